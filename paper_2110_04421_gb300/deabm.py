"""Thin ctypes binding of libdeabm.so (include/deabm.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing, loading
it raises.  PyTorch, when present, supplies the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdeabm.so")

MAX_NETS, N_AGE, N_STAGE, N_CLASS, POIS_CAP, N_REP_PARAMS = 4, 9, 11, 3, 15, 14
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5
STAGES = ("S", "ASYM", "PRE_MILD", "PRE_SEV", "MILD", "SEV", "HOSP", "ICU", "REC", "VAX", "DEAD")

EXPORTS = ("deabm_create", "deabm_create_batch", "deabm_step", "deabm_run", "deabm_get_state",
           "deabm_get_counters", "deabm_get_tables", "deabm_info", "deabm_sync", "deabm_last_error",
           "deabm_destroy", "deabm_relaxed_create", "deabm_relaxed_forward", "deabm_grad", "deabm_calibrate",
           "deabm_relaxed_last_error", "deabm_relaxed_destroy", "deabm_reset", "deabm_mlp_create",
           "deabm_mlp_param_count", "deabm_mlp_set_params", "deabm_mlp_get_params", "deabm_mlp_forward",
           "deabm_mlp_grad", "deabm_mlp_train_step", "deabm_mlp_sync", "deabm_mlp_last_error", "deabm_mlp_destroy",
           "deabm_lambda_noalloc", "deabm_lambda_noalloc_last_error", "deabm_create_ragged", "deabm_autotune",
           "deabm_mlp_use_tcgen05", "deabm_get_dose_days", "deabm_get_notified", "deabm_save", "deabm_restore",
           "deabm_mlp_apply_grads", "deabm_get_gathered", "deabm_mlp_set_wait_limit",
           "deabm_inject_alloc_failure", "deabm_grad_batch")
N_THETA = 13
NOALLOC_MAX_AGENTS = 1 << 20  # agents the library's fixed working array holds (deabm_lambda_noalloc)


class DeabmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"deabm error {code}: {msg}")
        self.code = code


class Graph(C.Structure):
    _fields_ = [("n_agents", C.c_uint32), ("n_nets", C.c_uint32),
                ("row_ptr", C.c_void_p * MAX_NETS), ("col", C.c_void_p * MAX_NETS),
                ("rand_mean", C.c_float),
                ("n_occ", C.c_uint32), ("occ_group", C.c_void_p), ("occ_k", C.c_void_p),
                ("occ_lattice", C.c_uint32), ("occ_rewire", C.c_float),
                ("rand_ws", C.c_uint32), ("rand_ws_k", C.c_uint32), ("rand_ws_beta", C.c_float),
                ("rand_by_age", C.c_uint32), ("rand_mean_age", C.c_float * N_AGE)]


class Agents(C.Structure):
    _fields_ = [("age_bin", C.c_void_p), ("stage", C.c_void_p), ("timer", C.c_void_p), ("tinf", C.c_void_p),
                ("flags", C.c_void_p), ("qt", C.c_void_p), ("seed_ids", C.c_void_p), ("n_seed", C.c_uint32),
                ("dose1_day", C.c_void_p), ("dose2_day", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [
        ("R", C.c_float), ("inv_Ibar", C.c_float), ("dt", C.c_float),
        ("B_net", C.c_float * MAX_NETS), ("B_rand", C.c_float),
        ("S_age", C.c_float * N_AGE), ("A_class", C.c_float * N_CLASS),
        ("inf_shape", C.c_double * N_CLASS), ("inf_scale", C.c_double * N_CLASS), ("inf_len", C.c_uint32),
        ("p_asym", C.c_double * N_AGE), ("p_sev", C.c_double * N_AGE), ("p_hosp", C.c_double * N_AGE),
        ("p_icu", C.c_double * N_AGE), ("p_death", C.c_double * N_AGE),
        ("dur_lo", (C.c_uint8 * N_AGE) * 8), ("dur_hi", (C.c_uint8 * N_AGE) * 8),
        ("test_on", C.c_uint32), ("test_sens", C.c_double), ("test_lo", C.c_uint32), ("test_hi", C.c_uint32),
        ("quar_on", C.c_uint32), ("quar_days", C.c_uint32), ("q_dropout", C.c_double),
        ("vax_on", C.c_uint32), ("vax_start", C.c_uint32), ("vax_onset", C.c_uint32), ("dose2_delay", C.c_uint32),
        ("vax_rate", C.c_double), ("vax_eff1", C.c_double), ("vax_eff2", C.c_double),
        ("seed", C.c_uint64), ("net_seed", C.c_uint64),
        ("max_steps", C.c_uint32), ("keep_lambda", C.c_uint32), ("vax_strategy", C.c_uint32),
        ("elderly_bin", C.c_uint32), ("vax_nonsterile", C.c_uint32), ("locality_order", C.c_uint32),
        ("den_on", C.c_uint32), ("den_adoption", C.c_double), ("den_compliance", C.c_double),
        ("den_window", C.c_uint32),
    ]


_lib = None


def lib():
    """Load libdeabm.so (build it with ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp, u32 = C.c_void_p, C.c_uint32
        L.deabm_create.argtypes = [C.POINTER(Graph), C.POINTER(Agents), C.POINTER(Params), vp, C.POINTER(vp)]
        L.deabm_create_batch.argtypes = [C.POINTER(Graph), C.POINTER(Agents), C.POINTER(Params), u32, vp, vp, vp,
                                         C.POINTER(vp)]
        L.deabm_step.argtypes = [vp, u32]
        L.deabm_run.argtypes = [vp, u32, vp, vp]
        L.deabm_get_state.argtypes = [vp] + [vp] * 7
        L.deabm_get_counters.argtypes = [vp, u32, vp, vp, vp]
        L.deabm_get_notified.argtypes = [vp, u32, vp]
        L.deabm_get_notified.restype = C.c_int
        L.deabm_save.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(u32)]
        L.deabm_save.restype = C.c_int
        L.deabm_restore.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, u32]
        L.deabm_restore.restype = C.c_int
        L.deabm_get_tables.argtypes = [vp, vp, vp, vp]
        L.deabm_info.argtypes = [vp, vp, vp, vp]
        L.deabm_sync.argtypes = [vp]
        L.deabm_last_error.argtypes = [vp]
        L.deabm_last_error.restype = C.c_char_p
        L.deabm_destroy.argtypes = [vp]
        L.deabm_destroy.restype = None
        L.deabm_relaxed_create.argtypes = [C.POINTER(Graph), C.POINTER(Agents), C.POINTER(Params), C.c_float, u32,
                                           u32, vp, C.POINTER(vp)]
        L.deabm_relaxed_forward.argtypes = [vp, u32, vp, vp]
        L.deabm_grad.argtypes = [vp, u32, vp, vp, vp, vp, vp]
        L.deabm_calibrate.argtypes = [vp, u32, vp, vp, u32, C.c_float, vp, vp]
        L.deabm_relaxed_last_error.argtypes = []
        L.deabm_relaxed_last_error.restype = C.c_char_p
        L.deabm_relaxed_destroy.argtypes = [vp]
        L.deabm_relaxed_destroy.restype = None
        L.deabm_reset.argtypes = [vp, vp, vp]
        L.deabm_get_dose_days.argtypes = [vp, vp, vp]
        L.deabm_get_dose_days.restype = C.c_int
        L.deabm_create_ragged.argtypes = [u32, C.POINTER(Graph), C.POINTER(Agents), C.POINTER(Params), vp, C.POINTER(vp)]
        L.deabm_create_ragged.restype = C.c_int
        L.deabm_autotune.argtypes = [vp, u32, C.POINTER(u32), C.POINTER(u32)]
        L.deabm_autotune.restype = C.c_int
        L.deabm_lambda_noalloc.argtypes = [C.POINTER(Graph), vp, vp, vp, vp, C.POINTER(Params), u32, vp, vp]
        L.deabm_lambda_noalloc.restype = C.c_int
        L.deabm_lambda_noalloc_last_error.argtypes = []
        L.deabm_lambda_noalloc_last_error.restype = C.c_char_p
        L.deabm_mlp_create.argtypes = [u32, u32, u32, u32, u32, vp, C.POINTER(vp)]
        L.deabm_mlp_param_count.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.deabm_mlp_set_params.argtypes = [vp, vp]
        L.deabm_mlp_get_params.argtypes = [vp, vp, vp]
        L.deabm_mlp_forward.argtypes = [vp, vp, u32, vp]
        L.deabm_mlp_grad.argtypes = [vp, vp, vp, u32, vp]
        L.deabm_mlp_train_step.argtypes = [vp, vp, vp, u32, C.c_float, vp]
        L.deabm_mlp_sync.argtypes = [vp]
        L.deabm_mlp_apply_grads.argtypes = [vp, vp, u32, C.c_float]
        L.deabm_get_gathered.argtypes = [vp, u32, vp]
        L.deabm_mlp_set_wait_limit.argtypes = [vp, u32]
        L.deabm_inject_alloc_failure.argtypes = [u32]
        L.deabm_grad_batch.argtypes = [vp, u32, u32, vp, vp, vp, vp, vp]
        L.deabm_inject_alloc_failure.restype = None
        L.deabm_mlp_use_tcgen05.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.deabm_mlp_use_tcgen05.restype = C.c_int
        L.deabm_mlp_last_error.argtypes = []
        L.deabm_mlp_last_error.restype = C.c_char_p
        L.deabm_mlp_destroy.argtypes = [vp]
        L.deabm_mlp_destroy.restype = None
        for name in ("deabm_create", "deabm_create_batch", "deabm_step", "deabm_run", "deabm_get_state",
                     "deabm_get_counters", "deabm_get_tables", "deabm_info", "deabm_sync", "deabm_relaxed_create",
                     "deabm_relaxed_forward", "deabm_grad", "deabm_calibrate", "deabm_reset", "deabm_mlp_create",
                     "deabm_mlp_param_count", "deabm_mlp_set_params", "deabm_mlp_get_params", "deabm_mlp_forward",
                     "deabm_mlp_grad", "deabm_mlp_train_step", "deabm_mlp_sync", "deabm_mlp_apply_grads",
                     "deabm_get_gathered", "deabm_mlp_set_wait_limit", "deabm_grad_batch"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, ctx=None):
    if rc != OK:
        msg = lib().deabm_last_error(ctx).decode(errors="replace")
        raise DeabmError(rc, msg)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def make_params(P: dict, max_steps: int = 1024, keep_lambda: bool = False, locality_order: bool = True) -> Params:
    p = Params()
    p.R, p.inv_Ibar, p.dt = P["R"], P["inv_Ibar"], P["dt"]
    for i in range(MAX_NETS):
        p.B_net[i] = P["B_net"][i] if i < len(P["B_net"]) else 0.0
    p.B_rand = P["B_rand"]
    for i in range(N_AGE):
        p.S_age[i] = P["S_age"][i]
    for c in range(N_CLASS):
        p.A_class[c] = P["A_class"][c]
        p.inf_shape[c] = P["inf_shape"][c]
        p.inf_scale[c] = P["inf_scale"][c]
    p.inf_len = P["inf_len"]
    for name in ("p_asym", "p_sev", "p_hosp", "p_icu", "p_death"):
        arr = getattr(p, name)
        for i in range(N_AGE):
            arr[i] = P[name][i]
    for st in range(8):
        for a in range(N_AGE):
            p.dur_lo[st][a] = P["dur_lo"][st][a]
            p.dur_hi[st][a] = P["dur_hi"][st][a]
    for name in ("test_on", "test_sens", "test_lo", "test_hi", "quar_on", "quar_days", "q_dropout", "vax_on",
                 "vax_start", "vax_onset", "dose2_delay", "vax_rate", "vax_eff1", "vax_eff2", "seed", "net_seed"):
        setattr(p, name, P[name])
    p.max_steps = max_steps
    p.keep_lambda = 1 if keep_lambda else 0
    p.vax_strategy = P.get("vax_strategy", 0)
    p.elderly_bin = P.get("elderly_bin", 6)
    p.vax_nonsterile = P.get("vax_nonsterile", 0)
    p.locality_order = 1 if locality_order else 0
    p.den_on = P.get("den_on", 0)
    p.den_adoption = P.get("den_adoption", 0.3)
    p.den_compliance = P.get("den_compliance", 0.8)
    p.den_window = P.get("den_window", 7)
    return p


def _graph_struct(graph: dict, rand_mean: float, keep: list, rand_mean_age=None) -> Graph:
    g = Graph()
    g.n_agents = int(graph["n"])
    g.n_nets = len(graph["row_ptr"])
    for i, (rp, cl) in enumerate(zip(graph["row_ptr"], graph["col"])):
        rp = np.ascontiguousarray(rp, dtype=np.uint32)
        cl = np.ascontiguousarray(cl, dtype=np.uint32)
        keep += [rp, cl]
        g.row_ptr[i] = rp.ctypes.data
        g.col[i] = cl.ctypes.data if cl.size else None
    g.rand_mean = rand_mean
    if rand_mean_age is not None:  # age-stratified Poisson means of the random network
        g.rand_by_age = 1
        for a in range(N_AGE):
            g.rand_mean_age[a] = float(rand_mean_age[a])
    if graph.get("occ_group") is not None:  # daily occupation networks
        og = np.ascontiguousarray(graph["occ_group"], dtype=np.uint32)
        ok = np.ascontiguousarray(graph["occ_k"], dtype=np.uint8)
        keep += [og, ok]
        g.n_occ = ok.size
        g.occ_group = og.ctypes.data
        g.occ_k = ok.ctypes.data
        g.occ_lattice = int(graph.get("occ_lattice", 0))
        g.occ_rewire = float(graph.get("occ_rewire", 0.0))
    if graph.get("rand_ws"):  # the random network as a daily Watts-Strogatz graph
        g.rand_ws = 1
        g.rand_ws_k = int(graph.get("rand_ws_k", 2))
        g.rand_ws_beta = float(graph.get("rand_ws_beta", 0.5))
    return g


def theta_of(params: dict) -> np.ndarray:
    """theta = (R, B_net[0], B_net[1], B_rand, S_age[0..8]) as float32."""
    B = list(params["B_net"]) + [0.0, 0.0]
    return np.array([params["R"], B[0], B[1], params["B_rand"], *params["S_age"]], np.float32)


def _rx_check(rc):
    if rc != OK:
        raise DeabmError(rc, lib().deabm_relaxed_last_error().decode(errors="replace"))


class Relaxed:
    """The relaxed (Gumbel-softmax) simulation on the GPU: forward, loss gradient
    by the library's reverse sweep, and on-device Adam calibration."""

    def __init__(self, graph: dict, params: dict, age, seed_ids=None, tau: float = 0.5, max_days: int = 90,
                 ckpt_every: int = 10, stream=None):
        L = lib()
        keep = []
        g = _graph_struct(graph, params["rand_mean"], keep, params.get("rand_mean_age"))
        a = Agents()
        age = np.ascontiguousarray(age, dtype=np.uint8)
        keep.append(age)
        a.age_bin = age.ctypes.data
        if seed_ids is not None and len(seed_ids):
            ids = np.ascontiguousarray(seed_ids, dtype=np.uint32)
            keep.append(ids)
            a.seed_ids = ids.ctypes.data
            a.n_seed = ids.size
        p = make_params(params)
        self._stream = C.c_void_p(stream) if isinstance(stream, int) else (stream or _current_stream())
        ctx = C.c_void_p()
        _rx_check(L.deabm_relaxed_create(C.byref(g), C.byref(a), C.byref(p), tau, max_days, ckpt_every,
                                         self._stream, C.byref(ctx)))
        self.ctx = ctx
        self.max_days = max_days

    def forward(self, theta, T: int) -> np.ndarray:
        th = np.ascontiguousarray(theta, dtype=np.float32)
        inc = np.zeros(T, np.float32)
        _rx_check(lib().deabm_relaxed_forward(self.ctx, T, _p(th), _p(inc)))
        return inc

    def grad(self, theta, target):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        y = np.ascontiguousarray(target, dtype=np.float32)
        T = y.size
        loss = np.zeros(1, np.float32)
        g = np.zeros(N_THETA, np.float32)
        inc = np.zeros(T, np.float32)
        _rx_check(lib().deabm_grad(self.ctx, T, _p(th), _p(y), _p(loss), _p(g), _p(inc)))
        return float(loss[0]), g, inc

    def grad_batch(self, theta, target):
        """Loss and gradient of B parameter columns at once (deabm_grad_batch):
        theta [B, 13], target [T, B] -> loss [B], grad [B, 13], incidence [T, B]."""
        th = np.ascontiguousarray(theta, dtype=np.float32)
        y = np.ascontiguousarray(target, dtype=np.float32)
        B = th.shape[0]
        assert th.shape == (B, N_THETA) and y.ndim == 2 and y.shape[1] == B
        T = y.shape[0]
        loss = np.zeros(B, np.float32)
        g = np.zeros((B, N_THETA), np.float32)
        inc = np.zeros((T, B), np.float32)
        _rx_check(lib().deabm_grad_batch(self.ctx, T, B, _p(th), _p(y), _p(loss), _p(g), _p(inc)))
        return loss, g, inc

    def calibrate(self, theta0, target, steps: int, lr: float):
        th0 = np.ascontiguousarray(theta0, dtype=np.float32)
        y = np.ascontiguousarray(target, dtype=np.float32)
        out = np.zeros(N_THETA, np.float32)
        trace = np.zeros(steps, np.float32)
        _rx_check(lib().deabm_calibrate(self.ctx, y.size, _p(th0), _p(y), steps, lr, _p(out), _p(trace)))
        return out, trace

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().deabm_relaxed_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def relaxed_loss(sim: "Relaxed", theta, target):
    """torch autograd entry: loss(theta) whose backward is the library's reverse sweep."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th, y):
            loss, g, _ = sim.grad(th.detach().cpu().numpy(), y.detach().cpu().numpy())
            ctx.save_for_backward(torch.from_numpy(g).to(th.device))
            return torch.tensor(loss, dtype=th.dtype, device=th.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g.to(gout.dtype), None

    return _Fn.apply(theta, target)


class RaggedSimulation:
    """A ragged batch of independent populations (different sizes, graphs,
    parameters) stepped together by one persistent kernel per day; ``run`` replays
    a captured CUDA graph of the days."""

    def __init__(self, pops: list, params: list, max_steps: int = 1024, stream=None, locality_order: bool = True,
                 states: list | None = None):
        """states: optional per-population initial state dicts (as Simulation's
        `state`, dose days included), None entries for the default state."""
        L = lib()
        keep = []
        n = len(pops)
        gs = (Graph * n)()
        ag = (Agents * n)()
        ps = (Params * n)()
        for q, (pop, par) in enumerate(zip(pops, params)):
            gs[q] = _graph_struct(pop, par["rand_mean"], keep, par.get("rand_mean_age"))
            age = np.ascontiguousarray(pop["age"], dtype=np.uint8)
            keep.append(age)
            ag[q].age_bin = age.ctypes.data
            ids = np.ascontiguousarray(pop.get("seed_ids", []), dtype=np.uint32)
            keep.append(ids)
            if ids.size:
                ag[q].seed_ids = ids.ctypes.data
                ag[q].n_seed = ids.size
            st = states[q] if states is not None else None
            if st is not None:
                for k, dt in (("stage", np.int8), ("timer", np.int16), ("tinf", np.int16), ("flags", np.uint8),
                              ("qt", np.uint8), ("dose1_day", np.int16), ("dose2_day", np.int16)):
                    if k in st:
                        arr = np.ascontiguousarray(st[k], dtype=dt)
                        keep.append(arr)
                        setattr(ag[q], k, arr.ctypes.data)
            ps[q] = make_params(par, max_steps=max_steps, locality_order=locality_order)
        self.sizes = [int(p["n"]) for p in pops]
        self.n_pops = n
        self.n = sum(self.sizes)
        self._stream = C.c_void_p(stream) if isinstance(stream, int) else (stream or C.c_void_p(0))
        ctx = C.c_void_p()
        _check(L.deabm_create_ragged(n, gs, ag, ps, self._stream, C.byref(ctx)))
        self.ctx = ctx

    def autotune(self, days_per_trial: int = 2):
        r, b = C.c_uint32(), C.c_uint32()
        _check(lib().deabm_autotune(self.ctx, days_per_trial, C.byref(r), C.byref(b)), self.ctx)
        return r.value, b.value

    def step(self, n_steps: int = 1):
        _check(lib().deabm_step(self.ctx, n_steps), self.ctx)

    def run(self, T: int, hist: bool = True):
        ni = np.zeros((T, self.n_pops), np.int32)
        h = np.zeros((T, self.n_pops, N_STAGE), np.int32) if hist else None
        _check(lib().deabm_run(self.ctx, T, _p(ni), _p(h)), self.ctx)
        return ni, h

    def reset(self):
        _check(lib().deabm_reset(self.ctx, None, None), self.ctx)

    def sync(self):
        _check(lib().deabm_sync(self.ctx), self.ctx)

    def counters(self, days: int):
        ni = np.zeros((days, self.n_pops), np.int32)
        h = np.zeros((days, self.n_pops, N_STAGE), np.int32)
        m = np.zeros(days, np.uint64)
        _check(lib().deabm_get_counters(self.ctx, days, _p(ni), _p(h), _p(m)), self.ctx)
        return ni, h, m

    def notified(self, days: int) -> np.ndarray:
        """Agents notified by exposure notification at the end of each day, [days, n_pops]
        (zeros in the columns of populations without it)."""
        out = np.zeros((days, self.n_pops), np.int32)
        _check(lib().deabm_get_notified(self.ctx, days, _p(out)), self.ctx)
        return out

    def gathered(self, days: int):
        """Messages gathered per day, summed over the populations (deabm_get_gathered)."""
        g = np.zeros(days, np.uint64)
        _check(lib().deabm_get_gathered(self.ctx, days, _p(g)), self.ctx)
        return g

    def dose_days(self) -> list:
        """Per population, each agent's first and second dose day under a priority
        strategy (0x7FFF = none), caller order."""
        d1 = np.zeros(self.n, np.int16)
        d2 = np.zeros(self.n, np.int16)
        _check(lib().deabm_get_dose_days(self.ctx, _p(d1), _p(d2)), self.ctx)
        res, b = [], 0
        for n in self.sizes:
            res.append((d1[b:b + n], d2[b:b + n]))
            b += n
        return res

    def state(self) -> list:
        """Per-population state dicts (caller ids)."""
        out = dict(stage=np.zeros(self.n, np.int8), timer=np.zeros(self.n, np.int16), tinf=np.zeros(self.n, np.int16),
                   flags=np.zeros(self.n, np.uint8), qt=np.zeros(self.n, np.uint8))
        _check(lib().deabm_get_state(self.ctx, _p(out["stage"]), _p(out["timer"]), _p(out["tinf"]),
                                     _p(out["flags"]), _p(out["qt"]), None, None), self.ctx)
        res, b = [], 0
        for n in self.sizes:
            res.append({k: v[b:b + n] for k, v in out.items()})
            b += n
        return res

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().deabm_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """A DeepABM-COVID simulation living on the GPU (one context of libdeabm).

    ``graph``: dict with ``n``, ``row_ptr`` and ``col`` (lists of u32 arrays, one
    per static network) and the parameters' ``rand_mean``; ``age``: u8 [n];
    ``seed_ids``: initial cases.  ``n_rep > 1`` with ``rep_params [n_rep, 14]``
    and ``rep_seeds [n_rep]`` creates a batch of replicates sharing the graph.
    """

    def __init__(self, graph: dict, params: dict, age, seed_ids=None, state: dict | None = None,
                 n_rep: int = 1, rep_params=None, rep_seeds=None, keep_lambda: bool = False,
                 max_steps: int = 1024, stream=None, locality_order: bool = True):
        L = lib()
        self.n = int(graph["n"])
        self.n_rep = int(n_rep)
        keep = []
        g = _graph_struct(graph, params["rand_mean"], keep, params.get("rand_mean_age"))
        a = Agents()
        age = np.ascontiguousarray(age, dtype=np.uint8)
        keep.append(age)
        a.age_bin = age.ctypes.data
        if state is not None:
            for k, dt in (("stage", np.int8), ("timer", np.int16), ("tinf", np.int16), ("flags", np.uint8),
                          ("qt", np.uint8), ("dose1_day", np.int16), ("dose2_day", np.int16)):
                if k not in state:
                    continue
                arr = np.ascontiguousarray(state[k], dtype=dt)
                keep.append(arr)
                setattr(a, k, arr.ctypes.data)
        if seed_ids is not None and len(seed_ids):
            ids = np.ascontiguousarray(seed_ids, dtype=np.uint32)
            keep.append(ids)
            a.seed_ids = ids.ctypes.data
            a.n_seed = ids.size
        p = make_params(params, max_steps=max_steps, keep_lambda=keep_lambda, locality_order=locality_order)
        self._stream = C.c_void_p(stream) if isinstance(stream, int) else (stream or _current_stream())
        ctx = C.c_void_p()
        if self.n_rep == 1 and rep_params is None:
            rc = L.deabm_create(C.byref(g), C.byref(a), C.byref(p), self._stream, C.byref(ctx))
        else:
            rp = np.ascontiguousarray(rep_params, dtype=np.float32).reshape(self.n_rep, N_REP_PARAMS)
            rs = np.ascontiguousarray(rep_seeds, dtype=np.uint64).reshape(self.n_rep)
            keep += [rp, rs]
            rc = L.deabm_create_batch(C.byref(g), C.byref(a), C.byref(p), self.n_rep, _p(rp), _p(rs),
                                      self._stream, C.byref(ctx))
        _check(rc)
        self.ctx = ctx
        self.keep_lambda = keep_lambda

    # -- the day loop
    def step(self, n_steps: int = 1):
        _check(lib().deabm_step(self.ctx, n_steps), self.ctx)

    def run(self, T: int, hist: bool = True):
        B = self.n_rep
        ni = np.zeros((T, B), np.int32)
        h = np.zeros((T, B, N_STAGE), np.int32) if hist else None
        _check(lib().deabm_run(self.ctx, T, _p(ni), _p(h)), self.ctx)
        return ni, h

    def sync(self):
        _check(lib().deabm_sync(self.ctx), self.ctx)

    def reset(self, rep_params=None, rep_seeds=None):
        """Back to day 0 (initial state and cases re-applied), optionally with new
        per-replicate parameters [n_rep, 14] and seeds."""
        rp = rs = None
        if rep_params is not None:
            rp = np.ascontiguousarray(rep_params, dtype=np.float32).reshape(self.n_rep, N_REP_PARAMS)
            rs = np.ascontiguousarray(rep_seeds, dtype=np.uint64).reshape(self.n_rep)
        _check(lib().deabm_reset(self.ctx, _p(rp), _p(rs)), self.ctx)

    # -- readback
    @property
    def day(self) -> int:
        d = C.c_uint32()
        _check(lib().deabm_info(self.ctx, C.byref(d), None, None), self.ctx)
        return d.value

    def state(self, with_lambda: bool = False) -> dict:
        nb = self.n * self.n_rep
        out = dict(stage=np.zeros(nb, np.int8), timer=np.zeros(nb, np.int16), tinf=np.zeros(nb, np.int16),
                   flags=np.zeros(nb, np.uint8), qt=np.zeros(nb, np.uint8))
        lam = p = None
        if with_lambda:
            lam, p = np.zeros(nb, np.float32), np.zeros(nb, np.float32)
            out["lambda"], out["p"] = lam, p
        _check(lib().deabm_get_state(self.ctx, _p(out["stage"]), _p(out["timer"]), _p(out["tinf"]),
                                     _p(out["flags"]), _p(out["qt"]), _p(lam), _p(p)), self.ctx)
        if self.n_rep > 1:
            out = {k: v.reshape(self.n, self.n_rep) for k, v in out.items()}
        return out

    def dose_days(self):
        """Each agent's first and second dose day under a priority strategy
        (0x7FFF = none): [N] arrays, or [N, B] in a batched context."""
        d1 = np.zeros(self.n * self.n_rep, np.int16)
        d2 = np.zeros(self.n * self.n_rep, np.int16)
        _check(lib().deabm_get_dose_days(self.ctx, _p(d1), _p(d2)), self.ctx)
        if self.n_rep > 1:
            return d1.reshape(self.n, self.n_rep), d2.reshape(self.n, self.n_rep)
        return d1, d2

    def counters(self, days: int | None = None):
        days = self.day if days is None else days
        B = self.n_rep
        ni = np.zeros((days, B), np.int32)
        h = np.zeros((days, B, N_STAGE), np.int32)
        m = np.zeros(days, np.uint64)
        _check(lib().deabm_get_counters(self.ctx, days, _p(ni), _p(h), _p(m)), self.ctx)
        return ni, h, m

    def gathered(self, days: int | None = None):
        """Messages gathered per day (deabm_get_gathered): the in-contacts of the
        destinations that evaluated Eq. 1 that day."""
        days = self.day if days is None else days
        g = np.zeros(days, np.uint64)
        _check(lib().deabm_get_gathered(self.ctx, days, _p(g)), self.ctx)
        return g

    def save(self) -> dict:
        """A checkpoint: the state at the start of the next day to run ([N, B] or
        [N] arrays in caller order), dose days under a priority strategy, the day."""
        shape = (self.n,) if self.n_rep == 1 else (self.n, self.n_rep)
        out = dict(stage=np.zeros(shape, np.int8), timer=np.zeros(shape, np.int16), tinf=np.zeros(shape, np.int16),
                   flags=np.zeros(shape, np.uint8), qt=np.zeros(shape, np.uint8),
                   dose1_day=np.zeros(shape, np.int16), dose2_day=np.zeros(shape, np.int16))
        day = C.c_uint32()
        _check(lib().deabm_save(self.ctx, *(_p(out[k]) for k in ("stage", "timer", "tinf", "flags", "qt",
                                                                 "dose1_day", "dose2_day")), C.byref(day)), self.ctx)
        out["day"] = int(day.value)
        return out

    def restore(self, ckpt: dict):
        """Resume from a checkpoint of save() (this context or another with the
        same graph and parameters): the next step runs day ckpt["day"]."""
        arrs = [np.ascontiguousarray(ckpt[k], dtype=t) for k, t in (("stage", np.int8), ("timer", np.int16),
                                                                  ("tinf", np.int16), ("flags", np.uint8),
                                                                  ("qt", np.uint8))]
        d1 = ckpt.get("dose1_day")
        d2 = ckpt.get("dose2_day")
        d1 = None if d1 is None else np.ascontiguousarray(d1, dtype=np.int16)
        d2 = None if d2 is None else np.ascontiguousarray(d2, dtype=np.int16)
        _check(lib().deabm_restore(self.ctx, *(_p(a) for a in arrs), _p(d1), _p(d2), int(ckpt["day"])), self.ctx)

    def notified(self, days: int | None = None) -> np.ndarray:
        """Agents notified by exposure notification at the end of each day: [days]
        in a plain context, [days, n_rep] in a batched one."""
        days = self.day if days is None else days
        out = np.zeros((days, self.n_rep) if self.n_rep > 1 else days, np.int32)
        _check(lib().deabm_get_notified(self.ctx, days, _p(out)), self.ctx)
        return out

    def tables(self, inf_len: int):
        t = np.zeros((N_CLASS, inf_len), np.float32)
        pois = np.zeros(POIS_CAP, np.uint64)
        d1 = np.zeros(self.n, np.int16)
        _check(lib().deabm_get_tables(self.ctx, _p(t), _p(pois), _p(d1)), self.ctx)
        return t, pois, d1

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().deabm_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _mlp_check(rc):
    if rc != OK:
        raise DeabmError(rc, lib().deabm_mlp_last_error().decode(errors="replace"))


class MLP:
    """The surrogate MLP in libdeabm: BF16 tensor-core forward / backward, FP32
    master weights, Adam.  Data are torch CUDA float32 tensors (device pointers)."""

    def __init__(self, n_in=14, hidden=256, depth=3, n_out=180, max_batch=65536, stream=None):
        L = lib()
        self.sizes = [n_in] + [hidden] * depth + [n_out]
        self.n_in, self.n_out, self.max_batch = n_in, n_out, max_batch
        self._stream = C.c_void_p(stream) if isinstance(stream, int) else (stream or _current_stream())
        ctx = C.c_void_p()
        _mlp_check(L.deabm_mlp_create(n_in, hidden, depth, n_out, max_batch, self._stream, C.byref(ctx)))
        self.ctx = ctx
        cnt = C.c_uint64()
        _mlp_check(L.deabm_mlp_param_count(ctx, C.byref(cnt)))
        self.n_params = cnt.value

    def use_tcgen05(self, enable: bool = True) -> bool:
        """Select the fused tcgen05 forward (True) or the per-layer mma.sync GEMMs;
        returns whether the fused path applies to this shape."""
        avail = C.c_int()
        _mlp_check(lib().deabm_mlp_use_tcgen05(self.ctx, 1 if enable else 0, C.byref(avail)))
        return bool(avail.value)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.n_params
        _mlp_check(lib().deabm_mlp_set_params(self.ctx, _p(p)))

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        _mlp_check(lib().deabm_mlp_get_params(self.ctx, _p(p), None))
        return p

    def get_grads(self):
        g = np.zeros(self.n_params, np.float32)
        _mlp_check(lib().deabm_mlp_get_params(self.ctx, None, _p(g)))
        return g

    @staticmethod
    def _dev(t, cols):
        assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous() and t.shape[-1] == cols
        return C.c_void_p(t.data_ptr())

    def forward(self, x, out=None):
        import torch
        B = x.shape[0]
        y = out if out is not None else torch.empty((B, self.n_out), dtype=torch.float32, device=x.device)
        _mlp_check(lib().deabm_mlp_forward(self.ctx, self._dev(x, self.n_in), B, self._dev(y, self.n_out)))
        return y

    def grad(self, x, y):
        loss = np.zeros(1, np.float32)
        _mlp_check(lib().deabm_mlp_grad(self.ctx, self._dev(x, self.n_in), self._dev(y, self.n_out), x.shape[0],
                                        _p(loss)))
        return float(loss[0])

    def train_step(self, x, y, lr, sync=False):
        loss = np.zeros(1, np.float32) if sync else None
        _mlp_check(lib().deabm_mlp_train_step(self.ctx, self._dev(x, self.n_in), self._dev(y, self.n_out), x.shape[0],
                                              lr, _p(loss)))
        return float(loss[0]) if sync else None

    def apply_grads(self, grads, lr):
        """One Adam step on caller-supplied gradients (numpy FP32 on the host, or a
        contiguous CUDA FP32 tensor) in the get_params layout."""
        if hasattr(grads, "is_cuda") and grads.is_cuda:
            assert grads.dtype.is_floating_point and grads.element_size() == 4 and grads.is_contiguous()
            assert grads.numel() == self.n_params
            _mlp_check(lib().deabm_mlp_apply_grads(self.ctx, C.c_void_p(grads.data_ptr()), 1, lr))
        else:
            g = np.ascontiguousarray(grads, np.float32)
            assert g.size == self.n_params
            _mlp_check(lib().deabm_mlp_apply_grads(self.ctx, _p(g), 0, lr))

    def set_wait_limit(self, polls: int):
        """Bound of the tcgen05 kernels' waits (deabm_mlp_set_wait_limit)."""
        _mlp_check(lib().deabm_mlp_set_wait_limit(self.ctx, int(polls)))

    def sync(self):
        _mlp_check(lib().deabm_mlp_sync(self.ctx))

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().deabm_mlp_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_noalloc_args(graph_dev: dict, arrays: dict, out):
    """Everything deabm_lambda_noalloc cannot check itself (its arrays are device
    memory): each tensor's dtype, that it is a contiguous CUDA tensor on one common
    device, and that it holds the entries the call reads or writes.  Raises
    ValueError; returns the common device."""
    import torch
    n = int(graph_dev["n"])
    rps, cols = list(graph_dev["row_ptr"]), list(graph_dev["col"])
    if len(rps) != len(cols) or len(rps) > 4:
        raise ValueError("graph_dev needs as many row_ptr as col tensors, at most 4")
    if n > NOALLOC_MAX_AGENTS:
        return None  # the library rejects the size itself, before touching any array
    idx = (torch.int32, torch.uint32) if hasattr(torch, "uint32") else (torch.int32,)
    want = {"age": ((torch.uint8,), n), "stage": ((torch.int8,), n), "tinf": ((torch.int16,), n),
            "qt": ((torch.uint8,), n), "out": ((torch.float32,), n)}
    items = dict(arrays, out=out)
    for k, (rp, cl) in enumerate(zip(rps, cols)):
        items[f"row_ptr[{k}]"], want[f"row_ptr[{k}]"] = rp, (idx, n + 1)
        items[f"col[{k}]"], want[f"col[{k}]"] = cl, (idx, 0)
    device = None
    for name, t in items.items():
        dtypes, count = want[name]
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}, expected {' or '.join(str(d) for d in dtypes)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < count:
            raise ValueError(f"{name} has {t.numel()} entries, the call needs {count}")
    for name, t in items.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if device is None:
            device = t.device
        elif t.device != device:
            raise ValueError(f"{name} is on {t.device}, the other arrays on {device}")
    return device


def lambda_noalloc(graph_dev: dict, age, stage, tinf, qt, params: dict, day: int, out, stream=None):
    """Infection rates of one day through deabm_lambda_noalloc, which allocates
    nothing: every argument is a caller-owned torch CUDA tensor on one device
    (graph_dev holds ``n``, ``row_ptr`` and ``col`` tensors of dtype int32/uint32;
    age and qt uint8, stage int8, tinf int16, out float32, n entries each;
    row_ptr n + 1; the column arrays as long as the row pointers say, which the
    library does not check).  The tensors' device is made current for the call."""
    import torch
    device = _check_noalloc_args(graph_dev, {"age": age, "stage": stage, "tinf": tinf, "qt": qt}, out)
    g = Graph()
    g.n_agents = int(graph_dev["n"])
    g.n_nets = len(graph_dev["row_ptr"])
    for i, (rp, cl) in enumerate(zip(graph_dev["row_ptr"], graph_dev["col"])):
        g.row_ptr[i] = rp.data_ptr()
        g.col[i] = cl.data_ptr()
    g.rand_mean = params["rand_mean"]
    p = make_params(params)
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        st = C.c_void_p(stream) if isinstance(stream, int) else (stream or _current_stream())
        rc = lib().deabm_lambda_noalloc(C.byref(g), C.c_void_p(age.data_ptr()), C.c_void_p(stage.data_ptr()),
                                        C.c_void_p(tinf.data_ptr()), C.c_void_p(qt.data_ptr()), C.byref(p), day,
                                        C.c_void_p(out.data_ptr()), st)
    if rc != OK:
        raise DeabmError(rc, lib().deabm_lambda_noalloc_last_error().decode(errors="replace"))
    return out
