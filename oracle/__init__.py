"""CPU oracle of the DeepABM-COVID simulation step (arXiv 2110.04421).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use this package; the product path never does.
The arithmetic lives in ``deabm_oracle.c`` (plain C, built with
``-ffp-contract=off`` so every FP32 product and sum is rounded on its own).
This module compiles it on first use and wraps it with ctypes.

What it follows:
  * Eq. 1 (Sec. 3 "Infection Transmission"): per-interaction rate
    R S_a A_s B_n / I * integral of the gamma infectiousness density over one day.
  * Eq. 2: P = 1 - exp(-lambda); aggregated per agent over independent
    interactions this is 1 - exp(-sum lambda).
  * Sec. 3 "Agent State Definition" (eleven stages), "Interaction Networks"
    (household, occupation, daily random network) and "Disease Progression".
  * Sec. 4.1 self-quarantine (14 days, daily dropout), Sec. 4.3 testing,
    Sec. 4.4/Sec. 5 two-dose vaccination with a 12-day onset.
Parity pins for every function here live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "deabm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "deabm_relaxed.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_STAGE, N_AGE, N_CLASS, MAX_NETS, POIS_CAP = 11, 9, 3, 4, 15
STAGES = ("S", "ASYM", "PRE_MILD", "PRE_SEV", "MILD", "SEV", "HOSP", "ICU", "REC", "VAX", "DEAD")


def build(force: bool = False) -> str:
    """Compile the oracle's C into ``oracle/_build/liboracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    import fcntl
    with open(os.path.join(_OUT_DIR, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        return _build_locked(force)


def _build_locked(force: bool) -> str:
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    # OpenMP over agents when the compiler has it (or_set_threads); one thread otherwise
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, *_SRCS, "-lm"], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, *_SRCS, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("n_nets", C.c_uint32),
        ("row_ptr", C.c_void_p * MAX_NETS), ("col", C.c_void_p * MAX_NETS),
        ("B_net", C.c_float * MAX_NETS),
        ("rand_mean", C.c_float), ("B_rand", C.c_float),
        ("R", C.c_float), ("inv_Ibar", C.c_float), ("dt", C.c_float),
        ("S_age", C.c_float * N_AGE), ("A_class", C.c_float * N_CLASS),
        ("inf_shape", C.c_double * N_CLASS), ("inf_scale", C.c_double * N_CLASS),
        ("inf_len", C.c_uint32),
        ("p_asym", C.c_double * N_AGE), ("p_sev", C.c_double * N_AGE), ("p_hosp", C.c_double * N_AGE),
        ("p_icu", C.c_double * N_AGE), ("p_death", C.c_double * N_AGE),
        ("dur_lo", (C.c_uint8 * N_AGE) * 8), ("dur_hi", (C.c_uint8 * N_AGE) * 8),
        ("test_on", C.c_uint32), ("test_sens", C.c_double), ("test_lo", C.c_uint32), ("test_hi", C.c_uint32),
        ("quar_on", C.c_uint32), ("quar_days", C.c_uint32), ("q_dropout", C.c_double),
        ("vax_on", C.c_uint32), ("vax_start", C.c_uint32), ("vax_onset", C.c_uint32),
        ("dose2_delay", C.c_uint32),
        ("vax_rate", C.c_double), ("vax_eff1", C.c_double), ("vax_eff2", C.c_double),
        ("seed", C.c_uint64), ("net_seed", C.c_uint64),
        ("vax_strategy", C.c_uint32), ("elderly_bin", C.c_uint32), ("vax_nonsterile", C.c_uint32),
        ("n_occ", C.c_uint32), ("occ_group", C.c_void_p), ("occ_k", C.c_void_p),
        ("occ_lattice", C.c_uint32), ("occ_rewire", C.c_float),
        ("den_on", C.c_uint32), ("den_adoption", C.c_double), ("den_compliance", C.c_double),
        ("den_window", C.c_uint32),
        ("rand_ws", C.c_uint32), ("rand_ws_k", C.c_uint32), ("rand_ws_beta", C.c_double),
        ("rand_by_age", C.c_uint32), ("rand_mean_age", C.c_float * N_AGE),
    ]


class _Diag(C.Structure):
    _fields_ = [
        ("lambda32", C.c_void_p), ("lambda64", C.c_void_p), ("p32", C.c_void_p), ("u32", C.c_void_p),
        ("inf32", C.c_void_p), ("near", C.c_void_p), ("rand_k", C.c_void_p),
        ("new_inf", C.c_int32), ("messages", C.c_int64), ("hist", C.c_int32 * N_STAGE),
        ("den_notified", C.c_int32), ("messages_sus", C.c_int64),
    ]


class _RxModel(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("n_nets", C.c_uint32),
        ("row_ptr", C.c_void_p * MAX_NETS), ("col", C.c_void_p * MAX_NETS),
        ("B_extra", C.c_double * MAX_NETS),
        ("rand_mean", C.c_double), ("inv_Ibar", C.c_double), ("tau", C.c_double),
        ("A_class", C.c_double * N_CLASS),
        ("inf_shape", C.c_double * N_CLASS), ("inf_scale", C.c_double * N_CLASS), ("inf_len", C.c_uint32),
        ("p_asym", C.c_double * N_AGE), ("p_sev", C.c_double * N_AGE),
        ("seed", C.c_uint64), ("net_seed", C.c_uint64),
        ("n_occ", C.c_uint32), ("occ_group", C.c_void_p), ("occ_k", C.c_void_p),
        ("occ_lattice", C.c_uint32), ("occ_rewire", C.c_double),
        ("rand_by_age", C.c_uint32), ("rand_mean_age", C.c_double * N_AGE),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.or_philox.argtypes = [vp, vp, vp]
            L.or_threshold.argtypes = [C.c_double]
            L.or_threshold.restype = C.c_uint64
            L.or_gamma_integral.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.or_gamma_integral.restype = C.c_double
            L.or_gamma_pdf.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_gamma_pdf.restype = C.c_double
            L.or_inf_table.argtypes = [C.POINTER(_Model), vp, vp]
            L.or_poisson_thresholds.argtypes = [C.c_double, vp]
            L.or_random_contacts.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_double, vp]
            L.or_random_contacts.restype = C.c_uint32
            L.or_occ_contacts.argtypes = [C.POINTER(_Model), C.c_uint32, C.c_uint32, vp]
            L.or_occ_contacts.restype = C.c_uint32
            L.or_vax_days.argtypes = [C.c_uint32, vp, C.c_uint32, C.c_double, vp]
            L.or_step.argtypes = [C.POINTER(_Model), vp, vp, C.c_uint32, vp, vp, vp, vp, vp, vp, vp, C.POINTER(_Diag)]
            L.or_step.restype = C.c_int
            L.or_seed_infections.argtypes = [C.POINTER(_Model), vp, vp, C.c_uint32, vp, vp, vp]
            L.or_seed_infections.restype = C.c_int
            L.or_run.argtypes = [C.POINTER(_Model), vp, vp, C.c_uint32, C.c_uint32,
                                 vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.or_den_apps.argtypes = [C.POINTER(_Model), vp]
            L.or_run.restype = C.c_int
            L.rx_run.argtypes = [C.POINTER(_RxModel), vp, vp, C.c_uint32, C.c_uint32, vp, vp, vp, vp, vp, vp]
            L.rx_run.restype = C.c_int
            L.rx_classes.argtypes = [C.POINTER(_RxModel), vp, vp]
            L.rx_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
            L.rx_noise.restype = C.c_double
            L.or_wsg_neighbours.argtypes = [C.POINTER(_Model), C.c_uint32, vp, vp, C.c_uint32]
            L.or_wsg_neighbours.restype = C.c_int
            L.or_set_threads.argtypes = [C.c_int]
            L.or_set_threads.restype = C.c_int
            _lib = L
    return _lib


def set_threads(threads: int) -> int:
    """Host threads for the oracle's per-agent loops (OpenMP over agents; results
    are the same for every count).  Returns the count in effect (1 when the
    library was built without OpenMP)."""
    return int(lib().or_set_threads(int(threads)))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------- primitives
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter (4 x u32) under a 64-bit key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def threshold(p: float) -> int:
    return int(lib().or_threshold(float(p)))


def gamma_integral(a: float, b: float, shape: float, scale: float) -> float:
    return float(lib().or_gamma_integral(a, b, shape, scale))


def poisson_thresholds(mean: float) -> np.ndarray:
    out = np.zeros(POIS_CAP, np.uint64)
    lib().or_poisson_thresholds(float(mean), _ptr(out))
    return out


def random_contacts(net_seed: int, n: int, j: int, step: int, mean: float) -> np.ndarray:
    buf = np.zeros(POIS_CAP, np.uint32)
    k = lib().or_random_contacts(int(net_seed), n, j, step, float(mean), _ptr(buf))
    return buf[:k].copy()


def vax_days(age: np.ndarray, start: int, rate: float) -> np.ndarray:
    age = np.ascontiguousarray(age, dtype=np.uint8)
    out = np.zeros(age.size, np.int16)
    lib().or_vax_days(age.size, _ptr(age), int(start), float(rate), _ptr(out))
    return out


# --------------------------------------------------------------------------- the model
class Model:
    """Graph + parameters packed for the C oracle.  ``graph`` holds ``row_ptr`` and
    ``col`` lists (u32 CSR, destination rows) and ``n``, and optionally the daily
    occupation networks: ``occ_group`` (u32 per agent) and ``occ_k`` (u8 per
    occupation, in-contacts a day), with ``occ_lattice`` = 1 and ``occ_rewire``
    for Watts-Strogatz contacts; ``params`` is a plain dict."""

    def __init__(self, graph: dict, params: dict):
        self.n = int(graph["n"])
        self._keep = []
        m = _Model()
        m.n = self.n
        rps, cols = graph["row_ptr"], graph["col"]
        m.n_nets = len(rps)
        for i, (rp, cl) in enumerate(zip(rps, cols)):
            rp = np.ascontiguousarray(rp, dtype=np.uint32)
            cl = np.ascontiguousarray(cl, dtype=np.uint32)
            self._keep += [rp, cl]
            m.row_ptr[i] = rp.ctypes.data
            m.col[i] = cl.ctypes.data
        P = params
        for i in range(MAX_NETS):
            m.B_net[i] = P["B_net"][i] if i < len(P["B_net"]) else 0.0
        m.rand_mean = P["rand_mean"]
        m.B_rand = P["B_rand"]
        m.R, m.inv_Ibar, m.dt = P["R"], P["inv_Ibar"], P["dt"]
        for i in range(N_AGE):
            m.S_age[i] = P["S_age"][i]
        for c in range(N_CLASS):
            m.A_class[c] = P["A_class"][c]
            m.inf_shape[c] = P["inf_shape"][c]
            m.inf_scale[c] = P["inf_scale"][c]
        m.inf_len = P["inf_len"]
        for name in ("p_asym", "p_sev", "p_hosp", "p_icu", "p_death"):
            arr = getattr(m, name)
            for a in range(N_AGE):
                arr[a] = P[name][a]
        for st in range(8):
            for a in range(N_AGE):
                m.dur_lo[st][a] = P["dur_lo"][st][a]
                m.dur_hi[st][a] = P["dur_hi"][st][a]
        for name in ("test_on", "test_sens", "test_lo", "test_hi", "quar_on", "quar_days", "q_dropout",
                     "vax_on", "vax_start", "vax_onset", "dose2_delay", "vax_rate", "vax_eff1", "vax_eff2",
                     "seed", "net_seed"):
            setattr(m, name, P[name])
        m.vax_strategy = P.get("vax_strategy", 0)
        m.elderly_bin = P.get("elderly_bin", 6)
        m.vax_nonsterile = P.get("vax_nonsterile", 0)
        m.den_on = P.get("den_on", 0)
        m.den_adoption = P.get("den_adoption", 0.3)
        m.den_compliance = P.get("den_compliance", 0.8)
        m.den_window = P.get("den_window", 7)
        if graph.get("occ_group") is not None:
            og = np.ascontiguousarray(graph["occ_group"], dtype=np.uint32)
            ok = np.ascontiguousarray(graph["occ_k"], dtype=np.uint8)
            self._keep += [og, ok]
            m.n_occ = ok.size
            m.occ_group = og.ctypes.data
            m.occ_k = ok.ctypes.data
            m.occ_lattice = int(graph.get("occ_lattice", 0))
            m.occ_rewire = float(graph.get("occ_rewire", 0.0))
        if P.get("rand_mean_age") is not None:  # age-stratified Poisson means
            m.rand_by_age = 1
            for a in range(N_AGE):
                m.rand_mean_age[a] = float(P["rand_mean_age"][a])
        if graph.get("rand_ws"):  # the global random network as a daily Watts-Strogatz graph
            m.rand_ws = 1
            m.rand_ws_k = int(graph.get("rand_ws_k", 2))
            m.rand_ws_beta = float(graph.get("rand_ws_beta", 0.5))
        self.m = m
        self.params = P

    def ws_neighbours(self, step: int):
        """The Watts-Strogatz random network of `step`: (start[n+1], neighbours) with
        agent j's neighbours, in summation order, at neighbours[start[j]:start[j+1]]."""
        n, k = self.n, int(self.m.rand_ws_k)
        start = np.zeros(n + 1, np.uint32)
        cap = 2 * k * n + 64
        nb = np.zeros(cap, np.uint32)
        if lib().or_wsg_neighbours(C.byref(self.m), step, _ptr(start), _ptr(nb), cap) != 0:
            raise ValueError("no Watts-Strogatz random network in this model")
        return start, nb[:start[-1]].copy()

    def occ_contacts(self, j: int, step: int) -> np.ndarray:
        """The daily occupation network's in-contacts of agent j on `step`."""
        buf = np.zeros(POIS_CAP, np.uint32)
        k = lib().or_occ_contacts(C.byref(self.m), j, step, _ptr(buf))
        return buf[:k].copy()

    def inf_table(self):
        L = self.m.inf_len
        t64 = np.zeros((N_CLASS, L), np.float64)
        t32 = np.zeros((N_CLASS, L), np.float32)
        lib().or_inf_table(C.byref(self.m), _ptr(t64), _ptr(t32))
        return t64, t32


class State:
    """Per-agent state arrays (SoA): stage int8, timer int16, tinf int16, flags u8, qt u8,
    and the days of dose 1 / dose 2 under a priority strategy (int16, 0x7FFF = none)."""

    def __init__(self, n: int):
        self.stage = np.zeros(n, np.int8)
        self.timer = np.zeros(n, np.int16)
        self.tinf = np.zeros(n, np.int16)
        self.flags = np.zeros(n, np.uint8)
        self.qt = np.zeros(n, np.uint8)
        self.vd1 = np.full(n, 0x7FFF, np.int16)
        self.vd2 = np.full(n, 0x7FFF, np.int16)

    def copy(self):
        s = State(0)
        for k in ("stage", "timer", "tinf", "flags", "qt", "vd1", "vd2"):
            setattr(s, k, getattr(self, k).copy())
        return s

    def ptrs(self):
        return [_ptr(self.stage), _ptr(self.timer), _ptr(self.tinf), _ptr(self.flags), _ptr(self.qt),
                _ptr(self.vd1), _ptr(self.vd2)]


class Sim:
    """One simulation on the oracle: ``Sim(graph, params, age, seed_ids)``; ``step()``
    runs one synchronous day and returns its diagnostics."""

    def __init__(self, graph: dict, params: dict, age: np.ndarray, seed_ids=None, state: State | None = None):
        self.model = Model(graph, params)
        self.n = self.model.n
        self.age = np.ascontiguousarray(age, dtype=np.uint8)
        if params["vax_on"]:
            self.vday1 = vax_days(self.age, params["vax_start"], params["vax_rate"])
        else:
            self.vday1 = np.full(self.n, 0x7FFF, np.int16)
        self.state = state.copy() if state is not None else State(self.n)
        self.t = 0
        self.den_notified = []  # per step: app holders notified (Sec. 4.2)
        if params.get("den_on", 0):
            lib().or_den_apps(C.byref(self.model.m), _ptr(self.state.flags))
        if seed_ids is not None and len(seed_ids):
            ids = np.ascontiguousarray(seed_ids, dtype=np.uint32)
            s = self.state
            rc = lib().or_seed_infections(C.byref(self.model.m), _ptr(self.age), _ptr(ids), ids.size,
                                          _ptr(s.stage), _ptr(s.timer), _ptr(s.tinf))
            assert rc == 0

    def step(self, diag: bool = True) -> dict:
        n = self.n
        out = {}
        d = _Diag()
        if diag:
            out = dict(lambda32=np.zeros(n, np.float32), lambda64=np.zeros(n, np.float64),
                       p32=np.zeros(n, np.float32), u32=np.zeros(n, np.float32), inf32=np.zeros(n, np.float32),
                       near=np.zeros(n, np.uint8), rand_k=np.zeros(n, np.uint32))
            for k, v in out.items():
                setattr(d, k, v.ctypes.data)
        rc = lib().or_step(C.byref(self.model.m), _ptr(self.age), _ptr(self.vday1), self.t,
                           *self.state.ptrs(), C.byref(d))
        if rc != 0:
            raise ValueError("oracle rejected the model parameters")
        out["new_inf"] = int(d.new_inf)
        out["messages"] = int(d.messages)
        out["messages_sus"] = int(d.messages_sus)
        out["hist"] = np.array(list(d.hist), np.int32)
        out["den_notified"] = int(d.den_notified)
        self.den_notified.append(out["den_notified"])
        out["t"] = self.t
        self.t += 1
        return out

    def run(self, T: int):
        new_inf = np.zeros(T, np.int32)
        hist = np.zeros((T, N_STAGE), np.int32)
        msgs = np.zeros(T, np.int64)
        den = np.zeros(T, np.int32)
        rc = lib().or_run(C.byref(self.model.m), _ptr(self.age), _ptr(self.vday1), self.t, T,
                          *self.state.ptrs(), _ptr(new_inf), _ptr(hist), _ptr(msgs), _ptr(den))
        if rc != 0:
            raise ValueError("oracle rejected the model parameters")
        self.den_notified += den.tolist()
        self.t += T
        return new_inf, hist, msgs


# --------------------------------------------------------------------------- relaxed model
THETA_NAMES = ("R", "B_household", "B_occupation", "B_random") + tuple(f"S_age{a}" for a in range(N_AGE))


def theta_of(params: dict) -> np.ndarray:
    """theta = (R, B_net[0], B_net[1], B_rand, S_age[0..8]) as FP64."""
    B = list(params["B_net"]) + [0.0, 0.0]
    return np.array([params["R"], B[0], B[1], params["B_rand"], *params["S_age"]], np.float64)


class Relaxed:
    """FP64 relaxed (Gumbel-softmax) model with full-history reverse sweep.
    Parameters are taken as the FP32 values the CUDA path receives."""

    def __init__(self, graph: dict, params: dict, age, seed_ids, tau: float = 0.5):
        self.n = int(graph["n"])
        self._keep = []
        m = _RxModel()
        m.n = self.n
        m.n_nets = len(graph["row_ptr"])
        for i, (rp, cl) in enumerate(zip(graph["row_ptr"], graph["col"])):
            rp = np.ascontiguousarray(rp, dtype=np.uint32)
            cl = np.ascontiguousarray(cl, dtype=np.uint32)
            self._keep += [rp, cl]
            m.row_ptr[i] = rp.ctypes.data
            m.col[i] = cl.ctypes.data
        f32 = lambda v: float(np.float32(v))
        B = list(params["B_net"]) + [0.0] * MAX_NETS
        for i in range(MAX_NETS):
            m.B_extra[i] = f32(B[i])
        m.rand_mean = f32(params["rand_mean"])
        m.inv_Ibar = f32(params["inv_Ibar"])
        m.tau = f32(tau)
        for c in range(N_CLASS):
            m.A_class[c] = f32(params["A_class"][c])
            m.inf_shape[c] = params["inf_shape"][c]
            m.inf_scale[c] = params["inf_scale"][c]
        m.inf_len = params["inf_len"]
        for a in range(N_AGE):
            m.p_asym[a] = params["p_asym"][a]
            m.p_sev[a] = params["p_sev"][a]
        m.seed, m.net_seed = params["seed"], params["net_seed"]
        if graph.get("occ_group") is not None:  # daily occupation networks
            og = np.ascontiguousarray(graph["occ_group"], dtype=np.uint32)
            ok = np.ascontiguousarray(graph["occ_k"], dtype=np.uint8)
            self._keep += [og, ok]
            m.n_occ = ok.size
            m.occ_group = og.ctypes.data
            m.occ_k = ok.ctypes.data
            m.occ_lattice = int(graph.get("occ_lattice", 0))
            m.occ_rewire = float(np.float32(graph.get("occ_rewire", 0.0)))
        if params.get("rand_mean_age") is not None:  # age-stratified Poisson means (FP32 values)
            m.rand_by_age = 1
            for a in range(N_AGE):
                m.rand_mean_age[a] = f32(params["rand_mean_age"][a])
        self.m = m
        self.age = np.ascontiguousarray(age, dtype=np.uint8)
        self.seeds = np.ascontiguousarray(seed_ids if seed_ids is not None else [], dtype=np.uint32)

    def classes(self) -> np.ndarray:
        out = np.zeros(self.n, np.uint8)
        lib().rx_classes(C.byref(self.m), _ptr(self.age), _ptr(out))
        return out

    def run(self, theta, T: int, target=None, grad: bool = False, want_x: bool = False, fp32_theta: bool = True):
        """theta is rounded to FP32 first (the values the CUDA path receives) unless
        fp32_theta=False (finite differences need the exact FP64 perturbation)."""
        th = np.asarray(theta, np.float64)
        th = np.ascontiguousarray(np.float32(th).astype(np.float64) if fp32_theta else th)
        y = None if target is None else np.ascontiguousarray(target, dtype=np.float64)
        inc = np.zeros(T, np.float64)
        loss = C.c_double(0.0)
        g = np.zeros(13, np.float64) if grad else None
        x = np.zeros((T, self.n), np.float64) if want_x else None
        rc = lib().rx_run(C.byref(self.m), _ptr(self.age), _ptr(self.seeds), self.seeds.size, T, _ptr(th), _ptr(y),
                          _ptr(inc), C.byref(loss), _ptr(g), _ptr(x))
        if rc != 0:
            raise ValueError("oracle rejected the relaxed model")
        out = dict(incidence=inc)
        if y is not None:
            out["loss"] = loss.value
        if grad:
            out["grad"] = g
        if want_x:
            out["x"] = x
        return out
