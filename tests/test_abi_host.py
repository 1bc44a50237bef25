"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point include/deabm.h declares, and create() rejects invalid
inputs during host validation, before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_04421_gb300 import build, deabm
    build.build()
    return deabm.lib()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(deabm_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert {"deabm_create", "deabm_step", "deabm_run", "deabm_destroy"} <= names
    for name in names:
        assert hasattr(lib, name), name


def _graph(n, rp, col, rand_mean=2.0):
    from paper_2110_04421_gb300.deabm import Graph
    g = Graph()
    g.n_agents, g.n_nets, g.rand_mean = n, 1, rand_mean
    g.row_ptr[0] = rp.ctypes.data
    g.col[0] = col.ctypes.data
    return g


def _create(lib, n, rp, col, age, params=None, rand_mean=2.0, stage=None, occ=None):
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Agents, make_params
    g = _graph(n, rp, col, rand_mean)
    if occ is not None:  # (occ_group, occ_k, n_nets[, occ_lattice, occ_rewire])
        g.n_occ, g.occ_group, g.occ_k = occ[1].size, occ[0].ctypes.data, occ[1].ctypes.data
        g.n_nets = occ[2]
        if len(occ) > 3:
            g.occ_lattice, g.occ_rewire = occ[3], occ[4]
        for q in range(1, occ[2]):
            g.row_ptr[q], g.col[q] = rp.ctypes.data, col.ctypes.data
    a = Agents()
    a.age_bin = age.ctypes.data
    if stage is not None:
        a.stage = stage.ctypes.data
    p = make_params(params or W.params_with())
    ctx = C.c_void_p()
    rc = lib.deabm_create(C.byref(g), C.byref(a), C.byref(p), None, C.byref(ctx))
    return rc, ctx, lib.deabm_last_error(None).decode()


@pytest.mark.parametrize("case", ["self_loop", "col_out_of_range", "row_ptr_decreases", "row_ptr_start",
                                  "bad_age", "bad_stage", "bad_test_delay", "bad_quarantine", "bad_prob",
                                  "random_net_single_agent", "occ_group_out_of_range", "occ_k_too_large",
                                  "occ_without_weight_slot", "den_without_testing", "den_bad_window",
                                  "den_bad_adoption", "occ_bad_lattice", "occ_bad_rewire"])
def test_create_rejects_invalid_input(lib, case):
    from paper_2110_04421_gb300 import workloads as W
    n = 4
    rp = np.array([0, 1, 2, 3, 4], np.uint32)
    col = np.array([1, 2, 3, 0], np.uint32)
    age = np.zeros(n, np.uint8)
    params, stage, rand_mean, occ = None, None, 2.0, None
    occ_group, occ_k = np.array([0, 1, 1, 0], np.uint32), np.array([3, 15], np.uint8)
    if case == "occ_group_out_of_range":
        occ_group[2] = 2
        occ = (occ_group, occ_k, 1)
    elif case == "occ_k_too_large":
        occ_k[1] = 16
        occ = (occ_group, occ_k, 1)
    elif case == "occ_without_weight_slot":  # four stored networks leave no B_net entry for it
        occ = (occ_group, occ_k, 4)
    elif case in ("occ_bad_lattice", "occ_bad_rewire"):
        occ = (occ_group, occ_k, 1, 2 if case == "occ_bad_lattice" else 1, -0.1 if case == "occ_bad_rewire" else 0.0)
    elif case == "den_without_testing":
        params = W.params_with(den_on=1, test_on=0)
    elif case == "den_bad_window":
        params = W.params_with(den_on=1, test_on=1, den_window=0)
    elif case == "den_bad_adoption":
        params = W.params_with(den_on=1, test_on=1, den_adoption=1.5)
    elif case == "self_loop":
        col[2] = 2
    elif case == "col_out_of_range":
        col[1] = 4
    elif case == "row_ptr_decreases":
        rp = np.array([0, 2, 1, 3, 4], np.uint32)
    elif case == "row_ptr_start":
        rp = np.array([1, 1, 2, 3, 4], np.uint32)
    elif case == "bad_age":
        age[3] = 9
    elif case == "bad_stage":
        stage = np.array([0, 11, 0, 0], np.int8)
    elif case == "bad_test_delay":
        params = W.params_with(test_lo=0)
    elif case == "bad_quarantine":
        params = W.params_with(quar_days=16)
    elif case == "bad_prob":
        params = W.params_with(p_sev=[1.5] * 9)
    elif case == "random_net_single_agent":
        n, rp, col, age = 1, np.array([0, 0], np.uint32), np.zeros(1, np.uint32), np.zeros(1, np.uint8)
    rc, ctx, msg = _create(lib, n, rp, col, age, params, rand_mean, stage, occ)
    assert rc == -1, (case, rc, msg)
    assert ctx.value is None and msg


@pytest.mark.parametrize("case", ["self_loop_first", "decrease_wins", "age_before_stage", "second_network"])
def test_create_reports_the_first_error_of_a_large_graph(lib, case):
    """n = 200,000 rows are checked on several host threads: the error reported is
    still the first one in the fixed order (network by network: row pointers,
    then columns; then ages, stages), whichever thread found it, and rows whose
    bounds leave col are never read."""
    n = 200_000
    rp = np.arange(n + 1, dtype=np.uint32)
    col = ((np.arange(n) + 1) % n).astype(np.uint32)
    age = np.zeros(n, np.uint8)
    stage, occ, want = None, None, None
    if case == "self_loop_first":
        col[150_000] = n
        col[10_000] = 10_000
        want = "self-loop at row 10000 of network 0"
    elif case == "decrease_wins":
        col[5] = n
        rp[100] = 4_000_000_000  # rows 99 and 100 point far past col: never read
        want = "row_ptr[0] decreases at row 100"
    elif case == "age_before_stage":
        age[170_000] = 9
        stage = np.zeros(n, np.int8)
        stage[1_000] = 11
        want = "age_bin[170000]"
    elif case == "second_network":
        rp2, col2 = rp.copy(), col.copy()
        col2[199_999] = 199_999
        age[3] = 9
        from paper_2110_04421_gb300 import workloads as W
        from paper_2110_04421_gb300.deabm import Agents, make_params
        g = _graph(n, rp, col, 2.0)
        g.n_nets = 2
        g.row_ptr[1], g.col[1] = rp2.ctypes.data, col2.ctypes.data
        a = Agents()
        a.age_bin = age.ctypes.data
        p = make_params(W.params_with())
        ctx = C.c_void_p()
        rc = lib.deabm_create(C.byref(g), C.byref(a), C.byref(p), None, C.byref(ctx))
        msg = lib.deabm_last_error(None).decode()
        assert rc == -1 and ctx.value is None and "self-loop at row 199999 of network 1" in msg, msg
        return
    rc, ctx, msg = _create(lib, n, rp, col, age, None, 2.0, stage, occ)
    assert rc == -1 and ctx.value is None, (case, rc, msg)
    assert want in msg, (case, msg)


def test_null_arguments(lib):
    ctx = C.c_void_p()
    assert lib.deabm_create(None, None, None, None, C.byref(ctx)) == -1
    assert lib.deabm_step(None, 1) == -1
    assert lib.deabm_run(None, 1, None, None) == -1
    lib.deabm_destroy(None)  # NULL-safe
    assert b"NULL" in lib.deabm_last_error(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2110_04421_gb300 import deabm
    monkeypatch.setattr(deabm, "_lib", None)
    monkeypatch.setattr(deabm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        deabm.lib()


def test_binding_passes_daily_occupations(lib):
    """The Python binding hands the occupation arrays to the library: an invalid
    daily count is rejected by the library's host validation, before any CUDA call."""
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import DeabmError, Simulation
    pop = W.population_daily_occupation(60, 1, 3)
    pop["occ_k"] = pop["occ_k"].copy()
    pop["occ_k"][0] = 16
    with pytest.raises(DeabmError, match="occ_k"):
        Simulation(pop, W.params_with(), pop["age"], pop["seed_ids"])
    pop["occ_k"][0] = 5
    pop["occ_group"] = pop["occ_group"].copy()
    pop["occ_group"][7] = pop["occ_k"].size
    with pytest.raises(DeabmError, match="occ_group"):
        Simulation(pop, W.params_with(), pop["age"], pop["seed_ids"])


def test_noalloc_wrapper_rejects_bad_tensors_before_the_call(lib):
    """lambda_noalloc's arrays are device memory the library cannot inspect, so the
    binding checks dtype, contiguity, length and device first: a wrong dtype or a
    short output is a ValueError and the C entry point is never reached."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import lambda_noalloc
    n = 50
    g = dict(n=n, row_ptr=[torch.zeros(n + 1, dtype=torch.int32)], col=[torch.zeros(4, dtype=torch.int32)])
    ok = dict(age=torch.zeros(n, dtype=torch.uint8), stage=torch.zeros(n, dtype=torch.int8),
              tinf=torch.zeros(n, dtype=torch.int16), qt=torch.zeros(n, dtype=torch.uint8))
    out = torch.zeros(n, dtype=torch.float32)
    p = W.params_with()

    def call(graph=g, out=out, **kw):
        a = dict(ok, **kw)
        return lambda_noalloc(graph, a["age"], a["stage"], a["tinf"], a["qt"], p, 0, out)

    with pytest.raises(ValueError, match="age has dtype torch.int64"):
        call(age=torch.zeros(n, dtype=torch.int64))
    with pytest.raises(ValueError, match="tinf has dtype"):
        call(tinf=torch.zeros(n, dtype=torch.int32))
    with pytest.raises(ValueError, match="out has 49 entries, the call needs 50"):
        call(out=torch.zeros(n - 1, dtype=torch.float32))
    with pytest.raises(ValueError, match=r"row_ptr\[0\] has 50 entries, the call needs 51"):
        call(graph=dict(g, row_ptr=[torch.zeros(n, dtype=torch.int32)]))
    with pytest.raises(ValueError, match="col.0. has dtype torch.int64"):
        call(graph=dict(g, col=[torch.zeros(4, dtype=torch.int64)]))
    with pytest.raises(ValueError, match="stage must be contiguous"):
        call(stage=torch.zeros(2 * n, dtype=torch.int8)[::2])
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        call()  # every check but the device passes on host tensors


def test_noalloc_rejects_oversized_population_before_any_gpu_work(lib):
    """The C entry point refuses more agents than its fixed array holds during its
    host checks, before it looks at the (here dummy) device pointers."""
    from paper_2110_04421_gb300.deabm import NOALLOC_MAX_AGENTS, Graph, make_params
    from paper_2110_04421_gb300 import workloads as W
    g = Graph()
    g.n_agents = NOALLOC_MAX_AGENTS + 1
    g.n_nets = 0
    g.rand_mean = 2.0
    p = make_params(W.params_with())
    dummy = C.c_void_p(16)
    rc = lib.deabm_lambda_noalloc(C.byref(g), dummy, dummy, dummy, dummy, C.byref(p), 0, dummy, None)
    assert rc == -1
    assert b"exceed the fixed working array" in lib.deabm_lambda_noalloc_last_error()
