"""CUDA path (through the C-ABI) against the CPU oracle, element by element.

Bar: stages, timers, flags and counters bit-exact; lambda bit-exact against the
oracle's FP32 path (same CSR order, no FMA) and within 1e-5 relative of its FP64
path; the only tolerated infection-draw difference is |u - p| < 1e-6 (counted,
and it ends the comparison)."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W
from tests.helpers import STATE_KEYS, compare_days, gpu_available, gpu_sim, oracle_sim

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_device_tables_match_oracle():
    pop = W.population(5000, 1, 10)
    for p in (W.params_with(vax_on=1, vax_start=7, vax_rate=0.013),
              W.params_with(inf_shape=[2.5, 4.0, 6.7], inf_scale=[2.0, 1.25, 0.9], A_class=[0.3, 1.0, 1.7],
                            inf_len=40, rand_mean=3.7, vax_on=1, vax_rate=0.002)):
        g = gpu_sim(pop, p)
        try:
            t, pois, d1 = g.tables(p["inf_len"])
        finally:
            g.close()
        _, t32 = oracle.Model(pop, p).inf_table()
        want = np.float32(p["A_class"])[:, None] * t32          # A_c * infT_c[t] in FP32
        assert np.array_equal(t.view(np.uint32), want.view(np.uint32)), np.nonzero(t != want)
        assert np.array_equal(pois, oracle.poisson_thresholds(float(np.float32(p["rand_mean"]))))  # FP32 parameter
        assert np.array_equal(d1, oracle.vax_days(pop["age"], p["vax_start"], p["vax_rate"]))


def test_plain_small_workload_60_days():
    """N=10,000, 60 days, 10 initial cases, seed 0 (the small plain workload)."""
    w = W.plain_small()
    pop = W.population(w["n"], 0, w["n_seed"])
    rep = compare_days(pop, w["params"], w["T"])
    assert rep["flips"] == 0 and rep["days"] == w["T"], rep
    assert rep["max_rel_lambda64"] <= 1e-5
    assert sum(rep["new_inf"]) > 1000


def test_interventions_all_on():
    pop = W.population(6001, 2, 40)
    p = W.params_with(test_on=1, quar_on=1, q_dropout=0.07, vax_on=1, vax_start=10, vax_rate=0.02,
                      dose2_delay=17, R=4.5, seed=77, net_seed=78, S_age=[0.5, 0.7, 0.9, 1.0, 1.1, 1.2, 1.3, 1.4, 1.6])
    rep = compare_days(pop, p, 100)
    assert rep["flips"] == 0 and rep["days"] == 100, rep
    assert rep["max_rel_lambda64"] <= 1e-5


@pytest.mark.parametrize("n", [2, 3, 31, 257, 1001])
def test_ragged_and_tiny_populations(n):
    pop = W.population(n, 5, max(1, n // 10))
    p = W.params_with(R=6.0, rand_mean=2.5, test_on=1, quar_on=1)
    rep = compare_days(pop, p, 30)
    assert rep["flips"] == 0 and rep["days"] == 30


def test_no_networks_and_no_random_network():
    pop = W.population(700, 6, 20)
    empty = dict(pop, row_ptr=[], col=[])
    rep = compare_days(empty, W.params_with(rand_mean=3.0), 20)
    assert rep["days"] == 20
    rep = compare_days(pop, W.params_with(rand_mean=0.0, R=8.0), 25)
    assert rep["days"] == 25
    one = dict(n=1, age=np.array([4], np.uint8), row_ptr=[np.zeros(2, np.uint32)], col=[np.zeros(0, np.uint32)],
               seed_ids=np.array([0], np.uint32))
    rep = compare_days(one, W.params_with(rand_mean=0.0), 15)
    assert rep["days"] == 15


def test_high_degree_rows_and_many_nets():
    """One household of 300 (in-degree 299) plus four networks."""
    rng = np.random.default_rng(3)
    n = 1200
    sizes = np.array([300] + [4] * 225)
    hh_rp, hh_col = W.household_csr(sizes)
    oc_rp, oc_col = W.occupation_csr(n, rng, group=50, links=40)
    x_rp, x_col = W.occupation_csr(n, rng, group=7, links=3)
    pop = dict(n=n, age=rng.integers(0, 9, n).astype(np.uint8), row_ptr=[hh_rp, oc_rp, x_rp, hh_rp],
               col=[hh_col, oc_col, x_col, hh_col], seed_ids=np.arange(0, n, 97, dtype=np.uint32))
    p = W.params_with(B_net=[0.5, 0.2, 1.3, 0.1], R=2.0, dt=0.75)
    rep = compare_days(pop, p, 30)
    assert rep["flips"] == 0 and rep["days"] == 30


def test_full_size_plain_workload_first_days():
    """N=2,000,000 with 10,000 initial cases and all interventions, launched as the
    benchmark launches it; the oracle runs the same first days in full."""
    w = W.plain_large()
    pop = W.population(w["n"], 0, w["n_seed"])
    p = dict(w["params"], vax_start=1)   # vaccination events inside the compared window
    rep = compare_days(pop, p, 4)
    assert rep["flips"] == 0 and rep["days"] == 4
    assert rep["max_rel_lambda64"] <= 1e-5


def test_full_size_bench_configuration_60_days():
    """The benchmark's launch configuration (no lambda kept, so only susceptible
    agents gather) at its full size, N = 2,000,000, through day 59: by then about
    half the agents are no longer susceptible.  Every day's counters and the final
    state equal the oracle's."""
    w = W.plain_large()
    pop = W.population(w["n"], 0, w["n_seed"])
    T = 60
    g = gpu_sim(pop, w["params"], keep_lambda=False, max_steps=T)
    ni, h = g.run(T)
    _, _, m = g.counters(T)
    s = g.state()
    g.close()
    o = oracle_sim(pop, w["params"])
    ni_o, h_o, m_o = o.run(T)
    assert np.array_equal(ni[:, 0], ni_o) and np.array_equal(h[:, 0], h_o)
    assert np.array_equal(m.astype(np.int64), m_o)
    for k in ("stage", "timer", "tinf", "flags", "qt"):
        assert np.array_equal(s[k], getattr(o.state, k)), k
    assert h_o[-1, 0] < 0.8 * w["n"]  # the skip path carried most agents


def test_more_than_2_pow_24_agents():
    """N = 2^24 + 3 agents (households only): the internal numbering's radix sort
    takes four 8-bit passes and row indices pass 2^24.  Three days' counters and
    the final state equal the oracle's."""
    n = (1 << 24) + 3
    pop = W.population(n, 5, 200_000)
    g = dict(pop, row_ptr=pop["row_ptr"][:1], col=pop["col"][:1])
    p = W.params_with(B_net=[1.0], R=4.0, test_on=1, quar_on=1, seed=3, net_seed=4)
    T = 3
    sim = gpu_sim(g, p, keep_lambda=False, max_steps=T)
    ni, h = sim.run(T)
    _, _, m = sim.counters(T)
    s = sim.state()
    sim.close()
    o = oracle_sim(g, p)
    ni_o, h_o, m_o = o.run(T)
    assert np.array_equal(ni[:, 0], ni_o) and np.array_equal(h[:, 0], h_o)
    assert np.array_equal(m.astype(np.int64), m_o)
    for k in ("stage", "timer", "tinf", "flags", "qt"):
        assert np.array_equal(s[k], getattr(o.state, k)), k
    assert ni_o.sum() > 1000


@pytest.mark.parametrize("B", [37, 36, 132])
def test_batched_columns_equal_plain_runs_and_oracle(B):
    """B = 37 runs the one-replicate-per-thread panel kernel; B = 36 and 132 (a
    partly filled second panel of 128) the four-replicates-per-thread kernel."""
    n, T = 3001, 40
    pop = W.population(n, 8, 30)
    base = W.params_with(vax_on=1, vax_start=5, vax_rate=0.01, test_on=1, quar_on=1, net_seed=5)
    rp, seeds = W.batch_params(B, 1)
    rp[:, 4:13] = np.random.default_rng(2).uniform(0.5, 1.5, (B, 9))
    from paper_2110_04421_gb300.deabm import Simulation
    gb = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds,
                    max_steps=T)
    ni_b, h_b = gb.run(T)
    sb = gb.state()
    gb.close()
    for r in sorted({0, 1, 17, 31, 32, B - 4, B - 1}):
        pr = dict(base, R=float(rp[r, 0]), B_net=[float(rp[r, 1]), float(rp[r, 2])], B_rand=float(rp[r, 3]),
                  S_age=[float(x) for x in rp[r, 4:13]], dose2_delay=int(rp[r, 13]), seed=int(seeds[r]))
        g = gpu_sim(pop, pr, keep_lambda=False, max_steps=T)
        ni, h = g.run(T)
        s = g.state()
        g.close()
        assert np.array_equal(ni[:, 0], ni_b[:, r]) and np.array_equal(h[:, 0], h_b[:, r])
        for k in ("stage", "timer", "tinf", "flags", "qt"):
            assert np.array_equal(s[k], sb[k][:, r]), (r, k)
        if r in (0, B - 1):
            o = oracle_sim(pop, pr)
            ni_o, h_o, _ = o.run(T)
            assert np.array_equal(ni_o, ni_b[:, r]) and np.array_equal(h_o, h_b[:, r])
            assert np.array_equal(o.state.stage, sb["stage"][:, r])


def test_counters_and_run_agree():
    pop = W.population(4000, 9, 20)
    p = W.params_with()
    g = gpu_sim(pop, p, keep_lambda=False, max_steps=50)
    ni, h = g.run(50)
    ni2, h2, m = g.counters()
    g.close()
    assert np.array_equal(ni, ni2) and np.array_equal(h, h2)
    assert np.all(h.sum(axis=2) == 4000)
    o = oracle_sim(pop, p)
    ni_o, h_o, m_o = o.run(50)
    assert np.array_equal(ni_o, ni[:, 0]) and np.array_equal(m_o, m.astype(np.int64))


@pytest.mark.parametrize("locality_order", [False, True])
def test_internal_numbering_changes_nothing(locality_order):
    """The library's internal agent numbering (agents grouped by the smallest id
    reaching them in the densest network) is invisible: the same days, draws and
    outputs, with or without it."""
    pop = W.population(5003, 11, 25)
    p = W.params_with(test_on=1, quar_on=1, vax_on=1, vax_start=3, vax_rate=0.03, R=4.0, seed=5, net_seed=6)
    rep = compare_days_kw(pop, p, 40, locality_order=locality_order)
    assert rep["flips"] == 0 and rep["days"] == 40


def compare_days_kw(pop, p, T, **kw):
    from tests import helpers
    orig = helpers.gpu_sim
    helpers.gpu_sim = lambda *a, **k: orig(*a, **{**k, **kw})
    try:
        return compare_days(pop, p, T)
    finally:
        helpers.gpu_sim = orig


def test_batched_without_internal_numbering():
    n, B, T = 2000, 40, 25
    pop = W.population(n, 12, 20)
    base = W.params_with(test_on=1, quar_on=1, net_seed=9)
    rp, seeds = W.batch_params(B, 3)
    from paper_2110_04421_gb300.deabm import Simulation
    out = []
    for lo in (False, True):
        g = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T,
                       locality_order=lo)
        ni, h = g.run(T)
        out.append((ni, h, g.state()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    for k in ("stage", "timer", "tinf", "flags", "qt"):
        assert np.array_equal(out[0][2][k], out[1][2][k])


def test_column_split_equals_full_batch():
    """The split the multi-GPU bench makes (bench.column_range): contexts over
    columns [0, 16) and [16, 40) of a 40-column ensemble give exactly the full
    batch's columns -- counters every day and the final state."""
    import bench
    pop = W.population(20_000, 9, 30)
    base = W.params_with(vax_on=1, vax_start=5, vax_rate=0.01)
    rp, seeds = W.batch_params(40, 3)
    T = 25
    full = gpu_sim(pop, base, keep_lambda=False, n_rep=40, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni, h = full.run(T)
    st = full.state()
    full.close()
    assert ni.sum() > 0
    for lo, hi in [bench.column_range(40, q, 2) for q in range(2)] + [(0, 16), (16, 40)]:
        part = gpu_sim(pop, base, keep_lambda=False, n_rep=hi - lo, rep_params=rp[lo:hi], rep_seeds=seeds[lo:hi],
                       max_steps=T)
        ni_p, h_p = part.run(T)
        st_p = part.state()
        part.close()
        assert np.array_equal(ni_p, ni[:, lo:hi]) and np.array_equal(h_p, h[:, lo:hi])
        for k in STATE_KEYS:
            assert np.array_equal(st_p[k].reshape(pop["n"], hi - lo), st[k][:, lo:hi]), k
