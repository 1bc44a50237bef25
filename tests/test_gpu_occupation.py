"""Daily occupation networks (Sec. 3, Interaction Networks) on the GPU against
the CPU oracle, through the C-ABI.

Same bar as the stored-network path: stages, timers, flags, counters and message
counts bit-exact; lambda bit-exact against the oracle's FP32 path and within
1e-5 relative of its FP64 path."""
import numpy as np
import pytest

from paper_2110_04421_gb300 import workloads as W
from tests.helpers import compare_days, gpu_available, gpu_sim, oracle_sim

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_23_occupations_with_households_and_interventions():
    """N = 10,000: households stored, 23 occupations drawn daily (5-15 contacts),
    random network, testing, quarantine and vaccination, 60 days."""
    pop = W.population_daily_occupation(10_000, 0, 20)
    p = W.params_with(test_on=1, quar_on=1, q_dropout=0.05, vax_on=1, vax_start=10, vax_rate=0.01, R=2.0,
                      seed=3, net_seed=4)
    rep = compare_days(pop, p, 60)
    assert rep["flips"] == 0 and rep["days"] == 60, rep
    assert rep["max_rel_lambda64"] <= 1e-5
    assert sum(rep["new_inf"]) > 500


def test_workplaces_only_ragged_last_group():
    """No stored network at all (the daily term comes first), workplaces of 20
    with a lone last member, several tiles and a ragged tail."""
    n = 20 * 301 + 1
    pop = W.population(n, 6, 25)
    group, k = W.workplaces(n, 6)
    assert np.bincount(group)[-1] == 1
    g = dict(pop, row_ptr=[], col=[], occ_group=group, occ_k=k)
    p = W.params_with(B_net=[1.3], R=5.0, test_on=1, quar_on=1, seed=8, net_seed=9)
    rep = compare_days(g, p, 45)
    assert rep["flips"] == 0 and rep["days"] == 45, rep
    assert sum(rep["new_inf"]) > 500


def test_occupations_without_random_network():
    pop = W.population_daily_occupation(4003, 2, 15)
    p = W.params_with(rand_mean=0.0, R=6.0, B_net=[1.0, 1.5], seed=1, net_seed=2)
    rep = compare_days(pop, p, 40)
    assert rep["flips"] == 0 and rep["days"] == 40, rep


@pytest.mark.parametrize("B", [37, 36])
def test_batched_columns_equal_plain_and_oracle(B):
    """B = 37: one replicate per thread; B = 36: four per thread."""
    n, T = 3001, 30
    pop = W.population_daily_occupation(n, 8, 30)
    base = W.params_with(vax_on=1, vax_start=5, vax_rate=0.01, test_on=1, quar_on=1, net_seed=5)
    rp, seeds = W.batch_params(B, 1)
    from paper_2110_04421_gb300.deabm import Simulation
    gb = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni_b, h_b = gb.run(T)
    _, _, m_b = gb.counters()
    sb = gb.state()
    gb.close()
    for r in (0, 5, B - 1):
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
            ni_o, h_o, m_o = o.run(T)
            assert np.array_equal(ni_o, ni_b[:, r]) and np.array_equal(h_o, h_b[:, r])
            assert np.array_equal(o.state.stage, sb["stage"][:, r])
            assert np.array_equal(m_o, m_b.astype(np.int64))


@pytest.mark.parametrize("beta", [0.0, 0.1, 1.0])
def test_watts_strogatz_occupations(beta):
    """Watts-Strogatz contacts rewired daily: 23 occupations, households stored."""
    pop = dict(W.population_daily_occupation(6_001, 9, 20), occ_lattice=1, occ_rewire=beta)
    p = W.params_with(test_on=1, quar_on=1, R=2.5, seed=5, net_seed=6)
    rep = compare_days(pop, p, 40)
    assert rep["flips"] == 0 and rep["days"] == 40, rep


def test_watts_strogatz_small_rings_and_notification():
    """Workplaces of 20 with a ragged last one of 3 members (lattice offsets that
    wrap onto the member itself are rewired), with exposure notification on, so
    the recorded contacts of the lattice feed the notification pass."""
    n = 20 * 250 + 3
    pop = W.population(n, 10, 30)
    group, k = W.workplaces(n, 10)
    g = dict(pop, row_ptr=pop["row_ptr"][:1], col=pop["col"][:1], occ_group=group, occ_k=k, occ_lattice=1,
             occ_rewire=0.2)
    p = W.params_with(test_on=1, quar_on=1, R=4.0, den_on=1, den_adoption=0.6, seed=2, net_seed=3)
    rep = compare_days(g, p, 45)
    assert rep["flips"] == 0 and rep["days"] == 45, rep
    assert sum(rep["notified"]) > 20


@pytest.mark.parametrize("B", [37, 36])
def test_watts_strogatz_batched(B):
    n, T = 2501, 25
    pop = dict(W.population_daily_occupation(n, 11, 25), occ_lattice=1, occ_rewire=0.15)
    base = W.params_with(test_on=1, quar_on=1, net_seed=7)
    rp, seeds = W.batch_params(B, 2)
    from paper_2110_04421_gb300.deabm import Simulation
    gb = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni_b, h_b = gb.run(T)
    sb = gb.state()
    gb.close()
    for r in (0, B - 1):
        pr = dict(base, R=float(rp[r, 0]), B_net=[float(rp[r, 1]), float(rp[r, 2])], B_rand=float(rp[r, 3]),
                  S_age=[float(x) for x in rp[r, 4:13]], dose2_delay=int(rp[r, 13]), seed=int(seeds[r]))
        o = oracle_sim(pop, pr)
        ni_o, h_o, _ = o.run(T)
        assert np.array_equal(ni_o, ni_b[:, r]) and np.array_equal(h_o, h_b[:, r])
        for k in ("stage", "timer", "tinf", "flags", "qt"):
            assert np.array_equal(getattr(o.state, k), sb[k][:, r]), (r, k)
