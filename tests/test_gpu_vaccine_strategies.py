"""Vaccination priority strategies on the GPU (daily dose selection kernels)
against the paper's worked example (Table 1) and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W
from tests.helpers import compare_days, gpu_available
from tests.test_oracle_vaccine_strategies import STRATEGY, age_bin, load_golden

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name", list(STRATEGY))
def test_table1_order_on_gpu(name):
    from paper_2110_04421_gb300.deabm import Simulation
    people, orders = load_golden()
    n = len(people)
    age = np.array([age_bin(a) for _, a, _ in people], np.uint8)
    flags = np.array([1 if e == "second" else 0 for _, _, e in people], np.uint8)
    d1 = np.array([-30 if e == "second" else 0x7FFF for _, _, e in people], np.int16)
    state = dict(stage=np.zeros(n, np.int8), timer=np.zeros(n, np.int16), tinf=np.zeros(n, np.int16), flags=flags,
                 qt=np.zeros(n, np.uint8), dose1_day=d1)
    p = W.params_with(rand_mean=0.0, vax_on=1, vax_start=0, vax_rate=1.0 / n, dose2_delay=21,
                      vax_strategy=STRATEGY[name])
    g = Simulation(dict(n=n, row_ptr=[], col=[]), p, age, None, state=state, max_steps=n)
    got = []
    for t in range(n):
        before = g.state()["flags"].copy()
        g.step(1)
        after = g.state()["flags"]
        changed = np.nonzero(after != before)[0]
        assert changed.size == 1, (t, changed)
        got.append(people[int(changed[0])][0])
    g.close()
    assert got == orders[name]


@pytest.mark.parametrize("strategy", [1, 2, 3])
def test_strategy_runs_match_oracle(strategy):
    pop = W.population(6001, 12, 40)
    p = W.params_with(vax_on=1, vax_start=3, vax_rate=0.03, dose2_delay=9, vax_strategy=strategy, R=4.0,
                      test_on=1, quar_on=1, seed=70 + strategy, net_seed=80)
    rep = compare_days(pop, p, 70)
    assert rep["flips"] == 0 and rep["days"] == 70
    # dose days equal the oracle's
    from paper_2110_04421_gb300.deabm import Simulation
    g = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=70)
    g.step(70)
    d1, d2 = g.dose_days()
    g.close()
    o = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
    o.run(70)
    assert np.array_equal(d1, o.state.vd1) and np.array_equal(d2, o.state.vd2)
    assert (d1 != 0x7FFF).sum() > 1000


@pytest.mark.parametrize("strategy", [0, 2])
def test_nonsterilising_immunity_matches_oracle(strategy):
    pop = W.population(5003, 13, 40)
    p = W.params_with(vax_on=1, vax_start=2, vax_rate=0.05, vax_eff1=0.85, dose2_delay=15, vax_strategy=strategy,
                      vax_nonsterile=1, R=4.5, seed=91, net_seed=92)
    rep = compare_days(pop, p, 60)
    assert rep["flips"] == 0 and rep["days"] == 60


@pytest.mark.parametrize("strategy,B", [(1, 8), (3, 5)])
def test_strategies_in_batched_contexts_match_oracle_columns(strategy, B):
    """A batched context under a priority strategy: every replicate column
    selects its doses from its own state with its own dose-2 delay (and the same
    supply); each column equals the oracle's plain run with that column's
    parameters and seed — incidence, stages and dose days."""
    from paper_2110_04421_gb300.deabm import Simulation
    T = 45
    pop = W.population(4001, 14, 30)
    base = W.params_with(vax_on=1, vax_start=3, vax_rate=0.03, vax_strategy=strategy, R=4.0, test_on=1, quar_on=1,
                         net_seed=85)
    rp, seeds = W.batch_params(B, 7)
    g = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni, _ = g.run(T)
    st = g.state()
    d1, d2 = g.dose_days()
    g.close()
    assert d1.shape == (pop["n"], B)
    delays = set()
    for c in range(B):
        pc = dict(base, R=float(rp[c, 0]), B_net=[float(rp[c, 1]), float(rp[c, 2])], B_rand=float(rp[c, 3]),
                  S_age=[float(x) for x in rp[c, 4:13]], dose2_delay=int(rp[c, 13]), seed=int(seeds[c]))
        delays.add(int(rp[c, 13]))
        o = oracle.Sim(pop, pc, pop["age"], pop["seed_ids"])
        o_ni, _, _ = o.run(T)
        assert np.array_equal(ni[:, c], o_ni), c
        assert np.array_equal(st["stage"][:, c], o.state.stage), c
        assert np.array_equal(d1[:, c], o.state.vd1) and np.array_equal(d2[:, c], o.state.vd2), c
        if int(rp[c, 13]) < T - 4:
            assert (d2[:, c] != 0x7FFF).sum() > 0, c  # second doses were given
    assert len(delays) > 1  # the columns' delays differ
