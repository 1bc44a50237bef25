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
