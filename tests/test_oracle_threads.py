"""The oracle's per-agent loops on several host threads (OpenMP over agents)
give the same trajectory bit for bit as one thread: every state array, lambda
in both precisions, the counters and the notifications, with every intervention
and exposure notification on."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W

KEYS = ("stage", "timer", "tinf", "flags", "qt")


def run(pop, p, T, threads):
    oracle.set_threads(threads)
    try:
        sim = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
        days = [sim.step(diag=True) for _ in range(T)]
        return days, {k: getattr(sim.state, k).copy() for k in KEYS}, list(sim.den_notified)
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("daily_occ", [False, True])
def test_thread_count_changes_nothing(daily_occ):
    if oracle.set_threads(4) != 4:
        oracle.set_threads(1)
        pytest.skip("oracle built without OpenMP")
    oracle.set_threads(1)
    pop = W.population_daily_occupation(6000, 2, 30) if daily_occ else W.population(6000, 2, 30)
    p = W.params_with(R=4.0, test_on=1, quar_on=1, q_dropout=0.05, vax_on=1, vax_start=3, vax_rate=0.02,
                      den_on=1, den_adoption=0.5, seed=5, net_seed=6)
    d1, s1, n1 = run(pop, p, 25, 1)
    d4, s4, n4 = run(pop, p, 25, 4)
    for a, b in zip(d1, d4):
        assert a["new_inf"] == b["new_inf"] and a["messages"] == b["messages"]
        assert np.array_equal(a["lambda32"].view(np.uint32), b["lambda32"].view(np.uint32))
        assert np.array_equal(a["lambda64"].view(np.uint64), b["lambda64"].view(np.uint64))
        assert np.array_equal(a["hist"], b["hist"])
    for k in KEYS:
        assert np.array_equal(s1[k], s4[k]), k
    assert n1 == n4 and sum(n1) > 0
    assert sum(d["new_inf"] for d in d1) > 100
