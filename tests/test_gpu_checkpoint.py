"""Checkpoint and resume through the C-ABI (deabm_save / deabm_restore).

Draws are keyed by (seed, agent, day, stream), so a run split at day T1 --
saved, restored into a fresh context, continued -- must equal the straight run
bit for bit: states, per-day counters, notifications."""
import numpy as np
import pytest

from paper_2110_04421_gb300 import workloads as W
from tests.helpers import STATE_KEYS, compare_days, gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def straight_and_split(pop, p, T1, T2, **kw):
    from paper_2110_04421_gb300.deabm import Simulation
    T = T1 + T2
    a = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=T, **kw)
    a.run(T)
    ni_a, h_a, m_a = a.counters(T)
    s_a = a.state()
    den_a = a.notified(T)
    a.close()

    b = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=T, **kw)
    b.run(T1)
    ck = b.save()
    assert ck["day"] == T1
    c = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=T, **kw)
    c.restore(ck)
    c.run(T2)
    ni_c, h_c, m_c = c.counters(T)
    s_c = c.state()
    den_c = c.notified(T)
    c.close()
    for k in STATE_KEYS:
        assert np.array_equal(s_a[k], s_c[k]), k
    assert np.array_equal(ni_a[T1:], ni_c[T1:]) and np.array_equal(h_a[T1:], h_c[T1:])
    assert np.array_equal(m_a[T1:], m_c[T1:]) and np.array_equal(den_a[T1:], den_c[T1:])
    # the same context rewound to the checkpoint
    b.restore(ck)
    b.run(T2)
    s_b = b.state()
    ni_b, _, _ = b.counters(T)
    b.close()
    for k in STATE_KEYS:
        assert np.array_equal(s_a[k], s_b[k]), k
    assert np.array_equal(ni_a[T1:], ni_b[T1:])
    return ni_a


def test_resume_with_strategy_notification_and_daily_occupations():
    pop = dict(W.population_daily_occupation(5000, 3, 30), occ_lattice=1, occ_rewire=0.1)
    p = W.params_with(test_on=1, quar_on=1, den_on=1, den_adoption=0.5, vax_on=1, vax_start=8, vax_rate=0.02,
                      vax_strategy=3, dose2_delay=9, R=4.0, seed=6, net_seed=7)
    ni = straight_and_split(pop, p, 23, 17)
    assert ni.sum() > 300


def test_resume_static_schedule_stored_networks():
    pop = W.population(6000, 4, 30)
    p = W.params_with(test_on=1, quar_on=1, vax_on=1, vax_start=5, vax_rate=0.01, R=3.5, seed=8, net_seed=9)
    straight_and_split(pop, p, 12, 25)
    straight_and_split(pop, p, 12, 25, locality_order=False)


def test_resume_batched():
    from paper_2110_04421_gb300.deabm import Simulation
    n, B, T1, T2 = 3001, 36, 15, 15
    pop = W.population(n, 5, 30)
    base = W.params_with(test_on=1, quar_on=1, vax_on=1, vax_start=5, vax_rate=0.01, net_seed=3)
    rp, seeds = W.batch_params(B, 4)
    kw = dict(n_rep=B, rep_params=rp, rep_seeds=seeds)
    straight_and_split(pop, base, T1, T2, **kw)


def test_restore_rejects_bad_input():
    from paper_2110_04421_gb300.deabm import DeabmError, RaggedSimulation, Simulation
    pop = W.population(500, 1, 5)
    p = W.params_with()
    g = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=10)
    g.run(3)
    ck = g.save()
    bad = dict(ck, stage=ck["stage"].copy())
    bad["stage"][7] = 11
    with pytest.raises(DeabmError):
        g.restore(bad)
    with pytest.raises(DeabmError):
        g.restore(dict(ck, day=11))
    g.close()
    r = RaggedSimulation([pop], [p], max_steps=5)
    with pytest.raises(DeabmError):
        from paper_2110_04421_gb300.deabm import lib
        import ctypes as C
        day = C.c_uint32()
        rc = lib().deabm_save(r.ctx, None, None, None, None, None, None, None, C.byref(day))
        if rc != 0:
            raise DeabmError(rc, "ragged")
    r.close()


def test_allocation_failure_in_create_reports_enomem_and_frees_everything():
    """The library's allocation-failure injection makes the k-th device allocation
    of deabm_create fail, for every k a create makes: each attempt returns
    DEABM_ENOMEM with no context, the device's free memory is back where it was,
    and a create without injection then runs and matches the oracle."""
    import torch
    from paper_2110_04421_gb300.deabm import ENOMEM, DeabmError, Simulation, lib
    pop = W.population(30_000, 2, 20)
    p = W.params_with(test_on=1, quar_on=1, vax_on=1, vax_start=2, vax_rate=0.02, R=3.0)
    Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=5).close()  # device code of create loaded once
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    k = 1
    try:
        while True:
            lib().deabm_inject_alloc_failure(k)
            try:
                s = Simulation(pop, p, pop["age"], pop["seed_ids"], max_steps=5)
            except DeabmError as e:
                assert e.code == ENOMEM, e
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free0, (k, free0 - torch.cuda.mem_get_info()[0])
                k += 1
                assert k < 200
                continue
            s.close()
            break
    finally:
        lib().deabm_inject_alloc_failure(0)
    assert k > 3  # create makes several device allocations, each one was made to fail
    rep = compare_days(pop, p, 5)
    assert rep["days"] == 5
