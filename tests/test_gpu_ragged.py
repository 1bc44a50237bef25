"""Ragged batch (several populations of different sizes in one persistent launch
per day, days replayed as a CUDA graph): each population must reproduce its own
single-population run exactly, before and after autotuning and reset."""
import numpy as np
import pytest

from paper_2110_04421_gb300 import workloads as W
from tests.helpers import gpu_available, oracle_sim

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def case():
    sizes = [2000, 157, 5003, 33, 1200, 9000]
    pops, params = [], []
    for q, n in enumerate(sizes):
        pops.append(W.population(n, 40 + q, max(1, n // 50)))
        params.append(W.params_with(R=2.5 + q * 0.6, seed=100 + q, net_seed=200 + q, test_on=q % 2, quar_on=q % 2,
                                    vax_on=int(q >= 3), vax_start=4, vax_rate=0.02))
    return pops, params


def single_runs(pops, params, T):
    from paper_2110_04421_gb300.deabm import Simulation
    out = []
    for pop, par in zip(pops, params):
        s = Simulation(pop, par, pop["age"], pop["seed_ids"], max_steps=T, locality_order=False)
        ni, h = s.run(T)
        out.append((ni[:, 0], h[:, 0], s.state()))
        s.close()
    return out


def check(ragged_out, singles):
    ni, h, states = ragged_out
    for q, (ni1, h1, st1) in enumerate(singles):
        assert np.array_equal(ni[:, q], ni1), q
        assert np.array_equal(h[:, q], h1), q
        for k in st1:
            assert np.array_equal(states[q][k], st1[k]), (q, k)


@pytest.mark.parametrize("locality", [True, False])
def test_each_population_matches_its_own_run(locality):
    """locality: each population numbered internally for locality (its random
    contacts through a caller id -> row map) or kept in caller order."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation
    pops, params = case()
    T = 35
    singles = single_runs(pops, params, T)
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    r.reset()
    ni2, h2 = r.run(T)  # graph replay after a reset
    assert np.array_equal(ni, ni2) and np.array_equal(h, h2)
    r.close()
    for q in (1, 3):  # the two smallest against the oracle
        o = oracle_sim(pops[q], params[q])
        ni_o, h_o, _ = o.run(T)
        assert np.array_equal(ni_o, ni[:, q]) and np.array_equal(h_o, h[:, q])


def test_autotuned_tiling_changes_nothing():
    from paper_2110_04421_gb300.deabm import RaggedSimulation
    pops, params = case()
    T = 20
    singles = single_runs(pops, params, T)
    r = RaggedSimulation(pops, params, max_steps=T)
    rows, bps = r.autotune(days_per_trial=2)
    assert rows in (256, 512, 1024, 2048, 4096) and bps in (2, 4, 6, 8)
    r.step(T)
    r.sync()
    ni, h, _ = r.counters(T)
    check((ni, h, r.state()), singles)
    r.close()


@pytest.mark.parametrize("locality", [True, False])
def test_daily_occupations_in_ragged_batches(locality):
    """Populations that draw their occupation contacts daily (one of them as
    rewired ring lattices) mixed with ones that store them: each population of
    the ragged batch equals its own single-population run, and the small one
    the oracle."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation
    pops, params = case()
    for q, lattice in ((0, 0), (2, 1), (3, 0)):
        p = pops[q]
        p["row_ptr"], p["col"] = p["row_ptr"][:1], p["col"][:1]  # households stay stored
        p["occ_group"], p["occ_k"] = W.occupations(p["n"], 60 + q, n_occ=4 if p["n"] < 100 else 23)
        if lattice:
            p["occ_lattice"], p["occ_rewire"] = 1, 0.2
    T = 30
    singles = single_runs(pops, params, T)
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    r.close()
    assert ni[:, 0].sum() > 0 and ni[:, 2].sum() > 0
    o = oracle_sim(pops[3], params[3])  # the 33-agent population with daily occupations
    ni_o, h_o, _ = o.run(T)
    assert np.array_equal(ni_o, ni[:, 3]) and np.array_equal(h_o, h[:, 3])


@pytest.mark.parametrize("locality", [True, False])
def test_priority_strategies_in_ragged_batches(locality):
    """Populations under the three vaccination priority strategies (Sec. 5,
    Table 1) mixed with ones on the static schedule and without vaccination: each
    population selects its own doses from its own state before each day, and each
    equals its own single-population run (states, dose bits included, and
    counters), the 33-agent one also the oracle; a reset and rerun gives the same."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation
    pops, params = case()
    for q, strategy in ((0, 1), (2, 2), (3, 3), (5, 3)):
        params[q] = dict(params[q], vax_on=1, vax_start=3, vax_rate=0.03, vax_strategy=strategy,
                         dose2_delay=6 + q, elderly_bin=6)
    T = 30
    singles = single_runs(pops, params, T)
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    r.reset()
    ni2, h2 = r.run(T)
    assert np.array_equal(ni2, ni) and np.array_equal(h2, h)
    states = r.state()
    r.close()
    for q in (0, 5):  # (strategy 2 puts every first dose before any second: none in 30 days there)
        assert (states[q]["flags"] & 0x02).sum() > 0, q  # second doses were given
    assert (states[2]["flags"] & 0x01).sum() > 3000
    o = oracle_sim(pops[3], params[3])
    ni_o, h_o, _ = o.run(T)
    assert np.array_equal(ni_o, ni[:, 3]) and np.array_equal(h_o, h[:, 3])


@pytest.mark.parametrize("locality", [True, False])
def test_watts_strogatz_random_networks_in_ragged_batches(locality):
    """Populations whose random network is a daily Watts-Strogatz graph (each its
    own, built before each day) mixed with Poisson ones: each population equals
    its own single-population run, the 33-agent one also the oracle."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation
    pops, params = case()
    for q, (k, beta) in ((1, (4, 0.2)), (2, (2, 0.5)), (3, (6, 0.1))):
        pops[q] = dict(pops[q], rand_ws=1, rand_ws_k=k, rand_ws_beta=beta)
    T = 30
    singles = single_runs(pops, params, T)
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    r.close()
    assert ni[:, 2].sum() > 0
    o = oracle_sim(pops[3], params[3])
    ni_o, h_o, _ = o.run(T)
    assert np.array_equal(ni_o, ni[:, 3]) and np.array_equal(h_o, h[:, 3])


@pytest.mark.parametrize("locality", [True, False])
def test_exposure_notification_in_ragged_batches(locality):
    """Populations with digital exposure notification (Sec. 4.2: each its own app
    holders, look-back window and compliance draws; one with daily occupation
    contacts, one under a priority strategy) mixed with ones without it: each
    population equals its own single-population run (states, counters and the
    daily notification counts, a column of [day][population]), the 157-agent one
    also the oracle; a reset and rerun gives the same."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation, Simulation
    pops, params = case()
    den = dict(test_on=1, quar_on=1, den_on=1, den_compliance=0.8)
    for q, (adopt, window) in ((1, (0.9, 7)), (2, (0.4, 7)), (3, (1.0, 3)), (5, (0.3, 12))):
        params[q] = dict(params[q], den_adoption=adopt, den_window=window, R=3.5, **den)
    p = pops[2]
    p["row_ptr"], p["col"] = p["row_ptr"][:1], p["col"][:1]
    p["occ_group"], p["occ_k"] = W.occupations(p["n"], 62, n_occ=23)
    params[5] = dict(params[5], vax_on=1, vax_start=3, vax_rate=0.03, vax_strategy=1, dose2_delay=8, elderly_bin=6)
    T = 40
    singles, notified = [], []
    for pop, par in zip(pops, params):
        s = Simulation(pop, par, pop["age"], pop["seed_ids"], max_steps=T, locality_order=False)
        ni1, h1 = s.run(T)
        singles.append((ni1[:, 0], h1[:, 0], s.state()))
        notified.append(s.notified(T))
        s.close()
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    nt = r.notified(T)
    for q in range(len(pops)):
        assert np.array_equal(nt[:, q], notified[q]), q
    assert not nt[:, [0, 4]].any()
    for q in (1, 2, 5):
        assert nt[:, q].sum() > 20, q
    r.reset()
    ni2, h2 = r.run(T)
    assert np.array_equal(ni2, ni) and np.array_equal(h2, h) and np.array_equal(r.notified(T), nt)
    r.close()
    o = oracle_sim(pops[1], params[1])
    ni_o, h_o, _ = o.run(T)
    assert np.array_equal(ni_o, ni[:, 1]) and np.array_equal(h_o, h[:, 1])
    assert list(nt[:, 1]) == o.den_notified


@pytest.mark.parametrize("locality", [True, False])
def test_notification_over_watts_strogatz_networks_in_ragged_batches(locality):
    """Populations with exposure notification whose random network is a daily
    Watts-Strogatz graph (each keeps its look-back window's graphs in a ring of
    its own, the day's slot chosen on the device inside the captured days),
    beside Poisson and notification-free ones: each population equals its own
    single-population run, notification counts included; the 157-agent one also
    the oracle."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation, Simulation
    pops, params = case()
    den = dict(test_on=1, quar_on=1, den_on=1, den_compliance=0.8, R=4.0)
    for q, (k, beta, adopt, window) in ((1, (4, 0.2, 0.9, 7)), (2, (6, 0.1, 0.5, 5)), (4, (2, 0.5, 0.7, 1))):
        pops[q] = dict(pops[q], rand_ws=1, rand_ws_k=k, rand_ws_beta=beta)
        params[q] = dict(params[q], den_adoption=adopt, den_window=window, **den)
    pops[0] = dict(pops[0], rand_ws=1, rand_ws_k=4, rand_ws_beta=0.3)  # no notification
    params[5] = dict(params[5], den_adoption=0.5, den_window=7, **den)  # Poisson network
    T = 40
    singles, notified = [], []
    for pop, par in zip(pops, params):
        s = Simulation(pop, par, pop["age"], pop["seed_ids"], max_steps=T, locality_order=False)
        ni1, h1 = s.run(T)
        singles.append((ni1[:, 0], h1[:, 0], s.state()))
        notified.append(s.notified(T))
        s.close()
    r = RaggedSimulation(pops, params, max_steps=T, locality_order=locality)
    ni, h = r.run(T)
    check((ni, h, r.state()), singles)
    nt = r.notified(T)
    for q in range(len(pops)):
        assert np.array_equal(nt[:, q], notified[q]), q
    for q in (1, 2, 5):
        assert nt[:, q].sum() > 20, q
    r.reset()
    r.step(T)  # the days one launch sequence at a time, outside the captured graph
    r.sync()
    ni2, h2, _ = r.counters(T)
    assert np.array_equal(ni2, ni) and np.array_equal(h2, h) and np.array_equal(r.notified(T), nt)
    r.close()
    o = oracle_sim(pops[1], params[1])
    ni_o, h_o, _ = o.run(T)
    assert np.array_equal(ni_o, ni[:, 1]) and np.array_equal(h_o, h[:, 1])
    assert list(nt[:, 1]) == o.den_notified


@pytest.mark.parametrize("locality", [True, False])
def test_ragged_strategies_resume_from_given_dose_days(locality):
    """A ragged batch started from saved states (dose days of a priority strategy
    included) continues each population exactly as a plain context started from
    the same state; the dose days read back per population equal the plain ones."""
    from paper_2110_04421_gb300.deabm import RaggedSimulation, Simulation
    pops, params = case()
    for q, strategy in ((0, 1), (2, 3), (5, 2)):
        params[q] = dict(params[q], vax_on=1, vax_start=2, vax_rate=0.03, vax_strategy=strategy,
                         dose2_delay=5 + q, elderly_bin=6)
    T0, T1 = 12, 20
    saved, singles, doses = [], [], []
    for pop, par in zip(pops, params):
        s = Simulation(pop, par, pop["age"], pop["seed_ids"], max_steps=T0 + T1, locality_order=False)
        s.run(T0)
        st = s.state()
        if par.get("vax_strategy", 0):
            st["dose1_day"], st["dose2_day"] = s.dose_days()
        s.close()
        saved.append(st)
        # the continuation: a plain context from the saved state (no initial cases again)
        s2 = Simulation(pop, par, pop["age"], [], state=st, max_steps=T1, locality_order=False)
        ni1, h1 = s2.run(T1)
        singles.append((ni1[:, 0], h1[:, 0], s2.state()))
        doses.append(s2.dose_days() if par.get("vax_strategy", 0) else None)
        s2.close()
    pops2 = [dict(p, seed_ids=[]) for p in pops]
    r = RaggedSimulation(pops2, params, max_steps=T1, locality_order=locality, states=saved)
    ni, h = r.run(T1)
    check((ni, h, r.state()), singles)
    dd = r.dose_days()
    r.close()
    for q, d in enumerate(doses):
        if d is None:
            assert (dd[q][0] == 0x7FFF).all() and (dd[q][1] == 0x7FFF).all(), q
        else:
            assert np.array_equal(dd[q][0], d[0]) and np.array_equal(dd[q][1], d[1]), q
    assert (dd[2][1] != 0x7FFF).sum() > 0  # second doses given after the resume
