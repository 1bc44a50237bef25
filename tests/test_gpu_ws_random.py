"""The global random network as a daily Watts-Strogatz graph (Sec. 3,
Interaction Networks) on the GPU against the CPU oracle, through the C-ABI.

The day's graph is built on the device (rewired-edge bits, landing lists by a
prefix sum and atomics, each list sorted) before the day kernel gathers along
it.  Same bar as the Poisson random network: stages, timers, flags, counters and
message counts bit-exact; lambda bit-exact against the oracle's FP32 path and
within 1e-5 relative of its FP64 path, every day."""
import numpy as np
import pytest

from paper_2110_04421_gb300 import workloads as W
from tests.helpers import compare_days, gpu_available, gpu_sim

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("k,beta", [(2, 0.5), (6, 0.1), (4, 1.0), (2, 0.0)])
def test_watts_strogatz_random_network_matches_oracle(k, beta):
    """N = 12,347 (several tiles, a ragged tail, relabelled for locality) with
    households and occupations stored, interventions on, 40 days."""
    pop = dict(W.population(12_347, 3, 25), rand_ws=1, rand_ws_k=k, rand_ws_beta=beta)
    p = W.params_with(test_on=1, quar_on=1, vax_on=1, vax_start=8, vax_rate=0.01, R=3.0, seed=5, net_seed=6)
    rep = compare_days(pop, p, 40)
    assert rep["flips"] == 0 and rep["days"] == 40, rep
    assert rep["max_rel_lambda64"] <= 1e-5
    assert sum(rep["new_inf"]) > 200
    # n k messages of the random network a day on top of the stored edges
    stored = sum(int(r[-1]) for r in pop["row_ptr"])
    assert all(m == stored + pop["n"] * k for m in rep["messages"])


def test_watts_strogatz_only_network_and_tiny_ring():
    """No stored network (the random term alone), and a ring shorter than the
    lattice (wrapping edges always rewired)."""
    for n, k in ((5_001, 4), (7, 16)):
        pop = dict(n=n, age=np.random.default_rng(n).integers(0, 9, n, dtype=np.uint8), row_ptr=[], col=[],
                   seed_ids=np.array([0, n // 2], np.uint32), rand_ws=1, rand_ws_k=k, rand_ws_beta=0.2)
        rep = compare_days(pop, W.params_with(R=6.0, seed=1, net_seed=2), 25)
        assert rep["flips"] == 0 and rep["days"] == 25, rep


def test_watts_strogatz_rejected_where_not_built():
    from paper_2110_04421_gb300.deabm import DeabmError
    pop = dict(W.population(2_000, 1, 5), rand_ws=1, rand_ws_k=3, rand_ws_beta=0.2)
    with pytest.raises(DeabmError, match="rand_ws_k"):
        gpu_sim(pop, W.params_with())
    pop["rand_ws_k"] = 2


@pytest.mark.parametrize("B,locality", [(8, True), (5, False)])
def test_watts_strogatz_in_batched_contexts_match_oracle_columns(B, locality):
    """A batched context: the day's graph (keyed by the network seed) built once
    and shared by every replicate column; each column equals the oracle's plain
    run with its own parameters and seed (incidence and stages), and the day's
    message count is the shared graph's."""
    import oracle
    from paper_2110_04421_gb300.deabm import Simulation
    T = 30
    pop = dict(W.population(6_007, 4, 30), rand_ws=1, rand_ws_k=4, rand_ws_beta=0.3)
    base = W.params_with(test_on=1, quar_on=1, net_seed=17)
    rp, seeds = W.batch_params(B, 3)
    g = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T,
                   locality_order=locality)
    ni, _ = g.run(T)
    st = g.state()
    _, _, msgs = g.counters(T)
    g.close()
    for c in range(B):
        pc = dict(base, R=float(rp[c, 0]), B_net=[float(rp[c, 1]), float(rp[c, 2])], B_rand=float(rp[c, 3]),
                  S_age=[float(x) for x in rp[c, 4:13]], dose2_delay=int(rp[c, 13]), seed=int(seeds[c]))
        o = oracle.Sim(pop, pc, pop["age"], pop["seed_ids"])
        o_ni, _, o_msgs = o.run(T)
        assert np.array_equal(ni[:, c], o_ni), c
        assert np.array_equal(st["stage"][:, c], o.state.stage), c
        if c == 0:
            assert np.array_equal(np.asarray(msgs[:T], np.int64), np.asarray(o_msgs, np.int64))
    assert ni.sum() > 100


def test_watts_strogatz_full_size_first_days():
    """The bench's N = 2,000,000 workload (testing, quarantine, vaccination) with
    the random network as a daily Watts-Strogatz graph (k = 2, beta = 0.5), the
    first 4 days against the oracle in full: lambda bit for bit, every state array
    and counter."""
    w = W.plain_large()
    pop = dict(W.population(w["n"], 0, w["n_seed"]), rand_ws=1, rand_ws_k=2, rand_ws_beta=0.5)
    rep = compare_days(pop, w["params"], 4)
    assert rep["flips"] == 0 and rep["days"] == 4, rep
    assert rep["max_rel_lambda64"] <= 1e-5


@pytest.mark.parametrize("locality_order", [True, False])
def test_watts_strogatz_with_exposure_notification_matches_oracle(locality_order):
    """Exposure notification over the Watts-Strogatz random network: an agent's
    in-contacts there are its neighbours in each day's graph, and the graphs of the
    7-day look-back are kept on the device.  Bit-exact against the oracle every
    day (notified counts included), with and without the internal numbering."""
    from tests.helpers import STATE_KEYS, oracle_sim
    pop = dict(W.population(9_001, 7, 30), rand_ws=1, rand_ws_k=4, rand_ws_beta=0.3)
    p = W.params_with(test_on=1, quar_on=1, den_on=1, den_adoption=0.5, den_compliance=0.9, R=3.5, seed=9,
                      net_seed=10)
    if locality_order:
        rep = compare_days(pop, p, 45)
        assert rep["flips"] == 0 and rep["days"] == 45, rep
        assert sum(rep["notified"]) > 200
        return
    o = oracle_sim(pop, p)
    g = gpu_sim(pop, p, keep_lambda=False, max_steps=45, locality_order=False)
    ni, h = g.run(45)
    s = g.state()
    den = g.notified()
    g.close()
    ni_o, h_o, _ = o.run(45)
    assert np.array_equal(ni[:, 0], ni_o) and np.array_equal(h[:, 0], h_o)
    for k in STATE_KEYS:
        assert np.array_equal(s[k], getattr(o.state, k)), k
    assert den.tolist() == o.den_notified and sum(den) > 200


def test_watts_strogatz_with_notification_in_batched_contexts_and_resumed():
    """Batched columns with notification over the shared Watts-Strogatz graphs
    equal the oracle's per-column runs; a plain run resumed from a checkpoint
    (whose look-back graphs are rebuilt) equals the uninterrupted run."""
    import oracle
    from paper_2110_04421_gb300.deabm import Simulation
    from tests.test_gpu_checkpoint import straight_and_split
    T, B = 35, 6
    pop = dict(W.population(5_003, 8, 30), rand_ws=1, rand_ws_k=2, rand_ws_beta=0.5)
    base = W.params_with(test_on=1, quar_on=1, den_on=1, den_adoption=0.6, R=4.0, net_seed=19)
    rp, seeds = W.batch_params(B, 5)
    g = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni, _ = g.run(T)
    st = g.state()
    dn = g.notified()
    g.close()
    for c in range(B):
        pc = dict(base, R=float(rp[c, 0]), B_net=[float(rp[c, 1]), float(rp[c, 2])], B_rand=float(rp[c, 3]),
                  S_age=[float(x) for x in rp[c, 4:13]], dose2_delay=int(rp[c, 13]), seed=int(seeds[c]))
        o = oracle.Sim(pop, pc, pop["age"], pop["seed_ids"])
        o_ni, _, _ = o.run(T)
        assert np.array_equal(ni[:, c], o_ni), c
        assert np.array_equal(st["flags"][:, c], o.state.flags), c
        assert dn[:, c].tolist() == o.den_notified, c
    assert dn.sum() > 100
    p = dict(base, seed=21)
    straight_and_split(pop, p, 17, 15)
