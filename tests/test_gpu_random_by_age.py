"""Age-stratified random interactions (Sec. 3 "Interaction Networks": each agent's
age-stratified number of random interactions parameterises the random network)
on the GPU against the CPU oracle, through the C-ABI: plain runs bit-exact (with
and without the internal numbering, with exposure notification), batched columns
against the oracle's per-column runs (four-replicate and general panel kernels,
exposure notification's redrawn contacts), a ragged population against its own
run, and the relaxed model's gradient against the oracle's reverse sweep."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W
from tests.helpers import compare_days, gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

MEANS = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 5.0]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_plain_runs_match_oracle():
    pop = W.population(8_000, 31, 20)
    p = W.params_with(rand_mean_age=MEANS, R=3.0, test_on=1, quar_on=1, vax_on=1, vax_start=10, vax_rate=0.02,
                      seed=5, net_seed=6)
    rep = compare_days(pop, p, 50)
    assert rep["flips"] == 0 and rep["days"] == 50, rep
    # the day's random in-contacts follow the agents' bins: their mean count is the
    # sum of the agents' means
    static = sum(int(rp[-1]) for rp in pop["row_ptr"])
    rand = np.mean(np.array(rep["messages"], np.float64) - static)
    want = float(np.sum(np.array(MEANS)[pop["age"]]))
    assert abs(rand / want - 1.0) < 0.01, (rand, want)


def test_plain_without_internal_numbering_and_with_notification():
    from tests.helpers import STATE_KEYS, gpu_sim, oracle_sim
    pop = W.population(6_000, 32, 25)
    p = W.params_with(rand_mean_age=MEANS, R=3.5, test_on=1, quar_on=1, den_on=1, seed=7, net_seed=8)
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
    assert den.tolist() == o.den_notified and sum(den) > 50


@pytest.mark.parametrize("B,den", [(4, False), (5, False), (8, True)])
def test_batched_columns_match_oracle_runs(B, den):
    from paper_2110_04421_gb300.deabm import Simulation
    T = 40
    pop = W.population(4_001, 33, 30)
    base = W.params_with(rand_mean_age=MEANS, R=3.0, test_on=1, quar_on=1, den_on=1 if den else 0, net_seed=85)
    rp, seeds = W.batch_params(B, 3)
    g = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds, max_steps=T)
    ni, _ = g.run(T)
    st = g.state()
    dn = g.notified() if den else None
    g.close()
    for c in range(B):
        pc = dict(base, R=float(rp[c, 0]), B_net=[float(rp[c, 1]), float(rp[c, 2])], B_rand=float(rp[c, 3]),
                  S_age=[float(x) for x in rp[c, 4:13]], dose2_delay=int(rp[c, 13]), seed=int(seeds[c]))
        o = oracle.Sim(pop, pc, pop["age"], pop["seed_ids"])
        o_ni, _, _ = o.run(T)
        assert np.array_equal(ni[:, c], o_ni), c
        assert np.array_equal(st["stage"][:, c], o.state.stage), c
        assert np.array_equal(st["flags"][:, c], o.state.flags), c
        if den:
            assert dn[:, c].tolist() == o.den_notified, c


def test_ragged_population_equals_its_own_run():
    from paper_2110_04421_gb300.deabm import RaggedSimulation, Simulation
    pops = [W.population(n, 40 + q, 10) for q, n in enumerate((3_001, 9_000))]
    params = [W.params_with(rand_mean_age=MEANS, R=3.5, seed=50, net_seed=51),
              W.params_with(R=3.0, seed=52, net_seed=53)]
    rg = RaggedSimulation(pops, params, max_steps=30)
    ni, _ = rg.run(30)
    rg.close()
    for q in range(2):
        s = Simulation(pops[q], params[q], pops[q]["age"], pops[q]["seed_ids"], max_steps=30)
        ni_q, _ = s.run(30)
        s.close()
        assert np.array_equal(ni[:, q], ni_q[:, 0]), q


def test_relaxed_gradient_matches_oracle():
    from paper_2110_04421_gb300.deabm import Relaxed
    pop = W.population(5_000, 34, 12)
    p = W.params_with(rand_mean_age=MEANS, R=3.0, seed=61, net_seed=62,
                      S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    T = 45
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    th = oracle.theta_of(p)
    hidden = th.copy()
    hidden[0], hidden[3] = 3.5, 1.3
    y = np.log(rx.run(hidden, T)["incidence"] + 1.0).astype(np.float32)
    g = Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5, max_days=T, ckpt_every=10)
    loss, grad, _ = g.grad(th, y)
    thetas = np.repeat(np.float32(th)[None, :], 2, axis=0)
    thetas[1, 3] *= np.float32(1.2)
    loss_b, grad_b, _ = g.grad_batch(thetas, np.repeat(y[:, None], 2, axis=1))
    g.close()
    o = rx.run(th, T, target=y.astype(np.float64), grad=True)
    scale = np.linalg.norm(o["grad"])
    assert abs(loss - o["loss"]) <= 1e-4 * o["loss"]
    assert np.max(np.abs(grad - o["grad"])) <= 1e-4 * scale, (grad, o["grad"])
    assert abs(loss_b[0] - loss) <= 1e-5 * loss and np.max(np.abs(grad_b[0] - grad)) <= 1e-5 * np.linalg.norm(grad)
