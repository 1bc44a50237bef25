"""Pins for the transmission step (Eq. 1-2) on tiny graphs.

* brute force: for every destination j, enumerate all 2^E outcomes of its
  independent interactions, each transmitting with P_e = 1 - exp(-lambda_e)
  (Eq. 2) where lambda_e is Eq. 1 for that single interaction; the probability
  that at least one transmits must equal the oracle's 1 - exp(-lambda_j).
* star graph: one infected centre gives every leaf the single-term closed form,
  and the number of infected leaves matches n*p within a binomial band.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W

# reading of the stage list: infectious stages and their symptom class
CLASS_OF_STAGE = {1: 0, 2: 1, 4: 1, 3: 2, 5: 2}


def erlang_day(t, k, theta):
    def F(x):
        if x <= 0:
            return 0.0
        y = x / theta
        return 1.0 - math.exp(-y) * sum(y**m / math.factorial(m) for m in range(k))
    return F(t) - F(t - 1)


def csr(n, edges):
    """edges: list of (src, dst) -> destination-sorted CSR keeping list order within a row"""
    rows = [[] for _ in range(n)]
    for s, d in edges:
        rows[d].append(s)
    rp = np.zeros(n + 1, np.uint32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([s for r in rows for s in r], np.uint32)
    return rp, col


def make_state(n, infected):
    st = oracle.State(n)
    for i, (stage, tinf, quar) in infected.items():
        st.stage[i] = stage
        st.tinf[i] = tinf
        st.timer[i] = 5
        st.qt[i] = quar
    return st


def per_edge_lambda(p, stage, tinf, qt, age_dst, src, net_weight):
    c = CLASS_OF_STAGE.get(int(stage[src]))
    if c is None or (qt[src] & 0x0F) or tinf[src] >= p["inf_len"]:
        return 0.0
    f = erlang_day(int(tinf[src]), int(p["inf_shape"][c]), p["inf_scale"][c])
    f32 = lambda x: float(np.float32(x))  # Eq. 1's scale factors are FP32 parameters
    return f32(p["R"]) * f32(p["S_age"][age_dst]) * f32(p["A_class"][c]) * f32(net_weight) * f32(p["inv_Ibar"]) * f


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_enumeration_matches_aggregate(seed):
    rng = np.random.default_rng(seed)
    n = 9
    hh = [(s, d) for s in range(n) for d in range(n) if s != d and rng.random() < 0.35]
    oc = [(s, d) for s in range(n) for d in range(n) if s != d and rng.random() < 0.25]
    # cap to at most 12 interactions per destination so 2^E stays small
    hh = [e for e in hh if sum(1 for x in hh if x[1] == e[1]) <= 6][:40]
    oc = [e for e in oc if sum(1 for x in oc if x[1] == e[1]) <= 6][:40]
    rp0, c0 = csr(n, hh)
    rp1, c1 = csr(n, oc)
    p = W.params_with(R=2.5, inv_Ibar=0.2, B_net=[2.0, 0.7], rand_mean=0.0,
                      S_age=list(rng.uniform(0.3, 1.5, 9)), A_class=[0.4, 1.0, 1.3],
                      inf_shape=[4.0, 3.0, 2.0], inf_scale=[1.25, 1.5, 2.0])
    age = rng.integers(0, 9, n).astype(np.uint8)
    infected = {}
    for i in range(n):
        r = rng.random()
        if r < 0.6:
            stage = int(rng.choice([1, 2, 3, 4, 5, 6, 7, 8]))
            infected[i] = (stage, int(rng.integers(0, 12)), int(rng.random() < 0.2) * 5)
    st = make_state(n, infected)
    g = dict(n=n, row_ptr=[rp0, rp1], col=[c0, c1])
    sim = oracle.Sim(g, p, age, None, state=st)
    d = sim.step()
    for j in range(n):
        lam_e = [per_edge_lambda(p, st.stage, st.tinf, st.qt, age[j], s, p["B_net"][0]) for s, dd in hh if dd == j]
        lam_e += [per_edge_lambda(p, st.stage, st.tinf, st.qt, age[j], s, p["B_net"][1]) for s, dd in oc if dd == j]
        P_e = [1.0 - math.exp(-x) for x in lam_e]
        p_any = 0.0
        for outcome in itertools.product([0, 1], repeat=len(P_e)):
            if any(outcome):
                pr = 1.0
                for o, pe in zip(outcome, P_e):
                    pr *= pe if o else (1.0 - pe)
                p_any += pr
        assert abs(d["lambda64"][j] - sum(lam_e)) <= 1e-12 * max(1.0, sum(lam_e))
        assert abs(-math.expm1(-d["lambda64"][j]) - p_any) <= 1e-12
        assert abs(float(d["p32"][j]) - p_any) <= 2e-7
        assert abs(float(d["lambda32"][j]) - d["lambda64"][j]) <= 1e-5 * max(d["lambda64"][j], 1e-30)


def test_star_graph_closed_form_and_frequency():
    n_leaves = 40
    n = n_leaves + 1
    centre = 0
    rp, col = csr(n, [(centre, d) for d in range(1, n)])
    rpr, colr = csr(n, [(s, centre) for s in range(1, n)])
    p = W.params_with(R=3.0, inv_Ibar=0.25, B_net=[1.5, 0.0], rand_mean=0.0, S_age=[0.8] * 9)
    age = np.zeros(n, np.uint8)
    tau = 4
    st = make_state(n, {centre: (4, tau, 0)})  # mild symptomatic, 4 days since infection
    g = dict(n=n, row_ptr=[rp, rpr], col=[col, colr])
    d = oracle.Sim(g, p, age, None, state=st).step()
    want = 3.0 * float(np.float32(0.8)) * 1.0 * 1.5 * 0.25 * erlang_day(tau, 4, 1.25)
    assert np.allclose(d["lambda64"][1:], want, rtol=1e-12, atol=0)
    assert d["lambda64"][centre] == 0.0
    p_leaf = -math.expm1(-want)
    # Monte Carlo over seeds: infected leaves ~ Binomial(n_leaves, p) each trial
    tot, trials = 0, 300
    for s in range(trials):
        p2 = dict(p, seed=1000 + s)
        dd = oracle.Sim(g, p2, age, None, state=st).step(diag=False)
        tot += dd["new_inf"]
    mean = n_leaves * trials * p_leaf
    sd = math.sqrt(n_leaves * trials * p_leaf * (1 - p_leaf))
    assert abs(tot - mean) < 5 * sd, (tot, mean, sd)


def test_reversed_star_sums_leaves():
    n_leaves = 12
    n = n_leaves + 1
    rp, col = csr(n, [(s, 0) for s in range(1, n)])
    p = W.params_with(R=2.0, inv_Ibar=0.5, B_net=[1.0], rand_mean=0.0)
    age = np.full(n, 3, np.uint8)
    inf = {i: (int([1, 2, 3, 4, 5][i % 5]), 1 + i % 9, 0) for i in range(1, n)}
    st = make_state(n, inf)
    g = dict(n=n, row_ptr=[rp], col=[col])
    d = oracle.Sim(g, p, age, None, state=st).step()
    want = sum(per_edge_lambda(p, st.stage, st.tinf, st.qt, 3, s, 1.0) for s in range(1, n))
    assert abs(d["lambda64"][0] - want) <= 1e-12 * want


def test_random_network_term_uses_the_days_contacts():
    pop = W.population(300, 5, 30)
    p = W.params_with(rand_mean=2.0, B_rand=1.7, net_seed=77)
    sim = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
    for _ in range(3):
        sim.step(diag=False)
    st0 = sim.state.copy()
    t = sim.t
    d = sim.step()
    # rebuild lambda_j from the static sums and the day's contacts
    inf = d["inf32"].astype(np.float64)
    for j in range(0, 300, 7):
        hh = sum(inf[pop["col"][0][pop["row_ptr"][0][j]:pop["row_ptr"][0][j + 1]]])
        oc = sum(inf[pop["col"][1][pop["row_ptr"][1][j]:pop["row_ptr"][1][j + 1]]])
        cts = oracle.random_contacts(77, 300, j, t, 2.0)
        assert d["rand_k"][j] == cts.size
        rn = sum(inf[cts])
        f32 = lambda x: float(np.float32(x))
        want = f32(p["R"]) * f32(p["inv_Ibar"]) * p["S_age"][pop["age"][j]] * (2.0 * hh + 1.0 * oc + f32(1.7) * rn)
        assert abs(d["lambda64"][j] - want) <= 1e-6 * max(want, 1e-12)
    # messages = static in-edges + random in-contacts
    assert d["messages"] == int(pop["row_ptr"][0][-1]) + int(pop["row_ptr"][1][-1]) + int(d["rand_k"].sum())
    del st0


def test_messages_of_susceptible_destinations(oracle_lib):
    """The oracle's messages_sus counts exactly the in-edges (stored rows, the day's
    random contacts) of the agents susceptible at the start of the day."""
    import oracle
    from paper_2110_04421_gb300 import workloads as W
    pop = W.population(3000, 4, 40)
    p = W.params_with(R=5.0, seed=3, net_seed=4)
    sim = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
    deg = sum(np.diff(rp.astype(np.int64)) for rp in pop["row_ptr"])
    seen_partial = False
    for _ in range(15):
        sus = sim.state.stage == 0
        d = sim.step(diag=True)
        want = int((deg[sus] + d["rand_k"][sus].astype(np.int64)).sum())
        assert d["messages_sus"] == want
        assert d["messages"] == int((deg + d["rand_k"].astype(np.int64)).sum())
        seen_partial |= 0 < d["messages_sus"] < d["messages"]
    assert seen_partial
