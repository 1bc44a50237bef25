"""Pins for the oracle's Watts-Strogatz global random network (Sec. 3
"Interaction Networks": one small-world Watts-Strogatz graph re-initialised
every step; Watts and Strogatz 1998), from what the construction fixes: at
beta = 0 the exact ring lattice and its textbook clustering coefficient
3(k-2)/(4(k-1)); undirected edges (symmetric adjacency, degree sum n k) at
every beta; the rewired share beta (binomial band); at beta = 1 far ends
uniform over the other agents (chi-square); rings shorter than the lattice
never give an agent itself; and the infection rate of a single infectious
agent's lattice neighbours in closed form."""
import math

import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W


def model(n, k, beta, seed=0, **kw):
    g = dict(n=n, row_ptr=[], col=[], rand_ws=1, rand_ws_k=k, rand_ws_beta=beta)
    return oracle.Model(g, W.params_with(net_seed=seed, **kw))


def adjacency(start, nb, n):
    A = np.zeros((n, n), np.int64)
    for j in range(n):
        for i in nb[start[j]:start[j + 1]]:
            A[j, i] += 1
    return A


@pytest.mark.parametrize("k", [2, 4, 6, 10])
def test_beta_zero_is_the_ring_lattice(k):
    n, h = 200, k // 2
    start, nb = model(n, k, 0.0).ws_neighbours(3)
    for j in range(n):
        want = [(j + m) % n for m in range(1, h + 1)] + [(j - m) % n for m in range(1, h + 1)]
        assert nb[start[j]:start[j + 1]].tolist() == want
    A = adjacency(start, nb, n)
    assert np.array_equal(A, A.T)
    if k >= 4:  # clustering coefficient of the ring lattice (Watts and Strogatz 1998)
        S = (A > 0).astype(np.int64)
        tri = np.einsum("ij,jk,ki->i", S, S, S) / 2
        deg = S.sum(1)
        C = np.mean(tri / (deg * (deg - 1) / 2))
        assert C == pytest.approx(3 * (k - 2) / (4 * (k - 1)), abs=1e-12)


@pytest.mark.parametrize("beta", [0.1, 0.5, 1.0])
def test_undirected_edges_and_degree_sum(beta):
    n, k = 300, 6
    m = model(n, k, beta, seed=7)
    for day in (0, 1, 9):
        start, nb = m.ws_neighbours(day)
        A = adjacency(start, nb, n)
        assert np.array_equal(A, A.T)          # each edge is heard at both ends
        assert int(start[-1]) == n * k         # n k / 2 edges, two ends each
        assert np.all(np.diag(A) == 0)         # no agent is its own neighbour


def test_rewired_share_is_beta():
    n, k, beta = 4000, 4, 0.3
    m = model(n, k, beta, seed=11)
    h = k // 2
    rewired = 0
    days = 5
    for day in range(days):
        start, nb = m.ws_neighbours(day)
        for j in range(n):
            own = nb[start[j]:start[j] + h]
            rewired += sum(int(v != (j + e + 1) % n) for e, v in enumerate(own))
    total = n * h * days
    # a rewired edge lands back on the lattice neighbour with probability 1/(n-1)
    p = beta * (1 - 1 / (n - 1))
    sd = math.sqrt(total * p * (1 - p))
    assert abs(rewired - total * p) < 5 * sd


def test_beta_one_far_ends_are_uniform():
    n, k = 50, 2
    m = model(n, k, 1.0, seed=5)
    counts = np.zeros(n, np.int64)
    j0 = 17
    for day in range(4000):
        start, nb = m.ws_neighbours(day)
        counts[nb[start[j0]]] += 1   # the far end of agent 17's own edge
        assert start[j0 + 1] - start[j0] >= 1
    assert counts[j0] == 0
    obs = np.delete(counts, j0)
    exp = obs.sum() / (n - 1)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < 95.0  # chi-square, 48 degrees of freedom: p ~ 1e-4


def test_short_rings_never_return_the_agent():
    for n in (2, 3, 5):
        start, nb = model(n, 16, 0.0, seed=2).ws_neighbours(1)
        for j in range(n):
            assert j not in nb[start[j]:start[j + 1]].tolist()
        assert int(start[-1]) == n * 16


def test_single_infectious_agent_reaches_its_lattice_neighbours():
    """beta = 0, k = 4, one infectious agent c: lambda_j = (R/I) S B_r inf_c for the
    four agents c +- 1, c +- 2 (one term each) and 0 elsewhere."""
    n, k, c = 60, 4, 25
    g = dict(n=n, row_ptr=[], col=[], rand_ws=1, rand_ws_k=k, rand_ws_beta=0.0)
    p = W.params_with(R=2.5, B_rand=1.5, net_seed=3)
    age = np.zeros(n, np.uint8)
    sim = oracle.Sim(g, p, age, np.array([c], np.uint32))
    d = sim.step(diag=True)
    inf_c = d["inf32"][c]
    assert inf_c > 0
    cR = np.float32(np.float32(p["R"]) * np.float32(p["inv_Ibar"]))
    want = np.float32(cR * np.float32(p["S_age"][0])) * np.float32(np.float32(p["B_rand"]) * inf_c)
    for j in range(n):
        exp = want if (j - c) % n in (1, 2, n - 1, n - 2) else np.float32(0.0)
        assert d["lambda32"][j] == exp, j
    assert d["messages"] == n * k
