"""Pins for the relaxed (differentiable) model's oracle.

* its reverse sweep equals central finite differences of its FP64 forward;
* day 0 on a star graph equals the closed form sigmoid((log expm1(lambda) + l)/tau);
* the logistic noise makes the tau -> 0 limit a Bernoulli(p) draw:
  P(l > -logit p) = p (the relaxation is unbiased in that limit)."""
import math

import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W


def erlang_day(t, k, theta):
    def F(x):
        y = x / theta
        return 0.0 if x <= 0 else 1.0 - math.exp(-y) * sum(y**m / math.factorial(m) for m in range(k))
    return F(t) - F(t - 1)


@pytest.fixture(scope="module")
def small():
    pop = W.population(1500, 4, 8)
    p = W.params_with(R=3.2, seed=11, net_seed=12, S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    th = oracle.theta_of(p)
    y = np.log(rx.run(th, 40)["incidence"] + 1.0) * 1.15 + 0.05
    return rx, th, y


def test_adjoint_matches_central_differences(small):
    rx, th, y = small
    g = rx.run(th, 40, target=y, grad=True, fp32_theta=False)["grad"]
    for i in range(13):
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (rx.run(tp, 40, target=y, fp32_theta=False)["loss"] - rx.run(tm, 40, target=y, fp32_theta=False)["loss"]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_loss_definition(small):
    rx, th, y = small
    o = rx.run(th, 40, target=y)
    assert abs(o["loss"] - np.mean((np.log(o["incidence"] + 1.0) - y) ** 2)) < 1e-14


def test_star_day_zero_closed_form():
    n = 30
    rp = np.zeros(n + 1, np.uint32)
    rp[2:] = np.arange(1, n)          # rows 1..n-1 each have the single in-edge from agent 0
    col = np.zeros(n - 1, np.uint32)
    g = dict(n=n, row_ptr=[rp], col=[col])
    p = W.params_with(R=2.0, inv_Ibar=0.5, B_net=[1.5], rand_mean=0.0, seed=3, A_class=[0.5, 1.0, 1.0])
    age = np.zeros(n, np.uint8)
    rx = oracle.Relaxed(g, p, age, np.array([0], np.uint32), tau=0.5)
    cls = rx.classes()
    o = rx.run(oracle.theta_of(p), 1, want_x=True)
    A = [0.5, 1.0, 1.0][cls[0]]
    lam = 2.0 * 0.5 * 1.0 * 1.5 * A * erlang_day(1, 4, 1.25)
    for j in range(1, n):
        w = oracle.philox([j, 0, 8, 0], [3, 0])[0]
        u = ((int(w) >> 8) + 0.5) / 2**24
        ell = math.log(u) - math.log1p(-u)
        want = 1.0 / (1.0 + math.exp(-(math.log(math.expm1(lam)) + ell) / 0.5))
        assert abs(o["x"][0, j] - want) < 1e-12
    assert o["x"][0, 0] == 0.0


def test_symptom_classes_follow_thresholds():
    pop = W.population(4000, 2, 0)
    p = W.params_with(seed=21)
    cls = oracle.Relaxed(pop, p, pop["age"], None).classes()
    for i in range(0, 4000, 37):
        w = oracle.philox([i, 0xFFFFFFFE, 1, 0], [21, 0])
        a = pop["age"][i]
        want = 0 if w[0] < oracle.threshold(p["p_asym"][a]) else (2 if w[2] < oracle.threshold(p["p_sev"][a]) else 1)
        assert cls[i] == want


def test_noise_is_logistic_and_unbiased_in_the_hard_limit():
    ell = np.array([oracle.lib().rx_noise(5, j, t) for j in range(4000) for t in range(5)])
    for p in (0.05, 0.3, 0.7):
        frac = np.mean(ell > -math.log(p / (1 - p)))
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / ell.size)
    assert abs(np.mean(ell)) < 0.05 and abs(np.var(ell) - math.pi**2 / 3) < 0.15


@pytest.mark.parametrize("lattice", [0, 1])
def test_daily_occupations_adjoint_matches_central_differences(lattice):
    """Daily occupation networks (households stored, 23 occupations drawn every
    day; uniform or Watts-Strogatz lattice contacts): the reverse sweep, which
    scatters along each day's redrawn occupation contacts, equals central
    differences of the FP64 forward on all 13 parameters (theta[2] is the
    occupation weight)."""
    pop = W.population_daily_occupation(1500, 5, 8)
    if lattice:
        pop = dict(pop, occ_lattice=1, occ_rewire=0.2)
    p = W.params_with(R=3.0, seed=13, net_seed=14, S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    th = oracle.theta_of(p)
    y = np.log(rx.run(th, 30)["incidence"] + 1.0) * 1.1 + 0.05
    g = rx.run(th, 30, target=y, grad=True, fp32_theta=False)["grad"]
    assert abs(g[2]) > 1e-4 * np.linalg.norm(g)  # the occupation weight matters
    for i in range(13):
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (rx.run(tp, 30, target=y, fp32_theta=False)["loss"] - rx.run(tm, 30, target=y, fp32_theta=False)["loss"]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])


@pytest.mark.parametrize("lattice", [0, 1])
def test_two_member_occupations_equal_a_stored_network(lattice):
    """In an occupation of two every daily contact is the partner (uniform or
    lattice), so the run equals, operation for operation, the same model with the
    occupation replaced by a stored network that lists the partner k times: the
    incidence, loss and gradient agree exactly."""
    n = 2000
    pop = W.population(n, 6, 12)
    rng = np.random.default_rng(7)
    perm = rng.permutation(n)
    group = np.empty(n, np.uint32)
    group[perm] = (np.arange(n) // 2).astype(np.uint32)
    k = rng.integers(1, 16, size=n // 2).astype(np.uint8)
    partner = np.empty(n, np.uint32)
    partner[perm[0::2]] = perm[1::2]
    partner[perm[1::2]] = perm[0::2]
    kk = k[group].astype(np.int64)
    rp = np.zeros(n + 1, np.uint32)
    rp[1:] = np.cumsum(kk)
    col = np.repeat(partner, kk).astype(np.uint32)
    daily = dict(n=n, row_ptr=pop["row_ptr"][:1], col=pop["col"][:1], occ_group=group, occ_k=k,
                 occ_lattice=lattice, occ_rewire=0.3)
    stored = dict(n=n, row_ptr=pop["row_ptr"][:1] + [rp], col=pop["col"][:1] + [col])
    p = W.params_with(R=4.0, B_net=[2.0, 0.7], seed=15, net_seed=16)
    th = oracle.theta_of(p)
    a = oracle.Relaxed(daily, p, pop["age"], pop["seed_ids"], tau=0.5)
    b = oracle.Relaxed(stored, p, pop["age"], pop["seed_ids"], tau=0.5)
    y = np.log(b.run(th, 25)["incidence"] + 1.0) * 0.9
    oa, ob = a.run(th, 25, target=y, grad=True), b.run(th, 25, target=y, grad=True)
    assert np.array_equal(oa["incidence"], ob["incidence"])
    assert oa["loss"] == ob["loss"]
    assert np.array_equal(oa["grad"], ob["grad"])
    assert oa["incidence"].sum() > 100
