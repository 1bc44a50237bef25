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
