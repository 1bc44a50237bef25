"""Pins for the age-stratified random network (Sec. 3, Interaction Networks: each
agent's age-stratified number of random interactions parameterises the random
network): with per-age means, agent j's daily in-contact count follows
Poisson(mean of j's age bin), its contacts are the uniform contacts of the
single-mean network of that mean, and equal means reduce to the single-mean run."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W

scipy_stats = pytest.importorskip("scipy.stats")

MEANS = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 5.0]


def test_counts_follow_each_age_bins_poisson_law():
    """One day's counts, pooled per age bin over 60,000 agents: each bin's
    histogram against its own Poisson pmf (chi-square), and its mean within a
    5-sigma band of the bin's mean."""
    n = 60_000
    pop = W.population(n, 11, 0)
    p = W.params_with(rand_mean_age=MEANS, net_seed=31)
    d = oracle.Sim(pop, p, pop["age"], None).step()
    k = d["rand_k"].astype(np.int64)
    for a, mu in enumerate(MEANS):
        ka = k[pop["age"] == a]
        assert abs(ka.mean() - mu) < 5 * np.sqrt(mu / ka.size), (a, ka.mean(), mu)
        top = 12
        obs = np.bincount(np.minimum(ka, top), minlength=top + 1)[: top + 1].astype(np.float64)
        pmf = scipy_stats.poisson.pmf(np.arange(top + 1), mu)
        pmf[top] = scipy_stats.poisson.sf(top - 1, mu)
        exp = pmf * ka.size
        keep = exp > 5
        chi2 = float(((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum())
        assert chi2 < 3 * keep.sum() + 20, (a, chi2)


def test_contacts_are_the_single_mean_networks_of_each_bin():
    """Agent j's contacts (its count, then the uniform sources in draw order) are
    those of the single-mean network whose mean is the mean of j's age bin: the
    day's lambda rebuilt from them equals the oracle's."""
    pop = W.population(400, 12, 40)
    p = W.params_with(rand_mean_age=MEANS, B_rand=1.3, net_seed=41)
    sim = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
    for _ in range(4):
        sim.step(diag=False)
    t = sim.t
    d = sim.step()
    inf = d["inf32"].astype(np.float64)
    f32 = lambda x: float(np.float32(x))
    for j in range(0, 400, 3):
        cts = oracle.random_contacts(41, 400, j, t, MEANS[pop["age"][j]])
        assert d["rand_k"][j] == cts.size
        hh = sum(inf[pop["col"][0][pop["row_ptr"][0][j]:pop["row_ptr"][0][j + 1]]])
        oc = sum(inf[pop["col"][1][pop["row_ptr"][1][j]:pop["row_ptr"][1][j + 1]]])
        want = f32(p["R"]) * f32(p["inv_Ibar"]) * p["S_age"][pop["age"][j]] * (
            2.0 * hh + 1.0 * oc + f32(1.3) * sum(inf[cts]))
        assert abs(d["lambda64"][j] - want) <= 1e-6 * max(want, 1e-12)


def test_equal_means_reduce_to_the_single_mean_run():
    """Per-age means all equal to rand_mean give the single-mean run exactly (whole
    runs with interventions: every array, counter and lambda identical)."""
    pop = W.population(3000, 13, 20)
    base = W.params_with(R=4.0, test_on=1, quar_on=1, vax_on=1, vax_start=5, vax_rate=0.02, seed=5, net_seed=6)
    a = oracle.Sim(pop, base, pop["age"], pop["seed_ids"])
    b = oracle.Sim(pop, dict(base, rand_mean_age=[base["rand_mean"]] * 9), pop["age"], pop["seed_ids"])
    for _ in range(30):
        da, db = a.step(), b.step()
        assert np.array_equal(da["lambda32"], db["lambda32"]) and da["messages"] == db["messages"]
    for k in ("stage", "timer", "tinf", "flags", "qt"):
        assert np.array_equal(getattr(a.state, k), getattr(b.state, k)), k


def test_relaxed_model_with_age_stratified_means():
    """The relaxed oracle with per-age means: equal means reduce to the single-mean
    model exactly, and its reverse sweep equals central differences."""
    pop = W.population(1200, 14, 8)
    p = W.params_with(R=3.0, seed=15, net_seed=16, S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    th = oracle.theta_of(p)
    a = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    b = oracle.Relaxed(pop, dict(p, rand_mean_age=[p["rand_mean"]] * 9), pop["age"], pop["seed_ids"], tau=0.5)
    y = np.log(a.run(th, 25)["incidence"] + 1.0) * 1.1
    oa, ob = a.run(th, 25, target=y, grad=True), b.run(th, 25, target=y, grad=True)
    assert np.array_equal(oa["incidence"], ob["incidence"]) and np.array_equal(oa["grad"], ob["grad"])
    rx = oracle.Relaxed(pop, dict(p, rand_mean_age=MEANS), pop["age"], pop["seed_ids"], tau=0.5)
    g = rx.run(th, 25, target=y, grad=True, fp32_theta=False)["grad"]
    assert not np.array_equal(g, oa["grad"])
    for i in (0, 3, 5):
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (rx.run(tp, 25, target=y, fp32_theta=False)["loss"] - rx.run(tm, 25, target=y, fp32_theta=False)["loss"]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, g[i])
