"""Relaxed (Gumbel-softmax) path on the GPU against the FP64 oracle.

Bars: incidence within 1e-4 relative of the FP64 forward (FP32 sums over 90
days); gradient within 1e-3 relative of central finite differences (h = 1e-3)
of the FP64 oracle and within 1e-4 (relative to the gradient's norm) of the
oracle's own reverse sweep; the checkpoint interval changes nothing but
rounding."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def case():
    pop = W.population(4000, 7, 12)
    p = W.params_with(R=3.3, seed=31, net_seed=32, S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    T = 60
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    th = oracle.theta_of(p)
    hidden = th.copy()
    hidden[0], hidden[1], hidden[2], hidden[3] = 3.8, 2.2, 0.9, 0.8
    y = np.log(rx.run(hidden, T)["incidence"] + 1.0).astype(np.float32)
    return pop, p, T, rx, th, y


def gpu(pop, p, **kw):
    from paper_2110_04421_gb300.deabm import Relaxed
    return Relaxed(pop, p, pop["age"], pop["seed_ids"], **kw)


def test_forward_matches_oracle(case):
    pop, p, T, rx, th, y = case
    g = gpu(pop, p, max_days=T)
    inc = g.forward(th, T)
    g.close()
    ref = rx.run(th, T)["incidence"]
    assert np.all(np.abs(inc - ref) <= 1e-4 * np.maximum(ref, 1.0)), np.max(np.abs(inc - ref) / np.maximum(ref, 1))


def test_gradient_matches_oracle_adjoint_and_fd(case):
    pop, p, T, rx, th, y = case
    g = gpu(pop, p, max_days=T, ckpt_every=10)
    loss, grad, inc = g.grad(th, y)
    g.close()
    o = rx.run(th, T, target=y.astype(np.float64), grad=True)
    assert abs(loss - o["loss"]) <= 1e-4 * o["loss"]
    scale = np.linalg.norm(o["grad"])
    assert np.max(np.abs(grad - o["grad"])) <= 1e-4 * scale, (grad, o["grad"])
    th64 = np.float32(th).astype(np.float64)
    for i in range(13):
        h = 1e-3
        tp, tm = th64.copy(), th64.copy()
        tp[i] += h
        tm[i] -= h
        fd = (rx.run(tp, T, target=y, fp32_theta=False)["loss"] - rx.run(tm, T, target=y, fp32_theta=False)["loss"]) / (2 * h)
        assert abs(grad[i] - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale), (i, grad[i], fd)


def test_checkpoint_interval_changes_only_rounding(case):
    pop, p, T, rx, th, y = case
    grads = []
    for k in (1, 7, 10, T):
        g = gpu(pop, p, max_days=T, ckpt_every=k)
        grads.append(g.grad(th, y)[1])
        g.close()
    for gr in grads[1:]:
        assert np.max(np.abs(gr - grads[0])) <= 1e-5 * np.linalg.norm(grads[0])


def test_autograd_function(case):
    import torch
    from paper_2110_04421_gb300.deabm import relaxed_loss
    pop, p, T, rx, th, y = case
    g = gpu(pop, p, max_days=T)
    theta = torch.tensor(np.float32(th), requires_grad=True)
    loss = relaxed_loss(g, theta, torch.tensor(y))
    (3.0 * loss).backward()
    _, grad, _ = g.grad(th, y)
    g.close()
    assert torch.allclose(theta.grad, torch.tensor(3.0 * grad), rtol=1e-5, atol=1e-7)


def test_calibration_reduces_loss(case):
    pop, p, T, rx, th, y = case
    g = gpu(pop, p, max_days=T)
    out, trace = g.calibrate(th, y, steps=40, lr=0.02)
    loss_after, _, _ = g.grad(out, y)
    g.close()
    assert trace[0] > 0 and loss_after < 0.5 * trace[0], (trace[0], loss_after)
    assert np.all(out >= 0)


def test_calibration_steps_match_oracle_adam_on_oracle_gradients(case):
    """deabm_calibrate for 6 steps against the oracle's projected Adam driven by
    the oracle's FP64 reverse sweep from the same start.  The GPU gradient is
    within 1e-4 of the gradient's norm, and Adam normalises each coordinate, so
    where the oracle's gradient coordinates stay well clear of 0 every step the
    parameters agree within 2e-3 of the total step (lr per step).  The loss trace
    agrees within 1e-4 of the starting loss: as the fit improves the loss shrinks
    towards the FP32 rounding of the incidence it is made of, so its error is
    bounded in absolute terms, not relative to itself."""
    from oracle.adam import Adam
    pop, p, T, rx, th, y = case
    steps, lr = 6, 0.02
    g = gpu(pop, p, max_days=T, ckpt_every=10)
    out, trace = g.calibrate(th, y, steps=steps, lr=lr)
    g.close()
    opt = Adam(13, lr, nonneg=True)
    ref = np.float32(th).astype(np.float64)
    loss0 = None
    for it in range(steps):
        o = rx.run(ref, T, target=y.astype(np.float64), grad=True)
        loss0 = o["loss"] if loss0 is None else loss0
        assert abs(trace[it] - o["loss"]) <= 1e-4 * loss0, (it, trace[it], o["loss"])
        gr = o["grad"]
        assert np.min(np.abs(gr)) > 1e-2 * np.linalg.norm(gr), (it, gr)
        ref = opt.step(ref, gr)
        # the GPU keeps theta in FP32
        ref = np.float32(ref).astype(np.float64)
    assert np.max(np.abs(out - ref)) <= 2e-3 * lr * steps, (out, ref)


def test_full_size_gradient():
    """N = 100,000, 90 days, tau = 0.5, checkpoint every 10 days; target simulated
    at hidden parameters R = 3.5, weights 2.0 / 1.0 / 0.7."""
    w = W.relaxed_workload()
    pop = W.population(w["n"], 0, w["n_seed"])
    p, T = w["params"], w["T"]
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=w["tau"])
    y = np.log(rx.run(w["hidden"], T)["incidence"] + 1.0).astype(np.float32)
    th = w["start"]
    g = gpu(pop, p, max_days=T, ckpt_every=10, tau=w["tau"])
    loss, grad, _ = g.grad(th, y)
    g.close()
    o = rx.run(th, T, target=y, grad=True)
    scale = np.linalg.norm(o["grad"])
    assert abs(loss - o["loss"]) <= 1e-4 * o["loss"]
    assert np.max(np.abs(grad - o["grad"])) <= 1e-4 * scale
    th64 = np.float32(th).astype(np.float64)
    for i in (0, 1, 3, 4):
        tp, tm = th64.copy(), th64.copy()
        tp[i] += 1e-3
        tm[i] -= 1e-3
        fd = (rx.run(tp, T, target=y, fp32_theta=False)["loss"] - rx.run(tm, T, target=y, fp32_theta=False)["loss"]) / 2e-3
        assert abs(grad[i] - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale), (i, grad[i], fd)


def test_batched_gradient_columns_match_oracle_and_single_runs(case):
    """deabm_grad_batch over 5 parameter columns (R, the network weights and the
    age susceptibilities varied per column; B = 5 leaves a partial 32-column warp):
    each column's loss, gradient and incidence equal a single deabm_grad at that
    theta (within FP32 rounding: the reverse sweep's random-network atomics add in
    a different order) and the oracle's reverse sweep within the single path's bar."""
    pop, p, T, rx, th, y = case
    rng = np.random.default_rng(3)
    B = 5
    thetas = np.repeat(np.float32(th)[None, :], B, axis=0)
    thetas[:, 0] *= rng.uniform(0.8, 1.25, B).astype(np.float32)
    thetas[:, 1:4] *= rng.uniform(0.7, 1.3, (B, 3)).astype(np.float32)
    thetas[:, 4:] *= rng.uniform(0.9, 1.1, (B, 9)).astype(np.float32)
    targets = np.stack([y + np.float32(0.05 * b) for b in range(B)], axis=1)
    g = gpu(pop, p, max_days=T, ckpt_every=10)
    loss_b, grad_b, inc_b = g.grad_batch(thetas, targets)
    singles = [g.grad(thetas[b], targets[:, b]) for b in range(B)]
    g.close()
    for b in range(B):
        ls, gs, inc = singles[b]
        scale = np.linalg.norm(gs)
        assert abs(loss_b[b] - ls) <= 1e-5 * ls, (b, loss_b[b], ls)
        assert np.max(np.abs(grad_b[b] - gs)) <= 1e-5 * scale, (b, grad_b[b], gs)
        assert np.allclose(inc_b[:, b], inc, rtol=1e-5, atol=1e-3)
    for b in (0, B - 1):
        o = rx.run(thetas[b], T, target=targets[:, b].astype(np.float64), grad=True)
        scale = np.linalg.norm(o["grad"])
        assert abs(loss_b[b] - o["loss"]) <= 1e-4 * o["loss"]
        assert np.max(np.abs(grad_b[b] - o["grad"])) <= 1e-4 * scale, (b, grad_b[b], o["grad"])
    assert len({round(float(v), 6) for v in loss_b}) == B  # the columns ran different problems
    from paper_2110_04421_gb300.deabm import DeabmError
    g = gpu(pop, p, max_days=T)
    bad = thetas.copy()
    bad[2, 5] = -1.0
    with pytest.raises(DeabmError, match="must be finite and >= 0"):
        g.grad_batch(bad, targets)
    g.close()


def test_batched_gradient_full_workload_sample_columns():
    """N = 100,000, 90 days, checkpoint every 10, B = 64 columns of the calibration
    box (R in [2, 6], weights in [0.5, 2]); columns 0, 31, 63 against the oracle's
    reverse sweep at the single path's bar."""
    w = W.relaxed_workload()
    pop = W.population(w["n"], 0, w["n_seed"])
    p, T = w["params"], w["T"]
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=w["tau"])
    y = np.log(rx.run(w["hidden"], T)["incidence"] + 1.0).astype(np.float32)
    B = 64
    rng = np.random.default_rng(9)
    thetas = np.repeat(w["start"][None, :], B, axis=0).astype(np.float32)
    thetas[:, 0] = rng.uniform(2.0, 6.0, B)
    thetas[:, 1:4] = rng.uniform(0.5, 2.0, (B, 3))
    g = gpu(pop, p, max_days=T, ckpt_every=10, tau=w["tau"])
    loss_b, grad_b, _ = g.grad_batch(thetas, np.repeat(y[:, None], B, axis=1))
    g.close()
    for b in (0, 31, 63):
        o = rx.run(thetas[b], T, target=y, grad=True)
        scale = np.linalg.norm(o["grad"])
        assert abs(loss_b[b] - o["loss"]) <= 1e-4 * o["loss"], b
        assert np.max(np.abs(grad_b[b] - o["grad"])) <= 1e-4 * scale, (b, grad_b[b], o["grad"])


@pytest.mark.parametrize("lattice", [0, 1])
def test_daily_occupations_gradient_matches_oracle(lattice):
    """The relaxed model with daily occupation networks (households stored, 23
    occupations drawn every day; uniform or Watts-Strogatz lattice contacts): the
    forward incidence, the loss and the gradient (its occupation weight theta[2]
    included) against the oracle's FP64 run and reverse sweep at the bars above,
    and the batched gradient's columns against single runs."""
    pop = W.population_daily_occupation(6000, 17, 15)
    if lattice:
        pop = dict(pop, occ_lattice=1, occ_rewire=0.2)
    p = W.params_with(R=3.1, seed=41, net_seed=42, S_age=[0.6, 0.8, 1.0, 1.1, 1.2, 0.9, 1.3, 1.0, 0.7])
    T = 50
    rx = oracle.Relaxed(pop, p, pop["age"], pop["seed_ids"], tau=0.5)
    th = oracle.theta_of(p)
    hidden = th.copy()
    hidden[0], hidden[2] = 3.6, 1.4
    y = np.log(rx.run(hidden, T)["incidence"] + 1.0).astype(np.float32)
    g = gpu(pop, p, max_days=T, ckpt_every=10)
    inc = g.forward(th, T)
    loss, grad, _ = g.grad(th, y)
    B = 3
    thetas = np.repeat(np.float32(th)[None, :], B, axis=0)
    thetas[:, 2] *= np.array([0.8, 1.0, 1.3], np.float32)
    loss_b, grad_b, _ = g.grad_batch(thetas, np.repeat(y[:, None], B, axis=1))
    singles = [g.grad(thetas[b], y) for b in range(B)]
    g.close()
    o = rx.run(th, T, target=y.astype(np.float64), grad=True)
    assert np.all(np.abs(inc - o["incidence"]) <= 1e-4 * np.maximum(o["incidence"], 1.0))
    assert abs(loss - o["loss"]) <= 1e-4 * o["loss"]
    scale = np.linalg.norm(o["grad"])
    assert abs(o["grad"][2]) > 1e-3 * scale  # the occupation weight matters
    assert np.max(np.abs(grad - o["grad"])) <= 1e-4 * scale, (grad, o["grad"])
    for b in range(B):
        ls, gs, _ = singles[b]
        assert abs(loss_b[b] - ls) <= 1e-5 * ls, (b, loss_b[b], ls)
        assert np.max(np.abs(grad_b[b] - gs)) <= 1e-5 * np.linalg.norm(gs), (b, grad_b[b], gs)
