"""Pins for the oracle's Adam (oracle/adam.py), from what Kingma and Ba's
Algorithm 1 fixes: a two-step update worked by hand, the closed form of a
constant gradient (the bias-corrected moments equal the gradient exactly, so
every step moves by alpha g / (|g| + eps)), the projection onto theta >= 0,
and torch.optim.Adam run as a library routine."""
import numpy as np
import pytest

from oracle.adam import Adam


def test_two_steps_worked_by_hand():
    # theta_0 = 1, alpha = 0.1, g_1 = 2, g_2 = -1
    # step 1: m = 0.2, v = 0.004, mhat = 0.2 / 0.1 = 2, vhat = 0.004 / 0.001 = 4
    #         theta_1 = 1 - 0.1 * 2 / (2 + 1e-8)
    # step 2: m = 0.9 * 0.2 - 0.1 = 0.08, v = 0.999 * 0.004 + 0.001 = 0.004996
    #         mhat = 0.08 / 0.19, vhat = 0.004996 / 0.001999
    a = Adam(1, lr=0.1)
    th1 = a.step(np.array([1.0]), np.array([2.0]))
    assert th1[0] == pytest.approx(1.0 - 0.1 * 2.0 / (2.0 + 1e-8), abs=1e-15)
    th2 = a.step(th1, np.array([-1.0]))
    mhat, vhat = 0.08 / 0.19, 0.004996 / 0.001999
    assert th2[0] == pytest.approx(th1[0] - 0.1 * mhat / (np.sqrt(vhat) + 1e-8), abs=1e-14)
    assert a.t == 2


def test_constant_gradient_closed_form():
    g = np.array([3.0, -0.5, 1e-3, 0.0, -7.0])
    a = Adam(g.size, lr=0.01)
    th = np.zeros(g.size)
    for t in range(1, 60):
        th = a.step(th, g)
        want = -0.01 * t * g / (np.abs(g) + 1e-8)
        assert np.allclose(th, want, rtol=1e-12, atol=1e-15), t


def test_projection_keeps_theta_non_negative():
    a = Adam(3, lr=0.5, nonneg=True)
    th = a.step(np.array([0.2, 0.2, 3.0]), np.array([1.0, -1.0, 1.0]))
    assert th[0] == 0.0  # 0.2 - 0.5 clipped
    assert th[1] == pytest.approx(0.7)
    assert th[2] == pytest.approx(2.5)


def test_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    th0 = rng.normal(size=200)
    grads = rng.normal(size=(25, 200)) * np.exp(rng.uniform(-6, 2, (25, 200)))
    p = torch.tensor(th0, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    a = Adam(200, lr=3e-3)
    th = th0.copy()
    for g in grads:
        p.grad = torch.tensor(g)
        opt.step()
        th = a.step(th, g)
    assert np.allclose(p.detach().numpy(), th, rtol=0, atol=1e-12)
