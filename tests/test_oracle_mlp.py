"""Pins for the MLP oracle: its exact-arithmetic backward equals central finite
differences and torch's autograd (a library routine); the BF16 rounding helper
matches torch's bfloat16 conversion (round to nearest, ties to even)."""
import numpy as np
import pytest

from oracle import mlp

SIZES = [14, 24, 24, 10]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(size=5000) * np.exp(np.random.default_rng(1).uniform(-20, 20, 5000))
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1 + 2**-8, 1 + 3 * 2**-9, 1 + 2**-9, 3.0e38]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gelu_against_its_closed_forms():
    """The tanh form against values that fix it independently: gelu(0) = 0;
    gelu(z) - gelu(-z) = z (tanh is odd); as z -> +inf gelu(z) -> z and
    gelu(-z) -> 0; and gelu(1) = (1 + tanh(1.044715 sqrt(2/pi))) / 2 written
    out with the exponential form of tanh."""
    z = np.linspace(-6.0, 6.0, 241)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-13)
    assert abs(mlp.gelu(np.array([30.0]))[0] - 30.0) < 1e-12 and abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-12
    u = 1.044715 * np.sqrt(2.0 / np.pi)
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.5 * (1.0 + (np.exp(2 * u) - 1) / (np.exp(2 * u) + 1))) < 1e-15
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = mlp.init_params(SIZES, 3).astype(np.float64)
    x = rng.uniform(0, 1, (7, 14))
    y = rng.normal(size=(7, 10))
    loss, g, _ = mlp.loss_and_grad(p, SIZES, x, y, bf16_round=False)
    for q in rng.choice(p.size, 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (mlp.loss_and_grad(pp, SIZES, x, y, False)[0] - mlp.loss_and_grad(pm, SIZES, x, y, False)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1e-3, abs(fd)), (q, fd, g[q])


def test_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p = mlp.init_params(SIZES, 5).astype(np.float64)
    x = rng.uniform(0, 1, (9, 14))
    y = rng.normal(size=(9, 10))
    loss, g, yhat = mlp.loss_and_grad(p, SIZES, x, y, bf16_round=False)
    tp = torch.tensor(p, requires_grad=True)
    a = torch.tensor(x)
    off = 0
    for l, (fi, fo) in enumerate(zip(SIZES[:-1], SIZES[1:])):
        W = tp[off:off + fi * fo].view(fi, fo)
        off += fi * fo
        b = tp[off:off + fo]
        off += fo
        a = a @ W + b
        if l < len(SIZES) - 2:
            a = torch.nn.functional.gelu(a, approximate="tanh")
    tl = ((a - torch.tensor(y)) ** 2).mean()
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    assert np.allclose(tp.grad.numpy(), g, rtol=1e-10, atol=1e-14)
