"""Surrogate MLP on the GPU (BF16 tensor cores, FP32 accumulation) against the
CPU oracle that rounds the same values to BF16 (oracle/mlp.py).

Bars: outputs within 1e-2 of the largest output (a hidden activation that lands
next to a BF16 rounding boundary may round the other way); loss within 1e-3
relative; every gradient tensor within 1e-2 of its norm."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2110_04421_gb300 import workloads as W
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SIZES = [14, 256, 256, 256, 180]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make(batch, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (batch, 14)).astype(np.float32)
    y = rng.normal(2.0, 1.0, (batch, 180)).astype(np.float32)
    return x, y


def layer_slices(sizes):
    out, off = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        out.append((off, off + fi * fo))
        off += fi * fo
        out.append((off, off + fo))
        off += fo
    return out


@pytest.mark.parametrize("tcgen05", [True, False])
@pytest.mark.parametrize("batch", [1, 131, 300])
def test_forward_matches_bf16_oracle(batch, tcgen05):
    """Both forward paths: the fused tcgen05 kernel (TMEM accumulator) and the
    per-layer mma.sync GEMMs."""
    import torch
    from paper_2110_04421_gb300.deabm import MLP
    p = M.init_params(SIZES, 7)
    x, _ = make(batch, 1)
    m = MLP(max_batch=512)
    assert m.use_tcgen05(tcgen05)
    m.set_params(p)
    y = m.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    m.sync()
    m.close()
    ref, _, _ = M.forward(p, SIZES, x)
    assert np.max(np.abs(y - ref)) <= 1e-2 * np.max(np.abs(ref)), np.max(np.abs(y - ref))


def test_gradients_match_bf16_oracle():
    import torch
    from paper_2110_04421_gb300.deabm import MLP
    p = M.init_params(SIZES, 8)
    x, y = make(257, 2)
    m = MLP(max_batch=512)
    m.set_params(p)
    loss = m.grad(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    g = m.get_grads()
    m.close()
    lref, gref, _ = M.loss_and_grad(p, SIZES, x, y)
    assert abs(loss - lref) <= 1e-3 * lref
    for a, b in layer_slices(SIZES):
        err = np.max(np.abs(g[a:b] - gref[a:b]))
        assert err <= 1e-2 * np.max(np.abs(gref[a:b])) + 1e-8, (a, b, err)


def test_training_fits_a_smooth_map():
    import torch
    from paper_2110_04421_gb300.deabm import MLP
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (4096, 14)).astype(np.float32)
    t = np.linspace(0, 1, 180)[None, :]
    y = (3 * np.exp(-((t - 0.3 - 0.4 * x[:, :1]) ** 2) / 0.01) * x[:, 1:2]).astype(np.float32)
    m = MLP(max_batch=4096)
    m.set_params(M.init_params(SIZES, 4))
    X, Y = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    l0 = m.grad(X, Y)
    for it in range(600):
        idx = torch.randint(0, 4096, (512,), device="cuda")
        m.train_step(X[idx].contiguous(), Y[idx].contiguous(), 2e-3)
    l1 = m.grad(X, Y)
    m.close()
    assert l1 < 0.1 * l0, (l0, l1)


def test_reset_reproduces_a_fresh_context():
    from paper_2110_04421_gb300.deabm import Simulation
    pop = W.population(3000, 5, 15)
    base = W.params_with(vax_on=1, vax_start=5, vax_rate=0.01)
    rp1, s1 = W.batch_params(40, 1)
    rp2, s2 = W.batch_params(40, 2)
    a = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=40, rep_params=rp1, rep_seeds=s1, max_steps=30)
    a.run(30)
    a.reset(rp2, s2)
    ni_a, h_a = a.run(30)
    st_a = a.state()
    a.close()
    b = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=40, rep_params=rp2, rep_seeds=s2, max_steps=30)
    ni_b, h_b = b.run(30)
    st_b = b.state()
    b.close()
    assert np.array_equal(ni_a, ni_b) and np.array_equal(h_a, h_b)
    for k in st_a:
        assert np.array_equal(st_a[k], st_b[k])


def test_surrogate_beats_the_mean_curve_and_falls_back_outside_its_box():
    """Trained on 2,048 runs of the N = 100,000 ensemble workload; checked on 256
    unseen runs against re-simulation."""
    import torch
    from paper_2110_04421_gb300 import surrogate as S
    from paper_2110_04421_gb300.deabm import MLP
    w = W.surrogate_workload()
    pop = W.population(w["n"], 0, 10)
    rp, seeds = W.surrogate_params(2048 + 256, 5)
    Y = S.simulate(pop, w["params"], rp, seeds, w["T"])
    X = torch.tensor(S.normalize(rp), device="cuda")
    Yt = torch.tensor(Y, device="cuda")
    m = MLP(max_batch=4096)
    m.set_params(M.init_params(SIZES, 9))
    S.train(m, X[:2048], Yt[:2048], steps=1500, batch=512, lr=2e-3)
    pred = m.forward(X[2048:]).cpu().numpy()
    err = S.curve_errors(pred, Y[2048:])
    base = float(np.mean((Y[2048:] - Y[:2048].mean(0)) ** 2))
    assert err["mse_log"] < 0.25 * base, (err, base)
    sur = S.Surrogate(m, pop, w["params"], w["T"])
    outside = rp[2048:2050].copy()
    outside[:, 0] = 7.5  # R beyond the training box -> simulated
    out, inside = sur.predict(outside, seeds[2048:2050])
    m.close()
    assert not inside.any()
    assert np.array_equal(out, S.simulate(pop, w["params"], outside, seeds[2048:2050], w["T"]))
