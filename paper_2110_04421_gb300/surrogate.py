"""Learned surrogate of the simulator: parameters -> daily log incidence.

Runs of the batched simulator (libdeabm, N agents, B replicates per launch)
give pairs (14 parameters, log(1 + new infections per day)); the MLP of
libdeabm is trained on them on the GPU; the simulator stays the fallback for
parameters outside the training box and the reference against which the
surrogate's error in peak day and cumulative infections is measured.

    python -m paper_2110_04421_gb300.surrogate [--runs 50000] [--steps 4000]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W
from .deabm import MLP, Simulation


def normalize(rp: np.ndarray) -> np.ndarray:
    """Min-max scaling of the 14 inputs to [0, 1] over the training box."""
    return ((rp - W.SURROGATE_LO) / (W.SURROGATE_HI - W.SURROGATE_LO)).astype(np.float32)


def simulate(pop, base, rp, seeds, T, B=256, sim=None):
    """log(1 + daily new infections) [n, T] of the runs rp (rows of 14) with the batched simulator."""
    n = rp.shape[0]
    out = np.zeros((n, T), np.float32)
    own = sim is None
    for s0 in range(0, n, B):
        rows = rp[s0:s0 + B]
        sd = seeds[s0:s0 + B]
        k = rows.shape[0]
        if k < B:  # pad the last launch with copies of its first row
            rows = np.concatenate([rows, np.repeat(rows[:1], B - k, 0)])
            sd = np.concatenate([sd, np.repeat(sd[:1], B - k)])
        if sim is None:
            sim = Simulation(pop, base, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rows, rep_seeds=sd,
                             max_steps=T)
        else:
            sim.reset(rows, sd)
        ni, _ = sim.run(T, hist=False)
        out[s0:s0 + k] = np.log1p(ni[:, :k].T.astype(np.float32))
    if own and sim is not None:
        sim.close()
    return out


def curve_errors(y_pred: np.ndarray, y_true: np.ndarray) -> dict:
    """Peak-day difference (days) and relative error of cumulative infections."""
    inc_p, inc_t = np.expm1(np.maximum(y_pred, 0.0)), np.expm1(y_true)
    peak = np.abs(np.argmax(inc_p, 1) - np.argmax(inc_t, 1))
    cum_t = inc_t.sum(1)
    cum = np.abs(inc_p.sum(1) - cum_t) / np.maximum(cum_t, 1.0)
    return {"peak_day_abs_err_median": float(np.median(peak)), "peak_day_abs_err_p90": float(np.percentile(peak, 90)),
            "cum_rel_err_median": float(np.median(cum)), "cum_rel_err_p90": float(np.percentile(cum, 90)),
            "mse_log": float(np.mean((y_pred - y_true) ** 2))}


def train(mlp: MLP, X, Y, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 0):
    """Adam on minibatches drawn with replacement (torch CUDA tensors X, Y)."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (batch,), device=X.device, generator=g)
        cur_lr = lr * 0.5 * (1 + np.cos(np.pi * it / steps))  # cosine decay
        loss = mlp.train_step(X[idx].contiguous(), Y[idx].contiguous(), cur_lr,
                              sync=bool(log_every) and it % log_every == 0)
        if loss is not None:
            losses.append((it, loss))
    mlp.sync()
    return losses


class Surrogate:
    """Trained MLP with the simulator as fallback outside the training box."""

    def __init__(self, mlp: MLP, pop, base, T):
        self.mlp, self.pop, self.base, self.T = mlp, pop, base, T

    def predict(self, rp: np.ndarray, seeds: np.ndarray | None = None):
        import torch
        rp = np.asarray(rp, np.float32)
        inside = np.all((rp >= W.SURROGATE_LO) & (rp <= W.SURROGATE_HI), axis=1)
        out = np.zeros((rp.shape[0], self.T), np.float32)
        if inside.any():
            x = torch.tensor(normalize(rp[inside]), device="cuda")
            out[inside] = self.mlp.forward(x).cpu().numpy()
        if (~inside).any():
            sd = seeds[~inside] if seeds is not None else np.arange((~inside).sum(), dtype=np.uint64)
            out[~inside] = simulate(self.pop, self.base, rp[~inside], sd, self.T)
        return out, inside


def fit_and_score(runs: int = 50_000, steps: int = 4000, batch: int = 1024, lr: float = 2e-3) -> dict:
    """Simulate `runs` parameter sets (batched simulator), train the MLP on 79 %
    of them, and score it on the next 20 % (validation) and on the last 1 %
    (held out: used neither in training nor in validation), each against the
    simulator's curves; also the error of the mean training curve, the method
    without the surrogate's parameter dependence."""
    import torch
    w = W.surrogate_workload()
    pop = W.population(w["n"], 0, 10)
    rp, seeds = W.surrogate_params(runs, 0)
    t0 = time.time()
    Y = simulate(pop, w["params"], rp, seeds, w["T"], B=w["B"])
    t_sim = time.time() - t0
    n_test = max(1, runs // 100)
    n_tr = int(0.79 * runs)
    val, test = slice(n_tr, runs - n_test), slice(runs - n_test, runs)
    X = torch.tensor(normalize(rp), device="cuda")
    Yt = torch.tensor(Y, device="cuda")
    mlp = MLP(14, w["hidden"], w["depth"], w["T"], max_batch=w["batch"])
    rng = np.random.default_rng(1)
    sizes = mlp.sizes
    init = np.concatenate([np.concatenate([rng.uniform(-1 / np.sqrt(fi), 1 / np.sqrt(fi), fi * fo), np.zeros(fo)])
                           for fi, fo in zip(sizes[:-1], sizes[1:])]).astype(np.float32)
    mlp.set_params(init)
    t1 = time.time()
    train(mlp, X[:n_tr], Yt[:n_tr], steps, batch, lr)
    t_train = time.time() - t1
    sur = Surrogate(mlp, pop, w["params"], w["T"])
    pred_val, _ = sur.predict(rp[val])
    pred_test, inside = sur.predict(rp[test], seeds[test])
    mean_curve = Y[:n_tr].mean(0, keepdims=True)
    out = {"runs": runs, "train": n_tr, "validation": runs - n_test - n_tr, "held_out": n_test,
           "sim_seconds": t_sim, "train_seconds": t_train, "steps": steps, "batch": batch,
           "validation_errors": curve_errors(pred_val, Y[val]),
           "held_out_errors": curve_errors(pred_test, Y[test]),
           "held_out_inside_box": int(inside.sum()),
           "mean_curve_errors_held_out": curve_errors(np.repeat(mean_curve, n_test, 0), Y[test])}
    mlp.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=50_000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=2e-3)
    args = ap.parse_args()
    print(json.dumps(fit_and_score(args.runs, args.steps, args.batch, args.lr)))


if __name__ == "__main__":
    main()
