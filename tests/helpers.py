"""Shared test helpers: running the oracle and the CUDA path side by side."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2110_04421_gb300 import workloads as W

STATE_KEYS = ("stage", "timer", "tinf", "flags", "qt")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def oracle_sim(pop, params, state=None, seed_ids="pop"):
    ids = pop["seed_ids"] if isinstance(seed_ids, str) else seed_ids
    st = None
    if state is not None:
        st = oracle.State(pop["n"])
        for k in STATE_KEYS:
            getattr(st, k)[:] = state[k]
    return oracle.Sim(pop, params, pop["age"], ids, state=st)


def gpu_sim(pop, params, keep_lambda=True, state=None, seed_ids="pop", **kw):
    from paper_2110_04421_gb300.deabm import Simulation
    ids = pop["seed_ids"] if isinstance(seed_ids, str) else seed_ids
    return Simulation(pop, params, pop["age"], ids, state=state, keep_lambda=keep_lambda, **kw)


def compare_days(pop, params, T, state=None, seed_ids="pop", check_lambda=True):
    """Run T days on both sides, comparing after every day.  Returns a report dict.
    A draw whose |u - p| < 1e-6 on the oracle side is a tolerated flip: it ends
    the comparison (the trajectories legitimately part there) and is counted.
    With check_lambda a second GPU context that does not keep lambda (the
    launch configuration of runs and of the benchmark) steps alongside and must
    equal the first bit for bit every day."""
    osim = oracle_sim(pop, params, state, seed_ids)
    g = gpu_sim(pop, params, keep_lambda=check_lambda, state=state, seed_ids=seed_ids, max_steps=max(T, 1))
    g2 = gpu_sim(pop, params, keep_lambda=False, state=state, seed_ids=seed_ids, max_steps=max(T, 1)) \
        if check_lambda else None
    report = dict(days=0, flips=0, max_rel_lambda64=0.0, new_inf=[], messages=[], messages_sus=[])
    try:
        s0 = g.state()
        for k in STATE_KEYS:
            assert np.array_equal(s0[k], getattr(osim.state, k)), f"initial {k} differs"
        for t in range(T):
            d = osim.step(diag=True)
            g.step(1)
            s = g.state(with_lambda=check_lambda)
            if g2 is not None:
                g2.step(1)
                s2 = g2.state()
                for k in STATE_KEYS:
                    assert np.array_equal(s2[k], s[k]), f"day {t}: {k} differs between the two launch configurations"
            if check_lambda:
                lam_o = d["lambda32"]
                bad = np.nonzero(s["lambda"].view(np.uint32) != lam_o.view(np.uint32))[0]
                assert bad.size == 0, f"day {t}: lambda differs at {bad[:10]} gpu={s['lambda'][bad[:5]]} oracle={lam_o[bad[:5]]}"
                rel = np.abs(s["lambda"].astype(np.float64) - d["lambda64"]) / np.maximum(d["lambda64"], 1e-30)
                rel[d["lambda64"] == 0] = np.abs(s["lambda"][d["lambda64"] == 0])
                report["max_rel_lambda64"] = max(report["max_rel_lambda64"], float(rel.max(initial=0.0)))
                # p: the library reports expm1f's value away from the decision boundary
                pd = np.abs(s["p"].view(np.int32).astype(np.int64) - d["p32"].view(np.int32).astype(np.int64))
                assert pd.max(initial=0) <= 2, f"day {t}: p differs by {pd.max()} ulp"
            diff = {k: np.nonzero(s[k] != getattr(osim.state, k))[0] for k in STATE_KEYS}
            if any(v.size for v in diff.values()):
                agents = np.unique(np.concatenate(list(diff.values())))
                near = d["near"][agents].astype(bool)
                if near.any():
                    report["flips"] += int(near.sum())
                    report["flip_day"] = t
                    return report
                k0 = next(k for k in STATE_KEYS if diff[k].size)
                j = diff[k0][0]
                raise AssertionError(f"day {t}: {k0} differs at {diff[k0][:10]} (agent {j}: gpu "
                                     f"{[int(s[k][j]) for k in STATE_KEYS]} oracle "
                                     f"{[int(getattr(osim.state, k)[j]) for k in STATE_KEYS]})")
            report["days"] = t + 1
            report["new_inf"].append(d["new_inf"])
            report["messages"].append(d["messages"])
            report["messages_sus"].append(d["messages_sus"])
        ni, h, m = g.counters(T)
        assert ni[:, 0].tolist() == report["new_inf"]
        assert m.astype(np.int64).tolist() == report["messages"]
        # messages gathered: every destination when lambda is kept (or with exposure
        # notification), else only the destinations susceptible at the start of the day
        gath = g.gathered(T).astype(np.int64).tolist()
        assert gath == report["messages"], "gathered messages with lambda kept"
        if g2 is not None:
            ni2, h2, m2 = g2.counters(T)
            assert np.array_equal(ni2, ni) and np.array_equal(h2, h) and np.array_equal(m2, m)
            want = report["messages"] if params.get("den_on") else report["messages_sus"]
            assert g2.gathered(T).astype(np.int64).tolist() == want, "gathered messages"
        if params.get("den_on"):
            assert g.notified(T).tolist() == osim.den_notified[:T]
            report["notified"] = osim.den_notified[:T]
        return report
    finally:
        g.close()
        if g2 is not None:
            g2.close()
