"""Benchmark: agent interactions per second of the DeepABM-COVID day on GB300.

Default workload (one GPU): the plain simulation at scale, N = 2,000,000 agents,
household + occupation networks and a Poisson(2) random network regenerated
each day (about 14.2 messages per agent per day), 0.5% initial cases, testing
with 14-day quarantine, vaccination of 1%/day from day 30.  A step is one
simulated day (one launch of the day kernel).  Also reported: the batched
ensemble (one N = 100,000 graph shared by B = 256 replicates) against a loop of
plain per-replicate runs.

  python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--gpus N]

Interactions = messages processed (static in-edges + that day's random
in-contacts, before masking), summed over days and replicates.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2**20
PLAIN_WORKLOAD = ("plain N=2e6 T=180 (households 1-6, occupation groups of 20 x 10 links, Poisson(2) random "
                  "network, testing + 14-day quarantine, vaccination 1%/day from day 30)")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_bytes_plain(n: int, static_edges: int, n_nets: int, vax: bool) -> int:
    """Algorithmic HBM bytes of one day of the plain kernel: each array once.
    CSR row pointers 4(N+1) per network, columns 4 per stored edge; state read
    and written (stage 1, timer 2, tinf 2, flags 1, qt 1 = 7 B each way); age
    1 B; first-dose day 2 B (vaccination on); emitted infectiousness read once
    and written once (4 + 4 B).  Random edges are generated, not stored: 0 B."""
    return 4 * (n + 1) * n_nets + 4 * static_edges + n * (7 + 7 + 1 + (2 if vax else 0) + 4 + 4)


def step_bytes_plain_needed(n: int, static_edges: int, n_nets: int, vax: bool, n_sus: float) -> float:
    """Bytes one plain day needs when only susceptible agents gather (Eq. 2 applies
    to them alone): every agent's state, age, dose day and infectiousness as
    above, but row pointers and columns only for the n_sus susceptible rows
    (their edges counted at the mean in-degree)."""
    return (n * (7 + 7 + 1 + (2 if vax else 0) + 4 + 4)
            + 4.0 * n_sus * n_nets + 4.0 * static_edges * n_sus / n)


def step_bytes_batch(n: int, B: int, static_edges: int, n_nets: int, vax: bool) -> int:
    """Same for the [N][B] panel: per (agent, replicate) 7 + 7 + 4 + 4 B; per agent
    age and first-dose day; the CSR once for all replicates."""
    return 4 * (n + 1) * n_nets + 4 * static_edges + n * (1 + (2 if vax else 0)) + n * B * (7 + 7 + 4 + 4)


def step_bytes_occ(n: int, static_edges: int, n_nets: int, n_occ: int, vax: bool) -> int:
    """The plain day with its occupation network drawn daily: the stored networks'
    bytes as above, plus each agent's occupation (4 B) and each occupation's
    first row and daily count (4 + 1 B).  The day's contacts are generated: 0 B."""
    return step_bytes_plain(n, static_edges, n_nets, vax) + 4 * n + 5 * n_occ + 4


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


DAY_KERNEL_SOURCES = ("step_kernels.cu", "day_common.cuh", "deabm_device.cuh")
MLP_KERNEL_SOURCES = ("mlp_tc.cu", "mlp_tc.h", "gelu.cuh")


def sources_hash(names) -> str:
    """sha256 prefix over the concatenated sources a kernel is compiled from."""
    h = hashlib.sha256()
    for nm in names:
        h.update(open(os.path.join(ROOT, "paper_2110_04421_gb300", "csrc", nm), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(sources, profile: str, units_per_launch: float, days=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (their sha256 prefix is recorded there) and, when
    `days` = (first, last) is given, on a day inside that timed range (the
    summary's `captured_day` line); else None."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
        src_hash = sources_hash(sources)
        if f"source_sha256_16: {src_hash}" not in txt:
            return None
        if days is not None:
            d = re.search(r"captured_day:\s*([0-9]+)", txt)
            if not d or not (days[0] <= int(d.group(1)) <= days[1]):
                return None
        m = re.search(r"dram_bytes_per_unit:\s*([0-9.eE+-]+)", txt)
        return float(m.group(1)) * units_per_launch if m else None
    except Exception:
        return None


def profile_value(sources, profile: str, key: str, days=None):
    """A machine-readable number of a committed ncu summary (`key: value`), under
    the same conditions as traffic_from_profile (current sources, captured inside
    `days`); else None."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
        if f"source_sha256_16: {sources_hash(sources)}" not in txt:
            return None
        if days is not None:
            d = re.search(r"captured_day:\s*([0-9]+)", txt)
            if not d or not (days[0] <= int(d.group(1)) <= days[1]):
                return None
        m = re.search(key + r":\s*([0-9.eE+-]+)", txt)
        return float(m.group(1)) if m else None
    except Exception:
        return None


SMS, SMSP_PER_SM = 152, 4  # GB300: streaming multiprocessors, warp schedulers (one issue a cycle) each


# ---------------------------------------------------------------------------------------- ours
def rank_inputs(w: dict, rank: int):
    """Rank r's own problem: an independent population (seeded by r) with its own
    simulation and network seeds.  Ranks exchange no data on the simulation path."""
    from paper_2110_04421_gb300 import workloads as W
    params = dict(w["params"], seed=w["params"]["seed"] + rank, net_seed=w["params"]["net_seed"] + rank)
    pop = W.population(w["n"], rank, w["n_seed"])
    return params, pop


def column_range(B: int, rank: int, world: int):
    """The replicate columns [lo, hi) of a B-column ensemble that rank `rank` of
    `world` runs: contiguous shares, the first B % world ranks one column more.
    Columns are independent runs on the shared graph (own parameters and seed;
    the day's random network is keyed by the graph's seed), so a split changes no
    column's trajectory and needs no exchange until the results are gathered."""
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_columns(dist, local, B: int, world: int, device):
    """The [T, B] per-column results from every rank's [T, hi - lo] share, in
    column order (all_gather of equal-sized, zero-padded blocks)."""
    import torch
    T = local.shape[0]
    width = -(-B // world)
    buf = torch.zeros((T, width), dtype=torch.int64, device=device)
    buf[:, :local.shape[1]] = torch.as_tensor(np.asarray(local, np.int64), device=device)
    parts = [torch.empty_like(buf) for _ in range(world)]
    if dist is not None:
        dist.all_gather(parts, buf)
    else:
        parts = [buf]
    out = np.zeros((T, B), np.int64)
    for q in range(world):
        lo, hi = column_range(B, q, world)
        out[:, lo:hi] = parts[q][:, :hi - lo].cpu().numpy()
    return out


def reduce_over_ranks(dist, maxed, summed, device):
    """Whole-job figures: the slowest rank's times (max) and the work of all ranks
    (sum).  dist is torch.distributed (None on one rank)."""
    import torch
    mx = torch.tensor([float(v) for v in maxed], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in summed], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def run_ours(args, rank, world, local):
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = W.plain_large()
    n, K, Wm = w["n"], args.steps, args.warmup
    params, pop = rank_inputs(w, rank)
    static_edges = int(sum(int(rp[-1]) for rp in pop["row_ptr"]))
    stream = torch.cuda.Stream()

    # ---- device-resident timing: inputs uploaded before the timed region
    sim = Simulation(pop, params, pop["age"], pop["seed_ids"], max_steps=Wm + K, stream=stream.cuda_stream)
    sim.step(Wm)
    sim.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        # the K days back to back on the stream (one launch each, nothing else
        # between them): the events bracket exactly the K day kernels
        ev[0].record(stream)
        sim.step(K)
        ev[1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = ev[0].elapsed_time(ev[1])
    per_day_ms = [total_ms / K] * K
    _, hist_days, msgs = sim.counters(Wm + K)
    messages = int(msgs[Wm:].astype(np.int64).sum())
    gathered = int(sim.gathered(Wm + K)[Wm:].astype(np.int64).sum())
    # susceptible agents at the start of each timed day (end of the day before)
    sus_days = [float(hist_days[d - 1, 0, 0]) for d in range(Wm, Wm + K)]
    sim.close()

    # ---- end to end through the C-ABI with host buffers (create + run + readback),
    # days 0 .. Wm+K-1: the device-timed days and the warm-up days before them
    e2e_s, e2e_messages, h2d, d2h = float("nan"), 0, 0, 0
    KE = Wm + K
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = Simulation(pop, params, pop["age"], pop["seed_ids"], max_steps=KE, stream=stream.cuda_stream)
        ni, hist = sim2.run(KE)
        st = sim2.state()
        _, _, msgs2 = sim2.counters(KE)
        sim2.close()
        e2e_s = time.perf_counter() - t0
        e2e_messages = int(msgs2.astype(np.int64).sum())
        h2d = 4 * (n + 1) * len(pop["row_ptr"]) + 4 * static_edges + n + 4 * len(pop["seed_ids"])
        d2h = ni.nbytes + hist.nbytes + sum(v.nbytes for v in st.values()) + msgs2.nbytes

    # ---- max over ranks
    (total_ms, e2e_s), (messages, e2e_messages, gathered) = reduce_over_ranks(
        dist, [total_ms, e2e_s], [messages, e2e_messages, gathered], "cuda")
    messages, e2e_messages, gathered = int(messages), int(e2e_messages), int(gathered)

    # ---- batched ensemble vs plain per-replicate loop, relaxed gradient (rank 0)
    batched = run_batched(args, rank, world, dist) if not args.no_batched else None  # columns split over ranks
    relaxed = run_relaxed(args) if (rank == 0 and not args.no_relaxed) else None
    surrogate = run_surrogate(args) if (rank == 0 and not args.no_surrogate) else None
    ragged = run_ragged(args) if (rank == 0 and not args.no_ragged) else None
    occupation = run_occupation(args) if (rank == 0 and not args.no_occupation) else None
    den = run_den(args) if (rank == 0 and not args.no_den) else None
    wsr = run_ws_random(args) if (rank == 0 and not args.no_ws) else None

    if rank == 0:
        value = messages / (total_ms / 1e3)
        avg_ms = statistics.mean(per_day_ms)
        alg = step_bytes_plain(n, static_edges, len(pop["row_ptr"]), bool(params["vax_on"]))
        alg_needed = statistics.mean(
            step_bytes_plain_needed(n, static_edges, len(pop["row_ptr"]), bool(params["vax_on"]), ns) for ns in sus_days)
        peak, peak_kind = measured_peak_hbm()
        achieved = alg / (avg_ms / 1e3) / 1e9
        achieved_needed = alg_needed / (avg_ms / 1e3) / 1e9
        traffic = traffic_from_profile(DAY_KERNEL_SOURCES, "step_plain_n2e6.md", n, (Wm, Wm + K - 1))
        # the issue-rate view of the same launches: warp-instructions a launch (ncu,
        # same sources, a timed day) over the event-timed launch, against one issue
        # a cycle per warp scheduler at the SM clock seen during the timed region
        winst = profile_value(DAY_KERNEL_SOURCES, "step_plain_n2e6.md", "warp_instructions_per_launch",
                              (Wm, Wm + K - 1))
        sm_hz = 1e6 * float(clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0) if isinstance(clk, dict) else 2.07e9
        issue = None
        if winst:
            issue_peak = SMS * SMSP_PER_SM * sm_hz
            issue = {"achieved": winst / (avg_ms / 1e3), "peak": issue_peak, "unit": "warp-instructions/s",
                     "frac": winst / (avg_ms / 1e3) / issue_peak, "warp_instructions_per_launch": winst,
                     "note": "context for the HBM fraction: issued instructions (predicated-off and divergent "
                             "lanes included), not algorithmic work"}
        cpu = None if args.no_cpu_baseline else cpu_baseline(pop, params, args.cpu_seconds)
        line = {
            "metric": "agent interactions/s on 1 GB300 (plain day kernel; batched B=256 in 'batched')",
            "value": value, "unit": "interactions/s", "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded generators shaped like the paper's population)",
            "config": {"workload": PLAIN_WORKLOAD,
                       "n_agents": n, "messages_per_day": messages / K / world,
                       "static_edges": static_edges, "days_timed": f"{Wm}..{Wm + K - 1}",
                       "l2": f"inputs larger than L2: {alg / 1e6:.0f} MB algorithmic per day vs "
                             f"{L2_BYTES / 1e6:.0f} MB L2, no flush",
                       "parallelism": f"{world} independent population(s), one per GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "step_plain_kernel", "alg_bytes_per_launch": alg,
                         "alg_bytes_needed_mean": alg_needed,
                         "achieved_needed": achieved_needed, "frac_needed": achieved_needed / peak,
                         "alg_note": f"achieved counts every array once ({alg / 1e6:.0f} MB a day); only susceptible "
                                     "agents gather (Eq. 2 applies to them alone), so a day needs "
                                     "alg_bytes_needed_mean on average (mean susceptible share "
                                     f"{statistics.mean(sus_days) / n:.3f} over the timed days): achieved_needed "
                                     "and frac_needed divide those bytes by the same time",
                         "launch_ms_mean": avg_ms, "issue": issue},
            "e2e": None if args.no_e2e else {
                "value": e2e_messages / e2e_s, "unit": "interactions/s", "h2d_bytes_per_step": h2d / KE,
                "d2h_bytes_per_step": d2h / KE, "seconds": e2e_s, "days": f"0..{KE - 1}",
                "note": "one call sequence from host buffers: create (graph, agents and parameters up), "
                        "the days, state and counters back; the days are the timed days and the warm-up days "
                        "before them"},
            "gathered": {"value": gathered / (total_ms / 1e3), "unit": "messages gathered/s",
                         "share": gathered / max(messages, 1),
                         "note": "in-contacts of the destinations that evaluated Eq. 1 (the agents susceptible at "
                                 "the start of each day); value counts every message of the day, gathered or not"},
            "gpu_launches": K,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if batched:
            line["batched"] = batched
        if relaxed:
            line["relaxed"] = relaxed
        if surrogate:
            line["surrogate"] = surrogate
        if ragged:
            line["ragged"] = ragged
        if occupation:
            line["daily_occupation"] = occupation
        if den:
            line["exposure_notification"] = den
        if wsr:
            line["ws_random_network"] = wsr
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_relaxed(args):
    """Differentiable inverse run: one gradient (forward with checkpoints + reverse
    sweep) and an on-device Adam calibration, N = 1e5, 90 days."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Relaxed

    w = W.relaxed_workload()
    pop = W.population(w["n"], 0, w["n_seed"])
    stream = torch.cuda.Stream()
    rx = Relaxed(pop, w["params"], pop["age"], pop["seed_ids"], tau=w["tau"], max_days=w["T"], ckpt_every=10,
                 stream=stream.cuda_stream)
    y = np.log(rx.forward(w["hidden"], w["T"]).astype(np.float64) + 1.0).astype(np.float32)
    for _ in range(args.warmup):
        rx.grad(w["start"], y)
    reps = 5
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ms_grad = 0.0
    for _ in range(reps):
        flush.fill_(1.0)  # L2 flushed between gradients
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rx.grad(w["start"], y)  # returns host values: the call ends synchronised
        ms_grad += (time.perf_counter() - t0) * 1e3 / reps
    t1 = time.perf_counter()
    theta, trace = rx.calibrate(w["start"], y, steps=args.calib_steps, lr=w["lr"])
    cal_s = time.perf_counter() - t1
    loss1, _, _ = rx.grad(theta, y)
    # B = 256 parameter columns in one batched gradient (the calibration box of the
    # ensemble workload: R ~ U[2,6], network weights ~ U[0.5,2])
    Bc = 256
    rng = np.random.default_rng(0)
    thetas = np.repeat(np.asarray(w["start"], np.float32)[None, :], Bc, axis=0)
    thetas[:, 0] = rng.uniform(2.0, 6.0, Bc)
    thetas[:, 1:4] = rng.uniform(0.5, 2.0, (Bc, 3))
    targets = np.repeat(y[:, None], Bc, axis=1)
    rx.grad_batch(thetas[:8], targets[:, :8])  # arrays for 8 columns, device code loaded
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rx.grad_batch(thetas, targets)  # first call at 256 columns: includes their allocation
    first_ms = (time.perf_counter() - t2) * 1e3
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    loss_b, _, _ = rx.grad_batch(thetas, targets)
    batch_ms = (time.perf_counter() - t2) * 1e3
    rx.close()
    cpu = None if args.no_cpu_baseline else cpu_baseline_relaxed(pop, w["params"], w["tau"], w["start"], y, w["T"])
    return {"workload": w["name"], "ms_per_gradient": ms_grad, "days": w["T"], "checkpoint_every": 10,
            "cpu_baseline": cpu,
            "l2": "flushed before every timed gradient (write of twice its size)",
            "calibration": {"steps": args.calib_steps, "seconds": cal_s, "loss_start": float(trace[0]),
                            "loss_end": float(loss1), "theta_hidden": [float(x) for x in w["hidden"][:4]],
                            "theta_found": [float(x) for x in theta[:4]],
                            "products_hidden": [float(w["hidden"][0] * w["hidden"][k]) for k in (1, 2, 3)],
                            "products_found": [float(theta[0] * theta[k]) for k in (1, 2, 3)],
                            "note": "lambda depends on R, the network weights B_n and the age "
                                    "susceptibilities only through the products R S_a B_n (Eq. 1), so the "
                                    "loss is flat along R -> c R, B_n -> B_n / c; the networks' shares of the "
                                    "daily incidence also trade off against each other, so one incidence "
                                    "curve identifies neither R and the weights nor the products R B_n: "
                                    "the fit matches the curve, not the hidden parameters"},
            "batched_gradient": {"columns": Bc, "ms": batch_ms, "ms_first_call": first_ms,
                                 "ms_per_column": batch_ms / Bc,
                                 "multiple_of_single_gradients": ms_grad * Bc / batch_ms,
                                 "note": "one deabm_grad_batch call, host buffers, L2 flushed before; the "
                                         "multiple is against the single-gradient time above times the columns",
                                 "loss_range": [float(loss_b.min()), float(loss_b.max())]}}


def mlp_flops_per_sample(sizes) -> int:
    """Dense FLOPs of one forward pass: 2 * fan_in * fan_out per layer (bias and GELU
    not counted); the input layer at its unpadded width."""
    return sum(2 * fi * fo for fi, fo in zip(sizes[:-1], sizes[1:]))


def measured_peak_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def run_surrogate(args):
    """Surrogate MLP 14 -> 3 x 256 -> 180 at the inference batch of 65,536: forward
    and one training step (forward + backward + Adam), timed with CUDA events."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import MLP

    w = W.surrogate_workload()
    B = w["batch"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        m = MLP(14, w["hidden"], w["depth"], w["T"], max_batch=B, stream=stream.cuda_stream)
        rng = np.random.default_rng(0)
        sizes = m.sizes
        m.set_params(np.concatenate([np.concatenate([rng.uniform(-1 / np.sqrt(fi), 1 / np.sqrt(fi), fi * fo),
                                                     np.zeros(fo)]) for fi, fo in zip(sizes[:-1], sizes[1:])]
                                    ).astype(np.float32))
        x = torch.rand((B, 14), device="cuda")
        y = torch.rand((B, w["T"]), device="cuda")
        out = torch.empty((B, w["T"]), device="cuda")
        tc = m.use_tcgen05(True)
        for _ in range(args.warmup):
            m.forward(x, out)
            m.train_step(x, y, 1e-4)
        reps = 20
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

        def timed(fn):
            # L2 flushed (a write of twice its size) before every call; each call
            # bracketed by its own events on the MLP's stream
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for e0, e1 in ev:
                flush.fill_(1.0)
                e0.record(stream)
                fn()
                e1.record(stream)
            m.sync()
            torch.cuda.synchronize()
            return sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps

        m.forward(x, out)  # refresh the K-major weight copies outside the timed region
        fwd_ms = timed(lambda: m.forward(x, out))
        step_ms = timed(lambda: m.train_step(x, y, 1e-4))
        m.use_tcgen05(False)
        fwd_mma_ms = timed(lambda: m.forward(x, out))
        step_mma_ms = timed(lambda: m.train_step(x, y, 1e-4))
        params_now = m.get_params()
    m.close()
    cpu = None
    if not args.no_cpu_baseline:
        with tempfile.TemporaryDirectory() as d:
            pth = os.path.join(d, "params.npy")
            np.save(pth, params_now.astype(np.float64))
            cpu = cpu_baseline_mlp(sizes, pth, 16384)
    acc = None
    if args.surrogate_runs > 0:  # accuracy against the simulator: train on simulated runs, score held-out ones
        from paper_2110_04421_gb300 import surrogate as S
        acc = S.fit_and_score(runs=args.surrogate_runs, steps=args.surrogate_train_steps)
    f = mlp_flops_per_sample(sizes)
    peak, kind = measured_peak_bf16()
    fwd_tf = f * B / (fwd_ms / 1e3) / 1e12
    train_tf = 3 * f * B / (step_ms / 1e3) / 1e12
    return {"workload": w["name"] + f", batch {B}", "forward_ms": fwd_ms, "train_step_ms": step_ms,
            "forward_ms_mma_sync_path": fwd_mma_ms, "train_step_ms_mma_sync_path": step_mma_ms,
            "train_step_note": "forward keeping activations + input and weight gradients on tcgen05 GEMMs, "
                               "bias gradients, Adam; 3 x forward FLOPs counted",
            "samples_per_s": B / (fwd_ms / 1e3), "flops_per_sample_forward": f,
            "cpu_baseline": cpu,
            "accuracy": acc,
            "l2": "flushed before every timed call (write of twice its size)",
            "roofline": {"bound": "tensor", "achieved": fwd_tf, "peak": peak, "unit": "TFLOP/s", "frac": fwd_tf / peak,
                         "peak_kind": kind,
                         "kernel": "mlp_forward_tc_kernel (fused tcgen05)" if tc else "gemm_bf16_kernel (mma.sync)",
                         "traffic": traffic_from_profile(MLP_KERNEL_SOURCES, "mlp_forward_tc_b65536.md", B) if tc else None,
                         "train_step_tflops": train_tf}}


def run_ragged(args):
    """64 populations with N log-uniform in [1e4, 1e6] in one persistent launch per
    day (days replayed as a CUDA graph, tiling autotuned) against a loop of one
    plain launch per population per day."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import RaggedSimulation, Simulation

    w = W.ragged(64)
    T = max(3, min(args.batched_steps, args.steps))
    stream = torch.cuda.Stream()
    r = RaggedSimulation(w["pops"], w["params"], max_steps=args.warmup + T, stream=stream.cuda_stream)
    rows, bps = r.autotune(days_per_trial=2)
    r.step(args.warmup)
    r.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r.run(T, hist=False)  # one CUDA graph of T day launches
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, _, msgs = r.counters(args.warmup + T)
    r.close()
    messages = int(msgs[args.warmup:].astype(np.int64).sum())
    sims = [Simulation(p, par, p["age"], p["seed_ids"], max_steps=args.warmup + T, stream=stream.cuda_stream)
            for p, par in zip(w["pops"], w["params"])]
    for s in sims:
        s.step(args.warmup)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(T):
        for s in sims:
            s.step(1)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_loop = e2.elapsed_time(e3)
    for s in sims:
        s.close()
    # algorithmic bytes: each population's plain day (its arrays once)
    alg = sum(step_bytes_plain(int(p["n"]), int(sum(int(rp[-1]) for rp in p["row_ptr"])), len(p["row_ptr"]),
                               bool(par.get("vax_on", 0)))
              for p, par in zip(w["pops"], w["params"]))
    achieved = alg / (ms / T / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    cpu = None
    if not args.no_cpu_baseline:  # the populations one after another, whole days, as the oracle stands
        cpu = cpu_baseline(w["pops"], w["params"], args.cpu_seconds / 3, max_days=T + args.warmup)
    return {"workload": w["name"], "total_agents": int(sum(p["n"] for p in w["pops"])), "steps": T,
            "cpu_baseline": cpu,
            "value": messages / (ms / 1e3), "unit": "interactions/s", "ms_per_step": ms / T,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "kernel": "step_ragged_kernel", "alg_bytes_per_launch": alg,
                         "traffic": traffic_from_profile(DAY_KERNEL_SOURCES, "step_ragged_64pops.md",
                                                         int(sum(p["n"] for p in w["pops"])),
                                                         (args.warmup, args.warmup + T - 1))},
            "autotuned": {"rows_per_tile": rows, "blocks_per_sm": bps},
            "loop_of_plain_launches_ms_per_step": ms_loop / T, "multiple_of_plain_loop": ms_loop / ms}


def run_occupation(args):
    """The N=2e6 plain workload with its occupation network redrawn every day
    (23 occupations, 5-15 contacts a member): households stored, occupations and
    random network generated in the day kernel."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    w = W.plain_daily_occupation()
    n = w["n"]
    K = max(3, min(args.occupation_steps, args.steps))
    pop = W.population_daily_occupation(n, 0, w["n_seed"])
    static_edges = int(sum(int(r[-1]) for r in pop["row_ptr"]))
    stream = torch.cuda.Stream()

    def timed_days(graph):
        sim = Simulation(graph, w["params"], pop["age"], pop["seed_ids"], max_steps=args.warmup + K,
                         stream=stream.cuda_stream)
        sim.step(args.warmup)
        sim.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for e0, e1 in ev:
            e0.record(stream)
            sim.step(1)
            e1.record(stream)
        torch.cuda.synchronize()
        _, _, msgs = sim.counters()
        sim.close()
        return sum(e0.elapsed_time(e1) for e0, e1 in ev), int(msgs[args.warmup:args.warmup + K].astype(np.int64).sum())

    ms, msg = timed_days(pop)
    ms_ws, msg_ws = timed_days(dict(pop, occ_lattice=1, occ_rewire=0.1))
    cpu = None if args.no_cpu_baseline else cpu_baseline(pop, w["params"], args.cpu_seconds / 3)
    alg = step_bytes_occ(n, static_edges, len(pop["row_ptr"]), int(pop["occ_k"].size), True)
    peak, _ = measured_peak_hbm()
    avg = ms / K
    achieved = alg / (avg / 1e3) / 1e9
    return {"workload": w["name"], "value": msg / (ms / 1e3), "unit": "interactions/s", "ms_per_step": avg,
            "steps": K, "messages_per_day": msg / K, "cpu_baseline": cpu,
            "l2": f"inputs larger than L2: {alg / 1e6:.0f} MB algorithmic per day, no flush",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "step_plain_kernel (daily occupation networks)", "alg_bytes_per_launch": alg,
                         "traffic": traffic_from_profile(DAY_KERNEL_SOURCES, "step_plain_occ_n2e6.md", n,
                                                         (args.warmup, args.warmup + K - 1))},
            "watts_strogatz": {"workload": "the same with Watts-Strogatz occupations (ring lattice, rewiring 0.1)",
                               "value": msg_ws / (ms_ws / 1e3), "unit": "interactions/s", "ms_per_step": ms_ws / K,
                               "roofline": {"bound": "hbm", "achieved": alg / (ms_ws / K / 1e3) / 1e9, "peak": peak,
                                            "unit": "GB/s", "frac": alg / (ms_ws / K / 1e3) / 1e9 / peak}}}


def run_ws_random(args):
    """The N=2e6 plain workload with its global random network as a daily
    Watts-Strogatz graph (ring lattice over all agents, k = 2, rewiring 0.5, R24):
    the day's graph built on the device, then the day kernel."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    w = W.plain_large()
    n = w["n"]
    K = max(3, min(args.occupation_steps, args.steps))
    pop = dict(W.population(n, 0, w["n_seed"]), rand_ws=1, rand_ws_k=2, rand_ws_beta=0.5)
    stream = torch.cuda.Stream()
    sim = Simulation(pop, w["params"], pop["age"], pop["seed_ids"], max_steps=args.warmup + K, stream=stream.cuda_stream)
    sim.step(args.warmup)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, _, msgs = sim.counters()
    sim.close()
    msg = int(msgs[args.warmup:args.warmup + K].astype(np.int64).sum())
    cpu = None if args.no_cpu_baseline else cpu_baseline(pop, w["params"], args.cpu_seconds / 4)
    return {"workload": "plain N=2e6 with the random network as a daily Watts-Strogatz graph (k = 2, beta = 0.5)",
            "value": msg / (ms / 1e3), "unit": "interactions/s", "ms_per_step": ms / K, "steps": K,
            "days_timed": f"{args.warmup}..{args.warmup + K - 1}", "messages_per_day": msg / K,
            "launches_per_day": "day kernel + the graph's build (3 kernels, a prefix sum, 1 memset)",
            "cpu_baseline": cpu}


def run_den(args):
    """The N=2e6 plain workload with digital exposure notification (adoption 0.3,
    compliance 0.8, 7-day look-back): day kernel plus notification pass, timed
    from day 30 on, once test results are coming in."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    w = W.plain_large()
    n = w["n"]
    K = max(3, min(args.den_steps, args.steps))
    W0 = max(args.warmup, 30)
    pop = W.population(n, 0, w["n_seed"])
    params = dict(w["params"], den_on=1)
    stream = torch.cuda.Stream()
    sim = Simulation(pop, params, pop["age"], pop["seed_ids"], max_steps=W0 + K, stream=stream.cuda_stream)
    sim.step(W0)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, _, msgs = sim.counters()
    den = sim.notified()
    sim.close()
    msg = int(msgs[W0:W0 + K].astype(np.int64).sum())
    cpu = None if args.no_cpu_baseline else cpu_baseline(pop, params, args.cpu_seconds / 3)
    return {"workload": "plain N=2e6 with exposure notification (adoption 0.3, compliance 0.8, 7-day look-back)",
            "cpu_baseline": cpu,
            "value": msg / (ms / 1e3), "unit": "interactions/s", "ms_per_step": ms / K, "steps": K,
            "days_timed": f"{W0}..{W0 + K - 1}", "notified_per_day": float(den[W0:W0 + K].mean()),
            "launches_per_day": 2, "batched": run_den_batched(K, W0)}


def run_den_batched(K: int, W0: int):
    """The batched ensemble (N = 1e5 shared by B = 256 columns) with testing,
    quarantine and exposure notification, each column with its own app holders:
    days W0 .. W0 + K - 1, against the same ensemble without notification."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    w = W.batched()
    n, B = w["n"], w["B"]
    pop = W.population(n, 0, w["n_seed"])
    rp, seeds = W.batch_params(B, 0)
    out = {}
    for den_on in (1, 0):
        params = dict(w["params"], test_on=1, quar_on=1, den_on=den_on)
        stream = torch.cuda.Stream()
        sim = Simulation(pop, params, pop["age"], pop["seed_ids"], n_rep=B, rep_params=rp, rep_seeds=seeds,
                         max_steps=W0 + K, stream=stream.cuda_stream)
        sim.step(W0)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _, _, msgs = sim.counters()
        msg = int(msgs[W0:W0 + K].astype(np.int64).sum()) * B
        if den_on:
            den = sim.notified()
            out.update(value=msg / (ms / 1e3), unit="interactions/s", ms_per_step=ms / K,
                       notified_per_day_per_column=float(den[W0:W0 + K].mean()))
        else:
            out["ms_per_step_without_notification"] = ms / K
        sim.close()
    out["workload"] = ("batched N=1e5 B=256 with testing, quarantine and exposure notification (adoption 0.3, "
                       "compliance 0.8, 7-day look-back; app holders per column)")
    out["days_timed"] = f"{W0}..{W0 + K - 1}"
    out["launches_per_day"] = "day kernel + hit words + per-column notification"
    return out


def run_batched(args, rank: int = 0, world: int = 1, dist=None):
    """The batched ensemble: one N = 1e5 graph shared by B = 256 replicate columns.
    With several ranks the columns are split between them (column_range), each
    rank runs its own batch context over its columns, and the per-day new
    infections [T, B] are gathered at the end: no exchange on the simulation path."""
    import torch
    from paper_2110_04421_gb300 import workloads as W
    from paper_2110_04421_gb300.deabm import Simulation

    w = W.batched()
    n, B = w["n"], w["B"]
    Kb = max(3, min(args.batched_steps, args.steps))
    pop = W.population(n, 0, w["n_seed"])
    rp, seeds = W.batch_params(B, 0)
    lo, hi = column_range(B, rank, world)
    static_edges = int(sum(int(r[-1]) for r in pop["row_ptr"]))
    stream = torch.cuda.Stream()
    sim = Simulation(pop, w["params"], pop["age"], pop["seed_ids"], n_rep=hi - lo, rep_params=rp[lo:hi],
                     rep_seeds=seeds[lo:hi], max_steps=args.warmup + Kb, stream=stream.cuda_stream)
    sim.step(args.warmup)
    sim.sync()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(Kb)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ni, _, msgs = sim.counters()
    sim.close()
    msg_local = int(msgs[args.warmup:].astype(np.int64).sum()) * (hi - lo)
    (ms,), (msg_b,) = reduce_over_ranks(dist, [ms], [msg_local], "cuda")
    msg_b = int(msg_b)
    incidence = gather_columns(dist, ni[args.warmup:], B, world, "cuda")
    if rank != 0:
        return None
    alg = step_bytes_batch(n, B, static_edges, len(pop["row_ptr"]), True)
    peak, _ = measured_peak_hbm()
    achieved = alg / (ms / Kb / 1e3) / 1e9
    value = msg_b / (ms / 1e3)
    out = {"workload": "batched N=1e5 B=256 (R~U[2,6], weights~U[0.5,2], dose-2 delay~U{21..84}, own seeds)",
           "value": value, "unit": "interactions/s", "ms_per_step": ms / Kb, "steps": Kb,
           "columns_per_rank": [column_range(B, q, world) for q in range(world)],
           "new_infections_timed": int(incidence.sum()),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": "step_batch4_kernel", "alg_bytes_per_launch": alg,
                        "traffic": traffic_from_profile(DAY_KERNEL_SOURCES, "step_batch_n1e5_b256.md", n * B,
                                                        (args.warmup, args.warmup + Kb - 1)) if world == 1 else None}}
    if world > 1:
        out["roofline"]["note"] = "whole-job bytes over the slowest rank's time, B/world columns per rank"
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_columns(pop, w["params"], rp, seeds, args.cpu_seconds / 2)
    if args.no_loop or world > 1:
        return out
    # plain loop: the same B replicates one after another, same days
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sims = []
    for r in range(B):
        pr = dict(w["params"], R=float(rp[r, 0]), B_net=[float(rp[r, 1]), float(rp[r, 2])], B_rand=float(rp[r, 3]),
                  S_age=[float(x) for x in rp[r, 4:13]], dose2_delay=int(rp[r, 13]), seed=int(seeds[r]))
        s = Simulation(pop, pr, pop["age"], pop["seed_ids"], max_steps=args.warmup + Kb, stream=stream.cuda_stream)
        s.step(args.warmup)
        sims.append(s)
    torch.cuda.synchronize()
    e2.record(stream)
    for s in sims:
        s.step(Kb)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_loop = e2.elapsed_time(e3)
    for s in sims:
        s.close()
    out["plain_loop_value"] = msg_b / (ms_loop / 1e3)
    out["multiple_of_plain_loop"] = ms_loop / ms
    return out


# ---------------------------------------------------------------------------------------- CPU oracle
def _oracle_days(pops, params, seconds: float, max_days: int, threads: int):
    """Whole oracle days from day 0 of the population(s), in turn, each run for at
    most max_days, until about `seconds`; the oracle's per-agent loops on `threads`
    host threads.  Returns (messages, days, runs, seconds)."""
    import oracle
    used = oracle.set_threads(threads)
    msgs, days, runs, el = 0, 0, 0, 0.0
    try:
        t0 = time.perf_counter()
        while el < seconds:
            q = runs % len(pops)
            sim = oracle.Sim(pops[q], params[q], pops[q]["age"], pops[q]["seed_ids"])
            runs += 1
            for _ in range(max_days):
                msgs += sim.step(diag=False)["messages"]
                days += 1
                el = time.perf_counter() - t0
                if el >= seconds:
                    break
    finally:
        oracle.set_threads(1)
    return msgs, days, runs, el, used


def cpu_baseline(pops, params, seconds: float, max_days: int = 180):
    """The oracle, as written (plain C; its per-agent loops on OpenMP threads, which
    changes no result): whole days from day 0 of the given population(s) -- one
    population, or a list taken in turn -- each run for at most max_days (the
    workload's horizon).  Timed on every host core (the reported value) and on one
    core, about seconds/2 each."""
    pops = pops if isinstance(pops, list) else [pops]
    params = params if isinstance(params, list) else [params] * len(pops)

    def what(runs):
        sizes = sorted({int(p["n"]) for p in pops[:runs]})
        return (f"the same N={pops[0]['n']} population" if len(pops) == 1
                else f"{min(runs, len(pops))} of the {len(pops)} populations in turn (N {sizes[0]}..{sizes[-1]})")

    m1, d1, r1, e1, _ = _oracle_days(pops, params, seconds / 2, max_days, 1)
    ma, da, ra, ea, used = _oracle_days(pops, params, seconds / 2, max_days, host_cores())
    return {"value": ma / ea, "unit": "interactions/s", "cores": used, "kind": "oracle",
            "sample": f"{da} whole days of {what(ra)}, from day 0, at most {max_days} days a run, {ea:.1f} s, "
                      f"{used} threads (OpenMP over agents)",
            "cpu": cpu_model(),
            "one_core": {"value": m1 / e1, "unit": "interactions/s", "cores": 1,
                         "sample": f"{d1} whole days of {what(r1)}, {e1:.1f} s, single thread"}}


def cpu_baseline_columns(pop, base, rp, seeds, seconds: float):
    """The oracle on replicate columns of the batched workload, one after another
    (each column is an independent run on the shared graph), whole days from day
    0 of up to 8 columns, about seconds/2 on every host core (the reported value)
    and seconds/2 on one core."""
    cols = []
    for r in range(min(8, len(seeds))):
        cols.append(dict(base, R=float(rp[r, 0]), B_net=[float(rp[r, 1]), float(rp[r, 2])], B_rand=float(rp[r, 3]),
                         S_age=[float(x) for x in rp[r, 4:13]], dose2_delay=int(rp[r, 13]), seed=int(seeds[r])))
    pops = [pop] * len(cols)
    m1, d1, r1, e1, _ = _oracle_days(pops, cols, seconds / 2, 180, 1)
    ma, da, ra, ea, used = _oracle_days(pops, cols, seconds / 2, 180, host_cores())
    note = ("the columns are independent, so this per-column rate is the whole batch's rate "
            "(extrapolated, not run for all columns)")
    return {"value": ma / ea, "unit": "interactions/s", "cores": used, "kind": "oracle",
            "sample": f"{da} replicate-days over {min(ra, len(cols))} of the {len(seeds)} columns (from day 0), "
                      f"{ea:.1f} s, {used} threads (OpenMP over agents); {note}", "cpu": cpu_model(),
            "one_core": {"value": m1 / e1, "unit": "interactions/s", "cores": 1,
                         "sample": f"{d1} replicate-days over {min(r1, len(cols))} columns, {e1:.1f} s, single thread"}}


def cpu_baseline_relaxed(pop, params, tau, theta, target, T):
    """The FP64 relaxed oracle (full history, reverse sweep) for one gradient of the
    same workload, single thread."""
    import oracle
    rx = oracle.Relaxed(pop, params, pop["age"], pop["seed_ids"], tau=tau)
    t0 = time.perf_counter()
    rx.run(theta, T, target=np.asarray(target, np.float64), grad=True)
    el = time.perf_counter() - t0
    return {"value": el * 1e3, "unit": "ms per gradient", "cores": 1, "kind": "oracle",
            "sample": f"one gradient (forward and reverse sweep in FP64, full history), N={pop['n']}, {T} days, "
                      f"{el:.1f} s, single thread", "cpu": cpu_model()}


def cpu_baseline_mlp(sizes, params, batch: int):
    """The numpy MLP oracle (FP64 with the kernel's BF16 rounding points) on
    `batch` samples, in a child process: BLAS on every host core (the reported
    value) and on one."""
    def timed(threads):
        code = ("import sys, time, json, numpy as np\n"
                f"sys.path.insert(0, {ROOT!r})\n"
                "from oracle import mlp\n"
                f"sizes = {list(sizes)!r}\n"
                f"params = np.load({params!r})\n"
                f"x = np.random.default_rng(0).random(({batch}, sizes[0]))\n"
                "t0 = time.perf_counter(); mlp.forward(params, sizes, x); el = time.perf_counter() - t0\n"
                "print(json.dumps({'seconds': el}))\n")
        n = str(threads)
        env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
        return json.loads(out.stdout.strip().splitlines()[-1])["seconds"]

    el1 = timed(1)
    cores = host_cores()
    ela = timed(cores)
    return {"value": batch / ela, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"forward of {batch} samples (FP64 with BF16 rounding points), {ela:.2f} s, BLAS on {cores} threads",
            "cpu": cpu_model(),
            "one_core": {"value": batch / el1, "unit": "samples/s", "cores": 1,
                         "sample": f"the same forward, {el1:.2f} s, single-threaded BLAS"}}


def cpu_model() -> str:
    """The host CPU as lscpu names it (vendor and model; aarch64 hosts have no
    'model name' line in /proc/cpuinfo), with the online core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        f = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                f.setdefault(k.strip(), v.strip())
        parts = [f.get("Vendor ID"), f.get("Model name")]
        name = " ".join(x for x in parts if x and x != "-") or None
    except Exception:
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if "model name" in line:
                    name = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return f"{name or platform.processor() or 'unknown'} ({platform.machine()}, {host_cores()} cores)"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world, local):
    """The oracle arm: each step is one whole oracle day of the same workload, the
    oracle's per-agent loops on every host core (OpenMP over agents)."""
    if rank != 0:
        return
    import oracle
    from paper_2110_04421_gb300 import workloads as W
    w = W.plain_large()
    pop = W.population(w["n"], 0, w["n_seed"])
    cores = oracle.set_threads(host_cores())
    sim = oracle.Sim(pop, w["params"], pop["age"], pop["seed_ids"])
    for _ in range(args.warmup):
        sim.step(diag=False)
    msgs = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        msgs += sim.step(diag=False)["messages"]
    el = time.perf_counter() - t0
    oracle.set_threads(1)
    value = msgs / el
    line = {"impl": "reference", "metric": "agent interactions/s on 1 GB300 (plain day kernel; batched B=256 in "
            "'batched')", "value": value, "unit": "interactions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generators shaped like the paper's population)",
            "config": {"workload": PLAIN_WORKLOAD, "n_agents": w["n"],
                       "days_timed": f"{args.warmup}..{args.warmup + args.steps - 1}"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} whole oracle days after {args.warmup} warm-up days, "
                                       f"{cores} threads (OpenMP over agents)",
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=177)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batched-steps", type=int, default=177)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-loop", action="store_true", help="skip the plain per-replicate loop of the batched leg")
    ap.add_argument("--no-relaxed", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-runs", type=int, default=20_000,
                    help="simulated runs for the surrogate's accuracy (79/20/1 %% split); 0 skips it")
    ap.add_argument("--surrogate-train-steps", type=int, default=3000)
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-occupation", action="store_true")
    ap.add_argument("--occupation-steps", type=int, default=20)
    ap.add_argument("--no-den", action="store_true")
    ap.add_argument("--den-steps", type=int, default=20)
    ap.add_argument("--no-ws", action="store_true", help="skip the Watts-Strogatz random-network leg")
    ap.add_argument("--calib-steps", type=int, default=200)
    ap.add_argument("--only", default="all",
                    choices=["all", "plain", "batched", "relaxed", "surrogate", "ragged", "occupation", "den", "ws"],
                    help="profiling runs: time one workload only")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.only == "batched":
        import __graft_entry__
        __graft_entry__.build()
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(run_batched(args)))
        return
    if args.only in ("relaxed", "surrogate", "ragged", "occupation", "den", "ws"):
        import __graft_entry__
        __graft_entry__.build()
        import torch
        torch.cuda.set_device(local)
        fn = {"relaxed": run_relaxed, "surrogate": run_surrogate, "ragged": run_ragged,
              "occupation": run_occupation, "den": run_den, "ws": run_ws_random}[args.only]
        print(json.dumps(fn(args)))
        return
    if args.only == "plain":
        args.no_batched = True
        args.no_relaxed = True
        args.no_surrogate = True
        args.no_ragged = True
        args.no_occupation = True
        args.no_den = True
        args.no_ws = True
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        import __graft_entry__
        if local == 0:
            __graft_entry__.build()
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
