"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it draws populations (ages,
households, occupation groups, initial cases) with numpy's seeded generator and
lists parameter sets.  Both the CUDA path and the CPU oracle consume what it
returns; neither is imported here.

The paper's populations come from King County census and mobility data
(Sec. 3 "Agent State Definition"), which is not available; these generators
stand in for it with the shapes the paper describes:
  * ages: 9 ten-year bins (Sec. 3 "Infection Transmission"), uniform;
  * households: complete graphs (Sec. 3 "Interaction Networks"), sizes 1-6 with
    probabilities (.28, .35, .15, .13, .06, .03), members given consecutive ids;
  * occupation: groups of 20 drawn from a random permutation of the agents,
    each agent receiving in-links from 10 distinct members of its group;
  * random network: regenerated every day by the method itself (not here);
  * daily occupation networks (optional): 23 occupations (Sec. 3 "Agent State
    Definition") with Dirichlet(2) shares of the agents, each with its own number
    of in-contacts a member has a day, uniform on {5..15}; the contacts
    themselves are drawn every day by the method (not here).
The disease parameters are placeholders: the paper cites other work for them
(Sec. 3 "Disease Progression") and prints none.
"""
from __future__ import annotations

import copy

import numpy as np

HOUSEHOLD_SIZE_P = (0.28, 0.35, 0.15, 0.13, 0.06, 0.03)
N_AGE = 9
N_REP_PARAMS = 14  # R, B_household, B_occupation, B_random, S_age[9], second-dose delay


def household_sizes(n: int, rng: np.random.Generator) -> np.ndarray:
    """Household sizes covering exactly n agents (the last household is truncated)."""
    mean = sum((i + 1) * p for i, p in enumerate(HOUSEHOLD_SIZE_P))
    sizes = rng.choice(np.arange(1, 7), size=int(n / mean * 1.2) + 16, p=HOUSEHOLD_SIZE_P)
    cs = np.cumsum(sizes)
    while cs[-1] < n:
        sizes = np.concatenate([sizes, rng.choice(np.arange(1, 7), size=64, p=HOUSEHOLD_SIZE_P)])
        cs = np.cumsum(sizes)
    k = int(np.searchsorted(cs, n))
    sizes = sizes[: k + 1].copy()
    sizes[-1] -= int(cs[k] - n)
    return sizes[sizes > 0].astype(np.int64)


def household_csr(sizes: np.ndarray):
    """Complete graph inside each household; destination-sorted CSR, sources ascending."""
    n = int(sizes.sum())
    start = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    deg = np.repeat(sizes - 1, sizes)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = np.zeros(int(row_ptr[-1]), np.uint32)
    for s in range(2, int(sizes.max(initial=1)) + 1):
        st = start[sizes == s]
        if st.size == 0:
            continue
        members = st[:, None] + np.arange(s)[None, :]
        for p in range(s):
            src = np.delete(members, p, axis=1)
            dst = members[:, p]
            col[row_ptr[dst][:, None] + np.arange(s - 1)[None, :]] = src
    return row_ptr.astype(np.uint32), col


def occupation_csr(n: int, rng: np.random.Generator, group: int = 20, links: int = 10):
    """Groups of `group` agents from a random permutation; each agent gets `links`
    distinct in-links from its group-mates (all of them if the group is smaller)."""
    perm = rng.permutation(n).astype(np.int64)
    deg = np.zeros(n, np.int64)
    parts = []  # (dst ids, src matrix)
    G = n // group
    if G:
        members = perm[: G * group].reshape(G, group)
        others = np.array([[q for q in range(group) if q != p] for p in range(group)])  # (group, group-1)
        k = min(links, group - 1)
        keys = rng.random((G, group, group - 1), dtype=np.float32)
        pick = np.argsort(keys, axis=2, kind="stable")[:, :, :k]          # (G, group, k)
        pos = np.take_along_axis(np.broadcast_to(others, (G, group, group - 1)), pick, axis=2)
        src = np.take_along_axis(members[:, None, :].repeat(group, axis=1), pos, axis=2)
        src = np.sort(src, axis=2)
        parts.append((members.reshape(-1), src.reshape(-1, k)))
        deg[members.reshape(-1)] = k
    rest = perm[G * group:]
    r = rest.size
    if r >= 2:
        k = min(links, r - 1)
        rows = []
        for p in range(r):
            cand = np.delete(rest, p)
            rows.append(np.sort(rng.choice(cand, size=k, replace=False)))
        parts.append((rest, np.array(rows, np.int64)))
        deg[rest] = k
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = np.zeros(int(row_ptr[-1]), np.uint32)
    for dst, src in parts:
        kk = src.shape[1]
        col[row_ptr[dst][:, None] + np.arange(kk)[None, :]] = src
    return row_ptr.astype(np.uint32), col


N_OCCUPATION = 23


def occupations(n: int, seed: int = 0, n_occ: int = N_OCCUPATION, k_lo: int = 5, k_hi: int = 15):
    """Occupation of every agent (u32, fixed for the run) and the number of daily
    in-contacts of a member of each occupation (u8)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x0CC]))
    share = rng.dirichlet(np.full(n_occ, 2.0))
    group = rng.choice(n_occ, size=n, p=share).astype(np.uint32)
    k = rng.integers(k_lo, k_hi + 1, size=n_occ, dtype=np.uint8)
    return group, k


def workplaces(n: int, seed: int = 0, size: int = 20, k: int = 10):
    """Occupation groups of `size` agents from a random permutation (the last one
    ragged), each member meeting k of them a day: the static occupation network's
    groups with their contacts redrawn daily."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x0CD]))
    perm = rng.permutation(n)
    group = np.empty(n, np.uint32)
    group[perm] = (np.arange(n) // size).astype(np.uint32)
    n_occ = (n + size - 1) // size
    return group, np.full(n_occ, k, np.uint8)


def population(n: int, seed: int = 0, n_seed_infections: int = 10) -> dict:
    """Ages, household and occupation CSRs and the initial cases for n agents."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5EED]))
    age = rng.integers(0, N_AGE, size=n, dtype=np.uint8)
    sizes = household_sizes(n, rng)
    hh_rp, hh_col = household_csr(sizes)
    oc_rp, oc_col = occupation_csr(n, rng)
    k = min(int(n_seed_infections), n)
    seeds = np.sort(rng.choice(n, size=k, replace=False)).astype(np.uint32)
    return dict(n=n, age=age, row_ptr=[hh_rp, oc_rp], col=[hh_col, oc_col], seed_ids=seeds,
                household_sizes=sizes)


# --------------------------------------------------------------------------- parameters
def default_params() -> dict:
    """Placeholder disease parameters.  Names follow Eq. 1: R, S_age (S_a),
    A_class (A_s for asymptomatic / mild / severe infectors), B_net (B_n per
    static network: household, occupation), B_rand (random network), inv_Ibar (1/I)."""
    dur_lo = [[0] * N_AGE for _ in range(8)]
    dur_hi = [[0] * N_AGE for _ in range(8)]
    # stage index: 1 asym, 2 presym-mild, 3 presym-severe, 4 mild, 5 severe, 6 hospital, 7 ICU
    for st, (lo, hi) in {1: (5, 10), 2: (2, 4), 3: (2, 4), 4: (5, 10), 5: (3, 7), 6: (5, 15), 7: (5, 15)}.items():
        dur_lo[st] = [lo] * N_AGE
        dur_hi[st] = [hi] * N_AGE
    return dict(
        R=3.0, inv_Ibar=1.0 / 14.0, dt=1.0,   # 1/I: I = mean daily interactions (about 14 here)
        B_net=[2.0, 1.0], B_rand=1.0, rand_mean=2.0,
        rand_mean_age=None,  # per-age-bin Poisson means of the random network (None: rand_mean for all)
        S_age=[1.0] * N_AGE,
        A_class=[0.5, 1.0, 1.0],
        inf_shape=[4.0, 4.0, 4.0], inf_scale=[1.25, 1.25, 1.25], inf_len=30,
        p_asym=[0.45, 0.40, 0.35, 0.30, 0.30, 0.25, 0.20, 0.20, 0.20],
        p_sev=[0.02, 0.03, 0.05, 0.08, 0.12, 0.18, 0.28, 0.38, 0.50],
        p_hosp=[0.20, 0.20, 0.25, 0.30, 0.35, 0.40, 0.50, 0.60, 0.70],
        p_icu=[0.10, 0.10, 0.15, 0.20, 0.25, 0.30, 0.35, 0.40, 0.45],
        p_death=[0.05, 0.05, 0.10, 0.15, 0.20, 0.30, 0.40, 0.50, 0.60],
        dur_lo=dur_lo, dur_hi=dur_hi,
        test_on=0, test_sens=0.95, test_lo=3, test_hi=5,          # RT-PCR (Sec. 4.3)
        quar_on=0, quar_days=14, q_dropout=0.0,                     # Sec. 4.1
        vax_on=0, vax_start=30, vax_onset=12, dose2_delay=21,       # Sec. 5
        vax_rate=0.01, vax_eff1=0.8, vax_eff2=0.95,
        vax_strategy=0,   # 0 static age-priority schedule; 1 standard, 2 delayed second dose, 3 delayed except 65+
        elderly_bin=6,    # first age bin treated as "65+" (the 61-70 bin holds Table 1's 68-year-olds)
        vax_nonsterile=0, # 1: vaccine immunity is non-sterilising (infections become asymptomatic)
        den_on=0, den_adoption=0.3, den_compliance=0.8, den_window=7,  # exposure notification (Sec. 4.2, 4.5)
        seed=0, net_seed=0,
    )


def params_with(**kw) -> dict:
    p = copy.deepcopy(default_params())
    for k, v in kw.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


# --------------------------------------------------------------------------- workloads
def plain_small():
    """N=10,000 agents, 60 days, 10 initial cases, seed 0, no interventions."""
    return dict(name="plain N=1e4 T=60", n=10_000, T=60, n_seed=10, params=params_with())


def plain_large():
    """N=2,000,000 agents, 180 days, 0.5% initial cases, testing + 14-day quarantine
    of symptomatic agents, vaccination of 1% of agents a day from day 30."""
    return dict(name="plain N=2e6 T=180", n=2_000_000, T=180, n_seed=10_000,
                params=params_with(test_on=1, quar_on=1, vax_on=1, vax_start=30, vax_rate=0.01))


def population_daily_occupation(n: int, seed: int = 0, n_seed_infections: int = 10) -> dict:
    """Households as a stored network and the 23 occupations as daily networks."""
    pop = population(n, seed, n_seed_infections)
    pop["row_ptr"], pop["col"] = pop["row_ptr"][:1], pop["col"][:1]
    pop["occ_group"], pop["occ_k"] = occupations(n, seed)
    return pop


def plain_daily_occupation():
    """The N=2e6 plain workload with its occupation network redrawn every day:
    23 occupations, 5-15 daily in-contacts per member by occupation."""
    w = plain_large()
    return dict(w, name="plain N=2e6 T=180, daily occupation networks (23 occupations)")


def batch_params(B: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Per-replicate parameter rows [B, 14] (R ~ U[2,6]; household, occupation and
    random weights ~ U[0.5,2]; S_age = 1; second-dose delay ~ U{21..84}) and seeds."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xBA7C]))
    rp = np.zeros((B, N_REP_PARAMS), np.float32)
    rp[:, 0] = rng.uniform(2.0, 6.0, B)
    rp[:, 1:4] = rng.uniform(0.5, 2.0, (B, 3))
    rp[:, 4:13] = 1.0
    rp[:, 13] = rng.integers(21, 85, B)
    seeds = rng.integers(0, 2**63 - 1, B, dtype=np.int64).astype(np.uint64)
    return rp, seeds


def batched():
    """One N=100,000 graph shared by B=256 replicates, 180 days, vaccination at
    0.3%/day from day 20 with a per-replicate second-dose delay."""
    return dict(name="batched N=1e5 B=256 T=180", n=100_000, B=256, T=180, n_seed=10,
                params=params_with(vax_on=1, vax_start=20, vax_rate=0.003))


def relaxed_workload():
    """Differentiable inverse run: N = 100,000, 90 days, tau = 0.5; the target curve
    comes from hidden parameters R = 3.5, weights 2.0 / 1.0 / 0.7 (household,
    occupation, random); calibration starts from R = 2.5, weights 1.0 / 1.0 / 1.0."""
    p = params_with(seed=0, net_seed=0)
    hidden = np.array([3.5, 2.0, 1.0, 0.7] + [1.0] * N_AGE, np.float32)
    start = np.array([2.5, 1.0, 1.0, 1.0] + [1.0] * N_AGE, np.float32)
    return dict(name="relaxed N=1e5 T=90 tau=0.5", n=100_000, T=90, tau=0.5, n_seed=10, params=p,
                hidden=hidden, start=start, steps=200, lr=0.02)


# parameter box of the surrogate's inputs: R, three network weights, nine age
# susceptibilities, second-dose delay (days)
SURROGATE_LO = np.array([2.0, 0.5, 0.5, 0.5] + [0.5] * N_AGE + [21.0], np.float32)
SURROGATE_HI = np.array([6.0, 2.0, 2.0, 2.0] + [1.5] * N_AGE + [84.0], np.float32)


def surrogate_params(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """[n, 14] parameter rows drawn uniformly in the surrogate's box (delay whole
    days) and a Philox seed per row."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5A77]))
    rp = rng.uniform(SURROGATE_LO, SURROGATE_HI, (n, N_REP_PARAMS)).astype(np.float32)
    rp[:, 13] = rng.integers(21, 85, n)
    seeds = rng.integers(0, 2**63 - 1, n, dtype=np.int64).astype(np.uint64)
    return rp, seeds


def surrogate_workload():
    """Surrogate: MLP 14 -> 3 x 256 (GELU) -> 180 trained on 50,000 batched runs of
    the N = 100,000 ensemble workload (80/20 split), inference batch 65,536."""
    return dict(name="surrogate MLP 14-256x3-180", n_runs=50_000, n=100_000, T=180, B=256, hidden=256, depth=3,
                batch=65_536, params=batched()["params"])


def ragged(n_pops: int = 64, lo: float = 1e4, hi: float = 1e6, seed: int = 0):
    """A ragged batch: n_pops populations with N log-uniform in [lo, hi], each with
    its own generated graph, 10 initial cases, own seeds, the plain disease model."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x4A66]))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_pops)).astype(np.int64)
    pops, params = [], []
    for q, n in enumerate(sizes):
        pops.append(population(int(n), seed=1000 + q, n_seed_infections=10))
        params.append(params_with(seed=int(rng.integers(0, 2**62)), net_seed=int(rng.integers(0, 2**62)),
                                  R=float(rng.uniform(2.0, 6.0))))
    return dict(name=f"ragged {n_pops} populations, N log-uniform [{lo:.0e}, {hi:.0e}]", pops=pops, params=params)
