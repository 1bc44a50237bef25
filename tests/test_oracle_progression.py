"""Pins for the disease-stage/timer machine (Sec. 3 "Disease Progression") and the
interventions (Sec. 4): invariants that hold at every step, plus exact replay of
each random decision from the (separately pinned) Philox words and thresholds."""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W

S, ASYM, PRE_MILD, PRE_SEV, MILD, SEV, HOSP, ICU, REC, VAX, DEAD = range(11)
ALLOWED = {S: {S, ASYM, PRE_MILD, PRE_SEV, VAX}, ASYM: {ASYM, REC}, PRE_MILD: {PRE_MILD, MILD},
           PRE_SEV: {PRE_SEV, SEV}, MILD: {MILD, REC}, SEV: {SEV, HOSP, REC}, HOSP: {HOSP, ICU, REC},
           ICU: {ICU, DEAD, REC}, REC: {REC}, VAX: {VAX}, DEAD: {DEAD}}
INFECTED = set(range(ASYM, ICU + 1))


def word(seed, agent, step, stream, idx=0):
    return int(oracle.philox([agent, step, stream, 0], [seed & 0xFFFFFFFF, seed >> 32])[idx])


def unif_int(w, lo, hi):
    return lo + ((w * (hi - lo + 1)) >> 32)


def run_traj(n=3000, T=90, **kw):
    pop = W.population(n, 3, 25)
    p = W.params_with(**kw)
    sim = oracle.Sim(pop, p, pop["age"], pop["seed_ids"])
    traj = [sim.state.copy()]
    diags = []
    for _ in range(T):
        diags.append(sim.step())
        traj.append(sim.state.copy())
    return pop, p, sim, traj, diags


@pytest.fixture(scope="module")
def traj_interventions():
    return run_traj(test_on=1, quar_on=1, q_dropout=0.05, vax_on=1, vax_start=15, vax_rate=0.02,
                    dose2_delay=21, seed=123, net_seed=321, R=4.0)


def test_invariants_every_step(traj_interventions):
    pop, p, sim, traj, diags = traj_interventions
    n = pop["n"]
    for t, d in enumerate(diags):
        a, b = traj[t], traj[t + 1]
        assert d["hist"].sum() == n
        assert np.array_equal(np.bincount(b.stage, minlength=11), d["hist"])
        for s in range(11):
            moved = np.unique(b.stage[a.stage == s])
            assert set(moved.tolist()) <= ALLOWED[s], (t, s, moved)
        newly = (a.stage == S) & np.isin(b.stage, [ASYM, PRE_MILD, PRE_SEV])
        assert newly.sum() == d["new_inf"]
        assert np.all(b.tinf[newly] == 1)
        stay = (a.stage == b.stage) & np.isin(a.stage, list(INFECTED))
        assert np.all(b.timer[stay] == a.timer[stay] - 1)
        assert np.all(b.timer[stay] >= 1)
        cont = np.isin(a.stage, list(INFECTED)) & np.isin(b.stage, list(INFECTED))
        assert np.all(b.tinf[cont] == a.tinf[cont] + 1)
        done = np.isin(b.stage, [S, REC, VAX, DEAD]) & np.isin(a.stage, list(INFECTED))
        assert np.all(b.timer[done] == 0)
        # only susceptible agents are ever infected, and only those with p > 0
        assert np.all(d["p32"][newly] > 0)
        assert np.all(d["u32"][newly] < d["p32"][newly])


def test_decisions_replay_from_philox(traj_interventions):
    pop, p, sim, traj, diags = traj_interventions
    age = pop["age"]
    seed = p["seed"]
    checked = 0
    for t in range(len(diags)):
        a, b = traj[t], traj[t + 1]
        idx = np.nonzero(a.stage != b.stage)[0]
        for j in idx[:60]:
            j = int(j)
            sa, sb, ag = int(a.stage[j]), int(b.stage[j]), int(age[j])
            if sb == VAX:
                continue
            w = oracle.philox([j, t, 1, 0], [seed & 0xFFFFFFFF, seed >> 32])
            if sa == S:
                if w[0] < oracle.threshold(p["p_asym"][ag]):
                    want = ASYM
                elif w[2] < oracle.threshold(p["p_sev"][ag]):
                    want = PRE_SEV
                else:
                    want = PRE_MILD
                assert sb == want
            elif sa == SEV:
                assert sb == (HOSP if w[3] < oracle.threshold(p["p_hosp"][ag]) else REC)
            elif sa == HOSP:
                assert sb == (ICU if w[3] < oracle.threshold(p["p_icu"][ag]) else REC)
            elif sa == ICU:
                assert sb == (DEAD if w[3] < oracle.threshold(p["p_death"][ag]) else REC)
            if sb in INFECTED:
                lo, hi = p["dur_lo"][sb][ag], p["dur_hi"][sb][ag]
                assert b.timer[j] == unif_int(int(w[1]), lo, hi)
            checked += 1
    assert checked > 500


def test_infection_decision_is_u_below_p(traj_interventions):
    pop, p, sim, traj, diags = traj_interventions
    for t in (5, 20, 40):
        d = diags[t]
        for j in range(0, pop["n"], 11):
            u = (word(p["seed"], j, t, 0) >> 8) * 2.0**-24
            assert d["u32"][j] == np.float32(u)
        sus = traj[t].stage == S
        assert np.array_equal((d["u32"] < d["p32"]) & sus,
                              (traj[t].stage == S) & np.isin(traj[t + 1].stage, [ASYM, PRE_MILD, PRE_SEV]))


def test_branch_frequencies(traj_interventions):
    pop, p, sim, traj, diags = traj_interventions
    age = pop["age"]
    new_stage, new_age = [], []
    for t in range(len(diags)):
        a, b = traj[t], traj[t + 1]
        m = (a.stage == S) & np.isin(b.stage, [ASYM, PRE_MILD, PRE_SEV])
        new_stage += b.stage[m].tolist()
        new_age += age[m].tolist()
    new_stage, new_age = np.array(new_stage), np.array(new_age)
    assert new_stage.size > 1000
    pa = np.array(p["p_asym"])[new_age]
    n_asym = (new_stage == ASYM).sum()
    mean, var = pa.sum(), (pa * (1 - pa)).sum()
    assert abs(n_asym - mean) < 5 * np.sqrt(var)


def test_quarantine_timeline(traj_interventions):
    """Symptom onset -> test (positive w.p. sensitivity, result after U{3..5} days)
    -> 14 days of quarantine with daily dropout; quarantined infectors emit nothing."""
    pop, p, sim, traj, diags = traj_interventions
    seed = p["seed"]
    n_onset = n_pos = 0
    for t in range(len(diags) - 20):
        a, b = traj[t], traj[t + 1]
        onset = ((a.stage == PRE_MILD) & (b.stage == MILD)) | ((a.stage == PRE_SEV) & (b.stage == SEV))
        onset &= ((a.qt & 0x0F) <= 1) & ((a.qt >> 4) == 0)
        for j in np.nonzero(onset)[0][:40]:
            j = int(j)
            if (b.qt[j] & 0x0F) != 0:
                continue
            w = oracle.philox([j, t, 5, 0], [seed & 0xFFFFFFFF, seed >> 32])
            pos = w[0] < oracle.threshold(p["test_sens"])
            delay = unif_int(int(w[1]), p["test_lo"], p["test_hi"])
            assert (b.qt[j] >> 4) == delay
            assert bool(b.flags[j] & 0x04) == bool(pos)
            n_onset += 1
            # the result lands `delay` updates later
            r = traj[t + 1 + delay]
            assert (r.qt[j] >> 4) == 0
            if pos:
                n_pos += 1
                assert (r.qt[j] & 0x0F) == p["quar_days"]
            else:
                assert (r.qt[j] & 0x0F) == 0
    assert n_onset > 50 and n_pos > 0.8 * n_onset
    # quarantined agents have zero infectiousness
    for t in range(len(diags)):
        q = (traj[t].qt & 0x0F) > 0
        assert np.all(diags[t]["inf32"][q] == 0)


def test_quarantine_lasts_exactly_14_days_without_dropout():
    pop, p, sim, traj, diags = run_traj(n=2000, T=80, test_on=1, quar_on=1, q_dropout=0.0, R=4.0, seed=9)
    q = np.array([(s.qt & 0x0F) > 0 for s in traj])     # [T+1, n]
    lengths = []
    for j in range(pop["n"]):
        x = q[:, j].astype(int)
        starts = np.nonzero(np.diff(np.concatenate([[0], x])) == 1)[0]
        ends = np.nonzero(np.diff(np.concatenate([x, [0]])) == -1)[0]
        for s_, e_ in zip(starts, ends):
            if e_ < len(traj) - 1:
                lengths.append(e_ - s_ + 1)
    assert len(lengths) > 20 and set(lengths) == {14}


def test_vaccination_schedule_priority():
    # priority: age bin descending, then id ascending; Q = floor(rate * N) per day
    age = np.array([3, 8, 8, 0, 5, 3], np.uint8)
    d = oracle.vax_days(age, 10, 2.0 / 6.0)   # Q = 2
    assert d.tolist() == [11, 10, 10, 12, 11, 12]
    assert oracle.vax_days(age, 10, 0.0).tolist() == [0x7FFF] * 6


def test_vaccine_onset_replays_from_philox():
    """No infections: dose 1 at the scheduled day; immune (stage VAX) 12 days later iff
    the agent's vaccine word < threshold(eff1); else immune 12 days after dose 2 iff
    the same word < threshold(eff2)."""
    n, T = 600, 80
    pop = W.population(n, 4, 0)
    p = W.params_with(vax_on=1, vax_start=3, vax_rate=0.05, dose2_delay=25, vax_eff1=0.6, vax_eff2=0.9,
                      seed=2024)
    sim = oracle.Sim(pop, p, pop["age"], None)
    for _ in range(T):
        sim.step(diag=False)
    d1 = oracle.vax_days(pop["age"], 3, 0.05)
    for j in range(n):
        w = word(2024, j, 0, 7)
        if d1[j] + 12 < T and w < oracle.threshold(0.6):
            want = VAX
        elif d1[j] + 25 + 12 < T and w < oracle.threshold(0.9):
            want = VAX
        else:
            want = S
        assert sim.state.stage[j] == want, j
        if d1[j] < T:
            assert sim.state.flags[j] & 0x01
        if d1[j] + 25 < T:
            assert sim.state.flags[j] & 0x02
