"""Pins for digital exposure notification (Sec. 4.2).

* app holders: a fraction den_adoption of the agents, drawn once (binomial band;
  0 and 1 give nobody and everybody).
* star, worked by hand: the centre's positive result lands on step 0; every
  leaf it had an in-edge to, holding the app, in the community and out of
  quarantine, is notified that step, complies (compliance 1), is tested on step
  1 and, when infected, tests positive (sensitivity 1), is quarantined when the
  result lands and notifies in turn.  Leaves without the app, in quarantine, in
  hospital, or linked only towards the centre are not notified.
* look-back window: with the random network only, the notified set is exactly
  the app holders that drew the positive agent among their in-contacts on one
  of the last den_window steps (this one included).
* compliance: the share of notified agents that take the test is
  den_compliance (binomial band).
"""
import numpy as np
import pytest

import oracle
from paper_2110_04421_gb300 import workloads as W

FL_POS, FL_DEN, FL_APP = 0x04, 0x10, 0x20
S, ASYM, MILD, HOSP = 0, 1, 4, 6


def qt(qd, cd):
    return (qd & 0x0F) | ((cd & 0x07) << 4)


def star_graph(n_leaves):
    n = n_leaves + 1
    rp = np.zeros(n + 1, np.uint32)
    rp[2:] = np.arange(1, n_leaves + 1)  # row 0 (centre) empty; leaf l has one in-edge from 0
    col = np.zeros(n_leaves, np.uint32)
    return dict(n=n, row_ptr=[rp], col=[col])


def den_params(**kw):
    base = dict(den_on=1, den_adoption=1.0, den_compliance=1.0, test_on=1, quar_on=1, test_sens=1.0,
                test_lo=2, test_hi=2, rand_mean=0.0, R=0.0, B_net=[1.0])
    base.update(kw)
    return W.params_with(**base)


def test_app_holders_share():
    n = 20000
    g = dict(n=n, row_ptr=[], col=[])
    for a in (0.0, 0.3, 1.0):
        s = oracle.Sim(g, den_params(den_adoption=a), np.zeros(n, np.uint8))
        k = int((s.state.flags & FL_APP).astype(bool).sum())
        if a in (0.0, 1.0):
            assert k == int(a * n)
        else:
            sd = np.sqrt(n * a * (1 - a))
            assert abs(k - n * a) < 5 * sd


def test_star_notification_by_hand():
    L = 8
    g = star_graph(L)
    n = g["n"]
    s = oracle.Sim(g, den_params(), np.zeros(n, np.uint8))
    st = s.state
    st.stage[0], st.timer[0], st.tinf[0] = MILD, 9, 4
    st.flags[0] |= FL_POS
    st.qt[0] = qt(0, 1)              # its positive result lands on step 0
    st.stage[1], st.timer[1], st.tinf[1] = ASYM, 9, 2   # infected leaf
    st.stage[2], st.timer[2], st.tinf[2] = ASYM, 9, 2   # infected leaf
    st.flags[3] &= 0xFF ^ FL_APP         # no app
    st.qt[4] = qt(5, 0)               # in quarantine
    st.stage[5], st.timer[5] = HOSP, 9  # in hospital
    d = s.step()
    notified = {1, 2, 6, 7, 8}
    assert d["den_notified"] == len(notified)
    assert {j for j in range(n) if st.flags[j] & FL_DEN} == notified
    assert st.qt[0] & 0x0F == 14      # the centre is in quarantine
    d = s.step()                      # step 1: the notified take a test (result after 2 steps)
    assert all((st.qt[j] >> 4) & 7 == 2 for j in notified)
    assert not any(st.flags[j] & FL_DEN for j in range(n))
    assert {j for j in range(n) if st.flags[j] & FL_POS} == {1, 2}
    s.step()
    d = s.step()                      # step 3: results land, the two infected leaves are quarantined
    assert st.qt[1] & 0x0F == 14 and st.qt[2] & 0x0F == 14
    # they notify whoever they had in-edges to: nobody (leaves have no out-edges)
    assert d["den_notified"] == 0
    assert all(st.qt[j] & 0x0F == 0 for j in (6, 7, 8))


def test_in_edge_direction_only():
    """Only agents the positive agent had an in-edge to (possible infectees) are
    notified: a centre whose in-edges come from the leaves notifies nobody."""
    L = 5
    n = L + 1
    rp = np.zeros(n + 1, np.uint32)
    rp[1:] = L                          # row 0 lists every leaf, leaf rows empty
    col = np.arange(1, n, dtype=np.uint32)
    s = oracle.Sim(dict(n=n, row_ptr=[rp], col=[col]), den_params(), np.zeros(n, np.uint8))
    st = s.state
    st.stage[0], st.timer[0], st.tinf[0] = MILD, 9, 4
    st.flags[0] |= FL_POS
    st.qt[0] = qt(0, 1)
    assert s.step()["den_notified"] == 0


@pytest.mark.parametrize("window", [7, 1, 3])
def test_look_back_window_over_random_contacts(window):
    n, t_pos, mean = 400, 9, 2.0
    g = dict(n=n, row_ptr=[], col=[])
    p = den_params(rand_mean=mean, den_window=window, net_seed=21, seed=5)
    s = oracle.Sim(g, p, np.zeros(n, np.uint8))
    for _ in range(t_pos):
        s.step(diag=False)
    st = s.state
    src = 17
    st.stage[src], st.timer[src], st.tinf[src] = MILD, 9, 4
    st.flags[src] |= FL_POS
    st.qt[src] = qt(0, 1)
    st.qt[3] = qt(6, 0)                 # one agent in quarantine
    d = s.step()
    want = set()
    for j in range(n):
        if j in (src, 3):
            continue
        for day in range(max(0, t_pos - window + 1), t_pos + 1):
            if src in oracle.random_contacts(p["net_seed"], n, j, day, float(np.float32(mean))).tolist():
                want.add(j)
    got = {j for j in range(n) if st.flags[j] & FL_DEN}
    assert got == want and d["den_notified"] == len(want)
    assert len(want) >= window  # about 2 * window on average


@pytest.mark.parametrize("window", [7, 2])
def test_look_back_window_over_the_watts_strogatz_graphs(window):
    """With the global random network as a daily Watts-Strogatz graph (edges
    undirected: an agent's in-contacts are its neighbours), the notified set is
    exactly the app holders that were the positive agent's neighbour in the graph
    of one of the last den_window steps (each step's graph listed by the oracle's
    own neighbour lists)."""
    n, t_pos = 500, 8
    g = dict(n=n, row_ptr=[], col=[], rand_ws=1, rand_ws_k=4, rand_ws_beta=0.5)
    p = den_params(den_window=window, net_seed=23, seed=6)
    s = oracle.Sim(g, p, np.zeros(n, np.uint8))
    for _ in range(t_pos):
        s.step(diag=False)
    st = s.state
    src = 41
    st.stage[src], st.timer[src], st.tinf[src] = MILD, 9, 4
    st.flags[src] |= FL_POS
    st.qt[src] = qt(0, 1)
    st.qt[7] = qt(5, 0)                 # one agent in quarantine
    d = s.step()
    want = set()
    for day in range(max(0, t_pos - window + 1), t_pos + 1):
        start, nb = s.model.ws_neighbours(day)
        for j in range(n):
            if j not in (src, 7) and src in nb[start[j]:start[j + 1]].tolist():
                want.add(j)
    got = {j for j in range(n) if st.flags[j] & FL_DEN}
    assert got == want and d["den_notified"] == len(want)
    assert len(want) >= 4


def test_compliance_share():
    L = 4000
    g = star_graph(L)
    n = g["n"]
    c = 0.8
    s = oracle.Sim(g, den_params(den_compliance=c, seed=3), np.zeros(n, np.uint8))
    st = s.state
    st.stage[0], st.timer[0], st.tinf[0] = MILD, 9, 4
    st.flags[0] |= FL_POS
    st.qt[0] = qt(0, 1)
    d = s.step()
    assert d["den_notified"] == L
    k = int((st.flags[1:] & FL_DEN).astype(bool).sum())
    assert abs(k - c * L) < 5 * np.sqrt(L * c * (1 - c))


def test_needs_testing():
    with pytest.raises(ValueError):
        oracle.Sim(dict(n=3, row_ptr=[], col=[]), den_params(test_on=0), np.zeros(3, np.uint8)).step()
