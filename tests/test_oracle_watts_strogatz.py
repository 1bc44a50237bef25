"""Pins for the Watts-Strogatz occupation contacts (Sec. 3, Interaction
Networks: small-world networks re-parameterised every step; Watts and Strogatz,
Nature 393, 1998).

* no rewiring: every member's in-contacts are its ring-lattice neighbours
  q+1, q-1, q+2, q-2, ... in that order, the relation is symmetric, and the
  clustering coefficient of the lattice is the textbook 3(k-2) / (4(k-1));
* full rewiring: contacts uniform over the other members (chi-square);
* partial rewiring: the share of contacts off the lattice is
  beta (1 - 1/(S-1)) within a binomial band;
* a ring smaller than the lattice never yields the member itself.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2110_04421_gb300 import workloads as W


def ws_model(S, k, beta, n_other=0, seed=3):
    """One occupation of S members whose ids interleave with n_other agents of a
    second occupation, so that places differ from ids."""
    n = S + n_other
    group = np.ones(n, np.uint32)
    members = np.sort(np.random.default_rng(seed).choice(n, size=S, replace=False))
    group[members] = 0
    g = dict(n=n, row_ptr=[], col=[], occ_group=group, occ_k=np.array([k, 2], np.uint8), occ_lattice=1,
             occ_rewire=beta)
    return oracle.Model(g, W.params_with(net_seed=17)), members


def lattice(S, k, q):
    out = []
    for e in range(k):
        m = e // 2 + 1
        out.append((q + m) % S if e % 2 == 0 else (q - m) % S)
    return out


def test_no_rewiring_is_the_ring_lattice():
    S, k = 50, 6
    m, members = ws_model(S, k, 0.0, n_other=37)
    for day in (0, 5):
        for q in range(S):
            got = m.occ_contacts(int(members[q]), day).tolist()
            assert got == [int(members[p]) for p in lattice(S, k, q)]


def test_lattice_clustering_coefficient():
    S, k = 200, 10
    m, members = ws_model(S, k, 0.0)
    place = {int(v): i for i, v in enumerate(members)}
    nb = [set() for _ in range(S)]
    for q in range(S):
        for v in m.occ_contacts(int(members[q]), 0).tolist():
            nb[q].add(place[v])
    for q in range(S):
        for p in nb[q]:
            assert q in nb[p]  # undirected
    cc = []
    for q in range(S):
        links = sum(1 for a, b in itertools.combinations(sorted(nb[q]), 2) if b in nb[a])
        cc.append(links / (k * (k - 1) / 2))
    assert np.allclose(cc, 3 * (k - 2) / (4 * (k - 1)))


def test_full_rewiring_is_uniform():
    S, k = 40, 8
    m, members = ws_model(S, k, 1.0, n_other=10)
    j = int(members[7])
    counts = dict.fromkeys((int(v) for v in members if v != j), 0)
    for day in range(600):
        for v in m.occ_contacts(j, day).tolist():
            counts[v] += 1
    obs = np.array(list(counts.values()), float)
    chi2 = ((obs - obs.mean()) ** 2 / obs.mean()).sum()
    assert stats.chi2.sf(chi2, obs.size - 1) > 1e-3


@pytest.mark.parametrize("beta", [0.05, 0.3])
def test_rewired_share(beta):
    S, k = 500, 10
    m, members = ws_model(S, k, beta)
    off, total = 0, 0
    for day in range(3):
        for q in range(0, S, 2):
            got = m.occ_contacts(int(members[q]), day).tolist()
            lat = [int(members[p]) for p in lattice(S, k, q)]
            off += sum(a != b for a, b in zip(got, lat))
            total += k
    p = float(np.float32(beta)) * (1 - 1 / (S - 1))
    assert abs(off - total * p) < 5 * np.sqrt(total * p * (1 - p))


def test_ring_smaller_than_lattice():
    S, k = 3, 8
    m, members = ws_model(S, k, 0.0, n_other=5)
    for day in range(50):
        for q in range(S):
            j = int(members[q])
            got = m.occ_contacts(j, day).tolist()
            assert len(got) == k and j not in got and all(v in members for v in got)


def test_runs_and_rejects_bad_rewiring():
    pop = W.population(800, 2, 10)
    group, k = W.workplaces(800, 2)
    g = dict(pop, row_ptr=pop["row_ptr"][:1], col=pop["col"][:1], occ_group=group, occ_k=k, occ_lattice=1,
             occ_rewire=0.1)
    ni, _, _ = oracle.Sim(g, W.params_with(R=5.0), pop["age"], pop["seed_ids"]).run(20)
    assert ni.sum() > 20
    with pytest.raises(ValueError):
        oracle.Sim(dict(g, occ_rewire=1.5), W.params_with(), pop["age"], pop["seed_ids"]).step()
