"""Pins for the daily occupation networks (Sec. 3, Interaction Networks: an
agent's occupation is fixed, but whom it meets there is drawn anew every step).

* law: each in-contact is uniform over the other members of the agent's
  occupation (chi-square), never the agent itself, never outside its
  occupation; a member meets exactly its occupation's daily count, a lone
  member nobody.
* reduction: when every occupation has exactly two members, the daily draw has
  one possible outcome (the partner, k times), so whole runs must equal, bit for
  bit, runs whose occupation network is the stored CSR listing the partner k
  times, with and without a household network in front of it.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2110_04421_gb300 import workloads as W


def graph_with_occ(pop, group, k, keep_static):
    g = dict(n=pop["n"], row_ptr=pop["row_ptr"][:keep_static], col=pop["col"][:keep_static])
    g["occ_group"], g["occ_k"] = group, k
    return g


def test_contacts_uniform_over_other_members():
    n = 240
    group = (np.arange(n) % 3).astype(np.uint32)  # three occupations of 80, interleaved ids
    k = np.array([7, 12, 15], np.uint8)
    p = W.params_with(net_seed=11)
    m = oracle.Model(dict(n=n, row_ptr=[], col=[], occ_group=group, occ_k=k), p)
    for j in (0, 4, 239):
        g = group[j]
        members = np.flatnonzero(group == g)
        others = members[members != j]
        counts = dict.fromkeys(others.tolist(), 0)
        for day in range(400):
            c = m.occ_contacts(j, day)
            assert c.size == k[g]
            for v in c.tolist():
                assert v != j and group[v] == g
                counts[v] += 1
        obs = np.array(list(counts.values()), float)
        chi2 = ((obs - obs.mean()) ** 2 / obs.mean()).sum()
        assert stats.chi2.sf(chi2, obs.size - 1) > 1e-3


def test_lone_member_meets_nobody():
    n = 50
    group = np.zeros(n, np.uint32)
    group[17] = 1  # alone in occupation 1
    m = oracle.Model(dict(n=n, row_ptr=[], col=[], occ_group=group, occ_k=np.array([9, 9], np.uint8)),
                     W.params_with())
    assert m.occ_contacts(17, 3).size == 0
    assert m.occ_contacts(3, 3).size == 9


def test_daily_differs_between_days():
    n = 400
    group, k = W.workplaces(n, 0)
    m = oracle.Model(dict(n=n, row_ptr=[], col=[], occ_group=group, occ_k=k), W.params_with())
    assert not np.array_equal(m.occ_contacts(5, 0), m.occ_contacts(5, 1))


@pytest.mark.parametrize("keep_household", [1, 0])
def test_pairs_reduce_to_stored_network(keep_household):
    n = 3000
    pop = W.population(n, 3, 30)
    rng = np.random.default_rng(5)
    perm = rng.permutation(n)
    group = np.empty(n, np.uint32)
    group[perm] = (np.arange(n) // 2).astype(np.uint32)  # occupations of two
    n_occ = n // 2
    k = rng.integers(1, 16, size=n_occ).astype(np.uint8)
    # the stored equivalent: row j lists its partner k[group[j]] times
    partner = np.empty(n, np.uint32)
    partner[perm[0::2]] = perm[1::2]
    partner[perm[1::2]] = perm[0::2]
    kk = k[group].astype(np.int64)
    rp = np.zeros(n + 1, np.uint32)
    rp[1:] = np.cumsum(kk)
    col = np.repeat(partner, kk).astype(np.uint32)

    p = W.params_with(B_net=[2.0, 0.7] if keep_household else [0.7], R=6.0, test_on=1, quar_on=1,
                      vax_on=1, vax_start=5, vax_rate=0.02, seed=4, net_seed=8)
    daily = graph_with_occ(pop, group, k, keep_household)
    stored = dict(n=n, row_ptr=pop["row_ptr"][:keep_household] + [rp], col=pop["col"][:keep_household] + [col])
    a = oracle.Sim(daily, p, pop["age"], pop["seed_ids"])
    b = oracle.Sim(stored, p, pop["age"], pop["seed_ids"])
    for _ in range(25):
        da, db = a.step(), b.step()
        np.testing.assert_array_equal(da["lambda32"], db["lambda32"])
        assert da["messages"] == db["messages"]
        assert da["new_inf"] == db["new_inf"]
    for f in ("stage", "timer", "tinf", "flags", "qt"):
        np.testing.assert_array_equal(getattr(a.state, f), getattr(b.state, f))
    assert int(a.state.stage.astype(bool).sum()) > 100  # the epidemic took off


def test_messages_count_daily_contacts():
    n = 600
    pop = W.population(n, 1, 5)
    group, k = W.occupations(n, 1, n_occ=4)
    p = W.params_with(rand_mean=0.0)
    s = oracle.Sim(graph_with_occ(pop, group, k, 1), p, pop["age"], pop["seed_ids"])
    d = s.step()
    sizes = np.bincount(group, minlength=k.size)
    expect = int(pop["row_ptr"][0][-1]) + int(sum(int(k[g]) for g in group if sizes[g] > 1))
    assert d["messages"] == expect


def test_rejects_bad_occupations():
    n = 10
    p = W.params_with()
    with pytest.raises(ValueError):
        oracle.Sim(dict(n=n, row_ptr=[], col=[], occ_group=np.zeros(n, np.uint32),
                        occ_k=np.array([16], np.uint8)), p, np.zeros(n, np.uint8)).step()
    with pytest.raises(ValueError):
        oracle.Sim(dict(n=n, row_ptr=[], col=[], occ_group=np.full(n, 2, np.uint32),
                        occ_k=np.array([3, 3], np.uint8)), p, np.zeros(n, np.uint8)).step()
