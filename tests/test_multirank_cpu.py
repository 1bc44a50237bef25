"""The N > 1 path of bench.py on CPU: two gloo ranks, each running its own
population (rank-seeded inputs) on the oracle, then the whole-job reduction
(max of times, sum of work).  The simulation path has no collective: each
rank's result must equal that population run alone."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small():
    from paper_2110_04421_gb300 import workloads as W
    w = W.plain_small()
    return dict(w, n=1500, T=6, n_seed=15)


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _small()
    params, pop = bench.rank_inputs(w, rank)
    sim = oracle.Sim(pop, params, pop["age"], pop["seed_ids"])
    new_inf, _, msgs = sim.run(w["T"])
    fake_ms = 10.0 * (rank + 1)
    mx, sm = bench.reduce_over_ranks(dist, [fake_ms], [int(msgs.sum()), int(new_inf.sum())], "cpu")
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([mx[0], sm[0], sm[1], msgs.sum(), new_inf.sum()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    r = [np.load(tmp_path / f"rank{q}.npy") for q in range(world)]
    w = _small()
    alone = []
    for q in range(world):
        params, pop = bench.rank_inputs(w, q)
        ni, _, m = oracle.Sim(pop, params, pop["age"], pop["seed_ids"]).run(w["T"])
        alone.append((int(m.sum()), int(ni.sum())))
        assert r[q][3] == alone[q][0] and r[q][4] == alone[q][1]   # no exchange changed a rank's result
    assert alone[0] != alone[1]                                     # the ranks ran different problems
    for q in range(world):
        assert r[q][0] == 20.0                                      # max of the ranks' times
        assert r[q][1] == sum(a[0] for a in alone) and r[q][2] == sum(a[1] for a in alone)


def _columns(B):
    from paper_2110_04421_gb300 import workloads as W
    w = W.batched()
    pop = W.population(1200, 3, 12)
    rp, seeds = W.batch_params(B, 4)
    params = []
    for r in range(B):
        params.append(dict(w["params"], R=float(rp[r, 0]), B_net=[float(rp[r, 1]), float(rp[r, 2])],
                           B_rand=float(rp[r, 3]), S_age=[float(x) for x in rp[r, 4:13]],
                           dose2_delay=int(rp[r, 13]), seed=int(seeds[r]), vax_start=2, vax_rate=0.05))
    return pop, params


def _column_rank_main(rank, world, port, out_dir, B, T):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pop, params = _columns(B)
    lo, hi = bench.column_range(B, rank, world)
    local = np.zeros((T, hi - lo), np.int64)
    for c in range(lo, hi):   # this rank's columns only
        ni, _, _ = oracle.Sim(pop, params[c], pop["age"], pop["seed_ids"]).run(T)
        local[:, c - lo] = ni
    full = bench.gather_columns(dist, local, B, world, "cpu")
    np.save(os.path.join(out_dir, f"cols{rank}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("B", [7, 8])
def test_ensemble_columns_split_over_two_gloo_ranks(tmp_path, B):
    """The batched ensemble's columns split over two ranks (uneven for B = 7):
    each rank runs its own columns, the gathered [T, B] incidence equals the
    unsplit run on every rank."""
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    T, world, port = 8, 2, _free_port()
    assert [bench.column_range(B, q, world) for q in range(world)] == ([(0, 4), (4, 7)] if B == 7 else [(0, 4), (4, 8)])
    mp.start_processes(_column_rank_main, args=(world, port, str(tmp_path), B, T), nprocs=world, start_method="spawn")
    pop, params = _columns(B)
    want = np.stack([oracle.Sim(pop, params[c], pop["age"], pop["seed_ids"]).run(T)[0] for c in range(B)], axis=1)
    assert want.sum() > 0 and len({tuple(want[:, c]) for c in range(B)}) > 1
    for q in range(world):
        assert np.array_equal(np.load(tmp_path / f"cols{q}.npy"), want)
