"""The N > 1 path on the host: two gloo ranks on 127.0.0.1 (world size 2).

Replicas only (trajectories are independent, Secs. I and V): each rank runs
its own trajectory ranges of the same seed (here with the oracle, on the
CPU), the ranks exchange only their sufficient statistics at the end and the
slowest rank's time.  Checked: the ranges of all ranks and steps are disjoint
and cover every counter once; the merged estimate (the library's host-side
merge of the gathered statistics) equals the single-process estimate over
all counters; the MAX all-reduce gives the slowest rank's time.
"""
import math
import socket

import numpy as np
import pytest

from paper_1710_03757_gb300 import build, replicas

SEED, L, CHI, BETA = 0x51AB, 4, 2, 0.44
B, STEPS, WORLD = 40, 2, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()       # the children only load the library


def _estimate(results):
    from paper_1710_03757_gb300 import mctrg
    sign = np.array([r[0] for r in results], dtype=np.float64)
    lnabs = np.array([r[1] for r in results])
    flags = np.array([r[2] for r in results])
    m = float(np.max(lnabs))
    x = sign * np.exp(lnabs - m)
    e = mctrg.Estimate()
    e.n, e.ln_scale, e.sum_x = len(x), m, float(np.sum(x))
    e.m2_x = float(np.sum((x - x.mean()) ** 2))
    e.n_negative, e.n_flagged = int(np.sum(sign < 0)), int(np.sum(flags != 0))
    return e


def _rank(rank, port, q):
    import os
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from oracle import ising
        from oracle.trg import Problem, run_trajectory
        from paper_1710_03757_gb300 import mctrg
        prob = Problem(ising.site_tensor(BETA, 0.0), L, CHI)
        ests, counters = [], []
        for step in range(STEPS):
            f0 = replicas.first_trajectory(step, rank, WORLD, B)
            ests.append(_estimate([run_trajectory(prob, SEED, t) for t in range(f0, f0 + B)]))
            counters.extend(range(f0, f0 + B))
        all_ests = replicas.gather_estimates(dist, ests)
        took = torch.tensor([0.5 + rank], dtype=torch.float64)      # a rank's "time"
        dist.all_reduce(took, op=dist.ReduceOp.MAX)
        c = torch.tensor(counters, dtype=torch.int64)
        parts = [torch.empty_like(c) for _ in range(WORLD)]
        dist.all_gather(parts, c)
        if rank == 0:
            merged = mctrg.mctrg_merge_estimates(all_ests)
            q.put((merged.ln_mean_Z, merged.se_ln_Z, int(merged.n), int(merged.n_negative),
                   float(took[0]), sorted(torch.cat(parts).tolist()), len(all_ests)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_first_trajectory_partitions_the_counters():
    for world in (1, 2, 3, 8):
        seen = []
        for step in range(4):
            for rank in range(world):
                f0 = replicas.first_trajectory(step, rank, world, 5)
                seen.extend(range(f0, f0 + 5))
        assert sorted(seen) == list(range(4 * world * 5))


def test_pack_roundtrip():
    from paper_1710_03757_gb300 import mctrg
    e = mctrg.Estimate()
    e.n, e.ln_scale, e.sum_x, e.m2_x, e.n_negative, e.n_flagged = 123, -4.5, 17.25, 3.5, 7, 2
    (f,) = replicas.unpack(replicas.pack([e]))
    assert (f.n, f.ln_scale, f.sum_x, f.m2_x, f.n_negative, f.n_flagged) == (123, -4.5, 17.25, 3.5, 7, 2)


def test_two_gloo_ranks_merge_to_the_single_process_estimate():
    import torch.multiprocessing as tmp
    from oracle import ising
    from oracle.estimator import estimate
    from oracle.trg import Problem, run_many
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    tmp.start_processes(_rank, args=(_free_port(), q), nprocs=WORLD, join=True, start_method="spawn")
    ln_mean, se_ln, n, n_neg, took, counters, n_ests = q.get(timeout=60)
    total = WORLD * STEPS * B
    assert counters == list(range(total)) and n == total and n_ests == WORLD * STEPS
    assert took == 0.5 + (WORLD - 1)
    sign, lnabs, _ = run_many(Problem(ising.site_tensor(BETA, 0.0), L, CHI), SEED, 0, total)
    ref = estimate(sign, lnabs)
    assert ln_mean == pytest.approx(ref["ln_mean_Z"], rel=1e-13)
    assert se_ln == pytest.approx(ref["se_ln_Z"], rel=1e-9)
    assert n_neg == ref["n_negative"] and math.isfinite(ln_mean)
