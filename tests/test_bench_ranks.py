"""The multi-GPU path of bench.py: one independent volume per rank (weak
scaling, no collective on the data path), the job time is the slowest
rank's, throughput counts every rank's work.  Run as two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(1.0 + rank, dist, "cpu")             # rank 1 is the slow one
    v = bench.throughput(world, 5, 1000, t)
    prob = bench.make_problem("potts3d", bench.rank_seed(rank), shape=(8, 12, 16))
    digest = float(np.asarray(prob.D, dtype=np.float64).sum())
    dist.barrier()
    out.put((rank, t, v, digest))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_independent_volumes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, d0), (r1, t1, v1, d1) = res
    assert t0 == t1 == 2.0                      # both see the slowest rank's time
    assert v0 == v1 == 2 * 5 * 1000 / 2.0       # whole-job units over that time
    assert d0 != d1                             # each rank has its own volume


def test_single_rank_helpers():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.throughput(1, 4, 10, 2.0) == 20.0
    assert bench.rank_seed(0) != bench.rank_seed(1)


def test_algorithmic_bytes_match_the_per_update_counts():
    """The roofline denominators bench.py reports: the fused schedule reads
    u, D, q and writes u, q once per iteration (d and the normaliser stay on
    chip), S once per voxel; the in-place schedule reads u and q twice.  Per
    voxel: Potts 8 labels FP32 8 * 36 + 4 = 292 B (BF16 storage 8 * 20 + 4),
    in place 8 * 52 + 4; HMF 12 end-labels / 15 flow nodes with per-node
    capacities 504 B; Ishikawa 8 labels / 7 flow-carrying levels 264 B; 2-D
    Potts 4 labels 4 * 28 B + 4."""
    import numpy as np
    import bench
    import synth
    cases = [
        (synth.potts3d_problem(seed=1, nl=8, shape=(4, 5, 6)), 0, 0, 8 * 36 + 4),
        (synth.potts3d_problem(seed=1, nl=8, shape=(4, 5, 6)), 1, 0, 8 * 20 + 4),
        (synth.potts3d_problem(seed=1, nl=8, shape=(4, 5, 6)), 0, 1, 8 * 52 + 4),
        (synth.hmf_problem(seed=1, shape=(4, 5, 6)), 0, 0, 504),
        (synth.ishikawa_problem(1, (4, 5, 6), nlev=7), 0, 0, 264),
        (synth.potts2d_problem(seed=1), 0, 0, 4 * 28 + 4),
    ]
    for prob, storage, schedule, per_voxel in cases:
        n = int(np.prod(prob.spatial))
        got = bench.algorithmic_bytes_per_iter(prob, storage, schedule)
        assert got == n * per_voxel, (prob.name, storage, schedule, got / n, per_voxel)
