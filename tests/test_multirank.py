"""The multi-rank (weak-scaling) path of bench.py on CPU: two gloo ranks, each with its own problem.

Every GPU run of this project has one GPU, so the N > 1 launch of bench.py (torchrun, one rank per GPU,
NCCL) is covered here on the host: each rank gets a different problem of the same shape, the only
collective is the MAX all-reduce of the timing, and the reported value counts every rank's problems.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        spec = bench.rank_spec(synth.CONFIGS["tiny_2x2x1"], rank)
        L, Cs, _ = synth.make_problem(spec)
        eri = oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real)
        ms = 10.0 * (rank + 1)  # the ranks finish at different times
        ms_job = bench.max_over_ranks(dist, ms, "cpu")
        digest = torch.tensor([float(np.abs(eri).sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, digest)  # (test only: compare what the ranks computed)
        out.put((rank, spec.seed, ms_job, bench.job_tflops(world, 1e9, 3, ms_job), [float(g) for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seed0, ms0, v0, g0), (r1, seed1, ms1, v1, g1) = res
    assert (r0, r1) == (0, 1)
    assert seed0 != seed1                      # each rank has its own problem
    assert g0 == g1 and g0[0] != g0[1]         # ... and they differ
    assert ms0 == ms1 == 20.0                  # the job time is the slowest rank's
    assert v0 == v1 == pytest.approx(2 * 1e9 * 3 / 0.020 / 1e12)  # both ranks' work over that time
