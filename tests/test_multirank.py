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


def _shard_main(rank, world, port, out):
    """One rank of a q-sharded problem: the oracle's partial ERI over this rank's q shard, then the FP64
    sum over ranks (the only exchange step)."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    import oracle
    import synth
    from oracle import mesh as omesh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        spec = synth.LatticeSpec((4, 3, 1), 3, 5, 5, 2, 0.6, 0.0, 77, "shard")
        L, Cs, _ = synth.make_problem(spec)
        lo, hi = bench.shard_ranges(spec.mesh, spec.n_ao, [spec.n_emb] * 2, world)[rank]
        lq = [oracle.embedded_3idx(L, C, spec.mesh) for C in Cs]
        nk = spec.nk
        parts = []
        for a, b in ((0, 0), (0, 1), (1, 1)):
            eri = np.zeros((5, 5, 5, 5), dtype=np.complex128)
            for q in range(nk):
                if lo <= min(q, omesh.k_neg(q, spec.mesh)) < hi:
                    eri += np.tensordot(lq[a][q], lq[b][omesh.k_neg(q, spec.mesh)], axes=([0], [0])) / nk
            parts.append(torch.from_numpy(np.ascontiguousarray(eri.real)))
        bench.sum_over_ranks(dist, parts)
        out.put((rank, (lo, hi), [p.numpy() for p in parts]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_q_shards_sum_to_the_full_eri():
    """Strong scaling of one problem: each rank contracts its q shard; the FP64 sum of the two partial
    ERIs (all_reduce SUM) equals the full ERI of the oracle on every rank."""
    import torch.multiprocessing as mp
    import oracle
    import synth
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = synth.LatticeSpec((4, 3, 1), 3, 5, 5, 2, 0.6, 0.0, 77, "shard")
    L, Cs, _ = synth.make_problem(spec)
    full = [oracle.embedded_eri(L, Cs[a], spec.mesh, Cb=Cs[b]).real for a, b in ((0, 0), (0, 1), (1, 1))]
    (r0, s0, p0), (r1, s1, p1) = res
    assert s0[0] == 0 and s0[1] == s1[0] and s1[1] == spec.nk and s0[0] < s0[1] < s1[1]
    for a, b, f in zip(p0, p1, full):
        assert np.array_equal(a, b)                      # every rank holds the sum
        assert np.abs(a - f).max() < 1e-13 * np.abs(f).max()


@pytest.mark.parametrize("mesh", [(4, 4, 4), (6, 6, 1), (3, 3, 1), (2, 2, 1)])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_cover_the_mesh(mesh, world):
    import bench
    r = bench.shard_ranges(mesh, 104, [300, 300], world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == int(np.prod(mesh))
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
