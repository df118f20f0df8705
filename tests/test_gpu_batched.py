"""Batched execution: one plan over problems of uneven sizes and both precisions, run
concurrently (own workspaces) or one after another (shared workspace), and replayed from a
CUDA graph; every problem must match its own single-problem result and the oracle."""
import numpy as np
import pytest

import oracle
import synth
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


def _problems(n=6, seed=77):
    specs = synth.batch_specs(n, seed=seed, n_ao_range=(4, 7), n_emb_range=(6, 20))
    probs = []
    for i, sp in enumerate(specs):
        L, Cs, _ = synth.make_problem(sp)
        prec = B.DMET_PREC_BF16X3 if i % 3 == 2 else B.DMET_PREC_FP64
        desc = B.make_desc(sp.mesh, sp.n_ao, sp.n_aux, sp.n_emb, n_spin=sp.n_spin, prec=prec)
        probs.append((sp, L, Cs, desc))
    return probs


def _run(torch, probs, workspace_limit=0, graph=False, calls=1, profile=False):
    Ls = [torch.from_numpy(L).cuda() for _, L, _, _ in probs]
    Cs = [[torch.from_numpy(c).cuda() for c in C] for _, _, C, _ in probs]
    outs = [[torch.full((B.dmet_emb_eri_bytes(d, b) // 8,), float("nan"), dtype=torch.float64, device="cuda")
             for b in range(1 if d.n_spin == 1 else 3)] for _, _, _, d in probs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = dm.dmet_emb_plan([d for *_, d in probs], stream=stream.cuda_stream, workspace_limit=workspace_limit)
        try:
            dm.dmet_emb_graph(plan, graph)
            dm.dmet_emb_profile(plan, profile)
            for _ in range(calls):
                dm.dmet_emb_eri(plan, Ls, Cs, outs)
            stream.synchronize()
            statuses = [dm.dmet_emb_status(plan, p)[0] for p in range(len(probs))]
            times = [dm.dmet_emb_problem_ms(plan, p) for p in range(len(probs))] if profile else None
            launches = dm.dmet_emb_launch_count(plan)
        finally:
            dm.dmet_emb_destroy(plan)
    return [[o.cpu().numpy() for o in row] for row in outs], statuses, times, launches


def _reference(sp, L, Cs, desc):
    tol = 1e-10 if desc.prec == B.DMET_PREC_FP64 else 1e-6
    blocks = [oracle.pack_s8(oracle.embedded_eri(L, Cs[0], sp.mesh).real)]
    if sp.n_spin == 2:
        blocks.append(oracle.pair_matrix(oracle.embedded_eri(L, Cs[0], sp.mesh, Cb=Cs[1]).real).ravel())
        blocks.append(oracle.pack_s8(oracle.embedded_eri(L, Cs[1], sp.mesh).real))
    return blocks, tol


def test_batched_concurrent_matches_oracle():
    torch = torch_cuda()
    probs = _problems()
    res, st, times, _ = _run(torch, probs, profile=True)
    assert all(s == B.DMET_OK for s in st)
    assert all(t > 0 for t in times)
    for (sp, L, Cs, d), got in zip(probs, res):
        refs, tol = _reference(sp, L, Cs, d)
        for g, r in zip(got, refs):
            assert rel_fro(g, r) < tol


def test_batched_shared_workspace_same_result():
    torch = torch_cuda()
    probs = _problems(seed=78)
    a, _, _, _ = _run(torch, probs)
    b, _, _, _ = _run(torch, probs, workspace_limit=1 << 26)  # too small for all: problems run in turn
    # The smaller limit can also change a problem's q-block size: FP64 sums then run in another order
    # (1e-12), and a tensor-core problem's last-wave K split may change, which can move its FP32 result
    # rounding by one unit in the last place (2^-24 relative).
    for (_, _, _, d), ra, rb in zip(probs, a, b):
        for x, y in zip(ra, rb):
            if d.prec == B.DMET_PREC_FP64:
                assert rel_fro(y, x) < 1e-12
            else:
                assert np.abs(x - y).max() <= 2.0 ** -22 * np.abs(x).max()


def test_graph_replay_same_result():
    torch = torch_cuda()
    probs = _problems(seed=79)
    a, _, _, l1 = _run(torch, probs)
    b, st, _, l3 = _run(torch, probs, graph=True, calls=3)
    assert all(s == B.DMET_OK for s in st)
    assert l3 == 3 * l1  # every replay counts the captured launches
    for ra, rb in zip(a, b):
        for x, y in zip(ra, rb):
            assert rel_fro(y, x) < 1e-12
