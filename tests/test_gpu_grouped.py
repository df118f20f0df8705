"""Grouped batch execution (dmet_emb_batch_mode 1): the tensor-core GEMMs of every problem of a plan
as persistent launches over a device table of per-problem tensor maps, segment lists and output
parameters. Every problem must match the oracle (tensor-core bounds), the side-stream execution of
the same plan (the only difference is the K split of the last wave's tiles), and itself when the
batch is replayed from a captured graph."""
import numpy as np
import pytest

import oracle
import synth
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _problems(n=8, seed=91, precs=None, complex_every=0):
    specs = synth.batch_specs(n, seed=seed, n_ao_range=(4, 8), n_emb_range=(6, 24))
    probs = []
    for i, sp in enumerate(specs):
        prec = precs[i % len(precs)] if precs else B.DMET_PREC_BF16X3
        if complex_every and i % complex_every == 1:
            L = synth.make_L(sp)
            Cs = [synth.bloch_orbitals(synth.complex_supercell_orbitals(sp, s), sp.mesh) for s in range(sp.n_spin)]
            ne = [sp.n_emb, sp.n_emb] if sp.n_spin == 2 else sp.n_emb
            desc = B.make_desc(sp.mesh, sp.n_ao, sp.n_aux, ne, n_spin=sp.n_spin, prec=prec, sym=B.DMET_SYM_NONE,
                               eri_pack=B.DMET_PACK_FULL)
        else:
            L, Cs, _ = synth.make_problem(sp)
            ne = [sp.n_emb, sp.n_emb] if sp.n_spin == 2 else sp.n_emb
            desc = B.make_desc(sp.mesh, sp.n_ao, sp.n_aux, ne, n_spin=sp.n_spin, prec=prec)
        probs.append((sp, L, Cs, desc))
    return probs


def _run(torch, probs, mode, graph=False, calls=1, autotune=False):
    Ls = [torch.from_numpy(L).cuda() for _, L, _, _ in probs]
    Cs = [[torch.from_numpy(c).cuda() for c in C] for _, _, C, _ in probs]

    def buf(d, b):
        nb = B.dmet_emb_eri_bytes(d, b)
        if d.sym == B.DMET_SYM_NONE:
            return torch.full((nb // 16,), complex("nan"), dtype=torch.complex128, device="cuda")
        return torch.full((nb // 8,), float("nan"), dtype=torch.float64, device="cuda")

    outs = [[buf(d, b) for b in range(1 if d.n_spin == 1 else 3)] for _, _, _, d in probs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = dm.dmet_emb_plan([d for *_, d in probs], stream=stream.cuda_stream)
        try:
            active = dm.dmet_emb_batch_mode(plan, mode)
            dm.dmet_emb_graph(plan, graph)
            if autotune:
                dm.dmet_emb_autotune(plan, Ls, Cs, outs)
            for _ in range(calls):
                dm.dmet_emb_eri(plan, Ls, Cs, outs)
            stream.synchronize()
            statuses = [dm.dmet_emb_status(plan, p)[0] for p in range(len(probs))]
            launches = dm.dmet_emb_launch_count(plan)
        finally:
            dm.dmet_emb_destroy(plan)
    return [[o.cpu().numpy() for o in row] for row in outs], statuses, active, launches


def _reference(sp, L, Cs, desc):
    if desc.sym == B.DMET_SYM_NONE:
        blocks = [oracle.embedded_eri(L, Cs[0], sp.mesh).ravel()]
        if sp.n_spin == 2:
            blocks.append(oracle.embedded_eri(L, Cs[0], sp.mesh, Cb=Cs[1]).ravel())
            blocks.append(oracle.embedded_eri(L, Cs[1], sp.mesh).ravel())
        return blocks
    blocks = [oracle.pack_s8(oracle.embedded_eri(L, Cs[0], sp.mesh).real)]
    if sp.n_spin == 2:
        blocks.append(oracle.pair_matrix(oracle.embedded_eri(L, Cs[0], sp.mesh, Cb=Cs[1]).real).ravel())
        blocks.append(oracle.pack_s8(oracle.embedded_eri(L, Cs[1], sp.mesh).real))
    return blocks


def _check_oracle(probs, res):
    for (sp, L, Cs, d), got in zip(probs, res):
        tol = 1e-6 if d.prec == B.DMET_PREC_BF16X3 else 5e-6
        for g, r in zip(got, _reference(sp, L, Cs, d)):
            assert np.isfinite(g).all()
            e = rel_fro(g, r)
            m = np.abs(g - r).max() / np.abs(r).max()
            assert e < tol and m < tol, (d.prec, e, m)


def test_grouped_matches_oracle_and_side_streams(torch):
    probs = _problems(precs=[B.DMET_PREC_BF16X3, B.DMET_PREC_BF16X3, B.DMET_PREC_FP16X2])
    g, st, active, _ = _run(torch, probs, 1)
    assert active
    assert all(s == B.DMET_OK for s in st)
    _check_oracle(probs, g)
    s_, st2, active2, _ = _run(torch, probs, 0)
    assert not active2 and all(s == B.DMET_OK for s in st2)
    # The side-stream run splits the last wave's tiles in K; the two groupings of the same segment
    # sums may round the FP32 result differently (one unit in the last place, 2^-24 relative).
    for ra, rb in zip(g, s_):
        for x, y in zip(ra, rb):
            assert np.abs(x - y).max() <= 2.0 ** -22 * np.abs(y).max()
            assert rel_fro(x, y) < 1e-7


def test_grouped_graph_replay_is_exact(torch):
    probs = _problems(seed=92)
    a, _, _, l1 = _run(torch, probs, 1)
    b, st, active, l3 = _run(torch, probs, 1, graph=True, calls=3)
    assert active and all(s == B.DMET_OK for s in st)
    assert l3 == 3 * l1
    for ra, rb in zip(a, b):
        for x, y in zip(ra, rb):
            assert np.array_equal(x, y)


def test_grouped_with_complex_orbitals(torch):
    probs = _problems(n=6, seed=93, complex_every=2)
    assert any(d.sym == B.DMET_SYM_NONE for *_, d in probs)
    g, st, active, _ = _run(torch, probs, 1)
    assert active and all(s == B.DMET_OK for s in st)
    _check_oracle(probs, g)


def test_grouped_after_autotune(torch):
    probs = _problems(n=5, seed=94)
    g, st, active, _ = _run(torch, probs, 1, autotune=True)
    assert active and all(s == B.DMET_OK for s in st)
    _check_oracle(probs, g)


def test_grouped_needs_tensor_core_problems(torch):
    probs = _problems(n=3, seed=95, precs=[B.DMET_PREC_BF16X3, B.DMET_PREC_FP64])
    _, st, active, _ = _run(torch, probs, 1)
    assert not active and all(s == B.DMET_OK for s in st)


def test_grouped_medium_problems(torch):
    """Grouped launches over problems of a few thousand pairs (several tile rows per block, uneven
    rounds), unrestricted and restricted: every block within the FP32 output rounding of the
    side-stream run, and one problem's 12-orbital subset against the oracle."""
    specs = [synth.LatticeSpec((2, 2, 2), 18, 150, 96, 2, 0.6, 0.0, 501, "g0"),
             synth.LatticeSpec((3, 3, 1), 22, 180, 130, 1, 0.6, 0.0, 502, "g1"),
             synth.LatticeSpec((2, 2, 1), 26, 220, 70, 1, 0.6, 0.0, 503, "g2")]
    probs = []
    for sp in specs:
        L, Cs, _ = synth.make_problem(sp)
        ne = [sp.n_emb, sp.n_emb] if sp.n_spin == 2 else sp.n_emb
        probs.append((sp, L, Cs, B.make_desc(sp.mesh, sp.n_ao, sp.n_aux, ne, n_spin=sp.n_spin,
                                             prec=B.DMET_PREC_BF16X3)))
    g, st, active, _ = _run(torch, probs, 1)
    assert active and all(s == B.DMET_OK for s in st)
    s_, st2, _, _ = _run(torch, probs, 0)
    assert all(s == B.DMET_OK for s in st2)
    for ra, rb in zip(g, s_):
        for x, y in zip(ra, rb):
            assert np.isfinite(x).all()
            assert np.abs(x - y).max() <= 2.0 ** -22 * np.abs(y).max()
    sp, L, Cs, _ = probs[1]
    S = np.sort(np.random.default_rng(3).choice(sp.n_emb, 12, replace=False))
    ref = oracle.embedded_eri(L, np.ascontiguousarray(Cs[0][:, :, S]), sp.mesh).real
    i, j, k, l = np.meshgrid(*([S] * 4), indexing="ij")
    from gpu_helpers import s8_index
    got = g[1][0][s8_index(i, j, k, l)]
    e = rel_fro(got, ref)
    assert e < 1e-6, e
