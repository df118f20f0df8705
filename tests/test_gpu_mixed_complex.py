"""GPU parity of the tensor-core path for general (complex) embedding orbitals (sym = NONE) against
the FP64 CPU oracle of Algorithm 1: every q contracted as one real GEMM of the bra rows (Re, Im of
L^q_ij) against the ket rows of L^{-q}_kl, only the tiles with kl <= ij of a same-spin block
computed, the rest by (kl|ij) = (ij|kl); FULL and 4-fold packed (S4) outputs, restricted and
unrestricted. Tolerance: 1e-6 relative Frobenius and max-abs over max for BF16X3 (as for real
orbitals), 5e-6 for the 22-bit precisions."""
import numpy as np
import pytest

import oracle
import synth
from oracle import checks
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def run(torch, desc, L, Cs):
    import paper_1909_08596_gb300 as dm
    nblk = 1 if desc.n_spin == 1 else 3
    outs = [torch.full((dm.dmet_emb_eri_bytes(desc, b) // 16,), complex("nan"), dtype=torch.complex128, device="cuda")
            for b in range(nblk)]
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    plan = dm.dmet_emb_plan(desc, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    return [o.cpu().numpy() for o in outs]


def close(got, ref, tol=1e-6):
    got = got.reshape(ref.shape)
    assert np.isfinite(got).all()
    e = rel_fro(got, ref)
    m = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < tol and m < tol, (e, m)
    return e


def problem(mesh, nao, naux, n, seed, n_b=None):
    spec = synth.LatticeSpec(tuple(mesh), nao, naux, n, 1 if n_b is None else 2, 0.6, 0.0, seed, "mc")
    L = synth.make_L(spec)
    ca = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec, 0), spec.mesh)
    if n_b is None:
        return spec, L, [ca]
    cb = synth.bloch_orbitals(synth.complex_supercell_orbitals(synth.spec_with(spec, n_emb=n_b), 1), spec.mesh)
    return spec, L, [ca, cb]


CASES = [
    ((2, 2, 1), 4, 9, 6),
    ((3, 1, 1), 5, 7, 1),
    ((3, 2, 1), 6, 20, 9),
    ((3, 3, 1), 8, 30, 23),    # n^2 = 529: five bra tiles, nine ket tiles, the diagonal inside tiles
    ((2, 2, 2), 6, 16, 36),    # n^2 = 1296: a multiple of neither 128 nor 64
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_n{c[3]}")
def test_full_matches_oracle(torch, case):
    mesh, nao, naux, n = case
    spec, L, Cs = problem(mesh, nao, naux, n, 71)
    d = B.make_desc(mesh, nao, naux, n, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_FULL, prec=B.DMET_PREC_BF16X3)
    (got,) = run(torch, d, L, Cs)
    ref = oracle.embedded_eri(L, Cs[0], spec.mesh)
    close(got, ref)
    # the imaginary parts are not small: the orbitals are general complex ones (with one orbital,
    # (00|00) is real by the exchange symmetry)
    if n > 1:
        assert np.abs(ref.imag).max() > 1e-2 * np.abs(ref.real).max()


@pytest.mark.parametrize("ck_norm", [0, 1])
def test_s4_matches_oracle(torch, ck_norm):
    mesh, nao, naux, n = (3, 2, 1), 6, 20, 13
    spec = synth.LatticeSpec(mesh, nao, naux, n, 1, 0.6, 0.0, 72, "mc")
    L = synth.make_L(spec)
    C = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec), mesh, ck_norm=ck_norm)
    d = B.make_desc(mesh, nao, naux, n, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_S4, prec=B.DMET_PREC_BF16X3,
                    ck_norm=ck_norm)
    (got,) = run(torch, d, L, [C])
    assert len(got) == checks.s4_size(n)
    close(got, checks.pack_s4(oracle.embedded_eri(L, C, mesh, ck_norm=ck_norm)))


@pytest.mark.parametrize("pack", [B.DMET_PACK_FULL, B.DMET_PACK_S4])
def test_unrestricted_blocks(torch, pack):
    spec, L, (ca, cb) = problem((3, 2, 1), 5, 14, 11, 73, n_b=17)
    d = B.make_desc(spec.mesh, 5, 14, [11, 17], n_spin=2, sym=B.DMET_SYM_NONE, eri_pack=pack,
                    prec=B.DMET_PREC_BF16X3)
    aa, ab, bb = run(torch, d, L, [ca, cb])
    raa = oracle.embedded_eri(L, ca, spec.mesh)
    rbb = oracle.embedded_eri(L, cb, spec.mesh)
    rab = oracle.embedded_eri(L, ca, spec.mesh, Cb=cb)
    if pack == B.DMET_PACK_S4:
        raa, rbb, rab = checks.pack_s4(raa), checks.pack_s4(rbb), checks.pack_s4_ab(rab)
    close(aa, raa)
    close(bb, rbb)
    close(ab, rab)


@pytest.mark.parametrize("prec,tol", [(B.DMET_PREC_FP16X2, 5e-6), (B.DMET_PREC_TF32X3, 5e-6)])
def test_other_precisions(torch, prec, tol):
    spec, L, Cs = problem((3, 2, 1), 6, 20, 14, 74)
    d = B.make_desc(spec.mesh, 6, 20, 14, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_FULL, prec=prec)
    (got,) = run(torch, d, L, Cs)
    close(got, oracle.embedded_eri(L, Cs[0], spec.mesh), tol)


def test_transform_3idx_complex_orbitals(torch):
    import paper_1909_08596_gb300 as dm
    spec, L, Cs = problem((3, 2, 1), 6, 20, 10, 75)
    d = B.make_desc(spec.mesh, 6, 20, 10, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_FULL, prec=B.DMET_PREC_BF16X3)
    nk = spec.nk
    out = torch.empty((nk, 20, 10, 10), dtype=torch.complex128, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_transform_3idx(plan, 0, torch.from_numpy(L).cuda(), [torch.from_numpy(Cs[0]).cuda()], 0, nk, [out])
        torch.cuda.synchronize()
    finally:
        dm.dmet_emb_destroy(plan)
    ref = oracle.embedded_3idx(L, Cs[0], spec.mesh)
    assert rel_fro(out.cpu().numpy().reshape(ref.shape), ref) < 1e-6


def test_hbn_sized_complex_sampled(torch):
    """h-BN-shaped cell (6x6x1 mesh, n_ao 26, n_aux 220, n_emb 104) with general complex orbitals,
    FULL output: 4000 sampled entries against the oracle's per-q factors (relative to the largest
    sampled magnitude), and the (ij|kl) = (kl|ij) symmetry the path relies on, exactly."""
    import time
    import paper_1909_08596_gb300 as dm
    spec, L, Cs = problem((6, 6, 1), 26, 220, 104, 76)
    n = 104
    d = B.make_desc(spec.mesh, 26, 220, n, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_FULL, prec=B.DMET_PREC_BF16X3)
    out = torch.empty(n ** 4, dtype=torch.complex128, device="cuda")
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(Cs[0]).cuda()]
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    print(f"complex h-BN-shaped call: {ms:.2f} ms")
    got = out.cpu().numpy().reshape(n, n, n, n)
    assert np.isfinite(got).all()
    assert np.array_equal(got, got.transpose(2, 3, 0, 1))
    rng = np.random.default_rng(5)
    idx = rng.integers(0, n, size=(4000, 4))
    Lq = oracle.embedded_3idx(L, Cs[0], spec.mesh)
    ref = oracle.eri_entries(Lq, Lq, spec.mesh, idx)
    g = got[idx[:, 0], idx[:, 1], idx[:, 2], idx[:, 3]]
    assert np.abs(g - ref).max() < 1e-6 * np.abs(ref).max()
    assert rel_fro(g, ref) < 1e-6
