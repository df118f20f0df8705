"""GPU parity of the FP16x2, TF32x3 and TF32 tensor-core precisions against the FP64 CPU oracle,
through the C ABI (the BF16x3 precision has its own file, test_gpu_mixed.py).

Bounds (relative Frobenius and max-abs over max|(ij|kl)|):
* FP16x2 and TF32x3: 5e-6. Each operand is carried by two slices of 11 significant bits (a
  representation error up to 2^-22 = 2.4e-7 relative), the dropped slice product is up to 2^-22 of
  the leading one, and three chained products (two transforms and the contraction) each add such
  errors, amplified where the sums cancel: measured up to 1.6e-6 on the NiO-shaped workload and 1.2e-6
  max-abs on the small cases here. These two precisions do not meet the mixed path's 1e-6 bound
  (BF16x3, three 8-bit slices, carries 2^-24); they are part of the precision study.
* TF32: one slice of 11 bits per operand (2^-12 relative rounding each), one product: about 2^-11
  relative per product, compounded over three chained products (two transforms and the contraction)
  with random-sign cancellation in the sums; the bound is 3 x 2^-11 x 4 = 6e-3 (the factor 4 covers
  the cancellation measured on these problems), and the error must also exceed 1e-6 (TF32 cannot meet
  the mixed-path bound: that is what the precision study shows).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, run_eri, torch_cuda

pytestmark = pytest.mark.gpu

PRECS = {"fp16x2": (B.DMET_PREC_FP16X2, 5e-6), "tf32x3": (B.DMET_PREC_TF32X3, 5e-6),
         "tf32": (B.DMET_PREC_TF32, 3 * 2.0 ** -11 * 4)}


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def spec_of(mesh, n_ao, n_aux, n_emb, n_spin=1, seed=23, c_log_range=0.0):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, n_spin, 0.6, c_log_range, seed, "p")


def check(got, ref, name):
    tol = PRECS[name][1]
    assert np.isfinite(got).all()
    e = rel_fro(got, ref)
    m = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < tol and m < tol, (name, e, m)
    if name == "tf32":
        assert e > 1e-6, e
    return e


CASES = [
    ((2, 2, 1), 8, 40, 16),
    ((1, 1, 1), 5, 7, 3),
    ((2, 3, 1), 6, 11, 33),
    ((3, 3, 1), 10, 37, 70),
    ((3, 2, 1), 24, 60, 130),   # more than one 128-row tile of pairs and of (P, j) rows
]


@pytest.mark.parametrize("name", sorted(PRECS))
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_ao{c[1]}_aux{c[2]}_n{c[3]}")
def test_precision_matches_oracle(torch, name, case):
    mesh, nao, naux, n = case
    spec = spec_of(mesh, nao, naux, n)
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(mesh, nao, naux, n, prec=PRECS[name][0])
    (got,), st, stats = run_eri(torch, d, L, Cs)
    assert st == B.DMET_OK, (st, stats)
    check(got, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], mesh).real), name)


@pytest.mark.parametrize("name", sorted(PRECS))
def test_precision_unrestricted(torch, name):
    spec = spec_of((3, 2, 1), 5, 9, 8, n_spin=2)
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(spec.mesh, 5, 9, [8, 8], n_spin=2, prec=PRECS[name][0])
    (aa, ab, bb), st, _ = run_eri(torch, d, L, Cs)
    assert st == B.DMET_OK
    check(aa, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real), name)
    check(bb, oracle.pack_s8(oracle.embedded_eri(L, Cs[1], spec.mesh).real), name)
    check(ab, oracle.pair_matrix(oracle.embedded_eri(L, Cs[0], spec.mesh, Cb=Cs[1]).real).ravel(), name)


@pytest.mark.parametrize("name", sorted(PRECS))
def test_precision_log_uniform_orbitals(torch, name):
    """Orbital entries spread over four decades (the silicon-shaped precision study's recipe)."""
    spec = spec_of((2, 2, 2), 6, 15, 24, c_log_range=4.0)
    L, Cs, _ = synth.make_problem(spec)
    (got,), st, _ = run_eri(torch, B.make_desc(spec.mesh, 6, 15, 24, prec=PRECS[name][0]), L, Cs)
    assert st == B.DMET_OK
    check(got, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real), name)


@pytest.mark.parametrize("scale", [1e-9, 1e7])
def test_fp16_scales_follow_the_inputs(torch, scale):
    """L far from unit magnitude: the FP16 operand scales (powers of two from the inputs' maxima)
    keep every slice inside FP16's range, and the result scales with L squared."""
    spec = spec_of((3, 3, 1), 6, 11, 20)
    L, Cs, _ = synth.make_problem(spec)
    L = L * scale
    d = B.make_desc(spec.mesh, 6, 11, 20, prec=B.DMET_PREC_FP16X2)
    (got,), st, _ = run_eri(torch, d, L, Cs)
    assert st == B.DMET_OK
    check(got, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real), "fp16x2")


@pytest.mark.parametrize("name", ["fp16x2", "tf32x3"])
@pytest.mark.parametrize("layout", [B.DMET_L_FULL, B.DMET_L_REDUCED])
def test_precision_close_to_bf16x3(torch, name, layout):
    """The same problem through two precisions agrees within both bounds."""
    import paper_1909_08596_gb300 as dm
    spec = spec_of((4, 2, 1), 7, 13, 25)
    L, Cs, _ = synth.make_problem(spec)
    d0 = B.make_desc(spec.mesh, 7, 13, 25, prec=B.DMET_PREC_BF16X3)
    d1 = B.make_desc(spec.mesh, 7, 13, 25, prec=PRECS[name][0], l_layout=layout)
    Lin = synth.make_L_pairs(spec, dm.dmet_emb_l_pairs(d1)) if layout == B.DMET_L_REDUCED else L
    (a,), st0, _ = run_eri(torch, d0, L, Cs)
    (b,), st1, _ = run_eri(torch, d1, Lin, Cs)
    assert st0 == st1 == B.DMET_OK
    assert rel_fro(b, a) < 5e-6


@pytest.mark.parametrize("name", ["bf16x3", "fp16x2", "tf32x3"])
@pytest.mark.parametrize("layout", [B.DMET_L_FULL, B.DMET_L_REDUCED])
def test_precision_transform_3idx_matches_oracle(torch, name, layout):
    """dmet_emb_transform_3idx of a tensor-core plan: the half transforms of that precision (every q,
    including the q of zero contraction weight, which the reduced layout takes from -q conjugated)."""
    import paper_1909_08596_gb300 as dm
    from gpu_helpers import run_3idx
    codes = {"bf16x3": (B.DMET_PREC_BF16X3, 1e-6), "fp16x2": (B.DMET_PREC_FP16X2, 5e-6),
             "tf32x3": (B.DMET_PREC_TF32X3, 5e-6)}
    code, tol = codes[name]
    spec = spec_of((3, 2, 1), 6, 11, 20, n_spin=2)
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(spec.mesh, 6, 11, [20, 20], n_spin=2, prec=code, l_layout=layout)
    Lin = synth.make_L_pairs(spec, dm.dmet_emb_l_pairs(d)) if layout == B.DMET_L_REDUCED else L
    got, st, _ = run_3idx(torch, d, Lin, Cs, 0, spec.nk)
    assert st == B.DMET_OK
    for s in range(2):
        ref = oracle.embedded_3idx(L, Cs[s], spec.mesh)
        assert rel_fro(got[s], ref) < tol, (name, s, rel_fro(got[s], ref))
