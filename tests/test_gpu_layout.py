"""GPU tests of the reduced L layout and of q shards, through the C ABI.

* The reduced layout holds only the (k1, k2) blocks the 8-fold schedule reads (dmet_emb_l_pairs);
  the kernels index L through the same tables, so the results must equal the full layout's bit
  for bit, on both paths, with device and host L.
* dmet_emb_transform_3idx on the reduced layout computes a q of zero contraction weight from -q
  and conjugates it: every L^q against the oracle (FP64 tolerance).
* Shards: the packed ERIs of disjoint q shards add up to the full ERI (Algorithm 1's sum over the
  aux momentum is a plain sum), FP64 to 1e-12 relative; each shard alone against the oracle's
  partial sum over its own q.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mesh as omesh
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, run_eri, run_3idx, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def spec_of(mesh, n_ao, n_aux, n_emb, n_spin=1, seed=31):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, n_spin, 0.6, 0.0, seed, "layout")


def reduced_L(spec, desc):
    return synth.make_L_pairs(spec, dm.dmet_emb_l_pairs(desc))


@pytest.mark.parametrize("mesh,n_spin", [((2, 2, 1), 1), ((3, 3, 1), 2), ((2, 2, 2), 1), ((4, 2, 1), 2)])
@pytest.mark.parametrize("prec", [B.DMET_PREC_FP64, B.DMET_PREC_BF16X3])
@pytest.mark.parametrize("host", [False, True])
def test_reduced_layout_equals_full(torch, mesh, n_spin, prec, host):
    spec = spec_of(mesh, 5, 11, 9, n_spin)
    L, Cs, _ = synth.make_problem(spec)
    ne = [9, 9] if n_spin == 2 else [9, 0]
    d_full = B.make_desc(mesh, 5, 11, ne, n_spin=n_spin, prec=prec)
    d_red = B.make_desc(mesh, 5, 11, ne, n_spin=n_spin, prec=prec, l_layout=B.DMET_L_REDUCED)
    full, st, _ = run_eri(torch, d_full, L, Cs)
    assert st == B.DMET_OK
    red, st, _ = run_eri(torch, d_red, reduced_L(spec, d_red), Cs, host=host)
    assert st == B.DMET_OK
    for a, b in zip(full, red):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mesh", [(3, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2)])
def test_reduced_layout_3idx_matches_oracle(torch, mesh):
    spec = spec_of(mesh, 4, 6, 7, 2)
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(mesh, 4, 6, [7, 7], n_spin=2, l_layout=B.DMET_L_REDUCED)
    nk = spec.nk
    got, st, _ = run_3idx(torch, d, reduced_L(spec, d), Cs, 0, nk)
    assert st == B.DMET_OK
    for s in range(2):
        ref = oracle.embedded_3idx(L, Cs[s], mesh)
        assert rel_fro(got[s], ref) < 1e-12


def test_reduced_layout_3idx_outside_shard_is_refused(torch):
    spec = spec_of((3, 1, 1), 4, 6, 7)
    d = B.make_desc((3, 1, 1), 4, 6, 7, l_layout=B.DMET_L_REDUCED, q_range=(0, 1))
    Ld = torch.from_numpy(reduced_L(spec, d)).cuda()
    _, Cs, _ = synth.make_problem(spec, with_L=False)
    Cd = [torch.from_numpy(Cs[0]).cuda()]
    out = [torch.empty((1, 6, 7, 7), dtype=torch.complex128, device="cuda")]
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_transform_3idx(plan, 0, Ld, Cd, 0, 1, out)   # q = 0 is in the shard
        with pytest.raises(B.DmetError) as e:
            dm.dmet_emb_transform_3idx(plan, 0, Ld, Cd, 1, 2, out)
        assert e.value.status == B.DMET_ERR_INVALID_ARG
    finally:
        dm.dmet_emb_destroy(plan)


SHARDS = {(4, 2, 1): [(0, 2), (2, 5), (5, 8)], (3, 3, 1): [(0, 1), (1, 4), (4, 9)], (2, 2, 2): [(0, 3), (3, 8)]}


def oracle_shard(L, Cs, mesh, lo, hi):
    """The oracle's ERI blocks restricted to the q with lo <= min(q, -q) < hi (Algorithm 1's sum over q
    taken over a subset)."""
    nk = int(np.prod(mesh))
    lq = [oracle.embedded_3idx(L, C, mesh) for C in Cs]
    keys = [(0, 0)] if len(Cs) == 1 else [(0, 0), (0, 1), (1, 1)]
    out = []
    for a, b in keys:
        eri = 0
        for q in range(nk):
            if lo <= min(q, omesh.k_neg(q, mesh)) < hi:
                eri = eri + np.tensordot(lq[a][q], lq[b][omesh.k_neg(q, mesh)], axes=([0], [0])) / nk
        eri = np.real(eri)
        out.append(oracle.pack_s8(eri) if a == b else oracle.pair_matrix(eri).ravel())
    return out


@pytest.mark.parametrize("mesh", sorted(SHARDS))
@pytest.mark.parametrize("prec", [B.DMET_PREC_FP64, B.DMET_PREC_BF16X3])
@pytest.mark.parametrize("layout", [B.DMET_L_FULL, B.DMET_L_REDUCED])
def test_shards_add_up_to_the_full_eri(torch, mesh, prec, layout):
    spec = spec_of(mesh, 5, 9, 8, 2)
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(mesh, 5, 9, [8, 8], n_spin=2, prec=prec)
    full, st, _ = run_eri(torch, d, L, Cs)
    assert st == B.DMET_OK
    total = [np.zeros_like(f) for f in full]
    tol = 1e-12 if prec == B.DMET_PREC_FP64 else 1e-6
    for lo, hi in SHARDS[mesh]:
        ds = B.make_desc(mesh, 5, 9, [8, 8], n_spin=2, prec=prec, l_layout=layout, q_range=(lo, hi))
        Lin = reduced_L(spec, ds) if layout == B.DMET_L_REDUCED else L
        part, st, _ = run_eri(torch, ds, Lin, Cs)
        assert st == B.DMET_OK
        ref = oracle_shard(L, Cs, mesh, lo, hi)
        for p, r in zip(part, ref):
            assert np.abs(p - r).max() <= tol * max(np.abs(r).max(), 1e-300) * 10
        for t, p in zip(total, part):
            t += p
    for t, f in zip(total, full):
        assert rel_fro(t, f) < (1e-12 if prec == B.DMET_PREC_FP64 else 2e-6)
