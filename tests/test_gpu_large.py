"""The split-BF16 unrestricted path at a shape that reaches the NiO-shaped workload's tiles and
contraction length: n_emb = 256 per spin (257 x 257 tiles of pairs), contraction rank
K = sum over contracted q of n_aux (1 or 2 slices) = 28 800 (4x4x2 mesh, 900 aux functions), L in the
reduced layout generated on the device. Every (ij|kl) of every spin block (aa, ab, bb) on seeded
48-orbital subsets is compared with the FP64 oracle, which receives every aux function's L block by
block (exact: an orbital-column subset of the ERI is the method applied to those columns, and the sum
over the aux index is additive). Tolerance: 1e-6 relative Frobenius and max-abs over max (the mixed
path's bound)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

import bench
from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-6


def test_mixed_uhf_long_contraction_matches_oracle():
    torch = torch_cuda()
    from synth import gpu as sgpu
    spec = synth.LatticeSpec((4, 4, 2), 24, 900, 256, 2, 0.6, 0.0, 3100, "uhf_4x4x2_k28800")
    desc = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, [256, 256], n_spin=2, prec=B.DMET_PREC_BF16X3,
                       l_layout=B.DMET_L_REDUCED)
    qw, _ = bench.schedule_counts(spec.mesh)
    assert sum(spec.n_aux * w for w in qw) == 28800
    _, Cs, _ = synth.make_problem(spec, with_L=False)
    Ld = sgpu.make_L_pairs_device(torch, spec, dm.dmet_emb_l_pairs(desc), p_block=32)
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    outs = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64, device="cuda") for b in range(3)]
    plan = dm.dmet_emb_plan(desc, stream=torch.cuda.current_stream().cuda_stream, workspace_limit=48 << 30)
    try:
        dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
        st, stats = dm.dmet_emb_status(plan, 0)
        assert st == B.DMET_OK, (dm.dmet_emb_last_error(), stats)
    finally:
        dm.dmet_emb_destroy(plan)
    del Ld
    S = bench.subset_orbitals(spec, 48, seed=1)
    got = bench.gather_subsets(torch, outs, bench.block_positions(spec, S))
    del outs
    torch.cuda.empty_cache()
    Csub = [np.ascontiguousarray(C[:, :, s]) for C, s in zip(Cs, S)]
    blocks = (sgpu.L_blocks_device(torch, spec, p0, min(spec.n_aux, p0 + 64)).cpu().numpy()
              for p0 in range(0, spec.n_aux, 64))
    ref = oracle.embedded_eri_pblocks(blocks, Csub, spec.mesh)
    for b, key in enumerate([(0, 0), (0, 1), (1, 1)]):
        r = ref[key].real.ravel()
        assert np.abs(ref[key].imag).max() < 1e-12 * np.abs(r).max()
        e = np.linalg.norm(got[b] - r) / np.linalg.norm(r)
        m = np.abs(got[b] - r).max() / np.abs(r).max()
        assert e < TOL and m < TOL, (key, e, m)
