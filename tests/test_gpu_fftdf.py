"""The FFTDF embedded ERI on the device (dmet_emb_eri_fftdf, Appendix B, Algorithm 2) against the
oracle's embedded_eri_fftdf (pinned against the Coulomb integral over the Born-von Karman supercell).
FP64 bound 1e-12 relative to max|(ij|kl)|. The alpha-beta block is checked against the oracle's ERI of
the concatenated orbital set [C_alpha | C_beta] (the ERI is bilinear in the orbitals)."""
import numpy as np
import pytest

import synth
import oracle.fftdf as of
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

CASES = [((1, 1, 1), (4, 4, 4)), ((2, 2, 1), (3, 4, 3)), ((3, 1, 1), (3, 5, 3)), ((3, 3, 1), (3, 3, 5)),
         ((2, 1, 1), (3, 2, 34))]   # an axis of more than 32 points takes the GEMM form of the DFT


def _inputs(mesh, grid, complex_orbitals, n_emb=3, spin=0):
    spec = synth.GridSpec(tuple(mesh), 2, tuple(grid), n_emb=n_emb, seed=3)
    rho = synth.pair_densities_k(spec)
    csc = synth.grid_orbitals(spec, spin=spin, complex_orbitals=complex_orbitals)
    return spec, rho, csc


def _run(torch, spec, rho, Cs, sym):
    ng = int(np.prod(spec.grid))
    ne = [c.shape[2] for c in Cs]
    d = dm.make_desc(spec.mesh, spec.n_ao, ng, ne if len(Cs) == 2 else ne[0], n_spin=len(Cs), sym=sym,
                     eri_pack=B.DMET_PACK_FULL)
    rd = torch.from_numpy(np.ascontiguousarray(rho.transpose(0, 1, 4, 2, 3))).cuda()   # [k1][k2][r][mu][nu]
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    outs = [torch.empty(dm.dmet_emb_eri_bytes(d, b) // 16, dtype=torch.complex128, device="cuda")
            for b in range(1 if len(Cs) == 1 else 3)]
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_eri_fftdf(plan, rd, Cd, spec.grid, spec.lattice, outs)
        st, stats = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK, stats
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("mesh,grid", CASES)
@pytest.mark.parametrize("complex_orbitals", [False, True])
def test_fftdf_matches_oracle(mesh, grid, complex_orbitals):
    torch = torch_cuda()
    spec, rho, csc = _inputs(mesh, grid, complex_orbitals)
    C = synth.bloch_orbitals(csc, mesh)
    sym = B.DMET_SYM_NONE if complex_orbitals else B.DMET_SYM_REAL
    (got,) = _run(torch, spec, rho, [C], sym)
    ref = of.embedded_eri_fftdf(rho, C, mesh, spec.lattice, spec.grid).ravel()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_fftdf_unrestricted_blocks():
    torch = torch_cuda()
    mesh, grid = (3, 1, 1), (3, 5, 3)
    spec, rho, ca = _inputs(mesh, grid, True, n_emb=3, spin=0)
    _, _, cb = _inputs(mesh, grid, True, n_emb=3, spin=1)
    Ca, Cb = synth.bloch_orbitals(ca, mesh), synth.bloch_orbitals(cb, mesh)
    aa, ab, bb = _run(torch, spec, rho, [Ca, Cb], B.DMET_SYM_NONE)
    both = of.embedded_eri_fftdf(rho, np.concatenate([Ca, Cb], axis=2), mesh, spec.lattice, grid)
    scale = np.abs(both).max()
    assert np.abs(aa - both[:3, :3, :3, :3].ravel()).max() < 1e-12 * scale
    assert np.abs(ab - both[:3, :3, 3:, 3:].ravel()).max() < 1e-12 * scale
    assert np.abs(bb - both[3:, 3:, 3:, 3:].ravel()).max() < 1e-12 * scale
