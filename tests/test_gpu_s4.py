"""4-fold packed complex ERIs (DMET_PACK_S4, FP64 path) against the oracle's pack_s4 / pack_s4_ab of
Algorithm 1's complex ERI: complex orbitals (sym = NONE), restricted and unrestricted, and real orbitals
packed the same way. FP64 bound: 1e-10 relative Frobenius and max-abs over max."""
import numpy as np
import pytest

import oracle
import synth
from oracle import checks
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


def run(torch, desc, L, Cs):
    import paper_1909_08596_gb300 as dm
    nblk = 1 if desc.n_spin == 1 else 3
    outs = [torch.empty(dm.dmet_emb_eri_bytes(desc, b) // 16, dtype=torch.complex128, device="cuda")
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


def close(got, ref):
    assert got.shape == ref.shape
    assert rel_fro(got, ref) < 1e-10
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("mesh,n", [((2, 2, 1), 6), ((3, 2, 1), 9), ((3, 1, 1), 1)])
def test_s4_complex_orbitals(mesh, n):
    torch = torch_cuda()
    spec = synth.LatticeSpec(tuple(mesh), 4, 7, n, 1, 0.6, 0.0, 61, "s4")
    L = synth.make_L(spec)
    C = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec), mesh)
    d = B.make_desc(mesh, 4, 7, n, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_S4)
    (got,) = run(torch, d, L, [C])
    assert len(got) == checks.s4_size(n)
    close(got, checks.pack_s4(oracle.embedded_eri(L, C, mesh)))


def test_s4_unrestricted_complex():
    torch = torch_cuda()
    spec = synth.LatticeSpec((3, 2, 1), 4, 7, 6, 2, 0.6, 0.0, 62, "s4u")
    L = synth.make_L(spec)
    ca = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec, 0), spec.mesh)
    cb = synth.bloch_orbitals(synth.complex_supercell_orbitals(synth.spec_with(spec, n_emb=8), 1), spec.mesh)
    d = B.make_desc(spec.mesh, 4, 7, [6, 8], n_spin=2, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_S4)
    aa, ab, bb = run(torch, d, L, [ca, cb])
    close(aa, checks.pack_s4(oracle.embedded_eri(L, ca, spec.mesh)))
    close(bb, checks.pack_s4(oracle.embedded_eri(L, cb, spec.mesh)))
    close(ab, checks.pack_s4_ab(oracle.embedded_eri(L, ca, spec.mesh, Cb=cb)))


def test_s4_real_orbitals():
    torch = torch_cuda()
    spec = synth.LatticeSpec((2, 2, 2), 3, 6, 7, 1, 0.6, 0.0, 63, "s4r")
    L, Cs, _ = synth.make_problem(spec)
    d = B.make_desc(spec.mesh, 3, 6, 7, eri_pack=B.DMET_PACK_S4)
    (got,) = run(torch, d, L, Cs)
    close(got, checks.pack_s4(oracle.embedded_eri(L, Cs[0], spec.mesh)))
    assert np.abs(got.imag).max() < 1e-12 * np.abs(got.real).max()
