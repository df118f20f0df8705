"""dmet_emb_eri_noalloc, the entry point for callers that cannot allocate device memory
(their memory belongs to another allocator, or an allocation must not synchronise the
device mid-loop): called twice in a row through the C ABI, each result must match the
plan-based dmet_emb_eri FP64 result within the FP64 tolerance of the other GPU tests.
The meshes include ones whose q differ from -q (weight-2 contractions, two stacked L^q slices),
unitary-normalised orbitals, and a shape whose scratch is close to the static array's size.
This file is collected last so that a stop-at-first-failure run has run everything else."""
import ctypes

import numpy as np
import pytest

import synth
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, run_eri, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = {
    "tiny_2x2x1": (synth.CONFIGS["tiny_2x2x1"], 0),
    "3x1x1": (synth.LatticeSpec((3, 1, 1), 4, 9, 6, 1, 0.6, 0.0, 41, "na3"), 0),
    "3x3x1_unitary": (synth.LatticeSpec((3, 3, 1), 4, 9, 10, 1, 0.6, 0.0, 42, "na33"), 1),
    # about 25 MB of the 32 MiB scratch when unrestricted: T 9.2 MB, Z 6.9 MB, two pair operands 7 MB
    "3x3x1_near_cap": (synth.LatticeSpec((3, 3, 1), 16, 120, 60, 1, 0.6, 0.0, 43, "nacap"), 0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_spin", [1, 2])
def test_noalloc_matches_eri_two_calls(case, n_spin):
    torch = torch_cuda()
    spec, ck_norm = CASES[case]
    spec = synth.spec_with(spec, n_spin=n_spin)
    L, Cs, _ = synth.make_problem(spec, ck_norm=ck_norm)
    desc = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb, n_spin=n_spin, ck_norm=ck_norm, check_l=1)
    refs, st, _ = run_eri(torch, desc, L, Cs)
    assert st == B.DMET_OK
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    outs = [torch.empty(B.dmet_emb_eri_bytes(desc, b) // 8, dtype=torch.float64, device="cuda")
            for b in range(len(refs))]
    stream = torch.cuda.current_stream().cuda_stream
    lib = B.lib()
    cs = (ctypes.c_void_p * len(Cd))(*[c.data_ptr() for c in Cd])
    os_ = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    for call in range(2):
        for o in outs:
            o.fill_(float("nan"))
        status = lib.dmet_emb_eri_noalloc(ctypes.byref(desc), ctypes.c_void_p(Ld.data_ptr()), cs, os_,
                                          ctypes.c_void_p(stream))
        assert status == B.DMET_OK, (call, lib.dmet_emb_last_error())
        for o, ref in zip(outs, refs):
            got = o.cpu().numpy()
            assert np.isfinite(got).all()
            assert rel_fro(got, ref) < TOL, call


def test_noalloc_reports_non_orthonormal_orbitals():
    """The device checks' status comes back from the call itself."""
    torch = torch_cuda()
    spec = synth.CONFIGS["tiny_2x2x1"]
    L, (C,), _ = synth.make_problem(spec)
    desc = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb)
    out = torch.empty(B.dmet_emb_eri_bytes(desc, 0) // 8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DmetError) as e:
        B.dmet_emb_eri_noalloc(desc, torch.from_numpy(L).cuda(), [torch.from_numpy(1.01 * C).cuda()], [out])
    assert e.value.status == B.DMET_ERR_NOT_ORTHONORMAL


def test_noalloc_rejects_oversized_problem():
    """A problem whose scratch exceeds the static array is refused before any work."""
    torch = torch_cuda()
    desc = B.make_desc((4, 4, 4), 52, 400, 200)
    buf = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DmetError) as e:
        B.dmet_emb_eri_noalloc(desc, buf, [buf], [buf])
    assert e.value.status == B.DMET_ERR_OOM
    assert "static scratch holds" in str(e.value)
