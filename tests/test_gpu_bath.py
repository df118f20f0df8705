"""GPU parity of the DMET bath and embedding orbitals (dmet_emb_bath; Eqs. "bath R SVD", "C loemb R"
and "C loemb k", section 2.1) with the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from paper_1909_08596_gb300 import binding as B
import paper_1909_08596_gb300 as dm

from gpu_helpers import out_buffers, rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def inputs(mesh, n_ao, n_occ, seed=11, n_aux=9, n_val=1, isolate=None):
    spec = synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_ao + n_val, 1, 0.6, 0.0, seed, "bath")
    h = synth.mean_field_hamiltonian(spec, n_occ)
    g = synth.mean_field_density(h, mesh, n_occ)
    if isolate is not None:
        # an impurity LO decoupled from every other orbital (an exact zero column of the block)
        occ = np.round(g[:, isolate, isolate].real)
        g[:, isolate, :] = 0.0
        g[:, :, isolate] = 0.0
        g[:, isolate, isolate] = occ
    return spec, g, synth.lo_rotation(spec)


def run_bath(torch, spec, gamma_k, U, val):
    d = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_ao + len(val))
    gd, Ud = torch.from_numpy(gamma_k).cuda(), torch.from_numpy(U).cuda()
    Cd = torch.empty((spec.nk, spec.n_ao, spec.n_ao + len(val)), dtype=torch.complex128, device="cuda")
    info = torch.zeros(len(val) + 5, dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_bath(plan, gd, Ud, val, Cd, info)
        torch.cuda.synchronize()
    finally:
        dm.dmet_emb_destroy(plan)
    return Cd.cpu().numpy(), info.cpu().numpy()


# (mesh, n_ao, n_occ, val): ragged and odd column counts, a single column, every impurity column,
# a 3D mesh, an odd mesh, the h-BN-shaped cell (26 LOs, 8 valence), the Si-shaped cell (52 LOs on
# 4x4x4) with 16 and with all 52 columns, 70 columns (more pairs per round than warps), and a block
# too large for shared memory.
CASES = [
    ((2, 2, 1), 6, 3, [0, 2, 3, 5]),
    ((3, 2, 1), 8, 4, [7, 1, 4]),
    ((2, 2, 2), 7, 3, list(range(7))),
    ((5, 1, 1), 5, 2, [3]),
    ((6, 6, 1), 26, 13, [0, 1, 2, 3, 13, 14, 15, 16]),
    ((4, 4, 4), 52, 26, [0, 13, 26, 39, 2, 6, 10, 14, 18, 22, 30, 34, 42, 46, 50, 51]),
    ((4, 4, 4), 52, 26, list(range(52))),   # 26 pairs per round: two passes of the 16 warps
    ((2, 2, 1), 70, 35, list(range(70))),   # 35 pairs per round: three passes
    # 104 LOs on 4x4x4, 64 columns: each CTA's rows (819 x 64, 410 KB) stay in global memory
    ((4, 4, 4), 104, 52, list(range(0, 104, 2)) + list(range(1, 24, 2))),
]


def case_id(c):
    return "x".join(map(str, c[0])) + f"_ao{c[1]}_v{len(c[3])}"


@pytest.mark.parametrize("case", CASES, ids=case_id)
def test_bath_matches_oracle(torch, case):
    mesh, n_ao, n_occ, val = case
    assert len(set(val)) == len(val)
    spec, g, U = inputs(mesh, n_ao, n_occ)
    got, info = run_bath(torch, spec, g, U, val)
    want, s = oracle.embedding_orbitals(g, U, mesh, val)
    nv = len(val)
    np.testing.assert_allclose(info[:nv], s, rtol=1e-12, atol=1e-14 * s.max())
    assert info[nv + 1] <= 1e-13 * info[nv]          # the block is real
    assert info[nv + 2] < 40 and (info[nv + 2] >= 1 or nv == 1)  # Jacobi sweeps, converged
    assert info[nv + 3] <= 1e-14 or nv == 1            # last sweep's largest pair cosine
    assert abs(info[nv + 4] - s.min() / s.max()) < 1e-12
    # the bath columns are determined (sign included) when the singular values are distinct
    gaps = np.diff(s[::-1]).min() / s.max() if nv > 1 else 1.0
    assert gaps > 1e-6
    err = np.abs(got - want).max()
    assert err < 1e-10, err
    np.testing.assert_array_equal(got[:, :, :n_ao], U)  # the impurity columns are C^{k,AO,LO}
    assert oracle.orthonormality_error(got) < 1e-12
    assert oracle.realness_error(got, mesh) < 1e-12


def test_bath_zero_singular_value_gives_zero_column(torch):
    mesh, val = (3, 2, 1), [2, 0, 4]
    spec, g, U = inputs(mesh, 6, 3, isolate=2)
    got, info = run_bath(torch, spec, g, U, val)
    want, s = oracle.embedding_orbitals(g, U, mesh, val)
    assert s[-1] < 1e-14 and info[2] == 0.0 and info[len(val) + 4] == 0.0
    np.testing.assert_allclose(info[:2], s[:2], rtol=1e-12)
    assert np.abs(got[:, :, spec.n_ao + 2]).max() == 0.0
    assert np.abs(got[:, :, :spec.n_ao + 2] - want[:, :, :spec.n_ao + 2]).max() < 1e-10


def test_bath_orbitals_feed_the_eri(torch):
    """The orbitals dmet_emb_bath leaves on the device go straight into dmet_emb_eri (which
    checks their orthonormality and realness); the ERI equals the oracle's on the oracle's
    orbitals."""
    mesh, val = (2, 2, 1), [1, 3, 4]
    spec, g, U = inputs(mesh, 8, 4, n_aux=40, n_val=len(val))
    d = B.make_desc(mesh, spec.n_ao, spec.n_aux, spec.n_emb)
    L = synth.make_L(spec)
    Ld, gd, Ud = (torch.from_numpy(x).cuda() for x in (L, g, U))
    Cd = torch.empty((spec.nk, spec.n_ao, spec.n_emb), dtype=torch.complex128, device="cuda")
    outs = out_buffers(torch, d)
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_bath(plan, gd, Ud, val, Cd)
        dm.dmet_emb_eri(plan, [Ld], [[Cd]], [outs])
        st, stats = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK and stats[0] < 1e-12
    C, _ = oracle.embedding_orbitals(g, U, mesh, val)
    ref = oracle.pack_s8(oracle.embedded_eri(L, C, mesh).real)
    assert rel_fro(outs[0].cpu().numpy(), ref) < 1e-12


def test_bath_rejects_bad_arguments(torch):
    spec, g, U = inputs((2, 2, 1), 6, 3, n_val=2)
    d = B.make_desc(spec.mesh, 6, 9, 8)
    gd, Ud = torch.from_numpy(g).cuda(), torch.from_numpy(U).cuda()
    Cd = torch.empty((4, 6, 8), dtype=torch.complex128, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        for val in ([0, 1, 2], [0, 0], [0, 6], [-1, 2], []):
            with pytest.raises(B.DmetError) as e:
                dm.dmet_emb_bath(plan, gd, Ud, val, Cd)
            assert e.value.status == B.DMET_ERR_INVALID_ARG
        with pytest.raises(B.DmetError) as e:
            dm.dmet_emb_bath(plan, g, Ud, [0, 1], Cd)  # host buffer
        assert e.value.status == B.DMET_ERR_INVALID_ARG
        with pytest.raises(B.DmetError) as e:
            dm.dmet_emb_bath(plan, gd, Ud, [0, 1], Cd, spin=1)
        assert e.value.status == B.DMET_ERR_INVALID_ARG
    finally:
        dm.dmet_emb_destroy(plan)
    # one cell has no environment: its plan cannot hold n_ao + n_val > n_ao orbitals
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(B.make_desc((1, 1, 1), 6, 9, 8), stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.status == B.DMET_ERR_INVALID_ARG


def _hand_cases():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_bath.json")))["cases"]


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_bath_hand_worked_examples(torch, case):
    """The device path against values derived by hand (C^{k,AO,LO} = 1, so C_out = C^{k,LO,EO})."""
    mesh, val = tuple(case["mesh"]), case["val"]
    gk = np.ascontiguousarray(np.asarray(case["gamma_k"], dtype=np.complex128))
    nk, n_lo = gk.shape[0], gk.shape[1]
    U = np.ascontiguousarray(np.broadcast_to(np.eye(n_lo, dtype=np.complex128), (nk, n_lo, n_lo)))
    spec = synth.LatticeSpec(mesh, n_lo, 3, n_lo + len(val), 1, 0.6, 0.0, 0, "hand")
    got, info = run_bath(torch, spec, gk, U, val)
    want = np.asarray(case["C_lo_eo_re"]) + 1j * np.asarray(case["C_lo_eo_im"])
    np.testing.assert_allclose(info[:len(val)], case["sigma"], rtol=1e-14)
    np.testing.assert_allclose(got, want, atol=1e-14)
