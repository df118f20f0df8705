"""GPU parity of the embedding one-particle Hamiltonian (dmet_emb_fock; Eqs. "fock transform" and
"fock double counting", section 2.1) with the oracle, through the C ABI."""
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


def spec_of(mesh, n_ao, n_aux, n_emb, seed=31, n_spin=1):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, n_spin, 0.6, 0.0, seed, "f")


def run_fock(torch, spec, prec, ck_norm=0, gamma_seed=7):
    """(fock from the GPU, its ERI as host array, F, C, gamma)."""
    L, (C,), _ = synth.make_problem(spec, ck_norm=ck_norm)
    F = synth.fock_k(synth.real_space_fock(spec), spec.mesh)
    gamma = synth.embedding_density(spec.n_emb, gamma_seed)
    d = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb, prec=prec, ck_norm=ck_norm)
    outs = out_buffers(torch, d)
    Ld, Cd = torch.from_numpy(L).cuda(), torch.from_numpy(C).cuda()
    Fd, gd = torch.from_numpy(F).cuda(), torch.from_numpy(gamma).cuda()
    fo = torch.empty((spec.n_emb, spec.n_emb), dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_eri(plan, [Ld], [[Cd]], [outs])
        dm.dmet_emb_fock(plan, Fd, Cd, outs[0], gd, fo)
        torch.cuda.synchronize()
        st, _ = dm.dmet_emb_status(plan, 0)
        assert st == B.DMET_OK
    finally:
        dm.dmet_emb_destroy(plan)
    return fo.cpu().numpy(), outs[0].cpu().numpy(), L, F, C, gamma


CASES = [((2, 2, 1), 8, 40, 16), ((3, 2, 1), 6, 11, 20), ((3, 3, 1), 10, 37, 70), ((1, 1, 1), 5, 7, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_n{c[3]}")
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_fock_fp64_matches_oracle(torch, case, ck_norm):
    mesh, nao, naux, n = case
    spec = spec_of(mesh, nao, naux, n)
    got, _, L, F, C, gamma = run_fock(torch, spec, B.DMET_PREC_FP64, ck_norm)
    F0 = oracle.fock_transform(F, C, ck_norm)
    eri = oracle.embedded_eri(L, C, mesh, ck_norm=ck_norm).real
    ref = oracle.embedded_fock(F0.real, eri, gamma)
    assert np.abs(F0.imag).max() < 1e-12 * max(1.0, np.abs(F0).max())
    assert rel_fro(got, ref) < 1e-10, rel_fro(got, ref)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(got - got.T).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: "x".join(map(str, c[0])) + f"_n{c[3]}")
def test_fock_mixed_eri_matches_oracle(torch, case):
    """With the split-BF16 ERI the Fock matrix carries that ERI's ~1e-6 relative error at most."""
    mesh, nao, naux, n = case
    spec = spec_of(mesh, nao, naux, n)
    got, _, L, F, C, gamma = run_fock(torch, spec, B.DMET_PREC_BF16X3)
    ref = oracle.embedded_fock(oracle.fock_transform(F, C).real, oracle.embedded_eri(L, C, mesh).real, gamma)
    assert rel_fro(got, ref) < 1e-6, rel_fro(got, ref)


def test_fock_on_its_own_eri_at_the_hbn_size(torch):
    """The h-BN-sized problem (n_emb = 104): the Fock kernels against the oracle's formulas applied
    to the same FP64 ERI the library produced (the ERI itself is checked elsewhere)."""
    spec = synth.CONFIGS["hbn_6x6x1"]
    got, eri_p, _, F, C, gamma = run_fock(torch, spec, B.DMET_PREC_FP64)
    eri = oracle.unpack_s8(eri_p, spec.n_emb)
    ref = oracle.embedded_fock(oracle.fock_transform(F, C).real, eri, gamma)
    assert rel_fro(got, ref) < 1e-12, rel_fro(got, ref)


def test_fock_rejects_unsupported_and_host_pointers(torch):
    spec = spec_of((2, 1, 1), 4, 6, 5, n_spin=2)
    d = B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, [5, 5], n_spin=2)
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    x = torch.zeros(64, dtype=torch.complex128, device="cuda")
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(B.DmetError) as e:
            dm.dmet_emb_fock(plan, x, x, y, y, y)
        assert e.value.status == B.DMET_ERR_UNSUPPORTED
    finally:
        dm.dmet_emb_destroy(plan)
    d = B.make_desc((2, 1, 1), 4, 6, 5)
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(B.DmetError) as e:
            dm.dmet_emb_fock(plan, x.cpu().numpy(), x, y, y, y)
        assert e.value.status == B.DMET_ERR_INVALID_ARG
    finally:
        dm.dmet_emb_destroy(plan)
