"""Density-fitted Coulomb and exchange on the device (dmet_emb_jk_df) against the oracle's
coulomb_exchange_df (pinned against the ERI route and the one-cell textbook formula), from the
factors L^q that dmet_emb_transform_3idx writes; FP64 throughout, bound 1e-12 relative to max|J|."""
import numpy as np
import pytest

import oracle
import synth
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh,n_ao,n_aux,n,real", [((2, 2, 1), 4, 9, 7, True), ((3, 2, 1), 5, 11, 12, True),
                                                   ((3, 1, 1), 3, 6, 5, False), ((1, 1, 1), 4, 7, 3, True)])
def test_jk_df_matches_oracle(mesh, n_ao, n_aux, n, real):
    torch = torch_cuda()
    spec = synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n, 1, 0.6, 0.0, 55, "jk")
    L = synth.make_L(spec)
    csc = synth.supercell_orbitals(spec) if real else synth.complex_supercell_orbitals(spec)
    C = synth.bloch_orbitals(csc, mesh)
    sym = B.DMET_SYM_REAL if real else B.DMET_SYM_NONE
    d = dm.make_desc(mesh, n_ao, n_aux, n, sym=sym)
    nk = spec.nk
    Ld, Cd = torch.from_numpy(L).cuda(), torch.from_numpy(C).cuda()
    Lq = torch.empty((nk, n_aux, n, n), dtype=torch.complex128, device="cuda")
    gamma = synth.embedding_density(n, 9).astype(np.complex128)
    if not real:
        gamma = gamma + 1j * 0.1 * np.triu(np.ones((n, n)), 1) - 1j * 0.1 * np.tril(np.ones((n, n)), -1)
    gd = torch.from_numpy(np.ascontiguousarray(gamma)).cuda()
    J = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(J)
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_transform_3idx(plan, 0, Ld, [Cd], 0, nk, [Lq])
        dm.dmet_emb_jk_df(plan, Lq, gd, J, K)
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    Jr, Kr = oracle.coulomb_exchange_df(oracle.embedded_3idx(L, C, mesh), gamma, mesh)
    scale = np.abs(Jr).max()
    assert np.abs(J.cpu().numpy() - Jr).max() < 1e-12 * scale
    assert np.abs(K.cpu().numpy() - Kr).max() < 1e-12 * scale
