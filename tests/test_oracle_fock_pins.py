"""Pins of the embedding one-particle Hamiltonian oracle (Eqs. "fock transform" and "fock double
counting", section 2.1) against routes that do not go through it: the real-space supercell Fock
matrix, the 3-index (density-fitted) form of J and K, and a one-orbital closed form. Planted
mistakes (a transposed Fock matrix, a dropped 1/Nk, exchange contracted like Coulomb, a dropped 1/2)
each fail one of them. (For real orbitals and a symmetric gamma the index orders (ik|lj), (il|kj),
(ki|jl) all give the same exchange; the planted exchange mistake contracts like Coulomb.)"""
import numpy as np
import pytest

import oracle
import synth
from oracle.mesh import k_neg


def _spec(mesh, n_ao, n_aux, n_emb, seed=5):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, 1, 0.6, 0.0, seed, "fock")


MESHES = [((1, 1, 1), 4, 3), ((2, 1, 1), 3, 4), ((3, 1, 1), 3, 5), ((2, 2, 1), 3, 6), ((3, 2, 1), 2, 5)]


@pytest.mark.parametrize("mesh,n_ao,n_emb", MESHES)
@pytest.mark.parametrize("complex_orbitals", [False, True])
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_fock_transform_matches_supercell(mesh, n_ao, n_emb, complex_orbitals, ck_norm):
    spec = _spec(mesh, n_ao, 2, n_emb)
    f = synth.real_space_fock(spec)
    csc = synth.complex_supercell_orbitals(spec) if complex_orbitals else synth.supercell_orbitals(spec)
    C = synth.bloch_orbitals(csc, mesh, ck_norm)
    F = synth.fock_k(f, mesh)
    got = oracle.fock_transform(F, C, ck_norm)
    ref = oracle.supercell_fock(f, mesh, csc)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert np.abs(got - got.conj().T).max() < 1e-12          # Hermitian
    if not complex_orbitals:
        assert np.abs(got.imag).max() < 1e-12                  # real orbitals: real F0


def test_fock_planted_mistakes_fail_supercell_pin():
    mesh = (3, 2, 1)
    spec = _spec(mesh, 3, 2, 5)
    f = synth.real_space_fock(spec)
    csc = synth.complex_supercell_orbitals(spec)
    C = synth.bloch_orbitals(csc, mesh)
    F = synth.fock_k(f, mesh)
    ref = oracle.supercell_fock(f, mesh, csc)
    nk = F.shape[0]
    transposed = sum(C[k].conj().T @ F[k].T @ C[k] for k in range(nk)) / nk
    no_norm = sum(C[k].conj().T @ F[k] @ C[k] for k in range(nk))
    for bad in (transposed, no_norm):
        assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("mesh,n_ao,n_emb", [((2, 1, 1), 3, 4), ((3, 1, 1), 3, 5), ((2, 2, 1), 2, 6)])
def test_coulomb_exchange_match_density_fitted_route(mesh, n_ao, n_emb):
    spec = _spec(mesh, n_ao, 5, n_emb)
    L, (C,), _ = synth.make_problem(spec)
    Lq = oracle.embedded_3idx(L, C, mesh)
    eri = oracle.embedded_eri(L, C, mesh, Lq_a=Lq).real
    gamma = synth.embedding_density(n_emb, 11)
    J, K = oracle.coulomb_exchange(eri, gamma)
    J3, K3 = oracle.coulomb_exchange_df(Lq, gamma, mesh)
    scale = np.abs(J3).max()
    assert np.abs(J - J3).max() < 1e-12 * scale and np.abs(K - K3).max() < 1e-12 * scale
    assert np.abs(J - J.T).max() < 1e-12 * scale and np.abs(K - K.T).max() < 1e-12 * scale
    # planted: exchange contracted like Coulomb, (ij|kl) gamma_kl instead of (ik|lj) gamma_kl
    K_bad = np.einsum("ijkl,kl->ij", eri, gamma)
    assert np.abs(K_bad - K3).max() > 1e-6 * scale


def test_density_fitted_jk_planted_momentum_mistake():
    # pairing L^q with L^q instead of L^{-q} breaks the agreement with the ERI route
    mesh = (3, 1, 1)
    spec = _spec(mesh, 3, 5, 5)
    L, (C,), _ = synth.make_problem(spec)
    Lq = oracle.embedded_3idx(L, C, mesh)
    gamma = synth.embedding_density(5, 11)
    J, K = oracle.coulomb_exchange(oracle.embedded_eri(L, C, mesh, Lq_a=Lq).real, gamma)
    Jb = sum(Lq[q][P] * np.trace(Lq[q][P] @ gamma) for q in range(3) for P in range(Lq.shape[1])) / 3
    assert np.abs(Jb - J).max() > 1e-6 * np.abs(J).max()


def test_density_fitted_jk_nk1_is_the_molecular_formula():
    # one cell: J = sum_P B_P tr(B_P gamma), K = sum_P B_P gamma B_P with B_P = C^T L_P C (textbook DF)
    mesh = (1, 1, 1)
    spec = _spec(mesh, 4, 6, 3)
    L, (C,), _ = synth.make_problem(spec)
    Bp = np.einsum("mi,Pmn,nj->Pij", C[0].conj(), L[0, 0], C[0])
    gamma = synth.embedding_density(3, 4)
    J, K = oracle.coulomb_exchange_df(oracle.embedded_3idx(L, C, mesh), gamma, mesh)
    Jt = sum(Bp[P] * np.trace(Bp[P] @ gamma) for P in range(Bp.shape[0]))
    Kt = sum(Bp[P] @ gamma @ Bp[P] for P in range(Bp.shape[0]))
    np.testing.assert_allclose(J, Jt, atol=1e-12)
    np.testing.assert_allclose(K, Kt, atol=1e-12)


def test_one_orbital_closed_form():
    """One embedding orbital: Ftilde = F0 - (00|00) gamma + (00|00) gamma / 2."""
    eri = np.array([[[[0.7]]]])
    gamma = np.array([[1.3]])
    F0 = np.array([[-0.4]])
    got = oracle.embedded_fock(F0, eri, gamma)
    assert got[0, 0] == pytest.approx(-0.4 - 0.7 * 1.3 / 2)
    J, K = oracle.coulomb_exchange(eri, gamma)
    assert (F0 - (J - K))[0, 0] != pytest.approx(got[0, 0])   # a dropped 1/2 is caught


def test_embedding_density_is_a_density():
    g = synth.embedding_density(9, 3)
    w = np.linalg.eigvalsh(g)
    assert np.allclose(g, g.T) and w.min() > -1e-12 and w.max() < 2 + 1e-12
