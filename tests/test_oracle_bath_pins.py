"""Pins of the bath oracle (section 2.1, Eqs. "bath R SVD", "C loemb R", "C loemb k") against
results that do not go through it: the mean-field density matrix written out over the
supercell with no k-points, the closed form of the singular values of an idempotent density
matrix, the Bloch sum of the synthetic-input generator, and worked examples derived by hand
(tests/golden/hand_bath.json)."""
import numpy as np
import pytest

import oracle
import synth

MESHES = [(2, 2, 1), (3, 2, 1), (2, 2, 2)]


def _case(mesh, n_lo=6, n_occ=3, seed=7):
    spec = synth.spec_with(synth.CONFIGS["tiny_2x2x1"], mesh=mesh, n_ao=n_lo, seed=seed)
    h = synth.mean_field_hamiltonian(spec, n_occ)
    return spec, h, synth.mean_field_density(h, mesh, n_occ)


@pytest.mark.parametrize("mesh", MESHES)
def test_offdiag_density_is_the_supercell_block(mesh):
    spec, h, g = _case(mesh)
    n = spec.n_ao
    G = oracle.supercell_density(h, mesh, 3 * spec.nk)
    g0 = oracle.offdiag_density(g, mesh)
    for r in range(spec.nk):
        np.testing.assert_allclose(g0[r], G[r * n:(r + 1) * n, :n], atol=1e-13)
    assert np.abs(g0.imag).max() < 1e-13


@pytest.mark.parametrize("mesh", MESHES)
def test_singular_values_closed_form(mesh):
    # Gamma idempotent: sum_{R != 0} gamma^{0,R} gamma^{R,0} = gamma^{00} - (gamma^{00})^2, so the
    # squared singular values on the columns val are the eigenvalues of that matrix on val x val.
    spec, h, g = _case(mesh)
    val = [0, 2, 3, 5]
    _, s, max_imag = oracle.bath_svd(g, mesh, val)
    G = oracle.supercell_density(h, mesh, 3 * spec.nk)
    g00 = G[:spec.n_ao, :spec.n_ao]
    ev = np.sort(np.linalg.eigvalsh((g00 - g00 @ g00)[np.ix_(val, val)]))[::-1]
    np.testing.assert_allclose(s, np.sqrt(np.maximum(ev, 0.0)), rtol=1e-10, atol=1e-14)
    assert np.all(np.diff(s) <= 0)
    assert max_imag < 1e-13


@pytest.mark.parametrize("mesh", MESHES)
def test_bath_span_matches_supercell_svd(mesh):
    spec, h, g = _case(mesh)
    val = [1, 4, 5]
    B, s, _ = oracle.bath_svd(g, mesh, val)
    u, s2 = oracle.supercell_bath(oracle.supercell_density(h, mesh, 3 * spec.nk), spec.n_ao, val)
    np.testing.assert_allclose(s, s2, rtol=1e-12)
    b = B.reshape(-1, len(val))
    np.testing.assert_allclose(b @ b.T, u @ u.T, atol=1e-12)


def test_bath_orthonormal_and_sign_convention():
    _, _, g = _case((3, 2, 1))
    B, _, _ = oracle.bath_svd(g, (3, 2, 1), [0, 1, 2, 3, 4])
    b = B.reshape(-1, 5)
    np.testing.assert_allclose(b.T @ b, np.eye(5), atol=1e-13)
    for t in range(5):
        assert b[np.argmax(np.abs(b[:, t])), t] > 0


@pytest.mark.parametrize("mesh", MESHES)
def test_bloch_sum_matches_generator(mesh):
    # Eq. "C loemb R" built from the supercell SVD, then the generator's own Bloch sum.
    spec, h, g = _case(mesh)
    n, val = spec.n_ao, [0, 3, 4]
    u, _ = oracle.supercell_bath(oracle.supercell_density(h, mesh, 3 * spec.nk), n, val)
    for t in range(u.shape[1]):
        if u[np.argmax(np.abs(u[:, t])), t] < 0:
            u[:, t] = -u[:, t]
    csc = np.zeros((spec.nk * n, n + len(val)))
    csc[:n, :n] = np.eye(n)
    csc[n:, n:] = u
    want = synth.bloch_orbitals(csc, mesh)
    B, _, _ = oracle.bath_svd(g, mesh, val)
    np.testing.assert_allclose(oracle.embedding_orbitals_lo(B, mesh), want, atol=1e-12)


@pytest.mark.parametrize("mesh", MESHES)
def test_embedding_orbitals_orthonormal_real_and_impurity_block(mesh):
    spec, h, g = _case(mesh)
    U = synth.lo_rotation(spec)
    C, s = oracle.embedding_orbitals(g, U, mesh, [0, 2, 5])
    assert C.shape == (spec.nk, spec.n_ao, spec.n_ao + 3)
    assert oracle.orthonormality_error(C) < 1e-13
    assert oracle.realness_error(C, mesh) < 1e-13
    np.testing.assert_allclose(C[:, :, :spec.n_ao], U, atol=1e-15)


@pytest.mark.parametrize("mesh", MESHES)
def test_full_impurity_embedding_space_holds_n_imp_electrons(mesh):
    # Every impurity column in the SVD: the embedding space is spanned by whole occupied and
    # virtual orbitals of the determinant (one electron per impurity-bath pair), so the projected
    # density matrix is idempotent with trace n_imp.
    spec, h, g = _case(mesh)
    n = spec.n_ao
    B, s, _ = oracle.bath_svd(g, mesh, list(range(n)))
    assert s.min() > 1e-6
    c = oracle.embedding_orbitals_lo(B, mesh)
    d = sum(c[k].conj().T @ g[k] @ c[k] for k in range(spec.nk)) / spec.nk
    np.testing.assert_allclose(d @ d, d, atol=1e-12)
    assert abs(np.trace(d).real - n) < 1e-11


def test_planted_fourier_sign_is_caught(monkeypatch):
    # The inverse transform with the wrong sign gives gamma^{-R,0}, which the supercell rejects.
    import oracle.bath as ob
    mesh = (3, 2, 1)
    spec, h, g = _case(mesh)
    good = ob._k_dot_r
    monkeypatch.setattr(ob, "_k_dot_r", lambda m: -good(m))
    g0 = ob.offdiag_density(g, mesh)
    G = oracle.supercell_density(h, mesh, 3 * spec.nk)
    n = spec.n_ao
    err = max(np.abs(g0[r] - G[r * n:(r + 1) * n, :n]).max() for r in range(spec.nk))
    assert err > 1e-3


def _hand_cases():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_bath.json")
    return json.load(open(path))["cases"]


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_hand_worked_examples(case):
    mesh, val = tuple(case["mesh"]), case["val"]
    gk = np.asarray(case["gamma_k"], dtype=np.complex128)
    g0 = oracle.offdiag_density(gk, mesh)
    g_rs = np.asarray(case["g_real_space"])
    nk = g_rs.shape[0]
    for r in range(nk):  # gamma^{R,0} = g(-R)
        np.testing.assert_allclose(g0[r], g_rs[(-r) % nk], atol=1e-15)
    B, s, _ = oracle.bath_svd(gk, mesh, val)
    np.testing.assert_allclose(s, case["sigma"], rtol=1e-14)
    np.testing.assert_allclose(B, np.asarray(case["bath"]), atol=1e-15)
    c = oracle.embedding_orbitals_lo(B, mesh)
    want = np.asarray(case["C_lo_eo_re"]) + 1j * np.asarray(case["C_lo_eo_im"])
    np.testing.assert_allclose(c, want, atol=1e-15)
