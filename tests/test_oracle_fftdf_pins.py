"""Pins of the FFTDF oracle (Appendix B, Algorithm 2 and Eq. "FFTDF") against results that do not go
through it: the Coulomb integral of the real-space orbitals over the Born-von Karman supercell, done
with the supercell's own FFT grid and no k-points; symmetries, realness and positivity of the ERI;
planted mistakes in the oracle each fail the supercell pin."""
import numpy as np
import pytest

import synth
import oracle.fftdf as of
from oracle.supercell import supercell_eri_grid

# (mesh, grid): even and odd grids; N_d g_d odd on every axis in the last two
CASES = [((1, 1, 1), (4, 4, 4)), ((2, 1, 1), (4, 4, 4)), ((2, 2, 1), (3, 4, 3)), ((3, 1, 1), (3, 5, 3)),
         ((3, 3, 1), (3, 3, 5))]


def _setup(mesh, grid, complex_orbitals=False, n_emb=3, seed=0):
    spec = synth.GridSpec(tuple(mesh), 2, tuple(grid), n_emb=n_emb, seed=seed)
    rho = synth.pair_densities_k(spec)
    csc = synth.grid_orbitals(spec, complex_orbitals=complex_orbitals)
    chi = synth.ao_supercell(spec)
    chiR = np.stack([synth.shift_cells(chi, spec, R) for R in range(spec.nk)])
    return spec, rho, csc, chiR


@pytest.mark.parametrize("mesh,grid", CASES)
@pytest.mark.parametrize("complex_orbitals", [False, True])
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_fftdf_matches_supercell_coulomb(mesh, grid, complex_orbitals, ck_norm):
    spec, rho, csc, chiR = _setup(mesh, grid, complex_orbitals)
    C = synth.bloch_orbitals(csc, mesh, ck_norm)
    eri = of.embedded_eri_fftdf(rho, C, mesh, spec.lattice, grid, ck_norm)
    ref = supercell_eri_grid(chiR, csc, mesh, spec.lattice, grid)
    assert np.abs(eri - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("mesh,grid", CASES[3:])
def test_fftdf_real_symmetric_for_real_orbitals_on_odd_grids(mesh, grid):
    # With N_d g_d odd the plane-wave set is symmetric under G -> -G, so real orbitals give a real,
    # 8-fold symmetric ERI (with even sizes the Nyquist plane, present once, breaks that slightly in both
    # routes alike).
    spec, rho, csc, _ = _setup(mesh, grid)
    eri = of.embedded_eri_fftdf(rho, synth.bloch_orbitals(csc, mesh), mesh, spec.lattice, grid)
    scale = np.abs(eri).max()
    assert np.abs(eri.imag).max() < 1e-14 * scale
    e = eri.real
    for perm in ("jikl", "ijlk", "klij", "lkji"):
        assert np.abs(e - np.einsum("ijkl->" + perm, e)).max() < 1e-14 * scale


@pytest.mark.parametrize("mesh,grid", CASES)
def test_fftdf_pair_supermatrix_is_hermitian_psd(mesh, grid):
    spec, rho, csc, _ = _setup(mesh, grid, complex_orbitals=True, n_emb=4)
    eri = of.embedded_eri_fftdf(rho, synth.bloch_orbitals(csc, mesh), mesh, spec.lattice, grid)
    n = eri.shape[0]
    m = eri.transpose(0, 1, 3, 2).reshape(n * n, n * n)      # M[(ij),(lk)] = (ij|kl)
    assert np.abs(m - m.conj().T).max() < 1e-13 * np.abs(m).max()
    assert np.linalg.eigvalsh(0.5 * (m + m.conj().T)).min() > -1e-13 * np.abs(m).max()


def _mutant_error(monkeypatch, name, value, mesh=(3, 1, 1), grid=(3, 5, 3)):
    spec, rho, csc, chiR = _setup(mesh, grid)
    ref = supercell_eri_grid(chiR, csc, mesh, spec.lattice, grid)
    monkeypatch.setattr(of, name, value)
    eri = of.embedded_eri_fftdf(rho, synth.bloch_orbitals(csc, mesh), mesh, spec.lattice, grid)
    return np.abs(eri - ref).max() / np.abs(ref).max()


def test_planted_no_bloch_phase_is_caught(monkeypatch):
    # the pair's phase exp(i q.r) left in before the FFT
    assert _mutant_error(monkeypatch, "_grid_frac", lambda grid: np.zeros((int(np.prod(grid)), 3))) > 1e-3


def test_planted_kernel_without_q_is_caught(monkeypatch):
    good = of.coulomb_kernel
    assert _mutant_error(monkeypatch, "coulomb_kernel", lambda q, mesh, lat, grid: good(0, mesh, lat, grid)) > 1e-3


def test_planted_second_factor_at_plus_q_is_caught(monkeypatch):
    assert _mutant_error(monkeypatch, "k_neg", lambda q, mesh: q) > 1e-3


def test_planted_kernel_sign_of_q_is_caught(monkeypatch):
    good = of.coulomb_kernel
    from oracle.mesh import k_neg
    assert _mutant_error(monkeypatch, "coulomb_kernel",
                         lambda q, mesh, lat, grid: good(k_neg(q, mesh), mesh, lat, grid)) > 1e-3


@pytest.mark.parametrize("mesh,grid", CASES[3:])
def test_plane_wave_gdf_form_reproduces_algorithm_2(mesh, grid):
    # L^q_{G,ij} = (Omega v(q+G) / Nk)^(1/2) rho_hat^q_ij(G); the -q factor is taken at the plane wave
    # opposite to q + G. Then (ij|kl) = sum_q sum_G L^q_{G,ij} L^{-q}_{G',kl} and L^{-q}_{G',kl} =
    # conj L^q_{G,lk}: the form of Algorithm 1's contraction, with the plane waves as the aux set.
    from oracle.mesh import k_neg, k_triplet
    spec, rho, csc, _ = _setup(mesh, grid, complex_orbitals=True)
    C = synth.bloch_orbitals(csc, mesh)
    eri = of.embedded_eri_fftdf(rho, C, mesh, spec.lattice, grid)
    nk, ng, n = spec.nk, int(np.prod(grid)), C.shape[2]
    omega = abs(np.linalg.det(np.asarray(spec.lattice)))
    frac = (np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), -1).reshape(-1, 3)
            / np.asarray(grid))
    Lq = []
    for q in range(nk):
        t = np.asarray(k_triplet(q, mesh)) / np.asarray(mesh)
        r = of.embedded_3idx_grid(rho, C, mesh, q) * np.exp(-2j * np.pi * (frac @ t))[:, None, None]
        hat = np.fft.fftn(r.reshape(tuple(grid) + (n, n)), axes=(0, 1, 2)) / ng
        v = of.coulomb_kernel(q, mesh, spec.lattice, grid)
        Lq.append((np.sqrt(omega * v / nk)[..., None, None] * hat).reshape(ng, n, n))

    def opposite(q):
        t = k_triplet(q, mesh)
        ax = [(-np.arange(g) - (1 if t[d] else 0)) % g for d, g in enumerate(grid)]
        j = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
        return (j[:, 0] * grid[1] + j[:, 1]) * grid[2] + j[:, 2]

    gdf = sum(np.einsum("Gij,Gkl->ijkl", Lq[q], Lq[k_neg(q, mesh)][opposite(q)]) for q in range(nk))
    assert np.abs(gdf - eri).max() < 1e-13 * np.abs(eri).max()
    for q in range(nk):
        assert np.abs(Lq[k_neg(q, mesh)][opposite(q)] - Lq[q].transpose(0, 2, 1).conj()).max() < 1e-13 * np.abs(Lq[q]).max()


def test_supercell_coulomb_closed_form_for_plane_waves():
    # Orbitals psi_i = exp(i G_i . r) / sqrt(Omega): rho_ij has the single plane wave G_j - G_i, so
    # (ij|kl) = 4 pi / (Omega |G_j - G_i|^2) when G_j - G_i = -(G_l - G_k) != 0, and 0 otherwise.
    lat = np.asarray(((2.0, 0.0, 0.0), (0.3, 2.2, 0.0), (0.1, 0.2, 2.5)))
    grid = (5, 5, 5)
    b = 2.0 * np.pi * np.linalg.inv(lat).T
    omega = abs(np.linalg.det(lat))
    frac = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), -1).reshape(-1, 3) / np.asarray(grid)
    ms = np.array([(0, 0, 0), (1, 0, 0), (0, -1, 1), (-1, 1, 0)])
    chi = np.exp(2j * np.pi * (frac @ ms.T)).T / np.sqrt(omega)          # [i][r]
    eri = supercell_eri_grid(chi[None], np.eye(len(ms)), (1, 1, 1), lat, grid)
    want = np.zeros(eri.shape)
    for i, j, k, l in np.ndindex(eri.shape):
        d = ms[j] - ms[i]
        if np.array_equal(d, -(ms[l] - ms[k])) and np.any(d != 0):
            g = d @ b
            want[i, j, k, l] = 4.0 * np.pi / (omega * (g @ g))
    np.testing.assert_allclose(eri, want, atol=1e-12 * want.max())
