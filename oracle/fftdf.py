"""Algorithm 2 (embedding ERIs with FFTDF, Appendix B) in plain FP64 (test infrastructure).

The auxiliary set is the plane waves of the cell's FFT grid (Eq. "FFTDF"): the 3-index quantity is
the AO pair density on the real-space grid of the reference cell, rho^{k1,k2}_{mu nu}(r) =
conj(phi_{mu k1}(r)) phi_{nu k2}(r), with Bloch AOs phi_{mu k} = sum_R exp(+i k.R) chi_{mu R}.
Algorithm 2, for every q:
  1. (r|0i 0j) = (1/Nk) sum_{k1} C^{k1 +} rho^{k1, k1+q}(r) C^{k1+q}   (k-AO -> k-EO, FT to R = 0);
  2. FFT to G, multiply by the Coulomb kernel 4 pi / |q + G|^2, inverse FFT back to r;
  3. the same transform for the pairs of momentum -q;
  4. (ij|kl) += (1/Nk) sum_r (0i 0j|r) (r|0k 0l).

Conventions, which the paper leaves open (its Omega^2 and 4 pi / Omega go with a normalisation of
(mu nu|G) it does not spell out):
* grid points r = sum_d (j_d / g_d) a_d, reciprocal vectors b_d with a_d . b_e = 2 pi delta;
  q = sum_d (n_d / N_d) b_d, G = sum_d m_d b_d with m_d = j_d mod g_d chosen so that q + G is one of the
  signed FFT frequencies of the supercell grid (N_d g_d points along a_d);
* the forward transform removes the Bloch phase of the pair, rho_hat(G) = (1/N_g) sum_r
  exp(-i (q + G).r) rho(r), and the kernel is 4 pi / |q + G|^2, zero at q + G = 0 (the neutralising
  background);
* step 4 integrates over the cell with the grid's volume element Omega / N_g.
With these the method equals the Coulomb integral over the Born-von Karman supercell of the
real-space orbitals (pinned against oracle.supercell.supercell_eri_grid). With C^k scaled by
Nk^-1/2 (ck_norm = 1) step 1 has no 1/Nk.
"""
import numpy as np

from .mesh import k_add, k_neg, k_triplet


def _recip(lattice):
    """Rows b_d with a_d . b_e = 2 pi delta_de."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def _grid_frac(grid):
    g = np.asarray(grid)
    j = np.stack(np.meshgrid(*[np.arange(n) for n in g], indexing="ij"), -1).reshape(-1, 3)
    return j / g


def _g_index(n_k, g):
    """m[n][j]: the reciprocal-lattice index m (m = j mod g) for which n + N m is the supercell's signed
    FFT frequency, i.e. lies in [-floor(N g / 2), ceil(N g / 2) - 1]. q + G then runs over exactly the
    plane waves of the Born-von Karman supercell's own grid, Nyquist convention included."""
    out = np.zeros((n_k, g), dtype=np.int64)
    for s_ in (np.fft.fftfreq(n_k * g) * (n_k * g)).round().astype(np.int64):
        n = s_ % n_k
        m = (s_ - n) // n_k
        out[n, m % g] = m
    return out


def coulomb_kernel(q, mesh, lattice, grid):
    """4 pi / |q + G|^2 on the FFT grid (array of shape grid), 0 where q + G = 0."""
    b = _recip(lattice)
    t = k_triplet(q, mesh)
    idx = [_g_index(int(mesh[d]), int(grid[d]))[t[d]] for d in range(3)]
    m = np.stack(np.meshgrid(*idx, indexing="ij"), -1).astype(np.float64)
    v = (m + np.asarray(t, dtype=np.float64) / np.asarray(mesh)) @ b
    g2 = (v * v).sum(-1)
    out = np.zeros(g2.shape)
    nz = g2 > 1e-12
    out[nz] = 4.0 * np.pi / g2[nz]
    return out


def embedded_3idx_grid(rho, C, mesh, q, ck_norm=0):
    """(r|0i 0j) for momentum q: [N_g, n, n] (step 1 of Algorithm 2)."""
    nk = int(np.prod(mesh))
    scale = 1.0 / nk if ck_norm == 0 else 1.0
    n, ng = C.shape[2], rho.shape[-1]
    out = np.zeros((ng, n, n), dtype=np.complex128)
    for k1 in range(nk):
        k2 = k_add(k1, q, mesh)
        pair = np.einsum("mi,mnr,nj->rij", C[k1].conj(), rho[k1, k2], C[k2])
        out += scale * pair
    return out


def embedded_eri_fftdf(rho, C, mesh, lattice, grid, ck_norm=0):
    """(ij|kl) [n, n, n, n] (complex) by Algorithm 2."""
    nk = int(np.prod(mesh))
    grid = tuple(int(x) for x in grid)
    ng = int(np.prod(grid))
    omega = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    frac = _grid_frac(grid)
    n = C.shape[2]
    eri = np.zeros((n, n, n, n), dtype=np.complex128)
    for q in range(nk):
        t = np.asarray(k_triplet(q, mesh), dtype=np.float64) / np.asarray(mesh)
        phase = np.exp(-2j * np.pi * (frac @ t))                      # exp(-i q.r)
        rq = embedded_3idx_grid(rho, C, mesh, q, ck_norm)
        hat = np.fft.fftn((phase[:, None, None] * rq).reshape(grid + (n, n)), axes=(0, 1, 2)) / ng
        hat *= coulomb_kernel(q, mesh, lattice, grid)[..., None, None]
        w = np.fft.ifftn(hat, axes=(0, 1, 2)).reshape(ng, n, n) * ng * phase.conj()[:, None, None]
        rm = embedded_3idx_grid(rho, C, mesh, k_neg(q, mesh), ck_norm)
        eri += (omega / ng) / nk * np.einsum("rij,rkl->ijkl", w, rm)
    return eri
