"""Brute-force real-space transformation over the Born-von Karman supercell.

With the embedding orbitals written in real space, orbital i = sum_{R, mu}
Csc[(R, mu), i] phi_{mu R}, and aux functions in every cell R0 of the supercell,
the density-fitted ERI of Eq. "density fitting" reads
    X[(P, R0), i, j] = sum_{R1 mu R2 nu} conj(Csc[(R1,mu), i]) (P R0 | mu R1, nu R2) Csc[(R2,nu), j],
    (ij|kl) = sum_{P, R0} X[(P,R0), i, j] X[(P,R0), k, l],
where translation invariance gives (P R0 | mu R1, nu R2) = B[P, mu, R1 - R0, nu, R2 - R0].
No k-points appear, so this pins the k-space method and all of its conventions.
"""
import numpy as np


def _cells(mesh):
    n1, n2, n3 = mesh
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return g.reshape(-1, 3)


def supercell_eri(B, mesh, Csc_a, Csc_b=None):
    """(ij|kl) [na, na, nb, nb] from B[P, mu, R1, nu, R2] and supercell orbitals (real or
    complex; the bra orbital of each pair is conjugated)."""
    Csc_b = Csc_a if Csc_b is None else Csc_b
    cells = _cells(mesh)
    nmesh = np.asarray(mesh)
    n_aux, n_ao, nk = B.shape[0], B.shape[1], B.shape[2]
    # B as [P, (R1, mu), (R2, nu)], matching the row order of Csc.
    Bt = B.transpose(0, 2, 1, 4, 3)
    xa, xb = [], []
    for r0 in cells:
        shifted = (cells - r0) % nmesh
        src = (shifted[:, 0] * nmesh[1] + shifted[:, 1]) * nmesh[2] + shifted[:, 2]
        Bs = Bt[:, src][:, :, :, src].reshape(n_aux, nk * n_ao, nk * n_ao)
        xa.append(np.matmul(Csc_a.conj().T[None], np.matmul(Bs, Csc_a)))
        xb.append(np.matmul(Csc_b.conj().T[None], np.matmul(Bs, Csc_b)))
    xa = np.concatenate(xa, 0)
    xb = np.concatenate(xb, 0)
    return np.tensordot(xa, xb, axes=([0], [0]))


def supercell_matrix(f, mesh):
    """Fsc[(R1, mu), (R2, nu)] = f[mu, nu, R2 - R1]: a translation-invariant one-particle operator
    written out over the supercell from its blocks f[:, :, R] between cell 0 and cell R."""
    cells = _cells(mesh)
    nmesh = np.asarray(mesh)
    n_ao, nk = f.shape[0], f.shape[2]
    Fsc = np.zeros((nk * n_ao, nk * n_ao), dtype=f.dtype)
    for a, r1 in enumerate(cells):
        d = (cells - r1) % nmesh
        idx = (d[:, 0] * nmesh[1] + d[:, 1]) * nmesh[2] + d[:, 2]
        for b in range(nk):
            Fsc[a * n_ao:(a + 1) * n_ao, b * n_ao:(b + 1) * n_ao] = f[:, :, idx[b]]
    return Fsc


def supercell_fock(f, mesh, Csc):
    """Csc^+ Fsc Csc with Fsc[(R1, mu), (R2, nu)] = f[mu, nu, R2 - R1]: the Fock matrix of the
    supercell orbitals, with no k-points (pins Eq. "fock transform" and its conventions)."""
    return Csc.conj().T @ supercell_matrix(f, mesh) @ Csc


def supercell_density(h, mesh, n_elec):
    """Gamma = sum over the n_elec lowest eigenvectors v of the supercell Hamiltonian built from
    h[i, j, R] of v v^T: the mean-field density matrix of the whole supercell, with no k-points."""
    w, v = np.linalg.eigh(supercell_matrix(h, mesh))
    occ = v[:, np.argsort(w, kind="stable")[:n_elec]]
    return occ @ occ.conj().T


def supercell_bath(Gamma, n_lo, val):
    """Left singular vectors and singular values of the block Gamma[(R != 0, i), (0, j in val)],
    taken straight from the supercell density matrix (Eq. "bath R SVD" without k-points)."""
    block = Gamma[n_lo:, :][:, list(val)]
    u, s, _ = np.linalg.svd(block, full_matrices=False)
    return u, s


def supercell_eri_grid(chi_R, Csc, mesh, lattice, grid):
    """(ij|kl) of the supercell orbitals psi_i(r) = sum_{R, mu} Csc[(R, mu), i] chi_R[R][mu](r), with
    chi_R the AOs of every cell on the supercell grid (N_d g_d points along a_d): the periodic Coulomb
    integral over the Born-von Karman supercell, Omega_sc sum_{G != 0} 4 pi / |G|^2 rho_ij(G) rho_kl(-G),
    rho(G) = (1/N) sum_r exp(-i G.r) rho(r), with the supercell's own reciprocal vectors. No k-points."""
    nk, na = chi_R.shape[0], chi_R.shape[1]
    big = tuple(int(m) * int(g) for m, g in zip(mesh, grid))
    npts = int(np.prod(big))
    a_sc = np.asarray(lattice, dtype=np.float64) * np.asarray(mesh, dtype=np.float64)[:, None]
    b_sc = 2.0 * np.pi * np.linalg.inv(a_sc).T
    omega_sc = abs(np.linalg.det(a_sc))
    psi = np.einsum("Rmi,Rmr->ir", Csc.reshape(nk, na, -1), chi_R)
    n = psi.shape[0]
    rho = psi.conj()[:, None, :] * psi[None, :, :]                     # [i][j][r]
    hat = np.fft.fftn(rho.reshape((n, n) + big), axes=(2, 3, 4)) / npts
    m = np.stack(np.meshgrid(*[np.fft.fftfreq(x) * x for x in big], indexing="ij"), -1)
    gv = m @ b_sc
    g2 = (gv * gv).sum(-1)
    v = np.zeros(g2.shape)
    v[g2 > 1e-12] = 4.0 * np.pi / g2[g2 > 1e-12]
    neg = np.roll(np.flip(hat, axis=(2, 3, 4)), 1, axis=(2, 3, 4))    # rho(-G)
    return omega_sc * np.einsum("ijG,klG->ijkl", (hat * v).reshape(n, n, -1), neg.reshape(n, n, -1))
