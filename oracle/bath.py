"""DMET bath and embedding orbitals, section 2.1, in plain FP64 (test infrastructure).

Eq. "bath R SVD": the block of the mean-field density matrix between the environment (every
cell R != 0) and the impurity (the LOs of the reference cell R = 0) is decomposed,
    gamma^{R != 0, 0}_{ij} = sum_t B^R_{it} Lambda_tt V^{0 +}_{tj},
with the impurity index j restricted to the valence LOs (the valence-only bath of the same
section, which gives n_imp + n_val embedding orbitals). The left singular vectors B^R are the
bath orbitals.
Eq. "C loemb R": C^{R,LO,EO} = [[1, 0], [0, B^{R != 0}]], impurity columns first (the identity on
the LOs of cell 0), bath columns after them.
Eq. "C loemb k": C^{k,LO,EO} = sum_R exp(-i k.R) C^{R,LO,EO} and C^{k,AO,EO} = C^{k,AO,LO} C^{k,LO,EO}.

Conventions, which the paper leaves open:
* gamma^k = sum_R exp(+i k.R) g(R), with g(R)_{ij} the density-matrix element between LO i of
  cell 0 and LO j of cell R (the convention of the Fock matrix F^k). Translation invariance
  then gives gamma^{R,0}_{ij} = g(-R)_{ij} = (1/Nk) sum_k exp(+i k.R) gamma^k_{ij}.
* The bath columns come in decreasing singular value. Each column's sign is chosen so that its
  largest-magnitude coefficient (the first one, in (R, i) order, of equal magnitudes) is positive.
* k.R = 2 pi sum_d n_d m_d / N_d, with k-points and cells in the C order of oracle.mesh.
"""
import numpy as np

from .mesh import k_triplet


def _k_dot_r(mesh):
    """[k, R] matrix of k.R on the mesh."""
    nk = int(np.prod(mesh))
    t = np.array([k_triplet(k, mesh) for k in range(nk)], dtype=np.float64)
    n = np.asarray(mesh, dtype=np.float64)
    return 2.0 * np.pi * (t[:, None, :] * t[None, :, :] / n).sum(-1)


def offdiag_density(gamma_k, mesh):
    """gamma^{R,0} [R, i, j] (complex; real when gamma^{-k} = conj gamma^k), every cell R."""
    nk = gamma_k.shape[0]
    kr = _k_dot_r(mesh)
    out = np.zeros(gamma_k.shape, dtype=np.complex128)
    for r in range(nk):
        for k in range(nk):
            out[r] += np.exp(1j * kr[k, r]) * gamma_k[k]
    return out / nk


def bath_svd(gamma_k, mesh, val):
    """Bath orbitals of Eq. "bath R SVD" on the valence columns val.

    Returns (B [Nk - 1, n_lo, n_val] real, the bath coefficient of LO i of cell R = b + 1;
    Lambda [n_val], decreasing; max |Im gamma^{R,0}| over the block)."""
    g = offdiag_density(gamma_k, mesh)
    nk, n_lo = g.shape[0], g.shape[1]
    block = g[1:, :, :][:, :, list(val)].reshape((nk - 1) * n_lo, len(val))
    max_imag = float(np.abs(block.imag).max()) if block.size else 0.0
    u, s, _ = np.linalg.svd(block.real, full_matrices=False)
    for t in range(u.shape[1]):
        a = int(np.argmax(np.abs(u[:, t])))
        if u[a, t] < 0:
            u[:, t] = -u[:, t]
    return u.reshape(nk - 1, n_lo, len(val)), s, max_imag


def embedding_orbitals_lo(B, mesh):
    """C^{k,LO,EO} [k, n_lo, n_lo + n_val] from the bath orbitals B [Nk - 1, n_lo, n_val]:
    Eq. "C loemb R" on every cell, then the Bloch sum of Eq. "C loemb k"."""
    nk = int(np.prod(mesh))
    n_lo, n_val = B.shape[1], B.shape[2]
    c_r = np.zeros((nk, n_lo, n_lo + n_val))
    c_r[0, :, :n_lo] = np.eye(n_lo)
    c_r[1:, :, n_lo:] = B
    kr = _k_dot_r(mesh)
    out = np.zeros((nk, n_lo, n_lo + n_val), dtype=np.complex128)
    for k in range(nk):
        for r in range(nk):
            out[k] += np.exp(-1j * kr[k, r]) * c_r[r]
    return out


def embedding_orbitals(gamma_k, C_ao_lo, mesh, val):
    """C^{k,AO,EO} [k, n_ao, n_lo + n_val] and Lambda [n_val]: the bath of Eq. "bath R SVD", the
    block form of Eq. "C loemb R" and the two transformations of Eq. "C loemb k"."""
    B, s, _ = bath_svd(gamma_k, mesh, val)
    c_lo = embedding_orbitals_lo(B, mesh)
    return np.matmul(C_ao_lo, c_lo), s
