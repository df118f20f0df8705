"""Input checks and the packed output format, written from their definitions.

* Orthonormality of the embedding orbitals: with the Bloch sum of Eq. "C loemb k",
  (1/Nk) sum_k C^k+ C^k = 1 (the normalisation Eq. "fock transform" implies with
  F = S = 1); with unitary-normalised C^k, sum_k C^k+ C^k = 1.
* Real orbitals (section 2.1: bottom-up local orbitals are real when phases are
  smooth): C^{-k} = conj(C^k).
* 8-fold packing of a real ERI (the paper fixes no order; this is the library's):
  pair index IJ = i(i+1)/2 + j for i >= j, packed index IJ(IJ+1)/2 + KL for IJ >= KL.
"""
import numpy as np

from .mesh import k_neg


def orthonormality_error(C, ck_norm=0):
    nk = C.shape[0]
    s = np.einsum("kmi,kmj->ij", C.conj(), C)
    if ck_norm == 0:
        s = s / nk
    return float(np.abs(s - np.eye(C.shape[2])).max())


def realness_error(C, mesh):
    nk = C.shape[0]
    return float(max(np.abs(C[k_neg(k, mesh)] - C[k].conj()).max() for k in range(nk)))


def pair_matrix(eri_ab):
    """M[IJ, KL] = (ij|kl) over lower-triangle pairs i >= j, k >= l."""
    na, nb = eri_ab.shape[0], eri_ab.shape[2]
    ia, ja = np.tril_indices(na)
    ib, jb = np.tril_indices(nb)
    return eri_ab[ia, ja][:, ib, jb]


def pack_s8(eri):
    """Packed lower triangle of the pair matrix of a real, 8-fold symmetric ERI."""
    m = pair_matrix(eri)
    return m[np.tril_indices(m.shape[0])]


def unpack_s8(packed, n):
    """Full [n, n, n, n] real ERI from its 8-fold packed form."""
    npair = n * (n + 1) // 2
    m = np.zeros((npair, npair))
    r, c = np.tril_indices(npair)
    m[r, c] = packed
    m[c, r] = packed
    i, j = np.tril_indices(n)
    full = np.zeros((n, n, n, n))
    for a, (p, q) in enumerate(zip(i, j)):
        row = np.zeros((n, n))
        row[i, j] = m[a]
        row[j, i] = m[a]
        full[p, q] = row
        full[q, p] = row
    return full
