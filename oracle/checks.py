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


# ---- 4-fold packing of a complex ERI (the paper fixes no order; this is the library's) ----
# A complex same-spin ERI has (ij|kl) = (kl|ij) and (ij|kl) = conj((ji|lk)). Every entry is then
# stored once, possibly as the conjugate of the stored value, in one of two blocks:
#   A: i >= j, k >= l, IJ >= KL (IJ = i(i+1)/2 + j), at IJ(IJ+1)/2 + KL;
#   B: i > j, k < l, a >= b with a = i(i-1)/2 + j and b = l(l-1)/2 + k, at nA + a(a+1)/2 + b,
#      nA = np(np+1)/2, np = n(n+1)/2.
# The alpha-beta block has only the conjugation symmetry: (ij|kl) for i >= j and every (k, l), at
# IJ n_b^2 + k n_b + l.


def s4_size(n):
    np_, ns = n * (n + 1) // 2, n * (n - 1) // 2
    return np_ * (np_ + 1) // 2 + ns * (ns + 1) // 2


def _s4_home(i, j, k, l, n):
    """(position, conjugate?) of (ij|kl) in the 4-fold layout, case by case from the definition."""
    np_ = n * (n + 1) // 2
    nA = np_ * (np_ + 1) // 2
    if i >= j and k >= l:                          # block A
        I, K = i * (i + 1) // 2 + j, k * (k + 1) // 2 + l
        I, K = max(I, K), min(I, K)
        return I * (I + 1) // 2 + K, False
    if i < j and k < l:                            # (ij|kl) = conj((ji|lk))
        p, c = _s4_home(j, i, l, k, n)
        return p, not c
    if i < j:                                      # k >= l: (ij|kl) = (kl|ij)
        return _s4_home(k, l, i, j, n)
    if i == j:                                     # k < l: (ii|kl) = conj((ii|lk))
        p, c = _s4_home(i, i, l, k, n)
        return p, not c
    a, b = i * (i - 1) // 2 + j, l * (l - 1) // 2 + k   # i > j, k < l: block B
    if a >= b:
        return nA + a * (a + 1) // 2 + b, False
    return nA + b * (b + 1) // 2 + a, True          # (ij|kl) = conj((lk|ji)), a' = b, b' = a


def pack_s4(eri):
    """The 4-fold packed array (complex) of a same-spin complex ERI [n, n, n, n]."""
    n = eri.shape[0]
    np_ = n * (n + 1) // 2
    nA = np_ * (np_ + 1) // 2
    out = np.zeros(s4_size(n), dtype=np.complex128)
    for i in range(n):
        for j in range(i + 1):
            I = i * (i + 1) // 2 + j
            for k in range(n):
                for l in range(k + 1):
                    K = k * (k + 1) // 2 + l
                    if I >= K:
                        out[I * (I + 1) // 2 + K] = eri[i, j, k, l]
    for i in range(n):
        for j in range(i):
            a = i * (i - 1) // 2 + j
            for l in range(n):
                for k in range(l):
                    b = l * (l - 1) // 2 + k
                    if a >= b:
                        out[nA + a * (a + 1) // 2 + b] = eri[i, j, k, l]
    return out


def unpack_s4(packed, n):
    """The full complex ERI [n, n, n, n] from its 4-fold packed form (the symmetries filled in)."""
    full = np.zeros((n, n, n, n), dtype=np.complex128)
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for l in range(n):
                    p, conj = _s4_home(i, j, k, l, n)
                    full[i, j, k, l] = np.conj(packed[p]) if conj else packed[p]
    return full


def pack_s4_ab(eri_ab):
    """The packed alpha-beta block (complex): (ij|kl) for i >= j and every (k, l)."""
    na, nb = eri_ab.shape[0], eri_ab.shape[2]
    ia, ja = np.tril_indices(na)
    return np.ascontiguousarray(eri_ab[ia, ja].reshape(-1))
