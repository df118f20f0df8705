"""Algorithm 1 (embedding ERI transformation with GDF), section 2.1, in plain FP64.

Notation. L[k1, k2, P, mu, nu] = (P | mu k1, nu k2), the k-point density-fitted
3-index integrals of Eq. "density fitting"; C[k, mu, i] = C^{k,AO,EO}, the embedding
orbitals at k of Eq. "C loemb k". q = k2 - k1 is the momentum the pair (k1, k2)
transfers; Algorithm 1's k_L = k_mu - k_nu is -q, so looping over every k_L is
looping over every q.

Normalisation. With the Bloch sum of Eq. "C loemb k" (ck_norm = 0), Algorithm 1
divides by Nk once when it Fourier-transforms each transformed pair to the reference
cell and once more in the final contraction, which reproduces the real-space ERIs of
the embedding orbitals (pinned against the supercell transformation). With C^k scaled
by Nk^-1/2 (ck_norm = 1) the first division is dropped and only the contraction's
1/Nk remains.
"""
import numpy as np

from .mesh import k_add, k_neg


def embedded_3idx(L, C, mesh, qs=None, ck_norm=0):
    """(L | 0i 0j) at momentum transfer q, for every q in qs: array [len(qs), P, n, n].

    Algorithm 1's inner loop: for every momentum-conserving pair (k1, k2 = k1 + q),
    transform (L | mu k1, nu k2) to the embedding orbitals,
        (L | i k1, j k2) = sum_{mu nu} conj(C^{k1}_{mu i}) (L | mu k1, nu k2) C^{k2}_{nu j},
    and add it, divided by Nk, to the reference-cell factor.
    """
    nk = int(np.prod(mesh))
    qs = list(range(nk)) if qs is None else list(qs)
    n_aux, n = L.shape[2], C.shape[2]
    scale = 1.0 / nk if ck_norm == 0 else 1.0
    out = np.zeros((len(qs), n_aux, n, n), dtype=np.complex128)
    for iq, q in enumerate(qs):
        for k1 in range(nk):
            k2 = k_add(k1, q, mesh)
            right = np.matmul(L[k1, k2], C[k2])                  # [P, mu, j]
            pair = np.matmul(C[k1].conj().T[None, :, :], right)  # [P, i, j]
            out[iq] += scale * pair
    return out


def embedded_eri(L, Ca, mesh, Cb=None, ck_norm=0, Lq_a=None, Lq_b=None):
    """(ij|kl) with i, j orbitals of Ca and k, l orbitals of Cb: complex [na, na, nb, nb].

    Algorithm 1's contraction: (ij|kl) += (1/Nk) sum_P (0i0j | L)(L | 0k0l) for every
    aux momentum. By momentum conservation the pair (k, l) carries the opposite
    transfer, so the q factor of (i, j) meets the -q factor of (k, l).
    """
    nk = int(np.prod(mesh))
    if Lq_a is None:
        Lq_a = embedded_3idx(L, Ca, mesh, ck_norm=ck_norm)
    if Lq_b is None:
        Lq_b = Lq_a if Cb is None else embedded_3idx(L, Cb, mesh, ck_norm=ck_norm)
    na, nb = Lq_a.shape[2], Lq_b.shape[2]
    eri = np.zeros((na, na, nb, nb), dtype=np.complex128)
    for q in range(nk):
        eri += np.tensordot(Lq_a[q], Lq_b[k_neg(q, mesh)], axes=([0], [0])) / nk
    return eri


def eri_entries(Lq_a, Lq_b, mesh, idx):
    """Selected (ij|kl) from the per-q factors of all q; idx is an int array [m, 4]."""
    nk = int(np.prod(mesh))
    idx = np.asarray(idx)
    i, j, k, l = idx.T
    total = np.zeros(len(idx), dtype=np.complex128)
    for q in range(nk):
        a = Lq_a[q][:, i, j]                       # [P, m]
        b = Lq_b[k_neg(q, mesh)][:, k, l]          # [P, m]
        total += (a * b).sum(0) / nk
    return total
