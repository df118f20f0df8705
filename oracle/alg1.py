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


def _embedded_3idx_block(Lb, C, mesh, scale):
    """Algorithm 1's inner loop for one block of aux functions: Lb[k1, k2, P, mu, nu] holds every
    (k1, k2) pair of the block; returns [Nk (q), P, n, n]. The same sums as embedded_3idx, with the
    block's P rows stacked into one matrix product per pair (a library GEMM per step)."""
    nk, pb, na = Lb.shape[0], Lb.shape[2], Lb.shape[3]
    n = C.shape[2]
    out = np.zeros((nk, pb, n, n), dtype=np.complex128)
    for q in range(nk):
        for k1 in range(nk):
            k2 = k_add(k1, q, mesh)
            right = (Lb[k1, k2].reshape(pb * na, na) @ C[k2]).reshape(pb, na, n)       # [P, mu, j]
            pair = C[k1].conj().T @ right.transpose(1, 0, 2).reshape(na, pb * n)      # [i, (P, j)]
            out[q] += scale * pair.reshape(n, pb, n).transpose(1, 0, 2)
    return out


def embedded_eri_pblocks(L_blocks, Cs, mesh, ck_norm=0):
    """Algorithm 1 with L supplied block by block over the aux index (section 2.1 loads the
    3-index integrals from disk blockwise): the contraction sums over P, so each block's
    transformed factors are contracted and added on their own.

    L_blocks: iterable of arrays [Nk, Nk, Pb, n_ao, n_ao] (every (k1, k2) pair of a block of aux
    functions; the blocks together cover every P once). Cs: orbitals per spin, [Nk, n_ao, n_s].
    Returns {(sa, sb): complex [n_sa, n_sa, n_sb, n_sb]} for sa <= sb, (i j) of spin sa and (k l) of
    spin sb."""
    nk = int(np.prod(mesh))
    scale = 1.0 / nk if ck_norm == 0 else 1.0
    ns = len(Cs)
    out = {(a, b): np.zeros((Cs[a].shape[2],) * 2 + (Cs[b].shape[2],) * 2, dtype=np.complex128)
           for a in range(ns) for b in range(a, ns)}
    for Lb in L_blocks:
        lq = [_embedded_3idx_block(Lb, C, mesh, scale) for C in Cs]
        for (a, b), eri in out.items():
            for q in range(nk):
                eri += np.tensordot(lq[a][q], lq[b][k_neg(q, mesh)], axes=([0], [0])) / nk
    return out
