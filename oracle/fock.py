"""The embedding one-particle Hamiltonian, section 2.1, in plain FP64 (test infrastructure).

Eq. "fock transform": the periodic mean-field Fock matrix F^{k,AO} is transformed to the
embedding orbitals and brought to the reference cell,
    F^{0,EO} = (1/Nk) sum_k C^{k,AO,EO +} F^{k,AO} C^{k,AO,EO},
with the Bloch-sum orbitals of Eq. "C loemb k" (ck_norm = 0); with C^k scaled by Nk^-1/2
(ck_norm = 1) the 1/Nk is already inside the orbitals.

Eq. "fock double counting": the mean-field Coulomb and exchange of the embedding density gamma,
evaluated with the embedding ERIs, are subtracted,
    Ftilde_ij = F^{0,EO}_ij - [ sum_kl (ij|kl) gamma_lk - 1/2 sum_kl (ik|lj) gamma_kl ],
with gamma spin-summed (restricted) and rotated to the embedding basis.
"""
import numpy as np


def fock_transform(F, C, ck_norm=0):
    """F^{0,EO} [n, n] (complex) from F[k, mu, nu] and C[k, mu, i]."""
    nk = F.shape[0]
    scale = 1.0 / nk if ck_norm == 0 else 1.0
    out = np.zeros((C.shape[2], C.shape[2]), dtype=np.complex128)
    for k in range(nk):
        out += scale * (C[k].conj().T @ F[k] @ C[k])
    return out


def coulomb_exchange(eri, gamma):
    """J_ij = sum_kl (ij|kl) gamma_lk and K_ij = sum_kl (ik|lj) gamma_kl, from the dense
    ERI [n, n, n, n] (chemists' notation)."""
    J = np.einsum("ijkl,lk->ij", eri, gamma)
    K = np.einsum("iklj,kl->ij", eri, gamma)
    return J, K


def embedded_fock(F0, eri, gamma):
    """Ftilde = F0 - (J - K / 2), Eq. "fock double counting"."""
    J, K = coulomb_exchange(eri, gamma)
    return F0 - (J - 0.5 * K)


def coulomb_exchange_df(Lq, gamma, mesh):
    """J and K straight from the density-fitted factors L^q (Algorithm 1's inner-loop output for
    every q, [q][P][i][j]), without forming the ERI: with (ij|kl) = (1/Nk) sum_q sum_P
    L^q_{P,ij} L^{-q}_{P,kl} (Algorithm 1's contraction),
        J_ij = (1/Nk) sum_q sum_P L^q_{P,ij} tr(L^{-q}_P gamma),
        K_ij = (1/Nk) sum_q sum_P (L^q_P gamma L^{-q}_P)_ij,
    the density-fitted use the paper mentions for solvers that take the factors directly."""
    from .mesh import k_neg
    nk = Lq.shape[0]
    J = np.zeros(gamma.shape, dtype=np.complex128)
    K = np.zeros(gamma.shape, dtype=np.complex128)
    for q in range(nk):
        a, b = Lq[q], Lq[k_neg(q, mesh)]
        for P in range(a.shape[0]):
            J += a[P] * np.trace(b[P] @ gamma) / nk
            K += a[P] @ gamma @ b[P] / nk
    return J, K
