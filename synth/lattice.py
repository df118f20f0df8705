"""Seeded synthetic lattice inputs for the embedded-ERI transformation.

This module builds the inputs of the lattice-to-embedded integral transformation
(Cui, Zhu & Chan, arXiv 1909.08596, section 2.1, Algorithm 1): the k-point
density-fitted 3-index integrals L^{k1,k2}_{P,mu nu} and the embedding orbitals
C^k (n_AO x n_emb per k). It holds none of the transformation's arithmetic:
it draws real-space tensors, orthonormalises the orbitals over the Born-von Karman
supercell and Fourier-transforms both to the k mesh. Both the CPU oracle and the
CUDA path consume what it returns.

Conventions (section 2.1, Eq. "C loemb k" and Eq. "density fitting"):

* k-points and cells share the C-order index kappa(n1,n2,n3) = (n1*N2 + n2)*N3 + n3
  on a Gamma-centred N1 x N2 x N3 mesh; k.R = 2 pi sum_d n_d m_d / N_d.
* Real-space 3-index tensor B[P, mu, R1, nu, R2] = (P, cell 0 | mu R1, nu R2), real,
  symmetric under the pair swap (mu,R1) <-> (nu,R2).
* L^{k1,k2}_{P,mu nu} = sum_{R1,R2} exp(-i k1.R1 + i k2.R2) B[P, mu, R1, nu, R2],
  so that L^{k2,k1}_{P,nu mu} = conj(L^{k1,k2}_{P,mu nu}) and, because B is real,
  L^{-k1,-k2} = conj(L^{k1,k2}).
* Supercell orbitals Csc[(R, mu), i], real and orthonormal over the supercell;
  C^k_{mu i} = sum_R exp(-i k.R) Csc[(R, mu), i] (the Bloch sum of Eq. "C loemb k",
  "paper" normalisation, Nk^-1 sum_k C^k+ C^k = 1), or that times Nk^-1/2
  ("unitary" normalisation, sum_k C^k+ C^k = 1).

Random numbers: the 3-index tensor B, the bulk of every input, is drawn from a counter-based
generator defined here (SplitMix64 of Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014, used as a hash of (seed, stream, counter), with the Box-Muller
transform), so that any P-block regenerates identically on its own and a device implementation
of the same definition (synth.gpu, for workloads whose L is too large to draw on the host) gives
the same numbers up to the last-bit rounding of log and cos. The orbitals and the other small
inputs come from numpy's counter-based Philox generator keyed by (seed, stream).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.fft

# Philox stream identifiers (second key word); the P index is added for B.
_STREAM_B = 1 << 40
_STREAM_C = 2 << 40
_STREAM_SCALE = 3 << 40
_STREAM_BATH = 4 << 40
_STREAM_FOCK = 5 << 40
_STREAM_DM = 6 << 40


@dataclasses.dataclass(frozen=True)
class LatticeSpec:
    """Shape and value recipe of one synthetic embedding problem."""

    mesh: tuple            # (N1, N2, N3), Gamma-centred
    n_ao: int              # AOs per cell
    n_aux: int             # auxiliary functions per cell (the P index)
    n_emb: int             # embedding orbitals per spin
    n_spin: int = 1        # 1 restricted, 2 unrestricted
    decay: float = 0.7     # a in exp(-a (|R1| + |R2|))
    c_log_range: float = 0.0  # >0: orbital entries scaled by 10**U(-c_log_range, 0)
    seed: int = 0
    name: str = ""

    @property
    def nk(self) -> int:
        return int(np.prod(self.mesh))


# Shapes of the paper's three solids (section 2.2: h-BN 6x6x1, Si 4x4x4, NiO 4x4x4
# meshes; aux basis about ten times the AO basis) plus a tiny case.
CONFIGS = {
    "tiny_2x2x1": LatticeSpec((2, 2, 1), 8, 40, 16, 1, 0.7, 0.0, 0, "tiny_2x2x1"),
    "hbn_6x6x1": LatticeSpec((6, 6, 1), 26, 220, 104, 1, 0.5, 0.0, 1000, "hbn_6x6x1"),
    # the same cell on a 4x4x1 mesh (L = 0.61 GB): the case the profiler captures kernel by kernel
    "hbn_4x4x1": LatticeSpec((4, 4, 1), 26, 220, 104, 1, 0.5, 0.0, 1100, "hbn_4x4x1"),
    "si_4x4x4": LatticeSpec((4, 4, 4), 52, 400, 200, 1, 0.6, 4.0, 2000, "si_4x4x4"),
    "nio_4x4x4_uhf": LatticeSpec((4, 4, 4), 104, 900, 300, 2, 0.6, 0.0, 3000, "nio_4x4x4_uhf"),
    # a few GB on the device with the NiO-shaped aux basis (900 per cell, K = 14 400): the case the
    # profiler captures kernel by kernel in place of the 270 GB NiO-shaped run
    "nio_proxy_4x4x1": LatticeSpec((4, 4, 1), 52, 900, 128, 1, 0.6, 0.0, 3500, "nio_proxy_4x4x1"),
}


# Meshes of the batched workload (Nk = 8, 27, 36, 64).
BATCH_MESHES = {8: (2, 2, 2), 27: (3, 3, 3), 36: (6, 6, 1), 64: (4, 4, 4)}


def batch_specs(n_problems: int = 48, seed: int = 4000, n_ao_range=(6, 12), n_emb_range=(16, 48),
                decay: float = 0.7):
    """Seeded list of uneven embedding problems: Nk drawn from {8, 27, 36, 64}, n_AO uniform in
    n_ao_range, n_aux = floor(8.5 n_AO + 1/2), n_emb uniform in n_emb_range (capped at Nk n_AO),
    every other problem unrestricted."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 5 << 40]))
    out = []
    for p in range(n_problems):
        nk = int(rng.choice([8, 27, 36, 64]))
        nao = int(rng.integers(n_ao_range[0], n_ao_range[1] + 1))
        naux = int(math.floor(8.5 * nao + 0.5))
        n = int(rng.integers(n_emb_range[0], min(n_emb_range[1], nk * nao) + 1))
        out.append(LatticeSpec(BATCH_MESHES[nk], nao, naux, n, 1 + (p % 2), decay, 0.0, seed * 100 + p,
                               f"batch{n_problems}_{p}"))
    return out


def cell_vectors(mesh) -> np.ndarray:
    """Integer cell vectors m = (m1, m2, m3) in C order, shape (Nk, 3)."""
    n1, n2, n3 = mesh
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return g.reshape(-1, 3)


def min_image_norm(mesh) -> np.ndarray:
    """|R| of each cell: Euclidean norm of the minimum-image integer vector."""
    m = cell_vectors(mesh).astype(np.float64)
    n = np.asarray(mesh, dtype=np.float64)
    m = np.where(m > n / 2, m - n, m)
    return np.sqrt((m * m).sum(-1))


def phases(mesh) -> np.ndarray:
    """E[k, R] = exp(-i k.R) with k.R = 2 pi sum_d n_d m_d / N_d."""
    v = cell_vectors(mesh).astype(np.float64)
    n = np.asarray(mesh, dtype=np.float64)
    kr = 2.0 * np.pi * (v[:, None, :] * v[None, :, :] / n).sum(-1)
    return np.exp(-1j * kr)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


# SplitMix64 (Steele, Lea & Flood 2014): state increment and output mixing constants.
SM_GAMMA = 0x9E3779B97F4A7C15
SM_M1 = 0xBF58476D1CE4E5B9
SM_M2 = 0x94D049BB133111EB
_U64 = (1 << 64) - 1


def _sm_mix_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * SM_M1) & _U64
    z = ((z ^ (z >> 27)) * SM_M2) & _U64
    return z ^ (z >> 31)


def counter_key(seed: int, stream: int) -> int:
    """Key of one stream: k0 = mix(seed + gamma), key = mix(k0 + (stream + 1) gamma), mod 2^64."""
    k0 = _sm_mix_int((int(seed) + SM_GAMMA) & _U64)
    return _sm_mix_int((k0 + (int(stream) + 1) * SM_GAMMA) & _U64)


def counter_normals(seed: int, stream: int, start: int, count: int, out: np.ndarray | None = None,
                    chunk: int = 1 << 20) -> np.ndarray:
    """Normals t = start .. start + count - 1 of stream (seed, stream).

    Normal t is the Box-Muller transform of the SplitMix64 outputs h(2t) and h(2t + 1), where
    h(c) = mix(key + (c + 1) gamma) (mod 2^64) and mix is SplitMix64's output function:
    u1 = (floor(h(2t) / 2^11) + 1) 2^-53 in (0, 1], u2 = floor(h(2t + 1) / 2^11) 2^-53 in [0, 1),
    z = sqrt(-2 ln u1) cos(2 pi u2)."""
    key = np.uint64(counter_key(seed, stream))
    if out is None:
        out = np.empty(count)
    g, m1, m2 = np.uint64(SM_GAMMA), np.uint64(SM_M1), np.uint64(SM_M2)
    for c0 in range(0, count, chunk):
        m = min(chunk, count - c0)
        t0 = start + c0
        c = np.arange(2 * t0 + 1, 2 * (t0 + m) + 1, dtype=np.uint64)   # c + 1 for c = 2t, 2t + 1
        c *= g
        c += key
        c ^= c >> np.uint64(30)
        c *= m1
        c ^= c >> np.uint64(27)
        c *= m2
        c ^= c >> np.uint64(31)
        c >>= np.uint64(11)
        f = c.view(np.int64).astype(np.float64).reshape(m, 2)
        u1 = (f[:, 0] + 1.0) * 2.0 ** -53
        r = np.log(u1)
        r *= -2.0
        np.sqrt(r, out=r)
        u2 = f[:, 1] * (2.0 ** -53 * 2.0 * np.pi)
        np.cos(u2, out=u2)
        np.multiply(r, u2, out=out[c0:c0 + m])
    return out


def real_space_B(spec: LatticeSpec, p_begin: int = 0, p_end: int | None = None) -> np.ndarray:
    """B[P, mu, R1, nu, R2] for P in [p_begin, p_end), real, pair-symmetrised.

    Entries are N(0,1) * exp(-a (|R1| + |R2|)); then B <- (B + B^T_pair) / 2 with the
    pair transpose (mu, R1) <-> (nu, R2). Aux function P draws its N(0,1) numbers, in C order
    over (mu, R1, nu, R2), from stream _STREAM_B + P of counter_normals.
    """
    p_end = spec.n_aux if p_end is None else p_end
    nk, na = spec.nk, spec.n_ao
    w = np.exp(-spec.decay * min_image_norm(spec.mesh))
    per = na * nk * na * nk
    out = np.empty((p_end - p_begin, na, nk, na, nk))
    b = np.empty(per)
    for p in range(p_begin, p_end):
        counter_normals(spec.seed, _STREAM_B + p, 0, per, out=b)
        g = b.reshape(na, nk, na, nk)
        g *= w[None, :, None, None]
        g *= w[None, None, None, :]
        out[p - p_begin] = 0.5 * (g + g.transpose(2, 3, 0, 1))
    return out


def fourier_L(Bblk: np.ndarray, mesh, workers: int = -1) -> np.ndarray:
    """L[k1, k2, P, mu, nu] = sum_{R1,R2} exp(-i k1.R1 + i k2.R2) B[P, mu, R1, nu, R2]."""
    npb, na, nk, _, _ = Bblk.shape
    n1, n2, n3 = mesh
    x = Bblk.reshape(npb, na, n1, n2, n3, na, n1, n2, n3)
    # exp(-i k.R) over R1 is the forward DFT; exp(+i k.R) over R2 is the unscaled inverse.
    x = scipy.fft.fftn(x, axes=(2, 3, 4), workers=workers)
    x = scipy.fft.ifftn(x, axes=(6, 7, 8), norm="forward", workers=workers)
    x = x.reshape(npb, na, nk, na, nk)
    return np.ascontiguousarray(x.transpose(2, 4, 0, 1, 3))


def make_L(spec: LatticeSpec, p_block: int = 64, out: np.ndarray | None = None) -> np.ndarray:
    """Full L[k1][k2][P][mu][nu], complex128, generated P-block by P-block."""
    nk, na = spec.nk, spec.n_ao
    if out is None:
        out = np.empty((nk, nk, spec.n_aux, na, na), dtype=np.complex128)
    for p0 in range(0, spec.n_aux, p_block):
        p1 = min(spec.n_aux, p0 + p_block)
        out[:, :, p0:p1] = fourier_L(real_space_B(spec, p0, p1), spec.mesh)
    return out


def _orthonormalise(a: np.ndarray) -> np.ndarray:
    """Householder QR; column phases chosen so that diag(R) is real and positive."""
    q, r = np.linalg.qr(a)
    d = np.diag(r)
    s = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return q * s.conj()[None, :]


def supercell_orbitals(spec: LatticeSpec, spin: int = 0) -> np.ndarray:
    """Csc[(R, mu), i], real, orthonormal over the supercell, shape (Nk*n_AO, n_emb).

    Entries N(0,1) * exp(-a |R|) (times 10**U(-c, 0) when c_log_range = c > 0), then QR.
    """
    nk, na, n = spec.nk, spec.n_ao, spec.n_emb
    if n > nk * na:
        raise ValueError("n_emb exceeds the supercell dimension Nk*n_AO")
    g = _rng(spec.seed + spin, _STREAM_C)
    a = g.standard_normal((nk, na, n))
    a *= np.exp(-spec.decay * min_image_norm(spec.mesh))[:, None, None]
    if spec.c_log_range > 0:
        a *= 10.0 ** _rng(spec.seed + spin, _STREAM_SCALE).uniform(-spec.c_log_range, 0.0, (nk, na, n))
    return _orthonormalise(a.reshape(nk * na, n))


def complex_supercell_orbitals(spec: LatticeSpec, spin: int = 0) -> np.ndarray:
    """Complex Csc[(R, mu), i], orthonormal over the supercell (entries (N(0,1) + i N(0,1)) *
    exp(-a |R|), then QR). Their Bloch sums are orthonormal but not time-reversal symmetric."""
    nk, na, n = spec.nk, spec.n_ao, spec.n_emb
    g = _rng(spec.seed + spin, _STREAM_C + 7)
    a = g.standard_normal((nk, na, n)) + 1j * g.standard_normal((nk, na, n))
    a *= np.exp(-spec.decay * min_image_norm(spec.mesh))[:, None, None]
    return _orthonormalise(a.reshape(nk * na, n))


def dmet_structured_orbitals(spec: LatticeSpec, n_imp: int | None = None, spin: int = 0) -> np.ndarray:
    """Csc in the block form of Eq. "C loemb R": impurity columns are unit vectors on
    the first n_imp AOs of cell R = 0; bath columns are orthonormal and live on R != 0."""
    nk, na, n = spec.nk, spec.n_ao, spec.n_emb
    n_imp = min(na, n) if n_imp is None else n_imp
    n_bath = n - n_imp
    if n_bath > (nk - 1) * na:
        raise ValueError("bath larger than the environment")
    csc = np.zeros((nk * na, n))
    csc[np.arange(n_imp), np.arange(n_imp)] = 1.0
    if n_bath:
        g = _rng(spec.seed + spin, _STREAM_BATH)
        b = g.standard_normal(((nk - 1) * na, n_bath))
        csc[na:, n_imp:] = _orthonormalise(b)
    return csc


def bloch_orbitals(csc: np.ndarray, mesh, ck_norm: int = 0) -> np.ndarray:
    """C[k, mu, i] = sum_R exp(-i k.R) Csc[(R, mu), i] (times Nk^-1/2 if ck_norm == 1)."""
    nk = int(np.prod(mesh))
    na = csc.shape[0] // nk
    c = np.einsum("kR,Rmi->kmi", phases(mesh), csc.reshape(nk, na, -1))
    if ck_norm == 1:
        c /= math.sqrt(nk)
    return np.ascontiguousarray(c)


def make_problem(spec: LatticeSpec, ck_norm: int = 0, with_L: bool = True):
    """(L, [C_alpha, C_beta?], [Csc_alpha, ...]) for one problem."""
    cscs = [supercell_orbitals(spec, s) for s in range(spec.n_spin)]
    cs = [bloch_orbitals(c, spec.mesh, ck_norm) for c in cscs]
    L = make_L(spec) if with_L else None
    return L, cs, cscs


def real_space_fock(spec: LatticeSpec, spin: int = 0) -> np.ndarray:
    """f[mu, nu, R], real: the mean-field Fock matrix between AO mu of cell 0 and AO nu of cell R.

    Entries N(0,1) * exp(-a |R|), then symmetrised so that f[nu, mu, -R] = f[mu, nu, R] (a
    real, Hermitian one-particle operator that is invariant under lattice translations).
    """
    nk, na = spec.nk, spec.n_ao
    g = _rng(spec.seed + spin, _STREAM_FOCK).standard_normal((na, na, nk))
    g *= np.exp(-spec.decay * min_image_norm(spec.mesh))[None, None, :]
    cells = cell_vectors(spec.mesh)
    n = np.asarray(spec.mesh)
    neg = (-cells) % n
    neg_idx = (neg[:, 0] * n[1] + neg[:, 1]) * n[2] + neg[:, 2]
    return 0.5 * (g + g.transpose(1, 0, 2)[:, :, neg_idx])


def fock_k(f: np.ndarray, mesh) -> np.ndarray:
    """F[k, mu, nu] = sum_R exp(+i k.R) f[mu, nu, R]: the Fock matrix at k, Hermitian."""
    return np.ascontiguousarray(np.einsum("kR,mnR->kmn", phases(mesh).conj(), f))


def embedding_density(n: int, seed: int, n_occ: int | None = None) -> np.ndarray:
    """gamma [n, n], real symmetric with eigenvalues in [0, 2] (a spin-summed one-particle
    density matrix of the embedding space): 2 on n_occ random orthonormal directions, U(0, 2)
    on the others."""
    g = _rng(seed, _STREAM_DM)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    n_occ = n // 2 if n_occ is None else n_occ
    occ = np.concatenate([np.full(n_occ, 2.0), g.uniform(0.0, 2.0, n - n_occ)])
    return np.ascontiguousarray((q * occ[None, :]) @ q.T)


def spec_with(spec: LatticeSpec, **kw) -> LatticeSpec:
    return dataclasses.replace(spec, **kw)


_STREAM_MF = 7 << 40
_STREAM_LO = 8 << 40


def mean_field_hamiltonian(spec: LatticeSpec, n_occ: int, spin: int = 0, hop: float = 0.9) -> np.ndarray:
    """h[i, j, R], real: a gapped, translation-invariant one-particle Hamiltonian on the n_AO
    localized orbitals of every cell (the LO basis of section 2.1).

    On-site energies are -1 on n_occ LOs drawn at random and +1 on the others. Every other
    element is N(0,1) exp(-a |R|), symmetrised so that h[j, i, -R] = h[i, j, R], and the whole
    perturbation is scaled so that the sum over R of its spectral norms is hop < 1. Each k then
    has exactly n_occ levels below zero, so the lowest n_occ bands are separated by a gap of at
    least 2 (1 - hop) and filling them gives the same determinant as filling the Nk n_occ lowest
    levels of the supercell.
    """
    nk, na = spec.nk, spec.n_ao
    g = _rng(spec.seed + spin, _STREAM_MF)
    v = g.standard_normal((na, na, nk)) * np.exp(-spec.decay * min_image_norm(spec.mesh))[None, None, :]
    cells = cell_vectors(spec.mesh)
    n = np.asarray(spec.mesh)
    neg = (-cells) % n
    neg_idx = (neg[:, 0] * n[1] + neg[:, 1]) * n[2] + neg[:, 2]
    v = 0.5 * (v + v.transpose(1, 0, 2)[:, :, neg_idx])
    v[:, :, 0][np.diag_indices(na)] = 0.0
    norm = sum(np.linalg.norm(v[:, :, r], 2) for r in range(nk))
    v *= hop / max(norm, 1e-300)
    occ = g.permutation(na)[:n_occ]
    eps = np.ones(na)
    eps[occ] = -1.0
    v[:, :, 0] += np.diag(eps)
    return v


def mean_field_density(h: np.ndarray, mesh, n_occ: int) -> np.ndarray:
    """gamma[k, i, j] = sum over the n_occ lowest eigenvectors c of h^k of c c^+ (one spin; an
    idempotent density matrix), with h^k = sum_R exp(+i k.R) h[:, :, R] as for the Fock matrix."""
    hk = fock_k(h, mesh)
    out = np.empty_like(hk)
    for k in range(hk.shape[0]):
        w, c = np.linalg.eigh(hk[k])
        c = c[:, np.argsort(w, kind="stable")[:n_occ]]
        out[k] = c @ c.conj().T
    return out


def lo_rotation(spec: LatticeSpec, spin: int = 0, scale: float = 0.5) -> np.ndarray:
    """C^{k,AO,LO} [k, mu, i]: a unitary matrix at every k with C^{-k} = conj C^k (a real,
    orthogonal, translation-invariant AO-to-LO rotation of the supercell), the Cayley transform
    (1 - X^k)(1 + X^k)^-1 of X^k = sum_R exp(-i k.R) x(R), where x(R) is real, N(0,1) scale
    exp(-a |R|), made antisymmetric under x(-R) = -x(R)^T."""
    nk, na = spec.nk, spec.n_ao
    x = _rng(spec.seed + spin, _STREAM_LO).standard_normal((na, na, nk))
    x *= scale * np.exp(-spec.decay * min_image_norm(spec.mesh))[None, None, :]
    cells = cell_vectors(spec.mesh)
    n = np.asarray(spec.mesh)
    neg = (-cells) % n
    neg_idx = (neg[:, 0] * n[1] + neg[:, 1]) * n[2] + neg[:, 2]
    x = 0.5 * (x - x.transpose(1, 0, 2)[:, :, neg_idx])
    xk = np.einsum("kR,mnR->kmn", phases(spec.mesh), x)
    eye = np.eye(na)
    out = np.empty_like(xk)
    for k in range(nk):
        out[k] = np.linalg.solve((eye + xk[k]).T, (eye - xk[k]).T).T
    return np.ascontiguousarray(out)


# ---- inputs of the FFTDF variant (Appendix B, Algorithm 2): AO pair densities on a real-space grid ----

_STREAM_FFTDF = 9 << 40


@dataclasses.dataclass(frozen=True)
class GridSpec:
    """A cell with lattice vectors `lattice` (rows a_1, a_2, a_3), sampled on `grid` points per cell
    (g_d points along a_d, even numbers), carrying n_ao Gaussian-shaped real AOs per cell."""

    mesh: tuple
    n_ao: int
    grid: tuple
    lattice: tuple = ((2.0, 0.0, 0.0), (0.3, 2.2, 0.0), (0.1, 0.2, 2.5))
    n_emb: int = 4
    seed: int = 0

    @property
    def nk(self) -> int:
        return int(np.prod(self.mesh))


def cell_grid_points(spec: GridSpec) -> np.ndarray:
    """Cartesian points r = sum_d (j_d / g_d) a_d of the cell grid, C order, shape (N_g, 3)."""
    g = np.asarray(spec.grid)
    j = np.stack(np.meshgrid(*[np.arange(n) for n in g], indexing="ij"), -1).reshape(-1, 3)
    return (j / g) @ np.asarray(spec.lattice)


def ao_supercell(spec: GridSpec) -> np.ndarray:
    """chi[mu][supercell grid point], real: AO mu of cell 0 on the grid of the whole Born-von Karman
    supercell (N_d g_d points along a_d), a Gaussian exp(-alpha |r - c|^2) in the minimum-image
    distance of the supercell, with its centre c inside cell 0 and alpha in [1.5, 3] drawn per AO.
    The AO of cell R is this array shifted by R_d g_d points along each axis."""
    g = np.asarray(spec.grid)
    n = np.asarray(spec.mesh)
    big = n * g
    a = np.asarray(spec.lattice)
    rng = _rng(spec.seed, _STREAM_FFTDF)
    centres = rng.uniform(0.0, 1.0, (spec.n_ao, 3))      # fractional, in cell 0
    alphas = rng.uniform(1.5, 3.0, spec.n_ao)
    j = np.stack(np.meshgrid(*[np.arange(m) for m in big], indexing="ij"), -1).reshape(-1, 3)
    frac = j / g                                           # in cell units
    out = np.empty((spec.n_ao, len(j)))
    for mu in range(spec.n_ao):
        d = frac - centres[mu]
        d -= n * np.round(d / n)                          # minimum image on the supercell
        x = d @ a
        out[mu] = np.exp(-alphas[mu] * (x * x).sum(-1))
    return out


def shift_cells(f: np.ndarray, spec: GridSpec, R: int) -> np.ndarray:
    """f (on the supercell grid, last axis) translated by cell R (C-order index)."""
    g = np.asarray(spec.grid)
    n = np.asarray(spec.mesh)
    big = tuple(n * g)
    Rv = cell_vectors(spec.mesh)[R]
    shaped = f.reshape(f.shape[:-1] + big)
    return np.roll(shaped, tuple(Rv * g), axis=(-3, -2, -1)).reshape(f.shape)


def pair_densities_k(spec: GridSpec) -> np.ndarray:
    """rho[k1][k2][mu][nu][r] = conj(phi_{mu k1}(r)) phi_{nu k2}(r) on the grid of cell 0, with the
    Bloch sums phi_{mu k}(r) = sum_R exp(+i k.R) chi_{mu R}(r) (the AO pair densities of Eq.
    "FFTDF"; pair (k1, k2) carries momentum k2 - k1)."""
    chi = ao_supercell(spec)
    nk, na = spec.nk, spec.n_ao
    ng = int(np.prod(spec.grid))
    g = np.asarray(spec.grid)
    big = np.asarray(spec.mesh) * g
    # indices of the cell-0 grid inside the supercell grid (C order)
    j = np.stack(np.meshgrid(*[np.arange(m) for m in g], indexing="ij"), -1).reshape(-1, 3)
    flat = (j[:, 0] * big[1] + j[:, 1]) * big[2] + j[:, 2]
    shifted = np.stack([shift_cells(chi, spec, R)[:, flat] for R in range(nk)])   # [R][mu][r]
    ph = phases(spec.mesh).conj()                                               # exp(+i k.R) [k][R]
    phi = np.einsum("kR,Rmr->kmr", ph, shifted)                                 # [k][mu][r]
    rho = np.einsum("amr,bnr->abmnr", phi.conj(), phi)
    assert rho.shape == (nk, nk, na, na, ng)
    return np.ascontiguousarray(rho)


def grid_orbitals(spec: GridSpec, spin: int = 0, complex_orbitals: bool = False) -> np.ndarray:
    """Csc[(R, mu), i], orthonormal over the supercell (N(0,1) entries, or N(0,1) + i N(0,1), then QR),
    n_emb columns."""
    g = _rng(spec.seed + spin, _STREAM_FFTDF + 1)
    a = g.standard_normal((spec.nk * spec.n_ao, spec.n_emb))
    if complex_orbitals:
        a = a + 1j * g.standard_normal((spec.nk * spec.n_ao, spec.n_emb))
    return _orthonormalise(a)


def make_L_pairs(spec: LatticeSpec, pairs, p_block: int = 64, out: np.ndarray | None = None) -> np.ndarray:
    """L[e][P][mu][nu] = L^{k1_e, k2_e} for the listed pairs (pair index k1 Nk + k2), complex128, generated
    P-block by P-block so that the full L is never held: the blocks a reduced input layout keeps (for
    real-space-real inputs, the pairs the 8-fold schedule reads, about a quarter of all)."""
    nk, na = spec.nk, spec.n_ao
    pairs = np.asarray(pairs, dtype=np.int64)
    if out is None:
        out = np.empty((len(pairs), spec.n_aux, na, na), dtype=np.complex128)
    k1, k2 = pairs // nk, pairs % nk
    for p0 in range(0, spec.n_aux, p_block):
        p1 = min(spec.n_aux, p0 + p_block)
        blk = fourier_L(real_space_B(spec, p0, p1), spec.mesh)     # [k1][k2][P][mu][nu] of this P block
        out[:, p0:p1] = blk[k1, k2]
    return out
