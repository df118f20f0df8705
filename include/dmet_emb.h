/*
 * dmet_emb.h -- C ABI of the GB300 embedded two-electron-integral transformation.
 *
 * The library computes the lattice-to-embedded ERI transformation of periodic
 * ab initio DMET (Cui, Zhu & Chan, arXiv 1909.08596, section 2.1, Algorithm 1):
 *
 *   L^q_{P,ij} = s_C * sum_{k1} sum_{mu nu} conj(C^{k1}_{mu i}) L^{k1,k1+q}_{P,mu nu} C^{k1+q}_{nu j}
 *   (ij|kl)    = (1/Nk) * sum_q sum_P L^q_{P,ij} L^{-q}_{P,kl}
 *
 * with s_C = 1/Nk for the Bloch-sum orbitals of Eq. "C loemb k" (ck_norm = 0) and
 * s_C = 1 for unitary-normalised orbitals (ck_norm = 1). q = k2 - k1 is the momentum
 * transfer of a pair; Algorithm 1's k_L is -q. All k arithmetic is modulo the
 * Gamma-centred mesh, with C-order index (n1*N2 + n2)*N3 + n3.
 *
 * Memory conventions (every call):
 *  - Complex numbers are interleaved double pairs (re, im) ("complex128"), row-major.
 *  - L  : complex128 [Nk][Nk][n_aux][n_ao][n_ao], L[k1][k2][P][mu][nu] = (P | mu k1, nu k2)
 *         (Eq. "density fitting"; the aux index carries the implicit momentum k1 - k2), or,
 *         with l_layout = DMET_L_REDUCED, only the blocks listed by dmet_emb_l_pairs().
 *  - C  : complex128 [Nk][n_ao][n_emb] per spin, C[k][mu][i] = C^{k,AO,EO}_{mu i}.
 *  - Lq : complex128 [q_end - q_begin][n_aux][n_emb][n_emb].
 *  - ERI blocks: see dmet_emb_eri.
 *  Pointers may be device pointers or host pointers (pageable or pinned); the library
 *  classifies each with cudaPointerGetAttributes. Host inputs are staged through
 *  plan-owned device buffers; host outputs are copied back and the call then waits for
 *  its stream. For a real-orbital (sym = REAL, 8-fold packed) problem without check_l,
 *  dmet_emb_eri transfers from a host L only the (k1, k2) blocks its schedule reads: one
 *  k1 per orbit {k1, -k1-q} and one q per pair {q, -q} (the others follow from the
 *  symmetries the caller declared), about a quarter of L; the blocks of each q-block are
 *  copied on an internal stream (ordered after the work already queued on the plan's
 *  stream) while the previous q-block is being transformed. Every pointer must be 16-byte aligned. The caller owns all input and
 *  output buffers; the plan owns only its workspace, staging buffers and tables.
 *
 * Errors: every entry point returns a dmet_status_t and never aborts or traps.
 * Argument errors are detected on the host before any work is queued. Checks that
 * run on the device (orthonormality, symmetry of the inputs) set a per-problem device
 * status word; dmet_emb_status() waits for the plan's stream and reports it.
 * dmet_emb_last_error() returns a human-readable message for the calling thread.
 */
#ifndef DMET_EMB_H
#define DMET_EMB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DMET_API __attribute__((visibility("default")))
#else
#define DMET_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmet_emb_plan_s* dmet_emb_plan_t;

typedef enum {
  DMET_OK = 0,
  DMET_ERR_INVALID_ARG = 1,     /* bad descriptor, index or null pointer */
  DMET_ERR_ALIGNMENT = 2,       /* a pointer is not 16-byte aligned */
  DMET_ERR_OOM = 3,             /* workspace or staging allocation failed / over the limit */
  DMET_ERR_NOT_ORTHONORMAL = 4, /* device check: |s_O sum_k C^k+ C^k - 1|_max > ortho_tol */
  DMET_ERR_CUDA = 5,            /* a CUDA runtime call failed (message in dmet_emb_last_error) */
  DMET_ERR_TIMEOUT = 6,         /* a bounded device wait expired */
  DMET_ERR_UNSUPPORTED = 7,     /* valid request that this build does not implement */
  DMET_ERR_SYMMETRY = 8         /* device check: inputs violate the declared symmetry */
} dmet_status_t;

/* Arithmetic of the transforms and the contraction. The tensor-core precisions split every FP64
 * operand into slices the tensor cores (tcgen05) multiply exactly, accumulate in FP32 within short
 * K segments and across segments in an exact two-float sum, and write FP64 results. Real orbitals
 * (sym = REAL) need 8-fold packing; general orbitals (sym = NONE) take FULL or S4 packing, every q
 * contracted as one real GEMM of the bra rows (Re, Im of L^q_ij) against the ket rows of
 * L^{-q}_kl arranged so that output column 2 kl + c is component c of (ij|kl), only for kl <= ij
 * in the same-spin blocks ((kl|ij) = (ij|kl) supplies the rest). Errors against FP64 (relative
 * Frobenius, measured): see the library's documentation; BF16X3 and FP16X2 meet 1e-6, TF32 does
 * not. */
typedef enum {
  DMET_PREC_FP64 = 0,    /* every product and sum in IEEE FP64 */
  DMET_PREC_BF16X3 = 1,  /* three bf16 slices per operand, six slice products per multiply-add */
  DMET_PREC_TF32 = 2,    /* one TF32 slice, one product (about 2^-11 relative per product) */
  DMET_PREC_TF32X3 = 3,  /* two TF32 slices, three products (about 2^-22), half the 16-bit rate */
  DMET_PREC_FP16X2 = 4   /* two fp16 slices of each operand times an exact power-of-two scale
                            computed on the device from the inputs' largest components, three
                            products (about 2^-22): half the products of BF16X3 */
} dmet_prec_t;

typedef enum {
  DMET_SYM_NONE = 0,     /* no symmetry assumed: all q, all (k1, k1+q) pairs */
  DMET_SYM_REAL = 1      /* real-space-real integrals and orbitals:
                            L^{k2,k1}_{P,nu mu} = conj(L^{k1,k2}_{P,mu nu}),
                            L^{-k1,-k2} = conj(L^{k1,k2}), C^{-k} = conj(C^k);
                            the ERI is real with 8-fold symmetry */
} dmet_sym_t;

/* Layout of the L input (Eq. "density fitting"; section 2.1 loads L blockwise from disk, one
 * block per k-point pair). */
typedef enum {
  DMET_L_FULL = 0,       /* complex128 [Nk][Nk][n_aux][n_ao][n_ao]: every (k1, k2) block */
  DMET_L_REDUCED = 1     /* complex128 [n_pairs][n_aux][n_ao][n_ao]: only the blocks the
                            8-fold schedule transforms (sym = REAL and S8 packing only), in the
                            order of dmet_emb_l_pairs(); about a quarter of the full L (the
                            others follow from L^{k2,k1} = conj(L^{k1,k2})^T and
                            L^{-k1,-k2} = conj(L^{k1,k2})). With a shard (q_begin, q_end) only
                            the shard's blocks. */
} dmet_l_layout_t;

typedef enum {
  DMET_PACK_AUTO = 0,    /* S8 for DMET_SYM_REAL, FULL otherwise */
  DMET_PACK_S8 = 1,      /* real, 8-fold packed (requires DMET_SYM_REAL) */
  DMET_PACK_FULL = 2,    /* complex128 [n][n][n][n] */
  DMET_PACK_S4 = 3       /* complex, 4-fold packed: (ij|kl) = (kl|ij) = conj((ji|lk)) (FP64 path) */
} dmet_pack_t;

/* One embedding problem. Sizes follow section 2.1/2.2: a Gamma-centred mesh, n_ao AOs and
 * n_aux density-fitting functions per cell, n_emb embedding orbitals per spin
 * (n_spin = 2 for the unrestricted solver of section 2.2). */
typedef struct {
  int32_t mesh[3];      /* N1, N2, N3 >= 1; Nk = N1*N2*N3 <= 4096 */
  int32_t n_ao;         /* >= 1 */
  int32_t n_aux;        /* >= 1 */
  int32_t n_spin;       /* 1 or 2 */
  int32_t n_emb[2];     /* 1 <= n_emb[s] <= Nk*n_ao; n_emb[1] ignored when n_spin == 1 */
  int32_t prec;         /* dmet_prec_t */
  int32_t ck_norm;      /* 0: Bloch sum of Eq. "C loemb k"; 1: unitary (times Nk^-1/2) */
  int32_t sym;          /* dmet_sym_t */
  int32_t eri_pack;     /* dmet_pack_t */
  int32_t check_l;      /* 1: also verify the symmetries of L on the device when sym = REAL
                           (one extra pass over L; ~3 ms on a 3 GB L); needs l_layout = FULL */
  int32_t l_layout;     /* dmet_l_layout_t: how the caller stores L */
  int32_t q_begin;      /* shard of the contraction (dmet_emb_eri): only the momentum transfers q */
  int32_t q_end;        /* with q_begin <= min(q, -q) < q_end contribute (q and -q stay together:
                           their imaginary parts cancel in the sum). q_begin = q_end = 0 selects
                           every q. The ERIs of disjoint shards that cover [0, Nk) add up to the
                           full ERI (Algorithm 1's sum over k_L is a plain sum), so a problem can
                           be split over GPUs with one FP64 sum of the packed blocks. A partial
                           shard needs sym = REAL and 8-fold packing (else DMET_ERR_UNSUPPORTED).
                           dmet_emb_transform_3idx ignores the shard. */
  double ortho_tol;     /* <= 0 selects 1e-10 */
  double sym_tol;       /* relative; <= 0 selects 1e-10 */
} dmet_emb_desc_t;

/* ERI output blocks per problem (dmet_emb_eri):
 *   n_spin == 1: block 0 = (ij|kl) over spin alpha.
 *   n_spin == 2: block 0 = alpha-alpha, block 1 = alpha-beta ((ij) alpha, (kl) beta),
 *                block 2 = beta-beta.
 * Layouts:
 *   S8, same-spin block: double[npair*(npair+1)/2], npair = n(n+1)/2, pair index
 *       IJ = i(i+1)/2 + j (i >= j), element IJ(IJ+1)/2 + KL (IJ >= KL).
 *   S8, alpha-beta block: double[npair_a][npair_b], element [IJ][KL].
 *   FULL: complex128 [n_a][n_a][n_b][n_b], element [i][j][k][l].
 *   S4, same-spin block: complex128, every entry stored once (possibly as the conjugate of the
 *       stored value) using (ij|kl) = (kl|ij) and (ij|kl) = conj((ji|lk)):
 *       block A: i >= j, k >= l, IJ >= KL (IJ = i(i+1)/2 + j) at IJ(IJ+1)/2 + KL;
 *       block B: i > j, k < l, a >= b (a = i(i-1)/2 + j, b = l(l-1)/2 + k) at nA + a(a+1)/2 + b,
 *       nA = npair(npair+1)/2, npair = n(n+1)/2. Any other entry: (ij|kl) = (kl|ij) brings an
 *       ordered pair first; a reversed first pair is conj((ji|lk)); (ii|kl) with k < l is
 *       conj((ii|lk)); in block B, a < b is conj((lk|ji)) stored at nA + b(b+1)/2 + a.
 *   S4, alpha-beta block: complex128 [npair_a][n_b][n_b], element [IJ][k][l] for i >= j (the
 *       others: (ij|kl) = conj((ji|lk))).
 * Returns the number of BYTES of block `block` of `desc`, or 0 for an invalid request. */
DMET_API size_t dmet_emb_eri_bytes(const dmet_emb_desc_t* desc, int32_t block);

/* Builds a plan for n_problems problems (section 2.1, Algorithm 1's loop structure:
 * the scheduler tables of momentum-conserving pairs per q). `stream` is a cudaStream_t
 * (NULL = legacy default stream) on which every later call of this plan queues its work.
 * workspace_limit bounds the plan's device workspace in bytes (0 = 8 GiB); the q-block
 * size (at most 8 values of q per block of work; every q of a weight class in one block when
 * that workspace stays under 512 MiB) is chosen to fit it. Environment variables read here:
 * DMET_QBLOCK (1..8) caps the q-block size (with host-resident L the blocks' L pairs are
 * copied one block ahead of the kernels that read them, so smaller blocks expose less of the
 * copy before the first kernels start, at some cost in kernel efficiency); DMET_TC_KSEG,
 * DMET_TC_KSEG1 and DMET_TC_CRUN set the tensor-core paths' FP32 segment lengths (K elements,
 * multiples of 32; defaults 128, 128) and correction-run length (segments; default 1);
 * DMET_TC_PACE selects the job pacing of the tensor-core launches (bit 1: contractions, the
 * default; bit 2: the transforms too; 0: none; it never changes a result); DMET_TUNE_CACHE
 * names the tuning cache (dmet_emb_autotune). Allocates device memory. Host-side validation
 * only; no kernel runs. */
DMET_API dmet_status_t dmet_emb_plan(const dmet_emb_desc_t* descs, int32_t n_problems, void* stream,
                            size_t workspace_limit, dmet_emb_plan_t* plan);

/* Embedded 3-index factors L^q_{P,ij} for q in [q_begin, q_end) (Algorithm 1's inner loop:
 * k-AO -> k-EO transform of every momentum-conserving pair, then the Fourier sum to the
 * reference cell; the paper notes that a density-fitting solver can consume these
 * directly and skip the contraction). C[s] and Lq_out[s] for s < n_spin.
 * The transforms run in the problem's precision: FP64 kernels for DMET_PREC_FP64, the
 * tensor-core half transforms of the contraction path otherwise (then the q must belong to the
 * descriptor's shard; L^q is summed from the FP32 two-float results exactly in FP64).
 * Also runs the orbital checks (orthonormality; realness when sym = REAL). */
DMET_API dmet_status_t dmet_emb_transform_3idx(dmet_emb_plan_t plan, int32_t problem, const void* L,
                                      const void* const* C, int32_t q_begin, int32_t q_end,
                                      void* const* Lq_out);

/* Embedded ERIs of every problem of the plan (Algorithm 1 including its final
 * contraction over the aux index and the sum over q). L[p], C[p][s], eri_out[p][b] for
 * problem p, spin s and output block b (see dmet_emb_eri_bytes). Output buffers are
 * overwritten. */
DMET_API dmet_status_t dmet_emb_eri(dmet_emb_plan_t plan, const void* const* L, const void* const* const* C,
                           void* const* const* eri_out);

/* Waits for the plan's stream and returns the device status of `problem`. If stats is not
 * NULL it receives 4 doubles: [0] orthonormality error max|s_O sum_k C^k+C^k - 1| (worst
 * spin), [1] relative realness error max|C^{-k} - conj C^k| / max|C|, [2] relative
 * Hermiticity error of L and [3] relative time-reversal error of L, both as the largest
 * real or imaginary component of the difference over the largest component of L
 * (negative = not checked). A bounded device wait that expired is reported as
 * DMET_ERR_TIMEOUT. */
DMET_API dmet_status_t dmet_emb_status(dmet_emb_plan_t plan, int32_t problem, double* stats);

/* The embedding one-particle Hamiltonian of section 2.1: the Fock matrix of Eq. "fock
 * transform", F0 = s sum_k C^{k+} F^k C^k (s = 1/Nk for ck_norm = 0, 1 for ck_norm = 1: the
 * normalisation under which the orbitals are orthonormal), minus the double counting of
 * Eq. "fock double counting", the Coulomb and exchange of the embedding density gamma in the
 * embedding ERIs:
 *     fock_out_ij = F0_ij - [ sum_kl (ij|kl) gamma_lk - 1/2 sum_kl (ik|lj) gamma_kl ].
 * For restricted problems with real orbitals and the 8-fold packed ERI (n_spin = 1, sym =
 * REAL, pack S8 or AUTO); others return DMET_ERR_UNSUPPORTED. Device pointers only:
 *   F        complex128 [Nk][n_ao][n_ao], F[k][mu][nu] = F^{k,AO}_{mu nu} (Hermitian; the
 *            Hartree-Fock operator of the mean-field calculation, as the paper specifies);
 *   C        the problem's orbitals, as for dmet_emb_eri;
 *   eri      the problem's packed ERI as dmet_emb_eri wrote it (FP64, n(n+1)/2 (n(n+1)/2 + 1)/2);
 *   gamma    FP64 [n][n], symmetric, spin-summed, in the embedding basis;
 *   fock_out FP64 [n][n] (the real part of F0, whose imaginary part vanishes for real orbitals).
 * FP64 throughout; queued on the plan's stream; grows a plan-owned scratch buffer on first use
 * (about 16 Nk n_AO n + 16 Nk n^2 bytes). */
DMET_API dmet_status_t dmet_emb_fock(dmet_emb_plan_t plan, int32_t problem, const void* F, const void* C,
                                     const double* eri, const double* gamma, double* fock_out);

/* The DMET bath and embedding orbitals of section 2.1, which produce the C input of
 * dmet_emb_eri on the device. The impurity is the n_ao localized orbitals (LOs) of the
 * reference cell R = 0. Steps:
 *   1. gamma^{R,0} = (1/Nk) sum_k exp(+i k.R) gamma^k for every cell R != 0, on the impurity
 *      valence columns val (Eq. "bath R SVD" with j restricted to the valence LOs);
 *   2. the SVD of that ((Nk - 1) n_ao) x n_val block (real part; one-sided Jacobi rotations):
 *      its left singular vectors B^R are the bath orbitals, in decreasing singular value, each
 *      signed so that its largest-magnitude coefficient (the first in (R, i) order of equal
 *      ones) is positive;
 *   3. C^{R,LO,EO} = [[1, 0], [0, B^{R != 0}]] (Eq. "C loemb R"), impurity columns first;
 *   4. C_out[k] = C^{k,AO,LO} sum_R exp(-i k.R) C^{R,LO,EO} (Eq. "C loemb k").
 * The density convention: gamma^k = sum_R exp(+i k.R) g(R), g(R)_{ij} the element between LO i of
 * cell 0 and LO j of cell R (as for the Fock matrix of dmet_emb_fock); a time-reversal-symmetric
 * mean field (gamma^{-k} = conj gamma^k) makes the block real. Arguments:
 *   problem, spin  which orbitals of the plan this builds; n_ao + n_val must equal n_emb[spin];
 *   gamma_k  device complex128 [Nk][n_ao][n_ao], the mean-field density matrix in the LO basis;
 *   C_lo     device complex128 [Nk][n_ao][n_ao], C^{k,AO,LO}[k][mu][i] (unitary at each k for
 *            orthonormal AOs);
 *   val      host int32 [n_val], distinct LO indices in [0, n_ao), 1 <= n_val <= min(n_ao, 128);
 *   C_out    device complex128 [Nk][n_ao][n_ao + n_val], written (the layout dmet_emb_eri reads);
 *   info     device double [n_val + 5] or NULL: the singular values (decreasing), then
 *            max |Re| and max |Im| of the block, the Jacobi sweeps used (at most 40), the largest
 *            pair cosine of the last sweep, and sigma_min / sigma_max. A zero singular value
 *            leaves a zero bath column (the orthonormality check of dmet_emb_eri then fails).
 * Needs Nk >= 2. FP64 throughout; queued on the plan's stream; grows a plan-owned scratch
 * buffer on first use (about 16 (Nk - 1) n_ao n_val + 16 Nk n_ao n_val bytes). Invalid
 * arguments return DMET_ERR_INVALID_ARG or DMET_ERR_ALIGNMENT before anything is queued. */
DMET_API dmet_status_t dmet_emb_bath(dmet_emb_plan_t plan, int32_t problem, int32_t spin, const void* gamma_k,
                                     const void* C_lo, const int32_t* val, int32_t n_val, void* C_out,
                                     double* info);

/* Coulomb and exchange of an embedding density straight from the density-fitted factors, without
 * forming the ERI (section 2.1: a solver that supports density fitting takes the factors and skips
 * Algorithm 1's contraction). With (ij|kl) = (1/Nk) sum_q sum_P L^q_{P,ij} L^{-q}_{P,kl}:
 *     J_ij = (1/Nk) sum_q sum_P L^q_{P,ij} tr(L^{-q}_P gamma),
 *     K_ij = (1/Nk) sum_q sum_P (L^q_P gamma L^{-q}_P)_ij,
 * i.e. J_ij = sum_kl (ij|kl) gamma_lk and K_ij = sum_kl (ik|lj) gamma_kl, the two terms of Eq.
 * "fock double counting". Device pointers only (16-byte aligned):
 *   Lq     complex128 [Nk][n_aux][n][n], L^q of spin `spin` for every q (as dmet_emb_transform_3idx
 *          writes them for q in [0, Nk));
 *   gamma  complex128 [n][n], the embedding density;
 *   J, K   complex128 [n][n], written (real for real orbitals and a real gamma).
 * FP64 throughout (batched complex GEMMs over the (q, P) entries in chunks, and reductions); queued
 * on the plan's stream; grows a plan-owned scratch buffer of at most about 1 GiB on first use. */
DMET_API dmet_status_t dmet_emb_jk_df(dmet_emb_plan_t plan, int32_t problem, int32_t spin, const void* Lq,
                                      const void* gamma, void* J, void* K);

/* Embedded ERIs with FFTDF (Appendix B, Algorithm 2, Eq. "FFTDF"): the auxiliary set is the plane
 * waves of the cell's real-space grid. The problem's n_aux must be the number of grid points N_g =
 * grid[0] grid[1] grid[2] (prec = FP64, FULL packing, full L layout). Arguments (device pointers):
 *   rho      complex128 [Nk][Nk][N_g][n_ao][n_ao], rho[k1][k2][r][mu][nu] = conj(phi_{mu k1}(r))
 *            phi_{nu k2}(r), the AO pair densities on the reference cell's grid (r in C order over
 *            the grid points sum_d (j_d / g_d) a_d) in place of L;
 *   C        the orbitals per spin, as for dmet_emb_eri;
 *   grid     host int32 [3], points per lattice vector;  lattice  host double [3][3], rows a_d;
 *   eri_out  complex128 [n_a][n_a][n_b][n_b] per block (FULL layout of dmet_emb_eri).
 * For every q: (r|0i 0j) = s_C sum_k1 C^{k1+} rho^{k1,k1+q}(r) C^{k1+q} (the half transforms of
 * dmet_emb_eri), then exp(-i q.r), the forward DFT over the grid, the Coulomb kernel 4 pi / |q + G|^2
 * (the plane waves and kernel of dmet_fftdf_plane_waves, 0 at q + G = 0), the inverse DFT,
 * exp(+i q.r), and (ij|kl) += Omega / (N_g Nk) sum_r w(r)_ij (r|0k 0l)^{-q} with the inverse DFT
 * normalised by 1/N_g (Omega the cell volume). The DFTs are dense per grid axis (batched complex
 * GEMMs). FP64 throughout; queued on the plan's stream; grows a plan-owned scratch buffer on first use
 * (2 N_g n^2 complex values). */
DMET_API dmet_status_t dmet_emb_eri_fftdf(dmet_emb_plan_t plan, int32_t problem, const void* rho,
                                          const void* const* C, const int32_t* grid, const double* lattice,
                                          void* const* eri_out);

/* Frees the plan's device memory, events and tables. Safe on NULL. Waits for the stream. */
DMET_API dmet_status_t dmet_emb_destroy(dmet_emb_plan_t plan);

/* The k-pair schedule of one problem (section 2.1, Algorithm 1's two loops; momentum
 * conservation of Eq. "density fitting"). Host-only; no GPU needed. Arrays of Nk or Nk*Nk
 * int32 entries, any may be NULL:
 *   k2_of[q*Nk + k1] = k1 + q;  neg[k] = -k;
 *   q_weight[q] = number of q values the contraction of q stands for (sym = REAL: 1 for
 *                 self-conjugate q, 2 for the representative min(q, -q), 0 for the other;
 *                 sym = NONE: 1 for every q);
 *   n_rep[q], rep_k1[q*Nk + r], rep_half[q*Nk + r]: the k1 values whose transformed pairs are
 *                 computed for q. sym = REAL: one k1 per orbit {k1, -k1-q} (the smaller), with
 *                 rep_half = 1 for the fixed points k1 = -k1-q; sym = NONE: every k1, rep_half 0. */
DMET_API dmet_status_t dmet_emb_schedule(const dmet_emb_desc_t* desc, int32_t* k2_of, int32_t* neg,
                                int32_t* q_weight, int32_t* n_rep, int32_t* rep_k1,
                                int32_t* rep_half);

/* The (k1, k2) blocks of L that dmet_emb_eri reads for a real-orbital, 8-fold packed problem
 * (sym = REAL, S8 packing), in the order of the DMET_L_REDUCED layout: the contracted q values
 * (those whose q_weight is nonzero and, with a shard, with q_begin <= q < q_end) with q = -q first
 * and then q < -q, each in increasing order; within one q, its representative k1 of each orbit
 * {k1, -k1-q} in increasing order (Algorithm 1's two loops with the symmetry reductions of
 * dmet_emb_schedule). pairs[e] = k1 * Nk + k2 with k2 = k1 + q. Host-only; no GPU needed.
 * *n_pairs receives the count; pairs may be NULL (count only). Other problems return
 * DMET_ERR_UNSUPPORTED. */
DMET_API dmet_status_t dmet_emb_l_pairs(const dmet_emb_desc_t* desc, int32_t* pairs, int64_t* n_pairs);

/* Plane waves of the FFTDF variant (Appendix B, Eq. "FFTDF"; the auxiliary set of Algorithm 2) for
 * momentum q of a Gamma-centred mesh, on a cell grid of grid[d] points along the lattice vectors a_d
 * (lattice: 3 x 3, row-major, row d = a_d). Host-only; no GPU needed. For each FFT index j (C order over
 * the grid; N_g = grid[0] grid[1] grid[2] entries, any output may be NULL):
 *   m[3 j .. 3 j + 2]: the reciprocal-lattice triple of G (m_d = j_d mod grid[d]), chosen so that q + G is
 *                      one of the signed FFT frequencies of the Born-von Karman supercell's grid
 *                      (mesh[d] grid[d] points along a_d, Nyquist convention included);
 *   v[j]:              the Coulomb kernel 4 pi / |q + G|^2, 0 at q + G = 0;
 *   opposite[j]:       the FFT index j' at momentum -q whose plane wave is -(q + G) (the -q factor of
 *                      Algorithm 2's contraction pairs with it), modulo the supercell grid: on an axis
 *                      with mesh[d] grid[d] even, -(q + G) at the Nyquist frequency folds back onto it.
 * Returns DMET_ERR_INVALID_ARG for sizes outside [1, 4096] per axis, Nk > 4096, N_g > 2^24, q outside
 * [0, Nk) or a singular lattice. */
DMET_API dmet_status_t dmet_fftdf_plane_waves(const int32_t* mesh, int32_t q, const int32_t* grid,
                                              const double* lattice, int32_t* m, double* v, int32_t* opposite);

/* Execution of the plan's problems (the batched form of Algorithm 1's loops; the paper runs
 * one embedding problem at a time). When every problem of a plan gets its own workspace
 * within the plan's workspace limit, dmet_emb_eri runs the problems concurrently on the
 * plan's side streams, forked from and joined back to the plan's stream; otherwise they run
 * one after another. enable != 0 makes dmet_emb_eri capture its work, on its first call with
 * device buffers, into a CUDA graph that later calls with the same buffers replay on the
 * plan's stream (different buffers: captured again; host buffers or profiling: no graph). */
DMET_API dmet_status_t dmet_emb_graph(dmet_emb_plan_t plan, int32_t enable);

/* Execution of a plan of several problems. mode 1 (the default) runs the batch as grouped
 * persistent launches whenever every problem is on a tensor-core precision, every problem got its
 * own workspace, the inputs and outputs are device buffers, and no complex ERI is 4-fold packed:
 * per round r (block r of the q-blocks of every problem that has one) and spin, one launch of the
 * first half transform and one of the second for all problems (one per precision and tile width),
 * and at the end one launch of the contraction of every ERI block of every problem, each a
 * persistent tcgen05 kernel over a device table of per-problem tensor maps, segment lists and
 * output parameters; each problem's element-wise kernels (checks, operand splitting, packing) run
 * on the side streams between them. Every problem then completes with the last launch, so the
 * per-problem times of dmet_emb_problem_ms are the batch's. mode 0 runs each problem on its own
 * side stream (or one after another), as described for dmet_emb_graph. *active (optional)
 * receives 1 if calls with device buffers will run grouped, else 0. A captured graph is discarded
 * when the mode changes. No counterpart in the paper (a GPU scheduling choice). */
DMET_API dmet_status_t dmet_emb_batch_mode(dmet_emb_plan_t plan, int32_t mode, int32_t* active);

/* Device milliseconds of problem `problem` in the last call made while profiling was enabled
 * (CUDA events around that problem's work on its stream). Waits for the stream. */
DMET_API dmet_status_t dmet_emb_problem_ms(dmet_emb_plan_t plan, int32_t problem, double* ms);

/* Autotuner of the split-BF16 path: for every problem it times the two transform GEMMs'
 * output tile widths (128, 112 and 96 columns; the width that wastes least on the problem's
 * 2 n_emb output columns is not always the fastest), each problem on its own side stream, by
 * running dmet_emb_eri on the given
 * buffers (device pointers; the outputs are overwritten with valid results), keeps the
 * fastest for each problem, then in the same way the K split of the contraction's last wave
 * (dmet_emb_split_parts) and, if the environment variable DMET_TUNE_CACHE names a file,
 * appends the choice there; dmet_emb_plan reads that file for later plans of the same shape.
 * A captured graph is discarded. No counterpart in the paper (it is a GPU tiling choice). */
DMET_API dmet_status_t dmet_emb_autotune(dmet_emb_plan_t plan, const void* const* L, const void* const* const* C,
                                         void* const* const* eri_out);

/* The K split of the contraction's last wave in use for `problem` (side-stream and single-problem
 * execution; grouped launches run whole tiles): for ERI block b (0 aa, 1 ab, 2 bb),
 * parts[2 b] = the number of tiles split and parts[2 b + 1] = the parts per tile (1 = none).
 * dmet_emb_autotune times the split factors 1, 2, 4 and 8 against the default (as many parts as
 * fill the GPU's SMs, at most 8) and keeps the fastest. */
DMET_API dmet_status_t dmet_emb_split_parts(dmet_emb_plan_t plan, int32_t problem, int32_t* parts);

/* The tile widths in use for `problem`: bn[0] (half transform 1), bn[1] (half transform 2). */
DMET_API dmet_status_t dmet_emb_tile_widths(dmet_emb_plan_t plan, int32_t problem, int32_t* bn);

/* Bounded waits. Every spin-wait of the tensor-core kernels (on an mbarrier: a stage loaded, a stage
 * or accumulator free, an accumulator ready) gives up after wait_ns nanoseconds of the GPU's global
 * timer (0 restores the default, 4 s); the kernel then records which kind of wait expired in the
 * plan's device error word, lets its copies in flight land, frees its tensor memory and returns, so
 * the context stays usable, and the next dmet_emb_status returns DMET_ERR_TIMEOUT (once; the word
 * is then cleared). test_withhold_loads != 0 is a test hook with no counterpart in the paper: the
 * producer thread of every later tensor-core launch of this plan issues no copies, so the waits for
 * loaded stages and ready accumulators expire with no copy and no MMA in flight (the results are
 * then meaningless). A captured graph is discarded. */
DMET_API dmet_status_t dmet_emb_wait_limit(dmet_emb_plan_t plan, uint64_t wait_ns, int32_t test_withhold_loads);

/* Per-kernel timing with CUDA events on the plan's stream. enable != 0 starts recording
 * (and clears the counters); 0 stops. */
DMET_API dmet_status_t dmet_emb_profile(dmet_emb_plan_t plan, int32_t enable);

/* Reads the counters of kernel class `kernel` (0 .. dmet_emb_profile_count()-1): name,
 * launches, total device milliseconds, algorithmic flops (the work the method needs, with
 * the symmetry reductions applied; a complex multiply-add counts 8), executed flops (what
 * the kernels issue: for the split-BF16 tensor-core kernels the 6 slice products over whole
 * 128 x 128 tiles, otherwise equal to the algorithmic count) and algorithmic bytes, summed
 * over the recorded launches. Waits for the stream. */
DMET_API int32_t dmet_emb_profile_count(void);
DMET_API dmet_status_t dmet_emb_profile_read(dmet_emb_plan_t plan, int32_t kernel, const char** name,
                                    int64_t* launches, double* total_ms, double* flops,
                                    double* exec_flops, double* bytes);

/* Number of kernel launches the plan has queued since it was created. */
DMET_API int64_t dmet_emb_launch_count(dmet_emb_plan_t plan);

/* Size of the static device scratch array used by dmet_emb_eri_noalloc (32 MiB). */
#define DMET_EMB_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory: a caller whose device memory is entirely owned by another
 * allocator (for example a framework's caching pool that must account for every byte), or
 * one that must not let an allocation synchronise the device in the middle of an embedding
 * self-consistency loop that shares the GPU with other streams.
 *
 * It computes the same result as dmet_emb_eri's FP64 path for one problem, allocating
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine, no host heap. All
 * scratch comes from one file-scope __device__ array of DMET_EMB_NOALLOC_SCRATCH_BYTES bytes,
 * which every GPU that loads the library holds until the process exits. The caller passes
 * device pointers (L, C[s], eri_out[b]) laid out as for dmet_emb_eri, and `stream`, a
 * cudaStream_t (NULL = legacy default stream).
 * Supported: prec = FP64, sym = REAL, 8-fold packing (AUTO or S8), the full L layout, no
 * shard, Nk <= 64 (each mesh dimension <= 64); descriptor fields outside dmet_emb_plan's bounds
 * are rejected before any size is computed, and a problem whose scratch would exceed the array
 * is rejected with DMET_ERR_OOM and a message giving both sizes, before any work is queued.
 * Host pointers are rejected (staging would allocate). Every call looks up the array's address
 * on the current device (cudaGetSymbolAddress, which allocates nothing: in host code the array's
 * name is only a host-side stand-in); the first call on a device loads the library's device code
 * there, so make it before any stream capture. The host-side tables live in one static
 * structure that a mutex guards for the whole call.
 * Calls share the array and leave their contents in it; the call clears what must start at
 * zero (its check maxima and the output blocks) itself. Two calls whose work overlaps on the
 * GPU (other streams, other host threads on the same device) race on the array: serialise
 * them. The call is synchronous: it waits for `stream` and returns the device checks' status
 * (DMET_ERR_NOT_ORTHONORMAL, DMET_ERR_SYMMETRY) like dmet_emb_status. */
DMET_API dmet_status_t dmet_emb_eri_noalloc(const dmet_emb_desc_t* desc, const void* L,
                                            const void* const* C, void* const* eri_out, void* stream);

/* Message describing the last error returned on the calling thread ("" if none). */
DMET_API const char* dmet_emb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DMET_EMB_H */
