// dmet_emb_eri_noalloc: the FP64 embedded-ERI path for callers that cannot allocate device
// memory. It runs the same kernels as dmet_emb_eri's FP64 path (orbital checks, the two
// half transforms per q, pair packing and the 8-fold packed contraction), but every scratch
// buffer is carved out of one file-scope __device__ array, so the call allocates nothing:
// no cudaMalloc, no cudaFree, no allocating library routine, and no host heap either (its
// schedule tables are built in one fixed-size static host structure).
//
// Who needs this: a caller whose device memory is entirely owned by another allocator
// (for example a framework's caching pool that must see every byte), or one that must not
// let an allocation synchronise the device in the middle of an embedding self-consistency
// loop that shares the GPU with other streams. Such callers pass their input and output
// buffers; the scratch comes from the library's static array.
//
// The array (DMET_EMB_NOALLOC_SCRATCH_BYTES) is part of the library's device image: every
// GPU on which the library's kernels are loaded holds it until the process exits. Its
// device address is looked up with cudaGetSymbolAddress on every call, with the caller's
// device current (no cached address can outlive a context that was torn down and created
// again); the first call on a device loads the library's device code there, so make it
// before any stream capture. All calls share the array and leave their contents in it, so
// two calls whose work overlaps on the GPU (different streams, or different host threads on
// one device) race on it: serialise them. The host side keeps its schedule tables in one
// static structure guarded by a mutex for the whole call, so calls from several host
// threads take turns there.

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/dmet_emb.h"
#include "internal.h"

using namespace dmet;

namespace {

static __device__ __align__(256) unsigned char g_scratch[DMET_EMB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxNk = 64;  // the schedule tables below are sized for this mesh bound
std::mutex g_mutex;         // guards g_tab for a whole call

dmet_status_t nfail(dmet_status_t st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dmet::last_error_buffer(), dmet::kLastErrorBytes, fmt, ap);
  va_end(ap);
  return st;
}

#define NCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return nfail(DMET_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Host-side schedule of one problem in fixed-size arrays (no heap).
struct NoAllocTables {
  int nk;
  int neg[kMaxNk];
  int order[kMaxNk];     // contracted q: self-conjugate ones first, then q < -q
  int weight[kMaxNk];
  int nq;
  int start[kMaxNk + 1];  // entries of order[i] are [start[i], start[i+1])
  int4 t1[kMaxNk * kMaxNk];
  int4 gather[kMaxNk * kMaxNk];
  int4 t2[kMaxNk];
};
NoAllocTables g_tab;

int kmod(int a, int n) { return ((a % n) + n) % n; }

void build_noalloc_tables(const dmet_emb_desc_t& d, NoAllocTables& t) {
  const int* m = d.mesh;
  const int nk = m[0] * m[1] * m[2];
  t.nk = nk;
  auto trip = [&](int k, int& a, int& b, int& c) {
    a = k / (m[1] * m[2]);
    b = (k / m[2]) % m[1];
    c = k % m[2];
  };
  auto idx = [&](int a, int b, int c) { return (kmod(a, m[0]) * m[1] + kmod(b, m[1])) * m[2] + kmod(c, m[2]); };
  for (int k = 0; k < nk; ++k) {
    int a, b, c;
    trip(k, a, b, c);
    t.neg[k] = idx(-a, -b, -c);
  }
  t.nq = 0;
  for (int w = 1; w <= 2; ++w)
    for (int q = 0; q < nk; ++q) {
      const int wq = q == t.neg[q] ? 1 : (q < t.neg[q] ? 2 : 0);
      if (wq == w) {
        t.order[t.nq] = q;
        t.weight[t.nq] = w;
        ++t.nq;
      }
    }
  int e = 0;
  for (int i = 0; i < t.nq; ++i) {
    const int q = t.order[i];
    int qa, qb, qc;
    trip(q, qa, qb, qc);
    t.start[i] = e;
    for (int k1 = 0; k1 < nk; ++k1) {
      int a, b, c;
      trip(k1, a, b, c);
      const int k2 = idx(a + qa, b + qb, c + qc);
      const int partner = t.neg[k2];  // -k1 - q
      if (k1 > partner) continue;
      t.t1[e] = make_int4(k2, k1 * nk + k2, e, d.n_ao);
      t.gather[e] = make_int4(k1, k1 == partner ? 1 : 0, 0, 0);
      ++e;
    }
    t.t2[i] = make_int4(t.start[i], t.start[i], i, (e - t.start[i]) * d.n_ao);
  }
  t.start[t.nq] = e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout arithmetic that reports overflow instead of wrapping: off = align256(off + a * b).
bool grow(size_t& off, size_t a, size_t b) {
  size_t p = 0, q = 0;
  if (__builtin_mul_overflow(a, b, &p) || __builtin_add_overflow(off, p, &q) || q > (SIZE_MAX - 255)) return false;
  off = align256(q);
  return true;
}

ZgemmArgs zdefault() {
  ZgemmArgs z;
  std::memset(&z, 0, sizeof(z));
  z.dm_div = INT_MAX;
  z.dn_div = INT_MAX;
  z.alpha = 1.0;
  z.batch = 1;
  return z;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" DMET_API dmet_status_t dmet_emb_eri_noalloc(const dmet_emb_desc_t* desc, const void* L,
                                                       const void* const* C, void* const* eri_out, void* stream) {
  dmet::last_error_buffer()[0] = 0;
  if (!desc || !L || !C || !eri_out) return nfail(DMET_ERR_INVALID_ARG, "NULL argument");
  const dmet_emb_desc_t& d = *desc;
  // The same descriptor rules as dmet_emb_plan, narrowed to what this variant runs.
  for (int i = 0; i < 3; ++i)
    if (d.mesh[i] < 1 || d.mesh[i] > kMaxNk) return nfail(DMET_ERR_INVALID_ARG, "mesh[%d] = %d", i, d.mesh[i]);
  const long long nk = (long long)d.mesh[0] * d.mesh[1] * d.mesh[2];
  if (nk > kMaxNk) return nfail(DMET_ERR_UNSUPPORTED, "Nk = %lld exceeds the no-allocation limit %d", nk, kMaxNk);
  if (d.n_ao < 1 || d.n_ao > 4096 || d.n_aux < 1 || d.n_aux > 65536 || (d.n_spin != 1 && d.n_spin != 2))
    return nfail(DMET_ERR_INVALID_ARG, "invalid descriptor (n_ao %d, n_aux %d, n_spin %d)", d.n_ao, d.n_aux, d.n_spin);
  if (d.check_l != 0 && d.check_l != 1) return nfail(DMET_ERR_INVALID_ARG, "check_l = %d", d.check_l);
  for (int s = 0; s < d.n_spin; ++s)
    if (d.n_emb[s] > 2047) return nfail(DMET_ERR_UNSUPPORTED, "n_emb[%d] = %d > 2047", s, d.n_emb[s]);
  if (d.l_layout != DMET_L_FULL || d.q_begin != 0 || d.q_end != 0)
    return nfail(DMET_ERR_UNSUPPORTED, "the no-allocation variant takes the full L layout and no shard");
  for (int s = 0; s < d.n_spin; ++s)
    if (d.n_emb[s] < 1 || (long long)d.n_emb[s] > nk * d.n_ao) return nfail(DMET_ERR_INVALID_ARG, "n_emb[%d]", s);
  if (d.prec != DMET_PREC_FP64 || d.sym != DMET_SYM_REAL ||
      (d.eri_pack != DMET_PACK_AUTO && d.eri_pack != DMET_PACK_S8) || (d.ck_norm != 0 && d.ck_norm != 1))
    return nfail(DMET_ERR_UNSUPPORTED, "the no-allocation variant runs FP64, sym = REAL, 8-fold packing only");
  {
    // the per-launch 32-bit sizes of the kernels (as in dmet_emb_plan)
    const long long nm = std::max(d.n_emb[0], d.n_spin == 2 ? d.n_emb[1] : 0);
    if ((long long)d.n_aux * nm > INT_MAX / 2 || (long long)d.n_aux * d.n_ao > INT_MAX / 2)
      return nfail(DMET_ERR_UNSUPPORTED, "n_aux*n too large for one launch");
  }
  const int nblk = d.n_spin == 1 ? 1 : 3;
  std::lock_guard<std::mutex> lock(g_mutex);
  NoAllocTables& tb = g_tab;
  build_noalloc_tables(d, tb);
  const int nao = d.n_ao, naux = d.n_aux, nspin = d.n_spin;
  const int n[2] = {d.n_emb[0], nspin == 2 ? d.n_emb[1] : 0};
  const long long npair[2] = {(long long)n[0] * (n[0] + 1) / 2, (long long)n[1] * (n[1] + 1) / 2};
  const int nmax = std::max(n[0], n[1]);
  int emax = 0;
  for (int i = 0; i < tb.nq; ++i) emax = std::max(emax, tb.start[i + 1] - tb.start[i]);
  int ng = 1;
  for (int g = (int)std::min<long long>(nk, 32); g >= 1; --g)
    if (nk % g == 0) {
      ng = g;
      break;
    }

  // Scratch layout (256-byte aligned pieces), one q at a time. Every size is a product of bounded
  // descriptor fields; grow() still checks each step for overflow.
  size_t off = 0;
  bool fits = true;
  const size_t o_stats = off;
  fits = fits && grow(off, 8, sizeof(double));
  const size_t o_neg = off;
  fits = fits && grow(off, (size_t)nk, sizeof(int));
  const size_t o_t1 = off;
  fits = fits && grow(off, (size_t)tb.start[tb.nq], sizeof(int4));
  const size_t o_gather = off;
  fits = fits && grow(off, (size_t)tb.start[tb.nq], sizeof(int4));
  const size_t o_t2 = off;
  fits = fits && grow(off, (size_t)tb.nq, sizeof(int4));
  const size_t o_S = off;
  fits = fits && grow(off, (size_t)ng * nmax, (size_t)nmax * 16);
  const size_t o_crep = off;
  fits = fits && grow(off, (size_t)emax * nao, (size_t)nmax * 16);
  const size_t o_T = off;
  fits = fits && grow(off, (size_t)emax * nao * naux, (size_t)nmax * 16);
  const size_t o_Z = off;
  fits = fits && grow(off, (size_t)naux * nmax, (size_t)nmax * 16);
  size_t o_X[2];
  for (int s = 0; s < 2; ++s) {
    o_X[s] = off;
    fits = fits && grow(off, s < nspin ? (size_t)naux * 2 : 0, (size_t)npair[s] * 8);
  }
  if (!fits) return nfail(DMET_ERR_OOM, "problem's scratch size overflows; the static scratch holds %zu bytes",
                          (size_t)DMET_EMB_NOALLOC_SCRATCH_BYTES);
  if (off > (size_t)DMET_EMB_NOALLOC_SCRATCH_BYTES)
    return nfail(DMET_ERR_OOM, "problem needs %zu bytes of scratch; the static scratch holds %zu", off,
                 (size_t)DMET_EMB_NOALLOC_SCRATCH_BYTES);
  if (!on_device(L)) return nfail(DMET_ERR_INVALID_ARG, "L must be device memory (host staging would allocate)");
  if ((uintptr_t)L & 15) return nfail(DMET_ERR_ALIGNMENT, "L not 16-byte aligned");
  for (int s = 0; s < d.n_spin; ++s) {
    if (!C[s] || !on_device(C[s])) return nfail(DMET_ERR_INVALID_ARG, "C[%d] must be device memory", s);
    if ((uintptr_t)C[s] & 15) return nfail(DMET_ERR_ALIGNMENT, "C[%d] not 16-byte aligned", s);
  }
  for (int b = 0; b < nblk; ++b) {
    if (!eri_out[b] || !on_device(eri_out[b])) return nfail(DMET_ERR_INVALID_ARG, "eri_out[%d] must be device memory", b);
    if ((uintptr_t)eri_out[b] & 15) return nfail(DMET_ERR_ALIGNMENT, "eri_out[%d] not 16-byte aligned", b);
  }


  // The array's address on the current device (host code cannot use the symbol itself: in host
  // code it names a host-side stand-in). Looked up on every call; it allocates nothing.
  unsigned char* base = nullptr;
  {
    void* p = nullptr;
    NCK(cudaGetSymbolAddress(&p, g_scratch));
    base = (unsigned char*)p;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* stats = (double*)(base + o_stats);
  int* dneg = (int*)(base + o_neg);
  int4* dt1 = (int4*)(base + o_t1);
  int4* dgather = (int4*)(base + o_gather);
  int4* dt2 = (int4*)(base + o_t2);
  double2* S = (double2*)(base + o_S);
  double2* crep = (double2*)(base + o_crep);
  double2* T = (double2*)(base + o_T);
  double2* Z = (double2*)(base + o_Z);
  double* X[2] = {(double*)(base + o_X[0]), (double*)(base + o_X[1])};

  // What must start at zero: the check maxima and the accumulated outputs.
  NCK(cudaMemsetAsync(stats, 0, 8 * sizeof(double), st));
  for (int b = 0; b < nblk; ++b) {
    const int sa = b == 2 ? 1 : 0, sb = b == 0 ? 0 : 1;
    const size_t bytes = b == 1 ? (size_t)npair[0] * npair[1] * 8 : (size_t)npair[sa] * (npair[sa] + 1) / 2 * 8;
    (void)sb;
    NCK(cudaMemsetAsync(eri_out[b], 0, bytes, st));
  }
  NCK(cudaMemcpyAsync(dneg, tb.neg, nk * sizeof(int), cudaMemcpyHostToDevice, st));
  NCK(cudaMemcpyAsync(dt1, tb.t1, tb.start[tb.nq] * sizeof(int4), cudaMemcpyHostToDevice, st));
  NCK(cudaMemcpyAsync(dgather, tb.gather, tb.start[tb.nq] * sizeof(int4), cudaMemcpyHostToDevice, st));
  NCK(cudaMemcpyAsync(dt2, tb.t2, tb.nq * sizeof(int4), cudaMemcpyHostToDevice, st));

  const double lq_scale = d.ck_norm == 0 ? 1.0 / nk : 1.0;
  const double2* Cd[2] = {(const double2*)C[0], nspin == 2 ? (const double2*)C[1] : nullptr};
  // Orbital checks (orthonormality and realness) and the symmetries of L.
  for (int s = 0; s < nspin; ++s) {
    ZgemmArgs z = zdefault();
    z.A = Cd[s];
    z.B = Cd[s];
    z.D = S;
    z.M = n[s];
    z.N = n[s];
    z.K = (int)(nk / ng) * nao;
    z.lda = n[s];
    z.ldb = n[s];
    z.sA = (long long)z.K * n[s];
    z.sB = z.sA;
    z.sD = (long long)n[s] * n[s];
    z.dm_lo = n[s];
    z.dn_lo = 1;
    z.batch = ng;
    NCK(launch_zgemm(z, A_KM, true, B_KN, st));
    NCK(launch_orth_reduce(S, ng, n[s], lq_scale, stats, st));
    NCK(launch_c_real_check(Cd[s], dneg, (int)nk, nao, n[s], stats, st));
  }
  if (d.check_l) NCK(launch_l_check((const double2*)L, dneg, (int)nk, naux, nao, stats, st));

  for (int i = 0; i < tb.nq; ++i) {
    const int e0 = tb.start[i], E = tb.start[i + 1] - e0, w = tb.weight[i];
    const int nc = w == 1 ? 1 : 2;
    for (int s = 0; s < nspin; ++s) {
      const int ns = n[s];
      NCK(launch_gather_orbitals(Cd[s], crep, dgather, e0, E, nao, ns, st));
      ZgemmArgs z = zdefault();  // T_e[mu][P][j] = sum_nu C^{k2}_{nu j} L^{k1,k2}_{P,mu nu}
      z.A = Cd[s];
      z.B = (const double2*)L;
      z.tab = dt1;
      z.tab0 = e0;
      z.M = ns;
      z.N = naux * nao;
      z.K = nao;
      z.lda = ns;
      z.ldb = nao;
      z.sA = (long long)nao * ns;
      z.sB = (long long)naux * nao * nao;
      z.sD = (long long)nao * naux * ns;
      z.dm_lo = 1;
      z.dn_div = nao;
      z.dn_hi = ns;
      z.dn_lo = (long long)naux * ns;
      z.batch = E;
      z.D = T - (long long)e0 * z.sD;
      NCK(launch_zgemm(z, A_KM, false, B_NK, st));
      ZgemmArgs y = zdefault();  // Z[P][i][j] = sum_(r,mu) w_r conj(C^{k1_r}_{mu i}) T_r[mu][P][j]
      y.A = crep - (long long)e0 * nao * ns;
      y.B = T - (long long)e0 * nao * naux * ns;
      y.tab = dt2;
      y.tab0 = i;
      y.M = ns;
      y.N = naux * ns;
      y.lda = ns;
      y.ldb = (long long)naux * ns;
      y.sA = (long long)nao * ns;
      y.sB = (long long)nao * naux * ns;
      y.sD = (long long)naux * ns * ns;
      y.dm_lo = ns;
      y.dn_div = ns;
      y.dn_hi = (long long)ns * ns;
      y.dn_lo = 1;
      y.batch = 1;
      y.D = Z - (long long)i * y.sD;
      NCK(launch_zgemm(y, A_KM, true, B_KN, st));
      NCK(launch_pack_pairs(Z, X[s], 1, naux, ns, nc, lq_scale, st));
    }
    for (int b = 0; b < nblk; ++b) {
      const int sa = b == 2 ? 1 : 0, sb = b == 0 ? 0 : 1;
      DsyrkArgs a;
      std::memset(&a, 0, sizeof(a));
      a.X = X[sa];
      a.Y = X[sb];
      a.out = (double*)eri_out[b];
      a.M = (int)npair[sa];
      a.N = (int)npair[sb];
      a.K = naux * nc;
      a.ldx = npair[sa];
      a.ldy = npair[sb];
      a.ldo = npair[sb];
      a.alpha = (double)w / nk;
      a.mode = b == 1 ? 1 : 0;
      NCK(launch_dsyrk(a, st));
    }
  }
  // The call is synchronous: it waits for its stream and reports the device checks.
  double h[8];
  NCK(cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  const double ortho_tol = d.ortho_tol > 0 ? d.ortho_tol : 1e-10, sym_tol = d.sym_tol > 0 ? d.sym_tol : 1e-10;
  if (!(h[0] <= ortho_tol)) return nfail(DMET_ERR_NOT_ORTHONORMAL, "orthonormality error %.3e", h[0]);
  if (!(h[1] <= sym_tol * std::max(h[2], 1e-300))) return nfail(DMET_ERR_SYMMETRY, "C^-k != conj C^k");
  if (d.check_l && !(h[3] <= sym_tol * std::max(h[5], 1e-300) && h[4] <= sym_tol * std::max(h[5], 1e-300)))
    return nfail(DMET_ERR_SYMMETRY, "L symmetry violated");
  return DMET_OK;
}
