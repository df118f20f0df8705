// Host side of the C ABI: plans, the k-pair scheduler, workspace, dispatch of the
// kernels of Algorithm 1 (section 2.1), staging of host buffers, checks and profiling.

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/dmet_emb.h"
#include "internal.h"
#include "tc_gemm.cuh"

using namespace dmet;

namespace dmet {
char* last_error_buffer() {
  static thread_local char buf[kLastErrorBytes];
  return buf;
}
}  // namespace dmet

namespace {

dmet_status_t fail(dmet_status_t st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dmet::last_error_buffer(), dmet::kLastErrorBytes, fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { dmet::last_error_buffer()[0] = 0; }

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(DMET_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)                          \
  do {                                     \
    dmet_status_t s_ = (expr);             \
    if (s_ != DMET_OK) return s_;          \
  } while (0)

enum KernelClass {
  KC_CHECK_C = 0,
  KC_CHECK_L,
  KC_GATHER,
  KC_TRANSFORM_1,
  KC_TRANSFORM_2,
  KC_PACK,
  KC_CONTRACT,
  KC_CONTRACT_FULL,
  KC_COPY,
  KC_SPLIT,
  KC_TC_TRANSFORM_1,
  KC_TC_TRANSFORM_2,
  KC_TC_PACK,
  KC_TC_CONTRACT,
  KC_FOCK,
  KC_BATH,
  KC_JK_DF,
  KC_FFTDF,
  KC_COUNT
};
const char* const kKcNames[KC_COUNT] = {"check_orbitals",      "check_L",          "gather_orbitals",
                                        "half_transform_1",    "half_transform_2", "pack_pairs",
                                        "contract_s8",         "contract_full",    "host_copy",
                                        "split_operands",      "tc_half_transform_1", "tc_half_transform_2",
                                        "tc_pack_split",       "tc_contract",      "embedding_fock",
                                        "dmet_bath",           "jk_density_fitted", "fftdf_grid"};

// ------------------------------------------------------------------------------------------
// Scheduler: momentum-conserving pairs (k1, k1 + q), negation, q weights and the
// representative k1 of each orbit {k1, -k1 - q} (real-space-real inputs).

struct Sched {
  int nk = 0;
  int mesh[3] = {1, 1, 1};
  std::vector<int> k2_of, neg, qw, nrep, rep_k1, rep_half;
};

int kidx(int a, int b, int c, const int* m) {
  a = ((a % m[0]) + m[0]) % m[0];
  b = ((b % m[1]) + m[1]) % m[1];
  c = ((c % m[2]) + m[2]) % m[2];
  return (a * m[1] + b) * m[2] + c;
}

void build_schedule(const dmet_emb_desc_t& d, Sched& s) {
  const int* m = d.mesh;
  s.nk = m[0] * m[1] * m[2];
  std::memcpy(s.mesh, m, sizeof(s.mesh));
  const int nk = s.nk;
  std::vector<int> t0(nk), t1(nk), t2(nk);
  for (int k = 0; k < nk; ++k) {
    t0[k] = k / (m[1] * m[2]);
    t1[k] = (k / m[2]) % m[1];
    t2[k] = k % m[2];
  }
  s.k2_of.assign((size_t)nk * nk, 0);
  s.neg.assign(nk, 0);
  for (int q = 0; q < nk; ++q)
    for (int k1 = 0; k1 < nk; ++k1)
      s.k2_of[(size_t)q * nk + k1] = kidx(t0[k1] + t0[q], t1[k1] + t1[q], t2[k1] + t2[q], m);
  for (int k = 0; k < nk; ++k) s.neg[k] = kidx(-t0[k], -t1[k], -t2[k], m);
  s.qw.assign(nk, 1);
  s.nrep.assign(nk, 0);
  s.rep_k1.assign((size_t)nk * nk, 0);
  s.rep_half.assign((size_t)nk * nk, 0);
  const bool real = d.sym == DMET_SYM_REAL;
  for (int q = 0; q < nk; ++q) {
    if (real) s.qw[q] = (q == s.neg[q]) ? 1 : (q < s.neg[q] ? 2 : 0);
    int r = 0;
    for (int k1 = 0; k1 < nk; ++k1) {
      if (real) {
        const int partner = s.neg[s.k2_of[(size_t)q * nk + k1]];  // -k1 - q
        if (k1 > partner) continue;
        s.rep_k1[(size_t)q * nk + r] = k1;
        s.rep_half[(size_t)q * nk + r] = (k1 == partner) ? 1 : 0;
      } else {
        s.rep_k1[(size_t)q * nk + r] = k1;
        s.rep_half[(size_t)q * nk + r] = 0;
      }
      ++r;
    }
    s.nrep[q] = r;
  }
}

// The contracted q values of an 8-fold packed problem in the library's order (q = -q first, then
// q < -q, each increasing), restricted to the descriptor's shard; weights alongside.
void contraction_order(const dmet_emb_desc_t& d, const Sched& s, std::vector<int>& order, std::vector<int>& wts) {
  order.clear();
  wts.clear();
  const bool all = d.q_begin == 0 && d.q_end == 0;
  for (int w = 1; w <= 2; ++w)
    for (int q = 0; q < s.nk; ++q)
      if (s.qw[q] == w && (all || (q >= d.q_begin && q < d.q_end))) {
        order.push_back(q);
        wts.push_back(w);
      }
}

// Entry tables for one ordering of q values. Entry e = (q, r) for the r-th representative.
struct Tables {
  std::vector<int> order;      // q values
  std::vector<int> start;      // prefix over order, size order+1 (entries)
  std::vector<int4> t1;        // per entry: {k2, k1*nk + k2, e, nao}
  std::vector<int4> t2;        // per q slot: {start, start, slot, nrep*nao}
  std::vector<int4> gather;    // per entry: {k1, half, 0, 0}
  int4* d_t1 = nullptr;
  int4* d_t2 = nullptr;
  int4* d_gather = nullptr;
};

void build_tables(const Sched& s, const std::vector<int>& order, int nao, Tables& t) {
  t.order = order;
  t.start.assign(order.size() + 1, 0);
  t.t1.clear();
  t.t2.clear();
  t.gather.clear();
  const int nk = s.nk;
  for (size_t i = 0; i < order.size(); ++i) {
    const int q = order[i];
    t.start[i] = (int)t.t1.size();
    for (int r = 0; r < s.nrep[q]; ++r) {
      const int k1 = s.rep_k1[(size_t)q * nk + r];
      const int k2 = s.k2_of[(size_t)q * nk + k1];
      const int e = (int)t.t1.size();
      t.t1.push_back(make_int4(k2, k1 * nk + k2, e, nao));
      t.gather.push_back(make_int4(k1, s.rep_half[(size_t)q * nk + r], 0, 0));
    }
    t.t2.push_back(make_int4(t.start[i], t.start[i], (int)i, s.nrep[q] * nao));
  }
  t.start[order.size()] = (int)t.t1.size();
}

struct Block {
  int b0, b1, w;  // slots [b0, b1) of an ordering, contraction weight
};

// Split-BF16 path: tables built at plan time (they depend on shapes only).
struct MixedPlan {
  int prec = DMET_PREC_BF16X3;         // operand precision (dmet_prec_t)
  int ns = 3, esz = 2, nprod = 6;      // slices per operand, bytes per slice element, slice products
  int K1 = 0, K2 = 0, kseg = 128, kseg1 = 0, crun = 0;
  // Defaults of the segment knobs. The tensor cores add each MMA's products into the FP32 accumulator
  // with an error of about 2^-24 of the accumulator per MMA that grows linearly with the MMAs a
  // segment accumulates (measured 5.5e-8 per MMA of K = 16 on an h-BN-shaped contraction), so every
  // FP32 sum is kept short: 128 K (8 MMAs) per leading-sum segment, also for the first transform, and
  // the correction sum read back after every segment (at the NiO-shaped workload, K = 57 600: the
  // alpha-beta block's error fell from 1.5e-6 with whole-job correction runs to 3.8e-7, at +3% time).
  // 64-K segments in the first transform lower the NiO-shaped errors further (4.6e-7 / 3.8e-7 against
  // 5.3e-7 / 4.5e-7) but cost 4% of the call: its epilogue then reads an accumulator every two K blocks
  // while the previous tile's stores keep it busy.
  int kseg_def = 128, kseg1_def = 128, crun_def = 1;
  // General (complex) orbitals: every q is contracted (weight 1, 2 n_aux K rows each: Re, Im), and
  // the contraction operand of spin s has 3 n_s^2 rows (bra rows ij, then ket rows 2 kl + c);
  // real orbitals: n_pair rows. xrows[s] is that row count.
  bool cplx = false;
  long long xrows[2] = {0, 0};
  int bn1 = 128, bn2 = 128;            // output tile widths of the two transform GEMMs
  long long Rtot = 0, R1 = 0;
  std::vector<Block> blocks;           // contraction order, q-blocks within one weight class
  std::vector<long long> row_base;     // first contraction row of each block
  std::vector<tc::TcJob> jobs;         // all job tables
  std::vector<tc::Segment> segs;       // all segment lists
  // offsets (first, count) into jobs: step 1 / step 2 per block and spin; contraction per block kind
  std::vector<int> j1_off[2], j1_cnt[2], j2_off[2], j2_cnt[2];
  int jc_off[3] = {0, 0, 0}, jc_cnt[3] = {0, 0, 0};
  // per contraction block: split tiles (their K parts are the last jc_split_n * jc_split_f jobs)
  int jc_split_n[3] = {0, 0, 0}, jc_split_f[3] = {1, 1, 1};
  int jc_seg0 = 0, jc_nseg = 0;  // the contraction's segment list (a whole tile's K)
  int jc_tail[3] = {0, 0, 0};    // tiles past the last multiple of the SM count
  // K parts of each last-wave tile: 0 = the heuristic (enough to fill the GPU, at most 8), 1 = no
  // split, 2..8 = that many (dmet_emb_autotune times them)
  int split_pref = 0;
  tc::TcJob* d_jobs = nullptr;
  tc::Segment* d_segs = nullptr;
  long long Ls_rows = 0, A2_rows[2] = {0, 0};
  double useful_t1 = 0, useful_t2 = 0, useful_c = 0;  // per call, all spins
};

struct Prob {
  dmet_emb_desc_t d;
  Sched s;
  int nk, nao, naux, nspin, n[2];
  long long npair[2];
  int pack;            // resolved: S8 or FULL
  double lq_scale;     // 1/Nk (Bloch sum) or 1 (unitary)
  double ortho_scale;  // same
  Tables nat, con;     // natural q order; contraction order (S8 only)
  std::vector<char> nat_conj;  // per q: computed from -q and conjugated (reduced L layout)
  std::vector<char> nat_ok;    // per q: its L blocks are in the caller's layout
  long long n_lblocks = 0;     // (k1, k2) blocks of the caller's L
  std::vector<Block> con_blocks;
  int bq = 1;          // q slots per block
  int* d_neg = nullptr;
  int orth_groups = 1;  // split-K groups of the orthonormality product (a divisor of Nk)
  bool mixed = false;
  MixedPlan mx;
};

struct KStat {
  long long launches = 0;
  double flops = 0, bytes = 0, exec = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};

}  // namespace

// Device scratch of one problem (or shared by every problem of a plan run one at a time).
struct Workspace {
  double2* crep = nullptr;
  double2* T = nullptr;
  double2* Z = nullptr;
  double2* S = nullptr;
  double* X[2] = {nullptr, nullptr};
  double2* lq_all[2] = {nullptr, nullptr};
  double2* full = nullptr;  // one complex ERI block before 4-fold packing
  size_t crep_b = 0, T_b = 0, Z_b = 0, S_b = 0, X_b[2] = {0, 0}, lq_all_b[2] = {0, 0}, full_b = 0;
  // split-BF16 operands
  void* Ls = nullptr;
  void* Cb[2] = {nullptr, nullptr};
  void* Cc = nullptr;
  void* A2 = nullptr;
  double* ZT = nullptr;
  void* Xt[2] = {nullptr, nullptr};
  MixScales* sc = nullptr;
  size_t Ls_b = 0, Cb_b[2] = {0, 0}, Cc_b = 0, A2_b = 0, ZT_b = 0, Xt_b[2] = {0, 0}, sc_b = 0;
};

// One grouped tensor-core launch: its job table (every job naming its entry of the group table),
// the group table, and the work it stands for.
struct GroupedLaunch {
  int kind = 0, prec = 0, bn = 128;
  int pace_bits = 2;  // DMET_TC_PACE bits that pace it
  tc::TcJob* d_jobs = nullptr;
  int njobs = 0;
  void* d_groups = nullptr;
  double flops = 0, bytes = 0, exec = 0;
};

// The batch as grouped launches: round r (block r of every problem that has one), spin s: the
// first and the second half transforms of all those problems, one launch per (precision, tile
// width) class; then the contraction of every ERI block of every problem, one launch per precision.
struct GroupedPlan {
  bool built = false;
  int rounds = 0;
  std::vector<std::vector<GroupedLaunch>> step1, step2;  // [r * 2 + s]
  std::vector<GroupedLaunch> contract;
  double** d_slots = nullptr;  // [problem * 3 + block]: the ERI block pointers of the call
};

struct dmet_emb_plan_s {
  cudaStream_t stream = nullptr;  // the caller's stream
  int device = 0;
  std::vector<Prob> probs;
  size_t ws_limit = 0;
  // One workspace per problem when they all fit the limit (problems then run concurrently on
  // the plan's side streams), else one shared workspace (problems run one after another).
  std::vector<Workspace> ws;
  std::vector<int> ws_of;          // problem -> workspace
  std::vector<cudaStream_t> side;  // side streams of the concurrent mode
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  Workspace* W = nullptr;          // workspace of the problem being enqueued
  cudaStream_t cs = nullptr;       // stream of the problem being enqueued
  double* dstats = nullptr;        // [n_problems][8]
  unsigned int* derr = nullptr;
  // staging of host buffers
  void* stage_in = nullptr;
  size_t stage_in_b = 0;
  void* stage_out = nullptr;
  size_t stage_out_b = 0;
  // scratch of dmet_emb_fock (grown on demand)
  void* fock_ws = nullptr;
  size_t fock_ws_b = 0;
  // scratch of dmet_emb_bath (grown on demand)
  void* bath_ws = nullptr;
  size_t bath_ws_b = 0;
  // scratch of dmet_emb_jk_df (grown on demand)
  void* jk_ws = nullptr;
  size_t jk_ws_b = 0;
  // scratch of dmet_emb_eri_fftdf (grown on demand)
  void* fft_ws = nullptr;
  size_t fft_ws_b = 0;
  // Host L transferred block by block on its own stream: the problem being enqueued waits on
  // xev[b] (its contraction block b's pairs have landed) before its first read of L in block b.
  cudaStream_t xs = nullptr;
  cudaEvent_t xstart = nullptr;
  std::vector<cudaEvent_t> xev;
  bool xpending = false;
  int xnext = 0;              // next block whose copies are still to be queued
  const char* xsrc = nullptr;  // host L of the problem being enqueued
  char* xdst = nullptr;        // its staging buffer
  size_t xbb = 0;              // bytes of one (k1, k2) block
  // per-problem device time of the last profiled call
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pev;
  // CUDA graph of the last device-pointer call (replayed while the pointers stay the same)
  bool use_graph = false;
  long long glaunches = 0;  // kernel launches in the captured graph
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gkey;
  cudaStream_t cap = nullptr;
  // profiling
  bool prof = false;
  KStat ks[KC_COUNT];
  std::vector<cudaEvent_t> pool;
  long long launches = 0;
  // grouped execution of a batch (dmet_emb_batch_mode): requested mode and the launch tables
  int batch_mode = 1;
  GroupedPlan grp;
  // bounded waits of the tensor-core kernels
  unsigned long long wait_ns = tc::kWaitLimitNs;
  int withhold_loads = 0;
  // job pacing (DMET_TC_PACE: bit 1 the contraction launches, the default; bit 2 the transforms too):
  // one counter per workspace and one for the grouped launches
  unsigned int* dsync = nullptr;
  int pace = 1;
  tc::TcCtl ctl(unsigned int* sync = nullptr) const {
    return tc::TcCtl{derr, wait_ns, withhold_loads, pace ? sync : nullptr};
  }
};


namespace {

// ------------------------------------------------------------------------------------------
// Validation and sizes

size_t eri_bytes_of(const dmet_emb_desc_t& d, int block) {
  const int nspin = d.n_spin;
  const int nblk = nspin == 1 ? 1 : 3;
  if (block < 0 || block >= nblk) return 0;
  const long long na = d.n_emb[0];
  const long long nb = nspin == 1 ? na : d.n_emb[1];
  const long long a = block == 2 ? nb : na;
  const long long b = block == 0 ? na : nb;
  int pack = d.eri_pack == DMET_PACK_AUTO ? (d.sym == DMET_SYM_REAL ? DMET_PACK_S8 : DMET_PACK_FULL) : d.eri_pack;
  if (pack == DMET_PACK_S8) {
    const long long pa = a * (a + 1) / 2, pb = b * (b + 1) / 2;
    if (block == 1) return (size_t)(pa * pb) * 8;
    return (size_t)(pa * (pa + 1) / 2) * 8;
  }
  if (pack == DMET_PACK_S4) {
    const long long pa = a * (a + 1) / 2, sa = a * (a - 1) / 2;
    if (block == 1) return (size_t)(pa * b * b) * 16;
    return (size_t)(pa * (pa + 1) / 2 + sa * (sa + 1) / 2) * 16;
  }
  return (size_t)(a * a * b * b) * 16;
}

dmet_status_t validate_desc(const dmet_emb_desc_t& d, int idx) {
  for (int i = 0; i < 3; ++i)
    if (d.mesh[i] < 1 || d.mesh[i] > 4096) return fail(DMET_ERR_INVALID_ARG, "problem %d: mesh[%d] = %d", idx, i, d.mesh[i]);
  const long long nk = (long long)d.mesh[0] * d.mesh[1] * d.mesh[2];
  if (nk > 4096) return fail(DMET_ERR_INVALID_ARG, "problem %d: Nk = %lld > 4096", idx, nk);
  if (d.n_ao < 1 || d.n_ao > 4096) return fail(DMET_ERR_INVALID_ARG, "problem %d: n_ao = %d", idx, d.n_ao);
  if (d.n_aux < 1 || d.n_aux > 65536) return fail(DMET_ERR_INVALID_ARG, "problem %d: n_aux = %d", idx, d.n_aux);
  if (d.n_spin != 1 && d.n_spin != 2) return fail(DMET_ERR_INVALID_ARG, "problem %d: n_spin = %d", idx, d.n_spin);
  for (int s = 0; s < d.n_spin; ++s) {
    if (d.n_emb[s] < 1 || (long long)d.n_emb[s] > nk * d.n_ao)
      return fail(DMET_ERR_INVALID_ARG, "problem %d: n_emb[%d] = %d not in [1, Nk*n_ao]", idx, s, d.n_emb[s]);
    if (d.n_emb[s] > 2047) return fail(DMET_ERR_UNSUPPORTED, "problem %d: n_emb > 2047", idx);
  }
  if (d.ck_norm != 0 && d.ck_norm != 1) return fail(DMET_ERR_INVALID_ARG, "problem %d: ck_norm = %d", idx, d.ck_norm);
  if (d.sym != DMET_SYM_NONE && d.sym != DMET_SYM_REAL) return fail(DMET_ERR_INVALID_ARG, "problem %d: sym = %d", idx, d.sym);
  if (d.eri_pack < 0 || d.eri_pack > 3) return fail(DMET_ERR_INVALID_ARG, "problem %d: eri_pack = %d", idx, d.eri_pack);
  if (d.eri_pack == DMET_PACK_S8 && d.sym != DMET_SYM_REAL)
    return fail(DMET_ERR_INVALID_ARG, "problem %d: 8-fold packing needs sym = DMET_SYM_REAL", idx);
  if (d.check_l != 0 && d.check_l != 1) return fail(DMET_ERR_INVALID_ARG, "problem %d: check_l = %d", idx, d.check_l);
  const int rpack = d.eri_pack == DMET_PACK_AUTO ? (d.sym == DMET_SYM_REAL ? DMET_PACK_S8 : DMET_PACK_FULL) : d.eri_pack;
  if (d.l_layout != DMET_L_FULL && d.l_layout != DMET_L_REDUCED)
    return fail(DMET_ERR_INVALID_ARG, "problem %d: l_layout = %d", idx, d.l_layout);
  if (d.l_layout == DMET_L_REDUCED && (d.sym != DMET_SYM_REAL || rpack != DMET_PACK_S8))
    return fail(DMET_ERR_INVALID_ARG, "problem %d: the reduced L layout needs sym = REAL and 8-fold packing", idx);
  if (d.l_layout == DMET_L_REDUCED && d.check_l)
    return fail(DMET_ERR_INVALID_ARG, "problem %d: check_l compares blocks the reduced L layout leaves out", idx);
  if (!(d.q_begin == 0 && d.q_end == 0)) {
    if (d.q_begin < 0 || d.q_end > nk || d.q_begin >= d.q_end)
      return fail(DMET_ERR_INVALID_ARG, "problem %d: shard [%d, %d) not inside [0, %lld)", idx, d.q_begin, d.q_end, nk);
    if (rpack != DMET_PACK_S8 && !(d.q_begin == 0 && d.q_end == nk))
      return fail(DMET_ERR_UNSUPPORTED, "problem %d: a q shard needs the 8-fold packed output", idx);
  }
  if (d.prec < DMET_PREC_FP64 || d.prec > DMET_PREC_FP16X2)
    return fail(DMET_ERR_INVALID_ARG, "problem %d: prec = %d", idx, d.prec);
  if (d.prec != DMET_PREC_FP64) {
    const int pack = d.eri_pack == DMET_PACK_AUTO ? (d.sym == DMET_SYM_REAL ? DMET_PACK_S8 : DMET_PACK_FULL) : d.eri_pack;
    if (d.sym == DMET_SYM_REAL && pack != DMET_PACK_S8)
      return fail(DMET_ERR_UNSUPPORTED, "problem %d: the tensor-core paths write real orbitals' ERIs 8-fold packed",
                  idx);
  }
  const long long nmax = std::max(d.n_emb[0], d.n_spin == 2 ? d.n_emb[1] : 0);
  if ((long long)d.n_aux * nmax > INT_MAX / 2 || (long long)d.n_aux * d.n_ao > INT_MAX / 2)
    return fail(DMET_ERR_UNSUPPORTED, "problem %d: n_aux*n too large for one launch", idx);
  return DMET_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }


// ------------------------------------------------------------------------------------------
// Launch helpers with per-class accounting and optional CUDA-event timing.

cudaEvent_t get_event(dmet_emb_plan_s* P) {
  if (!P->pool.empty()) {
    cudaEvent_t e = P->pool.back();
    P->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Queues on the copy stream the host-to-device copies of the L blocks that contraction block b of
// the problem being enqueued reads (runs of consecutive pair indices; each pair belongs to one q,
// so to one block), and records xev[b]. Block b + 1's copies are queued right after block b's
// kernels, so that they run on the copy engines while those kernels run.
static dmet_status_t queue_block_copies(dmet_emb_plan_s* P, const Prob& pr, int b) {
  if (!P->xpending || b != P->xnext || b >= (int)pr.con_blocks.size()) return DMET_OK;
  const Block& bl = pr.con_blocks[b];
  std::vector<int> pairs;
  for (int e = pr.con.start[bl.b0]; e < pr.con.start[bl.b1]; ++e) pairs.push_back(pr.con.t1[e].y);
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (P->prof) {
    ta = get_event(P);
    tb = get_event(P);
    if (ta) CK(cudaEventRecord(ta, P->xs));
  }
  // Runs of pair indices in arithmetic progression go as one copy each: contiguous runs as one
  // 1D copy, longer strides as one pitched 2D copy (one row per pair). Each copy call costs the
  // copy engine a few microseconds on top of its bytes (measured: 368 single-pair copies of
  // 2.4 MB move at 163 GB/s, the same pairs in 23 pitched copies at 207 GB/s).
  int max_pitch = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, dev) != cudaSuccess)
    max_pitch = 0;
  for (size_t i = 0; i < pairs.size();) {
    size_t j = i + 1;
    const long long d = j < pairs.size() ? (long long)pairs[j] - pairs[i] : 1;
    while (j < pairs.size() && (long long)pairs[j] - pairs[j - 1] == d) ++j;
    const size_t off = (size_t)pairs[i] * P->xbb, rows = j - i;
    if (d == 1 || rows == 1) {
      CK(cudaMemcpyAsync(P->xdst + off, P->xsrc + off, rows * P->xbb, cudaMemcpyHostToDevice, P->xs));
    } else if ((size_t)d * P->xbb <= (size_t)max_pitch) {
      CK(cudaMemcpy2DAsync(P->xdst + off, (size_t)d * P->xbb, P->xsrc + off, (size_t)d * P->xbb, P->xbb, rows,
                           cudaMemcpyHostToDevice, P->xs));
    } else {
      for (size_t r = i; r < j; ++r) {
        const size_t o = (size_t)pairs[r] * P->xbb;
        CK(cudaMemcpyAsync(P->xdst + o, P->xsrc + o, P->xbb, cudaMemcpyHostToDevice, P->xs));
      }
    }
    i = j;
  }
  CK(cudaEventRecord(P->xev[b], P->xs));
  if (ta && tb) {
    CK(cudaEventRecord(tb, P->xs));
    P->ks[KC_COPY].ev.emplace_back(ta, tb);
  }
  P->ks[KC_COPY].bytes += (double)pairs.size() * P->xbb;
  P->ks[KC_COPY].launches += 1;
  P->xnext = b + 1;
  return DMET_OK;
}

struct Timed {
  dmet_emb_plan_s* P;
  int kc;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(dmet_emb_plan_s* p, int k, double flops, double bytes, int nlaunch = 1, double exec = -1.0) : P(p), kc(k) {
    P->ks[kc].launches += nlaunch;
    P->ks[kc].flops += flops;
    P->ks[kc].bytes += bytes;
    P->ks[kc].exec += exec < 0 ? flops : exec;
    if (kc != KC_COPY) P->launches += nlaunch;
    if (P->prof) {
      a = get_event(P);
      b = get_event(P);
      if (a) cudaEventRecord(a, P->cs);
    }
  }
  ~Timed() {
    if (P->prof && a && b) {
      cudaEventRecord(b, P->cs);
      P->ks[kc].ev.emplace_back(a, b);
    }
  }
};

// Split-K groups of the orthonormality product C^+ C (K = Nk n_AO rows of C): a divisor of K
// whose chunks hold >= 8 rows (one k-step of the FP64 kernel), as many as make about four
// CTAs per SM over the lower-triangle tiles, with the partial products kept under 256 MB.
int orth_groups_for(int nk, int nao, int n) {
  const long long K = (long long)nk * nao;
  const long long tiles = (n + 63) / 64, lower = tiles * (tiles + 1) / 2;
  const long long want = std::max(1LL, 4 * 152 / lower);
  const long long cap = std::max(1LL, (256LL << 20) / std::max(1LL, (long long)n * n * 16));
  int best = 1;
  for (long long g = 1; g <= K; ++g) {
    if (K % g || K / g < 8 || g > want || g > cap) continue;
    best = (int)g;
  }
  return best;
}

ZgemmArgs zargs() {
  ZgemmArgs z;
  std::memset(&z, 0, sizeof(z));
  z.dm_div = INT_MAX;
  z.dn_div = INT_MAX;
  z.alpha = 1.0;
  z.batch = 1;
  return z;
}

dmet_status_t ensure(void** p, size_t* have, size_t need) {
  if (need <= *have) return DMET_OK;
  if (*p) {
    CK(cudaFree(*p));
    *p = nullptr;
    *have = 0;
  }
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(DMET_ERR_OOM, "cudaMalloc of %zu bytes failed", need);
  }
  *have = need;
  return DMET_OK;
}

// Orbital checks: orthonormality (Eq. "fock transform" normalisation with F = S = 1) and,
// for real-space-real inputs, C^{-k} = conj(C^k).
dmet_status_t run_orbital_checks(dmet_emb_plan_s* P, Prob& pr, int p, const double2* const* C) {
  double* st = P->dstats + 8 * p;
  for (int s = 0; s < pr.nspin; ++s) {
    const int n = pr.n[s];
    {
      // split-K over groups of k-points so that the small n x n product fills the GPU
      const int ng = pr.orth_groups;
      const int tiles = (n + 63) / 64;
      Timed t(P, KC_CHECK_C, 8.0 * 64 * 64 * (tiles * (tiles + 1) / 2) * (double)pr.nk * pr.nao,
              16.0 * pr.nk * pr.nao * n, 2);
      ZgemmArgs z = zargs();
      z.A = C[s];
      z.B = C[s];
      z.D = P->W->S;
      z.M = n;
      z.N = n;
      z.K = (pr.nk * pr.nao) / ng;  // the (k, mu) rows split into ng equal chunks
      z.lda = n;
      z.ldb = n;
      z.sA = (long long)z.K * n;
      z.sB = (long long)z.K * n;
      z.sD = (long long)n * n;
      z.dm_lo = n;
      z.dn_lo = 1;
      z.batch = ng;
      z.lower = 1;
      CK(launch_zgemm(z, A_KM, true, B_KN, P->cs));
      CK(launch_orth_reduce(P->W->S, ng, n, pr.ortho_scale, st + 0, P->cs));
    }
    if (pr.d.sym == DMET_SYM_REAL) {
      Timed t(P, KC_CHECK_C, 0.0, 32.0 * pr.nk * pr.nao * n);
      CK(launch_c_real_check(C[s], pr.d_neg, pr.nk, pr.nao, n, st, P->cs));
    }
  }
  return DMET_OK;
}

dmet_status_t run_l_check(dmet_emb_plan_s* P, Prob& pr, int p, const double2* L) {
  if (pr.d.sym != DMET_SYM_REAL || !pr.d.check_l) return DMET_OK;
  const double elems = (double)pr.nk * pr.nk * pr.naux * pr.nao * pr.nao;
  Timed t(P, KC_CHECK_L, 0.0, 16.0 * elems);
  CK(launch_l_check(L, pr.d_neg, pr.nk, pr.naux, pr.nao, P->dstats + 8 * p, P->cs));
  return DMET_OK;
}

// Transformed pairs and their Fourier sum for the q slots [b0, b1) of table `tb`, spin s.
// Writes Z (real-space-real inputs: the half sum over orbit representatives) or, for
// sym = NONE, L^q scaled by lq_scale directly into `dest` (slot-major, z0 = b0).
dmet_status_t run_half_transform(dmet_emb_plan_s* P, Prob& pr, const Tables& tb, int b0, int b1, int s,
                                 const double2* L, const double2* C, double2* dest, int dest_slot0) {
  const int n = pr.n[s], nao = pr.nao, naux = pr.naux;
  const int e0 = tb.start[b0], E = tb.start[b1] - e0;
  if (E <= 0) return DMET_OK;
  {
    Timed t(P, KC_GATHER, 0.0, 32.0 * E * nao * n);
    CK(launch_gather_orbitals(C, P->W->crep, tb.d_gather, e0, E, nao, n, P->cs));
  }
  {
    // T_e[mu][P][j] = sum_nu C^{k2}_{nu j} L^{k1,k2}_{P,mu nu}   (k-AO -> k-EO, ket side)
    ZgemmArgs z = zargs();
    z.A = C;
    z.B = L;
    z.D = P->W->T;
    z.tab = tb.d_t1;
    z.tab0 = e0;
    z.M = n;
    z.N = naux * nao;
    z.K = nao;
    z.lda = n;
    z.ldb = nao;
    z.sA = (long long)nao * n;
    z.sB = (long long)naux * nao * nao;
    z.sD = (long long)nao * naux * n;
    z.dm_lo = 1;
    z.dn_div = nao;
    z.dn_hi = n;
    z.dn_lo = (long long)naux * n;
    z.batch = E;
    // table entries carry absolute indices; T holds this block's entries only
    z.D = P->W->T - (long long)e0 * z.sD;
    Timed t(P, KC_TRANSFORM_1, 8.0 * n * (double)naux * nao * nao * E, 0.0);
    CK(launch_zgemm(z, A_KM, false, B_NK, P->cs));
  }
  {
    // Z_q[P][i][j] = sum_{(r, mu)} w_r conj(C^{k1_r}_{mu i}) T_r[mu][P][j]   (bra side + FT to R=0)
    const bool real = pr.d.sym == DMET_SYM_REAL;
    ZgemmArgs z = zargs();
    z.A = P->W->crep - (long long)e0 * nao * n;
    z.B = P->W->T - (long long)e0 * nao * naux * n;
    z.tab = tb.d_t2;
    z.tab0 = b0;
    z.M = n;
    z.N = naux * n;
    z.lda = n;
    z.ldb = (long long)naux * n;
    z.sA = (long long)nao * n;
    z.sB = (long long)nao * naux * n;
    z.sD = (long long)naux * n * n;
    z.dm_lo = n;
    z.dn_div = n;
    z.dn_hi = (long long)n * n;
    z.dn_lo = 1;
    z.batch = b1 - b0;
    z.alpha = real ? 1.0 : pr.lq_scale;
    z.D = (real ? P->W->Z : dest) - (long long)(real ? b0 : dest_slot0) * z.sD;
    double fl = 0;
    for (int i = b0; i < b1; ++i) fl += 8.0 * n * (double)naux * n * tb.t2[i].w;
    Timed t(P, KC_TRANSFORM_2, fl, 0.0);
    CK(launch_zgemm(z, A_KM, true, B_KN, P->cs));
  }
  return DMET_OK;
}

dmet_status_t transform_range(dmet_emb_plan_s* P, Prob& pr, const double2* L, const double2* const* C, int q_begin,
                              int q_end, double2* const* out, int bq) {
  const bool real = pr.d.sym == DMET_SYM_REAL;
  // q-blocks of at most bq consecutive q with the same conjugation flag
  for (int qa = q_begin; qa < q_end;) {
    int qb = qa + 1;
    while (qb < q_end && qb - qa < bq && pr.nat_conj[qb] == pr.nat_conj[qa]) ++qb;
    for (int s = 0; s < pr.nspin; ++s) {
      const long long slot = (long long)pr.naux * pr.n[s] * pr.n[s];
      double2* dest = out[s] + (long long)(qa - q_begin) * slot;
      TRY(run_half_transform(P, pr, pr.nat, qa, qb, s, L, C[s], dest, qa));
      if (real) {
        Timed t(P, KC_PACK, 0.0, 32.0 * (qb - qa) * (double)slot);
        CK(launch_symmetrize(P->W->Z, dest, qb - qa, pr.naux, pr.n[s], pr.lq_scale, pr.nat_conj[qa], P->cs));
      }
    }
    qa = qb;
  }
  return DMET_OK;
}

dmet_status_t eri_s8(dmet_emb_plan_s* P, Prob& pr, const double2* L, const double2* const* C, void* const* out) {
  for (size_t bi = 0; bi < pr.con_blocks.size(); ++bi) {
    const Block& bl = pr.con_blocks[bi];
    if (P->xpending) {
      TRY(queue_block_copies(P, pr, (int)bi));
      CK(cudaStreamWaitEvent(P->cs, P->xev[bi], 0));
    }
    const int nq = bl.b1 - bl.b0;
    const int nc = bl.w == 1 ? 1 : 2;
    for (int s = 0; s < pr.nspin; ++s) {
      TRY(run_half_transform(P, pr, pr.con, bl.b0, bl.b1, s, L, C[s], nullptr, 0));
      const double elems = (double)nq * pr.naux * pr.n[s] * pr.n[s];
      Timed t(P, KC_PACK, 0.0, 16.0 * elems + 8.0 * nq * pr.naux * nc * (double)pr.npair[s]);
      CK(launch_pack_pairs(P->W->Z, P->W->X[s], nq, pr.naux, pr.n[s], nc, pr.lq_scale, P->cs));
    }
    const int K = nq * pr.naux * nc;
    const double alpha = (double)bl.w / pr.nk;
    for (int blk = 0; blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
      const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
      DsyrkArgs a;
      std::memset(&a, 0, sizeof(a));
      a.X = P->W->X[sa];
      a.Y = P->W->X[sb];
      a.out = (double*)out[blk];
      a.M = (int)pr.npair[sa];
      a.N = (int)pr.npair[sb];
      a.K = K;
      a.ldx = pr.npair[sa];
      a.ldy = pr.npair[sb];
      a.ldo = pr.npair[sb];
      a.alpha = alpha;
      a.mode = blk == 1 ? 1 : 0;
      const double fl = a.mode == 0 ? (double)a.M * (a.M + 1.0) * K : 2.0 * a.M * (double)a.N * K;
      Timed t(P, KC_CONTRACT, fl, 0.0);
      CK(launch_dsyrk(a, P->cs));
    }
  }
  return DMET_OK;
}

dmet_status_t eri_full(dmet_emb_plan_s* P, Prob& pr, const double2* L, const double2* const* C, void* const* out) {
  double2* lq[2] = {P->W->lq_all[0], P->W->lq_all[1]};
  TRY(transform_range(P, pr, L, C, 0, pr.nk, lq, pr.bq));
  const bool s4 = pr.pack == DMET_PACK_S4;
  for (int blk = 0; blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
    const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
    const long long na2 = (long long)pr.n[sa] * pr.n[sa], nb2 = (long long)pr.n[sb] * pr.n[sb];
    // S4: the block's full ERI in the workspace first, then packed
    double2* dst = s4 ? P->W->full : (double2*)out[blk];
    if (s4) CK(cudaMemsetAsync(dst, 0, (size_t)na2 * nb2 * 16, P->cs));
    for (int q = 0; q < pr.nk; ++q) {
      // (ij|kl) += (1/Nk) sum_P L^q_{P,ij} L^{-q}_{P,kl}
      ZgemmArgs z = zargs();
      z.A = lq[sa] + (long long)q * pr.naux * na2;
      z.B = lq[sb] + (long long)pr.s.neg[q] * pr.naux * nb2;
      z.D = dst;
      z.M = (int)na2;
      z.N = (int)nb2;
      z.K = pr.naux;
      z.lda = na2;
      z.ldb = nb2;
      z.dm_lo = nb2;
      z.dn_lo = 1;
      z.alpha = 1.0 / pr.nk;
      z.beta = 1;
      Timed t(P, KC_CONTRACT_FULL, 8.0 * (double)na2 * nb2 * pr.naux, 0.0);
      CK(launch_zgemm(z, A_KM, false, B_KN, P->cs));
    }
    if (s4) {
      Timed t(P, KC_PACK, 0.0, 16.0 * (double)na2 * nb2 + (double)eri_bytes_of(pr.d, blk));
      CK(launch_pack_s4(P->W->full, pr.n[sa], pr.n[sb], blk == 1, (double2*)out[blk], P->cs));
    }
  }
  return DMET_OK;
}

// Workspace for a q-block size bq.
struct WsSizes {
  size_t crep, T, Z, S, X[2], lq_all[2], full;
  size_t total() const { return crep + T + Z + S + X[0] + X[1] + lq_all[0] + lq_all[1] + full; }
};

void partition(const Prob& pr, const Tables& t, const std::vector<int>& wts, int bq, std::vector<Block>& out) {
  out.clear();
  int i = 0;
  const int m = (int)t.order.size();
  while (i < m) {
    int j = i + 1;
    while (j < m && j - i < bq && wts[j] == wts[i]) ++j;
    out.push_back({i, j, wts[i]});
    i = j;
  }
  // Largest blocks first: with host inputs each block's L is copied while the previous block is
  // transformed, so the work left after the last copy is the smallest block's. (Each block
  // keeps its slots, rows and output terms; only the order of processing changes.)
  std::stable_sort(out.begin(), out.end(), [&](const Block& a, const Block& b) {
    return t.start[a.b1] - t.start[a.b0] > t.start[b.b1] - t.start[b.b0];
  });
  (void)pr;
}

int max_entries(const Tables& t, int bq) {
  int best = 0;
  const int m = (int)t.order.size();
  for (int i = 0; i < m; ++i) best = std::max(best, t.start[std::min(m, i + bq)] - t.start[i]);
  return best;
}

WsSizes ws_for(const Prob& pr, int bq) {
  WsSizes w;
  std::memset(&w, 0, sizeof(w));
  const int nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  w.S = (size_t)pr.orth_groups * nmax * nmax * 16;
  if (pr.pack == DMET_PACK_S4) w.full = (size_t)nmax * nmax * nmax * nmax * 16;
  // The tensor-core paths need only the orthonormality product here (and the full block before
  // 4-fold packing).
  if (pr.mixed) return w;
  int E = max_entries(pr.nat, bq);
  if (pr.pack == DMET_PACK_S8) E = std::max(E, max_entries(pr.con, bq));
  w.crep = (size_t)E * pr.nao * nmax * 16;
  w.T = (size_t)E * pr.nao * pr.naux * nmax * 16;
  w.Z = pr.d.sym == DMET_SYM_REAL ? (size_t)bq * pr.naux * nmax * nmax * 16 : 0;
  for (int s = 0; s < pr.nspin; ++s) {
    if (pr.pack == DMET_PACK_S8) w.X[s] = (size_t)bq * pr.naux * 2 * pr.npair[s] * 8;
    else w.lq_all[s] = (size_t)pr.nk * pr.naux * pr.n[s] * pr.n[s] * 16;
  }
  return w;
}

dmet_status_t upload_tables(Tables& t) {
  if (t.t1.empty()) return DMET_OK;
  CK(cudaMalloc(&t.d_t1, t.t1.size() * sizeof(int4)));
  CK(cudaMalloc(&t.d_t2, t.t2.size() * sizeof(int4)));
  CK(cudaMalloc(&t.d_gather, t.gather.size() * sizeof(int4)));
  CK(cudaMemcpy(t.d_t1, t.t1.data(), t.t1.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(t.d_t2, t.t2.data(), t.t2.size() * sizeof(int4), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(t.d_gather, t.gather.data(), t.gather.size() * sizeof(int4), cudaMemcpyHostToDevice));
  return DMET_OK;
}

void free_tables(Tables& t) {
  cudaFree(t.d_t1);
  cudaFree(t.d_t2);
  cudaFree(t.d_gather);
  t.d_t1 = t.d_t2 = t.d_gather = nullptr;
}

void free_workspace(Workspace& w) {
  void* ptrs[] = {w.crep, w.T, w.Z, w.S, w.X[0], w.X[1], w.lq_all[0], w.lq_all[1], w.full,
                  w.Ls, w.Cb[0], w.Cb[1], w.Cc, w.A2, w.ZT, w.Xt[0], w.Xt[1], w.sc};
  for (void* q : ptrs) cudaFree(q);
  w = Workspace();
}

void free_grouped(GroupedPlan& g) {
  for (auto* v : {&g.step1, &g.step2})
    for (auto& ls : *v)
      for (auto& l : ls) {
        cudaFree(l.d_jobs);
        cudaFree(l.d_groups);
      }
  for (auto& l : g.contract) {
    cudaFree(l.d_jobs);
    cudaFree(l.d_groups);
  }
  cudaFree(g.d_slots);
  g = GroupedPlan();
}

void destroy_plan(dmet_emb_plan_s* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  else cudaDeviceSynchronize();
  for (cudaStream_t st : P->side) cudaStreamSynchronize(st);
  for (auto& pr : P->probs) {
    free_tables(pr.nat);
    free_tables(pr.con);
    cudaFree(pr.d_neg);
    cudaFree(pr.mx.d_jobs);
    cudaFree(pr.mx.d_segs);
  }
  for (auto& w : P->ws) free_workspace(w);
  free_grouped(P->grp);
  cudaFree(P->dsync);
  cudaFree(P->derr);
  cudaFree(P->dstats);
  cudaFree(P->stage_in);
  cudaFree(P->stage_out);
  cudaFree(P->fock_ws);
  cudaFree(P->bath_ws);
  cudaFree(P->jk_ws);
  cudaFree(P->fft_ws);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  for (cudaStream_t st : P->side) cudaStreamDestroy(st);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->fork) cudaEventDestroy(P->fork);
  for (auto e : P->join) cudaEventDestroy(e);
  for (auto& e : P->pev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& k : P->ks)
    for (auto& e : k.ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  for (auto e : P->pool) cudaEventDestroy(e);
  if (P->xs) {
    cudaStreamSynchronize(P->xs);
    cudaStreamDestroy(P->xs);
  }
  if (P->xstart) cudaEventDestroy(P->xstart);
  for (auto e : P->xev) cudaEventDestroy(e);
  cudaGetLastError();
  delete P;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Split-BF16 path (tcgen05). Shapes and tables are fixed at plan time; see mixed.cu for the
// kernels and the real-GEMM form of each complex product.

struct MixedMaps {
  CUtensorMap Ls, Cb[2], Cc[2], A2[2], Xt[2];
};

long long padk(long long x) {
  const long long bk = mixed_kblock();
  return (x + bk - 1) / bk * bk;
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0)
    return 152;
  return n;
}

// Bytes of the step-2 output workspace (two-float pairs of one q-block's Z).
long long zt_bytes(const Prob& pr) {
  const long long nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  return (long long)pr.bq * pr.naux * nmax * 2 * nmax * 8;
}

void build_mixed(Prob& pr) {
  MixedPlan& m = pr.mx;
  const int BK = mixed_kblock();
  m.prec = pr.d.prec;
  m.ns = prec_slices(m.prec);
  m.esz = prec_elem_bytes(m.prec);
  m.nprod = prec_products(m.prec);
  // K elements per FP32 segment (a multiple of the K block) of the second transform and the
  // contraction (DMET_TC_KSEG), of the first transform (DMET_TC_KSEG1; 0 = one segment), and the most
  // segments one correction-sum run spans (DMET_TC_CRUN; 0 = no limit).
  auto knob = [](const char* name, int def, int lo, int hi, int mult) {
    const char* e = std::getenv(name);
    if (!e) return def;
    const int v = std::atoi(e);
    return (v >= lo && v <= hi && (mult <= 1 || v % mult == 0)) ? v : def;
  };
  m.kseg = knob("DMET_TC_KSEG", m.kseg_def, BK, 4096, BK);
  m.kseg1 = knob("DMET_TC_KSEG1", m.kseg1_def, 0, 4096, BK);
  m.crun = knob("DMET_TC_CRUN", m.crun_def, 0, 1 << 20, 1);
  const int nk = pr.nk, nao = pr.nao, naux = pr.naux;
  m.K1 = (int)padk(2LL * nao);
  int nrep_max = 1;
  for (int q : pr.con.order) nrep_max = std::max(nrep_max, pr.s.nrep[q]);
  m.K2 = (int)padk(2LL * nrep_max * nao);
  m.blocks = pr.con_blocks;
  m.cplx = pr.d.sym == DMET_SYM_NONE;
  for (int s = 0; s < 2; ++s) m.xrows[s] = s < pr.nspin ? (m.cplx ? 3LL * pr.n[s] * pr.n[s] : pr.npair[s]) : 0;
  int n1 = 0, n2 = 0;
  for (int q : pr.con.order) (pr.s.qw[q] == 1 ? n1 : n2)++;
  // K rows of a q: n_aux for a weight-1 q of real orbitals, 2 n_aux (Re, Im) otherwise
  const long long kq1 = m.cplx ? 2LL * naux : naux;
  m.R1 = padk((long long)n1 * kq1);
  m.Rtot = m.R1 + padk((long long)n2 * 2 * naux);
  m.row_base.clear();
  for (const Block& b : m.blocks)
    m.row_base.push_back(b.w == 1 ? (long long)b.b0 * kq1 : m.R1 + (long long)(b.b0 - n1) * 2 * naux);
  m.segs.clear();
  m.jobs.clear();
  // segments [0, n1seg): the K range of step 1
  const int seg1 = m.kseg1 > 0 ? m.kseg1 : m.K1;
  for (int k0 = 0; k0 < m.K1; k0 += seg1) m.segs.push_back({k0, std::min(m.K1 - k0, seg1), 1.0f, 0});
  const int n1seg = (int)m.segs.size();
  // step 2: per contraction slot, chunks of kseg over its K
  const int nslots = (int)pr.con.order.size();
  std::vector<int> s2_off(nslots), s2_cnt(nslots);
  for (int i = 0; i < nslots; ++i) {
    const long long K = padk(2LL * pr.s.nrep[pr.con.order[i]] * nao);
    s2_off[i] = (int)m.segs.size();
    for (long long k0 = 0; k0 < K; k0 += m.kseg)
      m.segs.push_back({(int)k0, (int)std::min<long long>(K - k0, m.kseg), 1.0f, 0});
    s2_cnt[i] = (int)m.segs.size() - s2_off[i];
  }
  // contraction: class 1 (weight 1) rows [0, R1), class 2 (weight 2) rows [R1, Rtot)
  const int sc_off = (int)m.segs.size();
  for (long long k0 = 0; k0 < m.R1; k0 += m.kseg)
    m.segs.push_back({(int)k0, (int)std::min<long long>(m.R1 - k0, m.kseg), 1.0f, 0});
  for (long long k0 = m.R1; k0 < m.Rtot; k0 += m.kseg)
    m.segs.push_back({(int)k0, (int)std::min<long long>(m.Rtot - k0, m.kseg), 2.0f, 0});
  const int sc_cnt = (int)m.segs.size() - sc_off;
  m.jc_seg0 = sc_off;
  m.jc_nseg = sc_cnt;
  // A correction-sum run never spans a change of weight, nor more than crun segments of one list.
  auto bound = [&](size_t i) {  // a run ends at segment i - 1 and the next starts at i
    m.segs[i - 1].flags |= tc::kRunLast;
    m.segs[i].flags |= tc::kRunFirst;
  };
  for (size_t i = 1; i < m.segs.size(); ++i)
    if (m.segs[i].w != m.segs[i - 1].w) bound(i);
  if (m.crun > 0) {
    std::vector<std::pair<int, int>> lists = {{0, n1seg}, {sc_off, (int)m.segs.size()}};
    for (int i = 0; i < nslots; ++i) lists.push_back({s2_off[i], s2_off[i] + s2_cnt[i]});
    for (auto& l : lists)
      for (int i = l.first + m.crun; i < l.second; i += m.crun) bound((size_t)i);
  }

  auto cdiv = [](long long a, long long b) { return (int)((a + b - 1) / b); };
  const int T = tc::kTile;
  m.Ls_rows = 0;
  for (int sp = 0; sp < pr.nspin; ++sp) {
    const int n = pr.n[sp];
    m.j1_off[sp].clear();
    m.j1_cnt[sp].clear();
    m.j2_off[sp].clear();
    m.j2_cnt[sp].clear();
    for (const Block& bl : m.blocks) {
      const int e0 = pr.con.start[bl.b0];
      m.Ls_rows = std::max(m.Ls_rows, (long long)(pr.con.start[bl.b1] - e0) * naux * nao);
      m.j1_off[sp].push_back((int)m.jobs.size());
      // Tile-major, entry-minor: consecutive jobs write the adjacent column segments (one per
      // representative r) of the same output rows, so L2 merges them into whole lines.
      const int B1 = m.bn1, B2 = m.bn2;
      for (int mt = 0; mt < cdiv((long long)naux * nao, T); ++mt)
        for (int nt = 0; nt < cdiv(2LL * n, B1); ++nt)
          for (int slot = bl.b0; slot < bl.b1; ++slot)
            for (int e = pr.con.start[slot]; e < pr.con.start[slot + 1]; ++e) {
              const int r = e - pr.con.start[slot], el = e - e0, k2 = pr.con.t1[e].x;
              m.jobs.push_back({el * naux * nao + mt * T, k2 * 2 * n + nt * B1,
                                (int)std::min<long long>(T, (long long)naux * nao - mt * T),
                                (int)std::min<long long>(B1, 2LL * n - nt * B1), 0, n1seg, mt * T, nt * B1,
                                (slot - bl.b0) * naux * n, r * 2 * nao});
            }
      m.j1_cnt[sp].push_back((int)m.jobs.size() - m.j1_off[sp].back());
      m.j2_off[sp].push_back((int)m.jobs.size());
      for (int slot = bl.b0; slot < bl.b1; ++slot) {
        const int sl = slot - bl.b0;
        for (int mt = 0; mt < cdiv((long long)naux * n, T); ++mt)
          for (int nt = 0; nt < cdiv(2LL * n, B2); ++nt)
            m.jobs.push_back({sl * naux * n + mt * T, sl * 2 * n + nt * B2,
                              (int)std::min<long long>(T, (long long)naux * n - mt * T),
                              (int)std::min<long long>(B2, 2LL * n - nt * B2), s2_off[slot], s2_cnt[slot],
                              sl * naux * n + mt * T, nt * B2, 0, 0});
      }
      m.j2_cnt[sp].push_back((int)m.jobs.size() - m.j2_off[sp].back());
    }
    m.A2_rows[sp] = (long long)pr.bq * naux * n;
  }
  for (int blk = 0; m.cplx && blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
    // General orbitals: bra rows ij (n_a^2) against ket rows 2 kl + c (2 n_b^2, from row n_b^2 of
    // the ket spin's operand). Same-spin blocks: only the tiles that hold some kl <= ij.
    const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
    const long long ma = (long long)pr.n[sa] * pr.n[sa], nb = 2LL * pr.n[sb] * pr.n[sb];
    m.jc_off[blk] = (int)m.jobs.size();
    m.jc_split_n[blk] = 0;
    m.jc_split_f[blk] = 1;
    const int mts = cdiv(ma, T), nts = cdiv(nb, T), band = 8;
    for (int m0b = 0; m0b < mts; m0b += band)
      for (int nt = 0; nt < nts; ++nt)
        for (int mt = m0b; mt < std::min(mts, m0b + band); ++mt) {
          if (blk != 1 && (long long)nt * (T / 2) > (long long)mt * T + T - 1) continue;
          m.jobs.push_back({mt * T, (int)(nb / 2 + (long long)nt * T), (int)std::min<long long>(T, ma - (long long)mt * T),
                            (int)std::min<long long>(T, nb - (long long)nt * T), sc_off, sc_cnt, mt * T, nt * T, 0, 0});
        }
    m.jc_cnt[blk] = (int)m.jobs.size() - m.jc_off[blk];
  }
  for (int blk = 0; !m.cplx && blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
    const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
    const long long pa = pr.npair[sa], pb = pr.npair[sb];
    m.jc_off[blk] = (int)m.jobs.size();
    // Bands of 8 tile rows, column-major inside a band: the CTAs running at the same time
    // share few row blocks of the operands, which raises their L2 hit rate.
    const int mts = cdiv(pa, T), nts = cdiv(pb, T), band = 8;
    for (int m0b = 0; m0b < mts; m0b += band)
      for (int nt = 0; nt < nts; ++nt)
        for (int mt = m0b; mt < std::min(mts, m0b + band); ++mt) {
          if (blk != 1 && nt > mt) continue;
          m.jobs.push_back({mt * T, nt * T, (int)std::min<long long>(T, pa - mt * T),
                            (int)std::min<long long>(T, pb - nt * T), sc_off, sc_cnt, mt * T, nt * T, 0, 0});
        }
    m.jc_cnt[blk] = (int)m.jobs.size() - m.jc_off[blk];
    // The persistent CTAs take jobs round-robin, so the tiles past the last multiple of the SM
    // count form a short last wave. Those tiles are split in K into f parts (summed afterwards
    // by combine_parts, in the two-float form) so that the last wave fills the GPU. The parts'
    // partial sums go to the step-2 workspace, which the contraction does not otherwise use.
    m.jc_split_n[blk] = 0;
    m.jc_split_f[blk] = 1;
    if (blk != 1) {
      const int G = device_sms();
      const int tail = m.jc_cnt[blk] % G;
      m.jc_tail[blk] = tail;
      int f = tail ? (m.split_pref >= 1 ? std::min(m.split_pref, 8) : std::min(G / tail, 8)) : 1;
      f = std::min(f, sc_cnt);
      const long long cap = zt_bytes(pr) / ((long long)T * T * 8);
      while (f >= 2 && (long long)tail * f > cap) --f;
      if (tail && f >= 2) {
        std::vector<tc::TcJob> tl(m.jobs.end() - tail, m.jobs.end());
        m.jobs.resize(m.jobs.size() - tail);
        for (int t = 0; t < tail; ++t)
          for (int q = 0; q < f; ++q) {
            tc::TcJob j = tl[t];
            const int a = q * sc_cnt / f, b = (q + 1) * sc_cnt / f;
            j.seg0 = sc_off + a;
            j.nseg = b - a;
            j.o2 = 1;
            j.o3 = t * f + q;
            m.jobs.push_back(j);
          }
        m.jc_cnt[blk] = (int)m.jobs.size() - m.jc_off[blk];
        m.jc_split_n[blk] = tail;
        m.jc_split_f[blk] = f;
      }
    }
  }
  // useful flops of one call (the same count as the FP64 path)
  m.useful_t1 = m.useful_t2 = m.useful_c = 0;
  long long K = 0;
  for (int q : pr.con.order) K += (long long)naux * (pr.s.qw[q] == 1 ? 1 : 2);
  for (int sp = 0; sp < pr.nspin; ++sp) {
    const double n = pr.n[sp];
    for (int q : pr.con.order) {
      m.useful_t1 += 8.0 * n * naux * nao * nao * pr.s.nrep[q];
      m.useful_t2 += 8.0 * n * naux * n * nao * pr.s.nrep[q];
    }
    if (m.cplx) {
      // complex products over every q: 8 flops per multiply-add of (ij|kl), kl <= ij, over the n_aux terms
      const double n2 = (double)pr.n[sp] * pr.n[sp];
      m.useful_c += 4.0 * n2 * (n2 + 1.0) * pr.naux * (double)pr.con.order.size();
    } else {
      m.useful_c += (double)pr.npair[sp] * (pr.npair[sp] + 1.0) * K;
    }
  }
  if (pr.nspin == 2)
    m.useful_c += m.cplx ? 8.0 * pr.n[0] * pr.n[0] * (double)pr.n[1] * pr.n[1] * pr.naux * (double)pr.con.order.size()
                         : 2.0 * pr.npair[0] * pr.npair[1] * K;
  (void)nk;
}

// Tensor flops a job range issues: the precision's slice products of 128 x bn x K tiles.
double exec_flops(const MixedPlan& m, int off, int cnt, int bn) {
  double f = 0;
  for (int i = off; i < off + cnt; ++i) {
    const tc::TcJob& j = m.jobs[i];
    long long k = 0;
    for (int g = j.seg0; g < j.seg0 + j.nseg; ++g) k += (long long)m.segs[g].nk;
    f += (double)m.nprod * 2.0 * tc::kTile * bn * (double)k;
  }
  return f;
}

struct MixedWs {
  size_t Ls, Cb[2], Cc, A2, ZT, Xt[2], sc;
};

MixedWs mixed_ws(const Prob& pr) {
  const MixedPlan& m = pr.mx;
  const long long nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  MixedWs w;
  const size_t se = (size_t)m.ns * m.esz;  // bytes of all slices of one element
  w.Ls = se * m.Ls_rows * m.K1;
  for (int s = 0; s < 2; ++s) {
    w.Cb[s] = s < pr.nspin ? se * pr.nk * 2 * pr.n[s] * m.K1 : 0;
    w.Xt[s] = s < pr.nspin ? se * m.xrows[s] * m.Rtot : 0;
  }
  w.Cc = se * pr.bq * 2 * nmax * m.K2;
  w.A2 = se * pr.bq * pr.naux * nmax * m.K2;
  w.ZT = (size_t)zt_bytes(pr);
  w.sc = sizeof(MixScales);
  return w;
}

size_t mixed_total(const MixedWs& w) {
  return w.Ls + w.Cb[0] + w.Cb[1] + w.Cc + w.A2 + w.ZT + w.Xt[0] + w.Xt[1] + w.sc;
}

dmet_status_t mixed_maps(dmet_emb_plan_s* P, const Prob& pr, MixedMaps& mm) {
  const MixedPlan& m = pr.mx;
  const int T = tc::kTile, pc = m.prec, ns = m.ns;
  const long long nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  const long long cc_rows = (long long)pr.bq * 2 * nmax;
  CK(make_tmap_3d(&mm.Ls, pc, P->W->Ls, m.K1, m.Ls_rows, ns, m.K1, m.Ls_rows * m.K1, T));
  for (int s = 0; s < pr.nspin; ++s) {
    const long long n = pr.n[s];
    CK(make_tmap_3d(&mm.Cb[s], pc, P->W->Cb[s], m.K1, pr.nk * 2 * n, ns, m.K1, pr.nk * 2 * n * m.K1, m.bn1));
    CK(make_tmap_3d(&mm.Cc[s], pc, P->W->Cc, m.K2, (long long)pr.bq * 2 * n, ns, m.K2, cc_rows * m.K2, m.bn2));
    CK(make_tmap_interleaved(&mm.A2[s], pc, P->W->A2, m.K2, (long long)pr.bq * pr.naux * n, ns, T));
    CK(make_tmap_3d(&mm.Xt[s], pc, P->W->Xt[s], m.Rtot, m.xrows[s], ns, m.Rtot, m.xrows[s] * m.Rtot, T));
  }
  return DMET_OK;
}

// Algorithmic work of block bi's half transforms, spin s: flops and bytes (operands read once,
// results written once).
void step1_work(const Prob& pr, int bi, int s, double& fl, double& by) {
  const MixedPlan& m = pr.mx;
  const Block& bl = m.blocks[bi];
  const int E = pr.con.start[bl.b1] - pr.con.start[bl.b0], n = pr.n[s];
  const double se = (double)m.ns * m.esz;
  fl = 8.0 * n * (double)pr.naux * pr.nao * pr.nao * E;
  by = se * E * pr.naux * pr.nao * (m.K1 + 2.0 * n);  // L slices read, T slices written
}
void step2_work(const Prob& pr, int bi, int s, double& fl, double& by) {
  const MixedPlan& m = pr.mx;
  const Block& bl = m.blocks[bi];
  const int n = pr.n[s];
  const double se = (double)m.ns * m.esz;
  fl = by = 0;
  for (int i = bl.b0; i < bl.b1; ++i) {
    fl += 8.0 * n * (double)pr.naux * n * pr.con.t2[i].w;
    // the slot's T slices (K = its padded 2 n_rep n_AO) read once, Z written as two-float pairs
    const double K = (double)padk(2LL * pr.s.nrep[pr.con.order[i]] * pr.nao);
    by += se * pr.naux * n * K + se * 2 * n * K + 8.0 * pr.naux * n * 2.0 * n;
  }
}
// Flops and bytes of ERI block blk's contraction.
void contract_work(const Prob& pr, int blk, double& fl, double& by) {
  const MixedPlan& m = pr.mx;
  const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
  const double se = (double)m.ns * m.esz;
  if (m.cplx) {
    const double na2 = (double)pr.n[sa] * pr.n[sa], nb2 = (double)pr.n[sb] * pr.n[sb];
    // 8 flops per complex multiply-add; a same-spin block counts its (ij|kl) with kl <= ij only
    // ((kl|ij) = (ij|kl)), as the real blocks count their symmetric half
    fl = (blk == 1 ? 8.0 * na2 * nb2 : 4.0 * na2 * (na2 + 1.0)) * pr.naux * (double)pr.con.order.size();
    // the bra rows' and ket rows' slices read once, the complex block written once
    by = se * m.Rtot * (na2 + 2 * nb2) + 16.0 * na2 * nb2;
    return;
  }
  long long K = 0;
  for (int q : pr.con.order) K += (long long)pr.naux * (pr.s.qw[q] == 1 ? 1 : 2);
  fl = blk == 1 ? 2.0 * pr.npair[0] * (double)pr.npair[1] * K : (double)pr.npair[sa] * (pr.npair[sa] + 1.0) * K;
  // both operands' slices read once, the packed FP64 result written once
  by = se * m.Rtot * (double)(pr.npair[sa] + (blk == 1 ? pr.npair[sb] : 0)) +
       8.0 * (blk == 1 ? (double)pr.npair[sa] * pr.npair[sb] : pr.npair[sa] * (pr.npair[sa] + 1.0) / 2);
}

// Phases of the tensor-core path of one problem (Algorithm 1), on P->cs with workspace P->W.
// (1) The FP16 operand scales (from the maxima of the L blocks the call reads and of C), the zero
// padding of the contraction operand (pad) and the ket-side orbital operands of every spin.
dmet_status_t mixed_prep(dmet_emb_plan_s* P, Prob& pr, const double2* L, const double2* const* C, bool pad) {
  MixedPlan& m = pr.mx;
  int n1 = 0;
  for (int q : pr.con.order) n1 += pr.s.qw[q] == 1;
  const long long used1 = (long long)n1 * pr.naux * (m.cplx ? 2 : 1);
  const long long used2 = ((long long)pr.con.order.size() - n1) * 2 * pr.naux;
  const int pc = m.prec;
  const double se = (double)m.ns * m.esz;
  MixScales* sc = P->W->sc;
  if (prec_scaled(pc)) {
    const int E_all = (int)pr.con.t1.size();
    int nrep_max = 1;
    for (int q : pr.con.order) nrep_max = std::max(nrep_max, pr.s.nrep[q]);
    const long long c_el[2] = {(long long)pr.nk * pr.nao * pr.n[0], (long long)pr.nk * pr.nao * pr.n[1]};
    Timed t(P, KC_SPLIT, 0.0, 16.0 * E_all * pr.naux * pr.nao * pr.nao + 16.0 * (c_el[0] + c_el[1]), 2 + pr.nspin);
    CK(launch_mix_scales(pc, L, pr.con.d_t1, E_all, (long long)pr.naux * pr.nao * pr.nao, C, c_el, pr.nspin, pr.nao,
                         nrep_max, sc, P->cs));
  }
  for (int s = 0; s < pr.nspin; ++s) {
    // padding columns of the contraction operand read as zeros
    const size_t pitch = (size_t)m.Rtot * m.esz;
    const long long h = (long long)m.ns * m.xrows[s];
    if (pad && m.R1 > used1)
      CK(cudaMemset2DAsync((char*)P->W->Xt[s] + used1 * m.esz, pitch, 0, (size_t)(m.R1 - used1) * m.esz, h, P->cs));
    if (pad && m.Rtot - m.R1 > used2)
      CK(cudaMemset2DAsync((char*)P->W->Xt[s] + (m.R1 + used2) * m.esz, pitch, 0,
                           (size_t)(m.Rtot - m.R1 - used2) * m.esz, h, P->cs));
    Timed t(P, KC_SPLIT, 0.0, 16.0 * pr.nk * pr.nao * pr.n[s] + se * pr.nk * 2 * pr.n[s] * m.K1);
    CK(launch_build_Cb(pc, C[s], pr.nk, pr.nao, pr.n[s], m.K1, P->W->Cb[s], (long long)pr.nk * 2 * pr.n[s] * m.K1,
                       &sc->sC[s], P->cs));
  }
  return DMET_OK;
}

// (2) Block bi's inputs for spin s: the split of its L blocks (with spin 0; both spins read it)
// and the bra-side orbital operand of spin s.
dmet_status_t mixed_block_in(dmet_emb_plan_s* P, Prob& pr, int bi, int s, const double2* L, const double2* const* C) {
  MixedPlan& m = pr.mx;
  const Block& bl = m.blocks[bi];
  const int e0 = pr.con.start[bl.b0], E = pr.con.start[bl.b1] - e0, nq = bl.b1 - bl.b0;
  const int pc = m.prec;
  const double se = (double)m.ns * m.esz;
  MixScales* sc = P->W->sc;
  if (s == 0) {
    if (P->xpending) {
      TRY(queue_block_copies(P, pr, bi));
      CK(cudaStreamWaitEvent(P->cs, P->xev[bi], 0));
    }
    const double rows = (double)E * pr.naux * pr.nao;
    Timed t(P, KC_SPLIT, 0.0, rows * (16.0 * pr.nao + se * m.K1));
    CK(launch_split_L(pc, L, pr.con.d_t1, e0, E, pr.naux, pr.nao, m.K1, P->W->Ls, m.Ls_rows * m.K1, sc, P->cs));
  }
  const long long nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  const long long cc_rows = (long long)pr.bq * 2 * nmax;
  Timed t(P, KC_SPLIT, 0.0, se * nq * 2 * pr.n[s] * m.K2);
  CK(launch_build_Cc(pc, C[s], pr.con.d_gather, pr.con.d_t2, bl.b0, nq, pr.nao, pr.n[s], m.K2, P->W->Cc,
                     cc_rows * m.K2, &sc->sC[s], P->cs));
  return DMET_OK;
}

// The pacing counter of the problem's workspace, cleared on the stream before a contraction launch.
// Not with concurrent problems on side streams: their grids share the SMs, so a grid's CTAs need not
// all be resident at once, and pacing would only wait for its limit.
static unsigned int* pace_counter(dmet_emb_plan_s* P, int bits = 1) {
  if (!(P->pace & bits) || !P->dsync || !P->side.empty()) return nullptr;
  unsigned int* c = P->dsync + (P->W - P->ws.data());
  return cudaMemsetAsync(c, 0, sizeof(unsigned int), P->cs) == cudaSuccess ? c : nullptr;
}

// (3) Block bi's two half transforms of spin s (this problem's own launches).
dmet_status_t mixed_block_gemms(dmet_emb_plan_s* P, Prob& pr, const MixedMaps& mm, int bi, int s) {
  MixedPlan& m = pr.mx;
  const int pc = m.prec, n = pr.n[s];
  const bool scaled = prec_scaled(pc);
  MixScales* sc = P->W->sc;
  double fl = 0, by = 0;
  step1_work(pr, bi, s, fl, by);
  {
    Timed t(P, KC_TC_TRANSFORM_1, fl, by, 1, exec_flops(m, m.j1_off[s][bi], m.j1_cnt[s][bi], m.bn1));
    // (a first transform of K <= 64 is bound by its epilogue's stores; pacing helped it, 10.8 -> 9.4 ms
    // per 10 h-BN-shaped calls, and slowed the K = 224 NiO-shaped one, so it goes with the default then)
    unsigned int* sync = pace_counter(P, m.K1 <= 64 ? 3 : 2);
    CK(launch_tc_split_t(pc, m.bn1, mm.Ls, mm.Cb[s], m.d_jobs + m.j1_off[s][bi], m.j1_cnt[s][bi], m.d_segs, P->W->A2,
                         m.K2, pr.nao, n, P->ctl(sync), scaled ? &sc->f1[s] : nullptr, P->cs));
  }
  step2_work(pr, bi, s, fl, by);
  Timed t(P, KC_TC_TRANSFORM_2, fl, by, 1, exec_flops(m, m.j2_off[s][bi], m.j2_cnt[s][bi], m.bn2));
  unsigned int* sync = pace_counter(P, 2);
  CK(launch_tc_pairs(pc, m.bn2, mm.A2[s], mm.Cc[s], m.d_jobs + m.j2_off[s][bi], m.j2_cnt[s][bi], m.d_segs, P->W->ZT,
                     2LL * n, P->ctl(sync), scaled ? &sc->f2[s] : nullptr, P->cs));
  return DMET_OK;
}

// What dmet_emb_transform_3idx asks of the tensor-core path: L^q for q in [q_begin, q_end) of every
// spin, from the contraction slot slot[q - q_begin] (conjugated where conj[q - q_begin]).
struct Lq3Req {
  int q_begin = 0, q_end = 0;
  std::vector<int> slot;
  std::vector<char> conj;
  double2* const* out = nullptr;
};

// (4) Block bi's rows of the contraction operand of spin s (pair packing), or with req the L^q it
// holds.
dmet_status_t mixed_block_out(dmet_emb_plan_s* P, Prob& pr, int bi, int s, const Lq3Req* req) {
  MixedPlan& m = pr.mx;
  const Block& bl = m.blocks[bi];
  const int nq = bl.b1 - bl.b0, n = pr.n[s], pc = m.prec;
  const double se = (double)m.ns * m.esz;
  MixScales* sc = P->W->sc;
  if (req) {
    for (int i = 0; i < req->q_end - req->q_begin; ++i) {
      const int sl = req->slot[i];
      if (sl < bl.b0 || sl >= bl.b1) continue;
      const long long slot_el = (long long)pr.naux * n * n;
      Timed t(P, KC_PACK, 0.0, 16.0 * slot_el + 16.0 * slot_el);
      CK(launch_lq_from_pairs((const char*)P->W->ZT + (size_t)(sl - bl.b0) * slot_el * 2 * sizeof(float2), pr.naux, n,
                              pr.lq_scale, req->conj[i], m.cplx ? 0 : 1, req->out[s] + i * slot_el, P->cs));
    }
    return DMET_OK;
  }
  if (m.cplx) {
    // every q of a general-orbital problem is its own slot (q = slot)
    Timed t(P, KC_TC_PACK, 0.0, 16.0 * nq * pr.naux * (double)n * n + se * 6.0 * nq * pr.naux * (double)n * n);
    CK(launch_pack_cplx(pc, P->W->ZT, nq, pr.naux, n, pr.con.order[bl.b0], pr.d_neg, P->W->Xt[s],
                        m.xrows[s] * m.Rtot, m.Rtot, &sc->sX[s], P->cs));
  } else {
    const int nc = bl.w == 1 ? 1 : 2;
    Timed t(P, KC_TC_PACK, 0.0, 16.0 * nq * pr.naux * (double)n * n + se * nq * pr.naux * nc * pr.npair[s]);
    CK(launch_pack_split(pc, P->W->ZT, nq, pr.naux, n, nc, P->W->Xt[s], pr.npair[s] * m.Rtot, m.Rtot,
                         m.row_base[bi], &sc->sX[s], P->cs));
  }
  return DMET_OK;
}

// The contraction's output scale: the operand holds Z + Z^T (general orbitals: Z); L^q = s (Z + Z^T)
// (s Z), so the product carries s^2, and 1/Nk.
double contract_scale(const Prob& pr) { return pr.lq_scale * pr.lq_scale / pr.nk; }

// (5) The contraction of every ERI block (this problem's own launches).
dmet_status_t mixed_contract(dmet_emb_plan_s* P, Prob& pr, const MixedMaps& mm, void* const* out) {
  MixedPlan& m = pr.mx;
  const int pc = m.prec;
  const bool scaled = prec_scaled(pc);
  MixScales* sc = P->W->sc;
  const double oscale = contract_scale(pr);
  for (int blk = 0; blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
    const int sa = blk == 2 ? 1 : 0;
    double fl = 0, by = 0;
    contract_work(pr, blk, fl, by);
    if (m.cplx) {
      const long long na2 = (long long)pr.n[sa] * pr.n[sa], nb2 = (long long)pr.n[blk == 0 ? 0 : 1] * pr.n[blk == 0 ? 0 : 1];
      // S4: the block's full ERI in the workspace first, then packed
      const bool s4 = pr.pack == DMET_PACK_S4;
      double* dst = s4 ? (double*)P->W->full : (double*)out[blk];
      {
        Timed t(P, KC_TC_CONTRACT, fl, by, 1, exec_flops(m, m.jc_off[blk], m.jc_cnt[blk], tc::kTile));
        unsigned int* sync = pace_counter(P);
        if (blk == 1)
          CK(launch_tc_rect(pc, mm.Xt[0], mm.Xt[1], m.d_jobs + m.jc_off[1], m.jc_cnt[1], m.d_segs, dst, 2 * nb2, oscale,
                            P->ctl(sync), scaled ? &sc->fc[1] : nullptr, P->cs));
        else
          CK(launch_tc_herm(pc, mm.Xt[sa], mm.Xt[sa], m.d_jobs + m.jc_off[blk], m.jc_cnt[blk], m.d_segs, dst, na2,
                            oscale, P->ctl(sync), scaled ? &sc->fc[blk] : nullptr, P->cs));
      }
      if (s4) {
        Timed t(P, KC_PACK, 0.0, 16.0 * (double)na2 * nb2 + (double)eri_bytes_of(pr.d, blk));
        CK(launch_pack_s4((const double2*)dst, pr.n[sa], pr.n[blk == 0 ? 0 : 1], blk == 1, (double2*)out[blk], P->cs));
      }
      continue;
    }
    const int nsplit = m.jc_split_n[blk], f = m.jc_split_f[blk];
    Timed t(P, KC_TC_CONTRACT, fl, by, nsplit ? 2 : 1, exec_flops(m, m.jc_off[blk], m.jc_cnt[blk], tc::kTile));
    unsigned int* sync = pace_counter(P);
    if (blk == 1) {
      CK(launch_tc_rect(pc, mm.Xt[0], mm.Xt[1], m.d_jobs + m.jc_off[1], m.jc_cnt[1], m.d_segs, (double*)out[1],
                        pr.npair[1], oscale, P->ctl(sync), scaled ? &sc->fc[1] : nullptr, P->cs));
    } else {
      CK(launch_tc_packed(pc, mm.Xt[sa], mm.Xt[sa], m.d_jobs + m.jc_off[blk], m.jc_cnt[blk], m.d_segs,
                          (double*)out[blk], oscale, P->W->ZT, P->ctl(sync), scaled ? &sc->fc[blk] : nullptr, P->cs));
      if (nsplit)
        CK(launch_combine_parts(m.d_jobs + m.jc_off[blk] + m.jc_cnt[blk] - nsplit * f, nsplit, f, P->W->ZT,
                                (double*)out[blk], oscale, P->cs));
    }
  }
  return DMET_OK;
}

// The tensor-core path of Algorithm 1 for one problem: the operand scales and the orbital operands,
// then block by block the split of L, the two half transforms and the pair packing, then the
// contraction. With `req`, only the blocks that hold requested q run, their L^q are written out,
// and nothing is packed or contracted (dmet_emb_transform_3idx).
dmet_status_t eri_mixed(dmet_emb_plan_s* P, Prob& pr, const double2* L, const double2* const* C, void* const* out,
                        const Lq3Req* req = nullptr) {
  MixedPlan& m = pr.mx;
  MixedMaps mm;
  TRY(mixed_maps(P, pr, mm));
  TRY(mixed_prep(P, pr, L, C, !req));
  for (int bi = 0; bi < (int)m.blocks.size(); ++bi) {
    const Block& bl = m.blocks[bi];
    if (req) {
      bool any = false;
      for (int sl : req->slot) any |= sl >= bl.b0 && sl < bl.b1;
      if (!any) continue;
    }
    for (int s = 0; s < pr.nspin; ++s) {
      TRY(mixed_block_in(P, pr, bi, s, L, C));
      TRY(mixed_block_gemms(P, pr, mm, bi, s));
      TRY(mixed_block_out(P, pr, bi, s, req));
    }
  }
  if (req) return DMET_OK;
  return mixed_contract(P, pr, mm, out);
}

// Clears the per-kernel counters (their events go back to the pool).
void reset_profile(dmet_emb_plan_s* P) {
  for (auto& k : P->ks) {
    for (auto& e : k.ev) {
      P->pool.push_back(e.first);
      P->pool.push_back(e.second);
    }
    k.ev.clear();
    k.launches = 0;
    k.flops = 0;
    k.bytes = 0;
    k.exec = 0;
  }
}

// Rebuilds the split-BF16 job tables of a problem (after its tile widths changed) and uploads them.
dmet_status_t upload_mixed(Prob& pr) {
  build_mixed(pr);
  MixedPlan& m = pr.mx;
  cudaFree(m.d_jobs);
  cudaFree(m.d_segs);
  m.d_jobs = nullptr;
  m.d_segs = nullptr;
  if (cudaMalloc(&m.d_jobs, m.jobs.size() * sizeof(tc::TcJob)) != cudaSuccess ||
      cudaMalloc(&m.d_segs, m.segs.size() * sizeof(tc::Segment)) != cudaSuccess ||
      cudaMemcpy(m.d_jobs, m.jobs.data(), m.jobs.size() * sizeof(tc::TcJob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m.d_segs, m.segs.data(), m.segs.size() * sizeof(tc::Segment), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return fail(DMET_ERR_CUDA, "job table upload failed");
  }
  return DMET_OK;
}

// Tuning cache: one line per problem shape, "mesh0 mesh1 mesh2 n_ao n_aux n0 n1 n_spin bn1 bn2".
std::string tune_key(const Prob& pr) {
  char b[160];
  snprintf(b, sizeof(b), "%d %d %d %d %d %d %d %d", pr.d.mesh[0], pr.d.mesh[1], pr.d.mesh[2], pr.nao, pr.naux, pr.n[0],
           pr.n[1], pr.nspin);
  return b;
}

bool tune_cache_lookup(const Prob& pr, int& bn1, int& bn2, int& split) {
  const char* path = std::getenv("DMET_TUNE_CACHE");
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  const std::string key = tune_key(pr);
  char line[256];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    int v[11];
    v[10] = 0;
    const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                           &v[7], &v[8], &v[9], &v[10]);
    if (got != 10 && got != 11) continue;
    char k[160];
    snprintf(k, sizeof(k), "%d %d %d %d %d %d %d %d", v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    if (key == k && (v[8] == 128 || v[8] == 112 || v[8] == 96) && (v[9] == 128 || v[9] == 112 || v[9] == 96) &&
        v[10] >= 0 && v[10] <= 8) {
      bn1 = v[8];
      bn2 = v[9];
      split = v[10];
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(const Prob& pr) {
  const char* path = std::getenv("DMET_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", tune_key(pr).c_str(), pr.mx.bn1, pr.mx.bn2, pr.mx.split_pref);
  fclose(f);
}

// ==========================================================================================
// C ABI

extern "C" {

size_t dmet_emb_eri_bytes(const dmet_emb_desc_t* desc, int32_t block) {
  if (!desc) return 0;
  if (validate_desc(*desc, 0) != DMET_OK) return 0;
  return eri_bytes_of(*desc, block);
}

const char* dmet_emb_last_error(void) { return dmet::last_error_buffer(); }

int32_t dmet_emb_profile_count(void) { return KC_COUNT; }

dmet_status_t dmet_emb_schedule(const dmet_emb_desc_t* desc, int32_t* k2_of, int32_t* neg, int32_t* q_weight,
                                int32_t* n_rep, int32_t* rep_k1, int32_t* rep_half) {
  clear_error();
  if (!desc) return fail(DMET_ERR_INVALID_ARG, "desc is NULL");
  TRY(validate_desc(*desc, 0));
  Sched s;
  build_schedule(*desc, s);
  const size_t nk = s.nk;
  if (k2_of) std::copy(s.k2_of.begin(), s.k2_of.end(), k2_of);
  if (neg) std::copy(s.neg.begin(), s.neg.end(), neg);
  if (q_weight) std::copy(s.qw.begin(), s.qw.end(), q_weight);
  if (n_rep) std::copy(s.nrep.begin(), s.nrep.end(), n_rep);
  if (rep_k1) std::copy(s.rep_k1.begin(), s.rep_k1.begin() + nk * nk, rep_k1);
  if (rep_half) std::copy(s.rep_half.begin(), s.rep_half.begin() + nk * nk, rep_half);
  return DMET_OK;
}

dmet_status_t dmet_emb_l_pairs(const dmet_emb_desc_t* desc, int32_t* pairs, int64_t* n_pairs) {
  clear_error();
  if (!desc || !n_pairs) return fail(DMET_ERR_INVALID_ARG, "desc or n_pairs is NULL");
  TRY(validate_desc(*desc, 0));
  const int pack = desc->eri_pack == DMET_PACK_AUTO ? (desc->sym == DMET_SYM_REAL ? DMET_PACK_S8 : DMET_PACK_FULL)
                                                    : desc->eri_pack;
  if (desc->sym != DMET_SYM_REAL || pack != DMET_PACK_S8)
    return fail(DMET_ERR_UNSUPPORTED, "the reduced pair list exists for sym = REAL with 8-fold packing");
  Sched s;
  build_schedule(*desc, s);
  std::vector<int> order, wts;
  contraction_order(*desc, s, order, wts);
  Tables t;
  build_tables(s, order, desc->n_ao, t);
  *n_pairs = (int64_t)t.t1.size();
  if (pairs)
    for (size_t e = 0; e < t.t1.size(); ++e) pairs[e] = t.t1[e].y;
  return DMET_OK;
}

dmet_status_t dmet_fftdf_plane_waves(const int32_t* mesh, int32_t q, const int32_t* grid, const double* lattice,
                                     int32_t* m_out, double* v_out, int32_t* opposite) {
  clear_error();
  if (!mesh || !grid || !lattice) return fail(DMET_ERR_INVALID_ARG, "NULL argument");
  long long nk = 1, ng = 1;
  for (int d = 0; d < 3; ++d) {
    if (mesh[d] < 1 || mesh[d] > 4096 || grid[d] < 1 || grid[d] > 4096)
      return fail(DMET_ERR_INVALID_ARG, "mesh[%d] = %d, grid[%d] = %d", d, mesh[d], d, grid[d]);
    nk *= mesh[d];
    ng *= grid[d];
  }
  if (nk > 4096 || ng > (1LL << 24)) return fail(DMET_ERR_INVALID_ARG, "Nk = %lld or N_g = %lld too large", nk, ng);
  if (q < 0 || q >= nk) return fail(DMET_ERR_INVALID_ARG, "q = %d outside [0, %lld)", q, nk);
  // reciprocal vectors b_d (rows) with a_d . b_e = 2 pi delta: b = 2 pi (a^-1)^T
  const double* a = lattice;
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  double scale = 0.0;
  for (int i = 0; i < 9; ++i) scale = std::max(scale, std::fabs(a[i]));
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) return fail(DMET_ERR_INVALID_ARG, "singular lattice");
  double b[9];
  const double f = 2.0 * M_PI / det;
  b[0] = f * (a[4] * a[8] - a[5] * a[7]);
  b[1] = f * (a[5] * a[6] - a[3] * a[8]);
  b[2] = f * (a[3] * a[7] - a[4] * a[6]);
  b[3] = f * (a[2] * a[7] - a[1] * a[8]);
  b[4] = f * (a[0] * a[8] - a[2] * a[6]);
  b[5] = f * (a[1] * a[6] - a[0] * a[7]);
  b[6] = f * (a[1] * a[5] - a[2] * a[4]);
  b[7] = f * (a[2] * a[3] - a[0] * a[5]);
  b[8] = f * (a[0] * a[4] - a[1] * a[3]);
  // q's mesh triple (C order) and that of -q
  const int n3[3] = {(int)(q / ((long long)mesh[1] * mesh[2])), (int)((q / mesh[2]) % mesh[1]), (int)(q % mesh[2])};
  // per axis: m_d of each FFT index j_d (m_d = j_d mod g_d with n_d + N_d m_d a signed frequency of the
  // supercell grid, N_d g_d points: [-floor(N g / 2), ceil(N g / 2) - 1]), and the opposite index
  std::vector<int> mj[3], opp[3];
  for (int d = 0; d < 3; ++d) {
    const long long N = mesh[d], g = grid[d], Ng = N * g;
    const long long lo = -(Ng / 2), hi = (Ng + 1) / 2 - 1;
    mj[d].assign(g, 0);
    opp[d].assign(g, 0);
    for (long long j = 0; j < g; ++j) {
      // m = j + g t for the integer t that puts s = n + N m in [lo, hi]
      long long m = j;
      while (n3[d] + N * m > hi) m -= g;
      while (n3[d] + N * m < lo) m += g;
      mj[d][j] = (int)m;
      // -(q + G): s' = -s = n' + N m' with n' = (-n) mod N
      const long long s_ = n3[d] + N * m;
      const long long np = ((-n3[d]) % N + N) % N;
      const long long mp = (-s_ - np) / N;
      opp[d][j] = (int)(((mp % g) + g) % g);
    }
  }
  const double t[3] = {(double)n3[0] / mesh[0], (double)n3[1] / mesh[1], (double)n3[2] / mesh[2]};
  for (long long j0 = 0; j0 < grid[0]; ++j0)
    for (long long j1 = 0; j1 < grid[1]; ++j1)
      for (long long j2 = 0; j2 < grid[2]; ++j2) {
        const long long idx = (j0 * grid[1] + j1) * grid[2] + j2;
        const int mm[3] = {mj[0][j0], mj[1][j1], mj[2][j2]};
        if (m_out) {
          m_out[3 * idx] = mm[0];
          m_out[3 * idx + 1] = mm[1];
          m_out[3 * idx + 2] = mm[2];
        }
        if (v_out) {
          double x[3] = {0.0, 0.0, 0.0};
          for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e) x[e] += (mm[d] + t[d]) * b[3 * d + e];
          const double g2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
          v_out[idx] = g2 > 1e-12 ? 4.0 * M_PI / g2 : 0.0;
        }
        if (opposite) opposite[idx] = (int32_t)(((long long)opp[0][j0] * grid[1] + opp[1][j1]) * grid[2] + opp[2][j2]);
      }
  return DMET_OK;
}

dmet_status_t dmet_emb_plan(const dmet_emb_desc_t* descs, int32_t n_problems, void* stream, size_t workspace_limit,
                            dmet_emb_plan_t* plan) {
  clear_error();
  if (!plan) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  if (!descs) return fail(DMET_ERR_INVALID_ARG, "descs is NULL");
  if (n_problems < 1 || n_problems > 65536) return fail(DMET_ERR_INVALID_ARG, "n_problems = %d", n_problems);
  for (int p = 0; p < n_problems; ++p) TRY(validate_desc(descs[p], p));

  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
    cudaGetLastError();
    return fail(DMET_ERR_CUDA, "no CUDA device visible");
  }
  dmet_emb_plan_s* P = new dmet_emb_plan_s();
  P->stream = (cudaStream_t)stream;
  cudaGetDevice(&P->device);
  P->ws_limit = workspace_limit ? workspace_limit : ((size_t)8 << 30);
  P->probs.resize(n_problems);
  std::vector<WsSizes> wneed(n_problems);
  std::vector<MixedWs> mneed(n_problems);
  for (int p = 0; p < n_problems; ++p) {
    Prob& pr = P->probs[p];
    pr.d = descs[p];
    if (pr.d.ortho_tol <= 0) pr.d.ortho_tol = 1e-10;
    if (pr.d.sym_tol <= 0) pr.d.sym_tol = 1e-10;
    build_schedule(pr.d, pr.s);
    pr.nk = pr.s.nk;
    pr.nao = pr.d.n_ao;
    pr.naux = pr.d.n_aux;
    pr.nspin = pr.d.n_spin;
    pr.n[0] = pr.d.n_emb[0];
    pr.n[1] = pr.nspin == 2 ? pr.d.n_emb[1] : 0;
    for (int s = 0; s < 2; ++s) pr.npair[s] = (long long)pr.n[s] * (pr.n[s] + 1) / 2;
    pr.pack = pr.d.eri_pack == DMET_PACK_AUTO ? (pr.d.sym == DMET_SYM_REAL ? DMET_PACK_S8 : DMET_PACK_FULL)
                                              : pr.d.eri_pack;
    pr.lq_scale = pr.d.ck_norm == 0 ? 1.0 / pr.nk : 1.0;
    pr.orth_groups = orth_groups_for(pr.nk, pr.nao, std::max(pr.n[0], pr.n[1]));
    pr.ortho_scale = pr.lq_scale;
    const bool reduced = pr.d.l_layout == DMET_L_REDUCED;
    std::vector<int> nat(pr.nk);
    pr.nat_conj.assign(pr.nk, 0);
    for (int q = 0; q < pr.nk; ++q) {
      // With the reduced layout a q whose contraction weight is 0 (q > -q) is computed from the
      // blocks of -q: L^q_{P,ij} = conj(L^{-q}_{P,ji}) = conj(L^{-q}_{P,ij}) for real orbitals.
      nat[q] = (reduced && pr.s.qw[q] == 0) ? pr.s.neg[q] : q;
      pr.nat_conj[q] = nat[q] != q;
    }
    build_tables(pr.s, nat, pr.nao, pr.nat);
    std::vector<int> con, wts;
    pr.mixed = pr.d.prec != DMET_PREC_FP64;
    if (pr.pack == DMET_PACK_S8 || pr.mixed) {
      // (general orbitals: every q, in increasing order, weight 1)
      contraction_order(pr.d, pr.s, con, wts);
      build_tables(pr.s, con, pr.nao, pr.con);
    }
    if (reduced) {
      // Block e of the reduced layout is contraction entry e (dmet_emb_l_pairs lists the same pairs).
      std::vector<int> red(pr.nk * pr.nk, -1);
      for (size_t e = 0; e < pr.con.t1.size(); ++e) {
        red[pr.con.t1[e].y] = (int)e;
        pr.con.t1[e].y = (int)e;
      }
      pr.n_lblocks = (long long)pr.con.t1.size();
      // transform_3idx reads the same blocks; a q outside the shard has none
      pr.nat_ok.assign(pr.nk, 1);
      for (int i = 0; i < pr.nk; ++i)
        for (int e = pr.nat.start[i]; e < pr.nat.start[i + 1]; ++e) {
          const int b = red[pr.nat.t1[e].y];
          if (b < 0) pr.nat_ok[i] = 0;
          pr.nat.t1[e].y = b < 0 ? 0 : b;
        }
    } else {
      pr.n_lblocks = (long long)pr.nk * pr.nk;
      pr.nat_ok.assign(pr.nk, 1);
    }
    // q-block size: the largest (<= 8, or <= DMET_QBLOCK, entries per launch <= 65535) whose
    // workspace fits.
    if (pr.mixed) tune_cache_lookup(pr, pr.mx.bn1, pr.mx.bn2, pr.mx.split_pref);
    auto total_for = [&](int b) {
      size_t t = ws_for(pr, b).total();
      if (pr.mixed) {
        pr.bq = b;
        partition(pr, pr.con, wts, b, pr.con_blocks);
        build_mixed(pr);
        t += mixed_total(mixed_ws(pr));
      }
      return t;
    };
    int bq = 8;
    bool capped = false;
    if (const char* e = std::getenv("DMET_QBLOCK")) {
      const int v = std::atoi(e);
      if (v >= 1 && v < bq) bq = v, capped = true;
    }
    // A small problem takes every q of a weight class in one block when that workspace stays under
    // 512 MiB: fewer, fuller launches (the batched workloads), the same results.
    const int all = std::max(1, (int)std::max(pr.con.order.size(), pr.nat.order.size()));
    if (!capped && all > bq) {
      const size_t small = std::min(P->ws_limit, (size_t)512 << 20);
      if (total_for(all) <= small && max_entries(pr.nat, all) <= 65535 && max_entries(pr.con, all) <= 65535) bq = all;
    }
    while (bq > 1 && (total_for(bq) > P->ws_limit || max_entries(pr.nat, bq) > 65535)) --bq;
    const size_t tot = total_for(bq);
    if (tot > P->ws_limit) {
      destroy_plan(P);
      return fail(DMET_ERR_OOM, "problem %d needs %zu bytes of workspace (limit %zu)", p, tot, P->ws_limit);
    }
    WsSizes w = ws_for(pr, bq);
    pr.bq = bq;
    if (pr.pack == DMET_PACK_S8 || pr.mixed) partition(pr, pr.con, wts, bq, pr.con_blocks);
    std::memset(&mneed[p], 0, sizeof(MixedWs));
    if (pr.mixed) {
      build_mixed(pr);
      mneed[p] = mixed_ws(pr);
    }
    wneed[p] = w;
  }
  // Workspace: one per problem if they all fit (concurrent problems), else one shared.
  size_t sum_all = 0;
  for (int p = 0; p < n_problems; ++p) sum_all += wneed[p].total() + mixed_total(mneed[p]);
  const bool concurrent = n_problems > 1 && sum_all <= P->ws_limit;
  P->ws.resize(concurrent ? n_problems : 1);
  P->ws_of.assign(n_problems, 0);
  std::vector<WsSizes> wsz(P->ws.size());
  std::vector<MixedWs> msz(P->ws.size());
  for (size_t i = 0; i < P->ws.size(); ++i) {
    std::memset(&wsz[i], 0, sizeof(WsSizes));
    std::memset(&msz[i], 0, sizeof(MixedWs));
  }
  for (int p = 0; p < n_problems; ++p) {
    const int i = concurrent ? p : 0;
    P->ws_of[p] = i;
    WsSizes& a = wsz[i];
    const WsSizes& b = wneed[p];
    a.crep = std::max(a.crep, b.crep);
    a.T = std::max(a.T, b.T);
    a.Z = std::max(a.Z, b.Z);
    a.S = std::max(a.S, b.S);
    a.full = std::max(a.full, b.full);
    MixedWs& c = msz[i];
    const MixedWs& d = mneed[p];
    c.Ls = std::max(c.Ls, d.Ls);
    c.Cc = std::max(c.Cc, d.Cc);
    c.A2 = std::max(c.A2, d.A2);
    c.ZT = std::max(c.ZT, d.ZT);
    c.sc = std::max(c.sc, d.sc);
    for (int s = 0; s < 2; ++s) {
      a.X[s] = std::max(a.X[s], b.X[s]);
      a.lq_all[s] = std::max(a.lq_all[s], b.lq_all[s]);
      c.Cb[s] = std::max(c.Cb[s], d.Cb[s]);
      c.Xt[s] = std::max(c.Xt[s], d.Xt[s]);
    }
  }
  dmet_status_t st = DMET_OK;
  auto alloc = [&](void** ptr, size_t* have, size_t bytes) {
    if (st == DMET_OK && bytes) st = ensure(ptr, have, bytes);
  };
  for (size_t i = 0; i < P->ws.size(); ++i) {
    Workspace& W = P->ws[i];
    const WsSizes& need = wsz[i];
    const MixedWs& mn = msz[i];
    alloc((void**)&W.crep, &W.crep_b, need.crep);
    alloc((void**)&W.T, &W.T_b, need.T);
    alloc((void**)&W.Z, &W.Z_b, need.Z);
    alloc((void**)&W.S, &W.S_b, need.S);
    alloc((void**)&W.full, &W.full_b, need.full);
    for (int s = 0; s < 2; ++s) {
      alloc((void**)&W.X[s], &W.X_b[s], need.X[s]);
      alloc((void**)&W.lq_all[s], &W.lq_all_b[s], need.lq_all[s]);
    }
    alloc(&W.Ls, &W.Ls_b, mn.Ls);
    alloc(&W.Cc, &W.Cc_b, mn.Cc);
    alloc(&W.A2, &W.A2_b, mn.A2);
    alloc((void**)&W.ZT, &W.ZT_b, mn.ZT);
    alloc((void**)&W.sc, &W.sc_b, mn.sc);
    for (int s = 0; s < 2; ++s) {
      alloc(&W.Cb[s], &W.Cb_b[s], mn.Cb[s]);
      alloc(&W.Xt[s], &W.Xt_b[s], mn.Xt[s]);
    }
    // The split-BF16 operands are read in whole K blocks: whatever a call does not write
    // must hold finite values, so they start at zero.
    if (st == DMET_OK && W.A2 && cudaMemset(W.A2, 0, W.A2_b) != cudaSuccess) st = fail(DMET_ERR_CUDA, "memset");
    for (int s = 0; s < 2; ++s)
      if (st == DMET_OK && W.Xt[s] && cudaMemset(W.Xt[s], 0, W.Xt_b[s]) != cudaSuccess)
        st = fail(DMET_ERR_CUDA, "memset");
  }
  if (st == DMET_OK && concurrent) {
    const int nside = std::min(n_problems, 8);
    P->side.assign(nside, nullptr);
    P->join.assign(nside, nullptr);
    for (int i = 0; st == DMET_OK && i < nside; ++i)
      if (cudaStreamCreateWithFlags(&P->side[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&P->join[i], cudaEventDisableTiming) != cudaSuccess)
        st = fail(DMET_ERR_CUDA, "side stream creation failed");
    if (st == DMET_OK && cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess)
      st = fail(DMET_ERR_CUDA, "event creation failed");
  }
  if (st == DMET_OK && cudaMalloc(&P->derr, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    st = fail(DMET_ERR_OOM, "error word allocation failed");
  }
  if (st == DMET_OK && cudaMemset(P->derr, 0, sizeof(unsigned int)) != cudaSuccess) st = fail(DMET_ERR_CUDA, "memset");
  if (st == DMET_OK && cudaMalloc(&P->dsync, sizeof(unsigned int) * (P->ws.size() + 1)) != cudaSuccess) {
    cudaGetLastError();
    st = fail(DMET_ERR_OOM, "pacing counter allocation failed");
  }
  if (const char* e = std::getenv("DMET_TC_PACE")) P->pace = std::atoi(e) & 3;
  if (st == DMET_OK && cudaMalloc(&P->dstats, sizeof(double) * 8 * n_problems) != cudaSuccess) {
    cudaGetLastError();
    st = fail(DMET_ERR_OOM, "stats allocation failed");
  }
  if (st == DMET_OK && cudaMemset(P->dstats, 0, sizeof(double) * 8 * n_problems) != cudaSuccess)
    st = fail(DMET_ERR_CUDA, "cudaMemset failed");
  for (int p = 0; st == DMET_OK && p < n_problems; ++p) {
    Prob& pr = P->probs[p];
    st = upload_tables(pr.nat);
    if (st == DMET_OK && (pr.pack == DMET_PACK_S8 || pr.mixed)) st = upload_tables(pr.con);
    if (st == DMET_OK && pr.mixed) {
      MixedPlan& m = pr.mx;
      if (cudaMalloc(&m.d_jobs, m.jobs.size() * sizeof(tc::TcJob)) != cudaSuccess ||
          cudaMalloc(&m.d_segs, m.segs.size() * sizeof(tc::Segment)) != cudaSuccess ||
          cudaMemcpy(m.d_jobs, m.jobs.data(), m.jobs.size() * sizeof(tc::TcJob), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(m.d_segs, m.segs.data(), m.segs.size() * sizeof(tc::Segment), cudaMemcpyHostToDevice) !=
              cudaSuccess) {
        cudaGetLastError();
        st = fail(DMET_ERR_CUDA, "job table upload failed");
      }
    }
    if (st == DMET_OK) {
      if (cudaMalloc(&pr.d_neg, sizeof(int) * pr.nk) != cudaSuccess ||
          cudaMemcpy(pr.d_neg, pr.s.neg.data(), sizeof(int) * pr.nk, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        st = fail(DMET_ERR_CUDA, "table upload failed");
      }
    }
  }
  if (st != DMET_OK) {
    char msg[dmet::kLastErrorBytes];
    std::memcpy(msg, dmet::last_error_buffer(), sizeof(msg));
    destroy_plan(P);
    std::memcpy(dmet::last_error_buffer(), msg, sizeof(msg));
    return st;
  }
  *plan = P;
  return DMET_OK;
}

dmet_status_t dmet_emb_destroy(dmet_emb_plan_t plan) {
  clear_error();
  destroy_plan(plan);
  return DMET_OK;
}

// Staging: device pointers pass through; host pointers are copied into plan buffers. With
// `subset`, a host L that the 8-fold-packed schedule reads only in part (one (k1, k2) block per
// transformed pair, see Tables::t1) is copied block run by block run into the same offsets of
// the staging buffer; the blocks the schedule never reads are not transferred (unless the L
// symmetry check, which reads every block, is on).
static dmet_status_t stage_inputs(dmet_emb_plan_s* P, const Prob& pr, const void* L, const void* const* C,
                                  const double2** Ld, const double2** Cd, bool subset = false) {
  const size_t blk = (size_t)pr.naux * pr.nao * pr.nao * 16;  // one (k1, k2) block
  const size_t lb = (size_t)pr.n_lblocks * blk;
  P->xpending = false;
  size_t need = 0;
  const bool lhost = L && !is_device_ptr(L);
  if (lhost) need += lb;
  bool chost[2] = {false, false};
  size_t cb[2] = {0, 0};
  for (int s = 0; s < pr.nspin; ++s) {
    cb[s] = (size_t)pr.nk * pr.nao * pr.n[s] * 16;
    chost[s] = !is_device_ptr(C[s]);
    if (chost[s]) need += cb[s];
  }
  if (need) TRY(ensure(&P->stage_in, &P->stage_in_b, need));
  char* cur = (char*)P->stage_in;
  // C first (small; the orbital checks need it before any L block)
  {
    char* cc = cur + (lhost ? lb : 0);
    for (int s = 0; s < pr.nspin; ++s) {
      Cd[s] = (const double2*)C[s];
      if (chost[s]) {
        Timed t(P, KC_COPY, 0.0, (double)cb[s]);
        CK(cudaMemcpyAsync(cc, C[s], cb[s], cudaMemcpyHostToDevice, P->cs));
        Cd[s] = (const double2*)cc;
        cc += cb[s];
      }
    }
  }
  if (L) *Ld = (const double2*)L;
  if (lhost) {
    if (subset && pr.pack == DMET_PACK_S8 && !pr.d.check_l && !pr.con.t1.empty()) {
      if (!P->xs) {
        CK(cudaStreamCreateWithFlags(&P->xs, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&P->xstart, cudaEventDisableTiming));
      }
      while (P->xev.size() < pr.con_blocks.size()) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        P->xev.push_back(e);
      }
      // the staging buffer is free once the work queued before this call has read it
      CK(cudaEventRecord(P->xstart, P->cs));
      CK(cudaStreamWaitEvent(P->xs, P->xstart, 0));
      P->xsrc = (const char*)L;
      P->xdst = cur;
      P->xbb = blk;
      P->xnext = 0;
      P->xpending = true;
      TRY(queue_block_copies(P, pr, 0));
    } else {
      Timed t(P, KC_COPY, 0.0, (double)lb);
      CK(cudaMemcpyAsync(cur, L, lb, cudaMemcpyHostToDevice, P->cs));
    }
    *Ld = (const double2*)cur;
    cur += lb;
  }
  return DMET_OK;
}

dmet_status_t dmet_emb_transform_3idx(dmet_emb_plan_t P, int32_t problem, const void* L, const void* const* C,
                                      int32_t q_begin, int32_t q_end, void* const* Lq_out) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  Prob& pr = P->probs[problem];
  if (!L || !C || !Lq_out) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  if (q_begin < 0 || q_end > pr.nk || q_begin > q_end) return fail(DMET_ERR_INVALID_ARG, "q range [%d, %d)", q_begin, q_end);
  if (!aligned16(L)) return fail(DMET_ERR_ALIGNMENT, "L not 16-byte aligned");
  for (int s = 0; s < pr.nspin; ++s) {
    if (!C[s] || !Lq_out[s]) return fail(DMET_ERR_INVALID_ARG, "NULL pointer for spin %d", s);
    if (!aligned16(C[s]) || !aligned16(Lq_out[s])) return fail(DMET_ERR_ALIGNMENT, "spin %d pointer not 16-byte aligned", s);
  }
  if (q_begin == q_end) return DMET_OK;
  for (int q = q_begin; q < q_end; ++q)
    if (!pr.nat_ok[q])
      return fail(DMET_ERR_INVALID_ARG, "q = %d: its L blocks are outside the shard of the reduced L layout", q);
  P->cs = P->stream;
  P->W = &P->ws[P->ws_of[problem]];
  const double2* Ld = nullptr;
  const double2* Cd[2] = {nullptr, nullptr};
  TRY(stage_inputs(P, pr, L, C, &Ld, Cd));
  CK(cudaMemsetAsync(P->dstats + 8 * problem, 0, 8 * sizeof(double), P->cs));
  TRY(run_orbital_checks(P, pr, problem, Cd));
  TRY(run_l_check(P, pr, problem, Ld));
  double2* out[2] = {nullptr, nullptr};
  size_t ob[2] = {0, 0}, need = 0;
  bool ohost[2] = {false, false};
  for (int s = 0; s < pr.nspin; ++s) {
    ob[s] = (size_t)(q_end - q_begin) * pr.naux * pr.n[s] * pr.n[s] * 16;
    ohost[s] = !is_device_ptr(Lq_out[s]);
    if (ohost[s]) need += ob[s];
    out[s] = (double2*)Lq_out[s];
  }
  if (need) {
    TRY(ensure(&P->stage_out, &P->stage_out_b, need));
    char* cur = (char*)P->stage_out;
    for (int s = 0; s < pr.nspin; ++s)
      if (ohost[s]) {
        out[s] = (double2*)cur;
        cur += ob[s];
      }
  }
  if (pr.mixed) {
    // the tensor-core transforms of the plan's precision, for the contraction slots that hold the q
    // (q of zero contraction weight: from -q, conjugated; real orbitals, section 2.1)
    Lq3Req req;
    req.q_begin = q_begin;
    req.q_end = q_end;
    req.out = out;
    for (int q = q_begin; q < q_end; ++q) {
      const int qe = pr.s.qw[q] > 0 ? q : pr.s.neg[q];
      const auto it = std::find(pr.con.order.begin(), pr.con.order.end(), qe);
      if (it == pr.con.order.end())
        return fail(DMET_ERR_INVALID_ARG, "q = %d is outside the plan's q shard", q);
      req.slot.push_back((int)(it - pr.con.order.begin()));
      req.conj.push_back(qe != q);
    }
    TRY(eri_mixed(P, pr, Ld, Cd, nullptr, &req));
  } else {
    TRY(transform_range(P, pr, Ld, Cd, q_begin, q_end, out, pr.bq));
  }
  if (need) {
    for (int s = 0; s < pr.nspin; ++s)
      if (ohost[s]) {
        Timed t(P, KC_COPY, 0.0, (double)ob[s]);
        CK(cudaMemcpyAsync(Lq_out[s], out[s], ob[s], cudaMemcpyDeviceToHost, P->cs));
      }
    CK(cudaStreamSynchronize(P->cs));
  }
  CK(cudaGetLastError());
  return DMET_OK;
}

// Queues problem p on P->cs with workspace P->W (Algorithm 1 for that problem).
static dmet_status_t enqueue_problem(dmet_emb_plan_s* P, int p, const void* L, const void* const* C,
                                     void* const* eri_out) {
  Prob& pr = P->probs[p];
  if (P->prof) {
    if ((int)P->pev.size() < (int)P->probs.size()) P->pev.resize(P->probs.size(), {nullptr, nullptr});
    for (cudaEvent_t* e : {&P->pev[p].first, &P->pev[p].second})
      if (!*e) CK(cudaEventCreate(e));
    CK(cudaEventRecord(P->pev[p].first, P->cs));
  }
  const double2* Ld = nullptr;
  const double2* Cd[2] = {nullptr, nullptr};
  TRY(stage_inputs(P, pr, L, C, &Ld, Cd, /*subset=*/true));
  CK(cudaMemsetAsync(P->dstats + 8 * p, 0, 8 * sizeof(double), P->cs));
  TRY(run_orbital_checks(P, pr, p, Cd));
  TRY(run_l_check(P, pr, p, Ld));
  const int nblk = pr.nspin == 1 ? 1 : 3;
  void* out[3] = {nullptr, nullptr, nullptr};
  size_t ob[3] = {0, 0, 0}, need = 0;
  bool ohost[3] = {false, false, false};
  for (int b = 0; b < nblk; ++b) {
    ob[b] = eri_bytes_of(pr.d, b);
    ohost[b] = !is_device_ptr(eri_out[b]);
    if (ohost[b]) need += ob[b];
    out[b] = eri_out[b];
  }
  if (need) {
    TRY(ensure(&P->stage_out, &P->stage_out_b, need));
    char* cur = (char*)P->stage_out;
    for (int b = 0; b < nblk; ++b)
      if (ohost[b]) {
        out[b] = cur;
        cur += ob[b];
      }
  }
  for (int b = 0; b < nblk; ++b) CK(cudaMemsetAsync(out[b], 0, ob[b], P->cs));
  dmet_status_t st = DMET_OK;
  if (pr.mixed) st = eri_mixed(P, pr, Ld, Cd, out);
  else if (pr.pack == DMET_PACK_S8) st = eri_s8(P, pr, Ld, Cd, out);
  else st = eri_full(P, pr, Ld, Cd, out);
  P->xpending = false;
  TRY(st);
  if (need) {
    for (int b = 0; b < nblk; ++b)
      if (ohost[b]) {
        Timed t(P, KC_COPY, 0.0, (double)ob[b]);
        CK(cudaMemcpyAsync(eri_out[b], out[b], ob[b], cudaMemcpyDeviceToHost, P->cs));
      }
  }
  if (P->prof) CK(cudaEventRecord(P->pev[p].second, P->cs));
  return DMET_OK;
}

// ------------------------------------------------------------------------------------------
// Grouped execution of a batch: the tensor-core GEMMs of every problem as persistent launches over
// device tables of per-problem tensor maps, segment lists and output parameters.

// Available when the plan holds several problems, all on tensor-core precisions, each with its own
// workspace (they all fit the limit together), and none whose complex ERI is 4-fold packed (that
// output passes through a per-problem full-block buffer).
bool grouped_available(const dmet_emb_plan_s* P) {
  if (P->probs.size() < 2 || P->side.empty()) return false;
  for (const Prob& pr : P->probs)
    if (!pr.mixed || (pr.mx.cplx && pr.pack == DMET_PACK_S4)) return false;
  return true;
}

bool grouped_active(const dmet_emb_plan_s* P) { return P->batch_mode == 1 && grouped_available(P); }

struct SlotArgs {
  double* p[256];
};
__global__ void set_slots_kernel(double** slots, SlotArgs a, int n) {
  if ((int)threadIdx.x < n) slots[threadIdx.x] = a.p[threadIdx.x];
}

// Uploads one launch: its jobs and its group table (entries filled on the host).
dmet_status_t upload_launch(GroupedLaunch& l, const std::vector<GroupSpec>& specs, const std::vector<tc::TcJob>& jobs) {
  const size_t gb = tc_group_bytes(l.kind, l.prec);
  if (!gb || specs.empty() || jobs.empty()) return fail(DMET_ERR_CUDA, "empty grouped launch");
  std::vector<unsigned char> host(gb * specs.size() + 128);
  unsigned char* h = host.data() + ((128 - ((uintptr_t)host.data() & 127)) & 127);
  CK(tc_group_fill(l.kind, l.prec, specs.data(), (int)specs.size(), h));
  if (cudaMalloc(&l.d_groups, gb * specs.size()) != cudaSuccess ||
      cudaMemcpy(l.d_groups, h, gb * specs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&l.d_jobs, jobs.size() * sizeof(tc::TcJob)) != cudaSuccess ||
      cudaMemcpy(l.d_jobs, jobs.data(), jobs.size() * sizeof(tc::TcJob), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(l.d_groups);
    cudaFree(l.d_jobs);
    l.d_groups = nullptr;
    l.d_jobs = nullptr;
    return fail(DMET_ERR_OOM, "grouped launch tables: device allocation or copy failed");
  }
  l.njobs = (int)jobs.size();
  return DMET_OK;
}

// A class of one grouped launch being assembled: its table entries and jobs.
struct LaunchBuild {
  GroupedLaunch l;
  std::vector<GroupSpec> specs;
  std::vector<tc::TcJob> jobs;
};

// Appends problem jobs [off, off + cnt) of table m.jobs to class lb as entry `spec`.
void add_group(LaunchBuild& lb, const GroupSpec& spec, const MixedPlan& m, int off, int cnt) {
  const int g = (int)lb.specs.size();
  lb.specs.push_back(spec);
  for (int i = off; i < off + cnt; ++i) {
    tc::TcJob j = m.jobs[i];
    j.grp = g;
    lb.jobs.push_back(j);
  }
}

// Drops the captured graph (its nodes refer to the launch tables of the mode it was captured in).
dmet_status_t drop_graph(dmet_emb_plan_s* P) {
  if (!P->gexec) return DMET_OK;
  CK(cudaStreamSynchronize(P->stream));
  CK(cudaGraphExecDestroy(P->gexec));
  P->gexec = nullptr;
  P->gkey.clear();
  return DMET_OK;
}

dmet_status_t build_grouped(dmet_emb_plan_s* P) {
  TRY(drop_graph(P));
  if (P->grp.built) CK(cudaStreamSynchronize(P->stream));
  free_grouped(P->grp);
  GroupedPlan& G = P->grp;
  const int np = (int)P->probs.size();
  // the workspace maps of every problem (the tables keep copies)
  std::vector<MixedMaps> maps(np);
  for (int p = 0; p < np; ++p) {
    P->W = &P->ws[P->ws_of[p]];
    TRY(mixed_maps(P, P->probs[p], maps[p]));
  }
  for (const Prob& pr : P->probs) G.rounds = std::max(G.rounds, (int)pr.mx.blocks.size());
  CK(cudaMalloc(&G.d_slots, sizeof(double*) * 3 * np));
  CK(cudaMemset(G.d_slots, 0, sizeof(double*) * 3 * np));
  G.step1.assign(2 * G.rounds, {});
  G.step2.assign(2 * G.rounds, {});
  for (int r = 0; r < G.rounds; ++r)
    for (int s = 0; s < 2; ++s) {
      std::map<std::pair<int, int>, LaunchBuild> c1, c2;  // by (precision, tile width)
      for (int p = 0; p < np; ++p) {
        Prob& pr = P->probs[p];
        const MixedPlan& m = pr.mx;
        if (r >= (int)m.blocks.size() || s >= pr.nspin) continue;
        Workspace& W = P->ws[P->ws_of[p]];
        const bool scaled = prec_scaled(m.prec);
        GroupSpec a{};
        a.a = &maps[p].Ls;
        a.b = &maps[p].Cb[s];
        a.segs = m.d_segs;
        a.fac = scaled ? &W.sc->f1[s] : nullptr;
        a.out = W.A2;
        a.ld = m.K2;
        a.nao = pr.nao;
        a.n = pr.n[s];
        LaunchBuild& b1 = c1[{m.prec, m.bn1}];
        b1.l.kind = kGroupSplitT;
        if (!b1.specs.empty() && b1.l.pace_bits == 3 && m.K1 > 64) b1.l.pace_bits = 2;
        if (b1.specs.empty()) b1.l.pace_bits = m.K1 <= 64 ? 3 : 2;
        b1.l.prec = m.prec;
        b1.l.bn = m.bn1;
        add_group(b1, a, m, m.j1_off[s][r], m.j1_cnt[s][r]);
        double fl = 0, by = 0;
        step1_work(pr, r, s, fl, by);
        b1.l.flops += fl;
        b1.l.bytes += by;
        b1.l.exec += exec_flops(m, m.j1_off[s][r], m.j1_cnt[s][r], m.bn1);
        GroupSpec z{};
        z.a = &maps[p].A2[s];
        z.b = &maps[p].Cc[s];
        z.segs = m.d_segs;
        z.fac = scaled ? &W.sc->f2[s] : nullptr;
        z.out = W.ZT;
        z.ld = 2LL * pr.n[s];
        LaunchBuild& b2 = c2[{m.prec, m.bn2}];
        b2.l.kind = kGroupPairs;
        b2.l.prec = m.prec;
        b2.l.bn = m.bn2;
        add_group(b2, z, m, m.j2_off[s][r], m.j2_cnt[s][r]);
        step2_work(pr, r, s, fl, by);
        b2.l.flops += fl;
        b2.l.bytes += by;
        b2.l.exec += exec_flops(m, m.j2_off[s][r], m.j2_cnt[s][r], m.bn2);
      }
      for (auto& kv : c1) {
        TRY(upload_launch(kv.second.l, kv.second.specs, kv.second.jobs));
        G.step1[2 * r + s].push_back(kv.second.l);
      }
      for (auto& kv : c2) {
        TRY(upload_launch(kv.second.l, kv.second.specs, kv.second.jobs));
        G.step2[2 * r + s].push_back(kv.second.l);
      }
    }
  // the contraction: every block of every problem, whole tiles (no K split: the tiles of all
  // problems share the launch's last wave)
  std::map<int, LaunchBuild> cc;
  for (int p = 0; p < np; ++p) {
    Prob& pr = P->probs[p];
    const MixedPlan& m = pr.mx;
    Workspace& W = P->ws[P->ws_of[p]];
    const bool scaled = prec_scaled(m.prec);
    for (int blk = 0; blk < (pr.nspin == 1 ? 1 : 3); ++blk) {
      const int sa = blk == 2 ? 1 : 0, sb = blk == 0 ? 0 : 1;
      GroupSpec c{};
      c.a = &maps[p].Xt[sa];
      c.b = &maps[p].Xt[sb];
      c.segs = m.d_segs;
      c.fac = scaled ? &W.sc->fc[blk] : nullptr;
      c.outp = G.d_slots + 3 * p + blk;
      c.scale = contract_scale(pr);
      if (m.cplx) {
        c.mode = blk == 1 ? 1 : 2;
        c.ld = 2LL * pr.n[sb] * pr.n[sb];
      } else {
        c.mode = blk == 1 ? 1 : 0;
        c.ld = pr.npair[sb];
      }
      LaunchBuild& b = cc[m.prec];
      b.l.kind = kGroupContract;
      b.l.prec = m.prec;
      b.l.bn = tc::kTile;
      const int g = (int)b.specs.size();
      b.specs.push_back(c);
      const int f = m.jc_split_f[blk], nsplit = m.jc_split_n[blk];
      const int whole = m.jc_cnt[blk] - nsplit * f;
      long long kc = 0;  // K of a whole tile
      for (int gi = m.jc_seg0; gi < m.jc_seg0 + m.jc_nseg; ++gi) kc += m.segs[gi].nk;
      const size_t before = b.jobs.size();
      for (int i = m.jc_off[blk]; i < m.jc_off[blk] + m.jc_cnt[blk]; ++i) {
        tc::TcJob j = m.jobs[i];
        if (i - m.jc_off[blk] >= whole) {
          // a split tile: its first part stands for the tile, over the whole K
          if ((i - m.jc_off[blk] - whole) % f) continue;
          j.seg0 = m.jc_seg0;
          j.nseg = m.jc_nseg;
          j.o2 = j.o3 = 0;
        }
        j.grp = g;
        b.jobs.push_back(j);
      }
      double fl = 0, by = 0;
      contract_work(pr, blk, fl, by);
      b.l.flops += fl;
      b.l.bytes += by;
      b.l.exec += (double)(b.jobs.size() - before) * m.nprod * 2.0 * tc::kTile * tc::kTile * (double)kc;
    }
  }
  for (auto& kv : cc) {
    TRY(upload_launch(kv.second.l, kv.second.specs, kv.second.jobs));
    G.contract.push_back(kv.second.l);
  }
  G.built = true;
  return DMET_OK;
}

// Fork: the side streams wait for `origin`'s work so far. Join: `origin` waits for theirs.
static dmet_status_t fork_sides(dmet_emb_plan_s* P, cudaStream_t origin) {
  CK(cudaEventRecord(P->fork, origin));
  for (cudaStream_t st : P->side) CK(cudaStreamWaitEvent(st, P->fork, 0));
  return DMET_OK;
}
static dmet_status_t join_sides(dmet_emb_plan_s* P, cudaStream_t origin) {
  for (size_t i = 0; i < P->side.size(); ++i) {
    CK(cudaEventRecord(P->join[i], P->side[i]));
    CK(cudaStreamWaitEvent(origin, P->join[i], 0));
  }
  return DMET_OK;
}

static dmet_status_t run_grouped(dmet_emb_plan_s* P, const GroupedLaunch& l, int kc) {
  unsigned int* sync = nullptr;
  if ((l.kind == kGroupContract ? (P->pace & 1) : (P->pace & l.pace_bits)) && P->dsync) {
    sync = P->dsync + P->ws.size();
    CK(cudaMemsetAsync(sync, 0, sizeof(unsigned int), P->cs));
  }
  Timed t(P, kc, l.flops, l.bytes, 1, l.exec);
  CK(launch_tc_grouped(l.kind, l.prec, l.bn, l.d_groups, l.d_jobs, l.njobs, P->ctl(sync), P->cs));
  return DMET_OK;
}

// The batch in grouped form (device inputs only). Per problem, on the side streams: the checks,
// the output clearing, the operand scales and the ket-side orbital operands. Then per round r and
// spin s: each problem's split of its block r and bra-side operand (side streams), the grouped
// first and second half transforms of all problems (the caller's stream), each problem's pair
// packing (side streams). Last, the grouped contraction of every ERI block.
static dmet_status_t enqueue_grouped(dmet_emb_plan_s* P, cudaStream_t origin, const void* const* L,
                                     const void* const* const* C, void* const* const* eri_out) {
  const int np = (int)P->probs.size(), ns = (int)P->side.size();
  GroupedPlan& G = P->grp;
  // this call's ERI block pointers, carried to the device by a kernel's parameters (so that a
  // captured graph replays them)
  for (int p0 = 0; p0 < 3 * np; p0 += 256) {
    SlotArgs a;
    std::memset(&a, 0, sizeof(a));
    const int cnt = std::min(256, 3 * np - p0);
    for (int i = 0; i < cnt; ++i) {
      const int p = (p0 + i) / 3, b = (p0 + i) % 3;
      a.p[i] = b < (P->probs[p].nspin == 1 ? 1 : 3) ? (double*)eri_out[p][b] : nullptr;
    }
    set_slots_kernel<<<1, 256, 0, origin>>>(G.d_slots + p0, a, cnt);
    CK(cudaGetLastError());
    P->launches += 1;
  }
  std::vector<const double2*> Ld(np, nullptr);
  std::vector<std::array<const double2*, 2>> Cd(np, {nullptr, nullptr});
  TRY(fork_sides(P, origin));
  for (int p = 0; p < np; ++p) {
    Prob& pr = P->probs[p];
    P->cs = P->side[p % ns];
    P->W = &P->ws[P->ws_of[p]];
    if (P->prof) {
      if ((int)P->pev.size() < np) P->pev.resize(np, {nullptr, nullptr});
      for (cudaEvent_t* e : {&P->pev[p].first, &P->pev[p].second})
        if (!*e) CK(cudaEventCreate(e));
      CK(cudaEventRecord(P->pev[p].first, P->cs));
    }
    TRY(stage_inputs(P, pr, L[p], C[p], &Ld[p], Cd[p].data()));
    CK(cudaMemsetAsync(P->dstats + 8 * p, 0, 8 * sizeof(double), P->cs));
    TRY(run_orbital_checks(P, pr, p, Cd[p].data()));
    TRY(run_l_check(P, pr, p, Ld[p]));
    for (int b = 0; b < (pr.nspin == 1 ? 1 : 3); ++b)
      CK(cudaMemsetAsync(eri_out[p][b], 0, eri_bytes_of(pr.d, b), P->cs));
    TRY(mixed_prep(P, pr, Ld[p], Cd[p].data(), true));
  }
  for (int r = 0; r < G.rounds; ++r)
    for (int s = 0; s < 2; ++s) {
      if (G.step1[2 * r + s].empty()) continue;
      for (int p = 0; p < np; ++p) {
        Prob& pr = P->probs[p];
        if (r >= (int)pr.mx.blocks.size() || s >= pr.nspin) continue;
        P->cs = P->side[p % ns];
        P->W = &P->ws[P->ws_of[p]];
        TRY(mixed_block_in(P, pr, r, s, Ld[p], Cd[p].data()));
      }
      TRY(join_sides(P, origin));
      P->cs = origin;
      for (const GroupedLaunch& l : G.step1[2 * r + s]) TRY(run_grouped(P, l, KC_TC_TRANSFORM_1));
      for (const GroupedLaunch& l : G.step2[2 * r + s]) TRY(run_grouped(P, l, KC_TC_TRANSFORM_2));
      TRY(fork_sides(P, origin));
      for (int p = 0; p < np; ++p) {
        Prob& pr = P->probs[p];
        if (r >= (int)pr.mx.blocks.size() || s >= pr.nspin) continue;
        P->cs = P->side[p % ns];
        P->W = &P->ws[P->ws_of[p]];
        TRY(mixed_block_out(P, pr, r, s, nullptr));
      }
    }
  TRY(join_sides(P, origin));
  P->cs = origin;
  for (const GroupedLaunch& l : G.contract) TRY(run_grouped(P, l, KC_TC_CONTRACT));
  if (P->prof)
    for (int p = 0; p < np; ++p) CK(cudaEventRecord(P->pev[p].second, origin));
  return DMET_OK;
}

// Queues every problem behind `origin`: concurrently on the side streams (fork/join) when each
// problem has its own workspace and no host staging is needed, else one after another.
static dmet_status_t enqueue_all(dmet_emb_plan_s* P, cudaStream_t origin, bool staged, const void* const* L,
                                 const void* const* const* C, void* const* const* eri_out) {
  const int np = (int)P->probs.size();
  if (!staged && grouped_active(P)) return enqueue_grouped(P, origin, L, C, eri_out);
  if (!staged && !P->side.empty()) {
    const int ns = (int)P->side.size();
    CK(cudaEventRecord(P->fork, origin));
    for (int i = 0; i < ns; ++i) CK(cudaStreamWaitEvent(P->side[i], P->fork, 0));
    for (int p = 0; p < np; ++p) {
      P->cs = P->side[p % ns];
      P->W = &P->ws[P->ws_of[p]];
      TRY(enqueue_problem(P, p, L[p], C[p], eri_out[p]));
    }
    for (int i = 0; i < ns; ++i) {
      CK(cudaEventRecord(P->join[i], P->side[i]));
      CK(cudaStreamWaitEvent(origin, P->join[i], 0));
    }
    return DMET_OK;
  }
  for (int p = 0; p < np; ++p) {
    P->cs = origin;
    P->W = &P->ws[P->ws_of[p]];
    TRY(enqueue_problem(P, p, L[p], C[p], eri_out[p]));
  }
  return DMET_OK;
}

dmet_status_t dmet_emb_eri(dmet_emb_plan_t P, const void* const* L, const void* const* const* C,
                           void* const* const* eri_out) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (!L || !C || !eri_out) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  const int np = (int)P->probs.size();
  bool staged = false;
  std::vector<const void*> key;
  for (int p = 0; p < np; ++p) {
    const Prob& pr = P->probs[p];
    if (!L[p] || !C[p] || !eri_out[p]) return fail(DMET_ERR_INVALID_ARG, "problem %d: NULL pointer", p);
    if (!aligned16(L[p])) return fail(DMET_ERR_ALIGNMENT, "problem %d: L not 16-byte aligned", p);
    staged |= !is_device_ptr(L[p]);
    key.push_back(L[p]);
    for (int s = 0; s < pr.nspin; ++s) {
      if (!C[p][s]) return fail(DMET_ERR_INVALID_ARG, "problem %d: C[%d] is NULL", p, s);
      if (!aligned16(C[p][s])) return fail(DMET_ERR_ALIGNMENT, "problem %d: C[%d] not 16-byte aligned", p, s);
      staged |= !is_device_ptr(C[p][s]);
      key.push_back(C[p][s]);
    }
    for (int b = 0; b < (pr.nspin == 1 ? 1 : 3); ++b) {
      if (!eri_out[p][b]) return fail(DMET_ERR_INVALID_ARG, "problem %d: eri_out[%d] is NULL", p, b);
      if (!aligned16(eri_out[p][b])) return fail(DMET_ERR_ALIGNMENT, "problem %d: eri_out[%d] not 16-byte aligned", p, b);
      staged |= !is_device_ptr(eri_out[p][b]);
      key.push_back(eri_out[p][b]);
    }
  }
  if (!staged && grouped_active(P) && !P->grp.built) TRY(build_grouped(P));
  if (!staged && P->use_graph && !P->prof) {
    // Replay the captured graph while the buffers are the same; otherwise capture anew.
    if (!(P->gexec && key == P->gkey)) {
      if (P->gexec) {
        CK(cudaGraphExecDestroy(P->gexec));
        P->gexec = nullptr;
      }
      if (!P->cap) CK(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
      const long long l0 = P->launches;
      CK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
      const dmet_status_t st = enqueue_all(P, P->cap, false, L, C, eri_out);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(P->cap, &g);
      if (st != DMET_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return fail(DMET_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&P->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        P->gexec = nullptr;
        return fail(DMET_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ei));
      }
      P->gkey = key;
      P->glaunches = P->launches - l0;
      P->launches = l0;
    }
    CK(cudaGraphLaunch(P->gexec, P->stream));
    P->launches += P->glaunches;
    return DMET_OK;
  }
  TRY(enqueue_all(P, P->stream, staged, L, C, eri_out));
  if (staged) CK(cudaStreamSynchronize(P->stream));
  CK(cudaGetLastError());
  return DMET_OK;
}

dmet_status_t dmet_emb_graph(dmet_emb_plan_t P, int32_t enable) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  P->use_graph = enable != 0;
  if (!P->use_graph && P->gexec) {
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
    P->gkey.clear();
  }
  return DMET_OK;
}

dmet_status_t dmet_emb_problem_ms(dmet_emb_plan_t P, int32_t problem, double* ms) {
  clear_error();
  if (!P || !ms) return fail(DMET_ERR_INVALID_ARG, "NULL argument");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  if (problem >= (int)P->pev.size() || !P->pev[problem].first)
    return fail(DMET_ERR_INVALID_ARG, "problem %d has no profiled call", problem);
  CK(cudaStreamSynchronize(P->stream));
  float t = 0;
  CK(cudaEventElapsedTime(&t, P->pev[problem].first, P->pev[problem].second));
  *ms = t;
  return DMET_OK;
}

dmet_status_t dmet_emb_autotune(dmet_emb_plan_t P, const void* const* L, const void* const* const* C,
                                void* const* const* eri_out) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  bool any = false;
  for (const Prob& pr : P->probs) any |= pr.mixed;
  if (!any) return DMET_OK;
  const bool prof = P->prof;
  TRY(drop_graph(P));
  // each problem is timed on its own (side-stream mode); the grouped tables are rebuilt afterwards
  const int mode = P->batch_mode;
  P->batch_mode = 0;
  CK(cudaStreamSynchronize(P->stream));
  free_grouped(P->grp);
  const int cand[3] = {128, 112, 96};
  const int np = (int)P->probs.size();
  int nmixed = 0;
  for (const Prob& pr : P->probs) nmixed += pr.mixed;
  // One mixed problem: the two transform GEMMs are timed (and chosen) separately from the
  // per-kernel CUDA events; several: each problem's whole time decides one width for both.
  std::vector<double> best(np, 1e300), best1(np, 1e300), best2(np, 1e300);
  std::vector<int> bn1(np, 128), bn2(np, 128);
  for (int c : cand) {
    for (Prob& pr : P->probs)
      if (pr.mixed) {
        pr.mx.bn1 = pr.mx.bn2 = c;
        TRY(upload_mixed(pr));
      }
    P->prof = false;
    TRY(dmet_emb_eri(P, L, C, eri_out));  // warm-up with this tile width
    reset_profile(P);
    P->prof = true;
    TRY(dmet_emb_eri(P, L, C, eri_out));
    CK(cudaStreamSynchronize(P->stream));
    double t1 = 0, t2 = 0;
    for (int k : {(int)KC_TC_TRANSFORM_1, (int)KC_TC_TRANSFORM_2})
      for (auto& e : P->ks[k].ev) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        (k == KC_TC_TRANSFORM_1 ? t1 : t2) += ms;
      }
    for (int p = 0; p < np; ++p) {
      if (!P->probs[p].mixed) continue;
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, P->pev[p].first, P->pev[p].second));
      if (nmixed == 1) {
        if (t1 < best1[p]) best1[p] = t1, bn1[p] = c;
        if (t2 < best2[p]) best2[p] = t2, bn2[p] = c;
      } else if (ms < best[p]) {
        best[p] = ms;
        bn1[p] = bn2[p] = c;
      }
    }
  }
  for (int p = 0; p < np; ++p) {
    Prob& pr = P->probs[p];
    if (!pr.mixed) continue;
    pr.mx.bn1 = bn1[p];
    pr.mx.bn2 = bn2[p];
    TRY(upload_mixed(pr));
  }
  // split-K of the contraction's last wave (problems whose packed blocks leave a partial wave):
  // the heuristic, no split, 2, 4 and 8 parts per tile, timed the same way
  bool tail = false;
  for (const Prob& pr : P->probs) tail |= pr.mixed && (pr.mx.jc_tail[0] > 0 || pr.mx.jc_tail[2] > 0);
  if (tail) {
    std::vector<double> bs(np, 1e300);
    std::vector<int> bf(np, 0);
    for (int f : {0, 1, 2, 4, 8}) {
      for (Prob& pr : P->probs)
        if (pr.mixed) {
          pr.mx.split_pref = f;
          TRY(upload_mixed(pr));
        }
      P->prof = false;
      TRY(dmet_emb_eri(P, L, C, eri_out));
      reset_profile(P);
      P->prof = true;
      TRY(dmet_emb_eri(P, L, C, eri_out));
      CK(cudaStreamSynchronize(P->stream));
      double tc = 0;
      for (auto& e : P->ks[KC_TC_CONTRACT].ev) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        tc += ms;
      }
      for (int p = 0; p < np; ++p) {
        if (!P->probs[p].mixed) continue;
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, P->pev[p].first, P->pev[p].second));
        const double t = nmixed == 1 ? tc : ms;
        if (t < bs[p]) bs[p] = t, bf[p] = f;
      }
    }
    for (int p = 0; p < np; ++p)
      if (P->probs[p].mixed) P->probs[p].mx.split_pref = bf[p];
  }
  for (int p = 0; p < np; ++p) {
    Prob& pr = P->probs[p];
    if (!pr.mixed) continue;
    TRY(upload_mixed(pr));
    tune_cache_store(pr);
  }
  reset_profile(P);
  P->prof = prof;
  TRY(drop_graph(P));
  P->batch_mode = mode;
  return DMET_OK;
}

dmet_status_t dmet_emb_batch_mode(dmet_emb_plan_t P, int32_t mode, int32_t* active) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (mode != 0 && mode != 1) return fail(DMET_ERR_INVALID_ARG, "batch mode %d", mode);
  if (mode != P->batch_mode) {
    TRY(drop_graph(P));
    P->batch_mode = mode;
  }
  if (active) *active = grouped_active(P) ? 1 : 0;
  return DMET_OK;
}

dmet_status_t dmet_emb_split_parts(dmet_emb_plan_t P, int32_t problem, int32_t* parts) {
  clear_error();
  if (!P || !parts) return fail(DMET_ERR_INVALID_ARG, "NULL argument");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  const Prob& pr = P->probs[problem];
  for (int b = 0; b < 3; ++b) {
    parts[2 * b] = pr.mixed ? pr.mx.jc_split_n[b] : 0;
    parts[2 * b + 1] = pr.mixed ? pr.mx.jc_split_f[b] : 1;
  }
  return DMET_OK;
}

dmet_status_t dmet_emb_tile_widths(dmet_emb_plan_t P, int32_t problem, int32_t* bn) {
  clear_error();
  if (!P || !bn) return fail(DMET_ERR_INVALID_ARG, "NULL argument");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  bn[0] = P->probs[problem].mx.bn1;
  bn[1] = P->probs[problem].mx.bn2;
  return DMET_OK;
}

dmet_status_t dmet_emb_fock(dmet_emb_plan_t P, int32_t problem, const void* F, const void* C, const double* eri,
                            const double* gamma, double* fock_out) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  Prob& pr = P->probs[problem];
  if (pr.nspin != 1 || pr.d.sym != DMET_SYM_REAL || pr.pack != DMET_PACK_S8)
    return fail(DMET_ERR_UNSUPPORTED, "problem %d: the embedding Fock matrix needs n_spin = 1, real orbitals and "
                "the 8-fold packed ERI", problem);
  if (!F || !C || !eri || !gamma || !fock_out) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  if ((long long)pr.n[0] * (pr.n[0] + 1) / 2 + 2LL * pr.n[0] > 227LL * 1024 / 8)
    return fail(DMET_ERR_UNSUPPORTED, "problem %d: n_emb %d is above the 232 orbitals that dmet_emb_fock handles "
                "(one ERI pair row must fit in shared memory)", problem, pr.n[0]);
  const void* ptrs[5] = {F, C, eri, gamma, fock_out};
  for (const void* q : ptrs)
    if (!is_device_ptr(q)) return fail(DMET_ERR_INVALID_ARG, "dmet_emb_fock takes device pointers only");
  if (!aligned16(F) || !aligned16(C)) return fail(DMET_ERR_ALIGNMENT, "F or C not 16-byte aligned");
  if (((uintptr_t)eri | (uintptr_t)gamma | (uintptr_t)fock_out) & 7u)
    return fail(DMET_ERR_ALIGNMENT, "eri, gamma or fock_out not 8-byte aligned");
  const long long nk = pr.nk, nao = pr.nao, n = pr.n[0], npair = n * (n + 1) / 2;
  // scratch: W = F^k C^k [k][mu][j], G = C^k+ W [k][i][j], F0, J, K [n][n]
  const size_t bW = (size_t)(nk * nao * n) * 16, bG = (size_t)(nk * n * n) * 16, bM = (size_t)(n * n) * 8;
  const size_t need = bW + bG + 3 * bM + 256;
  P->cs = P->stream;
  TRY(ensure(&P->fock_ws, &P->fock_ws_b, need));
  char* w = (char*)P->fock_ws;
  double2* W = (double2*)w;
  double2* G = (double2*)(w + bW);
  double* F0 = (double*)(w + bW + bG);
  double* J = F0 + n * n;
  double* K = J + n * n;
  // flops executed: the two complex GEMMs; per pair row {i, k}: 2 n^2 exchange and n(n+1)/2 Coulomb
  // multiply-adds
  Timed t(P, KC_FOCK, 8.0 * nk * (nao * nao * n + nao * n * n) + 2.0 * npair * (2.0 * n * n + npair),
          16.0 * nk * (nao * nao + nao * n) + 8.0 * npair * (npair + 1) / 2 + 8.0 * n * n * 2, 5);
  {
    // W[k] = F^k C^k: opA(mu, nu) = conj(F[k][nu][mu]) = F[k][mu][nu] (F^k is Hermitian)
    ZgemmArgs z = zargs();
    z.A = (const double2*)F;
    z.B = (const double2*)C;
    z.D = W;
    z.M = (int)nao;
    z.N = (int)n;
    z.K = (int)nao;
    z.lda = nao;
    z.ldb = n;
    z.sA = nao * nao;
    z.sB = nao * n;
    z.sD = nao * n;
    z.dm_lo = n;
    z.dn_lo = 1;
    z.batch = (int)nk;
    CK(launch_zgemm(z, A_KM, true, B_KN, P->cs));
  }
  {
    // G[k] = C^k+ W[k]
    ZgemmArgs z = zargs();
    z.A = (const double2*)C;
    z.B = W;
    z.D = G;
    z.M = (int)n;
    z.N = (int)n;
    z.K = (int)nao;
    z.lda = n;
    z.ldb = n;
    z.sA = nao * n;
    z.sB = nao * n;
    z.sD = n * n;
    z.dm_lo = n;
    z.dn_lo = 1;
    z.batch = (int)nk;
    CK(launch_zgemm(z, A_KM, true, B_KN, P->cs));
  }
  CK(launch_fock_reduce(G, (int)nk, (int)n, pr.ortho_scale, F0, P->cs));
  CK(cudaMemsetAsync(K, 0, bM, P->cs));
  CK(launch_coulomb_exchange(eri, gamma, (int)n, J, K, P->cs));
  CK(launch_fock_combine(F0, J, K, (int)n, fock_out, P->cs));
  return DMET_OK;
}

dmet_status_t dmet_emb_bath(dmet_emb_plan_t P, int32_t problem, int32_t spin, const void* gamma_k, const void* C_lo,
                            const int32_t* val, int32_t n_val, void* C_out, double* info) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  Prob& pr = P->probs[problem];
  if (spin < 0 || spin >= pr.nspin) return fail(DMET_ERR_INVALID_ARG, "spin %d of a problem with %d", spin, pr.nspin);
  if (!gamma_k || !C_lo || !val || !C_out) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  const int nk = pr.nk, nlo = pr.nao;
  if (nk < 2) return fail(DMET_ERR_INVALID_ARG, "the bath needs an environment (Nk >= 2)");
  if (n_val < 1 || n_val > nlo || n_val > kMaxBathCols)
    return fail(DMET_ERR_INVALID_ARG, "n_val %d outside [1, min(n_ao %d, %d)]", n_val, nlo, kMaxBathCols);
  if (nlo + n_val != pr.n[spin])
    return fail(DMET_ERR_INVALID_ARG, "n_ao + n_val = %d, but the problem has n_emb = %d", nlo + n_val, pr.n[spin]);
  BathCols cols;
  cols.n = n_val;
  {
    std::vector<char> seen(nlo, 0);
    for (int c = 0; c < n_val; ++c) {
      if (val[c] < 0 || val[c] >= nlo) return fail(DMET_ERR_INVALID_ARG, "val[%d] = %d outside [0, %d)", c, val[c], nlo);
      if (seen[val[c]]) return fail(DMET_ERR_INVALID_ARG, "val[%d] = %d repeats an earlier column", c, val[c]);
      seen[val[c]] = 1;
      cols.v[c] = val[c];
    }
  }
  const void* ptrs[4] = {gamma_k, C_lo, C_out, info};
  for (const void* q : ptrs)
    if (q && !is_device_ptr(q)) return fail(DMET_ERR_INVALID_ARG, "dmet_emb_bath takes device pointers only");
  if (!aligned16(gamma_k) || !aligned16(C_lo) || !aligned16(C_out))
    return fail(DMET_ERR_ALIGNMENT, "gamma_k, C_lo or C_out not 16-byte aligned");
  if ((uintptr_t)info & 7u) return fail(DMET_ERR_ALIGNMENT, "info not 8-byte aligned");
  const long long m = (long long)(nk - 1) * nlo, nemb = nlo + n_val;
  // scratch: A (column-major block, rotated in place), B (bath orbitals [m][n_val]), Cb (Bloch sum
  // of the bath columns [k][i][b]), stats, the table of the Nk roots of unity
  const size_t bA = (size_t)(m * n_val) * 8, bC = (size_t)nk * nlo * n_val * 16;
  const size_t oB = (bA + 255) & ~(size_t)255, oC = oB + ((bA + 255) & ~(size_t)255), oS = oC + bC, oT = oS + 256;
  P->cs = P->stream;
  TRY(ensure(&P->bath_ws, &P->bath_ws_b, oT + (size_t)nk * 16));
  char* w = (char*)P->bath_ws;
  double* A = (double*)w;
  double* B = (double*)(w + oB);
  double2* Cb = (double2*)(w + oC);
  double* stats = (double*)(w + oS);
  double2* tw = (double2*)(w + oT);
  Timed t(P, KC_BATH, 8.0 * nk * m * n_val + 4.0 * nk * m * n_val + 8.0 * nk * nlo * nlo * n_val,
          16.0 * nk * nlo * n_val + 16.0 * nk * nlo * nlo + 16.0 * nk * nlo * nemb, 5);
  CK(cudaMemsetAsync(stats, 0, 64, P->cs));
  CK(launch_bath_twiddle(nk, tw, P->cs));
  CK(launch_bath_offdiag((const double2*)gamma_k, tw, pr.d.mesh, nlo, cols, A, stats, P->cs));
  CK(launch_bath_jacobi(A, (int)m, n_val, B, info, stats, P->cs));
  CK(launch_bath_bloch(B, (const double2*)C_lo, tw, pr.d.mesh, nlo, n_val, Cb, (double2*)C_out, P->cs));
  CK(launch_bath_product((const double2*)C_lo, Cb, nk, nlo, n_val, (double2*)C_out, P->cs));
  if (info) CK(cudaMemcpyAsync(info + n_val, stats, 5 * sizeof(double), cudaMemcpyDeviceToDevice, P->cs));
  return DMET_OK;
}

dmet_status_t dmet_emb_jk_df(dmet_emb_plan_t P, int32_t problem, int32_t spin, const void* Lq, const void* gamma,
                             void* J, void* K) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  Prob& pr = P->probs[problem];
  if (spin < 0 || spin >= pr.nspin) return fail(DMET_ERR_INVALID_ARG, "spin %d of a problem with %d", spin, pr.nspin);
  if (!Lq || !gamma || !J || !K) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  const void* ptrs[4] = {Lq, gamma, J, K};
  for (const void* q : ptrs) {
    if (!is_device_ptr(q)) return fail(DMET_ERR_INVALID_ARG, "dmet_emb_jk_df takes device pointers only");
    if (!aligned16(q)) return fail(DMET_ERR_ALIGNMENT, "a pointer is not 16-byte aligned");
  }
  const int nk = pr.nk, naux = pr.naux, n = pr.n[spin];
  const long long nn = (long long)n * n, nz_all = (long long)nk * naux;
  // batch entries z = (q, P) in chunks whose two n x n scratch matrices per entry stay within 1 GiB
  const long long per = 2 * nn * 16 + 16 + 2 * (long long)sizeof(int4);
  const int chunk = (int)std::max(1LL, std::min({nz_all, (1LL << 30) / per, 65535LL}));
  const size_t oW = 0, oKb = oW + (size_t)chunk * nn * 16, ov = oKb + (size_t)chunk * nn * 16,
               ot1 = ov + ((size_t)chunk * 16 + 255) / 256 * 256, ot2 = ot1 + (size_t)chunk * sizeof(int4),
               ot3 = ot2 + (size_t)chunk * sizeof(int4);
  P->cs = P->stream;
  TRY(ensure(&P->jk_ws, &P->jk_ws_b, ot3 + (size_t)chunk * sizeof(int4)));
  char* w = (char*)P->jk_ws;
  double2* W = (double2*)(w + oW);
  double2* Kb = (double2*)(w + oKb);
  double2* v = (double2*)(w + ov);
  int4* d1 = (int4*)(w + ot1);
  int4* d2 = (int4*)(w + ot2);
  int4* d3 = (int4*)(w + ot3);
  const double2* L = (const double2*)Lq;
  // 8 flops per complex multiply-add: two n^3 products and the two n^2 reductions per entry
  const int nchunks = (int)((nz_all + chunk - 1) / chunk);
  Timed t(P, KC_JK_DF, 8.0 * nz_all * (2.0 * nn * n + 2.0 * nn), 16.0 * nz_all * nn * 5, 4 * nchunks);
  CK(cudaMemsetAsync(J, 0, (size_t)nn * 16, P->cs));
  CK(cudaMemsetAsync(K, 0, (size_t)nn * 16, P->cs));
  // (the batched GEMMs are written transposed: the FP64 GEMM kernel takes A K-major)
  std::vector<int4> t1(chunk), t2(chunk), t3(chunk);
  for (long long z0 = 0; z0 < nz_all; z0 += chunk) {
    const int nz = (int)std::min<long long>(chunk, nz_all - z0);
    for (int i = 0; i < nz; ++i) {
      const long long z = z0 + i;
      const int q = (int)(z / naux), Pp = (int)(z % naux);
      const int mz = pr.s.neg[q] * naux + Pp;  // the -q factor of the same aux function
      t1[i] = make_int4(0, (int)z, i, n);       // W: A = gamma (shared), B = L^q_P, D = W[i]
      t2[i] = make_int4(mz, i, i, n);           // Kb: A = L^{-q}_P, B = W[i], D = Kb[i]
      t3[i] = make_int4((int)z, mz, i, n);      // trace and sums: L^q_P, L^{-q}_P
    }
    CK(cudaMemcpyAsync(d1, t1.data(), nz * sizeof(int4), cudaMemcpyHostToDevice, P->cs));
    CK(cudaMemcpyAsync(d2, t2.data(), nz * sizeof(int4), cudaMemcpyHostToDevice, P->cs));
    CK(cudaMemcpyAsync(d3, t3.data(), nz * sizeof(int4), cudaMemcpyHostToDevice, P->cs));
    {
      // W[i][a][b] = (L^q_P gamma)_ab, as W^T = gamma^T (L^q_P)^T: m = b, n = a, k = l;
      // opA(b, l) = gamma[l][b], opB(l, a) = L[a][l], stored at a n + b
      ZgemmArgs z = zargs();
      z.A = (const double2*)gamma;
      z.B = L;
      z.D = W;
      z.tab = d1;
      z.M = n;
      z.N = n;
      z.K = n;
      z.lda = n;
      z.ldb = n;
      z.sA = 0;
      z.sB = nn;
      z.sD = nn;
      z.dm_lo = 1;
      z.dn_lo = n;
      z.batch = nz;
      CK(launch_zgemm(z, A_KM, false, B_NK, P->cs));
    }
    {
      // Kb[i][a][b] = (W[i] L^{-q}_P)_ab, as Kb^T = (L^{-q}_P)^T W[i]^T: m = b, n = a, k = l;
      // opA(b, l) = L^{-q}[l][b], opB(l, a) = W[a][l], stored at a n + b
      ZgemmArgs z = zargs();
      z.A = L;
      z.B = W;
      z.D = Kb;
      z.tab = d2;
      z.M = n;
      z.N = n;
      z.K = n;
      z.lda = n;
      z.ldb = n;
      z.sA = nn;
      z.sB = nn;
      z.sD = nn;
      z.dm_lo = 1;
      z.dn_lo = n;
      z.batch = nz;
      CK(launch_zgemm(z, A_KM, false, B_NK, P->cs));
    }
    CK(launch_jk_trace(L, d3, nz, n, (const double2*)gamma, v, P->cs));
    CK(launch_jk_accumulate(L, d3, v, Kb, nz, n, 1.0 / nk, (double2*)J, (double2*)K, P->cs));
  }
  return DMET_OK;
}

// out[o][k][x] = sum_j F[k][j] in[o][j][x] for o < outer (a dense DFT along one grid axis of length g,
// as one batched complex GEMM with m = x, n = k, k = j: opA(x, j) = in[o][j][x] (K-major),
// opB(j, k) = F[k][j], stored at out[o][k][x]).
static dmet_status_t dft_axis(dmet_emb_plan_s* P, const double2* F, int g, long long outer, long long inner,
                              const double2* in, double2* out) {
  if (fftdf_small_axis(g)) {
    // a short axis: one thread per column (the GEMM form would use a g-wide sliver of each tile)
    CK(launch_dft_axis_small(F, g, outer, inner, in, out, P->cs));
    return DMET_OK;
  }
  if (inner > INT_MAX || outer > 65535) return fail(DMET_ERR_UNSUPPORTED, "FFTDF grid too large for one DFT launch");
  ZgemmArgs z = zargs();
  z.A = in;
  z.B = F;
  z.D = out;
  z.M = (int)inner;
  z.N = g;
  z.K = g;
  z.lda = inner;
  z.ldb = g;
  z.sA = (long long)g * inner;
  z.sB = 0;
  z.sD = (long long)g * inner;
  z.dm_lo = 1;
  z.dn_lo = inner;
  z.batch = (int)outer;
  CK(launch_zgemm(z, A_KM, false, B_NK, P->cs));
  return DMET_OK;
}

dmet_status_t dmet_emb_eri_fftdf(dmet_emb_plan_t P, int32_t problem, const void* rho, const void* const* C,
                                 const int32_t* grid, const double* lattice, void* const* eri_out) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  Prob& pr = P->probs[problem];
  if (!rho || !C || !grid || !lattice || !eri_out) return fail(DMET_ERR_INVALID_ARG, "NULL pointer argument");
  if (pr.mixed || pr.pack != DMET_PACK_FULL || pr.d.l_layout != DMET_L_FULL)
    return fail(DMET_ERR_UNSUPPORTED, "problem %d: the FFTDF ERI needs prec = FP64, FULL packing and the full layout",
                problem);
  long long ng = 1;
  for (int d = 0; d < 3; ++d) {
    if (grid[d] < 1 || grid[d] > 4096) return fail(DMET_ERR_INVALID_ARG, "grid[%d] = %d", d, grid[d]);
    ng *= grid[d];
  }
  if (ng != pr.naux)
    return fail(DMET_ERR_INVALID_ARG, "problem %d: n_aux = %d must be the grid's %lld points", problem, pr.naux, ng);
  const int nblk = pr.nspin == 1 ? 1 : 3;
  std::vector<const void*> ptrs = {rho};
  for (int s = 0; s < pr.nspin; ++s) ptrs.push_back(C[s]);
  for (int b = 0; b < nblk; ++b) ptrs.push_back(eri_out[b]);
  for (const void* q : ptrs) {
    if (!q || !is_device_ptr(q)) return fail(DMET_ERR_INVALID_ARG, "dmet_emb_eri_fftdf takes device pointers only");
    if (!aligned16(q)) return fail(DMET_ERR_ALIGNMENT, "a pointer is not 16-byte aligned");
  }
  const int nk = pr.nk;
  const int nmax = std::max(pr.n[0], pr.nspin == 2 ? pr.n[1] : 0);
  const long long nx_max = (long long)nmax * nmax;
  // host tables: DFT matrices per axis (forward, then inverse = conjugate), the Coulomb kernel per q
  std::vector<double2> F;
  size_t f_off[3][2];
  for (int d = 0; d < 3; ++d)
    for (int inv = 0; inv < 2; ++inv) {
      f_off[d][inv] = F.size();
      const int g = grid[d];
      for (int k = 0; k < g; ++k)
        for (int j = 0; j < g; ++j) {
          const double a = 2.0 * M_PI * (double)((long long)j * k % g) / g;
          F.push_back(make_double2(std::cos(a), inv ? std::sin(a) : -std::sin(a)));
        }
    }
  std::vector<double> vq((size_t)nk * ng);
  for (int q = 0; q < nk; ++q)
    TRY(dmet_fftdf_plane_waves(pr.d.mesh, q, grid, lattice, nullptr, vq.data() + (size_t)q * ng, nullptr));
  const double a0[3] = {lattice[0], lattice[1], lattice[2]}, a1[3] = {lattice[3], lattice[4], lattice[5]},
               a2[3] = {lattice[6], lattice[7], lattice[8]};
  const double omega = std::fabs(a0[0] * (a1[1] * a2[2] - a1[2] * a2[1]) - a0[1] * (a1[0] * a2[2] - a1[2] * a2[0]) +
                                 a0[2] * (a1[0] * a2[1] - a1[1] * a2[0]));
  // The q values run in chunks of qc at once. Reindexed by q' = -q, step 4 reads
  //   (ij|kl) += Omega / (N_g^2 Nk) sum_q' sum_r w^{-q'}(r)_ij (r|0k 0l)^{q'},
  // so a chunk of consecutive q' pairs the transformed factors of q = -q' (computed in that order)
  // with a contiguous run of the untransformed ones: one GEMM over K = qc N_g per chunk and spin pair.
  const long long g0 = grid[0], g1 = grid[1], g2 = grid[2];
  int qc = nk;
  while (qc > 1 && ((size_t)qc * ng * nx_max * 16 * 2 > ((size_t)4 << 30) || (long long)qc * g0 * g1 > 65535 ||
                    (long long)qc * ng > INT_MAX))
    qc = (qc + 1) / 2;
  if ((long long)qc * g0 * g1 > 65535 || (long long)qc * ng > INT_MAX)
    return fail(DMET_ERR_UNSUPPORTED, "FFTDF grid too large for one DFT launch");
  std::vector<double> vp((size_t)nk * ng);  // kernels in q' order: v^{-q'}
  std::vector<int> qtab(nk);                // q' -> q = -q'
  for (int qq = 0; qq < nk; ++qq) {
    qtab[qq] = pr.s.neg[qq];
    std::memcpy(vp.data() + (size_t)qq * ng, vq.data() + (size_t)qtab[qq] * ng, sizeof(double) * ng);
  }
  // The contraction GEMM of a chunk is n^2 x n^2 with K = qc N_g: few output tiles over a long K, so
  // it is split in K into kparts batches (partial blocks, summed afterwards) that fill the GPU.
  const long long ktot = (long long)qc * ng, tiles_min = ((nx_max + 63) / 64) * ((nx_max + 63) / 64);
  int kparts = 1;
  while (kparts < 64 && tiles_min * kparts < 2 * 152 && ktot % (2 * kparts) == 0 && ktot / (2 * kparts) >= 64 &&
         (size_t)(2 * kparts) * nx_max * nx_max * 16 <= ((size_t)1 << 30))
    kparts *= 2;
  // scratch: two [qc][grid][n^2] buffers, the DFT matrices, the kernels, the q table, the K parts
  const size_t bbuf = (size_t)qc * ng * nx_max * 16, oF = 2 * bbuf, oV = oF + (F.size() * 16 + 255) / 256 * 256;
  const size_t oQ = oV + (vp.size() * 8 + 255) / 256 * 256;
  const size_t oP = oQ + (qtab.size() * sizeof(int) + 255) / 256 * 256;
  P->cs = P->stream;
  TRY(ensure(&P->fft_ws, &P->fft_ws_b, oP + (kparts > 1 ? (size_t)kparts * nx_max * nx_max * 16 : 0)));
  char* w = (char*)P->fft_ws;
  double2* buf0 = (double2*)w;
  double2* buf1 = (double2*)(w + bbuf);
  double2* dF = (double2*)(w + oF);
  double* dV = (double*)(w + oV);
  int* dQ = (int*)(w + oQ);
  double2* dPart = (double2*)(w + oP);
  CK(cudaMemcpyAsync(dF, F.data(), F.size() * 16, cudaMemcpyHostToDevice, P->cs));
  CK(cudaMemcpyAsync(dV, vp.data(), vp.size() * 8, cudaMemcpyHostToDevice, P->cs));
  CK(cudaMemcpyAsync(dQ, qtab.data(), qtab.size() * sizeof(int), cudaMemcpyHostToDevice, P->cs));
  // Step 1 of Algorithm 2 for every q and spin: (r|0i 0j) = s sum_k1 C^{k1+} rho^{k1,k1+q}(r) C^{k1+q}
  const double2* Cd[2] = {(const double2*)C[0], pr.nspin == 2 ? (const double2*)C[1] : nullptr};
  P->W = &P->ws[P->ws_of[problem]];
  CK(cudaMemsetAsync(P->dstats + 8 * problem, 0, 8 * sizeof(double), P->cs));
  TRY(run_orbital_checks(P, pr, problem, Cd));
  double2* lq[2] = {P->W->lq_all[0], P->W->lq_all[1]};
  TRY(transform_range(P, pr, (const double2*)rho, Cd, 0, nk, lq, pr.bq));
  for (int b = 0; b < nblk; ++b) CK(cudaMemsetAsync(eri_out[b], 0, eri_bytes_of(pr.d, b), P->cs));
  for (int sa = 0; sa < pr.nspin; ++sa) {
    const long long nx = (long long)pr.n[sa] * pr.n[sa];
    for (int c0 = 0; c0 < nk; c0 += qc) {
      const int nc = std::min(qc, nk - c0);
      {
        Timed t(P, KC_FFTDF, 8.0 * ng * nx * 2.0 * (g0 + g1 + g2) * nc, 16.0 * ng * nx * 14 * nc, 9);
        // 2. exp(-i q.r), forward DFT, 4 pi / |q + G|^2, inverse DFT, exp(+i q.r), for q = -q', q' in the chunk
        CK(launch_fftdf_phase_q(lq[sa], buf0, dQ + c0, nc, 1, grid, pr.d.mesh, -1.0, 1.0, nx, P->cs));
        TRY(dft_axis(P, dF + f_off[0][0], (int)g0, nc, g1 * g2 * nx, buf0, buf1));
        TRY(dft_axis(P, dF + f_off[1][0], (int)g1, nc * g0, g2 * nx, buf1, buf0));
        TRY(dft_axis(P, dF + f_off[2][0], (int)g2, nc * g0 * g1, nx, buf0, buf1));
        CK(launch_fftdf_kernel_mul(buf1, dV + (size_t)c0 * ng, (long long)nc * ng, nx, P->cs));
        TRY(dft_axis(P, dF + f_off[0][1], (int)g0, nc, g1 * g2 * nx, buf1, buf0));
        TRY(dft_axis(P, dF + f_off[1][1], (int)g1, nc * g0, g2 * nx, buf0, buf1));
        TRY(dft_axis(P, dF + f_off[2][1], (int)g2, nc * g0 * g1, nx, buf1, buf0));
        CK(launch_fftdf_phase_q(buf0, buf1, dQ + c0, nc, 0, grid, pr.d.mesh, 1.0, 1.0, nx, P->cs));
      }
      // 4. (ij|kl) += Omega / (N_g^2 Nk) sum_{q', r} w^{-q'}(r)_ij (r|0k 0l)^{q'} (one 1/N_g is the
      // unnormalised DFTs'), K = nc N_g
      for (int sb = sa; sb < pr.nspin; ++sb) {
        const long long nxb = (long long)pr.n[sb] * pr.n[sb];
        const int blk = pr.nspin == 1 ? 0 : (sa == 0 ? (sb == 0 ? 0 : 1) : 2);
        const long long kc = (long long)nc * ng;
        const int kp = (kparts > 1 && kc % kparts == 0) ? kparts : 1;
        ZgemmArgs z = zargs();
        z.A = buf1;
        z.B = lq[sb] + (long long)c0 * ng * nxb;
        z.D = kp > 1 ? dPart : (double2*)eri_out[blk];
        z.M = (int)nx;
        z.N = (int)nxb;
        z.K = (int)(kc / kp);
        z.lda = nx;
        z.ldb = nxb;
        z.dm_lo = nxb;
        z.dn_lo = 1;
        z.alpha = omega / ((double)ng * ng * nk);
        z.beta = kp > 1 ? 0 : 1;
        z.sA = (kc / kp) * nx;  // part p: K rows [p kc/kp, (p+1) kc/kp) of both operands
        z.sB = (kc / kp) * nxb;
        z.sD = nx * nxb;
        z.batch = kp;
        Timed tc(P, KC_FFTDF, 8.0 * (double)nx * nxb * ng * nc, kp > 1 ? 16.0 * kp * nx * nxb * 2 : 0.0,
                 kp > 1 ? 2 : 1);
        CK(launch_zgemm(z, A_KM, false, B_KN, P->cs));
        if (kp > 1) CK(launch_sum_parts(dPart, kp, nx * nxb, (double2*)eri_out[blk], P->cs));
      }
    }
  }
  CK(cudaGetLastError());
  return DMET_OK;
}

dmet_status_t dmet_emb_status(dmet_emb_plan_t P, int32_t problem, double* stats) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (problem < 0 || problem >= (int)P->probs.size()) return fail(DMET_ERR_INVALID_ARG, "problem %d", problem);
  CK(cudaStreamSynchronize(P->stream));
  double h[8];
  CK(cudaMemcpy(h, P->dstats + 8 * problem, sizeof(h), cudaMemcpyDeviceToHost));
  const Prob& pr = P->probs[problem];
  const bool real = pr.d.sym == DMET_SYM_REAL;
  const double rc = real ? h[1] / std::max(h[2], 1e-300) : -1.0;
  const bool lchk = real && pr.d.check_l;
  const double herm = lchk ? h[3] / std::max(h[5], 1e-300) : -1.0;
  const double tr = lchk ? h[4] / std::max(h[5], 1e-300) : -1.0;
  if (stats) {
    stats[0] = h[0];
    stats[1] = rc;
    stats[2] = herm;
    stats[3] = tr;
  }
  unsigned int werr = 0;
  if (P->derr) CK(cudaMemcpy(&werr, P->derr, sizeof(werr), cudaMemcpyDeviceToHost));
  if (werr) {
    // reported once: the word is cleared for the plan's later calls
    CK(cudaMemset(P->derr, 0, sizeof(unsigned int)));
    return fail(DMET_ERR_TIMEOUT, "a bounded device wait expired (flags 0x%x: 1 stage free, 2 accumulator free, "
                "4 stage loaded, 8 accumulator ready, 16 MMAs done, 32 copies landed)", werr);
  }
  if (!(h[0] <= pr.d.ortho_tol))
    return fail(DMET_ERR_NOT_ORTHONORMAL, "problem %d: orthonormality error %.3e > %.3e", problem, h[0], pr.d.ortho_tol);
  if (real && !(rc <= pr.d.sym_tol))
    return fail(DMET_ERR_SYMMETRY, "problem %d: C^-k != conj C^k (relative %.3e)", problem, rc);
  if (lchk && !(herm <= pr.d.sym_tol && tr <= pr.d.sym_tol))
    return fail(DMET_ERR_SYMMETRY, "problem %d: L symmetry violated (hermiticity %.3e, time reversal %.3e)", problem,
                herm, tr);
  return DMET_OK;
}

dmet_status_t dmet_emb_wait_limit(dmet_emb_plan_t P, uint64_t wait_ns, int32_t test_withhold_loads) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  P->wait_ns = wait_ns ? (unsigned long long)wait_ns : tc::kWaitLimitNs;
  P->withhold_loads = test_withhold_loads != 0;
  if (P->gexec) {
    // a captured graph holds the old launch parameters
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaGraphExecDestroy(P->gexec));
    P->gexec = nullptr;
    P->gkey.clear();
  }
  return DMET_OK;
}

dmet_status_t dmet_emb_profile(dmet_emb_plan_t P, int32_t enable) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  CK(cudaStreamSynchronize(P->stream));
  reset_profile(P);
  P->prof = enable != 0;
  return DMET_OK;
}

dmet_status_t dmet_emb_profile_read(dmet_emb_plan_t P, int32_t kernel, const char** name, int64_t* launches,
                                    double* total_ms, double* flops, double* exec_flops, double* bytes) {
  clear_error();
  if (!P) return fail(DMET_ERR_INVALID_ARG, "plan is NULL");
  if (kernel < 0 || kernel >= KC_COUNT) return fail(DMET_ERR_INVALID_ARG, "kernel %d", kernel);
  CK(cudaStreamSynchronize(P->stream));
  KStat& k = P->ks[kernel];
  double ms = 0;
  for (auto& e : k.ev) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, e.first, e.second));
    ms += t;
  }
  if (name) *name = kKcNames[kernel];
  if (launches) *launches = k.launches;
  if (total_ms) *total_ms = ms;
  if (flops) *flops = k.flops;
  if (exec_flops) *exec_flops = k.exec;
  if (bytes) *bytes = k.bytes;
  return DMET_OK;
}

int64_t dmet_emb_launch_count(dmet_emb_plan_t P) { return P ? P->launches : 0; }

}  // extern "C"
