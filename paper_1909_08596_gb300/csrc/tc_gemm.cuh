// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA).
//
//   result(m, n) = sum_g w_g * sum_{k in segment g} A(a_row0 + m, k) B(b_row0 + n, k)
//
// A and B are given as NSLICE bf16 slices, A = A_0 + A_1 + A_2 (K-major, [slice][row][K]).
// With three slices every product A_s B_t with s + t <= 2 is issued (6 products; the
// dropped terms are ~2^-24 relative). The leading product A_0 B_0 accumulates into its own
// FP32 TMEM accumulator and the five smaller ones into a second: the tensor cores add each
// MMA's result into the accumulator with an error of the accumulator's own magnitude, so
// mixing the small correction terms into the leading sum would multiply the number of lossy
// additions it suffers by six. That error still grows with the number of MMAs a segment
// accumulates, so the leading sum runs over short segments (a few K blocks); the epilogue
// warps add each segment's result, times its exact power-of-two weight w_g, into an
// unevaluated sum of two FP32 numbers (hi + lo, updated with the error-free TwoSum), which
// carries ~44 bits across segments at FP32-pipe cost, and hand hi + lo to the output
// functor once at the end. The correction sum is ~2^-8 of the leading one, so its own
// rounding error stays ~2^-8 below the leading sum's even over a whole job: it accumulates
// over a run of segments of equal weight (a job's segments, split where the weight
// changes) and is read once per run, which halves the accumulator traffic per segment.
//
// A persistent CTA of 12 warps (one per SM) works through the jobs blockIdx.x, blockIdx.x +
// gridDim.x, ...; each job is one 128 x BN output tile (jobs come from a table). The stage
// ring and the two accumulator buffers run on across jobs, so a job's final store overlaps
// the next job's MMAs.
//   warp 0      TMA producer (one thread): 3+3 slice tiles per K block into a stage ring;
//   warp 1      MMA issuer (one thread), also allocates / frees all 512 TMEM columns:
//               two leading-sum buffers (segment parity), so the epilogue of segment g
//               overlaps the MMAs of segment g+1, and two correction buffers (run parity);
//   warps 2, 3  idle (they complete the first warpgroup);
//   warps 4..11 epilogue: warp w reads TMEM lanes 32*(w%4).. and half (w-4)/4 of the BN columns;
//               most output functors store through a per-warp shared-memory transpose, so
//               that each store instruction writes whole row segments instead of 32 rows.
// Registers: the CTA launches with kLaunchRegs per thread; the first warpgroup gives most of
// its registers back (setmaxnreg.dec to kCtrlRegs) and the epilogue warpgroups take them
// (setmaxnreg.inc to kEpiRegs), which the two-float sums of up to 64 columns per thread need:
// 128 * kCtrlRegs + 128 * kEpiGroups * kEpiRegs <= kThreads * kLaunchRegs, and per SM
// sub-partition (one warp of each warpgroup) kCtrlRegs + kEpiGroups * kEpiRegs <= 512.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "prec.cuh"
#include "split.cuh"
#include "tc_common.cuh"

namespace dmet {
namespace tc {

struct Segment {
  int k0;     // first K element (a multiple of 32, so of every precision's K block)
  int nk;     // number of K elements (a multiple of 32)
  float w;    // weight of this segment (a power of two, so the scaling is exact)
  int flags;  // kRunFirst / kRunLast: bounds of a correction-sum run inside a job
};
// A job's first and last segments always bound a run; these flags add bounds inside a job.
// Every segment of a run must carry the same weight.
constexpr int kRunFirst = 1;
constexpr int kRunLast = 2;

// One output tile: rows [a_row0, a_row0 + 128) of A against rows [b_row0, b_row0 + 128) of B,
// of which m_valid x n_valid are stored; segments [seg0, seg0 + nseg). A job may also be one
// K part of a tile (the output functor then stores the unscaled two-float partial sum).
struct TcJob {
  int a_row0, b_row0;
  int m_valid, n_valid;
  int seg0, nseg;
  int o0, o1, o2, o3;  // output-functor parameters (tile origin in the output's own indexing)
  int grp;             // grouped launches: the job's entry of the group table (0 otherwise)
};

// One entry of a grouped launch's table (one problem, or one block of a problem): its operand
// tensor maps, segment list, output-functor parameters and result factor. The table lives in
// global memory, written by a host copy before the launch; the producer thread acquires each map
// for the tensor-map proxy (fence.proxy.tensormap, system scope, since a host copy wrote it)
// before its first copy through it.
template <class EPI>
struct alignas(128) TcGroup {
  CUtensorMap a, b;
  const Segment* segs;
  const float* fac;
  typename EPI::Params ep;
};

// Run-time controls of one launch.
struct TcCtl {
  unsigned int* err;           // error word: one bit per kind of bounded wait that expired
  unsigned long long wait_ns;  // limit of every bounded wait
  int withhold_loads;          // test hook: the producer issues no copies, so the MMA thread's and
                               // the epilogue's waits expire with no copy or MMA in flight
  unsigned int* jobsync;       // job pacing (or null): a counter, zero at launch, of the jobs whose
                               // loads the CTAs have issued. Before its (k+1)-th job a CTA's producer
                               // waits until every CTA has issued its k-th job's loads, so the CTAs
                               // work on neighbouring tiles at neighbouring K and share their operand
                               // blocks in L2 instead of drifting apart over a long job. A pacing wait
                               // that takes longer than kJobSyncLimitNs (CTAs that are not all
                               // resident) ends the pacing for the rest of the launch; it is a
                               // scheduling aid only and never changes a result.
};

constexpr int kTile = 128;
constexpr int kEpiGroups = 2;                    // epilogue warpgroups
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kThreads = 128 * (1 + kEpiGroups);
constexpr int kTmemCols = 512;
constexpr int kLaunchRegs = 168;  // 65536 / 384, in the 8-register allocation unit
constexpr int kCtrlRegs = 56;
constexpr int kEpiRegs = 224;
static_assert(kLaunchRegs * kThreads <= 65536, "register file");
static_assert(128 * kCtrlRegs + 128 * kEpiGroups * kEpiRegs <= kThreads * kLaunchRegs,
              "the register split must fit in what the CTA launches with");
static_assert(kCtrlRegs + kEpiGroups * kEpiRegs <= 512, "per sub-partition register file");

// PREC: the operand precision (prec.cuh). BN: output columns per tile (the UMMA N), 128, 112 or
// 96. Each of the four accumulators (two buffers of leading + correction sums) starts on a
// 128-column boundary of TMEM. STAGED: the output functor stores through the shared-memory
// transpose. The stage ring takes what the 227 KB of shared memory leave (4 to 8 stages).
// Operand rows are 64 bytes per K block (64-byte swizzle).
template <class PREC, int BN, bool STAGED>
struct TcCfg {
  static_assert(BN % 32 == 16 || BN % 32 == 0, "BN must be a multiple of 16");
  static_assert(BN <= 128 && BN >= 64, "4 BN TMEM columns must fit");
  static constexpr int ROWB = 64;
  static constexpr int NSLICE = PREC::kSlices;
  static constexpr int BK = kblock_elems<PREC>();               // elements per K block
  static constexpr int A_BYTES = kTile * ROWB;                  // one A slice tile
  static constexpr int B_BYTES = BN * ROWB;                     // one B slice tile
  static constexpr int STAGE_BYTES = NSLICE * (A_BYTES + B_BYTES);
  static constexpr int NPROD = PREC::kProducts;
  static constexpr int STAGING = STAGED ? kEpiWarps * 32 * 8 * 8 : 0;  // epilogue transpose: 32 x 8 words per warp
  static constexpr int RING = 232448 - 1024 - 256 - STAGING;    // 227 KB less alignment, barriers, staging
  static constexpr int STAGES = RING / STAGE_BYTES > 8 ? 8 : RING / STAGE_BYTES;
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + 256 + STAGING;
  static_assert(STAGES >= 2 && SMEM <= 232448, "shared memory");
  static constexpr int PART = BN / kEpiGroups;                  // columns per epilogue warp
  static_assert(PART % 4 == 0, "epilogue column share");
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bv = s - hi;
  const float e = (hi - (s - bv)) + (x - bv);
  hi = s;
  lo += e;
}

// Two columns at once on the paired FP32 pipe (add/sub.rn.f32x2): (hi, lo) += v with the same
// TwoSum, each lane rounded as the scalar form.
__device__ __forceinline__ void two_sum_acc2(float& h0, float& h1, float& l0, float& l1, uint32_t v0, uint32_t v1) {
  asm("{\n\t.reg .b64 h, l, x, s, bv, t;\n\t"
      "mov.b64 h, {%0, %1};\n\t"
      "mov.b64 l, {%2, %3};\n\t"
      "mov.b64 x, {%4, %5};\n\t"
      "add.rn.f32x2 s, h, x;\n\t"
      "sub.rn.f32x2 bv, s, h;\n\t"
      "sub.rn.f32x2 t, s, bv;\n\t"
      "sub.rn.f32x2 t, h, t;\n\t"
      "sub.rn.f32x2 bv, x, bv;\n\t"
      "add.rn.f32x2 t, t, bv;\n\t"
      "add.rn.f32x2 l, l, t;\n\t"
      "mov.b64 {%0, %1}, s;\n\t"
      "mov.b64 {%2, %3}, l;\n\t}"
      : "+f"(h0), "+f"(h1), "+f"(l0), "+f"(l1)
      : "r"(v0), "r"(v1));
}

// (l0, l1) += (v0, v1) on the paired pipe.
__device__ __forceinline__ void add_acc2(float& l0, float& l1, uint32_t v0, uint32_t v1) {
  asm("{\n\t.reg .b64 l, x;\n\t"
      "mov.b64 l, {%0, %1};\n\t"
      "mov.b64 x, {%2, %3};\n\t"
      "add.rn.f32x2 l, l, x;\n\t"
      "mov.b64 {%0, %1}, l;\n\t}"
      : "+f"(l0), "+f"(l1)
      : "r"(v0), "r"(v1));
}

// Stores a warp's 32 rows x H columns through a 32 x 8 transpose in shared memory (element
// (r, c) at r * 8 + (c ^ (r & 7)), a swizzle that keeps both phases at two to four
// wavefronts): each store instruction then covers 4 rows x 8 consecutive columns.
template <int H, class EPI>
__device__ __forceinline__ void staged_store(const typename EPI::Params& ep, const TcJob& job, int row0, int col0,
                                             const float* hi, const float* lo, unsigned long long* stg, int lane) {
  static_assert(H % 4 == 0, "column share");
#pragma unroll
  for (int c0 = 0; c0 < H; c0 += 8) {
    if (c0 + 8 > H) {
      // 4-column tail: the block is 32 x 4, each store instruction covers 8 rows x 4 columns.
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const unsigned long long v = EPI::value(ep, job, hi[c0 + c], lo[c0 + c]);
        uint32_t* w = reinterpret_cast<uint32_t*>(stg + lane * 8 + (c ^ (lane & 7)));
        w[0] = (uint32_t)v;
        w[1] = (uint32_t)(v >> 32);
      }
      __syncwarp();
      int ln;
      asm volatile("mov.b32 %0, %1;" : "=r"(ln) : "r"(lane));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = i * 8 + (ln >> 2), c = ln & 3;
        EPI::put(ep, job, row0 + r, col0 + c0 + c, stg[r * 8 + (c ^ (r & 7))]);
      }
      __syncwarp();
      break;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      // two 32-bit halves: no aligned register pair is needed for the 64-bit value
      const unsigned long long v = EPI::value(ep, job, hi[c0 + c], lo[c0 + c]);
      uint32_t* w = reinterpret_cast<uint32_t*>(stg + lane * 8 + (c ^ (lane & 7)));
      w[0] = (uint32_t)v;
      w[1] = (uint32_t)(v >> 32);
    }
    __syncwarp();
    // (An opaque copy of the lane index keeps the compiler from hoisting the eight row
    // addresses of every 8-column block out of the loop, which would spill.)
    int ln;
    asm volatile("mov.b32 %0, %1;" : "=r"(ln) : "r"(lane));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = i * 4 + (ln >> 3), c = ln & 7;
      EPI::put(ep, job, row0 + r, col0 + c0 + c, stg[r * 8 + (c ^ (r & 7))]);
    }
    __syncwarp();
  }
}

// Output functors whose parameters hold indirections (an output pointer kept in a device slot that
// each call rewrites) resolve them once per job of a grouped launch: EPI::resolve(params).
template <class E>
__device__ __forceinline__ auto epi_resolve(typename E::Params& p, int) -> decltype(E::resolve(p)) {
  E::resolve(p);
}
template <class E>
__device__ __forceinline__ void epi_resolve(typename E::Params&, long) {}

// Output functors either store per thread, EPI::store<H>(params, job, row, col0, hi, lo) with
// row = tile-local row (< 128) and columns col0 .. col0+H-1, or (kStaged) give the 8-byte
// value of an element, EPI::value(params, job, hi, lo), and write it, EPI::put(params, job, row,
// col, v), skipping elements outside the job's valid region.
// fac (device, or null for 1): a power of two that multiplies every result before the output functor
// sees it (it undoes the operand scaling of the FP16 precision).
// groups (device, or null): a grouped launch, in which every job names its entry of this table and
// takes the maps, segments, output parameters and factor from there instead of tmA, tmB, segs, ep
// and fac. One persistent launch then works through the tiles of many problems of one shape class.
template <class PREC, int BN, class EPI>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcJob* __restrict__ jobs, int njobs, const Segment* __restrict__ segs,
                   const typename EPI::Params ep, const TcCtl ctl, const float* __restrict__ fac,
                   const TcGroup<EPI>* __restrict__ groups) {
  using Cfg = TcCfg<PREC, BN, EPI::kStaged>;
  constexpr int NSLICE = Cfg::NSLICE;
  constexpr int ROWB = Cfg::ROWB;
  constexpr int S = Cfg::STAGES;
  constexpr int H = Cfg::PART;
  constexpr int kChunk = 32;  // TMEM columns per load round trip
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* bars = (uint64_t*)(smem + S * Cfg::STAGE_BYTES);
  // bars: full[S], empty[S], accf[2], acce[2], done; then the TMEM address and a counter.
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * S + 5);
  volatile int* consumed = (volatile int*)(bars + 2 * S + 5) + 1;
  unsigned long long* staging = (unsigned long long*)(smem + S * Cfg::STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned int* const err = ctl.err;
  const unsigned long long lim = ctl.wait_ns;

  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + S + s); };
  auto accf = [&](int b) { return smem_u32(bars + 2 * S + b); };
  auto acce = [&](int b) { return smem_u32(bars + 2 * S + 2 + b); };
  const uint32_t done_bar = smem_u32(bars + 2 * S + 4);
  auto a_tile = [&](int s, int t) { return smem_u32(tiles + s * Cfg::STAGE_BYTES + t * Cfg::A_BYTES); };
  auto b_tile = [&](int s, int t) {
    return smem_u32(tiles + s * Cfg::STAGE_BYTES + NSLICE * Cfg::A_BYTES + t * Cfg::B_BYTES);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), kEpiWarps);
    }
    mbar_init(done_bar, 1);
    *consumed = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(bars + 2 * S + 5), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kCtrlRegs));
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      const void* ma = &tmA;
      const void* mb = &tmB;
      const Segment* sgs = segs;
      if (!groups) {
        prefetch_tmap(ma);
        prefetch_tmap(mb);
      }
      int cur = -1;
      bool ok = !ctl.withhold_loads;
      bool pace = ctl.jobsync != nullptr;
      unsigned int kjob = 0;  // jobs of this CTA whose loads are issued
      for (int jb = blockIdx.x; jb < njobs && ok; jb += gridDim.x, ++kjob) {
      if (pace && kjob > 0) pace = counter_wait(ctl.jobsync, kjob * gridDim.x, kJobSyncLimitNs);
      const TcJob job = jobs[jb];
      if (groups && job.grp != cur) {
        cur = job.grp;
        ma = &groups[cur].a;
        mb = &groups[cur].b;
        sgs = groups[cur].segs;
        tmap_acquire(ma);
        tmap_acquire(mb);
      }
      for (int g = 0; g < job.nseg && ok; ++g) {
        const Segment sg = sgs[job.seg0 + g];
        const int nkb = sg.nk / Cfg::BK;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = issued % S, ph = (issued / S) & 1;
          if (!mbar_wait(empty(s), ph ^ 1, err, 1u, lim)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full(s), Cfg::STAGE_BYTES);
          const int k = sg.k0 + kb * Cfg::BK;
#pragma unroll
          for (int t = 0; t < NSLICE; ++t) {
            // A operands stored slice-interleaved ([row][K / 32][slice][32]) come through a 4D map
            if constexpr (EPI::kAInterleaved)
              tma_load_4d(a_tile(s, t), ma, full(s), 0, t, k / Cfg::BK, job.a_row0);
            else
              tma_load_3d(a_tile(s, t), ma, full(s), k, job.a_row0, t);
            tma_load_3d(b_tile(s, t), mb, full(s), k, job.b_row0, t);
          }
          ++issued;
        }
      }
      if (ctl.jobsync && ok) atomicAdd(ctl.jobsync, 1u);
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = idesc_f32acc(PREC::kFormat, kTile, BN);
      int it = 0, gs = 0, run = -1;  // K blocks, segments and correction runs so far (across jobs)
      bool ok = true;
      for (int jb = blockIdx.x; jb < njobs && ok; jb += gridDim.x) {
      const TcJob job = jobs[jb];
      const Segment* sgs = groups ? groups[job.grp].segs : segs;
      for (int g = 0; g < job.nseg && ok; ++g, ++gs) {
        const int b = gs & 1, u = gs >> 1;
        // The buffer of segment gs - 2 is free once the epilogue has read it; the epilogue
        // reads a run's correction sum before it releases the run's last segment, so this
        // also frees the correction buffer of run `run - 1` (every run has >= 1 segment).
        if (!mbar_wait(acce(b), (u & 1) ^ 1, err, 2u, lim)) break;
        tc_fence_after();
        const Segment sg = sgs[job.seg0 + g];
        const bool first = g == 0 || (sg.flags & kRunFirst);
        run += first;
        // 128-column aligned: leading sums at 0 / 128, correction sums at 256 / 384
        const uint32_t d_main = tmem + b * kTile, d_corr = tmem + (2 + (run & 1)) * kTile;
        const int nkb = sg.nk / Cfg::BK;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % S, ph = (it / S) & 1;
          if (!mbar_wait(full(s), ph, err, 4u, lim)) {
            ok = false;
            break;
          }
          // (TMA wrote the stage and the MMAs read it, both through the async proxy; the
          // mbarrier's phase completion orders them, so no tcgen05 fence belongs here.)
          // each MMA takes 32 bytes of K from every operand row
#pragma unroll
          for (int kk = 0; kk < ROWB / 32; ++kk) {
#pragma unroll
            for (int p = 0; p < Cfg::NPROD; ++p) {
              const uint64_t ad = smem_desc<ROWB>(a_tile(s, PREC::prod_a(p)) + kk * 32);
              const uint64_t bd = smem_desc<ROWB>(b_tile(s, PREC::prod_b(p)) + kk * 32);
              if (p == 0) umma<PREC::kKind>(d_main, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
              else umma<PREC::kKind>(d_corr, ad, bd, idesc, (!first || (kb | kk) != 0 || p > 1) ? 1u : 0u);
            }
          }
          umma_commit(empty(s));
          ++it;
          *consumed = it;
        }
        if (ok) umma_commit(accf(b));
      }
      }
      // Every MMA issued above must be complete before the accumulators are released.
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, err, 16u, lim);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kEpiRegs));
    // ---------------- epilogue ----------------
    const int quad = warp & 3, half = (warp - 4) >> 2;  // (half: this warp's column share)
    const int row = quad * 32 + lane;
    const float f0 = fac ? *fac : 1.f;
    float hi[H], lo[H];
    float wc = 1.f;
    bool ok = true;
    int gs = 0, run = -1;
    for (int jb = blockIdx.x; jb < njobs && ok; jb += gridDim.x) {
      const TcJob job = jobs[jb];
      const Segment* sgs = groups ? groups[job.grp].segs : segs;
      wc = 1.f;
      for (int g = 0; g < job.nseg; ++g, ++gs) {
        const int b = gs & 1, u = gs >> 1;
        if (!mbar_wait(accf(b), u & 1, err, 8u, lim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const Segment sg = sgs[job.seg0 + g];
        // The sums are kept in units of the current segment weight wc (powers of two, so every
        // rescaling is exact and the result is that of adding w * v): a weight change inside a job
        // rescales them, the job's end multiplies by wc.
        const float w = sg.w;
        if (g == 0) {
          wc = w;
        } else if (w != wc) {
          const float r = wc / w;
#pragma unroll
          for (int c = 0; c < H; ++c) {
            hi[c] *= r;
            lo[c] *= r;
          }
          wc = w;
        }
        run += g == 0 || (sg.flags & kRunFirst);
        const bool last = Cfg::NPROD > 1 && (g == job.nseg - 1 || (sg.flags & kRunLast));
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + half * H;
        const uint32_t tm_main = lane_base + b * kTile, tm_corr = lane_base + (2 + (run & 1)) * kTile;
        // Up to kChunk columns per round trip: all loads, then one wait.
#pragma unroll
        for (int g0 = 0; g0 < H; g0 += kChunk) {
          uint32_t v[kChunk];
          if (g0 + kChunk <= H) {
            tmem_ld_32x32b_x32(tm_main + g0, v);
          } else {
#pragma unroll
            for (int q = 0; q < kChunk / 8; ++q)
              if (g0 + q * 8 < H) tmem_ld_32x32b_x8(tm_main + g0 + q * 8, v + q * 8);
          }
          tmem_ld_wait();
          // A job's first segment starts the two-float sums (no TwoSum needed).
          if (g == 0) {
#pragma unroll
            for (int c = 0; c < kChunk; ++c)
              if (g0 + c < H) {
                hi[g0 + c] = __uint_as_float(v[c]);
                lo[g0 + c] = 0.f;
              }
          } else {
#pragma unroll
            for (int c = 0; c < kChunk; c += 2)
              if (g0 + c < H) two_sum_acc2(hi[g0 + c], hi[g0 + c + 1], lo[g0 + c], lo[g0 + c + 1], v[c], v[c + 1]);
          }
        }
        if (last) {
          // The correction sum is ~2^-8 of the leading one: it joins the low word.
#pragma unroll
          for (int g0 = 0; g0 < H; g0 += kChunk) {
            uint32_t v[kChunk];
            if (g0 + kChunk <= H) {
              tmem_ld_32x32b_x32(tm_corr + g0, v);
            } else {
#pragma unroll
              for (int q = 0; q < kChunk / 8; ++q)
                if (g0 + q * 8 < H) tmem_ld_32x32b_x8(tm_corr + g0 + q * 8, v + q * 8);
            }
            tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < kChunk; c += 2)
              if (g0 + c < H) add_acc2(lo[g0 + c], lo[g0 + c + 1], v[c], v[c + 1]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce(b));
      }
      const float f = wc * (groups ? (groups[job.grp].fac ? *groups[job.grp].fac : 1.f) : f0);
      if (f != 1.f) {
#pragma unroll
        for (int c = 0; c < H; ++c) {
          hi[c] *= f;
          lo[c] *= f;
        }
      }
      if (groups) {
        typename EPI::Params gep = groups[job.grp].ep;
        epi_resolve<EPI>(gep, 0);
        if constexpr (EPI::kStaged) {
          if (ok) staged_store<H, EPI>(gep, job, quad * 32, half * H, hi, lo, staging + (warp - 4) * 256, lane);
        } else {
          if (ok && row < job.m_valid) EPI::template store<H>(gep, job, row, half * H, hi, lo);
        }
      } else {
        if constexpr (EPI::kStaged) {
          if (ok) staged_store<H, EPI>(ep, job, quad * 32, half * H, hi, lo, staging + (warp - 4) * 256, lane);
        } else {
          if (ok && row < job.m_valid) EPI::template store<H>(ep, job, row, half * H, hi, lo);
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0) {
    // Copies issued but never consumed (only after an expired wait) must land before exit.
    for (int i = *consumed; i < issued; ++i) mbar_wait(full(i % S), (i / S) & 1, err, 32u, lim);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------- output functors ----------------

// scale * (hi + lo) rounded once to FP32 and widened exactly, with scale = sh + sl given as
// two floats: the product of the two pairs is formed with an exact FMA residual (the dropped
// lo * sl is ~2^-48 relative), so the only rounding is the final one, 2^-24 relative, which
// is below the split-BF16 path's own error and keeps the FP64 pipe (1/64 of the FP32 rate on
// this part) out of the epilogue.
__device__ __forceinline__ double scaled_pair(float hi, float lo, float sh, float sl) {
  const float p = hi * sh;
  const float e = fmaf(hi, sh, -p) + fmaf(hi, sl, lo * sh);
  return f2d(p + e);
}

// Lower triangle of a symmetric result, 8-fold packed: element (m, n), m >= n, at
// m(m+1)/2 + n, m = o0 + row, n = o1 + col. Value = scale * (hi + lo), scale = sh + sl.
// A job with o2 != 0 is K part o3 of a split tile: it stores the unscaled pair (hi, lo) of
// every element of the tile to part[o3][row][col] (128 x 128), for combine_parts to sum.
struct EpiPacked {
  static constexpr bool kAInterleaved = false;
  struct Params {
    double* out;
    float sh, sl;
    unsigned long long* part;
  };
  static constexpr bool kStaged = true;
  static __device__ __forceinline__ unsigned long long value(const Params& p, const TcJob& j, float hi, float lo) {
    if (j.o2) return (unsigned long long)__float_as_uint(hi) | ((unsigned long long)__float_as_uint(lo) << 32);
    return (unsigned long long)__double_as_longlong(scaled_pair(hi, lo, p.sh, p.sl));
  }
  static __device__ __forceinline__ void put(const Params& p, const TcJob& j, int row, int col,
                                             unsigned long long v) {
    if (row >= j.m_valid || col >= j.n_valid) return;
    if (j.o2) {
      p.part[((long long)j.o3 * kTile + row) * kTile + col] = v;
      return;
    }
    const long long m = (long long)j.o0 + row, n = (long long)j.o1 + col;
    if (n <= m) p.out[m * (m + 1) / 2 + n] = __longlong_as_double((long long)v);
  }
};

// Rectangular: out[(o0 + row) * ldo + o1 + col] = scale * (hi + lo), scale = sh + sl.
struct EpiRect {
  static constexpr bool kAInterleaved = false;
  struct Params {
    double* out;
    long long ldo;
    float sh, sl;
  };
  static constexpr bool kStaged = true;
  static __device__ __forceinline__ unsigned long long value(const Params& p, const TcJob&, float hi, float lo) {
    return (unsigned long long)__double_as_longlong(scaled_pair(hi, lo, p.sh, p.sl));
  }
  static __device__ __forceinline__ void put(const Params& p, const TcJob& j, int row, int col,
                                             unsigned long long v) {
    if (row < j.m_valid && col < j.n_valid)
      p.out[((long long)j.o0 + row) * p.ldo + j.o1 + col] = __longlong_as_double((long long)v);
  }
};

// A same-spin block of complex ERIs (general orbitals): row ij of the GEMM against the ket rows
// 2 kl + c gives component c of (ij|kl); the output holds (re, im) doubles, out[ij * ldo + 2 kl + c]
// with ldo = 2 n^2. Only elements with kl <= ij are stored from their own tile, each also at its
// mirror (kl|ij) = (ij|kl) (the electron exchange symmetry; it holds exactly after the sum over q),
// so the tiles wholly above the diagonal are never computed.
struct EpiHerm {
  static constexpr bool kAInterleaved = false;
  struct Params {
    double* out;
    long long ldo;
    float sh, sl;
  };
  static constexpr bool kStaged = true;
  static __device__ __forceinline__ unsigned long long value(const Params& p, const TcJob&, float hi, float lo) {
    return (unsigned long long)__double_as_longlong(scaled_pair(hi, lo, p.sh, p.sl));
  }
  static __device__ __forceinline__ void put(const Params& p, const TcJob& j, int row, int col,
                                             unsigned long long v) {
    if (row >= j.m_valid || col >= j.n_valid) return;
    const long long ij = (long long)j.o0 + row, c = (long long)j.o1 + col, kl = c >> 1;
    if (kl > ij) return;
    const double x = __longlong_as_double((long long)v);
    p.out[ij * p.ldo + c] = x;
    if (kl < ij) p.out[kl * p.ldo + 2 * ij + (c & 1)] = x;
  }
};

// The contraction of a grouped launch, one table entry per ERI block of every problem: mode 0 is
// EpiPacked's 8-fold packed layout, 1 EpiRect's rectangular one, 2 EpiHerm's complex same-spin
// block. The block's output pointer sits in a device slot (outp) that each call rewrites, so the
// table itself is written once, when the plan is made.
struct EpiAny {
  static constexpr bool kAInterleaved = false;
  struct Params {
    double* const* outp;
    double* out;  // *outp, resolved per job
    long long ldo;
    float sh, sl;
    int mode;
  };
  static constexpr bool kStaged = true;
  static __device__ __forceinline__ void resolve(Params& p) { p.out = *p.outp; }
  static __device__ __forceinline__ unsigned long long value(const Params& p, const TcJob&, float hi, float lo) {
    return (unsigned long long)__double_as_longlong(scaled_pair(hi, lo, p.sh, p.sl));
  }
  static __device__ __forceinline__ void put(const Params& p, const TcJob& j, int row, int col,
                                             unsigned long long v) {
    if (row >= j.m_valid || col >= j.n_valid) return;
    const long long m = (long long)j.o0 + row, n = (long long)j.o1 + col;
    const double x = __longlong_as_double((long long)v);
    if (p.mode == 0) {
      if (n <= m) p.out[m * (m + 1) / 2 + n] = x;
    } else if (p.mode == 1) {
      p.out[m * p.ldo + n] = x;
    } else {
      const long long kl = n >> 1;
      if (kl > m) return;
      p.out[m * p.ldo + n] = x;
      if (kl < m) p.out[kl * p.ldo + 2 * m + (n & 1)] = x;
    }
  }
};

}  // namespace tc
}  // namespace dmet
