// fst_tc.cuh -- c = S_T^T y for a whole batch on the 5th-generation tensor cores.
//
// The rank-r correction of the fast projection (Section 4, the term S_T (D o S_T^T y))
// starts with the skinny product C = Y S_T, Y = [signals x N], S_T = [N x r].  This
// kernel computes it as one K-split GEMM per CTA:
//
//   rows    : 128 real signals, or the (re, im) rows of 64 complex signals (MMA M = 128)
//   columns : j < nB (MMA N = nB, a multiple of 32 covering r; rows j >= r of S are zero)
//   K       : nks = tc_slices(N) interleaved slices of k-tiles of 32 samples (slice s takes
//             k-tiles s, s + nks, s + 2 nks, ...); the CTAs walk the (row block, slice) items
//             round-robin with one continuous pipeline and store one partial per item, so the
//             summation order depends on N only, not on the batch or the grid.  Neighbouring
//             CTAs read neighbouring 128-byte pieces of the same rows at the same time, which
//             the DRAM serves as long runs.
//
// Each k-tile of y arrives by TMA, 128-byte swizzled, in a ring of raw buffers together
// with the k-tile of S_T^T (stored K-major in FP32 at plan time).  Eight worker warps split
// both into TF32 (hi, lo) parts: each thread reads its own row of y (conflict-free thanks to
// the swizzle), de-interleaving complex samples, and writes hi and lo straight into tensor
// memory with tcgen05.st, where the MMA takes its A operand; S hi and lo go to a small
// shared-memory ring as the B operand.  Keeping A out of shared memory matters: each TF32
// MMA has K = 8 only, and with A in shared memory its operand fetch, not the tensor core,
// set the pace.  One thread issues, per 8-sample k-step, the three products
// hi*hi + hi*lo + lo*hi into FP32 accumulators in TMEM (the missing lo*lo term is below FP32
// rounding).  Every TC_GROUP k-tiles the worker warps read the accumulators with
// tcgen05.ld into FP32 registers while the MMA fills a second set; each item ends with one
// partial row per (signal, slice), and a separate fixed-order reduction sums the slices, so
// results do not depend on scheduling.
//
// Every mbarrier wait is bounded (TC_TIMEOUT_NS of wall time): on expiry the CTA stops
// issuing work, waits (again bounded) for the copies and products it already issued,
// releases its TMEM, writes NaN partials and raises the error word.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace fst {

constexpr int TC_M = 128;                 // MMA rows
constexpr int TC_KT = 32;                 // samples per k-tile (128 bytes of FP32 per row)
constexpr int TC_WORKERS = 8;             // split + drain warps (two per TMEM lane quarter)
constexpr int TC_THREADS = 64 + 32 * TC_WORKERS;   // warp 0 TMA, warp 1 MMA + TMEM owner, then the workers
constexpr int TC_SLICE_MIN = 16;          // k-tiles per slice at least (512 samples)
constexpr int TC_SLICES_MAX = 1024;       // slices per signal at most
constexpr int TC_RAW_BYTES = TC_M * TC_KT * 4;   // 16 KB: one k-tile of y
constexpr unsigned long long TC_TIMEOUT_NS = 2000000000ull;

struct TcArgs {
  int64_t N;       // samples per signal
  int64_t rows;    // real signals, or complex signals
  int cplx;
  int nB;          // MMA N (32, 64, 96 or 128)
  int r, rpad;     // partial rows hold rpad floats, the first r meaningful
  int ktiles;      // ceil(N / TC_KT)
  int nks;         // interleaved slices
  int nitems;      // nks x row blocks
  float *part;     // [pair][nks][2][rpad]
  int *err;        // set to 1 when a wait timed out (host-mapped word, read by the host)
  unsigned long long timeout_ns;   // limit of every mbarrier wait (TC_TIMEOUT_NS)
  int stall;       // test hook: the producer first waits on a barrier nothing completes
};

// raw ring stage (shared memory): y tile + S tile; operand stage: S hi + S lo in shared
// memory, y hi + y lo in TMEM (2 TC_KT columns)
__host__ __device__ constexpr int tc_op_depth(int nB) { return nB == 64 ? 2 : 3; }
__host__ __device__ constexpr int tc_raw_stage(int nB) { return TC_RAW_BYTES + nB * 128; }
__host__ __device__ constexpr int tc_op_stage(int nB) { return 2 * nB * 128; }
__host__ __device__ constexpr int tc_raw_depth(int nB) {
  return nB <= 32 ? 8 : (nB <= 64 ? 7 : (nB <= 96 ? 5 : 4));
}
__host__ __device__ constexpr int tc_smem_bytes(int nB) {
  return tc_raw_depth(nB) * tc_raw_stage(nB) + tc_op_depth(nB) * tc_op_stage(nB) + 512 + 1024;
}
// Each tcgen05.mma costs a roughly fixed time when it is as small as these (K = 8), so the
// count matters more than the size.  For nB <= 64 the S hi and lo tiles, adjacent in shared
// memory, form one B operand of 2 nB rows: one MMA gives hi*hi and hi*lo side by side, a
// second lo*hi, into three nB-column accumulators (nacc = 3).  Wider S falls back to three
// MMAs into one accumulator.  TMEM: op-depth A stages of 2 TC_KT columns, then 2 buffers of
// nacc x nB columns.
__host__ __device__ constexpr int tc_nacc(int nB) { return nB <= 64 ? 3 : 1; }
constexpr uint32_t TC_TMEM_COLS = 512;
static_assert(3 * 2 * TC_KT + 2 * 3 * 32 <= 512 && 2 * 2 * TC_KT + 2 * 3 * 64 <= 512 &&
                  3 * 2 * TC_KT + 2 * 128 <= 512,
              "TMEM budget");

// instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, shape M x N (A in tensor memory is K-major by construction)
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// k-tiles per slice of the sample axis for signal length N (even: whole MMA groups), and
// the number of slices; both depend on N only
__host__ __device__ inline int tc_slice_len(int64_t N) {
  const int64_t kt = (N + TC_KT - 1) / TC_KT;
  int64_t L = (kt + TC_SLICES_MAX - 1) / TC_SLICES_MAX;
  L = L < TC_SLICE_MIN ? TC_SLICE_MIN : L;
  return (int)((L + 1) / 2 * 2);
}
__host__ __device__ inline int tc_slices(int64_t N) {
  const int64_t kt = (N + TC_KT - 1) / TC_KT;
  return (int)((kt + tc_slice_len(N) - 1) / tc_slice_len(N));
}

// kernels: compiled only in the translation unit that launches them
#if defined(__CUDACC__) && defined(FST_TC_KERNELS)

__device__ __forceinline__ uint64_t tc_gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity.  Returns false when the CTA gave up:
// either the shared abort flag is up (honoured only if `honour_abort`) or this wait ran
// past `limit_ns` of wall time, which raises the flag.
__device__ __noinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, bool honour_abort,
                                     unsigned long long limit_ns) {
  if (tc_mbar_try(bar, parity)) return true;
  const uint64_t t0 = tc_gtimer();
  for (;;) {
    if (tc_mbar_try(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if (tc_gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tc_tma_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared memory descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes in
// 8-row atoms (stride 1024 bytes); `addr` is the shared-window byte address
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (not used by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// A operand from tensor memory (`a` = TMEM address of its first column), B from shared memory
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 16 consecutive TMEM columns of this thread's lane (no wait)
__device__ __forceinline__ void tc_st16(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tc_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's TMEM lane (no wait)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t *u) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tc_hi(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// TMEM accumulation is coarser than FP32 round-to-nearest, so each accumulator buffer holds
// only TC_GROUP k-tiles (TC_GROUP x 4 x 3 accumulation steps); the epilogue warps drain it
// into FP32 registers while the MMA fills the other buffer.
constexpr int TC_GROUP = 2;

// item it of a CTA: row block it / nks, slice ks = it % nks: k-tiles ks + tt nks, tt < ntile
struct TcItem {
  int rb, ks, ntile;
};
__device__ __forceinline__ TcItem tc_item(const TcArgs &t, int it) {
  TcItem x;
  x.rb = it / t.nks;
  x.ks = it % t.nks;
  x.ntile = (t.ktiles - x.ks + t.nks - 1) / t.nks;
  return x;
}

template <int NB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_corr_tc(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmS, const TcArgs t) {
  extern __shared__ uint8_t tc_smem[];
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(tc_smem);
  const uint32_t base = (s0 + 1023u) & ~1023u;        // 128-byte swizzle atoms need 1024-byte alignment
  uint8_t *gbase = tc_smem + (base - s0);
  constexpr int SA = tc_raw_stage(NB), SO = tc_op_stage(NB), RA = tc_raw_depth(NB), RB = tc_op_depth(NB);
  constexpr int NACC = tc_nacc(NB);
  constexpr uint32_t ACC0 = RB * 2 * TC_KT;            // TMEM: A stages first, then the accumulators
  const uint32_t opb = base + RA * SA;                 // S hi/lo ring
  // barriers: fullA[a] (TMA landed), freeA[a] (raw read), fullB[b] (operands written),
  // emptyB[b] (products retired), accfull[c], accempty[c] (accumulator buffer c), done
  const uint32_t bars = opb + RB * SO;
  const uint32_t fullA = bars, freeA = bars + 64, fullB = bars + 128, emptyB = bars + 160;
  const uint32_t afull0 = bars + 192, aempty0 = bars + 208, done = bars + 224;
  const uint32_t stall = bars + 240;   // test hook only: never completed
  uint8_t *gbars = gbase + (bars - base);
  uint32_t *tslot = (uint32_t *)(gbars + 232);
  volatile int *abort_flag = (volatile int *)(gbars + 236);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int a = 0; a < RA; ++a) {
      tc_mbar_init(fullA + 8 * a, 1);
      tc_mbar_init(freeA + 8 * a, TC_WORKERS);
    }
    for (int b = 0; b < RB; ++b) {
      tc_mbar_init(fullB + 8 * b, TC_WORKERS);
      tc_mbar_init(emptyB + 8 * b, 1);
    }
    for (int c = 0; c < 2; ++c) {
      tc_mbar_init(afull0 + 8 * c, 1);
      tc_mbar_init(aempty0 + 8 * c, TC_WORKERS);
    }
    tc_mbar_init(done, 1);
    tc_mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(bars + 232),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- producer: y tile (swizzled) + S tile per raw stage, item after item
    if (lane == 0) {
      int i = 0, issued = 0;
      bool go = true;
      // test hook: give up before the first copy, on a wait that nothing can complete
      if (t.stall) go = tc_wait(stall, 0u, abort_flag, true, t.timeout_ns);
      for (int it = blockIdx.x; it < t.nitems && go; it += gridDim.x) {
        const TcItem x = tc_item(t, it);
        for (int tt = 0; tt < x.ntile; ++tt, ++i) {
          const int a = i % RA;
          if (i >= RA && !tc_wait(freeA + 8 * a, (uint32_t)((i / RA) - 1) & 1u, abort_flag, true, t.timeout_ns)) {
            go = false;
            break;
          }
          const uint32_t st = base + (uint32_t)(a * SA);
          tc_mbar_expect_tx(fullA + 8 * a, (uint32_t)SA);
          const int kt = x.ks + tt * t.nks;
          if (t.cplx) {
            // two halves of 16 complex samples (128 bytes per row each)
            tc_tma_2d(st, &tmY, fullA + 8 * a, kt * 2 * TC_KT, x.rb * (TC_M / 2));
            tc_tma_2d(st + TC_RAW_BYTES / 2, &tmY, fullA + 8 * a, kt * 2 * TC_KT + TC_KT, x.rb * (TC_M / 2));
          } else {
            tc_tma_2d(st, &tmY, fullA + 8 * a, kt * TC_KT, x.rb * TC_M);
          }
          tc_tma_2d(st + TC_RAW_BYTES, &tmS, fullA + 8 * a, kt * TC_KT, 0);
          issued = i + 1;
        }
      }
      // the copies issued last must land before the CTA may exit
      for (int j = max(0, issued - RA); j < issued; ++j)
        tc_wait(fullA + 8 * (j % RA), (uint32_t)(j / RA) & 1u, abort_flag, false, t.timeout_ns);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer: groups of TC_GROUP k-tiles of one item into accumulator buffer g & 1
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_tf32(TC_M, NB);
      const uint32_t idesc2 = tc_idesc_tf32(TC_M, 2 * NB);   // B = [S hi; S lo]
      int i = 0, g = 0;
      bool go = true;
      for (int it = blockIdx.x; it < t.nitems && go; it += gridDim.x) {
        const TcItem x = tc_item(t, it);
        for (int tt = 0; tt < x.ntile; ++tt, ++i) {
          const int b = i % RB, c = g & 1;
          const bool first = (tt % TC_GROUP) == 0;
          if (first && g >= 2 && !tc_wait(aempty0 + 8 * c, (uint32_t)((g / 2) - 1) & 1u, abort_flag, true, t.timeout_ns)) {
            go = false;
            break;
          }
          if (!tc_wait(fullB + 8 * b, (uint32_t)(i / RB) & 1u, abort_flag, true, t.timeout_ns)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t ahi = tmem + (uint32_t)(b * 2 * TC_KT), alo = ahi + TC_KT;
          const uint32_t bh = opb + (uint32_t)(b * SO);
          const uint32_t acc = tmem + ACC0 + (uint32_t)(c * NACC * NB);
          // a k-step of 8 samples is 32 bytes along the 128-byte rows: +2 in the address field
          const uint64_t dbh = tc_desc_sw128(bh), dbl = tc_desc_sw128(bh + 128 * NB);
#pragma unroll
          for (int k = 0; k < TC_KT / 8; ++k) {
            const uint32_t fresh = (first && k == 0) ? 0u : 1u;
            if (NACC == 3) {
              tc_mma_ts(acc, ahi + 8 * k, dbh + 2 * k, idesc2, fresh);
              tc_mma_ts(acc + 2 * NB, alo + 8 * k, dbh + 2 * k, idesc, fresh);
            } else {
              tc_mma_ts(acc, ahi + 8 * k, dbh + 2 * k, idesc, fresh);
              tc_mma_ts(acc, ahi + 8 * k, dbl + 2 * k, idesc, 1u);
              tc_mma_ts(acc, alo + 8 * k, dbh + 2 * k, idesc, 1u);
            }
          }
          tc_commit(emptyB + 8 * b);
          if ((tt % TC_GROUP) == TC_GROUP - 1 || tt == x.ntile - 1) {
            tc_commit(afull0 + 8 * c);
            ++g;
          }
        }
      }
      // every product issued has retired once `done` completes (also after an abort)
      tc_commit(done);
    }
    __syncwarp();
  } else {
    // ---- workers: TF32 split of y (rows into TMEM) and S (shared); drains; partials
    constexpr int NH = NB / 2;        // accumulator columns drained by this warp
    const int tw = threadIdx.x - 64;  // 0 .. 32 TC_WORKERS - 1
    const int q = warp & 3;           // TMEM lane quarter of this warp: rows 32 q + lane
    const int h = (warp - 2) >> 2;    // samples [16 h, 16 h + 16) of a k-tile; columns [h NH, (h + 1) NH)
    const int m = 32 * q + lane;
    const uint32_t lq = (uint32_t)(32 * q) << 16;
    float sum[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) sum[j] = 0.f;
    bool ok = true;
    // store the partial row of item it (NaN after an abort) and restart the sums
    auto flush = [&](int it) {
      const TcItem x = tc_item(t, it);
      int64_t sig, pair;
      int comp;
      if (!t.cplx) {
        sig = (int64_t)x.rb * TC_M + m;
        pair = sig >> 1;
        comp = (int)(sig & 1);
      } else {
        sig = (int64_t)x.rb * (TC_M / 2) + (m & 63);
        pair = sig;
        comp = m >> 6;
      }
      // real: the partner of an odd last signal gets its (zero) row too
      const bool valid = t.cplx ? sig < t.rows : pair < (t.rows + 1) / 2;
      if (valid) {
        float *dst = t.part + ((pair * t.nks + x.ks) * 2 + comp) * t.rpad + h * NH;
#pragma unroll
        for (int j = 0; j < NH; ++j)
          if (h * NH + j < t.rpad) dst[j] = ok ? sum[j] : __int_as_float(0x7fc00000);
      }
#pragma unroll
      for (int j = 0; j < NH; ++j) sum[j] = 0.f;
    };
    // add finished group g (of item it; the item's last group if `last`) into the sums
    auto drain = [&](int g, int it, bool last) {
      const int c = g & 1;
      if (ok) ok = tc_wait(afull0 + 8 * c, (uint32_t)(g / 2) & 1u, abort_flag, true, t.timeout_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
        uint32_t u[NACC][NH];
#pragma unroll
        for (int ac = 0; ac < NACC; ++ac)
#pragma unroll
          for (int cb = 0; cb < NH / 16; ++cb)
            tc_ld16(tmem + lq + ACC0 + (uint32_t)((c * NACC + ac) * NB + h * NH + 16 * cb), &u[ac][16 * cb]);
        tc_ld_wait();
        // fixed order: the accumulators, then into the running sum
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          float g0 = __uint_as_float(u[0][j]);
#pragma unroll
          for (int ac = 1; ac < NACC; ++ac) g0 += __uint_as_float(u[ac][j]);
          sum[j] += g0;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) tc_mbar_arrive(aempty0 + 8 * c);
      }
      if (last) flush(it);
    };
    int i = 0, g = 0;
    int prev_it = -1;
    bool prev_last = false;
    for (int it = blockIdx.x; it < t.nitems; it += gridDim.x) {
      const TcItem x = tc_item(t, it);
      for (int tt = 0; tt < x.ntile; ++tt, ++i) {
        const int a = i % RA, b = i % RB;
        if (ok) ok = tc_wait(fullA + 8 * a, (uint32_t)(i / RA) & 1u, abort_flag, true, t.timeout_ns);
        if (ok && i >= RB) ok = tc_wait(emptyB + 8 * b, (uint32_t)((i / RB) - 1) & 1u, abort_flag, true, t.timeout_ns);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          tc_fence_after();
          const uint8_t *ra = gbase + a * SA;
          float v[16];
          if (!t.cplx) {
            // row m, samples 16 h .. 16 h + 15: chunks 4 h .. 4 h + 3, chunk c stored at c ^ (m & 7)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int c = 4 * h + k;
              const float4 f = *(const float4 *)(ra + m * 128 + ((c ^ (m & 7)) << 4));
              v[4 * k] = f.x;
              v[4 * k + 1] = f.y;
              v[4 * k + 2] = f.z;
              v[4 * k + 3] = f.w;
            }
          } else {
            // row m: part m >> 6 (re, im) of signal m & 63; half h holds complex samples 16 h ..
            const int sg = m & 63;
            const bool im = m >= 64;
            const uint8_t *hb = ra + h * (TC_RAW_BYTES / 2) + sg * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const float4 f = *(const float4 *)(hb + ((c ^ (sg & 7)) << 4));
              v[2 * c] = im ? f.y : f.x;
              v[2 * c + 1] = im ? f.w : f.z;
            }
          }
          float vh[16], vl[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            vh[j] = tc_hi(v[j]);
            vl[j] = v[j] - vh[j];
          }
          const uint32_t acol = (uint32_t)(b * 2 * TC_KT + 16 * h);
          tc_st16(tmem + lq + acol, vh);
          tc_st16(tmem + lq + acol + TC_KT, vl);
          // S tile: already swizzled by the TMA; hi and lo keep its layout
          constexpr int NS = NB * 8 / (32 * TC_WORKERS);
          const float4 *sraw = (const float4 *)(ra + TC_RAW_BYTES);
          float4 *shi = (float4 *)(gbase + (opb - base) + b * SO), *slo = shi + NB * 8;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            const int qq = k * 32 * TC_WORKERS + tw;
            const float4 sv = sraw[qq];
            const float4 hs = make_float4(tc_hi(sv.x), tc_hi(sv.y), tc_hi(sv.z), tc_hi(sv.w));
            shi[qq] = hs;
            slo[qq] = make_float4(sv.x - hs.x, sv.y - hs.y, sv.z - hs.z, sv.w - hs.w);
          }
          tc_st_wait();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            tc_mbar_arrive(freeA + 8 * a);
            tc_mbar_arrive(fullB + 8 * b);
          }
        }
        if ((tt % TC_GROUP) == TC_GROUP - 1 || tt == x.ntile - 1) {
          // group g is fully split: drain the group before it
          if (g >= 1) drain(g - 1, prev_it, prev_last);
          prev_it = it;
          prev_last = tt == x.ntile - 1;
          ++g;
        }
      }
    }
    if (g >= 1) drain(g - 1, prev_it, prev_last);
    // every product must retire before the TMEM is released
    tc_wait(done, 0u, abort_flag, false, t.timeout_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) {
    *(volatile int *)t.err = 1;
    __threadfence_system();
  }
}

// S_T^T in FP32, K-major: STt[j][n] (zero for j >= r, n >= N)
__global__ void k_tc_prep(const float *ST, int64_t N, int rpad, int r, int nB, int64_t Npad, float *STt) {
  const int64_t total = (int64_t)nB * Npad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / Npad);
    const int64_t n = e % Npad;
    STt[e] = (j < r && n < N) ? ST[n * rpad + j] : 0.f;
  }
}

#endif  // __CUDACC__ && FST_TC_KERNELS


}  // namespace fst
