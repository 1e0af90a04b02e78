// fst_tc.cuh -- c = S_T^T y for a whole batch on the 5th-generation tensor cores.
//
// The rank-r correction of the fast projection (Section 4, the term S_T (D o S_T^T y))
// starts with the skinny product C = Y S_T, Y = [signals x N], S_T = [N x r].  This
// kernel computes it as one K-split GEMM per CTA:
//
//   rows    : 128 real signals, or the (re, im) rows of 64 complex signals (MMA M = 128)
//   columns : j < nB (MMA N = nB, a multiple of 32 covering r; rows j >= r of S are zero)
//   K       : slices of TC_SLICE k-tiles of 32 samples; the CTAs walk the (row block, slice)
//             items round-robin with one continuous pipeline and store one partial per item,
//             so the summation order depends on N only, not on the batch or the grid
//
// Each k-tile of y arrives by TMA (no swizzle) into a raw buffer; four worker warps split it
// into TF32 (hi, lo) parts written in the 128-byte-swizzled K-major layout the MMA reads,
// de-interleaving complex samples on the way.  S_T^T is stored K-major at plan time as
// TF32 hi and lo parts and arrives by TMA already swizzled.  One thread issues, per 8-sample
// k-step, the three products hi*hi + hi*lo + lo*hi into an FP32 accumulator in TMEM (the
// missing lo*lo term is below FP32 rounding).  Every TC_GROUP k-tiles the epilogue warps
// read the accumulator with tcgen05.ld into FP32 registers while the MMA fills a second
// accumulator; at the end each stores one partial row per (signal, slice), and a separate
// fixed-order reduction sums the slices, so results do not depend on scheduling.
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
constexpr int TC_THREADS = 192;           // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2-5 split + epilogue
constexpr int TC_SLICE = 16;              // k-tiles per slice (512 samples)
constexpr int TC_RAW_BYTES = TC_M * TC_KT * 4;   // 16 KB: one k-tile of y
constexpr unsigned long long TC_TIMEOUT_NS = 2000000000ull;

struct TcArgs {
  int64_t N;       // samples per signal
  int64_t rows;    // real signals, or complex signals
  int cplx;
  int nB;          // MMA N (32, 64, 96 or 128)
  int r, rpad;     // partial rows hold rpad floats, the first r meaningful
  int ktiles;      // ceil(N / TC_KT)
  int nks;         // slices: ceil(ktiles / TC_SLICE)
  int nitems;      // nks x row blocks
  int stages;      // pipeline depth (2 or 3)
  float *part;     // [pair][nks][2][rpad]
  int *err;        // set to 1 when a wait timed out
};

// bytes of one pipeline stage: raw y tile, hi tile, lo tile, S hi and lo tiles
__host__ __device__ constexpr int tc_stage_bytes(int nB) { return 3 * TC_RAW_BYTES + 2 * nB * 128; }
__host__ __device__ constexpr int tc_smem_bytes(int nB, int stages) { return stages * tc_stage_bytes(nB) + 256 + 1024; }
// two accumulator buffers of nB columns, allocated as a power of two >= 32
__host__ __device__ constexpr uint32_t tc_tmem_cols(int nB) { return 2 * nB <= 32 ? 32u : (2 * nB <= 64 ? 64u : (2 * nB <= 128 ? 128u : 256u)); }

// instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, shape M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// slices of the sample axis for signal length N
__host__ __device__ inline int tc_slices(int64_t N) {
  return (int)(((N + TC_KT - 1) / TC_KT + TC_SLICE - 1) / TC_SLICE);
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
// past the time limit, which raises the flag.
__device__ __noinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, bool honour_abort) {
  if (tc_mbar_try(bar, parity)) return true;
  const uint64_t t0 = tc_gtimer();
  for (;;) {
    if (tc_mbar_try(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if (tc_gtimer() - t0 > TC_TIMEOUT_NS) {
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
// 32 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float *v) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ float tc_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// TMEM accumulation is coarser than FP32 round-to-nearest, so each accumulator buffer holds
// only TC_GROUP k-tiles (TC_GROUP x 4 x 3 accumulation steps); the epilogue warps drain it
// into FP32 registers while the MMA fills the other buffer.
constexpr int TC_GROUP = 2;

// item it of a CTA: row block it / nks, slice it % nks, k-tiles [ks TC_SLICE, ...)
struct TcItem {
  int rb, ks, kt0, ntile;
};
__device__ __forceinline__ TcItem tc_item(const TcArgs &t, int it) {
  TcItem x;
  x.rb = it / t.nks;
  x.ks = it % t.nks;
  x.kt0 = x.ks * TC_SLICE;
  x.ntile = min(TC_SLICE, t.ktiles - x.kt0);
  return x;
}

template <int NB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_corr_tc(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmS, const TcArgs t) {
  extern __shared__ uint8_t tc_smem[];
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(tc_smem);
  const uint32_t base = (s0 + 1023u) & ~1023u;        // 128-byte swizzle atoms need 1024-byte alignment
  uint8_t *gbase = tc_smem + (base - s0);
  constexpr int SB = tc_stage_bytes(NB);
  const int S = t.stages;
  // barriers: full[s] (TMA landed), split[s] (hi/lo written), freeb[s] (products retired),
  // accfull[b] (buffer b holds a finished group), accempty[b] (buffer b drained), done
  const uint32_t bars = base + (uint32_t)(S * SB);
  const uint32_t full0 = bars, split0 = bars + 32, free0 = bars + 64;
  const uint32_t afull0 = bars + 96, aempty0 = bars + 112, done = bars + 128;
  uint32_t *tslot = (uint32_t *)(gbase + S * SB + 136);
  volatile int *abort_flag = (volatile int *)(gbase + S * SB + 140);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t ncols = tc_tmem_cols(NB);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc_mbar_init(full0 + 8 * s, 1);
      tc_mbar_init(split0 + 8 * s, 4);
      tc_mbar_init(free0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc_mbar_init(afull0 + 8 * b, 1);
      tc_mbar_init(aempty0 + 8 * b, 4);
    }
    tc_mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(bars + 136), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- producer: y tile + S hi/lo tiles per stage, item after item
    if (lane == 0) {
      const uint32_t tx = (uint32_t)TC_RAW_BYTES + 256u * (uint32_t)NB;
      int i = 0, issued = 0;
      bool go = true;
      for (int it = blockIdx.x; it < t.nitems && go; it += gridDim.x) {
        const TcItem x = tc_item(t, it);
        for (int tt = 0; tt < x.ntile; ++tt, ++i) {
          const int s = i % S;
          if (i >= S && !tc_wait(free0 + 8 * s, (uint32_t)((i / S) - 1) & 1u, abort_flag, true)) {
            go = false;
            break;
          }
          const uint32_t st = base + (uint32_t)(s * SB);
          tc_mbar_expect_tx(full0 + 8 * s, tx);
          const int kt = x.kt0 + tt;
          if (t.cplx) tc_tma_2d(st, &tmY, full0 + 8 * s, kt * 2 * TC_KT, x.rb * (TC_M / 2));
          else tc_tma_2d(st, &tmY, full0 + 8 * s, kt * TC_KT, x.rb * TC_M);
          tc_tma_2d(st + 3 * TC_RAW_BYTES, &tmS, full0 + 8 * s, kt * TC_KT, 0);
          tc_tma_2d(st + 3 * TC_RAW_BYTES + 128 * NB, &tmS, full0 + 8 * s, kt * TC_KT, NB);
          issued = i + 1;
        }
      }
      // the copies issued last must land before the CTA may exit
      for (int j = max(0, issued - S); j < issued; ++j)
        tc_wait(full0 + 8 * (j % S), (uint32_t)(j / S) & 1u, abort_flag, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer: groups of TC_GROUP k-tiles of one item into accumulator buffer g & 1
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_tf32(TC_M, NB);
      int i = 0, g = 0;
      bool go = true;
      for (int it = blockIdx.x; it < t.nitems && go; it += gridDim.x) {
        const TcItem x = tc_item(t, it);
        for (int tt = 0; tt < x.ntile; ++tt, ++i) {
          const int s = i % S, b = g & 1;
          const bool first = (tt % TC_GROUP) == 0;
          if (first && g >= 2 && !tc_wait(aempty0 + 8 * b, (uint32_t)((g / 2) - 1) & 1u, abort_flag, true)) {
            go = false;
            break;
          }
          if (!tc_wait(split0 + 8 * s, (uint32_t)(i / S) & 1u, abort_flag, true)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + (uint32_t)(s * SB);
          const uint32_t ah = st + TC_RAW_BYTES, al = st + 2 * TC_RAW_BYTES;
          const uint32_t bh = st + 3 * TC_RAW_BYTES, bl = bh + 128 * NB;
          const uint32_t acc = tmem + (uint32_t)(b * NB);
#pragma unroll
          for (int k = 0; k < TC_KT / 8; ++k) {
            const uint64_t dah = tc_desc_sw128(ah + 32 * k), dal = tc_desc_sw128(al + 32 * k);
            const uint64_t dbh = tc_desc_sw128(bh + 32 * k), dbl = tc_desc_sw128(bl + 32 * k);
            tc_mma(acc, dah, dbh, idesc, (first && k == 0) ? 0u : 1u);
            tc_mma(acc, dah, dbl, idesc, 1u);
            tc_mma(acc, dal, dbh, idesc, 1u);
          }
          tc_commit(free0 + 8 * s);
          if ((tt % TC_GROUP) == TC_GROUP - 1 || tt == x.ntile - 1) {
            tc_commit(afull0 + 8 * b);
            ++g;
          }
        }
      }
      // every product issued has retired once `done` completes (also after an abort)
      tc_commit(done);
    }
    __syncwarp();
  } else {
    // ---- workers: TF32 split into the swizzled K-major hi/lo tiles; drains; partials
    const int tw = threadIdx.x - 64;
    const int q = warp & 3;   // TMEM lane quarter of this warp: rows 32 q + lane
    const int m = 32 * q + lane;
    float sum[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) sum[j] = 0.f;
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
        float *dst = t.part + ((pair * t.nks + x.ks) * 2 + comp) * t.rpad;
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < t.rpad) dst[j] = ok ? sum[j] : __int_as_float(0x7fc00000);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) sum[j] = 0.f;
    };
    // add finished group g (of item it; the item's last group if `last`) into the sums
    auto drain = [&](int g, int it, bool last) {
      const int b = g & 1;
      if (ok) ok = tc_wait(afull0 + 8 * b, (uint32_t)(g / 2) & 1u, abort_flag, true);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
#pragma unroll
        for (int cb = 0; cb < NB / 32; ++cb) {
          float v[32];
          tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * NB + 32 * cb), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[32 * cb + j] += v[j];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) tc_mbar_arrive(aempty0 + 8 * b);
      }
      if (last) flush(it);
    };
    int i = 0, g = 0;
    int prev_it = -1;
    bool prev_last = false;
    for (int it = blockIdx.x; it < t.nitems; it += gridDim.x) {
      const TcItem x = tc_item(t, it);
      for (int tt = 0; tt < x.ntile; ++tt, ++i) {
        const int s = i % S;
        if (ok) ok = tc_wait(full0 + 8 * s, (uint32_t)(i / S) & 1u, abort_flag, true);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          uint8_t *st = gbase + s * SB;
          const float4 *raw = (const float4 *)st;
          uint8_t *hi = st + TC_RAW_BYTES, *lo = st + 2 * TC_RAW_BYTES;
          if (!t.cplx) {
            // raw: [128 rows][32 floats]; 16-byte chunk c of row r goes to chunk c ^ (r & 7)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int qq = k * 128 + tw;
              const int r = qq >> 3, c = qq & 7;
              const float4 v = raw[qq];
              const float4 h = make_float4(tc_hi(v.x), tc_hi(v.y), tc_hi(v.z), tc_hi(v.w));
              const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
              const int off = r * 128 + ((c ^ (r & 7)) << 4);
              *(float4 *)(hi + off) = h;
              *(float4 *)(lo + off) = l;
            }
          } else {
            // raw: [64 rows][32 complex]; real parts to row r, imaginary parts to row 64 + r
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int qq = k * 128 + tw;
              const int r = qq >> 4, cc = qq & 15;
              const float4 v = raw[qq];   // (re, im) of samples 2 cc and 2 cc + 1
              const int sub = (cc & 1) * 8, c = cc >> 1;
              const int offr = r * 128 + ((c ^ (r & 7)) << 4) + sub;
              const int offi = offr + 64 * 128;   // (r + 64) & 7 == r & 7
              const float2 hr = make_float2(tc_hi(v.x), tc_hi(v.z)), hm = make_float2(tc_hi(v.y), tc_hi(v.w));
              *(float2 *)(hi + offr) = hr;
              *(float2 *)(lo + offr) = make_float2(v.x - hr.x, v.z - hr.y);
              *(float2 *)(hi + offi) = hm;
              *(float2 *)(lo + offi) = make_float2(v.y - hm.x, v.w - hm.y);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) tc_mbar_arrive(split0 + 8 * s);
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
    tc_wait(done, 0u, abort_flag, false);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(t.err, 1);
}

// S_T^T as K-major TF32 parts: STt[j][n] = hi, STt[nB + j][n] = lo (zero for j >= r, n >= N)
__global__ void k_tc_prep(const float2 *hl, int64_t N, int rpad, int r, int nB, int64_t Npad, float *STt) {
  const int64_t total = (int64_t)nB * Npad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / Npad);
    const int64_t n = e % Npad;
    float2 v = make_float2(0.f, 0.f);
    if (j < r && n < N) v = hl[n * rpad + j];
    STt[e] = v.x;
    STt[(int64_t)nB * Npad + e] = v.y;
  }
}

#endif  // __CUDACC__ && FST_TC_KERNELS

}  // namespace fst
