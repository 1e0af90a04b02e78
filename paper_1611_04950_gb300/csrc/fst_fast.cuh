// fst_fast.cuh -- FP32 four-step kernels for P = 8, 16, 32 column rows (device only).
//
// Same algorithm and data layout as the generic passA/passB/passC bodies of
// fst_kernels.cuh (n = n1 Q + n2, k = k1 + P k2, inter[pair][k1][n2]), restructured
// for the GB300 memory system:
//   * column passes: one thread owns one whole column (all P rows of one n2 of one
//     pair) in registers, so the P-point DFT needs no shared memory and every
//     global access is coalesced across the 32 columns of a warp;
//   * the rank-r correction runs on the tensor cores: per CTA tile (8 pairs = 16
//     real signals x 32 columns x Pnz rows) the partial sums S_T^T y and the
//     epilogue S_T a are small matrix products done with mma.sync m16n8k8 TF32,
//     each operand split as hi + lo (both TF32) and three products kept
//     (hi*hi + hi*lo + lo*hi), which keeps FP32-level accuracy;
//   * row pass: the first radix-16 stage reads straight from global memory, the
//     forward transform's last stage, the spectrum multiply and the inverse
//     transform's first stage stay in registers, and the last stage writes straight
//     to global memory (4 shared-memory round trips per row instead of 8).
#pragma once
#include "fst_kernels.cuh"

namespace fst {

constexpr int FAST_G = 8;      // pairs per column tile
constexpr int FAST_NB = 32;    // columns (n2 values) per pair per tile
constexpr int FAST_THREADS = FAST_G * FAST_NB;   // one thread per column
constexpr int YT_STRIDE = 516; // padded row stride (floats) of the signal-major tile

struct FastArgs {
  ConvArgs<float> a;
  const float2 *ST_hl;  // [N][rpad] (TF32-rounded S_T, TF32 of the remainder) interleaved
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
// D += A(16x8, row) * B(8x8, col), TF32 inputs, FP32 accumulate
__device__ __forceinline__ void mma_tf32(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma3(float *d, const uint32_t *ahi, const uint32_t *alo, const uint32_t *bhi,
                                     const uint32_t *blo) {
  mma_tf32(d, alo, bhi);
  mma_tf32(d, ahi, blo);
  mma_tf32(d, ahi, bhi);
}

// In-register DFT of length P (8, 16 or 32) in natural order, unnormalised.
template <int P, bool INV> struct RegDft;
template <bool INV> struct RegDft<2, INV> {
  __device__ __forceinline__ static void run(float2 *v) { Dft<float, 2, INV>::run(v); }
};
template <bool INV> struct RegDft<4, INV> {
  __device__ __forceinline__ static void run(float2 *v) { Dft<float, 4, INV>::run(v); }
};
template <bool INV> struct RegDft<8, INV> {
  __device__ __forceinline__ static void run(float2 *v) { Dft<float, 8, INV>::run(v); }
};
template <bool INV> struct RegDft<16, INV> {
  __device__ __forceinline__ static void run(float2 *v) { Dft<float, 16, INV>::run(v); }
};
template <bool INV> struct RegDft<32, INV> {
  // 32 = 16 x 2: Y_b = DFT16 over a of x[2a + b]; Y_1[c] *= W32^c; X[c + 16d] = Y_0[c] +- Y_1[c]
  __device__ __forceinline__ static void run(float2 *v) {
    float2 e[16], o[16];
#pragma unroll
    for (int a = 0; a < 16; ++a) { e[a] = v[2 * a]; o[a] = v[2 * a + 1]; }
    Dft<float, 16, INV>::run(e);
    Dft<float, 16, INV>::run(o);
    constexpr double C[8] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                             0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                             0.19509032201612826785};
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      // W32^c = cos(2 pi c/32) - i sin(2 pi c/32)
      const int cc = c & 7;
      float cr, si;
      if (c < 8) { cr = (float)C[cc]; si = (float)C[(8 - cc) & 7]; if (cc == 0) si = 0.f; }
      else { cr = -(float)C[(8 - cc) & 7]; si = (float)C[cc]; if (cc == 0) cr = 0.f; }
      if (c == 8) { cr = 0.f; si = 1.f; }
      const float2 w = make_float2(cr, INV ? si : -si);
      const float2 t = (c == 0) ? o[c] : cmul(o[c], w);
      v[c] = cadd(e[c], t);
      v[c + 16] = csub(e[c], t);
    }
  }
};

// exp(-+2 pi i n / P) for P in {8, 16, 32}, n < P (compile-time n: folds to constants)
template <int P, bool INV> __device__ __forceinline__ float2 wP(int n) {
  constexpr double C[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                           0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                           0.19509032201612826785, 0.0};   // cos(2 pi k / 32), k = 0..8
  const int k = n * (32 / P), q = k >> 3, r = k & 7;
  const double c = C[r], sn = C[8 - r];                    // cos, sin of 2 pi r / 32
  double re, im;                                           // cos, sin of 2 pi k / 32
  if (q == 0) { re = c; im = sn; } else if (q == 1) { re = -sn; im = c; }
  else if (q == 2) { re = -c; im = -sn; } else { re = sn; im = -c; }
  return make_float2((float)re, INV ? (float)im : (float)-im);
}

// Forward P-point DFT of a column whose rows n >= P/2 are zero (M >= 2N): with e = x and
// o[n] = x[n] W_P^n (n < P/2), X[2m] = DFT_{P/2}(e)[m] and X[2m+1] = DFT_{P/2}(o)[m].
// In: v[0 .. P/2); out: v[0 .. P) in natural order.
template <int P> __device__ __forceinline__ void dft_half_in(float2 *v) {
  constexpr int H = P / 2;
  // o in the upper half (its rows are zero on input), e in place
#pragma unroll
  for (int n = 0; n < H; ++n) v[H + n] = (n == 0) ? v[0] : cmul(v[n], wP<P, false>(n));
  Dft<float, H, false>::run(v);
  Dft<float, H, false>::run(v + H);
  float2 t[P];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    t[2 * m] = v[m];
    t[2 * m + 1] = v[H + m];
  }
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = t[k];
}

// The first P/2 outputs of the inverse P-point DFT of v (natural order in), into out:
// X[n] = IDFT_{P/2}(even rows)[n] + W_P^{-n} IDFT_{P/2}(odd rows)[n], n < P/2.
template <int P> __device__ __forceinline__ void idft_half_out(const float2 *v, float2 *out) {
  constexpr int H = P / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  Dft<float, H, true>::run(e);
  Dft<float, H, true>::run(o);
#pragma unroll
  for (int n = 0; n < H; ++n) out[n] = cadd(e[n], (n == 0) ? o[0] : cmul(o[n], wP<P, true>(n)));
}

// P-point DFT of column n2 (v; rows n1 >= P/2 zero), times W_M^{n2 k1}, stored to
// inter[row0 + k1 Q + n2].
template <int P>
__device__ __forceinline__ void fastA_finish(const ConvArgs<float> &a, float2 *v, int64_t row0, int64_t n2) {
  const int Q = 1 << a.log2Q;
  dft_half_in<P>(v);
  float2 *dst = a.inter + row0 + n2;
  // k1 = 8h + b, W^{k1} = W^{8h} W^b: table lookups for W, W^8, W^16, small powers by at most
  // two products, each factor applied and stored right away
  const float2 w1 = a.tw.root<false>((uint64_t)n2, a.log2M);
  const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1), w4 = cmul(w2, w2);
  float2 wh[4];
  wh[0] = make_float2(1.f, 0.f);
  if (P > 8) wh[1] = a.tw.root<false>(8 * (uint64_t)n2, a.log2M);
  if (P > 16) {
    wh[2] = a.tw.root<false>(16 * (uint64_t)n2, a.log2M);
    wh[3] = cmul(wh[2], wh[1]);
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int l = b & 3;
    float2 wb = (l == 0) ? make_float2(1.f, 0.f) : (l == 1 ? w1 : (l == 2 ? w2 : w3));
    if (b >= 4) wb = (l == 0) ? w4 : cmul(w4, wb);
#pragma unroll
    for (int h = 0; h < P / 8; ++h) {
      const int k1 = 8 * h + b;
      const float2 w = (h == 0) ? wb : (b == 0 ? wh[h] : cmul(wh[h], wb));
      dst[(int64_t)k1 * Q] = (k1 == 0) ? v[0] : cmul(v[k1], w);
    }
  }
}

// ---------------------------------------------------------------------------
// pass A without the correction (B y alone, or a = D o S_T^T y computed beforehand), real
// signals: tiles of FASTW_G pairs x FASTW_NB columns, so each warp load reads 256 contiguous
// bytes of a signal row; the tile is transposed through shared memory to one column per
// thread.  Persistent CTAs walk the tiles with two shared-memory buffers: the cp.async copies
// of the next tile are in flight while the current one is transformed, so the load latency
// is not exposed once per tile.
// grid: at most 3 CTAs per SM, FAST_THREADS threads (warp w -> pair w / 2, columns
// 32 (w & 1) + lane); dynamic shared memory fastw_smem(P).  Rows need 8-byte alignment.
// ---------------------------------------------------------------------------
constexpr int FASTW_NB = 64, FASTW_G = 4;
__host__ __device__ constexpr int fastw_tile_floats(int P) { return 2 * FASTW_G * (P / 2) * FASTW_NB; }
__host__ __device__ constexpr int fastw_smem(int P) { return 2 * fastw_tile_floats(P) * 4; }

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <int P>
__global__ void __launch_bounds__(FAST_THREADS, 3) k_fastAw(const ConvArgs<float> a) {
  constexpr int R = P / 2;   // rows n1 that can hold samples (M >= 2N)
  constexpr int TF = fastw_tile_floats(P);
  extern __shared__ __align__(16) float wtile[];
  const int Q = 1 << a.log2Q;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncol = Q / FASTW_NB;
  const int64_t ngrp = (a.npairs + FASTW_G - 1) / FASTW_G;
  const int64_t total = ngrp * ncol;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(wtile);
  // copies of tile t into buffer b: rows (signal s of 2 FASTW_G, n1), 64 floats, 8 bytes a lane;
  // samples past N or absent signals read as zero
  auto issue = [&](int64_t t, int b) {
    const int64_t g0 = (t / ncol) * FASTW_G;
    const int64_t col0 = (t % ncol) * FASTW_NB;
#pragma unroll
    for (int k = 0; k < 2 * FASTW_G * R / 8; ++k) {
      const int row = w + 8 * k;
      const int s = row / R, n1 = row % R;
      const int64_t sig = 2 * (a.pair0 + g0) + s;
      const int64_t n = (int64_t)n1 * Q + col0 + 2 * lane;
      int bytes = 0;
      const float *src = a.y;
      if (sig < a.batch && g0 + (s >> 1) < a.npairs && n1 < a.Pnz && n < a.N) {
        src = a.y + sig * a.ld + n;
        bytes = (n + 1 < a.N) ? 8 : 4;
      }
      cp_async8(sbase + (uint32_t)((b * TF + row * FASTW_NB + 2 * lane) * 4), src, bytes);
    }
  };
  int64_t t = blockIdx.x;
  if (t < total) issue(t, 0);
  cp_async_commit();
  for (int i = 0; t < total; ++i, t += gridDim.x) {
    const int64_t tn = t + gridDim.x;
    if (tn < total) issue(tn, (i + 1) & 1);
    cp_async_commit();
    cp_async_wait1();   // this thread's copies of tile t have landed
    __syncthreads();    // ... and everyone's
    const float *tb = wtile + (i & 1) * TF;
    const int64_t g0 = (t / ncol) * FASTW_G;
    const int64_t col0 = (t % ncol) * FASTW_NB;
    const int pl = w >> 1, c = 32 * (w & 1) + lane;
    float2 v[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) v[n1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int n1 = 0; n1 < R; ++n1)
      v[n1] = make_float2(tb[((2 * pl) * R + n1) * FASTW_NB + c], tb[((2 * pl + 1) * R + n1) * FASTW_NB + c]);
    __syncthreads();    // buffer i & 1 is refilled at the next iteration
    if (g0 + pl < a.npairs) fastA_finish<P>(a, v, (g0 + pl) * P * (int64_t)Q, col0 + c);
  }
}

// ---------------------------------------------------------------------------
// pass A: load columns, correction partials (tensor cores), P-point DFT, twiddle
// grid (ntiles, ngroups), FAST_THREADS threads; thread = (pair g = warp, column c = lane)
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(FAST_THREADS, 3) k_fastA(const FastArgs f) {
  const ConvArgs<float> &a = f.a;
  __shared__ __align__(16) float yt[2 * FAST_G * YT_STRIDE];   // [signal][n_local], n_local = n1 * 32 + c
  __shared__ float red[FAST_G][2 * FAST_G][8 * 3 + 1];         // per-warp partial C^T blocks
  const int Q = 1 << a.log2Q;
  const int g = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int64_t tile = blockIdx.x, g0 = (int64_t)blockIdx.y * FAST_G;
  const int64_t n2 = tile * FAST_NB + c;
  const bool live = (g0 + g) < a.npairs;
  const bool corr = a.mode == MODE_FULL && a.r > 0;

  float2 v[P];
#pragma unroll
  for (int i = 0; i < P; ++i) v[i] = make_float2(0.f, 0.f);
#pragma unroll
  for (int n1 = 0; n1 < P / 2; ++n1) {
    const int64_t n = (int64_t)n1 * Q + n2;
    if (live && n1 < a.Pnz && n < a.N) v[n1] = load_pair(a, g0 + g, n);
    if (corr) {
      yt[(2 * g) * YT_STRIDE + n1 * 32 + c] = v[n1].x;
      yt[(2 * g + 1) * YT_STRIDE + n1 * 32 + c] = v[n1].y;
    }
  }

  if (live) {
  fastA_finish<P>(a, v, (g0 + g) * P * (int64_t)Q, n2);
  }
  if (corr) {
    __syncthreads();
    // C^T (16 signals x rpad) = Y^T (16 x nel) * S (nel x rpad); warp w takes the
    // k-slice n_local in [w * nk, (w+1) * nk); the j range in n-tiles of 8
    const int lane = c, gid = lane >> 2, tig = lane & 3;
    const int nel = (P / 2) * 32;
    const int nk = nel / FAST_G;            // k per warp (multiple of 8)
    const int ntj = a.rpad / 8;             // j tiles of 8 (rpad multiple of 8)
    for (int jt0 = 0; jt0 < ntj; jt0 += 3) {
      float acc[3][4];
#pragma unroll
      for (int t = 0; t < 3; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < P / 4; ++ks) {   // nk / 8 = P / 4 k-steps per warp
        const int k0 = g * nk + ks * 8;
        uint32_t ahi[4], alo[4];
        split_tf32(yt[gid * YT_STRIDE + k0 + tig], ahi[0], alo[0]);
        split_tf32(yt[(gid + 8) * YT_STRIDE + k0 + tig], ahi[1], alo[1]);
        split_tf32(yt[gid * YT_STRIDE + k0 + tig + 4], ahi[2], alo[2]);
        split_tf32(yt[(gid + 8) * YT_STRIDE + k0 + tig + 4], ahi[3], alo[3]);
        // rows of S for n_local = k0 + tig and k0 + tig + 4
        const int nl0 = k0 + tig, nl1 = k0 + tig + 4;
        const int64_t nA = (int64_t)(nl0 >> 5) * Q + tile * FAST_NB + (nl0 & 31);
        const int64_t nB = (int64_t)(nl1 >> 5) * Q + tile * FAST_NB + (nl1 & 31);
        const bool okA = nA < a.N, okB = nB < a.N;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const int jt = jt0 + t;
          if (jt < ntj) {
            const int j = jt * 8 + gid;
            const float2 sa = okA ? __ldg(f.ST_hl + nA * a.rpad + j) : make_float2(0.f, 0.f);
            const float2 sb = okB ? __ldg(f.ST_hl + nB * a.rpad + j) : make_float2(0.f, 0.f);
            const uint32_t bhi[2] = {__float_as_uint(sa.x), __float_as_uint(sb.x)};
            const uint32_t blo[2] = {__float_as_uint(sa.y), __float_as_uint(sb.y)};
            mma3(acc[t], ahi, alo, bhi, blo);
          }
        }
      }
      // acc[t]: rows (signals) gid, gid+8; cols (j) 2 tig, 2 tig + 1 of tile jt0 + t
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        red[g][gid][t * 8 + 2 * tig] = acc[t][0];
        red[g][gid][t * 8 + 2 * tig + 1] = acc[t][1];
        red[g][gid + 8][t * 8 + 2 * tig] = acc[t][2];
        red[g][gid + 8][t * 8 + 2 * tig + 1] = acc[t][3];
      }
      __syncthreads();
      // sum over the 8 warps in a fixed order: thread -> (signal s, column jj)
      for (int t = threadIdx.x; t < 2 * FAST_G * 24; t += FAST_THREADS) {
        const int s = t / 24, jj = t % 24;
        const int j = jt0 * 8 + jj;
        const int gp = s >> 1;
        if (j < a.r && g0 + gp < a.npairs) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < FAST_G; ++w) sum += red[w][s][jj];
          const int ntiles = Q / FAST_NB;
          a.part[(((g0 + gp) * ntiles + tile) * 2 + (s & 1)) * a.rpad + j] = sum;
        }
      }
      __syncthreads();
    }
  }

}

// ---------------------------------------------------------------------------
// pass B for Q = 4096 = 16^3 (256 threads, 16 values per thread)
// grid (P, npairs)
// ---------------------------------------------------------------------------
// x[t] times W^{k t} (t = 1..15) from a [t][ldk] table (conjugated for the inverse):
// lanes with consecutive k read consecutive entries
// (COHERENT: plain loads, which the compiler keeps between the barriers around them; read-only
// cache loads may be hoisted over a whole transform and then spill in a kernel with several)
template <bool COHERENT = false>
__device__ __forceinline__ void tw_table16(const float2 *tab, int ldk, int k, bool inv, float2 *x) {
#pragma unroll
  for (int t = 1; t < 16; ++t) {
    const float2 w = COHERENT ? tab[t * ldk + k] : __ldg(tab + t * ldk + k);
    x[t] = inv ? make_float2(x[t].x * w.x + x[t].y * w.y, x[t].y * w.x - x[t].x * w.y) : cmul(x[t], w);
  }
}

// 4096-point row transforms with 256 threads x 16 values (buf: padded_size(4096) float2 of
// scratch; every thread of the block calls these, they contain barriers)
//   row4096_fwd: forward DFT of `row` (global) -> x[t] = X[j + 256 t] (natural order)
//   row4096_inv: inverse DFT of x[t] = Z[j + 256 t] -> x[t] = z[j + 256 t]
//   row4096_store: row[j + 256 t] = x[t] W_M^{-n2 k1}, n2 = j + 256 t
template <bool COHERENT = false, bool SMEM_IN = false>
__device__ __forceinline__ void row4096_fwd(const float2 *row, float2 *buf, const float2 *twB, int j, float2 *x) {
  constexpr int T = 256;
  // stage 1 (Ns = 1): inputs x[j + 256 t] straight from global memory (SMEM_IN: already copied
  // to buf[pad(n)], read before the stage's writes)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = SMEM_IN ? buf[pad(j + T * t)] : row[j + T * t];
  Dft<float, 16, false>::run(x);
  if (SMEM_IN) __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf[pad(16 * j + t)] = x[t];
  __syncthreads();
  // stage 2 (Ns = 16)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf[pad(j + T * t)];
  tw_table16<COHERENT>(twB, 16, j & 15, false, x);
  Dft<float, 16, false>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf[pad(((j >> 4) << 8) + (j & 15) + 16 * t)] = x[t];
  __syncthreads();
  // stage 3 (Ns = 256): outputs land at j + 256 t = natural k2
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf[pad(j + T * t)];
  tw_table16<COHERENT>(twB + 256, 256, j, false, x);
  Dft<float, 16, false>::run(x);
}
template <bool COHERENT = false>
__device__ __forceinline__ void row4096_inv(float2 *buf, const float2 *twB, int j, float2 *x) {
  constexpr int T = 256;
  // stage 1: its inputs x[j + 256 t] are already in registers
  Dft<float, 16, true>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf[pad(16 * j + t)] = x[t];
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf[pad(j + T * t)];
  tw_table16<COHERENT>(twB, 16, j & 15, true, x);
  Dft<float, 16, true>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf[pad(((j >> 4) << 8) + (j & 15) + 16 * t)] = x[t];
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf[pad(j + T * t)];
  tw_table16<COHERENT>(twB + 256, 256, j, true, x);
  Dft<float, 16, true>::run(x);
}
__device__ __forceinline__ void row4096_store(float2 *row, const Tw<float> &tw, int log2M, int k1, int j,
                                              const float2 *x) {
  constexpr int T = 256;
  const float2 wj = tw.root<true>((uint64_t)j * (uint64_t)k1, log2M);
  const float2 wstep = tw.root<true>((uint64_t)T * (uint64_t)k1, log2M);
  float2 wt = wj;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    row[j + T * t] = cmul(x[t], wt);
    if (t == 7) wt = cmul(wj, tw.root<true>((uint64_t)(8 * T) * (uint64_t)k1, log2M));
    else wt = cmul(wt, wstep);
  }
}

__global__ void __launch_bounds__(256, 4) k_fastB4096(const ConvArgs<float> a) {
  constexpr int Q = 4096, T = 256;
  __shared__ float2 buf[padded_size(Q)];
  const int P = 1 << a.log2P;
  const int k1 = blockIdx.x;
  const int64_t pl = blockIdx.y;
  float2 *row = a.inter + (pl * P + k1) * (int64_t)Q;
  const int j = threadIdx.x;
  if (k1 == 0 && a.mode == MODE_FULL && a.r > 0) {
    // a = D o (sum of the column-tile partials of S_T^T y), fixed order
    const int ntiles = Q / FAST_NB;
    for (int t = j; t < 2 * a.r; t += T) {
      const int c = t / a.r, jj = t % a.r;
      float sum = 0.f;
      for (int tile = 0; tile < ntiles; ++tile) sum += a.part[((pl * ntiles + tile) * 2 + c) * a.rpad + jj];
      a.acoef[(pl * 2 + c) * a.rpad + jj] = __ldg(a.D + jj) * sum;
    }
  }
  float2 x[16];
  row4096_fwd(row, buf, a.twB, j, x);
  if (a.mode == MODE_FORWARD) {
#pragma unroll
    for (int t = 0; t < 16; ++t) row[j + T * t] = x[t];
    return;
  }
  const float *sp = spec_of(a, pl) + (int64_t)k1 * Q;
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = cscale(x[t], __ldg(sp + j + T * t));
  row4096_inv(buf, a.twB, j, x);
  row4096_store(row, a.tw, a.log2M, k1, j, x);
}

// ---------------------------------------------------------------------------
// pass B of a ragged slot holding two real signals with different spectra Ca, Cb (their own
// plans, same FFT length).  With x = ya + i yb, X = FFT(x): Ya = (X[k] + conj X[-k]) / 2,
// i Yb = (X[k] - conj X[-k]) / 2, so the filtered spectrum Ca Ya + i Cb Yb is
//   Z[k] = (Ca + Cb)/2 X[k] + (Ca - Cb)/2 conj X[-k],
// and IFFT(Z) = (B_a ya) + i (B_b yb) (Ca, Cb real and even).  For k = k1 + P k2 the index -k
// lies in row P - k1, column Q - 1 - k2 (row 0: column (Q - k2) mod Q).  A CTA takes rows
// r0 = blockIdx.x and r1 = P - r0 (rows 0 and P/2 pair with themselves): both rows' inputs are
// copied into shared memory with cp.async up front (the second row's load overlaps the first
// row's transform), both forward transforms land in shared memory, each thread then forms Z for
// an index and its mirror in
// place (the map k2 -> Q - 1 - k2 pairs the two buffers one to one), and the two inverse
// transforms follow one after the other.
// grid (P/2 + 1, slots), 256 threads, dynamic shared memory 2 padded_size(4096) float2.
// ---------------------------------------------------------------------------
constexpr size_t fastb2s_smem() { return 2 * (size_t)padded_size(4096) * sizeof(float2); }
__device__ __forceinline__ float2 two_spec_z(float2 xk, float2 xm, float ca, float cb) {
  const float A = 0.5f * (ca + cb), Bm = 0.5f * (ca - cb);
  return make_float2(A * xk.x + Bm * xm.x, A * xk.y - Bm * xm.y);
}
__global__ void __launch_bounds__(256, 3) k_fastB4096_2s(const ConvArgs<float> a) {
  constexpr int Q = 4096, T = 256;
  extern __shared__ __align__(16) float2 b2s[];
  float2 *buf0 = b2s, *buf1 = b2s + padded_size(Q);
  const int P = 1 << a.log2P;
  const int r0 = blockIdx.x, r1 = (P - r0) & (P - 1);
  const int64_t pl = blockIdx.y;
  const int j = threadIdx.x;
  const RPair<float> &q = a.rp[a.pair0 + pl];
  const float *ca = q.spec, *cb = q.spec2 ? q.spec2 : q.spec;
  float2 *row0 = a.inter + (pl * P + r0) * (int64_t)Q;
  float2 *row1 = a.inter + (pl * P + r1) * (int64_t)Q;
  // both rows' inputs in flight at once: 8-byte copies into the padded layout
  {
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(buf0), s1 = (uint32_t)__cvta_generic_to_shared(buf1);
#pragma unroll
    for (int t = 0; t < 16; ++t) cp_async8(s0 + (uint32_t)(pad(j + T * t) * 8), row0 + j + T * t);
    cp_async_commit();
    if (r1 != r0) {
#pragma unroll
      for (int t = 0; t < 16; ++t) cp_async8(s1 + (uint32_t)(pad(j + T * t) * 8), row1 + j + T * t);
    }
    cp_async_commit();
  }
  cp_async_wait1();
  __syncthreads();
  float2 x[16];
  row4096_fwd<true, true>(row0, buf0, a.twB, j, x);
  __syncthreads();   // the last stage's reads of buf0 are done
#pragma unroll
  for (int t = 0; t < 16; ++t) buf0[pad(j + T * t)] = x[t];
  if (r1 == r0) {
    __syncthreads();
    const float *sa = ca + (int64_t)r0 * Q, *sb = cb + (int64_t)r0 * Q;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int k2 = j + T * t;
      const int m = (r0 == 0) ? ((Q - k2) & (Q - 1)) : (Q - 1 - k2);
      x[t] = two_spec_z(x[t], buf0[pad(m)], __ldg(sa + k2), __ldg(sb + k2));
    }
    row4096_inv<true>(buf0, a.twB, j, x);   // begins with a barrier: every mirror read is done
    row4096_store(row0, a.tw, a.log2M, r0, j, x);
    return;
  }
  cp_async_wait0();
  __syncthreads();
  row4096_fwd<true, true>(row1, buf1, a.twB, j, x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf1[pad(j + T * t)] = x[t];
  __syncthreads();
  {
    const float *sa0 = ca + (int64_t)r0 * Q, *sb0 = cb + (int64_t)r0 * Q;
    const float *sa1 = ca + (int64_t)r1 * Q, *sb1 = cb + (int64_t)r1 * Q;
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
      const int k2 = j + T * t, m = Q - 1 - k2;
      const float2 x0 = buf0[pad(k2)], x1 = buf1[pad(m)];
      buf0[pad(k2)] = two_spec_z(x0, x1, __ldg(sa0 + k2), __ldg(sb0 + k2));
      buf1[pad(m)] = two_spec_z(x1, x0, __ldg(sa1 + m), __ldg(sb1 + m));
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf0[pad(j + T * t)];
  row4096_inv<true>(buf0, a.twB, j, x);
  row4096_store(row0, a.tw, a.log2M, r0, j, x);
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf1[pad(j + T * t)];
  row4096_inv<true>(buf1, a.twB, j, x);
  row4096_store(row1, a.tw, a.log2M, r1, j, x);
}

// ---------------------------------------------------------------------------
// pass B for Q = 8192 = 16^3 x 2 (512 threads, 16 values per thread), no fused reduce
// grid (P, npairs).  Stockham stages (radix R at sub-length Ns, butterfly j reads
// x[j + t Q/R], twiddles by W_{Ns R}^{(j mod Ns) t}, writes y[(j/Ns) Ns R + j mod Ns + t Ns]):
//   forward  R16 Ns=1 (from global), R16 Ns=16, R16 Ns=256, R2 Ns=4096 (natural order out,
//            8 butterflies per thread at j = tid + 512 q: values at j and j + 4096)
//   spectrum in registers
//   inverse  R2 Ns=1 (same positions), R16 Ns=2, R16 Ns=32, R16 Ns=512 (natural order out)
// tw8: W_8192^j (j < 4096), then [t][k] W_32^{k t} (k < 2), [t][k] W_512^{k t} (k < 32),
//      [t][k] W_8192^{k t} (k < 512), t < 16
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(512, 2) k_fastB8192(const ConvArgs<float> a, const float2 *tw8) {
  constexpr int Q = 8192, T = 512;
  extern __shared__ __align__(16) float2 buf8[];
  const int P = 1 << a.log2P;
  const int k1 = blockIdx.x;
  const int64_t pl = blockIdx.y;
  float2 *row = a.inter + (pl * P + k1) * (int64_t)Q;
  const int j = threadIdx.x;
  float2 x[16];
  // forward stage 1 (R16, Ns = 1): inputs x[j + 512 t] from global
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = row[j + T * t];
  Dft<float, 16, false>::run(x);
#pragma unroll
  for (int t = 0; t < 16; ++t) buf8[pad(16 * j + t)] = x[t];
  __syncthreads();
  // stage 2 (R16, Ns = 16)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf8[pad(j + T * t)];
  tw_table16(a.twB, 16, j & 15, false, x);
  Dft<float, 16, false>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf8[pad(((j >> 4) << 8) + (j & 15) + 16 * t)] = x[t];
  __syncthreads();
  // stage 3 (R16, Ns = 256)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf8[pad(j + T * t)];
  tw_table16(a.twB + 256, 256, j & 255, false, x);
  Dft<float, 16, false>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf8[pad(((j >> 8) << 12) + (j & 255) + 256 * t)] = x[t];
  __syncthreads();
  // stage 4 (R2, Ns = 4096): butterflies jq = j + 512 q, values at jq (x[2q]) and jq + 4096 (x[2q+1])
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int jq = j + T * q;
    const float2 u0 = buf8[pad(jq)];
    const float2 u1 = cmul(buf8[pad(jq + 4096)], __ldg(tw8 + TW8_R2 + jq));
    x[2 * q] = cadd(u0, u1);
    x[2 * q + 1] = csub(u0, u1);
  }
  if (a.mode == MODE_FORWARD) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      row[j + T * q] = x[2 * q];
      row[j + T * q + 4096] = x[2 * q + 1];
    }
    return;
  }
  const float *sp = spec_of(a, pl) + (int64_t)k1 * Q;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    x[2 * q] = cscale(x[2 * q], __ldg(sp + j + T * q));
    x[2 * q + 1] = cscale(x[2 * q + 1], __ldg(sp + j + T * q + 4096));
  }
  // inverse stage 1 (R2, Ns = 1): butterflies jq read x[jq], x[jq + 4096] (in registers) and
  // write y[2 jq], y[2 jq + 1]
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int jq = j + T * q;
    buf8[pad(2 * jq)] = cadd(x[2 * q], x[2 * q + 1]);
    buf8[pad(2 * jq + 1)] = csub(x[2 * q], x[2 * q + 1]);
  }
  __syncthreads();
  // inverse stage 2 (R16, Ns = 2)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf8[pad(j + T * t)];
  tw_table16(tw8 + TW8_32, 2, j & 1, true, x);
  Dft<float, 16, true>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf8[pad(((j >> 1) << 5) + (j & 1) + 2 * t)] = x[t];
  __syncthreads();
  // inverse stage 3 (R16, Ns = 32)
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf8[pad(j + T * t)];
  tw_table16(tw8 + TW8_512, 32, j & 31, true, x);
  Dft<float, 16, true>::run(x);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) buf8[pad(((j >> 5) << 9) + (j & 31) + 32 * t)] = x[t];
  __syncthreads();
  // inverse stage 4 (R16, Ns = 512): outputs at j + 512 t = natural n2
#pragma unroll
  for (int t = 0; t < 16; ++t) x[t] = buf8[pad(j + T * t)];
  tw_table16(tw8 + TW8_8192, 512, j, true, x);
  Dft<float, 16, true>::run(x);
  // times W_M^{-n2 k1}, n2 = j + 512 t, straight to global memory
  const float2 wj = a.tw.root<true>((uint64_t)j * (uint64_t)k1, a.log2M);
  const float2 wstep = a.tw.root<true>((uint64_t)T * (uint64_t)k1, a.log2M);
  float2 wt = wj;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    row[j + T * t] = cmul(x[t], wt);
    if (t == 7) wt = cmul(wj, a.tw.root<true>((uint64_t)(8 * T) * (uint64_t)k1, a.log2M));
    else wt = cmul(wt, wstep);
  }
}
__host__ __device__ constexpr int fastb8192_smem() { return padded_size(8192) * 8; }

// ---------------------------------------------------------------------------
// pass C: load columns, inverse P-point DFT, correction epilogue (tensor cores), store
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(FAST_THREADS, 3) k_fastC(const FastArgs f) {
  const ConvArgs<float> &a = f.a;
  __shared__ __align__(16) float zt[(P / 2) * 32][2 * FAST_G + 1];   // Z tile [n_local][signal]
  __shared__ float acs[2][32][2 * FAST_G + 1];                        // a (hi, lo) [j][signal]
  const int Q = 1 << a.log2Q;
  const int g = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int64_t tile = blockIdx.x, g0 = (int64_t)blockIdx.y * FAST_G;
  const int64_t n2 = tile * FAST_NB + c;
  const bool live = (g0 + g) < a.npairs;
  const bool corr = (a.mode == MODE_FULL || a.mode == MODE_ZONLY) && a.r > 0;

  if (corr) {
    const int lane = c, gid = lane >> 2, tig = lane & 3;
    const int nel = (P / 2) * 32;
    const int ntj = a.rpad / 8;
    for (int jt0 = 0; jt0 < ntj; jt0 += 4) {
      // a (coefficients D o c) for j in [8 jt0, 8 jt0 + 32), all 16 signals, split hi/lo
      for (int t = threadIdx.x; t < 32 * 2 * FAST_G; t += FAST_THREADS) {
        const int jj = t / (2 * FAST_G), s = t % (2 * FAST_G);
        const int j = jt0 * 8 + jj, gp = s >> 1;
        float val = 0.f;
        if (j < a.r && g0 + gp < a.npairs) val = a.acoef[((g0 + gp) * 2 + (s & 1)) * a.rpad + j];
        uint32_t hi, lo;
        split_tf32(val, hi, lo);
        acs[0][jj][s] = __uint_as_float(hi);
        acs[1][jj][s] = __uint_as_float(lo);
      }
      __syncthreads();
      // Z (nel x 16) = S (nel x 32 j) * A (32 j x 16); warp w takes m-tiles of 16 rows
#pragma unroll
      for (int mi = 0; mi < P / 8; ++mi) {
        const int mt = g + FAST_G * mi;
        float acc[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
        const int nl0 = mt * 16 + gid, nl1 = nl0 + 8;
        const int64_t nA = (int64_t)(nl0 >> 5) * Q + tile * FAST_NB + (nl0 & 31);
        const int64_t nB = (int64_t)(nl1 >> 5) * Q + tile * FAST_NB + (nl1 & 31);
        const bool okA = nA < a.N, okB = nB < a.N;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
          const int jt = jt0 + kt;
          if (jt < ntj) {
            const int j0 = jt * 8 + tig, j1 = j0 + 4;
            const float2 z2 = make_float2(0.f, 0.f);
            const float2 s0 = okA ? __ldg(f.ST_hl + nA * a.rpad + j0) : z2;
            const float2 s1 = okB ? __ldg(f.ST_hl + nB * a.rpad + j0) : z2;
            const float2 s2 = okA ? __ldg(f.ST_hl + nA * a.rpad + j1) : z2;
            const float2 s3 = okB ? __ldg(f.ST_hl + nB * a.rpad + j1) : z2;
            const uint32_t ahi[4] = {__float_as_uint(s0.x), __float_as_uint(s1.x), __float_as_uint(s2.x),
                                     __float_as_uint(s3.x)};
            const uint32_t alo[4] = {__float_as_uint(s0.y), __float_as_uint(s1.y), __float_as_uint(s2.y),
                                     __float_as_uint(s3.y)};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              // B (8 j x 8 signals): b0 = A[j = kt*8 + tig][s = u*8 + gid], b1 = A[j + 4][s]
              uint32_t bhi[2], blo[2];
              bhi[0] = __float_as_uint(acs[0][kt * 8 + tig][u * 8 + gid]);
              bhi[1] = __float_as_uint(acs[0][kt * 8 + tig + 4][u * 8 + gid]);
              blo[0] = __float_as_uint(acs[1][kt * 8 + tig][u * 8 + gid]);
              blo[1] = __float_as_uint(acs[1][kt * 8 + tig + 4][u * 8 + gid]);
              mma3(acc[u], ahi, alo, bhi, blo);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float add0 = (jt0 == 0) ? 0.f : zt[nl0][u * 8 + 2 * tig];
          const float add1 = (jt0 == 0) ? 0.f : zt[nl0][u * 8 + 2 * tig + 1];
          const float add2 = (jt0 == 0) ? 0.f : zt[nl1][u * 8 + 2 * tig];
          const float add3 = (jt0 == 0) ? 0.f : zt[nl1][u * 8 + 2 * tig + 1];
          zt[nl0][u * 8 + 2 * tig] = add0 + acc[u][0];
          zt[nl0][u * 8 + 2 * tig + 1] = add1 + acc[u][1];
          zt[nl1][u * 8 + 2 * tig] = add2 + acc[u][2];
          zt[nl1][u * 8 + 2 * tig + 1] = add3 + acc[u][3];
        }
      }
      __syncthreads();
    }
  }

  if (!live) return;
  float2 o[P / 2];   // inverse DFT outputs n1 < P/2 (M >= 2N: no output in the other rows)
  {
    const float2 *src = a.inter + ((g0 + g) * P) * (int64_t)Q + n2;
    float2 v[P];
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) v[k1] = src[(int64_t)k1 * Q];
    idft_half_out<P>(v, o);
  }
#pragma unroll
  for (int n1 = 0; n1 < P / 2; ++n1) {
    const int64_t n = (int64_t)n1 * Q + n2;
    if (n1 < a.Pnz && n < a.N) {
      float2 val = o[n1];
      if (corr) {
        val.x += zt[n1 * 32 + c][2 * g];
        val.y += zt[n1 * 32 + c][2 * g + 1];
      }
      store_pair(a, g0 + g, n, val);
    }
  }
}

}  // namespace fst

namespace fst {

// ---------------------------------------------------------------------------
// Standalone rank-r correction with mma.sync, for FP32 batches whose signal rows no TMA
// tensor map can address (otherwise the tcgen05 kernel computes S_T^T y): the same
// tensor-core products as the fast column kernels, on contiguous row blocks of CORR_ROWS
// samples:
//   k_corr_c : partial S_T^T y per (pair group, row block)   (before pass C)
//   k_corr_z : out += S_T (D o c) per (pair group, row block) (after pass C)
// ---------------------------------------------------------------------------


template <typename T> __device__ __forceinline__ void add_pair(const ConvArgs<T> &a, int64_t pl, int64_t n, c2<T> z) {
  const int64_t p = a.pair0 + pl;
  if (a.cplx) {
    c2<T> *o = reinterpret_cast<c2<T> *>(a.out) + p * a.ld + n;
    c2<T> v = *o;
    v.x += z.x;
    v.y += z.y;
    *o = v;
    return;
  }
  const int64_t s0 = 2 * p, s1 = 2 * p + 1;
  a.out[s0 * a.ld + n] += z.x;
  if (s1 < a.batch) a.out[s1 * a.ld + n] += z.y;
}

__global__ void __launch_bounds__(FAST_THREADS, 2) k_corr_c(const FastArgs f) {
  const ConvArgs<float> &a = f.a;
  // one buffer: the signal-major tile during the products, the per-warp results after
  constexpr int RED_STRIDE = 65;
  constexpr int BUF = (2 * FAST_G * YT_STRIDE > FAST_G * 2 * FAST_G * RED_STRIDE) ? 2 * FAST_G * YT_STRIDE
                                                                                  : FAST_G * 2 * FAST_G * RED_STRIDE;
  __shared__ __align__(16) float buf[BUF];
  float *yt = buf;
  const int nK = (int)((a.N + CORR_BLOCK - 1) / CORR_BLOCK);
  const int64_t blk = blockIdx.x, g0 = (int64_t)blockIdx.y * FAST_G;
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int nk = CORR_ROWS / FAST_G;   // 64 rows per warp and tile
  const int ntj = a.rpad / 8;
  for (int jt0 = 0; jt0 < ntj; jt0 += 8) {
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    for (int sub = 0; sub < CORR_BLOCK / CORR_ROWS; ++sub) {
      const int64_t n0 = blk * CORR_BLOCK + (int64_t)sub * CORR_ROWS;
      __syncthreads();
      // yt[s][k] = signal s (pair s/2, part s%2) at sample n0 + k
      for (int e = threadIdx.x; e < FAST_G * CORR_ROWS; e += FAST_THREADS) {
        const int gg = e / CORR_ROWS, k = e % CORR_ROWS;
        const int64_t n = n0 + k;
        float2 v = make_float2(0.f, 0.f);
        if (g0 + gg < a.npairs && n < a.N) v = load_pair(a, g0 + gg, n);
        yt[(2 * gg) * YT_STRIDE + k] = v.x;
        yt[(2 * gg + 1) * YT_STRIDE + k] = v.y;
      }
      __syncthreads();
#pragma unroll 2
      for (int ks = 0; ks < nk / 8; ++ks) {
        const int k0 = g * nk + ks * 8;
        uint32_t ahi[4], alo[4];
        split_tf32(yt[gid * YT_STRIDE + k0 + tig], ahi[0], alo[0]);
        split_tf32(yt[(gid + 8) * YT_STRIDE + k0 + tig], ahi[1], alo[1]);
        split_tf32(yt[gid * YT_STRIDE + k0 + tig + 4], ahi[2], alo[2]);
        split_tf32(yt[(gid + 8) * YT_STRIDE + k0 + tig + 4], ahi[3], alo[3]);
        const int64_t nA = n0 + k0 + tig, nB = nA + 4;
        const bool okA = nA < a.N, okB = nB < a.N;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int jt = jt0 + t;
          if (jt < ntj) {
            const int j = jt * 8 + gid;
            const float2 sa = okA ? __ldg(f.ST_hl + nA * a.rpad + j) : make_float2(0.f, 0.f);
            const float2 sb = okB ? __ldg(f.ST_hl + nB * a.rpad + j) : make_float2(0.f, 0.f);
            const uint32_t bhi[2] = {__float_as_uint(sa.x), __float_as_uint(sb.x)};
            const uint32_t blo[2] = {__float_as_uint(sa.y), __float_as_uint(sb.y)};
            mma3(acc[t], ahi, alo, bhi, blo);
          }
        }
      }
    }
    __syncthreads();
    float *red = buf;   // [warp][signal][64 j]
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float *r0 = red + (g * 2 * FAST_G + gid) * RED_STRIDE + t * 8 + 2 * tig;
      float *r1 = red + (g * 2 * FAST_G + gid + 8) * RED_STRIDE + t * 8 + 2 * tig;
      r0[0] = acc[t][0];
      r0[1] = acc[t][1];
      r1[0] = acc[t][2];
      r1[1] = acc[t][3];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * FAST_G * 64; t += FAST_THREADS) {
      const int sgl = t / 64, jj = t % 64;
      const int j = jt0 * 8 + jj, gp = sgl >> 1;
      if (j < a.r && g0 + gp < a.npairs) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < FAST_G; ++w) sum += red[(w * 2 * FAST_G + sgl) * RED_STRIDE + jj];
        a.part[(((g0 + gp) * nK + blk) * 2 + (sgl & 1)) * a.rpad + j] = sum;
      }
    }
  }
}

// a[pair][c][j] = scale_j * sum over row blocks of the partials: warp per output,
// lanes stride the blocks, fixed xor-tree across lanes (deterministic)
// grid (pairs, ceil(2 r / warps)): one warp per (pair, component, j), lanes over the blocks
__global__ void k_corr_reduce(const ConvArgs<float> a, const float *scale) {
  const int nK = a.nkb;
  const int64_t pl = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = blockIdx.y * nw + w; t < 2 * a.r; t += nw * gridDim.y) {
    const int c = t / a.r, j = t % a.r;
    float s = 0.f;
    for (int b = lane; b < nK; b += 32) s += a.part[((pl * nK + b) * 2 + c) * a.rpad + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.acoef[(pl * 2 + c) * a.rpad + j] = __ldg(scale + j) * s;
  }
}

// ---------------------------------------------------------------------------
// out += S_T a for every signal (the last step of the separate correction, a = D o S_T^T y
// already summed): r <= RMAX FP32 FMAs per output value, on CUDA cores.
// A block takes ZR_N consecutive samples and ZR_ROWS rows of a (real signals, or the (re, im)
// rows of ZR_ROWS / 2 complex signals).  The S_T rows of its samples are contiguous in memory:
// staged through shared memory with coalesced loads, then each thread keeps the row of its
// sample in registers and walks half of the a rows (read as shared-memory broadcasts),
// adding into out.  grid (ceil(N / ZR_N), ceil(rows / ZR_ROWS)), ZR_THREADS threads.
// ---------------------------------------------------------------------------
template <int RMAX>
__global__ void __launch_bounds__(ZR_THREADS) k_z_rmw(const ConvArgs<float> a, const float *ST) {
  __shared__ float st[ZR_N][RMAX + 1];
  __shared__ float as[ZR_ROWS][RMAX];
  const int r = a.r;
  const int64_t n0 = (int64_t)blockIdx.x * ZR_N;
  const int nsig = a.cplx ? ZR_ROWS / 2 : ZR_ROWS;
  const int64_t sig0 = (int64_t)blockIdx.y * nsig;
  // S_T rows n0 .. n0 + ZR_N - 1: ZR_N x rpad contiguous floats (rpad <= RMAX)
  const int64_t nn = (a.N - n0 < ZR_N) ? a.N - n0 : ZR_N;
  for (int t = threadIdx.x; t < ZR_N * a.rpad; t += ZR_THREADS) {
    const int row = t / a.rpad, j = t % a.rpad;
    st[row][j] = (row < nn && j < r) ? __ldg(ST + n0 * a.rpad + t) : 0.f;
  }
  for (int t = threadIdx.x; t < ZR_N * (RMAX - a.rpad); t += ZR_THREADS) {
    const int row = t / (RMAX - a.rpad), j = a.rpad + t % (RMAX - a.rpad);
    st[row][j] = 0.f;
  }
  // a rows: real signal sig0 + rr; complex signal sig0 + rr / 2, part rr & 1.  The rows of
  // acoef are (pair 2 + part); for real signals that index is the signal itself.
  for (int t = threadIdx.x; t < ZR_ROWS * RMAX; t += ZR_THREADS) {
    const int rr = t / RMAX, j = t % RMAX;
    const int64_t sg = a.cplx ? sig0 + rr / 2 : sig0 + rr;
    const int64_t arow = a.cplx ? 2 * sg + (rr & 1) : sg;
    as[rr][j] = (sg < a.batch && j < r) ? a.acoef[arow * a.rpad + j] : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x % ZR_N, half = threadIdx.x / ZR_N;
  const int64_t n = n0 + i;
  if (n >= a.N) return;
  float sv[RMAX];
#pragma unroll
  for (int j = 0; j < RMAX; ++j) sv[j] = st[i][j];
  if (!a.cplx) {
    const int rows = (int)(a.batch - sig0 < ZR_ROWS ? a.batch - sig0 : ZR_ROWS);
    for (int rr = half; rr < rows; rr += 2) {
      float z = 0.f;
#pragma unroll
      for (int j = 0; j < RMAX; ++j) z = fmaf(sv[j], as[rr][j], z);
      a.out[(sig0 + rr) * a.ld + n] += z;
    }
  } else {
    const int sigs = (int)(a.batch - sig0 < ZR_ROWS / 2 ? a.batch - sig0 : ZR_ROWS / 2);
    for (int q = half; q < sigs; q += 2) {
      float zr = 0.f, zi = 0.f;
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        zr = fmaf(sv[j], as[2 * q][j], zr);
        zi = fmaf(sv[j], as[2 * q + 1][j], zi);
      }
      float2 *o = reinterpret_cast<float2 *>(a.out) + (sig0 + q) * a.ld + n;
      float2 v = *o;
      v.x += zr;
      v.y += zi;
      *o = v;
    }
  }
}

// ---------------------------------------------------------------------------
// out += S_T a over the whole batch on CUDA cores (rpad <= 64): a block of ZA_THREADS threads
// takes ns = ZA_THREADS / ng samples and up to 16 ng signal rows (ng = ceil(rows / 16), at
// most 8: real signals, or the (re, im) rows of complex ones; row b of a is acoef row b).  The
// block's S_T rows are staged once in shared memory, [sample][j] with a 16-byte aligned odd
// stride (conflict-free float4 reads), and its a rows transposed to [j][row] (float4
// broadcasts).  Thread (sample i, row group g) keeps ZA_RG sums in registers: per 4 j, one
// float4 of S and ZA_RG / 4 float4 of a feed 4 ZA_RG FMAs.  Then the sums are added into out
// (coalesced along the samples).
// 1-D grid of ceil(N / ns) x (row blocks) blocks, block b = sample block b / nrb, row block
// b % nrb: the row blocks of the same samples run side by side, so their S_T rows come from L2.
// ---------------------------------------------------------------------------
constexpr int ZA_THREADS = 256, ZA_RG = 16, ZA_ROWS = 128;
// row groups per block: ceil(rows / 16) rounded up to a power of two, at most 8, so that
// ZA_THREADS / ng samples times ng groups is exactly the block
__host__ __device__ inline int za_groups(int64_t rows) {
  int g = 1;
  while (g < ZA_ROWS / ZA_RG && (int64_t)g * ZA_RG < rows) g *= 2;
  return g;
}
__host__ __device__ inline int za_smem(int rpad, int ng) {
  return ((ZA_THREADS / ng) * (rpad + 4) + rpad * (ng * ZA_RG + 4)) * 4;
}

__global__ void __launch_bounds__(ZA_THREADS) k_zadd(const ConvArgs<float> a) {
  extern __shared__ __align__(16) float zsm[];
  const int rpad = a.rpad, sst = rpad + 4;
  const int64_t rows = a.cplx ? 2 * a.batch : a.batch;
  const int ng = za_groups(rows), ns = ZA_THREADS / ng, brows = ng * ZA_RG, ast = brows + 4;
  float *st = zsm;                        // [ns][sst]
  float *as = zsm + ns * sst;             // [rpad][ast]
  const int64_t nrb = (rows + brows - 1) / brows;
  const int64_t row0 = ((int64_t)blockIdx.x % nrb) * brows;
  const int nrow = (int)(rows - row0 < brows ? rows - row0 : brows);
  const int64_t n0 = ((int64_t)blockIdx.x / nrb) * ns;
  // S_T rows n0 .. n0 + ns - 1 (zero past N)
  for (int e = threadIdx.x; e < ns * (rpad / 4); e += ZA_THREADS) {
    const int i = e / (rpad / 4), q = e % (rpad / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n0 + i < a.N) v = __ldg(reinterpret_cast<const float4 *>(a.ST + (n0 + i) * rpad) + q);
    *reinterpret_cast<float4 *>(st + i * sst + 4 * q) = v;
  }
  // a rows of this block, transposed: as[j][row]
  for (int e = threadIdx.x; e < rpad * brows; e += ZA_THREADS) {
    const int rr = e / rpad, j = e % rpad;
    as[j * ast + rr] = (rr < nrow && j < a.r) ? a.acoef[(row0 + rr) * rpad + j] : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x % ns, g = threadIdx.x / ns;
  const int64_t n = n0 + i;
  float acc[ZA_RG];
#pragma unroll
  for (int q = 0; q < ZA_RG; ++q) acc[q] = 0.f;
  const float *srow = st + i * sst;
  const float *acol = as + g * ZA_RG;
  for (int j = 0; j < rpad; j += 4) {
    const float4 s4 = *reinterpret_cast<const float4 *>(srow + j);
#pragma unroll
    for (int q = 0; q < ZA_RG; q += 4) {
      const float4 a0 = *reinterpret_cast<const float4 *>(acol + (j + 0) * ast + q);
      const float4 a1 = *reinterpret_cast<const float4 *>(acol + (j + 1) * ast + q);
      const float4 a2 = *reinterpret_cast<const float4 *>(acol + (j + 2) * ast + q);
      const float4 a3 = *reinterpret_cast<const float4 *>(acol + (j + 3) * ast + q);
      acc[q + 0] = fmaf(s4.w, a3.x, fmaf(s4.z, a2.x, fmaf(s4.y, a1.x, fmaf(s4.x, a0.x, acc[q + 0]))));
      acc[q + 1] = fmaf(s4.w, a3.y, fmaf(s4.z, a2.y, fmaf(s4.y, a1.y, fmaf(s4.x, a0.y, acc[q + 1]))));
      acc[q + 2] = fmaf(s4.w, a3.z, fmaf(s4.z, a2.z, fmaf(s4.y, a1.z, fmaf(s4.x, a0.z, acc[q + 2]))));
      acc[q + 3] = fmaf(s4.w, a3.w, fmaf(s4.z, a2.w, fmaf(s4.y, a1.w, fmaf(s4.x, a0.w, acc[q + 3]))));
    }
  }
  if (n >= a.N) return;
  if (!a.cplx) {
#pragma unroll
    for (int q = 0; q < ZA_RG; ++q) {
      const int rr = g * ZA_RG + q;
      if (rr < nrow) a.out[(row0 + rr) * a.ld + n] += acc[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < ZA_RG; q += 2) {
      const int rr = g * ZA_RG + q;
      if (rr < nrow) {
        float2 *o = reinterpret_cast<float2 *>(a.out) + ((row0 + rr) >> 1) * a.ld + n;
        float2 v = *o;
        v.x += acc[q];
        v.y += acc[q + 1];
        *o = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// S_T^T y for small batches (at most CC_ROWS signal rows: real signals, or the (re, im) rows
// of complex ones) on CUDA cores, in FP32: the MMA tile of the tensor-core kernel would be
// mostly empty there and each k-tile's fixed cost dominates.  A block takes CORR_BLOCK
// samples in sub-chunks of CC_SUB; y (transposed to [sample][row]) and S_T ([sample][j]) of
// a sub-chunk are staged in shared memory.  Thread (row group of 4, j group of 8, sample
// slice s) keeps 32 sums; per sample one float4 of y and two of S feed 32 FMAs.  The slices
// are summed in a fixed order at the end and one partial per (pair, block, part, j) is
// written, the layout k_corr_reduce reads (nkb = ceil(N / CORR_BLOCK)).
// grid ceil(N / CORR_BLOCK), CC_THREADS threads, dynamic shared memory cc_smem(rpad).
// ---------------------------------------------------------------------------
constexpr int CC_ROWS = 32, CC_SUB = 128, CC_THREADS = 256;
// staging area: y [CC_SUB][CC_ROWS + 4] and S_T [CC_SUB][rpad + 4]; at the end it holds the
// slice sums [CC_THREADS][33]
__host__ __device__ constexpr int cc_smem(int rpad) {
  return ((CC_SUB * (CC_ROWS + 4) + CC_SUB * (rpad + 4)) > CC_THREADS * 33
              ? (CC_SUB * (CC_ROWS + 4) + CC_SUB * (rpad + 4))
              : CC_THREADS * 33) * 4;
}

__global__ void __launch_bounds__(CC_THREADS) k_corr_cc(const ConvArgs<float> a) {
  extern __shared__ __align__(16) float csm2[];
  const int rpad = a.rpad, sst = rpad + 4;
  constexpr int YST = CC_ROWS + 4;
  float *yt = csm2;                     // [CC_SUB][YST]
  float *st = csm2 + CC_SUB * YST;      // [CC_SUB][sst]
  const int rows = (int)(a.cplx ? 2 * a.batch : a.batch);
  const int nrg = (rows + 3) / 4, njg = rpad / 8;
  const int combos = nrg * njg;
  const int nslice = CC_THREADS / combos;            // host guarantees combos <= CC_THREADS
  const int tid = threadIdx.x;
  const int combo = tid % combos, slice = tid / combos;
  const bool active = slice < nslice;
  const int rg = combo % nrg, jg = combo / nrg;
  const int64_t blk = blockIdx.x;
  float acc[4][8];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  for (int sub = 0; sub < CORR_BLOCK / CC_SUB; ++sub) {
    const int64_t n0 = blk * CORR_BLOCK + (int64_t)sub * CC_SUB;
    if (n0 >= a.N) break;
    __syncthreads();
    // S_T rows by cp.async (zero past N), y rows (the 4 nrg rows used; zero past N and past the
    // last row) transposed through registers meanwhile
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(st);
    for (int e = tid; e < CC_SUB * (rpad / 4); e += CC_THREADS) {
      const int i = e / (rpad / 4), q = e % (rpad / 4);
      const bool ok = n0 + i < a.N;
      cp_async16(sbase + (uint32_t)((i * sst + 4 * q) * 4), ok ? a.ST + (n0 + i) * rpad + 4 * q : a.ST, ok ? 16 : 0);
    }
    cp_async_commit();
    for (int e = tid; e < 4 * nrg * CC_SUB; e += CC_THREADS) {
      const int row = e / CC_SUB, i = e % CC_SUB;
      const int64_t n = n0 + i;
      float v = 0.f;
      if (row < rows && n < a.N) {
        if (!a.cplx) v = a.y[(int64_t)row * a.ld + n];
        else v = a.y[((int64_t)(row >> 1) * a.ld + n) * 2 + (row & 1)];
      }
      yt[i * YST + row] = v;
    }
    cp_async_wait0();
    __syncthreads();
    if (active) {
      for (int i = slice; i < CC_SUB; i += nslice) {
        const float4 y4 = *reinterpret_cast<const float4 *>(yt + i * YST + 4 * rg);
        const float4 s0 = *reinterpret_cast<const float4 *>(st + i * sst + 8 * jg);
        const float4 s1 = *reinterpret_cast<const float4 *>(st + i * sst + 8 * jg + 4);
        const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
        const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(yv[u], sv[v], acc[u][v]);
      }
    }
  }
  // sum the slices in a fixed order: red[slice][combo][32] over the staging area
  __syncthreads();
  float *red = csm2;
  if (active) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) red[(slice * combos + combo) * 33 + u * 8 + v] = acc[u][v];
  }
  __syncthreads();
  const int nK = (int)((a.N + CORR_BLOCK - 1) / CORR_BLOCK);
  for (int e = tid; e < combos * 32; e += CC_THREADS) {
    const int cb = e / 32, w = e % 32, u = w / 8, v = w % 8;
    float sum = 0.f;
    for (int sl = 0; sl < nslice; ++sl) sum += red[(sl * combos + cb) * 33 + w];
    const int row = (cb % nrg) * 4 + u, j = (cb / nrg) * 8 + v;
    if (row < rows && j < rpad) {
      // row -> (pair, part): real signal row = 2 pair + part; complex row = 2 signal + part
      const int64_t pair = row >> 1;
      const int comp = row & 1;
      a.part[((pair * nK + blk) * 2 + comp) * rpad + j] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// Rank-r correction of a ragged batch, one plan per signal (FP32, CUDA cores).  Every Slepian
// vector is symmetric or antisymmetric, s_l(N-1-n) = (-1)^l s_l(n) (B commutes with the
// exchange J), so only the rows n < H = ceil(N/2) of S_T are read, halving its traffic:
//   c_j = sum_{n<H} s_j(n) (y(n) +- y(N-1-n))   (the middle sample of an odd N once)
//   z(n) = z+(n) + z-(n),  z(N-1-n) = z+(n) - z-(n),  z+- = sums over the (anti)symmetric j
//   k_rcorr_part   item (signal, chunk of CORR_BLOCK of the H folded samples): partial c, the
//                  8 warps split the samples, lanes split j (coalesced S_T rows), fixed order
//   k_rcorr_reduce block per signal: a = D o (sum of its partials in chunk order)
//   k_rzadd        item: out(n) and out(N-1-n) += ... for the chunk's n (thread per n)
// acoef: [signal][2][RC_RMAX]
// ---------------------------------------------------------------------------
// The chunk's S_T rows are one contiguous block ([n][rpad]).  The block streams it through a
// ring of RC_NST shared-memory tiles of rpr * RC_U rows (rpr = 256 / tpr rows per round, tpr =
// rpad / 4 threads per row) with 16-byte cp.async copies, RC_NST - 1 tiles in flight, together
// with each row's y(n) and y(N-1-n).  Thread t takes the float4 jq = t mod tpr of rows t / tpr,
// t / tpr + rpr, ... (in increasing order), folds y(n) +- y(N-1-n) by the parity of each of its
// four columns and accumulates; fixed-order sums at the end.
constexpr int RC_U = 4, RC_NST = 3;
constexpr int RC_S_F = 256 * RC_U * 4;            // S floats per tile (1024 float4 at most)
constexpr int RC_STAGE_F = RC_S_F + 4 * 512;      // + y: up to 512 rows x (re, im) x (n, N-1-n)
constexpr int rcorr_smem() { return RC_NST * RC_STAGE_F * 4; }
__device__ __forceinline__ void cp_async_wait_ring() {
  asm volatile("cp.async.wait_group %0;" ::"n"(RC_NST - 1) : "memory");
}
__global__ void __launch_bounds__(256) k_rcorr_part(const RSig *sigs, const RItem *items, int cplx, float *part) {
  extern __shared__ __align__(16) float rsm[];
  const RItem it = items[blockIdx.x];
  const RSig q = sigs[it.sig];
  const int tpr = q.rpad / 4, rpr = 256 / tpr;
  const int slot = threadIdx.x / tpr, jq = threadIdx.x % tpr;
  const bool active = slot < rpr;
  const int64_t H = (q.N + 1) / 2;
  const int64_t n0 = (int64_t)it.chunk * CORR_BLOCK;
  const int rows_total = (int)((H - n0 < CORR_BLOCK) ? H - n0 : CORR_BLOCK);
  const int trows = rpr * RC_U;
  const int ntiles = (rows_total + trows - 1) / trows;
  const int jb = (4 * jq) & (RC_RMAX - 1);
  // 4 j never straddle a word (jb % 4 == 0); the word is read from the descriptor in global
  // memory (a runtime index into the register copy would put it in local memory)
  const unsigned odd = (__ldg(&sigs[it.sig].odd[jb >> 5]) >> (jb & 31)) & 15u;
  const float4 *S4 = reinterpret_cast<const float4 *>(q.ST);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(rsm);
  auto issue = [&](int tile) {
    const uint32_t st = sbase + (uint32_t)((tile % RC_NST) * RC_STAGE_F * 4);
    const int r0 = tile * trows;
    const int rows = (rows_total - r0 < trows) ? rows_total - r0 : trows;
    const float4 *src = S4 + (n0 + r0) * tpr;
    for (int e = threadIdx.x; e < rows * tpr; e += 256) cp_async16(st + (uint32_t)(e * 16), src + e, 16);
    const uint32_t yv = st + (uint32_t)(RC_S_F * 4);
    for (int r = threadIdx.x; r < rows; r += 256) {
      const int64_t n = n0 + r0 + r, m = q.N - 1 - n;
      if (cplx) {
        cp_async8(yv + (uint32_t)(r * 16), q.y + 2 * n);
        cp_async8(yv + (uint32_t)(r * 16 + 8), q.y + 2 * m);
      } else {
        cp_async4(yv + (uint32_t)(r * 8), q.y + n);
        cp_async4(yv + (uint32_t)(r * 8 + 4), q.y + m);
      }
    }
  };
#pragma unroll
  for (int t = 0; t < RC_NST - 1; ++t) {
    if (t < ntiles) issue(t);
    cp_async_commit();
  }
  float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
  for (int t = 0; t < ntiles; ++t) {
    if (t + RC_NST - 1 < ntiles) issue(t + RC_NST - 1);
    cp_async_commit();
    cp_async_wait_ring();   // this thread's copies of tile t have landed
    __syncthreads();        // and everyone else's
    if (active) {
      const float *st = rsm + (t % RC_NST) * RC_STAGE_F;
      const float *yv = st + RC_S_F;
      const int r0 = t * trows;
      const int rows = (rows_total - r0 < trows) ? rows_total - r0 : trows;
#pragma unroll
      for (int u = 0; u < RC_U; ++u) {
        const int r = slot + rpr * u;
        if (r < rows) {
          const float4 s4 = reinterpret_cast<const float4 *>(st)[r * tpr + jq];
          const int64_t n = n0 + r0 + r, m = q.N - 1 - n;
          float yr, yi = 0.f, mr = 0.f, mi = 0.f;
          if (cplx) {
            const float4 v = reinterpret_cast<const float4 *>(yv)[r];
            yr = v.x;
            yi = v.y;
            if (m != n) {
              mr = v.z;
              mi = v.w;
            }
          } else {
            const float2 v = reinterpret_cast<const float2 *>(yv)[r];
            yr = v.x;
            if (m != n) mr = v.y;
          }
          const float pr = yr + mr, dr = yr - mr, pi = yi + mi, di = yi - mi;
          ar[0] = fmaf(s4.x, (odd & 1u) ? dr : pr, ar[0]);
          ar[1] = fmaf(s4.y, (odd & 2u) ? dr : pr, ar[1]);
          ar[2] = fmaf(s4.z, (odd & 4u) ? dr : pr, ar[2]);
          ar[3] = fmaf(s4.w, (odd & 8u) ? dr : pr, ar[3]);
          ai[0] = fmaf(s4.x, (odd & 1u) ? di : pi, ai[0]);
          ai[1] = fmaf(s4.y, (odd & 2u) ? di : pi, ai[1]);
          ai[2] = fmaf(s4.z, (odd & 4u) ? di : pi, ai[2]);
          ai[3] = fmaf(s4.w, (odd & 8u) ? di : pi, ai[3]);
        }
      }
    }
    __syncthreads();        // tile t's slot is refilled by tile t + RC_NST at the next issue
  }
  cp_async_wait0();
  // the ring is free: [row slot][comp][j], rpr * 2 * rpad <= 2048 floats
  float *red = rsm;
  if (active) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      red[(slot * 2 + 0) * q.rpad + 4 * jq + u] = ar[u];
      red[(slot * 2 + 1) * q.rpad + 4 * jq + u] = ai[u];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * q.rpad; t += 256) {
    const int comp = t / q.rpad, j = t % q.rpad;
    float sum = 0.f;
    for (int sl = 0; sl < rpr; ++sl) sum += red[(sl * 2 + comp) * q.rpad + j];
    part[q.part + ((int64_t)it.chunk * 2 + comp) * q.rpad + j] = sum;
  }
}

__global__ void k_rcorr_reduce(const RSig *sigs, const float *part, float *acoef) {
  const RSig q = sigs[blockIdx.x];
  for (int t = threadIdx.x; t < 2 * q.rpad; t += blockDim.x) {
    const int comp = t / q.rpad, j = t % q.rpad;
    float sum = 0.f;
    for (int c = 0; c < q.nK; ++c) sum += part[q.part + ((int64_t)c * 2 + comp) * q.rpad + j];
    acoef[((int64_t)blockIdx.x * 2 + comp) * RC_RMAX + j] = j < q.r ? __ldg(q.D + j) * sum : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_rzadd(const RSig *sigs, const RItem *items, int cplx, const float *acoef) {
  // a split by parity: as[c][0][j] = a_j for symmetric j (else 0), as[c][1][j] for antisymmetric
  __shared__ __align__(16) float as[2][2][RC_RMAX];
  const RItem it = items[blockIdx.x];
  const RSig q = sigs[it.sig];
  for (int t = threadIdx.x; t < 2 * RC_RMAX; t += blockDim.x) {
    const int c = t / RC_RMAX, j = t % RC_RMAX;
    const float v = acoef[((int64_t)it.sig * 2) * RC_RMAX + t];
    const bool o = (__ldg(&sigs[it.sig].odd[j >> 5]) >> (j & 31)) & 1u;
    as[c][0][j] = o ? 0.f : v;
    as[c][1][j] = o ? v : 0.f;
  }
  __syncthreads();
  const int64_t H = (q.N + 1) / 2;
  const int64_t n0 = (int64_t)it.chunk * CORR_BLOCK;
  for (int i = threadIdx.x; i < CORR_BLOCK; i += blockDim.x) {
    const int64_t n = n0 + i;
    if (n >= H) break;
    const int64_t m = q.N - 1 - n;
    const float4 *row = reinterpret_cast<const float4 *>(q.ST + n * q.rpad);
    float zp = 0.f, zm = 0.f, wp = 0.f, wm = 0.f;   // re (z) and im (w), symmetric / antisymmetric
    for (int j4 = 0; j4 < q.rpad / 4; ++j4) {
      const float4 s4 = __ldg(row + j4);
      const float4 ap = *reinterpret_cast<const float4 *>(&as[0][0][4 * j4]);
      const float4 am = *reinterpret_cast<const float4 *>(&as[0][1][4 * j4]);
      zp = fmaf(s4.w, ap.w, fmaf(s4.z, ap.z, fmaf(s4.y, ap.y, fmaf(s4.x, ap.x, zp))));
      zm = fmaf(s4.w, am.w, fmaf(s4.z, am.z, fmaf(s4.y, am.y, fmaf(s4.x, am.x, zm))));
      if (cplx) {
        const float4 bp = *reinterpret_cast<const float4 *>(&as[1][0][4 * j4]);
        const float4 bm = *reinterpret_cast<const float4 *>(&as[1][1][4 * j4]);
        wp = fmaf(s4.w, bp.w, fmaf(s4.z, bp.z, fmaf(s4.y, bp.y, fmaf(s4.x, bp.x, wp))));
        wm = fmaf(s4.w, bm.w, fmaf(s4.z, bm.z, fmaf(s4.y, bm.y, fmaf(s4.x, bm.x, wm))));
      }
    }
    if (cplx) {
      float2 *o = reinterpret_cast<float2 *>(q.out);
      float2 v = o[n];
      v.x += zp + zm;
      v.y += wp + wm;
      o[n] = v;
      if (m != n) {
        float2 u = o[m];
        u.x += zp - zm;
        u.y += wp - wm;
        o[m] = u;
      }
    } else {
      q.out[n] += zp + zm;
      if (m != n) q.out[m] += zp - zm;
    }
  }
}

__global__ void __launch_bounds__(FAST_THREADS, 3) k_corr_z(const FastArgs f) {
  const ConvArgs<float> &a = f.a;
  __shared__ __align__(16) float zt[CORR_ROWS][2 * FAST_G + 1];
  __shared__ float acs[2][32][2 * FAST_G + 1];
  const int64_t blk = blockIdx.x, g0 = (int64_t)blockIdx.y * FAST_G;
  const int64_t n0 = blk * CORR_ROWS;
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int ntj = a.rpad / 8;
  for (int jt0 = 0; jt0 < ntj; jt0 += 4) {
    for (int t = threadIdx.x; t < 32 * 2 * FAST_G; t += FAST_THREADS) {
      const int jj = t / (2 * FAST_G), s = t % (2 * FAST_G);
      const int j = jt0 * 8 + jj, gp = s >> 1;
      float val = 0.f;
      if (j < a.r && g0 + gp < a.npairs) val = a.acoef[((g0 + gp) * 2 + (s & 1)) * a.rpad + j];
      uint32_t hi, lo;
      split_tf32(val, hi, lo);
      acs[0][jj][s] = __uint_as_float(hi);
      acs[1][jj][s] = __uint_as_float(lo);
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < CORR_ROWS / 16 / FAST_G; ++mi) {
      const int mt = g + FAST_G * mi;
      float acc[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
      const int nl0 = mt * 16 + gid, nl1 = nl0 + 8;
      const int64_t nA = n0 + nl0, nB = n0 + nl1;
      const bool okA = nA < a.N, okB = nB < a.N;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const int jt = jt0 + kt;
        if (jt < ntj) {
          const int j0 = jt * 8 + tig, j1 = j0 + 4;
          const float2 z2 = make_float2(0.f, 0.f);
          const float2 s0 = okA ? __ldg(f.ST_hl + nA * a.rpad + j0) : z2;
          const float2 s1 = okB ? __ldg(f.ST_hl + nB * a.rpad + j0) : z2;
          const float2 s2 = okA ? __ldg(f.ST_hl + nA * a.rpad + j1) : z2;
          const float2 s3 = okB ? __ldg(f.ST_hl + nB * a.rpad + j1) : z2;
          const uint32_t ahi[4] = {__float_as_uint(s0.x), __float_as_uint(s1.x), __float_as_uint(s2.x),
                                   __float_as_uint(s3.x)};
          const uint32_t alo[4] = {__float_as_uint(s0.y), __float_as_uint(s1.y), __float_as_uint(s2.y),
                                   __float_as_uint(s3.y)};
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint32_t bhi[2], blo[2];
            bhi[0] = __float_as_uint(acs[0][kt * 8 + tig][u * 8 + gid]);
            bhi[1] = __float_as_uint(acs[0][kt * 8 + tig + 4][u * 8 + gid]);
            blo[0] = __float_as_uint(acs[1][kt * 8 + tig][u * 8 + gid]);
            blo[1] = __float_as_uint(acs[1][kt * 8 + tig + 4][u * 8 + gid]);
            mma3(acc[u], ahi, alo, bhi, blo);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const bool first = (jt0 == 0);
        float *z0 = &zt[nl0][u * 8 + 2 * tig], *z1 = &zt[nl1][u * 8 + 2 * tig];
        z0[0] = (first ? 0.f : z0[0]) + acc[u][0];
        z0[1] = (first ? 0.f : z0[1]) + acc[u][1];
        z1[0] = (first ? 0.f : z1[0]) + acc[u][2];
        z1[1] = (first ? 0.f : z1[1]) + acc[u][3];
      }
    }
    __syncthreads();
  }
  // out += Z, coalesced along the samples of each signal
  for (int e = threadIdx.x; e < FAST_G * CORR_ROWS; e += FAST_THREADS) {
    const int gp = e / CORR_ROWS, k = e % CORR_ROWS;
    const int64_t n = n0 + k;
    if (g0 + gp < a.npairs && n < a.N) add_pair(a, g0 + gp, n, make_float2(zt[k][2 * gp], zt[k][2 * gp + 1]));
  }
}

}  // namespace fst
