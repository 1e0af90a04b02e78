// fst_big.cuh -- FP32 column passes of the four-step transform for P = 32 P2 rows,
// 2 <= P2 <= 32 (M = P Q from 2^18 up; device only).
//
// Same decomposition as the other passes (n = n1 Q + n2, k = k1 + P k2, inter[pair][k1][n2]);
// the P-point column DFT is split once more:
//   forward, n1 = P2 a + b (a < 32, b < P2), k1 = k + 32 m (k < 32, m < P2):
//     X[k + 32 m] = sum_b W_P2^{b m} ( W_P^{b k} sum_a x[P2 a + b] W_32^{a k} )
//     stage 1: per (b, column) a 32-point DFT over a; the signal occupies rows n1 < P/2
//              (M >= 2N), i.e. a < 16, so it is a half-input DFT; times W_P^{b k};
//     stage 2: per (k, column) a P2-point DFT over b; times W_M^{n2 k1}; stored.
//   inverse (pass C), the transpose: per (k, column) a P2-point inverse DFT over m, times
//     W_P^{-b k}; then per (b, column) the first 16 outputs a of a 32-point inverse DFT over k
//     (rows n1 = P2 a + b < P/2 are the only ones that hold output).
// Both stages keep their values in registers; the exchange between them goes through one
// shared-memory tile S[b][k][column] of the CTA's NB = 256 / P2 columns of one pair (64 KB).
// The rank-r correction is not fused here (a tile covers one pair only): the caller computes
// a = D o S_T^T y before and adds S_T a after, over the whole batch.
#pragma once
#include "fst_fast.cuh"

namespace fst {

// W_P^{t} (forward) or W_P^{-t} (inverse), t < P <= 1024, from the W_1024 table
template <bool INV> __device__ __forceinline__ float2 big_wP(const ConvArgs<float> &a, int t, int log2P) {
  const float2 w = __ldg(a.twB + TWB_P_OFF + (t << (10 - log2P)));
  return INV ? make_float2(w.x, -w.y) : w;
}

// ---------------------------------------------------------------------------
// pass A: grid (Q / NB, npairs), 256 threads, dynamic shared memory big_smem_bytes(P2)
// ---------------------------------------------------------------------------
template <int P2>
__global__ void __launch_bounds__(256, 3) k_colA(const ConvArgs<float> a) {
  constexpr int NB = big_nb(P2), BS = big_bs(P2), P = 32 * P2;
  extern __shared__ __align__(16) float2 bsm[];
  const int Q = 1 << a.log2Q;
  const int log2P = a.log2P;
  const int64_t pl = blockIdx.y;
  const int64_t n2_0 = (int64_t)blockIdx.x * NB;
  const int col = threadIdx.x % NB, hi = threadIdx.x / NB;   // hi: b in stage 1, k group in stage 2
  const int64_t n2 = n2_0 + col;
  {
    // stage 1: b = hi; x[P2 a + b] for a < 16
    const int b = hi;
    float2 v[32];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int n1 = P2 * q + b;
      const int64_t n = (int64_t)n1 * Q + n2;
      v[q] = (n1 < a.Pnz && n < a.N) ? load_pair(a, pl, n) : make_float2(0.f, 0.f);
    }
    dft_half_in<32>(v);
    float2 *s = bsm + b * BS + col;
    s[0] = v[0];
#pragma unroll
    for (int k = 1; k < 32; ++k) s[k * NB] = (b == 0) ? v[k] : cmul(v[k], big_wP<false>(a, b * k, log2P));
  }
  __syncthreads();
  // stage 2: tasks k = hi + P2 i; outputs k1 = k + 32 m, times W_M^{n2 k1}
  float2 *dst = a.inter + (pl * P) * (int64_t)Q + n2;
  // W_M^{n2 (k + 32 m)} = alpha_k beta^m, beta = W_M^{32 n2}: every 8th m from an exact lookup
  // of W_M^{n2 (k + 32 m)}, the others by at most 7 products with beta
  const float2 beta = a.tw.root<false>(32 * (uint64_t)n2, a.log2M);
#pragma unroll 2
  for (int i = 0; i < 32 / P2; ++i) {
    const int k = hi + P2 * i;
    float2 u[P2];
#pragma unroll
    for (int b = 0; b < P2; ++b) u[b] = bsm[b * BS + k * NB + col];
    RegDft<P2, false>::run(u);
    float2 t;
#pragma unroll
    for (int m = 0; m < P2; ++m) {
      if ((m & 7) == 0) t = a.tw.root<false>((uint64_t)n2 * (uint64_t)(k + 32 * m), a.log2M);
      else t = cmul(t, beta);
      dst[(int64_t)(k + 32 * m) * Q] = (k == 0 && m == 0) ? u[0] : cmul(u[m], t);
    }
  }
}

// ---------------------------------------------------------------------------
// pass C: grid (Q / NB, npairs), 256 threads, dynamic shared memory big_smem_bytes(P2)
// out[n] for n < N (no correction: the caller adds S_T a afterwards)
// ---------------------------------------------------------------------------
template <int P2>
__global__ void __launch_bounds__(256, 3) k_colC(const ConvArgs<float> a) {
  constexpr int NB = big_nb(P2), BS = big_bs(P2), P = 32 * P2;
  extern __shared__ __align__(16) float2 bsm[];
  const int Q = 1 << a.log2Q;
  const int log2P = a.log2P;
  const int64_t pl = blockIdx.y;
  const int64_t n2_0 = (int64_t)blockIdx.x * NB;
  const int col = threadIdx.x % NB, hi = threadIdx.x / NB;
  const int64_t n2 = n2_0 + col;
  {
    // stage 1: tasks k = hi + P2 i; inverse P2-point DFT over m of X[k + 32 m], times W_P^{-b k}
    const float2 *src = a.inter + (pl * P) * (int64_t)Q + n2;
#pragma unroll 2
    for (int i = 0; i < 32 / P2; ++i) {
      const int k = hi + P2 * i;
      float2 u[P2];
#pragma unroll
      for (int m = 0; m < P2; ++m) u[m] = src[(int64_t)(k + 32 * m) * Q];
      RegDft<P2, true>::run(u);
      float2 *s = bsm + k * NB + col;
      s[0] = u[0];
#pragma unroll
      for (int b = 1; b < P2; ++b) s[b * BS] = (k == 0) ? u[b] : cmul(u[b], big_wP<true>(a, b * k, log2P));
    }
  }
  __syncthreads();
  // stage 2: b = hi; outputs n1 = P2 a + b for a < 16
  const int b = hi;
  float2 v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = bsm[b * BS + k * NB + col];
  float2 o[16];
  idft_half_out<32>(v, o);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int n1 = P2 * q + b;
    const int64_t n = (int64_t)n1 * Q + n2;
    if (n1 < a.Pnz && n < a.N) store_pair(a, pl, n, o[q]);
  }
}

}  // namespace fst
