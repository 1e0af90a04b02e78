// fst_fft.cuh -- FFT building blocks for the prolate-matrix convolution B_{N,W} y
// (Section 1.3, fast projections: B y by an FFT; Section 4.1: zero-padded FFT of
// power-of-two length M >= 2N).
//
// Everything is templated on the real type T (float for the FP32 apply path,
// double for the FP64 apply path and for the plan's eigenvalue convolutions), and
// is __host__ __device__ so the kernel bodies can also be executed by the host
// emulator (fst_emu.cu), one phase at a time, for CPU tests of the index maths.
//
//  * Radix-2/4/8/16 DFTs held in registers (compile-time twiddles).
//  * Stockham auto-sort stages in shared memory over a tile of `ncols` independent
//    transforms of length L: element i of column c lives at pad(i * ncols + c).
//    With ncols = 1 this is one row transform (contiguous); with ncols > 1 the
//    columns of a tile are transformed side by side and consecutive threads touch
//    consecutive columns (bank-conflict free).
//  * Twiddles exp(-+2 pi i k / 2^24) come from a two-level table
//    (hi[k >> 12] * lo[k & 4095]) built in FP64 at plan time.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FST_HD __host__ __device__ __forceinline__

namespace fst {

constexpr int TW_LOG2 = 24;                  // twiddle root: exp(-2 pi i / 2^24)
constexpr int TW_SPLIT = 12;                 // two-level table split
constexpr int TW_LO_SIZE = 1 << TW_SPLIT;    // 4096
constexpr int TW_HI_SIZE = 1 << (TW_LOG2 - TW_SPLIT);

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2 = typename C2<T>::type;

template <typename T> FST_HD c2<T> mk(T x, T y) { c2<T> r; r.x = x; r.y = y; return r; }
template <typename V> FST_HD V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> FST_HD V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> FST_HD V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V> FST_HD V cconj(V a) { a.y = -a.y; return a; }
template <typename V, typename S> FST_HD V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> FST_HD V mul_mi(V a) {
  V r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <typename P> FST_HD P ldg(const P *p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// padded shared-memory index: one spare element every 16 keeps the strided
// Stockham writes of the early stages at most 2-way bank conflicted
FST_HD int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_size(int n) { return n + (n >> 4) + 1; }

// exp(-2 pi i k / 16), k = 0..15, as constants
FST_HD double w16re(int k) {
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, H = 0.70710678118654752440;
  switch (k & 15) {
    case 0: return 1.0;  case 1: return C1;  case 2: return H;   case 3: return S1;
    case 4: return 0.0;  case 5: return -S1; case 6: return -H;  case 7: return -C1;
    case 8: return -1.0; case 9: return -C1; case 10: return -H; case 11: return -S1;
    case 12: return 0.0; case 13: return S1; case 14: return H;  default: return C1;
  }
}
FST_HD double w16im(int k) {
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, H = 0.70710678118654752440;
  switch (k & 15) {
    case 0: return 0.0;  case 1: return -S1; case 2: return -H;  case 3: return -C1;
    case 4: return -1.0; case 5: return -C1; case 6: return -H;  case 7: return -S1;
    case 8: return 0.0;  case 9: return S1;  case 10: return H;  case 11: return C1;
    case 12: return 1.0; case 13: return C1; case 14: return H;  default: return S1;
  }
}
// W_R^k (R divides 16), conjugated for the inverse transform
template <typename T, int R, bool INV> FST_HD c2<T> wconst(int k) {
  const int kk = (k * (16 / R)) & 15;
  return mk<T>((T)w16re(kk), INV ? (T)(-w16im(kk)) : (T)w16im(kk));
}

// ----- register DFTs (unnormalised; INV uses exp(+2 pi i nk/R)) ---------------

template <typename T, bool INV> FST_HD void dft2(c2<T> &a, c2<T> &b) {
  c2<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename T, bool INV> FST_HD void dft4(c2<T> &x0, c2<T> &x1, c2<T> &x2, c2<T> &x3) {
  c2<T> s02 = cadd(x0, x2), d02 = csub(x0, x2);
  c2<T> s13 = cadd(x1, x3), d13 = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

// R = R1 * R2 split: with x[R2 a + b], Y_b[c] = DFT_R1 over a, Y_b[c] *= W_R^{bc},
// X[c + R1 d] = DFT_R2 over b of Y_b[c].
template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 2, INV> {
  FST_HD static void run(c2<T> *v) { dft2<T, INV>(v[0], v[1]); }
};
template <typename T, bool INV> struct Dft<T, 4, INV> {
  FST_HD static void run(c2<T> *v) { dft4<T, INV>(v[0], v[1], v[2], v[3]); }
};
template <typename T, bool INV> struct Dft<T, 8, INV> {
  // 8 = 4 x 2
  FST_HD static void run(c2<T> *v) {
    dft4<T, INV>(v[0], v[2], v[4], v[6]);
    dft4<T, INV>(v[1], v[3], v[5], v[7]);
    v[3] = cmul(v[3], wconst<T, 8, INV>(1));
    v[5] = cmul(v[5], wconst<T, 8, INV>(2));
    v[7] = cmul(v[7], wconst<T, 8, INV>(3));
    c2<T> o[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      c2<T> e0 = v[2 * c], e1 = v[2 * c + 1];
      o[c] = cadd(e0, e1);
      o[c + 4] = csub(e0, e1);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  }
};
template <typename T, bool INV> struct Dft<T, 16, INV> {
  // 16 = 4 x 4
  FST_HD static void run(c2<T> *v) {
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<T, INV>(v[b], v[4 + b], v[8 + b], v[12 + b]);
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
      for (int c = 1; c < 4; ++c)
        // W_16^4 = -i (conjugated: +i) is a swap and a sign, not a product
        v[4 * c + b] = (b * c == 4) ? mul_mi<INV>(v[4 * c + b]) : cmul(v[4 * c + b], wconst<T, 16, INV>(b * c));
    c2<T> o[16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      c2<T> y0 = v[4 * c], y1 = v[4 * c + 1], y2 = v[4 * c + 2], y3 = v[4 * c + 3];
      dft4<T, INV>(y0, y1, y2, y3);
      o[c] = y0; o[c + 4] = y1; o[c + 8] = y2; o[c + 12] = y3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
};

// ----- twiddles ---------------------------------------------------------------

template <typename T> struct Tw {
  const c2<T> *hi;   // exp(-2 pi i (a << 12) / 2^24), a < 4096
  const c2<T> *lo;   // exp(-2 pi i b / 2^24), b < 4096
  // exp(-+2 pi i k / 2^24), k in [0, 2^24)
  template <bool INV> FST_HD c2<T> get(uint32_t k) const {
    c2<T> w = cmul(ldg(hi + ((k >> TW_SPLIT) & (TW_HI_SIZE - 1))), ldg(lo + (k & (TW_LO_SIZE - 1))));
    return INV ? cconj(w) : w;
  }
  // exp(-+2 pi i m / 2^log2n) for any m (reduced mod 2^log2n), log2n <= 24
  template <bool INV> FST_HD c2<T> root(uint64_t m, int log2n) const {
    uint32_t k = (uint32_t)((m & ((1ull << log2n) - 1)) << (TW_LOG2 - log2n));
    return get<INV>(k);
  }
};

// ----- Stockham stages in shared memory -----------------------------------------
// One stage of radix R on a tile of `ncols` transforms of length L (power of 2)
// with current sub-transform length Ns.  Each thread owns up to 16/R butterflies
// (butterfly b = tid + q * nthr; column b % ncols, index j = b / ncols):
//   v_t = x[j + t L/R] * W_{Ns R}^{(j mod Ns) t},  DFT_R(v),
//   y[(j / Ns) Ns R + (j mod Ns) + t Ns] = v_t.
// The read phase of every thread completes (barrier) before any write phase, so
// the stage works in place.  `v` holds 16 complex values per thread.

template <int R> struct LogR { static constexpr int v = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : 4; };

template <typename T, int R, bool INV>
FST_HD void stage_read(const c2<T> *buf, c2<T> *v, int log2L, int log2Ns, int ncols, int tid, int nthr,
                       const Tw<T> &tw) {
  constexpr int PER = 16 / R;
  constexpr int LOGR = LogR<R>::v;
  const int L = 1 << log2L;
  const int nb = ncols * (L >> LOGR);
  const int stride = L >> LOGR;
  const int Ns = 1 << log2Ns;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = tid + q * nthr;
    if (b < nb) {
      c2<T> *w = v + q * R;
      const int col = b % ncols, j = b / ncols;
#pragma unroll
      for (int t = 0; t < R; ++t) w[t] = buf[pad((j + t * stride) * ncols + col)];
      if (Ns > 1) {
        const int k = j & (Ns - 1);
        // W_{Ns R}^{k t} = exp(-2 pi i k t / 2^(log2Ns + LOGR)); powers of the base
        // root from the table (t = 1, 2, 4, 8, 12) and at most two products
        const uint32_t base = (uint32_t)k << (TW_LOG2 - log2Ns - LOGR);
        const c2<T> w1 = tw.template get<INV>(base);
        w[1] = cmul(w[1], w1);
        if (R >= 4) {
          const c2<T> w2 = tw.template get<INV>(2 * base);
          const c2<T> w3 = cmul(w2, w1);
          w[2] = cmul(w[2], w2);
          w[3] = cmul(w[3], w3);
          if (R >= 8) {
            const c2<T> w4 = tw.template get<INV>(4 * base);
            w[4] = cmul(w[4], w4);
            w[5] = cmul(w[5], cmul(w4, w1));
            w[6] = cmul(w[6], cmul(w4, w2));
            w[7] = cmul(w[7], cmul(w4, w3));
            if (R >= 16) {
              const c2<T> w8 = tw.template get<INV>(8 * base);
              const c2<T> w12 = tw.template get<INV>(12 * base);
              w[8] = cmul(w[8], w8);
              w[9] = cmul(w[9], cmul(w8, w1));
              w[10] = cmul(w[10], cmul(w8, w2));
              w[11] = cmul(w[11], cmul(w8, w3));
              w[12] = cmul(w[12], w12);
              w[13] = cmul(w[13], cmul(w12, w1));
              w[14] = cmul(w[14], cmul(w12, w2));
              w[15] = cmul(w[15], cmul(w12, w3));
            }
          }
        }
      }
      Dft<T, R, INV>::run(w);
    }
  }
}

template <typename T, int R>
FST_HD void stage_write(c2<T> *buf, const c2<T> *v, int log2L, int log2Ns, int ncols, int tid, int nthr) {
  constexpr int PER = 16 / R;
  constexpr int LOGR = LogR<R>::v;
  const int L = 1 << log2L;
  const int nb = ncols * (L >> LOGR);
  const int Ns = 1 << log2Ns;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = tid + q * nthr;
    if (b < nb) {
      const c2<T> *w = v + q * R;
      const int col = b % ncols, j = b / ncols;
      const int k = j & (Ns - 1);
      const int d0 = ((j >> log2Ns) << (log2Ns + LOGR)) + k;
#pragma unroll
      for (int t = 0; t < R; ++t) buf[pad((d0 + t * Ns) * ncols + col)] = w[t];
    }
  }
}

// Radix of each stage of a length-2^log2L transform: a first radix-2^(log2L mod 4)
// stage (when log2L is not a multiple of 4), then radix 16.
FST_HD int first_radix_log2(int log2L) { return log2L & 3; }

// Full transform of the tile, driven by an executor `ex` whose phase(f) runs
// f(tid, state) for every thread and then synchronises.  Requires
// nthr * 16 >= ncols * 2^log2L.  Natural order in and out.
template <typename T, bool INV, typename Ex>
FST_HD void tile_fft(Ex &ex, c2<T> *buf, int log2L, int ncols, const Tw<T> &tw) {
  int log2Ns = 0;
  const int nthr = ex.nthr;
  const int r0 = first_radix_log2(log2L);
  if (r0 == 1) {
    ex.phase([&](int tid, typename Ex::State &st) { stage_read<T, 2, INV>(buf, st.v, log2L, 0, ncols, tid, nthr, tw); });
    ex.phase([&](int tid, typename Ex::State &st) { stage_write<T, 2>(buf, st.v, log2L, 0, ncols, tid, nthr); });
  } else if (r0 == 2) {
    ex.phase([&](int tid, typename Ex::State &st) { stage_read<T, 4, INV>(buf, st.v, log2L, 0, ncols, tid, nthr, tw); });
    ex.phase([&](int tid, typename Ex::State &st) { stage_write<T, 4>(buf, st.v, log2L, 0, ncols, tid, nthr); });
  } else if (r0 == 3) {
    ex.phase([&](int tid, typename Ex::State &st) { stage_read<T, 8, INV>(buf, st.v, log2L, 0, ncols, tid, nthr, tw); });
    ex.phase([&](int tid, typename Ex::State &st) { stage_write<T, 8>(buf, st.v, log2L, 0, ncols, tid, nthr); });
  }
  log2Ns = r0;
  while (log2Ns < log2L) {
    const int ns = log2Ns;
    ex.phase([&](int tid, typename Ex::State &st) { stage_read<T, 16, INV>(buf, st.v, log2L, ns, ncols, tid, nthr, tw); });
    ex.phase([&](int tid, typename Ex::State &st) { stage_write<T, 16>(buf, st.v, log2L, ns, ncols, tid, nthr); });
    log2Ns += 4;
  }
}

}  // namespace fst
