// fst_kernels.cuh -- bodies of the apply kernels of the fast Slepian projection
//
//     out = beta * B_{N,W} y + S_T (D o (S_T^T y))          (Section 1.3, Corollary 2)
//
// B_{N,W} y is the first N samples of a length-M circular convolution of the
// zero-padded signal with the even sinc embedding c (c[k] = c[M-k] = b[k], k < N;
// Section 4.1), done as FFT -> multiply by the real spectrum DFT_M(c)/M -> inverse FFT.
// Real signals travel two at a time as the real and imaginary part of one complex
// transform: the spectrum is real and even, so B acts on both parts separately and
// the two results come back in the real and imaginary parts ("pairs").  A complex
// signal is one pair.
//
// Two layouts of the length-M transform:
//   small  (M <= one CTA's shared memory): one CTA per pair does everything.
//   3-pass (M = P * Q):  n = n1 Q + n2, k = k1 + P k2 (four-step decomposition)
//     pass A: per column n2, P-point DFT over n1, times W_M^{n2 k1}   -> inter[k1][n2]
//             (+ the partial sums of S_T^T y over the tile, written per tile)
//     reduce: c = sum of the partials in a fixed order, a = D o c
//     pass B: per row k1, Q-point DFT over n2 (natural k2 order), times
//             spec[k1 + P k2], inverse Q-point DFT, times W_M^{-n2 k1} -> inter[k1][n2]
//     pass C: per column n2, inverse P-point DFT over k1 -> n1; the first N samples
//             plus S_T a are written out.
// No floating-point atomics anywhere: every sum has a fixed order, so results are
// bit-for-bit repeatable.
//
// Each body is a sequence of phases separated by block barriers.  The device
// executor (DevEx) runs one thread per phase call and __syncthreads() between
// phases; the host executor (fst_emu.cu) loops the threads of a block, which lets
// the CPU tests run these exact bodies.
#pragma once
#include "fst_fft.cuh"

namespace fst {

// MODE_ZONLY: B y + S_T a with a = D o S_T^T y computed beforehand (fast column passes)
enum { MODE_FULL = 0, MODE_CONV = 1, MODE_FORWARD = 2, MODE_ZONLY = 3 };

constexpr int CORR_ROWS = 512;    // samples per tensor-core tile of the separate correction kernels
constexpr int CORR_BLOCK = 2048;  // samples per partial sum of S_T^T y (four tiles)
// CUDA-core out += S_T a: threads, samples and signal rows per block
constexpr int ZR_THREADS = 256, ZR_N = 128, ZR_ROWS = 64;

// Launch layout of the length-M transform for one real type.
struct Layout {
  bool small = true;
  bool fast = false;   // FP32 four-step with P <= 32: register column passes + tensor-core correction
  bool fused_reduce = false;  // the row pass also sums the correction partials (device fast path, Q = 4096)
  bool split_corr = false;    // correction outside the column passes (device FP32 four-step, P > 32)
  bool big = false;    // FP32 four-step with P = 32 P2, 2 <= P2 <= 32: two-stage register column passes
  int P2 = 0;
  int log2M = 0, log2P = 0, log2Q = 0;
  int Pnz = 0, NB = 0, G = 1, ntiles = 0;
  int nthr_small = 0, nthr_A = 0, nthr_B = 0, nthr_C = 0;
  size_t smem_small = 0, smem_A = 0, smem_B = 0, smem_C = 0;
  int64_t chunk = 1;   // pairs per launch group
};

// two-stage column passes (P = 32 P2): columns per CTA, float2 stride between the b-blocks of
// the shared tile (NB < 16 columns take a 16-word shift, so the two b-blocks a half-warp
// touches fall in different banks), and the tile's bytes
__host__ __device__ constexpr int big_nb(int P2) { return 256 / P2; }
__host__ __device__ constexpr int big_bs(int P2) { return 32 * big_nb(P2) + (big_nb(P2) < 16 ? 8 : 0); }
__host__ __device__ constexpr int big_smem_bytes(int P2) { return P2 * big_bs(P2) * 8; }

// position of natural frequency index k in the layout's spectrum array
__host__ __device__ inline int64_t spec_pos(const Layout &L, int64_t k) {
  if (L.small) return k;
  const int64_t P = 1LL << L.log2P;
  return (k & (P - 1)) * (1LL << L.log2Q) + (k >> L.log2P);
}



// A pair slot of a ragged four-step batch: one complex signal, or two real signals of the same
// FFT length with their own plans (the second travels as the imaginary part; y2 == nullptr
// when the slot holds one real signal)
template <typename T> struct RPair {
  const T *y;
  T *out;
  const T *spec;   // its spectrum, in the length class's [k1][k2] layout
  int64_t N;
  const T *y2;     // second real signal of the slot (or nullptr), its output, spectrum, length
  T *out2;
  const T *spec2;
  int64_t N2;
};

// Rank-r correction of the four-step signals of a ragged batch (FP32 device): one entry per
// signal, and work items of CORR_BLOCK samples
struct RSig {
  const float *y;      // real: N floats; complex: N (re, im) pairs
  float *out;
  const float *ST;     // [N][rpad] FP32; only rows n < ceil(N/2) are read (J-symmetry below)
  const float *D;      // [r]
  int64_t N;
  int r, rpad;
  int nK;              // ceil(ceil(N/2) / CORR_BLOCK) partial blocks
  int64_t part;        // offset (floats) of its partials [nK][2][rpad] in the partial buffer
  uint32_t odd[4];     // bit j: column j is antisymmetric, s(N-1-n) = -s(n) (its index l is odd)
};
struct RItem {
  int sig, chunk;
};
constexpr int RC_RMAX = 128;   // coefficient slots per signal and part (rpad <= RC_RMAX)

template <typename T> struct ConvArgs {
  // signals
  const T *y;         // real: batch rows of N (stride ld); complex: batch rows of N pairs (stride ld pairs)
  T *out;
  int64_t ld;
  int64_t batch;      // number of signals (real) or complex signals
  int cplx;           // 0: real signals paired (2p, 2p+1); 1: complex signals
  int64_t pair0;      // first global pair handled by this launch
  int64_t npairs;     // pairs handled by this launch (local pair index < npairs)
  int64_t N;
  int log2M;
  // 3-pass decomposition
  int log2P, log2Q;
  int Pnz;            // rows n1 with n1 * Q < N
  int NB;             // columns per pair in a pass-A/C tile
  int G;              // pairs per pass-A/C tile
  // plan data
  const T *spec;      // DFT_M(c) * beta / M, natural order (small) or [k1][k2] (3-pass)
  const T *ST;        // [N][rpad], row n = (s_j[n])_j, zero padded
  const c2<T> *ST_hl; // FP32 tensor-core path: (TF32-rounded S_T, TF32 remainder) interleaved
  int r, rpad;
  const T *D;         // [r]
  Tw<T> tw;
  // workspace (3-pass)
  c2<T> *inter;       // [npairs][P][Q] (small, forward mode: [npairs][M])
  T *part;            // [npairs][ntiles][2][rpad]
  T *acoef;           // [npairs][2][rpad]: D o c for (re, im)
  int mode;
  int nkb;            // partial blocks per pair summed by the separate correction's reduction
  const float *STt;   // FP32 device plans: S_T^T, K-major, [tc_nB][tc_Npad]
  int tc_nB;
  int64_t tc_Npad;
  const float2 *twB;  // FP32 device plans: stage twiddles of the 4096-point row FFT, then W_1024^t
  const float2 *tw8;  // FP32 device plans: stage twiddles of the 8192-point row FFT
  const RPair<T> *rp; // ragged batch: per pair slot signal, length and spectrum (else nullptr)
  int two_spec;       // ragged real slots hold two signals with their own spectra (pass B pairs rows)
};
// twB: [t][k] W_256^{k t} (k, t < 16), [t][k] W_4096^{k t} (t < 16, k < 256), W_1024^t (t < 1024)
constexpr int TWB_P_OFF = 16 * 16 + 16 * 256;
constexpr int TWB_WORDS = TWB_P_OFF + 1024;
// tw8 (8192-point rows): W_8192^j (j < 4096), then [t][k] W_32^{k t} (k < 2), W_512^{k t} (k < 32),
// W_8192^{k t} (k < 512), t < 16
constexpr int TW8_R2 = 0, TW8_32 = 4096, TW8_512 = TW8_32 + 16 * 2, TW8_8192 = TW8_512 + 16 * 32;
constexpr int TW8_WORDS = TW8_8192 + 16 * 512;

// TF32 rounding (round to nearest, ties away from zero, 10 mantissa bits kept)
FST_HD float tf32_round(float x) {
  union { float f; uint32_t u; } v;
  v.f = x;
  if ((v.u & 0x7f800000u) == 0x7f800000u) return x;
  v.u = (v.u + 0x1000u) & 0xffffe000u;
  return v.f;
}

// One signal of a ragged batch processed by the single-CTA kernel (its own plan).
template <typename T> struct RaggedDesc {
  const T *y;
  T *out;
  const T *spec;
  const T *ST;
  const T *D;
  int64_t N;
  int r, rpad;
};

template <typename T> struct KState {
  c2<T> v[16];
};

// ---- signal access ---------------------------------------------------------
template <typename T> FST_HD c2<T> load_pair(const ConvArgs<T> &a, int64_t pl, int64_t n) {
  const int64_t p = a.pair0 + pl;
  if (a.rp) {
    const RPair<T> &q = a.rp[p];
    if (a.cplx) return n < q.N ? reinterpret_cast<const c2<T> *>(q.y)[n] : mk<T>(0, 0);
    return mk<T>(n < q.N ? q.y[n] : (T)0, (q.y2 && n < q.N2) ? q.y2[n] : (T)0);
  }
  if (a.cplx) {
    const c2<T> *y2 = reinterpret_cast<const c2<T> *>(a.y);
    return y2[p * a.ld + n];
  }
  const int64_t s0 = 2 * p, s1 = 2 * p + 1;
  const T re = a.y[s0 * a.ld + n];
  const T im = (s1 < a.batch) ? a.y[s1 * a.ld + n] : (T)0;
  return mk<T>(re, im);
}
template <typename T> FST_HD void store_pair(const ConvArgs<T> &a, int64_t pl, int64_t n, c2<T> v) {
  const int64_t p = a.pair0 + pl;
  if (a.rp) {
    const RPair<T> &q = a.rp[p];
    if (a.cplx) {
      if (n < q.N) reinterpret_cast<c2<T> *>(q.out)[n] = v;
      return;
    }
    if (n < q.N) q.out[n] = v.x;
    if (q.out2 && n < q.N2) q.out2[n] = v.y;
    return;
  }
  if (a.cplx) {
    reinterpret_cast<c2<T> *>(a.out)[p * a.ld + n] = v;
    return;
  }
  const int64_t s0 = 2 * p, s1 = 2 * p + 1;
  a.out[s0 * a.ld + n] = v.x;
  if (s1 < a.batch) a.out[s1 * a.ld + n] = v.y;
}

// spectrum of local pair pl (its own for a ragged batch)
template <typename T> FST_HD const T *spec_of(const ConvArgs<T> &a, int64_t pl) {
  return a.rp ? a.rp[a.pair0 + pl].spec : a.spec;
}

// correction epilogue value: S_T[n,:] . (a_re, a_im)
template <typename T> FST_HD c2<T> corr_value(const ConvArgs<T> &a, int64_t n, const T *are, const T *aim) {
  const T *row = a.ST + n * a.rpad;
  T zr = 0, zi = 0;
  for (int j = 0; j < a.r; ++j) {
    const T s = ldg(row + j);
    zr += s * are[j];
    zi += s * aim[j];
  }
  return mk<T>(zr, zi);
}

// ---- small: one CTA per pair, M <= shared-memory capacity ----------------------
// smem: buf[padded_size(M)] complex, red[nwarps][2][64] reals, coef[2][rpad] reals
template <typename T, typename Ex>
FST_HD void small_body(Ex &ex, const ConvArgs<T> &a, int64_t pl, c2<T> *buf, T *red, T *coef) {
  using St = typename Ex::State;
  const int log2L = a.log2M;
  const int L = 1 << log2L;
  const int N = (int)a.N;
  const int nthr = ex.nthr;
  const int nwarps = (nthr + 31) / 32;

  ex.phase([&](int tid, St &) {
    for (int i = tid; i < L; i += nthr) buf[pad(i)] = (i < N) ? load_pair(a, pl, i) : mk<T>(0, 0);
  });

  const bool corr = (a.mode == MODE_FULL) && a.r > 0;
  for (int j0 = 0; corr && j0 < a.r; j0 += 64) {
    // warps split the samples, lanes split j: red[w][c][jj] = sum over the warp's samples
    ex.phase([&](int tid, St &) {
      const int w = tid >> 5, lane = tid & 31;
      T acc[4] = {0, 0, 0, 0};
      const int ja = j0 + lane, jb = j0 + lane + 32;
      for (int i = w; i < N; i += nwarps) {
        const c2<T> v = buf[pad(i)];
        const T *row = a.ST + (int64_t)i * a.rpad;
        const T sa = (ja < a.r) ? ldg(row + ja) : (T)0;
        const T sb = (jb < a.r) ? ldg(row + jb) : (T)0;
        acc[0] += sa * v.x; acc[1] += sa * v.y;
        acc[2] += sb * v.x; acc[3] += sb * v.y;
      }
      T *rw = red + w * 128;
      rw[lane] = acc[0]; rw[64 + lane] = acc[1];
      rw[32 + lane] = acc[2]; rw[96 + lane] = acc[3];
    });
    ex.phase([&](int tid, St &) {
      for (int t = tid; t < 128; t += nthr) {
        const int c = t >> 6, jj = t & 63;
        T s = 0;
        for (int w = 0; w < nwarps; ++w) s += red[w * 128 + c * 64 + jj];
        const int j = j0 + jj;
        if (j < a.r) coef[c * a.rpad + j] = ldg(a.D + j) * s;
      }
    });
  }

  tile_fft<T, false>(ex, buf, log2L, 1, a.tw);

  if (a.mode == MODE_FORWARD) {
    ex.phase([&](int tid, St &) {
      for (int i = tid; i < L; i += nthr) a.inter[pl * L + i] = buf[pad(i)];
    });
    return;
  }

  ex.phase([&](int tid, St &) {
    for (int i = tid; i < L; i += nthr) buf[pad(i)] = cscale(buf[pad(i)], ldg(a.spec + i));
  });

  tile_fft<T, true>(ex, buf, log2L, 1, a.tw);

  ex.phase([&](int tid, St &) {
    for (int i = tid; i < N; i += nthr) {
      c2<T> v = buf[pad(i)];
      if (corr) v = cadd(v, corr_value(a, i, coef, coef + a.rpad));
      store_pair(a, pl, i, v);
    }
  });
}

// ---- pass A: forward column DFTs over n1 for a tile of G pairs x NB columns ----
// tile element (n1, col), col = g * NB + c, lives at buf[pad(n1 * ncols + col)]
// smem: buf[padded_size(P * ncols)] complex, red[nwarps][2][64] reals
template <typename T, typename Ex>
FST_HD void passA_body(Ex &ex, const ConvArgs<T> &a, int64_t tile, int64_t group, c2<T> *buf, T *red) {
  using St = typename Ex::State;
  const int P = 1 << a.log2P;
  const int Q = 1 << a.log2Q;
  const int ncols = a.G * a.NB;
  const int nthr = ex.nthr;
  const int nwarps = (nthr + 31) / 32;
  const int64_t n2_0 = tile * a.NB;
  const int64_t g0 = group * a.G;
  const int ntiles = Q / a.NB;

  ex.phase([&](int tid, St &) {
    for (int e = tid; e < P * ncols; e += nthr) {
      const int n1 = e / ncols, col = e % ncols;
      const int g = col / a.NB, c = col % a.NB;
      const int64_t n = (int64_t)n1 * Q + n2_0 + c;
      c2<T> v = mk<T>(0, 0);
      if (n1 < a.Pnz && n < a.N && g0 + g < a.npairs) v = load_pair(a, g0 + g, n);
      buf[pad(e)] = v;
    }
  });

  if (a.mode == MODE_FULL && a.r > 0) {
    // warps of pair g: w = g * wpp + u, u < wpp; lanes split j (j = lane, lane + 32)
    const int wpp = nwarps / a.G;  // host guarantees nwarps % G == 0
    const int nel = a.Pnz * a.NB;
    for (int j0 = 0; j0 < a.r; j0 += 64) {
      ex.phase([&](int tid, St &) {
        const int w = tid >> 5, lane = tid & 31;
        const int g = w / wpp, u = w % wpp;
        T acc[4] = {0, 0, 0, 0};
        const int ja = j0 + lane, jb = j0 + lane + 32;
        for (int e = u; e < nel; e += wpp) {
          const int n1 = e / a.NB, c = e % a.NB;
          const int64_t n = (int64_t)n1 * Q + n2_0 + c;
          if (n >= a.N) continue;
          const c2<T> v = buf[pad(n1 * ncols + g * a.NB + c)];
          const T *row = a.ST + n * a.rpad;
          const T sa = (ja < a.r) ? ldg(row + ja) : (T)0;
          const T sb = (jb < a.r) ? ldg(row + jb) : (T)0;
          acc[0] += sa * v.x; acc[1] += sa * v.y;
          acc[2] += sb * v.x; acc[3] += sb * v.y;
        }
        T *rw = red + w * 128;
        rw[lane] = acc[0]; rw[64 + lane] = acc[1];
        rw[32 + lane] = acc[2]; rw[96 + lane] = acc[3];
      });
      ex.phase([&](int tid, St &) {
        for (int t = tid; t < a.G * 128; t += nthr) {
          const int g = t / 128, c = (t % 128) / 64, jj = t % 64;
          const int j = j0 + jj;
          if (j >= a.r || g0 + g >= a.npairs) continue;
          T s = 0;
          for (int u = 0; u < wpp; ++u) s += red[(g * wpp + u) * 128 + c * 64 + jj];
          a.part[(((g0 + g) * ntiles + tile) * 2 + c) * a.rpad + j] = s;
        }
      });
    }
  }

  tile_fft<T, false>(ex, buf, a.log2P, ncols, a.tw);

  ex.phase([&](int tid, St &) {
    for (int e = tid; e < P * ncols; e += nthr) {
      const int k1 = e / ncols, col = e % ncols;
      const int g = col / a.NB, c = col % a.NB;
      if (g0 + g >= a.npairs) continue;
      const int64_t n2 = n2_0 + c;
      const c2<T> w = a.tw.template root<false>((uint64_t)n2 * (uint64_t)k1, a.log2M);
      a.inter[((g0 + g) * P + k1) * (int64_t)Q + n2] = cmul(buf[pad(e)], w);
    }
  });
}

// ---- reduce: a[pair][c][j] = D_j * sum over tiles of part[pair][tile][c][j] ---------
template <typename T>
FST_HD void reduce_body(const ConvArgs<T> &a, int64_t pl, int tid, int nthr) {
  const int Q = 1 << a.log2Q;
  const int ntiles = Q / a.NB;
  for (int t = tid; t < 2 * a.r; t += nthr) {
    const int c = t / a.r, j = t % a.r;
    T s = 0;
    for (int tile = 0; tile < ntiles; ++tile) s += a.part[((pl * ntiles + tile) * 2 + c) * a.rpad + j];
    a.acoef[(pl * 2 + c) * a.rpad + j] = ldg(a.D + j) * s;
  }
}

// ---- pass B: row k1 of pair pl: forward Q-point DFT, spectrum, inverse, twiddle -----
// smem: buf[padded_size(Q)] complex
template <typename T, typename Ex>
FST_HD void passB_body(Ex &ex, const ConvArgs<T> &a, int64_t pl, int k1, c2<T> *buf) {
  using St = typename Ex::State;
  const int P = 1 << a.log2P;
  const int Q = 1 << a.log2Q;
  const int nthr = ex.nthr;
  c2<T> *row = a.inter + ((pl * P) + k1) * (int64_t)Q;

  ex.phase([&](int tid, St &) {
    for (int i = tid; i < Q; i += nthr) buf[pad(i)] = row[i];
  });
  tile_fft<T, false>(ex, buf, a.log2Q, 1, a.tw);
  if (a.mode == MODE_FORWARD) {
    ex.phase([&](int tid, St &) {
      for (int i = tid; i < Q; i += nthr) row[i] = buf[pad(i)];
    });
    return;
  }
  ex.phase([&](int tid, St &) {
    const T *sp = spec_of(a, pl) + (int64_t)k1 * Q;
    for (int i = tid; i < Q; i += nthr) buf[pad(i)] = cscale(buf[pad(i)], ldg(sp + i));
  });
  tile_fft<T, true>(ex, buf, a.log2Q, 1, a.tw);
  ex.phase([&](int tid, St &) {
    for (int i = tid; i < Q; i += nthr) {
      const c2<T> w = a.tw.template root<true>((uint64_t)i * (uint64_t)k1, a.log2M);
      row[i] = cmul(buf[pad(i)], w);
    }
  });
}

// ---- pass C: inverse column DFTs over k1, first N samples + correction ----------------
// smem: buf[padded_size(P * ncols)] complex; the coefficients a = D o c are read
// from global memory (L1-resident broadcast)
template <typename T, typename Ex>
FST_HD void passC_body(Ex &ex, const ConvArgs<T> &a, int64_t tile, int64_t group, c2<T> *buf) {
  using St = typename Ex::State;
  const int P = 1 << a.log2P;
  const int Q = 1 << a.log2Q;
  const int ncols = a.G * a.NB;
  const int nthr = ex.nthr;
  const int64_t n2_0 = tile * a.NB;
  const int64_t g0 = group * a.G;
  const bool corr = (a.mode == MODE_FULL) && a.r > 0;

  ex.phase([&](int tid, St &) {
    for (int e = tid; e < P * ncols; e += nthr) {
      const int k1 = e / ncols, col = e % ncols;
      const int g = col / a.NB, c = col % a.NB;
      c2<T> v = mk<T>(0, 0);
      if (g0 + g < a.npairs) v = a.inter[((g0 + g) * P + k1) * (int64_t)Q + n2_0 + c];
      buf[pad(e)] = v;
    }
  });

  tile_fft<T, true>(ex, buf, a.log2P, ncols, a.tw);

  ex.phase([&](int tid, St &) {
    for (int e = tid; e < a.Pnz * ncols; e += nthr) {
      const int n1 = e / ncols, col = e % ncols;
      const int g = col / a.NB, c = col % a.NB;
      const int64_t n = (int64_t)n1 * Q + n2_0 + c;
      if (n >= a.N || g0 + g >= a.npairs) continue;
      c2<T> v = buf[pad(e)];
      if (corr) {
        const T *cg = a.acoef + (g0 + g) * 2 * a.rpad;
        v = cadd(v, corr_value(a, n, cg, cg + a.rpad));
      }
      store_pair(a, g0 + g, n, v);
    }
  });
}

}  // namespace fst
