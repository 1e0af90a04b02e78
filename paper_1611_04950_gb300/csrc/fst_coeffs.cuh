// fst_coeffs.cuh -- kernel bodies of the fast coefficient vector T2^* y of the fast
// factorization S_K S_K^* ~ T1 T2^* (Section 1.3; T2 = [F_{N,W}  L2  U2], L2 from the
// constructive proof of Theorem 1 in Section 2, U2 from the proof of Corollary 2).
//
//   F^* y : the length-N DFT bins k = -h..h (2h+1 = 2NW') divided by sqrt(N), from the
//           library's forward FFT (forward mode of the convolution kernels) + gather.
//   L2^* y: eight blocks, every column a real weight times a phase ramp:
//             (D_A J Z)^* y, (D_A Z)^* y, (D_A^* J Z)^* y, (D_A^* Z)^* y,
//             C_A V_A^T D_A^* y, C_A V_A^T D_A y, C_B V_B^T D_B^* y, C_B V_B^T D_B y,
//           with D_A = diag(exp(j 2 pi W' n)), D_B = diag(exp(j pi (W + W') n)),
//           Z the CF-ADI factor of the Hilbert matrix (columns by the recurrence of
//           the appendix, x = n + 1/2), V_A, V_B centred monomials u_n^i,
//           u_n = (n - (N-1)/2)/N.  The kernel forms the sums over n (partials per
//           n-chunk); the reduce kernel adds the chunks in a fixed order and applies
//           C_A, C_B.
//   U2^* y: sqrt|D_l| s_l^T y (partials per n-chunk, then a fixed-order reduce).
//
// and of its expansion T1 c (fst_expand), T1 = [F_{N,W}  L1  U1]:
//   F c_F : the bins scattered (conjugated) into a length-N row, the library's forward DFT,
//           conjugated and divided by sqrt(N) (= the inverse DFT restricted to -h..h).
//   L1 c_L: per sample, the same generated columns as above (ADI Z and J Z, centred monomials,
//           phase ramps D_A, D_B) summed against the eight coefficient blocks; no reduction
//           across samples.
//   U1 c_U: sum_l sign(D_l) sqrt|D_l| s_l c_U[l].
#pragma once
#include "fst_kernels.cuh"

namespace fst {

constexpr int COEF_THREADS = 256;
constexpr int COEF_E = 8;      // samples per thread per chunk
constexpr int COEF_CHUNK = COEF_THREADS * COEF_E;
constexpr int COEF_GROUP = 8;  // complex outputs reduced per round

template <typename T> struct CoefArgs {
  const T *y;        // signals (real rows of N, or complex rows of N pairs)
  int64_t ld, batch;
  int cplx;
  int64_t N;
  int rH, DA, DB;    // ADI rank, 2 r_A, 2 r_B - 1
  const T *zfirst;   // [rH]: zfirst[0] = sqrt(2 p_1); zfirst[k] = sqrt(p_{k+1}/p_k) (1-based p)
  const T *zshift;   // [rH]: p_k (k = 1..rH), 1-based p stored at [k-1]
  const c2<T> *phA;  // [N]: exp(-j 2 pi W' n)
  const c2<T> *phB;  // [N]: exp(-j pi (W + W') n)
  int nraw;          // raw outputs per signal: 4 rH + 2 DA + 2 DB
  int nchunks;
  T *part;           // [batch][nchunks][nraw][2]
  // U2 part
  const T *ST;       // [N][rpad]
  int r, rpad;
  T *partU;          // [batch][nchunks][r][2]
  int upairs;        // 1: U2^* y already reduced per pair in acoefU ([pair][re/im][rpad])
  const T *acoefU;
};

template <typename T> struct CState {
  c2<T> v[COEF_E];   // phase-multiplied samples
  T zf[COEF_E], zr[COEF_E], up[COEF_E];
  T acc[2 * COEF_GROUP];
};

// a / b: the device's fast FP32 division (2 ulp) for the ADI recurrence; exact otherwise
FST_HD float coef_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
FST_HD double coef_div(double a, double b) { return a / b; }

template <typename T> FST_HD c2<T> coef_sample(const CoefArgs<T> &a, int64_t sig, int64_t n) {
  if (a.cplx) return reinterpret_cast<const c2<T> *>(a.y)[sig * a.ld + n];
  return mk<T>(a.y[sig * a.ld + n], (T)0);
}

// Block-wide fixed-order reduction of every thread's acc[0 .. 2*cnt) into dst[0 .. 2*cnt).
// red: COEF_RED_WORDS reals of shared memory, laid out [q][COEF_RED_LD] (the thread values,
// rows padded by 16 so that both passes below are free of bank conflicts), then
// [q][COEF_RED_PARTS] part sums; dst may be red + COEF_RED_DST.  Part p of value q sums the
// thread values p, p + 16, p + 32, ... in that order; then the parts are summed in order.
constexpr int COEF_RED_PARTS = 16;
constexpr int COEF_RED_LD = COEF_THREADS + 16;
constexpr int COEF_RED_DST = 2 * COEF_GROUP * COEF_RED_LD + 2 * COEF_GROUP * COEF_RED_PARTS;
constexpr int COEF_RED_WORDS = COEF_RED_DST + 2 * COEF_GROUP;
static_assert(2 * COEF_GROUP * COEF_RED_PARTS <= COEF_THREADS, "one thread per (value, part)");
template <typename T, typename Ex>
FST_HD void coef_block_reduce(Ex &ex, T *red, int cnt, T *dst) {
  using St = typename Ex::State;
  ex.phase([&](int tid, St &st) {
#pragma unroll
    for (int q = 0; q < 2 * COEF_GROUP; ++q)
      if (q < 2 * cnt) red[q * COEF_RED_LD + tid] = st.acc[q];
  });
  ex.phase([&](int tid, St &) {
    const int q = tid / COEF_RED_PARTS, pidx = tid % COEF_RED_PARTS;
    if (q < 2 * cnt) {
      T s = 0;
#pragma unroll
      for (int i = 0; i < COEF_THREADS / COEF_RED_PARTS; ++i) s += red[q * COEF_RED_LD + pidx + COEF_RED_PARTS * i];
      red[2 * COEF_GROUP * COEF_RED_LD + q * COEF_RED_PARTS + pidx] = s;
    }
  });
  ex.phase([&](int tid, St &) {
    if (tid < 2 * cnt) {
      T s = 0;
      for (int pidx = 0; pidx < COEF_RED_PARTS; ++pidx)
        s += red[2 * COEF_GROUP * COEF_RED_LD + tid * COEF_RED_PARTS + pidx];
      dst[tid] = s;
    }
  });
}

// Raw low-rank sums of one signal over one chunk of samples.
// Output order (complex): [b2 | b1 | qA-] for the D_A^* y variant, then
// [b4 | b3 | qA+] for D_A y, then qB- (D_B^* y) and qB+ (D_B y), where
// bZ = sum Z(n) v(n), bJ = sum Z(N-1-n) v(n), q[i] = sum u_n^i v(n).
template <typename T, typename Ex>
FST_HD void coef_lowrank_body(Ex &ex, const CoefArgs<T> &a, int64_t sig, int chunk, T *red) {
  using St = typename Ex::State;
  const int nthr = ex.nthr;
  const int64_t n0 = (int64_t)chunk * COEF_CHUNK;
  T *out = a.part + ((sig * a.nchunks + chunk) * a.nraw) * 2;
  const T half = (T)0.5, Nd = (T)a.N, cen = (T)(0.5 * (double)(a.N - 1)), invN = (T)(1.0 / (double)a.N);
  const int vbase[4] = {0, 2 * a.rH + a.DA, 4 * a.rH + 2 * a.DA, 4 * a.rH + 2 * a.DA + a.DB};
  for (int variant = 0; variant < 4; ++variant) {
    const bool useA = variant < 2, conjph = (variant & 1) != 0;
    // real input: the D_A y and D_B y sums are the conjugates of the D_A^* y, D_B^* y ones
    if (!a.cplx && conjph) continue;
    int obase = vbase[variant];
    // v(n) = phase(n) y(n) with phase = exp(-j..) (conjph: exp(+j..)); reset recurrences
    ex.phase([&](int tid, St &st) {
#pragma unroll
      for (int e = 0; e < COEF_E; ++e) {
        const int64_t n = n0 + tid + (int64_t)e * nthr;
        c2<T> v = mk<T>(0, 0);
        T zf = 0, zr = 0;
        if (n < a.N) {
          c2<T> ph = useA ? a.phA[n] : a.phB[n];
          if (conjph) ph = cconj(ph);
          v = cmul(ph, coef_sample(a, sig, n));
          const T x = (T)n + half, xr = Nd - x;      // x for n and for N-1-n
          zf = coef_div(a.zfirst[0], x + a.zshift[0]);
          zr = coef_div(a.zfirst[0], xr + a.zshift[0]);
        }
        st.v[e] = v;
        st.zf[e] = zf;
        st.zr[e] = zr;
        st.up[e] = (T)1;
      }
    });
    if (useA) {
      // Z columns, COEF_GROUP / 2 of them per round (two outputs each: Z and JZ)
      for (int k0 = 0; k0 < a.rH; k0 += COEF_GROUP / 2) {
        const int kc = (a.rH - k0 < COEF_GROUP / 2) ? a.rH - k0 : COEF_GROUP / 2;
        ex.phase([&](int tid, St &st) {
#pragma unroll
          for (int q = 0; q < 2 * COEF_GROUP; ++q) st.acc[q] = 0;
#pragma unroll
          for (int kk = 0; kk < COEF_GROUP / 2; ++kk) {
            if (kk >= kc) break;
            const int k = k0 + kk;
#pragma unroll
            for (int e = 0; e < COEF_E; ++e) {
              const int64_t n = n0 + tid + (int64_t)e * nthr;
              if (k > 0 && n < a.N) {
                const T x = (T)n + half, xr = Nd - x;
                const T pk = a.zshift[k], pk1 = a.zshift[k - 1], sc = a.zfirst[k];
                st.zf[e] = coef_div(sc * (x - pk1) * st.zf[e], x + pk);
                st.zr[e] = coef_div(sc * (xr - pk1) * st.zr[e], xr + pk);
              }
              st.acc[4 * kk + 0] += st.zf[e] * st.v[e].x;
              st.acc[4 * kk + 1] += st.zf[e] * st.v[e].y;
              st.acc[4 * kk + 2] += st.zr[e] * st.v[e].x;
              st.acc[4 * kk + 3] += st.zr[e] * st.v[e].y;
            }
          }
        });
        T res[2 * COEF_GROUP];
        coef_block_reduce<T>(ex, red, 2 * kc, red + COEF_RED_DST);
        ex.phase([&](int tid, St &) {
          const T *r = red + COEF_RED_DST;
          if (tid < kc) {
            const int k = k0 + tid;
            out[2 * (obase + k)] = r[4 * tid + 0];                 // sum Z v
            out[2 * (obase + k) + 1] = r[4 * tid + 1];
            out[2 * (obase + a.rH + k)] = r[4 * tid + 2];          // sum JZ v
            out[2 * (obase + a.rH + k) + 1] = r[4 * tid + 3];
          }
        });
        (void)res;
      }
      obase += 2 * a.rH;
    }
    (void)obase;
    // monomials u^i, i < D
    const int D = useA ? a.DA : a.DB;
    for (int i0 = 0; i0 < D; i0 += COEF_GROUP) {
      const int ic = (D - i0 < COEF_GROUP) ? D - i0 : COEF_GROUP;
      ex.phase([&](int tid, St &st) {
#pragma unroll
        for (int q = 0; q < 2 * COEF_GROUP; ++q) st.acc[q] = 0;
#pragma unroll
        for (int ii = 0; ii < COEF_GROUP; ++ii) {
          if (ii >= ic) break;
#pragma unroll
          for (int e = 0; e < COEF_E; ++e) {
            const int64_t n = n0 + tid + (int64_t)e * nthr;
            const T u = ((T)n - cen) * invN;
            if (i0 + ii > 0) st.up[e] *= u;
            st.acc[2 * ii] += st.up[e] * st.v[e].x;
            st.acc[2 * ii + 1] += st.up[e] * st.v[e].y;
          }
        }
      });
      coef_block_reduce<T>(ex, red, ic, red + COEF_RED_DST);
      ex.phase([&](int tid, St &) {
        const T *r = red + COEF_RED_DST;
        if (tid < ic) {
          out[2 * (obase + i0 + tid)] = r[2 * tid];
          out[2 * (obase + i0 + tid) + 1] = r[2 * tid + 1];
        }
      });
    }
  }
  if (!a.cplx) {
    ex.phase([&](int tid, St &) {
      const int n0c = 2 * a.rH + a.DA, n2c = a.DB;
      for (int i = tid; i < n0c + n2c; i += nthr) {
        const int src = (i < n0c) ? vbase[0] + i : vbase[2] + (i - n0c);
        const int dst = (i < n0c) ? vbase[1] + i : vbase[3] + (i - n0c);
        out[2 * dst] = out[2 * src];
        out[2 * dst + 1] = -out[2 * src + 1];
      }
    });
  }
}

// S_T^T y partial sums of one signal over one chunk: warps split the samples, lanes
// split j (j = lane + 32 q).  red: nwarps * 2 * 64 reals.
template <typename T, typename Ex>
FST_HD void coef_st_body(Ex &ex, const CoefArgs<T> &a, int64_t sig, int chunk, T *red) {
  using St = typename Ex::State;
  const int nthr = ex.nthr, nwarps = nthr / 32;
  const int64_t n0 = (int64_t)chunk * COEF_CHUNK;
  const int64_t n1 = (n0 + COEF_CHUNK < a.N) ? n0 + COEF_CHUNK : a.N;
  for (int j0 = 0; j0 < a.r; j0 += 64) {
    ex.phase([&](int tid, St &) {
      const int w = tid >> 5, lane = tid & 31;
      T acc[4] = {0, 0, 0, 0};
      const int ja = j0 + lane, jb = j0 + lane + 32;
      for (int64_t n = n0 + w; n < n1; n += nwarps) {
        const c2<T> v = coef_sample(a, sig, n);
        const T *row = a.ST + n * a.rpad;
        const T sa = (ja < a.r) ? ldg(row + ja) : (T)0;
        const T sb = (jb < a.r) ? ldg(row + jb) : (T)0;
        acc[0] += sa * v.x; acc[1] += sa * v.y;
        acc[2] += sb * v.x; acc[3] += sb * v.y;
      }
      T *rw = red + w * 128;
      rw[2 * lane] = acc[0]; rw[2 * lane + 1] = acc[1];
      rw[64 + 2 * lane] = acc[2]; rw[64 + 2 * lane + 1] = acc[3];
    });
    ex.phase([&](int tid, St &) {
      if (tid < 128) {
        const int jj = tid >> 1, c = tid & 1;   // output j0 + jj, component c
        T s = 0;
        for (int w = 0; w < nwarps; ++w) s += red[w * 128 + 2 * jj + c];
        const int j = j0 + jj;
        if (j < a.r) a.partU[((sig * a.nchunks + chunk) * a.r + j) * 2 + c] = s;
      }
    });
  }
}

// F^* y bins of signal `sig` for k = -h..h from the forward DFT X of its pair
// (natural index kk stored at pos(kk) of the forward layout): real pairs split as
// X_a = (Z[kk] + conj Z[-kk]) / 2, X_b = (Z[kk] - conj Z[-kk]) / (2j).
template <typename T>
FST_HD void coef_gather_body(const c2<T> *X, const Layout &Lf, int64_t N, int cplx, int64_t sig, int64_t pl,
                             int64_t h, int64_t k, c2<T> *out) {
  const int64_t kk = ((k - h) % N + N) % N;
  const int64_t nk = (N - kk) % N;
  const c2<T> *Xp = X + pl * N;
  const c2<T> z = Xp[spec_pos(Lf, kk)];
  c2<T> v;
  if (cplx) {
    v = z;
  } else {
    const c2<T> zc = cconj(Xp[spec_pos(Lf, nk)]);
    if ((sig & 1) == 0) v = cscale(cadd(z, zc), (T)0.5);
    else {
      const c2<T> d = csub(z, zc);
      v = mk<T>((T)0.5 * d.y, (T)(-0.5) * d.x);     // d / (2j)
    }
  }
  const T s = (T)(1.0 / sqrt((double)N));
  out[k] = cscale(v, s);
}

// totals[sig][o] = sum over chunks (fixed order) of part[sig][chunk][o]
template <typename T>
FST_HD void coef_reduce_body(const T *part, int nchunks, int nout, int64_t sig, int o, T *tot) {
  T sr = 0, si = 0;
  for (int c = 0; c < nchunks; ++c) {
    const T *q = part + ((sig * nchunks + c) * (int64_t)nout + o) * 2;
    sr += q[0];
    si += q[1];
  }
  tot[(sig * (int64_t)nout + o) * 2] = sr;
  tot[(sig * (int64_t)nout + o) * 2 + 1] = si;
}

// final L2^* y and U2^* y entries (index o in [0, r1 + r)) from the raw totals
template <typename T>
FST_HD c2<T> coef_mix_value(const CoefArgs<T> &a, const T *raw, const T *rawU, const T *CA, const T *CB,
                            const T *sqrtD, int o, int64_t sig) {
  const int rH = a.rH, DA = a.DA, DB = a.DB;
  auto R = [&](int i) { return mk<T>(raw[2 * i], raw[2 * i + 1]); };
  const int r1 = 4 * rH + 2 * DA + 2 * DB;
  if (o < rH) return R(rH + o);                                  // (D_A J Z)^* y
  if (o < 2 * rH) return R(o - rH);                              // (D_A Z)^* y
  if (o < 3 * rH) return R(2 * rH + DA + rH + (o - 2 * rH));     // (D_A^* J Z)^* y
  if (o < 4 * rH) return R(2 * rH + DA + (o - 3 * rH));          // (D_A^* Z)^* y
  if (o < r1) {
    int base, D, i;
    const T *C;
    if (o < 4 * rH + DA) { i = o - 4 * rH; base = 2 * rH; D = DA; C = CA; }                     // C_A qA-
    else if (o < 4 * rH + 2 * DA) { i = o - 4 * rH - DA; base = 4 * rH + DA; D = DA; C = CA; }   // C_A qA+
    else if (o < 4 * rH + 2 * DA + DB) { i = o - 4 * rH - 2 * DA; base = 4 * rH + 2 * DA; D = DB; C = CB; }
    else { i = o - 4 * rH - 2 * DA - DB; base = 4 * rH + 2 * DA + DB; D = DB; C = CB; }
    T sr = 0, si = 0;
    for (int l = 0; l < D; ++l) {
      const T c = C[i * D + l];
      sr += c * raw[2 * (base + l)];
      si += c * raw[2 * (base + l) + 1];
    }
    return mk<T>(sr, si);
  }
  const int j = o - r1;
  if (a.upairs) {
    // sqrt|D| already applied; real pairs hold signals 2p (re part) and 2p+1 (im part)
    if (a.cplx) return mk<T>(a.acoefU[(sig * 2) * a.rpad + j], a.acoefU[(sig * 2 + 1) * a.rpad + j]);
    return mk<T>(a.acoefU[((sig / 2) * 2 + (sig & 1)) * a.rpad + j], (T)0);
  }
  return mk<T>(sqrtD[j] * rawU[2 * j], sqrtD[j] * rawU[2 * j + 1]);
}

// ---------------------------------------------------------------------------
// T1 c (fst_expand)
// ---------------------------------------------------------------------------
template <typename T> struct ExpArgs {
  const c2<T> *coef;    // [batch][Kp]: F bins k = -h..h, L blocks b1..b8, U part
  int64_t Kp, h, N;
  int rH, DA, DB, r, rpad;
  const T *zfirst, *zshift;   // ADI recurrence factors (as CoefArgs)
  const c2<T> *phA, *phB;     // exp(-j 2 pi W' n) = conj(D_A), exp(-j pi (W + W') n) = conj(D_B)
  const T *ST;                // [N][rpad]
  const T *D, *sqrtD;         // [r]
  const c2<T> *X;             // forward DFT of the launch group's scattered rows, layout Lf
  Layout Lf;
  int64_t sig0;               // first signal of the launch group
  c2<T> *out;                 // [batch][N]
};

// row sl of the launch group: Xs[n] = conj(c_F[k]) at the bin k = n (n <= h) or n - N
// (n >= N - h), zero elsewhere (2h + 1 <= N, so the two ranges do not meet)
template <typename T> FST_HD void exp_scatter_body(const ExpArgs<T> &a, int64_t sl, int64_t n, c2<T> *Xs) {
  const int64_t k = (n <= a.h) ? n : n - a.N;
  c2<T> v = mk<T>(0, 0);
  if (k >= -a.h && k <= a.h) v = cconj(a.coef[(a.sig0 + sl) * a.Kp + (k + a.h)]);
  Xs[sl * a.N + n] = v;
}

// (T1 c)[n] of signal sig0 + sl for the EXP_E samples n = n0 + i stride (i < EXP_E, n < N):
// every coefficient and table value is loaded once for all of them
constexpr int EXP_E = 4;
template <typename T> FST_HD void exp_samples_body(const ExpArgs<T> &a, int64_t sl, int64_t n0, int64_t stride) {
  const int64_t sig = a.sig0 + sl;
  const c2<T> *b1 = a.coef + sig * a.Kp + (2 * a.h + 1);
  const c2<T> *b2 = b1 + a.rH, *b3 = b2 + a.rH, *b4 = b3 + a.rH, *b5 = b4 + a.rH;
  const c2<T> *b6 = b5 + a.DA, *b7 = b6 + a.DA, *b8 = b7 + a.DB, *cu = b8 + a.DB;
  int64_t n[EXP_E];
  bool ok[EXP_E];
#pragma unroll
  for (int i = 0; i < EXP_E; ++i) {
    n[i] = n0 + i * stride;
    ok[i] = n[i] < a.N;
    if (!ok[i]) n[i] = a.N - 1;   // computed, not stored
  }
  // Z_k at x = n + 1/2 and at N - x (J Z), by the recurrence of the coefficient kernels
  T x[EXP_E], xr[EXP_E], zf[EXP_E], zr[EXP_E];
  c2<T> s1[EXP_E], s2[EXP_E], s3[EXP_E], s4[EXP_E];
#pragma unroll
  for (int i = 0; i < EXP_E; ++i) {
    x[i] = (T)n[i] + (T)0.5;
    xr[i] = (T)a.N - x[i];
    zf[i] = coef_div(a.zfirst[0], x[i] + a.zshift[0]);
    zr[i] = coef_div(a.zfirst[0], xr[i] + a.zshift[0]);
    s1[i] = s2[i] = s3[i] = s4[i] = mk<T>(0, 0);
  }
  for (int k = 0; k < a.rH; ++k) {
    const T pk = a.zshift[k], pk1 = k > 0 ? a.zshift[k - 1] : (T)0, sc = a.zfirst[k];
    const c2<T> c1 = b1[k], c2v = b2[k], c3 = b3[k], c4 = b4[k];
#pragma unroll
    for (int i = 0; i < EXP_E; ++i) {
      if (k > 0) {
        zf[i] = coef_div(sc * (x[i] - pk1) * zf[i], x[i] + pk);
        zr[i] = coef_div(sc * (xr[i] - pk1) * zr[i], xr[i] + pk);
      }
      s1[i] = cadd(s1[i], cscale(c1, zf[i]));
      s2[i] = cadd(s2[i], cscale(c2v, zr[i]));
      s3[i] = cadd(s3[i], cscale(c3, zf[i]));
      s4[i] = cadd(s4[i], cscale(c4, zr[i]));
    }
  }
  // centred monomials u^i, u = (n - (N - 1)/2) / N
  T u[EXP_E], up[EXP_E];
  c2<T> m5[EXP_E], m6[EXP_E], m7[EXP_E], m8[EXP_E];
#pragma unroll
  for (int i = 0; i < EXP_E; ++i) {
    u[i] = ((T)n[i] - (T)(0.5 * (double)(a.N - 1))) * (T)(1.0 / (double)a.N);
    up[i] = 1;
    m5[i] = m6[i] = m7[i] = m8[i] = mk<T>(0, 0);
  }
  const int D = a.DA > a.DB ? a.DA : a.DB;
  for (int d = 0; d < D; ++d) {
    const bool inA = d < a.DA, inB = d < a.DB;
    const c2<T> c5 = inA ? b5[d] : mk<T>(0, 0), c6 = inA ? b6[d] : mk<T>(0, 0);
    const c2<T> c7 = inB ? b7[d] : mk<T>(0, 0), c8 = inB ? b8[d] : mk<T>(0, 0);
#pragma unroll
    for (int i = 0; i < EXP_E; ++i) {
      m5[i] = cadd(m5[i], cscale(c5, up[i]));
      m6[i] = cadd(m6[i], cscale(c6, up[i]));
      m7[i] = cadd(m7[i], cscale(c7, up[i]));
      m8[i] = cadd(m8[i], cscale(c8, up[i]));
      up[i] *= u[i];
    }
  }
  // U1 c_U: weights sign(D) sqrt|D| c_U[j], applied to the S_T rows of the samples
  c2<T> v[EXP_E];
#pragma unroll
  for (int i = 0; i < EXP_E; ++i) v[i] = mk<T>(0, 0);
  for (int j = 0; j < a.r; ++j) {
    const c2<T> w = cscale(cu[j], a.D[j] < 0 ? -a.sqrtD[j] : a.sqrtD[j]);
#pragma unroll
    for (int i = 0; i < EXP_E; ++i) v[i] = cadd(v[i], cscale(w, a.ST[n[i] * a.rpad + j]));
  }
  // L1 c_L = D_A (c (s1 - s2) + m5 / 2j) + D_A^* (c (s4 - s3) - m6 / 2j) + D_B m7 / 2 + D_B^* m8 / 2,
  // c = 1 / (2 j pi) = -j / (2 pi), 1 / 2j = -j / 2; then F c_F = conj(DFT_N(conj bins)) / sqrt(N)
  const T ip = (T)0.15915494309189533577;   // 1 / (2 pi)
  const T rs = (T)(1.0 / sqrt((double)a.N));
#pragma unroll
  for (int i = 0; i < EXP_E; ++i) {
    if (!ok[i]) continue;
    const c2<T> dA = cconj(a.phA[n[i]]), dB = cconj(a.phB[n[i]]);
    const c2<T> d12 = csub(s1[i], s2[i]), d43 = csub(s4[i], s3[i]);
    const c2<T> tA = mk<T>(ip * d12.y + (T)0.5 * m5[i].y, -ip * d12.x - (T)0.5 * m5[i].x);
    const c2<T> tC = mk<T>(ip * d43.y - (T)0.5 * m6[i].y, -ip * d43.x + (T)0.5 * m6[i].x);
    c2<T> r = cadd(v[i], cadd(cmul(dA, tA), cmul(cconj(dA), tC)));
    r = cadd(r, cadd(cmul(dB, cscale(m7[i], (T)0.5)), cmul(cconj(dB), cscale(m8[i], (T)0.5))));
    const c2<T> xf = a.X[sl * a.N + spec_pos(a.Lf, n[i])];
    r = cadd(r, cscale(cconj(xf), rs));
    a.out[sig * a.N + n[i]] = r;
  }
}
}  // namespace fst
