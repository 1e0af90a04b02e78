// fst_plan_kernels.cuh -- FP64 plan-time kernel bodies: the Slepian basis vectors
// of the eigen-window around K (precomputation paragraph of Section 1.3).
//
// The DPSS are the eigenvectors of Slepian's tridiagonal matrix T_{N,W}
// (diag ((N-1)/2 - n)^2 cos(2 pi W), off-diagonal n (N - n) / 2), which commutes
// with the prolate matrix B_{N,W}; its l-th largest eigenvector is s^(l).  T is
// centro-symmetric, so its eigenvectors are symmetric (even l) or antisymmetric
// (odd l) and each parity is the eigenproblem of a tridiagonal matrix of half the
// size ("reduced" matrices, built on the host):
//   N = 2m:    both parities: leading m x m block, last diagonal d[m-1] +- e[m].
//   N = 2m+1:  symmetric: leading (m+1) x (m+1) block with the coupling between
//              m-1 and m multiplied by sqrt(2) (the centre sample is sqrt(2) u_m);
//              antisymmetric: leading m x m block (the centre sample is 0).
// Bodies here: multisection bisection on Sturm counts, inverse iteration with
// partially pivoted tridiagonal LU, and the expansion of a reduced vector to the
// unit-norm, sign-fixed full vector.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>
#include "fst_fft.cuh"

namespace fst {

constexpr int BISECT_THREADS = 64;
constexpr int BISECT_MS_MAX_TARGETS = 512;   // batches up to this many targets use multisection
constexpr int BISECT_MAX_ROUNDS = 24;

// biased exponent field of a double (0 for zeros and subnormals)
FST_HD int dexp_field(double v) {
#ifdef __CUDA_ARCH__
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
#else
  uint64_t u;
  memcpy(&u, &v, 8);
  return (int)((u >> 52) & 0x7ff);
#endif
}

// Number of eigenvalues of the reduced matrix smaller than x: the sign changes of the Sturm
// sequence of leading principal minors p_i = det(T_i - x I), p_i = (d_i - x) p_{i-1} -
// e_i^2 p_{i-2} (p_{-1} = 1), which equal the negative pivots q_i = p_i / p_{i-1} of
// T - x I = L D L^T.  The recurrence needs no division (the serial chain is one FMA per step);
// every 4 steps the pair (p_i, p_{i-1}) is rescaled by an exact power of two when both are
// beyond 2^(+-400) (a step grows them by at most about 2^87 for N <= 2^23), and an exact zero
// p_i is replaced by -pivmin p_{i-1} (the pivot -pivmin of the LDL^T form).
FST_HD int sturm_count(const double *d, const double *e2, int n, double x, double pivmin) {
  double pm = 1.0, p = ldg(d) - x;
  if (p == 0.0) p = -pivmin;
  int c = (p < 0.0);
  for (int i = 1; i < n; ++i) {
    const double t = ldg(e2 + i) * pm;
    double pn = fma(ldg(d + i) - x, p, -t);
    if (pn == 0.0) pn = -pivmin * p;
    c += ((pn < 0.0) != (p < 0.0));
    pm = p;
    p = pn;
    if ((i & 3) == 0) {
      const int ex = dexp_field(p), exm = dexp_field(pm);
      const int mx = ex > exm ? ex : exm;
      if (mx > 1023 + 400) {
        p *= 0x1p-512;
        pm *= 0x1p-512;
      } else if (mx < 1023 - 400) {
        p *= 0x1p512;
        pm *= 0x1p512;
      }
    }
  }
  return c;
}

struct BisectShared {
  double lo, hi;
  int done;
  int cnt[BISECT_THREADS];
};

// Block computes the eigenvalue of ascending index `target` of the reduced matrix:
// each round evaluates the Sturm count at 64 interior points of [lo, hi] and keeps
// the sub-interval that holds it (6 bits per round), until the interval is within 4 ulp
// of its ends plus abstol (about eps ||T||: an eigenvalue near 0, e.g. every transition
// eigenvalue at W = 1/4 where the diagonal vanishes, needs no more for the inverse
// iteration).  flag != 0 on non-convergence.
template <typename Ex>
FST_HD void bisect_body(Ex &ex, const double *d, const double *e2, int n, int target, double glo, double ghi,
                        double pivmin, double abstol, double *out, int *flag, BisectShared *sh) {
  using St = typename Ex::State;
  ex.phase([&](int tid, St &) {
    if (tid == 0) { sh->lo = glo; sh->hi = ghi; sh->done = 0; }
  });
  for (int round = 0; round < BISECT_MAX_ROUNDS; ++round) {
    ex.phase([&](int tid, St &) {
      const double lo = sh->lo, hi = sh->hi;
      const double x = lo + (hi - lo) * (double)(tid + 1) / (double)(BISECT_THREADS + 1);
      sh->cnt[tid] = sturm_count(d, e2, n, x, pivmin);
    });
    ex.phase([&](int tid, St &) {
      if (tid == 0) {
        const double lo = sh->lo, hi = sh->hi;
        int t = 0;
        while (t < BISECT_THREADS && sh->cnt[t] <= target) ++t;
        // count(x_t) > target >= count(x_{t-1}): eigenvalue in [x_{t-1}, x_t]
        const double nlo = (t == 0) ? lo : lo + (hi - lo) * (double)t / (double)(BISECT_THREADS + 1);
        const double nhi = (t == BISECT_THREADS) ? hi : lo + (hi - lo) * (double)(t + 1) / (double)(BISECT_THREADS + 1);
        sh->lo = nlo;
        sh->hi = nhi;
        const double tol = 4.0 * 2.220446049250313e-16 * fmax(fabs(nlo), fabs(nhi)) + abstol;
        if (nhi - nlo <= tol || (nlo == lo && nhi == hi)) sh->done = 1;
      }
    });
    if (sh->done) break;
  }
  ex.phase([&](int tid, St &) {
    if (tid == 0) {
      *out = 0.5 * (sh->lo + sh->hi);
      if (!sh->done) *flag = 1;
    }
  });
}

// Plain bisection for one target (one thread), used when many plans are built at
// once: the throughput of thousands of independent targets matters more than the
// latency of one.  flag != 0 if it did not converge.
FST_HD void bisect1_body(const double *d, const double *e2, int n, int target, double glo, double ghi, double pivmin,
                         double abstol, double *out, int *flag) {
  double lo = glo, hi = ghi;
  int it = 0;
  for (; it < 256; ++it) {
    const double tol = 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)) + abstol;
    if (hi - lo <= tol) break;
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(d, e2, n, mid, pivmin) > target) hi = mid;
    else lo = mid;
  }
  *out = 0.5 * (lo + hi);
  if (it == 256) *flag = 1;
}

// Descriptor of one eigen-target of a batch of plans (fst_plan_many).
struct TargetDesc {
  int64_t mat_off;   // reduced matrix: d, e, e2 at [mat_off, mat_off + n) of the concatenations
  int64_t x_off;     // this target's vector and factor arrays at [x_off, x_off + n)
  double *S;         // output: the full unit-norm Slepian vector (length N)
  int64_t N;
  int n, target, parity, pad_;
  double glo, ghi, pivmin, tol;
};

// Inverse iteration for one eigenvalue sigma of the reduced matrix (diag d,
// coupling e[i] between i-1 and i): LU with partial pivoting of T - sigma I (the
// classical tridiagonal elimination; row interchanges create a second
// superdiagonal), zero pivots lifted to tol, then `iters` solves with the same
// factors, each followed by scaling to max-norm 1.  Vector t of nt: element i at
// [i * nt + t] in x and in the factor arrays.  fd holds the reciprocals of the
// (lifted) U diagonal, so the back substitution multiplies.
//
// Each phase is a serial chain over i.  The entries a step updates travel to the next
// step in registers (cd, cu: U diagonal and super-diagonal at i; cur: x[i]; x1, x2:
// x[i+1], x[i+2]), and the inputs of the next INVIT_B steps are loaded while the current
// ones are processed (the loads never touch an entry the current block writes), so the
// chain waits on arithmetic, not on memory.
constexpr int INVIT_B = 8;
FST_HD void invit_body(const double *d, const double *e, int n, double sigma, double tol, int iters, int t, int nt,
                       double *x, double *fd, double *fdl, double *fdu, double *fdu2, uint8_t *piv) {
#define AT(a, i) a[(int64_t)(i) * nt + t]
  constexpr int B = INVIT_B;
  auto lift = [&](double p) { return (fabs(p) < tol) ? ((p < 0.0) ? -tol : tol) : p; };
  // ---- factor: steps i = 0 .. n-2 read e[i+1], d[i+1], e[i+2]
  {
    double cd = ldg(d) - sigma;
    double cu = (n > 1) ? ldg(e + 1) : 0.0;
    double E[B + 1], D[B];
    auto load = [&](int i0, double *Ev, double *Dv) {
#pragma unroll
      for (int k = 0; k <= B; ++k) Ev[k] = (i0 + 1 + k < n) ? ldg(e + i0 + 1 + k) : 0.0;
#pragma unroll
      for (int k = 0; k < B; ++k) Dv[k] = (i0 + 1 + k < n) ? ldg(d + i0 + 1 + k) : 0.0;
    };
    load(0, E, D);
    for (int i0 = 0; i0 + 1 < n; i0 += B) {
      double En[B + 1], Dn[B];
      load(i0 + B, En, Dn);
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int i = i0 + k;
        if (i + 1 < n) {
          const double li = E[k], nd = D[k] - sigma, nu = (i + 2 < n) ? E[k + 1] : 0.0;
          if (fabs(cd) >= fabs(li)) {
            const double f = (cd != 0.0) ? li / cd : 0.0;
            AT(fdl, i) = f;
            AT(fd, i) = 1.0 / lift(cd);
            AT(fdu, i) = cu;
            AT(fdu2, i) = 0.0;
            AT(piv, i) = 0;
            cd = nd - f * cu;
            cu = nu;
          } else {
            const double f = cd / li;
            AT(fdl, i) = f;
            AT(fd, i) = 1.0 / lift(li);
            AT(fdu, i) = nd;
            AT(fdu2, i) = nu;
            AT(piv, i) = 1;
            cd = cu - f * nd;
            cu = -f * nu;
          }
        }
      }
#pragma unroll
      for (int k = 0; k <= B; ++k) E[k] = En[k];
#pragma unroll
      for (int k = 0; k < B; ++k) D[k] = Dn[k];
    }
    AT(fd, n - 1) = 1.0 / lift(cd);
    AT(fdu, n - 1) = 0.0;
    AT(fdl, n - 1) = 0.0;
    AT(fdu2, n - 1) = 0.0;
    AT(piv, n - 1) = 0;
  }
  // start vector: deterministic, no structure shared with any eigenvector
  for (int i = 0; i < n; ++i) {
    const double g = (double)i * 0.6180339887498949;
    AT(x, i) = 0.5 + (g - floor(g));
  }
  for (int it = 0; it < iters; ++it) {
    // ---- L solve with the row interchanges: step i reads x[i+1] (not yet written), fdl[i], piv[i]
    {
      double cur = AT(x, 0);
      double X[B], L[B];
      unsigned PV;
      auto load = [&](int i0, double *Xv, double *Lv, unsigned &pv) {
        pv = 0u;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const bool ok = i0 + k + 1 < n;
          Xv[k] = ok ? AT(x, i0 + k + 1) : 0.0;
          Lv[k] = ok ? AT(fdl, i0 + k) : 0.0;
          pv |= (ok && AT(piv, i0 + k)) ? (1u << k) : 0u;
        }
      };
      load(0, X, L, PV);
      for (int i0 = 0; i0 + 1 < n; i0 += B) {
        double Xn[B], Ln[B];
        unsigned PVn;
        load(i0 + B, Xn, Ln, PVn);
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int i = i0 + k;
          if (i + 1 < n) {
            if (((PV >> k) & 1u) == 0u) {
              AT(x, i) = cur;
              cur = X[k] - L[k] * cur;
            } else {
              AT(x, i) = X[k];
              cur = cur - L[k] * X[k];
            }
          }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          X[k] = Xn[k];
          L[k] = Ln[k];
        }
        PV = PVn;
      }
      AT(x, n - 1) = cur;
    }
    // ---- U solve (descending), max-norm: step i reads x[i], fdu[i], fdu2[i], fd[i]
    double mx = 0.0;
    {
      double x1 = 0.0, x2 = 0.0;
      double X[B], U1[B], U2[B], R[B];
      auto load = [&](int i1, double *Xv, double *U1v, double *U2v, double *Rv) {
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int i = i1 - k;
          const bool ok = i >= 0;
          Xv[k] = ok ? AT(x, i) : 0.0;
          U1v[k] = ok ? AT(fdu, i) : 0.0;
          U2v[k] = ok ? AT(fdu2, i) : 0.0;
          Rv[k] = ok ? AT(fd, i) : 0.0;
        }
      };
      load(n - 1, X, U1, U2, R);
      for (int i1 = n - 1; i1 >= 0; i1 -= B) {
        double Xn[B], U1n[B], U2n[B], Rn[B];
        load(i1 - B, Xn, U1n, U2n, Rn);
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int i = i1 - k;
          if (i >= 0) {
            double v = X[k];
            if (i + 1 < n) v -= U1[k] * x1;
            if (i + 2 < n) v -= U2[k] * x2;
            v *= R[k];
            AT(x, i) = v;
            mx = fmax(mx, fabs(v));
            x2 = x1;
            x1 = v;
          }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          X[k] = Xn[k];
          U1[k] = U1n[k];
          U2[k] = U2n[k];
          R[k] = Rn[k];
        }
      }
    }
    const double s = (mx > 0.0) ? 1.0 / mx : 1.0;
    for (int i = 0; i < n; ++i) AT(x, i) = AT(x, i) * s;
  }
#undef AT
}

// Expansion of reduced vector t (interleaved x[i * nt + t], size n, parity p) to the
// full unit-norm Slepian vector s (length N, contiguous) with the sign convention:
// symmetric vectors have positive sum, antisymmetric ones positive
// sum((N-1-2i) s[i]).  Block reduction in a fixed order.  sh: 2 * nthr doubles.
template <typename Ex>
FST_HD void finalize_body(Ex &ex, const double *x, int n, int nt, int t, int parity, int64_t N, double *s, double *sh) {
  using St = typename Ex::State;
  const int nthr = ex.nthr;
  const bool odd = (N & 1) != 0;
  const int64_t m = N / 2;  // full index m is the centre when N is odd
  ex.phase([&](int tid, St &) {
    double nrm = 0.0, ref = 0.0;
    for (int i = tid; i < n; i += nthr) {
      const double u = x[(int64_t)i * nt + t];
      nrm += u * u;
      if (parity == 0) ref += (odd && i == m) ? 0.7071067811865476 * u : u;  // centre counts once, times sqrt(2)/2
      else ref += (double)(N - 1 - 2 * (int64_t)i) * u;
    }
    sh[tid] = nrm;
    sh[nthr + tid] = ref;
  });
  ex.phase([&](int tid, St &) {
    if (tid == 0) {
      double nrm = 0.0, ref = 0.0;
      for (int k = 0; k < nthr; ++k) { nrm += sh[k]; ref += sh[nthr + k]; }
      // full norm^2 = 2 * reduced norm^2 (centre sample sqrt(2) u_m when present)
      const double scale = (ref < 0.0 ? -1.0 : 1.0) / sqrt(2.0 * nrm);
      sh[0] = scale;
    }
  });
  ex.phase([&](int tid, St &) {
    const double scale = sh[0];
    const double sgn = (parity == 0) ? 1.0 : -1.0;
    for (int64_t i = tid; i < N; i += nthr) {
      double v;
      if (odd && i == m) {
        v = (parity == 0) ? 1.4142135623730951 * x[(int64_t)m * nt + t] * scale : 0.0;
      } else if (i < m || (odd && i < m)) {
        v = x[i * nt + t] * scale;
      } else {
        v = sgn * x[(N - 1 - i) * nt + t] * scale;
      }
      s[i] = v;
    }
  });
}

// sum_i a[i] * b[i] for vector t (contiguous, length N), fixed-order block reduction
template <typename Ex>
FST_HD void dot_body(Ex &ex, const double *a, const double *b, int64_t N, double *out, double *sh) {
  using St = typename Ex::State;
  const int nthr = ex.nthr;
  ex.phase([&](int tid, St &) {
    double acc = 0.0;
    for (int64_t i = tid; i < N; i += nthr) acc += a[i] * b[i];
    sh[tid] = acc;
  });
  ex.phase([&](int tid, St &) {
    if (tid == 0) {
      double acc = 0.0;
      for (int k = 0; k < nthr; ++k) acc += sh[k];
      *out = acc;
    }
  });
}

FST_HD double sinpi_hd(double x) {
#ifdef __CUDA_ARCH__
  return sinpi(x);
#else
  return sin(M_PI * x);
#endif
}

// b[k] = sin(2 pi W k) / (pi k), b[0] = 2W (first row of B_{N,W}, Eq. "Prolate
// matrix").  The product 2Wk is formed exactly as hi + lo (fma) and reduced mod 2
// before the sine, so large k lose no accuracy to the argument.
FST_HD double sinc_row_value(int64_t k, double W) {
  if (k == 0) return 2.0 * W;
  const double a = 2.0 * W, kd = (double)k;
  const double hi = a * kd;
  const double lo = fma(a, kd, -hi);
  double r = fmod(hi, 2.0) + lo;
  if (r > 1.0) r -= 2.0;
  return sinpi_hd(r) / (M_PI * kd);
}

// circulant embedding c of length M: c[k] = c[M-k] = b[k] for 0 <= k < N, else 0
FST_HD double sinc_embed_at(int64_t k, int64_t N, int64_t M, double W) {
  if (k < N) return sinc_row_value(k, W);
  if (k > M - N) return sinc_row_value(M - k, W);
  return 0.0;
}

}  // namespace fst
