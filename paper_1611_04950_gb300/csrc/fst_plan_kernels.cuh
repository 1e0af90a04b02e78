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
#include "fst_fft.cuh"

namespace fst {

constexpr int BISECT_THREADS = 64;
constexpr int BISECT_MAX_ROUNDS = 24;

// number of eigenvalues of the reduced matrix smaller than x (negative LDL^T pivots)
FST_HD int sturm_count(const double *d, const double *e2, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  c += (q < 0.0);
  for (int i = 1; i < n; ++i) {
    q = (ldg(d + i) - x) - ldg(e2 + i) / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += (q < 0.0);
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
// the sub-interval that holds it (6 bits per round).  flag != 0 on non-convergence.
template <typename Ex>
FST_HD void bisect_body(Ex &ex, const double *d, const double *e2, int n, int target, double glo, double ghi,
                        double pivmin, double *out, int *flag, BisectShared *sh) {
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
        const double tol = 4.0 * 2.220446049250313e-16 * fmax(fabs(nlo), fabs(nhi)) + pivmin;
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
                         double *out, int *flag) {
  double lo = glo, hi = ghi;
  int it = 0;
  for (; it < 256; ++it) {
    const double tol = 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)) + pivmin;
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
// [i * nt + t] in x and in the factor arrays (interleaved: coalesced across t).
FST_HD void invit_body(const double *d, const double *e, int n, double sigma, double tol, int iters, int t, int nt,
                       double *x, double *fd, double *fdl, double *fdu, double *fdu2, uint8_t *piv) {
#define AT(a, i) a[(int64_t)(i) * nt + t]
  // The elimination and both sweeps carry the entries they update from one step to the next in
  // registers (cd, cu: the current U diagonal and super-diagonal at i; cur: x[i]; x1, x2: x[i+1],
  // x[i+2]), so each step reads only inputs and the serial chain never waits on a memory round
  // trip.  Same operations, same order as the textbook in-place form.
  auto lift = [&](double p) { return (fabs(p) < tol) ? ((p < 0.0) ? -tol : tol) : p; };
  // factor: fd = U diagonal (zero pivots lifted to tol), fdu / fdu2 = U super-diagonals,
  // fdl = multipliers
  double cd = ldg(d) - sigma;
  double cu = (n > 1) ? ldg(e + 1) : 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double li = ldg(e + i + 1);
    const double nd = ldg(d + i + 1) - sigma;
    const double nu = (i + 2 < n) ? ldg(e + i + 2) : 0.0;
    if (fabs(cd) >= fabs(li)) {
      const double f = (cd != 0.0) ? li / cd : 0.0;
      AT(fdl, i) = f;
      AT(fd, i) = lift(cd);
      AT(fdu, i) = cu;
      AT(fdu2, i) = 0.0;
      AT(piv, i) = 0;
      cd = nd - f * cu;
      cu = nu;
    } else {
      const double f = cd / li;
      AT(fdl, i) = f;
      AT(fd, i) = lift(li);
      AT(fdu, i) = nd;
      AT(fdu2, i) = (i + 2 < n) ? nu : 0.0;
      AT(piv, i) = 1;
      cd = cu - f * nd;
      cu = (i + 2 < n) ? -f * nu : 0.0;
    }
  }
  AT(fd, n - 1) = lift(cd);
  AT(fdu, n - 1) = 0.0;
  AT(fdl, n - 1) = 0.0;
  AT(fdu2, n - 1) = 0.0;
  AT(piv, n - 1) = 0;
  // start vector: deterministic, no structure shared with any eigenvector
  for (int i = 0; i < n; ++i) {
    const double g = (double)i * 0.6180339887498949;
    AT(x, i) = 0.5 + (g - floor(g));
  }
  for (int it = 0; it < iters; ++it) {
    // L solve with the row interchanges
    double cur = AT(x, 0);
    for (int i = 0; i + 1 < n; ++i) {
      const double nx = AT(x, i + 1), l = AT(fdl, i);
      if (AT(piv, i) == 0) {
        AT(x, i) = cur;
        cur = nx - l * cur;
      } else {
        AT(x, i) = nx;
        cur = cur - l * nx;
      }
    }
    AT(x, n - 1) = cur;
    // U solve, max-norm
    double mx = 0.0, x1 = 0.0, x2 = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      double v = AT(x, i);
      if (i + 1 < n) v -= AT(fdu, i) * x1;
      if (i + 2 < n) v -= AT(fdu2, i) * x2;
      v /= AT(fd, i);
      AT(x, i) = v;
      mx = fmax(mx, fabs(v));
      x2 = x1;
      x1 = v;
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
