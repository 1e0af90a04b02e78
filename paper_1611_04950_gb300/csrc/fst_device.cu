// fst_device.cu -- CUDA back-end of the fast Slepian projection library (sm_103a):
// the __global__ wrappers of the kernel bodies, the device Runner, and the
// host-buffer entry point with overlapped copies.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "fst_internal.h"
#include "../../include/fst_testing.h"
#include "fst_fast.cuh"
#include "fst_big.cuh"
#define FST_TC_KERNELS
#include "fst_tc.cuh"

namespace fst {

template <typename T> struct DevEx {
  using State = KState<T>;
  int nthr;
  int tid;
  State st;
  __device__ DevEx() : nthr(blockDim.x), tid(threadIdx.x) {}
  template <typename F> __device__ __forceinline__ void phase(F &&f) {
    f(tid, st);
    __syncthreads();
  }
};

struct NoState {
  c2<double> v[1];
};
struct DevExPlan {
  using State = NoState;
  int nthr;
  int tid;
  State st;
  __device__ DevExPlan() : nthr(blockDim.x), tid(threadIdx.x) {}
  template <typename F> __device__ __forceinline__ void phase(F &&f) {
    f(tid, st);
    __syncthreads();
  }
};

template <typename S> struct DevExS {
  using State = S;
  int nthr;
  int tid;
  State st;
  __device__ DevExS() : nthr(blockDim.x), tid(threadIdx.x) {}
  template <typename F> __device__ __forceinline__ void phase(F &&f) {
    f(tid, st);
    __syncthreads();
  }
};

// ---------------------------------------------------------------------------
// apply kernels
// ---------------------------------------------------------------------------

template <typename T> __global__ void __launch_bounds__(1024) k_small(const ConvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = 1 << a.log2M;
  c2<T> *buf = reinterpret_cast<c2<T> *>(smem);
  T *red = reinterpret_cast<T *>(smem + padded_size(L) * sizeof(c2<T>));
  T *coef = red + ((blockDim.x + 31) / 32) * 128;
  DevEx<T> ex;
  small_body<T>(ex, a, (int64_t)blockIdx.x, buf, red, coef);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_small_ragged(const RaggedDesc<T> *d, const ConvArgs<T> base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = 1 << base.log2M;
  c2<T> *buf = reinterpret_cast<c2<T> *>(smem);
  T *red = reinterpret_cast<T *>(smem + padded_size(L) * sizeof(c2<T>));
  T *coef = red + ((blockDim.x + 31) / 32) * 128;
  const RaggedDesc<T> q = d[blockIdx.x];
  ConvArgs<T> a = base;
  a.y = q.y;
  a.out = q.out;
  a.ld = q.N;
  a.N = q.N;
  a.spec = q.spec;
  a.ST = q.ST;
  a.D = q.D;
  a.r = q.r;
  a.rpad = q.rpad;
  DevEx<T> ex;
  small_body<T>(ex, a, 0, buf, red, coef);
}

template <typename T> __global__ void __launch_bounds__(1024) k_passA(const ConvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int P = 1 << a.log2P;
  const int ncols = a.G * a.NB;
  c2<T> *buf = reinterpret_cast<c2<T> *>(smem);
  T *red = reinterpret_cast<T *>(smem + padded_size(P * ncols) * sizeof(c2<T>));
  DevEx<T> ex;
  passA_body<T>(ex, a, (int64_t)blockIdx.x, (int64_t)blockIdx.y, buf, red);
}

template <typename T> __global__ void k_reduce(const ConvArgs<T> a) {
  reduce_body<T>(a, (int64_t)blockIdx.x, threadIdx.x, blockDim.x);
}

template <typename T> __global__ void __launch_bounds__(1024) k_passB(const ConvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T> *buf = reinterpret_cast<c2<T> *>(smem);
  DevEx<T> ex;
  passB_body<T>(ex, a, (int64_t)blockIdx.y, (int)blockIdx.x, buf);
}

template <typename T> __global__ void __launch_bounds__(1024) k_passC(const ConvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T> *buf = reinterpret_cast<c2<T> *>(smem);
  DevEx<T> ex;
  passC_body<T>(ex, a, (int64_t)blockIdx.x, (int64_t)blockIdx.y, buf);
}

// ---------------------------------------------------------------------------
// plan kernels
// ---------------------------------------------------------------------------

__global__ void k_bisect_ms_many(const TargetDesc *td, const double *dcat, const double *e2cat, double *theta,
                                 int *flag) {
  __shared__ BisectShared sh;
  DevExPlan ex;
  const TargetDesc q = td[blockIdx.x];
  bisect_body(ex, dcat + q.mat_off, e2cat + q.mat_off, q.n, q.target, q.glo, q.ghi, q.pivmin, q.tol, theta + blockIdx.x,
              flag, &sh);
}

__global__ void k_bisect_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat, double *theta,
                              int *flag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const TargetDesc q = td[t];
  bisect1_body(dcat + q.mat_off, e2cat + q.mat_off, q.n, q.target, q.glo, q.ghi, q.pivmin, q.tol, theta + t, flag);
}
__global__ void k_invit_many(const TargetDesc *td, int nt, const double *dcat, const double *ecat,
                             const double *theta, double *x, double *fd, double *fdl, double *fdu, double *fdu2,
                             uint8_t *piv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const TargetDesc q = td[t];
  invit_body(dcat + q.mat_off, ecat + q.mat_off, q.n, theta[t], q.tol, 3, 0, 1, x + q.x_off, fd + q.x_off,
             fdl + q.x_off, fdu + q.x_off, fdu2 + q.x_off, piv + q.x_off);
}
__global__ void k_finalize_many(const TargetDesc *td, const double *x) {
  __shared__ double sh[2 * 256];
  DevExPlan ex;
  const TargetDesc q = td[blockIdx.x];
  finalize_body(ex, x + q.x_off, q.n, 1, 0, q.parity, q.N, q.S, sh);
}

__global__ void k_dot(const double *a, const double *b, int64_t N, double *out) {
  __shared__ double sh[256];
  DevExPlan ex;
  const int64_t off = (int64_t)blockIdx.x * N;
  dot_body(ex, a + off, b + off, N, out + blockIdx.x, sh);
}

__global__ void k_sinc(double *c, int64_t N, int64_t M, double W) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x)
    c[k] = sinc_embed_at(k, N, M, W);
}

__global__ void k_spec_store(const double2 *X, Layout L64, Layout L32, int64_t M, double scale, double *spec64,
                             float *spec32) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p64 = spec_pos(L64, k);
    const double v = X[p64].x * scale;
    spec64[p64] = v;
    spec32[spec_pos(L32, k)] = (float)v;
  }
}

__global__ void k_gather(const double *S, int64_t N, const int *sel, int r, int rpad, double *ST64, float *ST32) {
  const int64_t total = N * rpad;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / rpad;
    const int j = (int)(t % rpad);
    const double v = (j < r) ? S[(int64_t)sel[j] * N + n] : 0.0;
    ST64[t] = v;
    ST32[t] = (float)v;
  }
}

// ---- T1 c (fst_expand) ----
template <typename T> __global__ void k_exp_scatter(const ExpArgs<T> a, int64_t nsig, c2<T> *Xs) {
  const int64_t total = nsig * a.N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    exp_scatter_body<T>(a, t / a.N, t % a.N, Xs);
}
// block b of a signal row: samples b (EXP_E 256) + tid + i 256, i < EXP_E
template <typename T> __global__ void __launch_bounds__(256) k_expand(const ExpArgs<T> a, int64_t nsig) {
  const int64_t per = (a.N + EXP_E * 256 - 1) / (EXP_E * 256);
  for (int64_t bb = blockIdx.x; bb < nsig * per; bb += gridDim.x)
    exp_samples_body<T>(a, bb / per, (bb % per) * (EXP_E * 256) + threadIdx.x, 256);
}

// ---- fast coefficient vector kernels ----
template <typename T> __global__ void __launch_bounds__(COEF_THREADS) k_coef_lowrank(const CoefArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  DevExS<CState<T>> ex;
  coef_lowrank_body<T>(ex, a, (int64_t)blockIdx.y, (int)blockIdx.x, reinterpret_cast<T *>(smem));
}
// The raw low-rank sums of coef_lowrank_body for real FP32 signals, CL_SG signals per block:
// the generated columns (CF-ADI Z and J Z, centred monomials) and the phase ramps do not depend
// on the signal, so each value is formed once per sample and weighted by every signal of the
// group (for real y, v = ph y: sum col ph y = sum (col ph) y).  Same partial layout as
// coef_lowrank_body (the conjugate variants are copied at the end).  A round reduces 32 values
// (two columns' f and r sums, or four monomials, for the group's signals; re and im) over the
// block in a fixed order: [value][thread] in shared memory, 8 parts of 32 threads, then the
// parts.  grid (nchunks, ceil(batch / CL_SG)), COEF_THREADS threads.
constexpr int CL_SG = 4, CL_VALS = 32, CL_PARTS = COEF_THREADS / CL_VALS;
constexpr int CL_LD = COEF_THREADS + 16;
__global__ void __launch_bounds__(COEF_THREADS, 2) k_coef_lowrank_r4(const CoefArgs<float> a) {
  __shared__ float red[CL_VALS * CL_LD + CL_VALS * CL_PARTS];
  const int tid = threadIdx.x;
  const int chunk = blockIdx.x;
  const int64_t s0 = (int64_t)blockIdx.y * CL_SG;
  const int ns = (int)((a.batch - s0 < CL_SG) ? a.batch - s0 : CL_SG);
  const int64_t n0 = (int64_t)chunk * COEF_CHUNK;
  const float half = 0.5f, Nd = (float)a.N, cen = (float)(0.5 * (double)(a.N - 1)), invN = (float)(1.0 / (double)a.N);
  float y[COEF_E][CL_SG];
  bool in[COEF_E];
#pragma unroll
  for (int e = 0; e < COEF_E; ++e) {
    const int64_t n = n0 + tid + (int64_t)e * COEF_THREADS;
    in[e] = n < a.N;
#pragma unroll
    for (int s = 0; s < CL_SG; ++s) y[e][s] = (in[e] && s < ns) ? a.y[(s0 + s) * a.ld + n] : 0.f;
  }
  // fixed-order block sum of acc[0 .. CL_VALS) -> red's tail (value v at red[CL_VALS*CL_LD + v])
  auto reduce = [&](const float *acc) {
#pragma unroll
    for (int v = 0; v < CL_VALS; ++v) red[v * CL_LD + tid] = acc[v];
    __syncthreads();
    {
      const int v = tid / CL_PARTS, p = tid % CL_PARTS;
      float sum = 0.f;
#pragma unroll 8
      for (int i = 0; i < COEF_THREADS / CL_PARTS; ++i) sum += red[v * CL_LD + p + CL_PARTS * i];
      __syncthreads();
      red[CL_VALS * CL_LD + v * CL_PARTS + p] = sum;
    }
    __syncthreads();
    if (tid < CL_VALS) {
      float sum = 0.f;
#pragma unroll
      for (int p = 0; p < CL_PARTS; ++p) sum += red[CL_VALS * CL_LD + tid * CL_PARTS + p];
      red[tid] = sum;   // the first values of the (now free) thread area
    }
    __syncthreads();
  };
  auto out_of = [&](int s) { return a.part + (((s0 + s) * a.nchunks + chunk) * (int64_t)a.nraw) * 2; };
  const int vbase[4] = {0, 2 * a.rH + a.DA, 4 * a.rH + 2 * a.DA, 4 * a.rH + 2 * a.DA + a.DB};
  for (int variant = 0; variant < 4; variant += 2) {   // real y: the conjugate variants are copies
    const bool useA = variant == 0;
    float2 ph[COEF_E];
#pragma unroll
    for (int e = 0; e < COEF_E; ++e) {
      const int64_t n = n0 + tid + (int64_t)e * COEF_THREADS;
      ph[e] = in[e] ? (useA ? a.phA[n] : a.phB[n]) : make_float2(0.f, 0.f);
    }
    int obase = vbase[variant];
    if (useA) {
      float zf[COEF_E], zr[COEF_E];
#pragma unroll
      for (int e = 0; e < COEF_E; ++e) {
        const float x = (float)(n0 + tid + (int64_t)e * COEF_THREADS) + half, xr = Nd - x;
        zf[e] = in[e] ? coef_div(a.zfirst[0], x + a.zshift[0]) : 0.f;
        zr[e] = in[e] ? coef_div(a.zfirst[0], xr + a.zshift[0]) : 0.f;
      }
      for (int k0 = 0; k0 < a.rH; k0 += 2) {
        const int kc = (a.rH - k0 < 2) ? a.rH - k0 : 2;
        float acc[CL_VALS];   // [column kk][f / r][signal][re / im]
#pragma unroll
        for (int v = 0; v < CL_VALS; ++v) acc[v] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          if (kk >= kc) break;
          const int k = k0 + kk;
          const float pk = a.zshift[k], pk1 = k > 0 ? a.zshift[k - 1] : 0.f, sc = a.zfirst[k];
#pragma unroll
          for (int e = 0; e < COEF_E; ++e) {
            const float x = (float)(n0 + tid + (int64_t)e * COEF_THREADS) + half, xr = Nd - x;
            if (k > 0 && in[e]) {
              zf[e] = coef_div(sc * (x - pk1) * zf[e], x + pk);
              zr[e] = coef_div(sc * (xr - pk1) * zr[e], xr + pk);
            }
            const float cfx = zf[e] * ph[e].x, cfy = zf[e] * ph[e].y;
            const float crx = zr[e] * ph[e].x, cry = zr[e] * ph[e].y;
#pragma unroll
            for (int s = 0; s < CL_SG; ++s) {
              acc[kk * 16 + 0 * 8 + 2 * s] = fmaf(cfx, y[e][s], acc[kk * 16 + 0 * 8 + 2 * s]);
              acc[kk * 16 + 0 * 8 + 2 * s + 1] = fmaf(cfy, y[e][s], acc[kk * 16 + 0 * 8 + 2 * s + 1]);
              acc[kk * 16 + 1 * 8 + 2 * s] = fmaf(crx, y[e][s], acc[kk * 16 + 1 * 8 + 2 * s]);
              acc[kk * 16 + 1 * 8 + 2 * s + 1] = fmaf(cry, y[e][s], acc[kk * 16 + 1 * 8 + 2 * s + 1]);
            }
          }
        }
        reduce(acc);
        if (tid < 16 * kc) {
          const int kk = tid / 16, fr = (tid / 8) & 1, s = (tid / 2) & 3, c = tid & 1;
          if (s < ns) out_of(s)[2 * (obase + fr * a.rH + k0 + kk) + c] = red[tid];
        }
        __syncthreads();
      }
      obase += 2 * a.rH;
    }
    // centred monomials u^i, four per round
    const int D = useA ? a.DA : a.DB;
    float up[COEF_E];
#pragma unroll
    for (int e = 0; e < COEF_E; ++e) up[e] = 1.f;
    for (int i0 = 0; i0 < D; i0 += 4) {
      const int ic = (D - i0 < 4) ? D - i0 : 4;
      float acc[CL_VALS];   // [monomial ii][signal][re / im]
#pragma unroll
      for (int v = 0; v < CL_VALS; ++v) acc[v] = 0.f;
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        if (ii >= ic) break;
#pragma unroll
        for (int e = 0; e < COEF_E; ++e) {
          const float u = ((float)(n0 + tid + (int64_t)e * COEF_THREADS) - cen) * invN;
          if (i0 + ii > 0) up[e] *= u;
          const float cx = up[e] * ph[e].x, cy = up[e] * ph[e].y;
#pragma unroll
          for (int s = 0; s < CL_SG; ++s) {
            acc[ii * 8 + 2 * s] = fmaf(cx, y[e][s], acc[ii * 8 + 2 * s]);
            acc[ii * 8 + 2 * s + 1] = fmaf(cy, y[e][s], acc[ii * 8 + 2 * s + 1]);
          }
        }
      }
      reduce(acc);
      if (tid < 8 * ic) {
        const int ii = tid / 8, s = (tid / 2) & 3, c = tid & 1;
        if (s < ns) out_of(s)[2 * (obase + i0 + ii) + c] = red[tid];
      }
      __syncthreads();
    }
  }
  // conjugate variants (D_A y, D_B y) of real input
  const int n0c = 2 * a.rH + a.DA, n2c = a.DB;
  for (int s = 0; s < ns; ++s) {
    float *out = out_of(s);
    for (int i = tid; i < n0c + n2c; i += COEF_THREADS) {
      const int src = (i < n0c) ? vbase[0] + i : vbase[2] + (i - n0c);
      const int dst = (i < n0c) ? vbase[1] + i : vbase[3] + (i - n0c);
      out[2 * dst] = out[2 * src];
      out[2 * dst + 1] = -out[2 * src + 1];
    }
  }
}

template <typename T> __global__ void __launch_bounds__(COEF_THREADS) k_coef_st(const CoefArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  DevExS<CState<T>> ex;
  coef_st_body<T>(ex, a, (int64_t)blockIdx.y, (int)blockIdx.x, reinterpret_cast<T *>(smem));
}
template <typename T> __global__ void k_coef_reduce(const T *part, int nchunks, int nout, T *tot) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < nout) coef_reduce_body<T>(part, nchunks, nout, (int64_t)blockIdx.y, o, tot);
}
template <typename T>
__global__ void k_coef_gather(const c2<T> *X, Layout Lf, int64_t N, int cplx, int64_t sig0, int64_t nsig, int64_t h,
                              c2<T> *out, int64_t Kp) {
  const int64_t nF = 2 * h + 1, total = nsig * nF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = sig0 + t / nF, k = t % nF;
    const int64_t pl = cplx ? (s - sig0) : (s / 2 - sig0 / 2);
    coef_gather_body<T>(X, Lf, N, cplx, s, pl, h, k, out + s * Kp);
  }
}
template <typename T>
__global__ void k_coef_mix(const CoefArgs<T> a, const T *tot, const T *totU, const T *CA, const T *CB, const T *sq,
                           c2<T> *out, int64_t Kp, int64_t nF) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sig = blockIdx.y;
  const int nfin = 4 * a.rH + 2 * a.DA + 2 * a.DB + a.r;
  if (o >= nfin) return;
  out[sig * Kp + nF + o] =
      coef_mix_value<T>(a, tot + sig * (int64_t)a.nraw * 2, totU + sig * (int64_t)(a.r > 0 ? a.r : 1) * 2, CA, CB, sq, o, sig);
}

__global__ void k_split_tf32(const float *src, float2 *hl, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const float h = tf32_round(src[t]);
    hl[t] = make_float2(h, tf32_round(src[t] - h));
  }
}

__global__ void k_to_f32(const double *src, float *dst, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (float)src[t];
}

// ---------------------------------------------------------------------------
// device runner
// ---------------------------------------------------------------------------

static fst_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? FST_ENOMEM : FST_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}
#define CU(call, what)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, what);  \
  } while (0)
#define LAUNCHED(what) CU(cudaGetLastError(), what)
#define TRY(expr)                \
  do {                           \
    fst_status _s = (expr);      \
    if (_s != FST_OK) return _s; \
  } while (0)

static bool g_attr_done = false;
static fst_status set_attrs() {
  if (g_attr_done) return FST_OK;
  const int mx = 227 * 1024;
  CU(cudaFuncSetAttribute(k_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_small_ragged<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_small_ragged<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passA<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passA<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passB<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passB<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passC<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_passC<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_fastAw<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, fastw_smem(32)), "attr");
  CU(cudaFuncSetAttribute(k_fastAw<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fastw_smem(16)), "attr");
  CU(cudaFuncSetAttribute(k_fastAw<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, fastw_smem(8)), "attr");
  CU(cudaFuncSetAttribute(k_corr_cc, cudaFuncAttributeMaxDynamicSharedMemorySize, cc_smem(64)), "attr");
  CU(cudaFuncSetAttribute(k_zadd, cudaFuncAttributeMaxDynamicSharedMemorySize, za_smem(64, 1)), "attr");
  CU(cudaFuncSetAttribute(k_fastB8192, cudaFuncAttributeMaxDynamicSharedMemorySize, fastb8192_smem()), "attr");
  CU(cudaFuncSetAttribute(k_fastB4096_2s, cudaFuncAttributeMaxDynamicSharedMemorySize, fastb2s_smem()), "attr");
  CU(cudaFuncSetAttribute(k_rcorr_part, cudaFuncAttributeMaxDynamicSharedMemorySize, rcorr_smem()), "attr");
  CU(cudaFuncSetAttribute(k_colA<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(2)), "attr");
  CU(cudaFuncSetAttribute(k_colA<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(4)), "attr");
  CU(cudaFuncSetAttribute(k_colA<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(8)), "attr");
  CU(cudaFuncSetAttribute(k_colA<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(16)), "attr");
  CU(cudaFuncSetAttribute(k_colA<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(32)), "attr");
  CU(cudaFuncSetAttribute(k_colC<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(2)), "attr");
  CU(cudaFuncSetAttribute(k_colC<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(4)), "attr");
  CU(cudaFuncSetAttribute(k_colC<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(8)), "attr");
  CU(cudaFuncSetAttribute(k_colC<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(16)), "attr");
  CU(cudaFuncSetAttribute(k_colC<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_smem_bytes(32)), "attr");
  CU(cudaFuncSetAttribute(k_corr_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_corr_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_corr_tc<96>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  CU(cudaFuncSetAttribute(k_corr_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr");
  g_attr_done = true;
  return FST_OK;
}

// ---- launch accounting (fst_launch_count / fst_profile_*) --------------------
static long long g_launches = 0;
static int g_prof_on = 0;
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
  long long units;
};
static std::vector<ProfRec> g_prof;
static void prof_begin(cudaStream_t s, const char *name, long long units, cudaEvent_t *ea) {
  ++g_launches;
  *ea = nullptr;
  if (!g_prof_on) return;
  cudaEventCreate(ea);
  cudaEventRecord(*ea, s);
  ProfRec r{name, *ea, nullptr, units};
  g_prof.push_back(r);
}
static void prof_end(cudaStream_t s, cudaEvent_t ea) {
  if (!g_prof_on || !ea) return;
  cudaEvent_t eb;
  cudaEventCreate(&eb);
  cudaEventRecord(eb, s);
  g_prof.back().b = eb;
}
#define PROF(name, units, launch)            \
  do {                                       \
    cudaEvent_t _ea;                         \
    prof_begin(cur, name, (units), &_ea);    \
    launch;                                  \
    prof_end(cur, _ea);                      \
  } while (0)

#define PROF_S(stream, name, units, launch) \
  do {                                       \
    cudaEvent_t _ea;                         \
    prof_begin(stream, name, (units), &_ea); \
    launch;                                  \
    prof_end(stream, _ea);                   \
  } while (0)

bool profiling_enabled() { return g_prof_on != 0; }

// ---- TMA tensor maps (driver entry point, resolved once) --------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D FP32 tensor map: rows of `inner` elements `row_bytes` apart, box inner x outer
static fst_status encode_2d(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                            uint32_t box_inner, uint32_t box_outer, bool swizzle128) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(FST_ECUDA, "cuTensorMapEncodeTiled not available");
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(FST_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return FST_OK;
}

// test hook (fst_test_tc_stall): the next g_tc_stall launches of the tcgen05 correction give
// up after g_tc_stall_limit_ns on a wait that nothing completes
static std::atomic<int> g_tc_stall{0};
static unsigned long long g_tc_stall_limit_ns = 20000000ull;
bool tc_stall_pending() { return g_tc_stall.load() > 0; }
bool tc_stall_take() {
  int v = g_tc_stall.load();
  while (v > 0)
    if (g_tc_stall.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

static inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

struct DevRunner : Runner {
  cudaStream_t s = nullptr;     // caller's stream
  cudaStream_t cur = nullptr;   // stream the apply kernels go to (s, or a capture lane)
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};   // two lanes and the side lane
  cudaEvent_t fork = nullptr, join = nullptr, ev_mid = nullptr, ev_side = nullptr, join_side = nullptr;
  bool capturing = false;
  long long launches_at_begin = 0;
  int sms = 1;
  // raised by k_corr_tc when one of its waits timed out: a host-mapped word, so the host
  // reads it without a copy (fst_sync, and the next call on the plan)
  int *tc_err = nullptr;     // device address
  int *tc_err_h = nullptr;   // host address
  bool device() const override { return true; }
  int sm_count() const override { return sms; }
  void set_stream(void *st) override { s = (cudaStream_t)st; cur = s; }
  void *stream() const override { return (void *)s; }
  ~DevRunner() override {
    for (int i = 0; i < 3; ++i)
      if (cap[i]) cudaStreamDestroy(cap[i]);
    for (cudaEvent_t e : {fork, join, ev_mid, ev_side, join_side, t0, t1})
      if (e) cudaEventDestroy(e);
    if (tc_err_h) cudaFreeHost(tc_err_h);
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  fst_status timer(int phase, double *ms) override {
    if (!t0) {
      CU(cudaEventCreate(&t0), "event");
      CU(cudaEventCreate(&t1), "event");
    }
    if (phase == 0) {
      CU(cudaEventRecord(t0, cur), "event");
      return FST_OK;
    }
    CU(cudaEventRecord(t1, cur), "event");
    CU(cudaEventSynchronize(t1), "event sync");
    float f = 0.f;
    CU(cudaEventElapsedTime(&f, t0, t1), "elapsed");
    if (ms) *ms = f;
    return FST_OK;
  }
  fst_status device_status(bool sync) override {
    if (sync) CU(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (tc_err_h && *(volatile int *)tc_err_h) {
      *(volatile int *)tc_err_h = 0;
      return fail(FST_ETIMEOUT, "a bounded wait of the tensor-core correction ran past its limit; the outputs "
                                "of that call are NaN");
    }
    return FST_OK;
  }

  int lanes() const override { return capturing ? 2 : 1; }
  void use_lane(int i) override { cur = capturing ? cap[i & 1] : s; }
  void lanes_after_first() override {
    if (!capturing) return;
    cudaEventRecord(ev_mid, cap[0]);
    cudaStreamWaitEvent(cap[1], ev_mid, 0);
  }
  void lanes_join_first() override {
    if (!capturing) return;
    cudaEventRecord(ev_mid, cap[1]);
    cudaStreamWaitEvent(cap[0], ev_mid, 0);
  }
  void use_side() override { cur = capturing ? cap[2] : s; }
  void side_done() override {
    if (capturing) cudaEventRecord(ev_side, cap[2]);
  }
  void wait_side() override {
    if (capturing) cudaStreamWaitEvent(cur, ev_side, 0);
  }
  bool user_stream_capturing() override {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
      cudaGetLastError();
      return true;
    }
    return st != cudaStreamCaptureStatusNone;
  }
  bool graph_begin() override {
    if (!cap[0]) {
      for (int i = 0; i < 3; ++i)
        if (cudaStreamCreateWithFlags(&cap[i], cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return false; }
      for (cudaEvent_t *e : {&fork, &join, &ev_mid, &ev_side, &join_side})
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          return false;
        }
    }
    if (set_attrs() != FST_OK) return false;
    if (cudaStreamBeginCapture(cap[0], cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaEventRecord(fork, cap[0]);
    cudaStreamWaitEvent(cap[1], fork, 0);
    cudaStreamWaitEvent(cap[2], fork, 0);
    capturing = true;
    cur = cap[0];
    launches_at_begin = g_launches;
    return true;
  }
  fst_status graph_end(void **exec, long long *nodes) override {
    *exec = nullptr;
    cudaEventRecord(join, cap[1]);
    cudaStreamWaitEvent(cap[0], join, 0);
    cudaEventRecord(join_side, cap[2]);
    cudaStreamWaitEvent(cap[0], join_side, 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap[0], &g);
    capturing = false;
    cur = s;
    *nodes = g_launches - launches_at_begin;
    g_launches = launches_at_begin;   // captured, not yet run
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    *exec = (void *)ex;
    return FST_OK;
  }
  fst_status graph_launch(void *exec, long long nodes) override {
    CU(cudaGraphLaunch((cudaGraphExec_t)exec, s), "cudaGraphLaunch");
    g_launches += nodes;
    return FST_OK;
  }
  void graph_destroy(void *exec) override {
    if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
  }

  fst_status alloc(void **p, size_t bytes) override {
    *p = nullptr;
    CU(cudaMalloc(p, std::max<size_t>(bytes, 16)), "cudaMalloc");
    return FST_OK;
  }
  void release(void *p) override {
    if (p) cudaFree(p);
  }
  fst_status h2d(void *dst, const void *src, size_t bytes) override {
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "h2d");
    CU(cudaStreamSynchronize(s), "h2d sync");
    return FST_OK;
  }
  fst_status d2h(void *dst, const void *src, size_t bytes) override {
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "d2h");
    CU(cudaStreamSynchronize(s), "d2h sync");
    return FST_OK;
  }
  fst_status d2d(void *dst, const void *src, size_t bytes) override {
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s), "d2d");
    return FST_OK;
  }
  fst_status zero(void *p, size_t bytes) override {
    CU(cudaMemsetAsync(p, 0, bytes, s), "memset");
    return FST_OK;
  }
  fst_status sync() override {
    CU(cudaStreamSynchronize(s), "sync");
    return FST_OK;
  }

  template <typename T> fst_status small_t(const ConvArgs<T> &a, const Layout &L) {
    if (set_attrs() != FST_OK) return FST_ECUDA;
    PROF(sizeof(T) == 4 ? "k_small<f32>" : "k_small<f64>", a.npairs,
         (k_small<T><<<(unsigned)a.npairs, L.nthr_small, L.smem_small, cur>>>(a)));
    LAUNCHED("k_small");
    return FST_OK;
  }
  template <typename T> fst_status passA_t(const ConvArgs<T> &a, const Layout &L) {
    if (set_attrs() != FST_OK) return FST_ECUDA;
    dim3 grid((unsigned)L.ntiles, (unsigned)((a.npairs + L.G - 1) / L.G));
    PROF(sizeof(T) == 4 ? "k_passA<f32>" : "k_passA<f64>", a.npairs, (k_passA<T><<<grid, L.nthr_A, L.smem_A, cur>>>(a)));
    LAUNCHED("k_passA");
    return FST_OK;
  }
  template <typename T> fst_status reduce_t(const ConvArgs<T> &a, const Layout &) {
    const int thr = std::min(1024, std::max(32, ((2 * a.r + 31) / 32) * 32));
    PROF(sizeof(T) == 4 ? "k_reduce<f32>" : "k_reduce<f64>", a.npairs, (k_reduce<T><<<(unsigned)a.npairs, thr, 0, cur>>>(a)));
    LAUNCHED("k_reduce");
    return FST_OK;
  }
  template <typename T> fst_status passB_t(const ConvArgs<T> &a, const Layout &L) {
    if (set_attrs() != FST_OK) return FST_ECUDA;
    dim3 grid((unsigned)(1u << L.log2P), (unsigned)a.npairs);
    PROF(sizeof(T) == 4 ? "k_passB<f32>" : "k_passB<f64>", a.npairs, (k_passB<T><<<grid, L.nthr_B, L.smem_B, cur>>>(a)));
    LAUNCHED("k_passB");
    return FST_OK;
  }
  template <typename T> fst_status passC_t(const ConvArgs<T> &a, const Layout &L) {
    if (set_attrs() != FST_OK) return FST_ECUDA;
    dim3 grid((unsigned)L.ntiles, (unsigned)((a.npairs + L.G - 1) / L.G));
    PROF(sizeof(T) == 4 ? "k_passC<f32>" : "k_passC<f64>", a.npairs, (k_passC<T><<<grid, L.nthr_C, L.smem_C, cur>>>(a)));
    LAUNCHED("k_passC");
    return FST_OK;
  }
  template <typename T>
  fst_status small_ragged_t(const RaggedDesc<T> *d, int count, const ConvArgs<T> &base, const Layout &L) {
    if (set_attrs() != FST_OK) return FST_ECUDA;
    PROF(sizeof(T) == 4 ? "k_small_ragged<f32>" : "k_small_ragged<f64>", count,
         (k_small_ragged<T><<<(unsigned)count, L.nthr_small, L.smem_small, cur>>>(d, base)));
    LAUNCHED("k_small_ragged");
    return FST_OK;
  }
  fst_status small_ragged(const RaggedDesc<float> *d, int count, const ConvArgs<float> &base,
                          const Layout &L) override { return small_ragged_t(d, count, base, L); }
  fst_status small_ragged(const RaggedDesc<double> *d, int count, const ConvArgs<double> &base,
                          const Layout &L) override { return small_ragged_t(d, count, base, L); }
  fst_status small(const ConvArgs<float> &a, const Layout &L) override { return small_t(a, L); }
  fst_status small(const ConvArgs<double> &a, const Layout &L) override { return small_t(a, L); }
  template <int P2> fst_status colA_t(const ConvArgs<float> &a, const Layout &L) {
    TRY(set_attrs());
    dim3 grid((unsigned)L.ntiles, (unsigned)a.npairs);
    PROF(P2 == 2 ? "k_colA<2>" : P2 == 4 ? "k_colA<4>" : P2 == 8 ? "k_colA<8>" : P2 == 16 ? "k_colA<16>" : "k_colA<32>",
         a.npairs, (k_colA<P2><<<grid, 256, big_smem_bytes(P2), cur>>>(a)));
    LAUNCHED("k_colA");
    return FST_OK;
  }
  template <int P2> fst_status colC_t(const ConvArgs<float> &a, const Layout &L) {
    TRY(set_attrs());
    dim3 grid((unsigned)L.ntiles, (unsigned)a.npairs);
    PROF(P2 == 2 ? "k_colC<2>" : P2 == 4 ? "k_colC<4>" : P2 == 8 ? "k_colC<8>" : P2 == 16 ? "k_colC<16>" : "k_colC<32>",
         a.npairs, (k_colC<P2><<<grid, 256, big_smem_bytes(P2), cur>>>(a)));
    LAUNCHED("k_colC");
    return FST_OK;
  }
  fst_status passA(const ConvArgs<float> &a, const Layout &L) override {
    if (L.big) {
      switch (L.P2) {
        case 2: return colA_t<2>(a, L);
        case 4: return colA_t<4>(a, L);
        case 8: return colA_t<8>(a, L);
        case 16: return colA_t<16>(a, L);
        case 32: return colA_t<32>(a, L);
        default: return fail(FST_EINVAL, "column pass width out of range");
      }
    }
    if (!L.fast) return passA_t(a, L);
    const int P = 1 << L.log2P;
    // no fused correction, real signals: 256-byte row loads when the rows allow float2 loads
    // (measured faster for real rows, slower for complex ones)
    const bool wide_ok = !a.rp && !a.cplx && (uintptr_t)a.y % 8 == 0 && a.ld % 2 == 0;
    if (a.mode != MODE_FULL && wide_ok) {
      TRY(set_attrs());
      const int64_t tiles = ((1 << L.log2Q) / FASTW_NB) * ((a.npairs + FASTW_G - 1) / FASTW_G);
      const unsigned grid = (unsigned)std::min<int64_t>(tiles, 3 * (int64_t)sms);
      if (P == 32) PROF("k_fastAw<32>", a.npairs, (k_fastAw<32><<<grid, FAST_THREADS, fastw_smem(32), cur>>>(a)));
      else if (P == 16) PROF("k_fastAw<16>", a.npairs, (k_fastAw<16><<<grid, FAST_THREADS, fastw_smem(16), cur>>>(a)));
      else PROF("k_fastAw<8>", a.npairs, (k_fastAw<8><<<grid, FAST_THREADS, fastw_smem(8), cur>>>(a)));
      LAUNCHED("k_fastAw");
      return FST_OK;
    }
    FastArgs f{a, a.ST_hl};
    dim3 grid((unsigned)L.ntiles, (unsigned)((a.npairs + FAST_G - 1) / FAST_G));
    if (P == 32) PROF("k_fastA<32>", a.npairs, (k_fastA<32><<<grid, FAST_THREADS, 0, cur>>>(f)));
    else if (P == 16) PROF("k_fastA<16>", a.npairs, (k_fastA<16><<<grid, FAST_THREADS, 0, cur>>>(f)));
    else PROF("k_fastA<8>", a.npairs, (k_fastA<8><<<grid, FAST_THREADS, 0, cur>>>(f)));
    LAUNCHED("k_fastA");
    return FST_OK;
  }
  fst_status passA(const ConvArgs<double> &a, const Layout &L) override { return passA_t(a, L); }
  fst_status reduce(const ConvArgs<float> &a, const Layout &L) override { return reduce_t(a, L); }
  fst_status reduce(const ConvArgs<double> &a, const Layout &L) override { return reduce_t(a, L); }
  fst_status passB(const ConvArgs<float> &a, const Layout &L) override {
    if (a.two_spec && !((L.fast || L.big) && L.log2Q == 12))
      return fail(FST_EINVAL, "two-spectrum row pass needs 4096-point rows");
    if ((L.fast || L.big) && L.log2Q == 13 && a.tw8) {
      TRY(set_attrs());
      dim3 grid((unsigned)(1u << L.log2P), (unsigned)a.npairs);
      PROF("k_fastB8192", a.npairs, (k_fastB8192<<<grid, 512, fastb8192_smem(), cur>>>(a, a.tw8)));
      LAUNCHED("k_fastB8192");
      return FST_OK;
    }
    if (!(L.fast || L.big) || L.log2Q != 12) return passB_t(a, L);
    if (a.two_spec) {
      if (!a.rp || a.cplx || a.mode != MODE_CONV)
        return fail(FST_EINVAL, "two-spectrum row pass needs real ragged slots");
      TRY(set_attrs());
      dim3 grid((unsigned)((1u << L.log2P) / 2 + 1), (unsigned)a.npairs);
      PROF("k_fastB4096_2s", a.npairs, (k_fastB4096_2s<<<grid, 256, fastb2s_smem(), cur>>>(a)));
      LAUNCHED("k_fastB4096_2s");
      return FST_OK;
    }
    dim3 grid((unsigned)(1u << L.log2P), (unsigned)a.npairs);
    PROF("k_fastB4096", a.npairs, (k_fastB4096<<<grid, 256, 0, cur>>>(a)));
    LAUNCHED("k_fastB4096");
    return FST_OK;
  }
  fst_status passB(const ConvArgs<double> &a, const Layout &L) override { return passB_t(a, L); }
  fst_status corr_c(const ConvArgs<float> &a) override {
    FastArgs f{a, a.ST_hl};
    dim3 grid((unsigned)((a.N + CORR_BLOCK - 1) / CORR_BLOCK), (unsigned)((a.npairs + FAST_G - 1) / FAST_G));
    PROF("k_corr_c", a.npairs, (k_corr_c<<<grid, FAST_THREADS, 0, cur>>>(f)));
    LAUNCHED("k_corr_c");
    return FST_OK;
  }
  fst_status tc_prep(const float *ST, int64_t N, int rpad, int r, int nB, int64_t Npad, float *STt) override {
    // plan time (never inside a stream capture): kernel attributes and the error word
    TRY(set_attrs());
    if (!tc_err_h) {
      CU(cudaHostAlloc((void **)&tc_err_h, sizeof(int), cudaHostAllocMapped), "cudaHostAlloc");
      *(volatile int *)tc_err_h = 0;
      CU(cudaHostGetDevicePointer((void **)&tc_err, tc_err_h, 0), "cudaHostGetDevicePointer");
    }
    k_tc_prep<<<grid_for((int64_t)nB * Npad, 256), 256, 0, s>>>(ST, N, rpad, r, nB, Npad, STt);
    LAUNCHED("k_tc_prep");
    return FST_OK;
  }
  fst_status corr_tc(const ConvArgs<float> &a) override {
    if (!tc_err) return fail(FST_EUNSUPPORTED, "tcgen05 correction used before its plan-time set-up");
    CUtensorMap mY, mS;
    // y in 128-byte swizzled boxes: 32 floats of 128 rows (real) or of 64 complex rows
    if (a.cplx)
      TRY(encode_2d(&mY, a.y, 2 * (uint64_t)a.N, (uint64_t)a.batch, (uint64_t)a.ld * 8, TC_KT, TC_M / 2, true));
    else
      TRY(encode_2d(&mY, a.y, (uint64_t)a.N, (uint64_t)a.batch, (uint64_t)a.ld * 4, TC_KT, TC_M, true));
    TRY(encode_2d(&mS, a.STt, (uint64_t)a.N, (uint64_t)a.tc_nB, (uint64_t)a.tc_Npad * 4, TC_KT, (uint32_t)a.tc_nB,
                  true));
    TcArgs t{};
    t.N = a.N;
    t.rows = a.batch;
    t.cplx = a.cplx;
    t.nB = a.tc_nB;
    t.r = a.r;
    t.rpad = a.rpad;
    t.ktiles = (int)((a.N + TC_KT - 1) / TC_KT);
    t.nks = tc_slices(a.N);
    const int64_t rb = a.cplx ? (a.batch + TC_M / 2 - 1) / (TC_M / 2) : (a.batch + TC_M - 1) / TC_M;
    if ((int64_t)t.nks * rb >= (1LL << 31)) return fail(FST_EINVAL, "batch too large for the tcgen05 correction");
    t.nitems = (int)(t.nks * rb);
    t.part = a.part;
    t.err = tc_err;
    t.timeout_ns = TC_TIMEOUT_NS;
    t.stall = 0;
    if (tc_stall_take()) {
      t.stall = 1;
      t.timeout_ns = g_tc_stall_limit_ns;
    }
    // persistent: one CTA per SM walks the items
    dim3 grid((unsigned)std::min<int64_t>(t.nitems, sms));
    const size_t smem = (size_t)tc_smem_bytes(t.nB);
    switch (t.nB) {
      case 32: PROF("k_corr_tc", a.npairs, (k_corr_tc<32><<<grid, TC_THREADS, smem, cur>>>(mY, mS, t))); break;
      case 64: PROF("k_corr_tc", a.npairs, (k_corr_tc<64><<<grid, TC_THREADS, smem, cur>>>(mY, mS, t))); break;
      case 96: PROF("k_corr_tc", a.npairs, (k_corr_tc<96><<<grid, TC_THREADS, smem, cur>>>(mY, mS, t))); break;
      case 128: PROF("k_corr_tc", a.npairs, (k_corr_tc<128><<<grid, TC_THREADS, smem, cur>>>(mY, mS, t))); break;
      default: return fail(FST_EINVAL, "tcgen05 correction width out of range");
    }
    LAUNCHED("k_corr_tc");
    return FST_OK;
  }
  fst_status rcorr(const RSig *sigs, int nsig, const RItem *items, int nitems, int cplx, float *part,
                   float *acoef) override {
    if (nitems <= 0) return FST_OK;
    TRY(set_attrs());
    PROF("k_rcorr_part", nitems, (k_rcorr_part<<<(unsigned)nitems, 256, rcorr_smem(), cur>>>(sigs, items, cplx, part)));
    LAUNCHED("k_rcorr_part");
    PROF("k_rcorr_reduce", nsig, (k_rcorr_reduce<<<(unsigned)nsig, 128, 0, cur>>>(sigs, part, acoef)));
    LAUNCHED("k_rcorr_reduce");
    return FST_OK;
  }
  fst_status rzadd(const RSig *sigs, const RItem *items, int nitems, int cplx, const float *acoef) override {
    if (nitems <= 0) return FST_OK;
    PROF("k_rzadd", nitems, (k_rzadd<<<(unsigned)nitems, 256, 0, cur>>>(sigs, items, cplx, acoef)));
    LAUNCHED("k_rzadd");
    return FST_OK;
  }
  fst_status corr_cc(const ConvArgs<float> &a) override {
    TRY(set_attrs());
    PROF("k_corr_cc", a.npairs,
         (k_corr_cc<<<(unsigned)((a.N + CORR_BLOCK - 1) / CORR_BLOCK), CC_THREADS, cc_smem(a.rpad), cur>>>(a)));
    LAUNCHED("k_corr_cc");
    return FST_OK;
  }
  fst_status zadd(const ConvArgs<float> &a) override {
    TRY(set_attrs());
    const int64_t rows = a.cplx ? 2 * a.batch : a.batch;
    const int ng = za_groups(rows), ns = ZA_THREADS / ng;
    const int64_t nrb = (rows + ng * ZA_RG - 1) / (ng * ZA_RG);
    const int64_t blocks = nrb * ((a.N + ns - 1) / ns);
    if (blocks >= (1LL << 31)) return fail(FST_EINVAL, "batch too large for the correction pass");
    PROF("k_zadd", a.npairs, (k_zadd<<<(unsigned)blocks, ZA_THREADS, za_smem(a.rpad, ng), cur>>>(a)));
    LAUNCHED("k_zadd");
    return FST_OK;
  }
  fst_status z_rmw(const ConvArgs<float> &a, const float *ST) override {
    const int nsig = a.cplx ? ZR_ROWS / 2 : ZR_ROWS;
    dim3 grid((unsigned)((a.N + ZR_N - 1) / ZR_N), (unsigned)((a.batch + nsig - 1) / nsig));
    if (a.rpad <= 32) PROF("k_z_rmw", a.npairs, (k_z_rmw<32><<<grid, ZR_THREADS, 0, cur>>>(a, ST)));
    else PROF("k_z_rmw", a.npairs, (k_z_rmw<64><<<grid, ZR_THREADS, 0, cur>>>(a, ST)));
    LAUNCHED("k_z_rmw");
    return FST_OK;
  }
  fst_status corr_reduce(const ConvArgs<float> &a, const float *scale) override {
    dim3 grid((unsigned)a.npairs, (unsigned)((2 * a.r + 7) / 8));
    PROF("k_corr_reduce", a.npairs, (k_corr_reduce<<<grid, 256, 0, cur>>>(a, scale)));
    LAUNCHED("k_corr_reduce");
    return FST_OK;
  }
  fst_status corr_z(const ConvArgs<float> &a) override {
    FastArgs f{a, a.ST_hl};
    dim3 grid((unsigned)((a.N + CORR_ROWS - 1) / CORR_ROWS), (unsigned)((a.npairs + FAST_G - 1) / FAST_G));
    PROF("k_corr_z", a.npairs, (k_corr_z<<<grid, FAST_THREADS, 0, cur>>>(f)));
    LAUNCHED("k_corr_z");
    return FST_OK;
  }
  fst_status passC(const ConvArgs<float> &a, const Layout &L) override {
    if (L.big) {
      switch (L.P2) {
        case 2: return colC_t<2>(a, L);
        case 4: return colC_t<4>(a, L);
        case 8: return colC_t<8>(a, L);
        case 16: return colC_t<16>(a, L);
        case 32: return colC_t<32>(a, L);
        default: return fail(FST_EINVAL, "column pass width out of range");
      }
    }
    if (!L.fast) return passC_t(a, L);
    FastArgs f{a, a.ST_hl};
    dim3 grid((unsigned)L.ntiles, (unsigned)((a.npairs + FAST_G - 1) / FAST_G));
    const int P = 1 << L.log2P;
    if (P == 32) PROF("k_fastC<32>", a.npairs, (k_fastC<32><<<grid, FAST_THREADS, 0, cur>>>(f)));
    else if (P == 16) PROF("k_fastC<16>", a.npairs, (k_fastC<16><<<grid, FAST_THREADS, 0, cur>>>(f)));
    else PROF("k_fastC<8>", a.npairs, (k_fastC<8><<<grid, FAST_THREADS, 0, cur>>>(f)));
    LAUNCHED("k_fastC");
    return FST_OK;
  }
  fst_status passC(const ConvArgs<double> &a, const Layout &L) override { return passC_t(a, L); }

  fst_status bisect_ms_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat, double *theta,
                            int *flag) override {
    if (nt <= 0) return FST_OK;
    PROF_S(s, "k_bisect_ms_many", nt, (k_bisect_ms_many<<<nt, BISECT_THREADS, 0, s>>>(td, dcat, e2cat, theta, flag)));
    LAUNCHED("k_bisect_ms_many");
    return FST_OK;
  }
  fst_status bisect_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat, double *theta,
                         int *flag) override {
    // one warp per block: the targets spread over every SM (each one's FP64 pipe is the limit)
    PROF_S(s, "k_bisect_many", nt, (k_bisect_many<<<(nt + 31) / 32, 32, 0, s>>>(td, nt, dcat, e2cat, theta, flag)));
    LAUNCHED("k_bisect_many");
    return FST_OK;
  }
  fst_status invit_many(const TargetDesc *td, int nt, const double *dcat, const double *ecat, const double *theta,
                        double *x, double *fd, double *fdl, double *fdu, double *fdu2, uint8_t *piv) override {
    PROF_S(s, "k_invit_many", nt, (k_invit_many<<<(nt + 63) / 64, 64, 0, s>>>(td, nt, dcat, ecat, theta, x, fd, fdl, fdu, fdu2, piv)));
    LAUNCHED("k_invit_many");
    return FST_OK;
  }
  fst_status finalize_many(const TargetDesc *td, int nt, const double *x) override {
    PROF_S(s, "k_finalize_many", nt, (k_finalize_many<<<nt, 256, 0, s>>>(td, x)));
    LAUNCHED("k_finalize_many");
    return FST_OK;
  }
  fst_status dot(const double *a, const double *b, int64_t N, int nvec, double *out) override {
    k_dot<<<nvec, 256, 0, s>>>(a, b, N, out);
    LAUNCHED("k_dot");
    return FST_OK;
  }
  fst_status sinc_embed(double *c, int64_t N, int64_t M, double W) override {
    k_sinc<<<grid_for(M, 256), 256, 0, s>>>(c, N, M, W);
    LAUNCHED("k_sinc");
    return FST_OK;
  }
  fst_status spec_store(const double2 *X, const Layout &L64, const Layout &L32, int64_t M, double scale,
                        double *spec64, float *spec32) override {
    k_spec_store<<<grid_for(M, 256), 256, 0, s>>>(X, L64, L32, M, scale, spec64, spec32);
    LAUNCHED("k_spec_store");
    return FST_OK;
  }
  fst_status gather_ST(const double *S, int64_t N, const int *sel, int r, int rpad, double *ST64,
                       float *ST32) override {
    k_gather<<<grid_for(N * rpad, 256), 256, 0, s>>>(S, N, sel, r, rpad, ST64, ST32);
    LAUNCHED("k_gather");
    return FST_OK;
  }
  template <typename T> fst_status coef_lowrank_t(const CoefArgs<T> &a) {
    if (sizeof(T) == 4 && !a.cplx && a.batch >= 2) {
      // real FP32 batches: four signals share every generated column
      const CoefArgs<float> &af = *reinterpret_cast<const CoefArgs<float> *>(&a);
      dim3 grid((unsigned)af.nchunks, (unsigned)((af.batch + CL_SG - 1) / CL_SG));
      PROF("k_coef_lowrank_r4", 0, (k_coef_lowrank_r4<<<grid, COEF_THREADS, 0, cur>>>(af)));
      LAUNCHED("k_coef_lowrank_r4");
      return FST_OK;
    }
    const size_t smem = (size_t)COEF_RED_WORDS * sizeof(T);
    dim3 grid((unsigned)a.nchunks, (unsigned)a.batch);
    PROF("k_coef_lowrank", 0, (k_coef_lowrank<T><<<grid, COEF_THREADS, smem, cur>>>(a)));
    LAUNCHED("k_coef_lowrank");
    return FST_OK;
  }
  template <typename T> fst_status coef_st_t(const CoefArgs<T> &a) {
    const size_t smem = (COEF_THREADS / 32) * 128 * sizeof(T);
    dim3 grid((unsigned)a.nchunks, (unsigned)a.batch);
    PROF("k_coef_st", 0, (k_coef_st<T><<<grid, COEF_THREADS, smem, cur>>>(a)));
    LAUNCHED("k_coef_st");
    return FST_OK;
  }
  template <typename T> fst_status coef_reduce_t(const T *part, int nchunks, int nout, int64_t batch, T *tot) {
    dim3 grid((unsigned)((nout + 127) / 128), (unsigned)batch);
    PROF("k_coef_reduce", 0, (k_coef_reduce<T><<<grid, 128, 0, cur>>>(part, nchunks, nout, tot)));
    LAUNCHED("k_coef_reduce");
    return FST_OK;
  }
  template <typename T>
  fst_status coef_gather_t(const c2<T> *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0, int64_t nsig,
                           int64_t h, c2<T> *out, int64_t Kp) {
    PROF("k_coef_gather", 0, (k_coef_gather<T><<<grid_for(nsig * (2 * h + 1), 256), 256, 0, cur>>>(X, Lf, N, cplx, sig0, nsig, h, out, Kp)));
    LAUNCHED("k_coef_gather");
    return FST_OK;
  }
  template <typename T>
  fst_status coef_mix_t(const CoefArgs<T> &a, const T *tot, const T *totU, const T *CA, const T *CB, const T *sq,
                        c2<T> *out, int64_t Kp, int64_t nF) {
    const int nfin = 4 * a.rH + 2 * a.DA + 2 * a.DB + a.r;
    dim3 grid((unsigned)((nfin + 127) / 128), (unsigned)a.batch);
    PROF("k_coef_mix", 0, (k_coef_mix<T><<<grid, 128, 0, cur>>>(a, tot, totU, CA, CB, sq, out, Kp, nF)));
    LAUNCHED("k_coef_mix");
    return FST_OK;
  }
  template <typename T> fst_status exp_scatter_t(const ExpArgs<T> &a, int64_t nsig, c2<T> *Xs) {
    PROF("k_exp_scatter", nsig, (k_exp_scatter<T><<<grid_for(nsig * a.N, 256), 256, 0, cur>>>(a, nsig, Xs)));
    LAUNCHED("k_exp_scatter");
    return FST_OK;
  }
  template <typename T> fst_status expand_t(const ExpArgs<T> &a, int64_t nsig) {
    const int64_t blocks = nsig * ((a.N + EXP_E * 256 - 1) / (EXP_E * 256));
    PROF("k_expand", nsig, (k_expand<T><<<(unsigned)std::min<int64_t>(blocks, 152 * 64), 256, 0, cur>>>(a, nsig)));
    LAUNCHED("k_expand");
    return FST_OK;
  }
  fst_status exp_scatter(const ExpArgs<float> &a, int64_t nsig, float2 *Xs) override { return exp_scatter_t(a, nsig, Xs); }
  fst_status exp_scatter(const ExpArgs<double> &a, int64_t nsig, double2 *Xs) override { return exp_scatter_t(a, nsig, Xs); }
  fst_status expand(const ExpArgs<float> &a, int64_t nsig) override { return expand_t(a, nsig); }
  fst_status expand(const ExpArgs<double> &a, int64_t nsig) override { return expand_t(a, nsig); }
  fst_status coef_lowrank(const CoefArgs<float> &a) override { return coef_lowrank_t(a); }
  fst_status coef_lowrank(const CoefArgs<double> &a) override { return coef_lowrank_t(a); }
  fst_status coef_st(const CoefArgs<float> &a) override { return coef_st_t(a); }
  fst_status coef_st(const CoefArgs<double> &a) override { return coef_st_t(a); }
  fst_status coef_reduce(const float *part, int nchunks, int nout, int64_t batch, float *tot) override {
    return coef_reduce_t(part, nchunks, nout, batch, tot);
  }
  fst_status coef_reduce(const double *part, int nchunks, int nout, int64_t batch, double *tot) override {
    return coef_reduce_t(part, nchunks, nout, batch, tot);
  }
  fst_status coef_gather(const float2 *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0, int64_t nsig,
                         int64_t h, float2 *out, int64_t Kp) override {
    return coef_gather_t<float>(X, Lf, N, cplx, sig0, nsig, h, out, Kp);
  }
  fst_status coef_gather(const double2 *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0, int64_t nsig,
                         int64_t h, double2 *out, int64_t Kp) override {
    return coef_gather_t<double>(X, Lf, N, cplx, sig0, nsig, h, out, Kp);
  }
  fst_status coef_mix(const CoefArgs<float> &a, const float *tot, const float *totU, const float *CA, const float *CB,
                      const float *sq, float2 *out, int64_t Kp, int64_t nF) override {
    return coef_mix_t(a, tot, totU, CA, CB, sq, out, Kp, nF);
  }
  fst_status coef_mix(const CoefArgs<double> &a, const double *tot, const double *totU, const double *CA,
                      const double *CB, const double *sq, double2 *out, int64_t Kp, int64_t nF) override {
    return coef_mix_t(a, tot, totU, CA, CB, sq, out, Kp, nF);
  }

  fst_status split_tf32(const float *src, float2 *hl, int64_t n) override {
    k_split_tf32<<<grid_for(n, 256), 256, 0, s>>>(src, hl, n);
    LAUNCHED("k_split_tf32");
    return FST_OK;
  }
  fst_status to_f32(const double *src, float *dst, int64_t n) override {
    k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    LAUNCHED("k_to_f32");
    return FST_OK;
  }
};

Runner *make_dev_runner() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return nullptr;
  }
  DevRunner *R = new DevRunner();
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&R->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  if (R->sms < 1) R->sms = 1;
  return R;
}

}  // namespace fst

using namespace fst;

extern "C" long long fst_launch_count(void) { return g_launches; }

// ---------------------------------------------------------------------------
// fst_project_noalloc: fst_project for callers that cannot allocate device memory
// when they project (for example a process whose memory manager owns all device
// memory after start-up).  The four-step path's scratch (intermediate spectra,
// per-tile partial sums and the correction coefficients) lives in one fixed
// file-scope device array instead of the plan's on-demand workspace.  Every device
// that loads this library holds the array until the process exits.
// ---------------------------------------------------------------------------
#define FST_NOALLOC_SCRATCH_BYTES (128ull << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[FST_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};   // context the address was looked up in
// the calling thread's current context (the primary context of the current device,
// re-created after a device reset)
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext *);
  static Fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (Fn)p;
    else
      cudaGetLastError();
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}
}  // namespace

extern "C" fst_status fst_project_noalloc(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld,
                                          int dtype, void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (!p->R->device()) return fail(FST_EINVAL, "fst_project_noalloc needs a device plan");
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(FST_EUNSUPPORTED, "device ordinal out of range");
  void *scratch = nullptr;
  {
    // set-up per device and context (with that device current): the host-side name of
    // the array is only a stand-in, its device address comes from the runtime; a new
    // context (after a device reset) gets the array at a new address
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    const CUcontext ctx = current_context();
    if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
      void *a = nullptr;
      CU(cudaGetSymbolAddress(&a, g_noalloc_scratch), "cudaGetSymbolAddress");
      g_scratch_addr[dev] = a;
      g_scratch_ctx[dev] = current_context();   // the runtime has made its context current
    }
    scratch = g_scratch_addr[dev];
  }
  p->R->set_stream(stream);
  // nothing in the scratch has to start at zero: every kernel writes the part it
  // later reads before reading it
  return run_apply_ws(p, y, out, batch, ld, dtype, true, scratch, (size_t)FST_NOALLOC_SCRATCH_BYTES);
}

extern "C" unsigned long long fst_noalloc_scratch_bytes(void) { return FST_NOALLOC_SCRATCH_BYTES; }

extern "C" fst_status fst_profile_enable(int on) {
  for (auto &r : g_prof) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  g_prof.clear();
  g_prof_on = on ? 1 : 0;
  return FST_OK;
}

extern "C" fst_status fst_profile_read(int i, const char **name, double *ms, long long *units) {
  if (i < 0 || i >= (int)g_prof.size()) return fail(FST_EINVAL, "profile index out of range");
  ProfRec &r = g_prof[i];
  float t = 0.f;
  if (r.a && r.b) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "event sync");
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "elapsed");
  }
  if (name) *name = r.name;
  if (ms) *ms = t;
  if (units) *units = r.units;
  return FST_OK;
}

extern "C" int fst_profile_count(void) { return (int)g_prof.size(); }

// ---------------------------------------------------------------------------
// host-buffer entry point: chunks of the batch go host -> device -> host on two
// copy streams while the previous / next chunk is projected on `stream`
// ---------------------------------------------------------------------------
namespace {
constexpr int HP_SLOTS = 4;   // chunks in flight: copy in, compute and copy out overlap freely
struct HostPipe {
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t in_done[HP_SLOTS] = {}, comp_done[HP_SLOTS] = {}, out_done[HP_SLOTS] = {};
  void *din[HP_SLOTS] = {}, *dout[HP_SLOTS] = {};
  size_t slot_bytes = 0;
  int dev = -1;
};
thread_local HostPipe *g_pipe = nullptr;
}  // namespace

extern "C" fst_status fst_project_host(fst_plan_t p, const void *y, void *out, int64_t batch, int dtype,
                                       void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FST_EINVAL, "batch < 0");
  if (batch == 0) return FST_OK;
  if (!y || !out) return fail(FST_EINVAL, "NULL signal pointer");
  if (!p->R->device()) return run_apply(p, y, out, batch, 0, dtype, true);
  size_t esz;
  switch (dtype) {
    case FST_F32: esz = 4; break;
    case FST_F64: esz = 8; break;
    case FST_C64: esz = 8; break;
    case FST_C128: esz = 16; break;
    default: return fail(FST_EINVAL, "unknown dtype");
  }
  const size_t sig_bytes = esz * (size_t)p->N;
  // chunk of the pipeline: FST_HOST_CHUNK_MB (default 64) MiB of signals
  const char *env = getenv("FST_HOST_CHUNK_MB");
  const int64_t chunk_mb = std::max<int64_t>(1, env ? atoll(env) : 64);
  int64_t per = std::max<int64_t>(2, (int64_t)(((size_t)chunk_mb << 20) / sig_bytes));
  per = (per / 2) * 2;
  per = std::min<int64_t>(per, ((batch + 1) / 2) * 2);
  const size_t slot = (size_t)per * sig_bytes;
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  if (!g_pipe || g_pipe->dev != dev || g_pipe->slot_bytes < slot) {
    if (g_pipe) {
      for (int i = 0; i < HP_SLOTS; ++i) {
        cudaFree(g_pipe->din[i]);
        cudaFree(g_pipe->dout[i]);
      }
    } else {
      g_pipe = new HostPipe();
    }
    if (!g_pipe->cin) {
      CU(cudaStreamCreateWithFlags(&g_pipe->cin, cudaStreamNonBlocking), "stream");
      CU(cudaStreamCreateWithFlags(&g_pipe->cout, cudaStreamNonBlocking), "stream");
      for (int i = 0; i < HP_SLOTS; ++i) {
        CU(cudaEventCreateWithFlags(&g_pipe->in_done[i], cudaEventDisableTiming), "event");
        CU(cudaEventCreateWithFlags(&g_pipe->comp_done[i], cudaEventDisableTiming), "event");
        CU(cudaEventCreateWithFlags(&g_pipe->out_done[i], cudaEventDisableTiming), "event");
      }
    }
    for (int i = 0; i < HP_SLOTS; ++i) {
      g_pipe->din[i] = g_pipe->dout[i] = nullptr;
      CU(cudaMalloc(&g_pipe->din[i], slot), "cudaMalloc");
      CU(cudaMalloc(&g_pipe->dout[i], slot), "cudaMalloc");
    }
    g_pipe->slot_bytes = slot;
    g_pipe->dev = dev;
  }
  HostPipe &hp = *g_pipe;
  cudaStream_t sc = (cudaStream_t)stream;
  p->R->set_stream(stream);
  // the copies must not start before earlier work on the compute stream is done
  CU(cudaEventRecord(hp.comp_done[0], sc), "event");
  CU(cudaStreamWaitEvent(hp.cin, hp.comp_done[0], 0), "wait");
  // chunk schedule: a short first chunk (compute starts after less copying), full chunks, and a
  // short last chunk (less copying after the last compute); every chunk but the last has an even
  // size, so real signals pair as in one call over the whole batch
  std::vector<int64_t> sizes;
  const int64_t small = std::max<int64_t>(2, (per / 4) / 2 * 2);
  if (per >= 8 && batch >= 2 * per + 2 * small) {
    const int64_t tail = small + (batch & 1);
    int64_t mid = batch - small - tail;
    sizes.push_back(small);
    while (mid > per) {
      sizes.push_back(per);
      mid -= per;
    }
    if (mid > 0) sizes.push_back(mid);
    sizes.push_back(tail);
  } else {
    for (int64_t b0 = 0; b0 < batch; b0 += per) sizes.push_back(std::min<int64_t>(per, batch - b0));
  }
  int64_t b0 = 0;
  for (size_t i = 0; i < sizes.size(); b0 += sizes[i], ++i) {
    const int k = (int)(i % HP_SLOTS);
    const int64_t nb = sizes[i];
    const size_t bytes = (size_t)nb * sig_bytes;
    if (i >= (size_t)HP_SLOTS) CU(cudaStreamWaitEvent(hp.cin, hp.out_done[k], 0), "wait");
    CU(cudaMemcpyAsync(hp.din[k], (const char *)y + b0 * sig_bytes, bytes, cudaMemcpyHostToDevice, hp.cin), "h2d");
    CU(cudaEventRecord(hp.in_done[k], hp.cin), "event");
    CU(cudaStreamWaitEvent(sc, hp.in_done[k], 0), "wait");
    fst_status s = run_apply(p, hp.din[k], hp.dout[k], nb, 0, dtype, true);
    if (s != FST_OK) return s;
    CU(cudaEventRecord(hp.comp_done[k], sc), "event");
    CU(cudaStreamWaitEvent(hp.cout, hp.comp_done[k], 0), "wait");
    CU(cudaMemcpyAsync((char *)out + b0 * sig_bytes, hp.dout[k], bytes, cudaMemcpyDeviceToHost, hp.cout), "d2h");
    CU(cudaEventRecord(hp.out_done[k], hp.cout), "event");
  }
  CU(cudaStreamSynchronize(hp.cout), "sync");
  CU(cudaStreamSynchronize(sc), "sync");
  return p->R->device_status(false);
}

// ---------------------------------------------------------------------------
// fst_project_ragged: the first call with a given (plans, signals) signature runs
// directly (allocating what it needs), the second records the whole batch into a
// CUDA graph, later ones replay it.
// ---------------------------------------------------------------------------
namespace {
struct RaggedCtx {
  std::vector<const void *> sig;
  std::vector<fst_plan_t> plans;   // the batch's plans, in call order
  std::vector<uint64_t> gens;      // their workspace generations when the graph was recorded
  fst::RaggedState state;          // descriptor arrays and workspaces (cudaMalloc), launch choices
  cudaGraphExec_t exec = nullptr;
  long long nodes = 0;
  int seen = 0;
};
std::recursive_mutex g_ragged_mu;
std::vector<RaggedCtx *> g_ragged;
// frees a context after every launch that may still use it has finished
void free_ctx(RaggedCtx *c) {
  cudaDeviceSynchronize();
  if (c->exec) cudaGraphExecDestroy(c->exec);
  for (void *b : c->state.bufs) cudaFree(b);
  delete c;
}
bool ctx_current(const RaggedCtx *c) {
  for (size_t i = 0; i < c->plans.size(); ++i)
    if (c->plans[i]->ws_gen != c->gens[i]) return false;
  return true;
}
cudaStream_t g_ragged_cap = nullptr;
bool ragged_graphs_enabled() {
  const char *s = getenv("FST_GRAPHS");
  return !(s && s[0] == '0');
}
}  // namespace

extern "C" fst_status fst_project_ragged(const fst_plan_t *plans, const void *const *y, void *const *out,
                                         int64_t count, int dtype, void *stream) {
  if (count < 0 || (count > 0 && (!plans || !y || !out))) return fail(FST_EINVAL, "bad arguments");
  if (count == 0) return FST_OK;
  for (int64_t i = 0; i < count; ++i)
    if (!plans[i]) return fail(FST_EINVAL, "NULL plan");
  if (!plans[0]->R->device()) {
    RaggedState rs;
    fst_status st = run_ragged(plans, y, out, count, dtype, rs);
    for (void *b : rs.bufs) plans[0]->R->release(b);
    return st;
  }
  std::lock_guard<std::recursive_mutex> lk(g_ragged_mu);
  std::vector<const void *> sig;
  sig.reserve(3 * count + 1);
  sig.push_back((const void *)(intptr_t)dtype);
  for (int64_t i = 0; i < count; ++i) {
    sig.push_back(plans[i]);
    sig.push_back(y[i]);
    sig.push_back(out[i]);
  }
  RaggedCtx *ctx = nullptr;
  for (RaggedCtx *c : g_ragged)
    if (c->sig == sig) ctx = c;
  cudaStream_t us = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(us, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;
  }
  const bool graphs = ragged_graphs_enabled() && !profiling_enabled() && cs == cudaStreamCaptureStatusNone;
  if (ctx && ctx->exec && !ctx_current(ctx)) {
    // a plan's workspace moved since the recording: run directly, record again next time
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(ctx->exec);
    ctx->exec = nullptr;
    ctx->seen = 0;
  }
  if (ctx && ctx->exec && graphs) {
    CU(cudaGraphLaunch(ctx->exec, us), "cudaGraphLaunch");
    g_launches += ctx->nodes;
    return FST_OK;
  }
  if (!ctx) {
    if (g_ragged.size() >= 4) {
      free_ctx(g_ragged.front());
      g_ragged.erase(g_ragged.begin());
    }
    ctx = new RaggedCtx();
    ctx->sig = sig;
    ctx->plans.assign(plans, plans + count);
    g_ragged.push_back(ctx);
  }
  for (int64_t i = 0; i < count; ++i) plans[i]->R->set_stream(stream);
  if (ctx->seen == 0 || !graphs) {
    ctx->seen = 1;
    return run_ragged(plans, y, out, count, dtype, ctx->state);
  }
  // second call: record the batch into a graph on a private stream
  if (!g_ragged_cap) CU(cudaStreamCreateWithFlags(&g_ragged_cap, cudaStreamNonBlocking), "stream");
  for (int64_t i = 0; i < count; ++i) plans[i]->R->set_stream((void *)g_ragged_cap);
  const long long l0 = g_launches;
  CU(cudaStreamBeginCapture(g_ragged_cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  fst_status st = run_ragged(plans, y, out, count, dtype, ctx->state);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(g_ragged_cap, &g);
  for (int64_t i = 0; i < count; ++i) plans[i]->R->set_stream(stream);
  ctx->nodes = g_launches - l0;
  g_launches = l0;
  if (st != FST_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&ctx->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  ctx->gens.resize(count);
  for (int64_t i = 0; i < count; ++i) ctx->gens[i] = plans[i]->ws_gen;
  CU(cudaGraphLaunch(ctx->exec, us), "cudaGraphLaunch");
  g_launches += ctx->nodes;
  return FST_OK;
}

namespace fst {
// A plan about to be destroyed: every recorded ragged batch that uses it points at its
// device data and is dropped (after its launches finish), with its descriptor arrays.
void forget_ragged(fst_plan_t p) {
  std::lock_guard<std::recursive_mutex> lk(g_ragged_mu);
  for (size_t i = 0; i < g_ragged.size();) {
    RaggedCtx *c = g_ragged[i];
    if (std::find(c->plans.begin(), c->plans.end(), p) != c->plans.end()) {
      free_ctx(c);
      g_ragged.erase(g_ragged.begin() + i);
    } else {
      ++i;
    }
  }
}
}  // namespace fst

extern "C" fst_status fst_ragged_tuning(const fst_plan_t *plans, const void *const *y, void *const *out,
                                        int64_t count, int dtype, int64_t *pairs, double *ms) {
  if (count <= 0 || !plans || !y || !out || !pairs) return fail(FST_EINVAL, "bad arguments");
  std::lock_guard<std::recursive_mutex> lk(g_ragged_mu);
  std::vector<const void *> sig;
  sig.reserve(3 * count + 1);
  sig.push_back((const void *)(intptr_t)dtype);
  for (int64_t i = 0; i < count; ++i) {
    sig.push_back(plans[i]);
    sig.push_back(y[i]);
    sig.push_back(out[i]);
  }
  for (RaggedCtx *c : g_ragged)
    if (c->sig == sig) {
      for (int lg = 0; lg < 32; ++lg) {
        pairs[lg] = lg < (int)c->state.chunk.size() ? c->state.chunk[lg] : 0;
        if (ms) ms[lg] = lg < (int)c->state.tune_ms.size() ? c->state.tune_ms[lg] : 0.0;
      }
      return FST_OK;
    }
  return fail(FST_EINVAL, "no ragged call with this signature has run");
}

extern "C" fst_status fst_test_tc_stall(int launches, double limit_s) {
  if (launches < 0 || !(limit_s > 0.0) || limit_s > 2.0) return fail(FST_EINVAL, "bad stall request");
  fst::g_tc_stall_limit_ns = (unsigned long long)(limit_s * 1e9);
  fst::g_tc_stall.store(launches);
  return FST_OK;
}
