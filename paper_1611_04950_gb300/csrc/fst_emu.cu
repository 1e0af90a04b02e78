// fst_emu.cu -- host emulation back-end: runs the library's kernel bodies on the
// CPU, one thread block at a time, with the block's threads looped inside each
// phase (a phase ends where the device kernel has a __syncthreads()).  Buffers live
// in host memory.  Used by the CPU test-suite to check index arithmetic, layouts
// and the plan logic without a GPU.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fst_internal.h"

namespace fst {

template <typename S> struct HostEx {
  using State = S;
  int nthr;
  std::vector<State> st;
  explicit HostEx(int n) : nthr(n), st(n) {}
  template <typename F> void phase(F &&f) {
    for (int t = 0; t < nthr; ++t) f(t, st[t]);
  }
};
struct NoStateH {
  c2<double> v[1];
};

struct EmuRunner : Runner {
  bool device() const override { return false; }
  fst_status alloc(void **p, size_t bytes) override {
    *p = calloc(1, std::max<size_t>(bytes, 16));
    if (!*p) return fail(FST_ENOMEM, "host allocation failed");
    return FST_OK;
  }
  void release(void *p) override { free(p); }
  fst_status h2d(void *dst, const void *src, size_t bytes) override { memcpy(dst, src, bytes); return FST_OK; }
  fst_status d2h(void *dst, const void *src, size_t bytes) override { memcpy(dst, src, bytes); return FST_OK; }
  fst_status d2d(void *dst, const void *src, size_t bytes) override { memmove(dst, src, bytes); return FST_OK; }
  fst_status zero(void *p, size_t bytes) override { memset(p, 0, bytes); return FST_OK; }
  fst_status sync() override { return FST_OK; }

  template <typename T> fst_status small_t(const ConvArgs<T> &a, const Layout &L) {
    std::vector<unsigned char> smem(L.smem_small + 64);
    const int Lsz = 1 << a.log2M;
    c2<T> *buf = reinterpret_cast<c2<T> *>(smem.data());
    T *red = reinterpret_cast<T *>(smem.data() + padded_size(Lsz) * sizeof(c2<T>));
    T *coef = red + ((L.nthr_small + 31) / 32) * 128;
    for (int64_t pl = 0; pl < a.npairs; ++pl) {
      HostEx<KState<T>> ex(L.nthr_small);
      small_body<T>(ex, a, pl, buf, red, coef);
    }
    return FST_OK;
  }
  template <typename T> fst_status passA_t(const ConvArgs<T> &a, const Layout &L) {
    std::vector<unsigned char> smem(L.smem_A + 64);
    const int P = 1 << a.log2P;
    c2<T> *buf = reinterpret_cast<c2<T> *>(smem.data());
    T *red = reinterpret_cast<T *>(smem.data() + padded_size(P * a.G * a.NB) * sizeof(c2<T>));
    const int64_t ngroups = (a.npairs + L.G - 1) / L.G;
    for (int64_t g = 0; g < ngroups; ++g)
      for (int64_t t = 0; t < L.ntiles; ++t) {
        HostEx<KState<T>> ex(L.nthr_A);
        passA_body<T>(ex, a, t, g, buf, red);
      }
    return FST_OK;
  }
  template <typename T> fst_status reduce_t(const ConvArgs<T> &a, const Layout &) {
    for (int64_t pl = 0; pl < a.npairs; ++pl)
      for (int t = 0; t < 64; ++t) reduce_body<T>(a, pl, t, 64);
    return FST_OK;
  }
  template <typename T> fst_status passB_t(const ConvArgs<T> &a, const Layout &L) {
    if (a.two_spec) return FST_EUNSUPPORTED;   // two-spectrum ragged slots run on the device only
    std::vector<unsigned char> smem(L.smem_B + 64);
    c2<T> *buf = reinterpret_cast<c2<T> *>(smem.data());
    for (int64_t pl = 0; pl < a.npairs; ++pl)
      for (int k1 = 0; k1 < (1 << L.log2P); ++k1) {
        HostEx<KState<T>> ex(L.nthr_B);
        passB_body<T>(ex, a, pl, k1, buf);
      }
    return FST_OK;
  }
  template <typename T> fst_status passC_t(const ConvArgs<T> &a, const Layout &L) {
    std::vector<unsigned char> smem(L.smem_C + 64);
    c2<T> *buf = reinterpret_cast<c2<T> *>(smem.data());
    const int64_t ngroups = (a.npairs + L.G - 1) / L.G;
    for (int64_t g = 0; g < ngroups; ++g)
      for (int64_t t = 0; t < L.ntiles; ++t) {
        HostEx<KState<T>> ex(L.nthr_C);
        passC_body<T>(ex, a, t, g, buf);
      }
    return FST_OK;
  }
  template <typename T>
  fst_status small_ragged_t(const RaggedDesc<T> *d, int count, const ConvArgs<T> &base, const Layout &L) {
    std::vector<unsigned char> smem(L.smem_small + 64);
    const int Lsz = 1 << base.log2M;
    c2<T> *buf = reinterpret_cast<c2<T> *>(smem.data());
    T *red = reinterpret_cast<T *>(smem.data() + padded_size(Lsz) * sizeof(c2<T>));
    T *coef = red + ((L.nthr_small + 31) / 32) * 128;
    for (int i = 0; i < count; ++i) {
      ConvArgs<T> a = base;
      a.y = d[i].y;
      a.out = d[i].out;
      a.ld = d[i].N;
      a.N = d[i].N;
      a.spec = d[i].spec;
      a.ST = d[i].ST;
      a.D = d[i].D;
      a.r = d[i].r;
      a.rpad = d[i].rpad;
      HostEx<KState<T>> ex(L.nthr_small);
      small_body<T>(ex, a, 0, buf, red, coef);
    }
    return FST_OK;
  }
  fst_status small_ragged(const RaggedDesc<float> *d, int count, const ConvArgs<float> &base,
                          const Layout &L) override { return small_ragged_t(d, count, base, L); }
  fst_status small_ragged(const RaggedDesc<double> *d, int count, const ConvArgs<double> &base,
                          const Layout &L) override { return small_ragged_t(d, count, base, L); }
  fst_status small(const ConvArgs<float> &a, const Layout &L) override { return small_t(a, L); }
  fst_status small(const ConvArgs<double> &a, const Layout &L) override { return small_t(a, L); }
  fst_status passA(const ConvArgs<float> &a, const Layout &L) override { return passA_t(a, L); }
  fst_status passA(const ConvArgs<double> &a, const Layout &L) override { return passA_t(a, L); }
  fst_status reduce(const ConvArgs<float> &a, const Layout &L) override { return reduce_t(a, L); }
  fst_status reduce(const ConvArgs<double> &a, const Layout &L) override { return reduce_t(a, L); }
  fst_status passB(const ConvArgs<float> &a, const Layout &L) override { return passB_t(a, L); }
  fst_status passB(const ConvArgs<double> &a, const Layout &L) override { return passB_t(a, L); }
  fst_status passC(const ConvArgs<float> &a, const Layout &L) override { return passC_t(a, L); }
  fst_status passC(const ConvArgs<double> &a, const Layout &L) override { return passC_t(a, L); }

  fst_status bisect_ms_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat, double *theta,
                            int *flag) override {
    for (int t = 0; t < nt; ++t) {
      const TargetDesc &q = td[t];
      BisectShared sh;
      HostEx<NoStateH> ex(BISECT_THREADS);
      bisect_body(ex, dcat + q.mat_off, e2cat + q.mat_off, q.n, q.target, q.glo, q.ghi, q.pivmin, q.tol, theta + t, flag,
                  &sh);
    }
    return FST_OK;
  }
  fst_status bisect_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat, double *theta,
                         int *flag) override {
    for (int t = 0; t < nt; ++t) {
      const TargetDesc &q = td[t];
      bisect1_body(dcat + q.mat_off, e2cat + q.mat_off, q.n, q.target, q.glo, q.ghi, q.pivmin, q.tol, theta + t, flag);
    }
    return FST_OK;
  }
  fst_status invit_many(const TargetDesc *td, int nt, const double *dcat, const double *ecat, const double *theta,
                        double *x, double *fd, double *fdl, double *fdu, double *fdu2, uint8_t *piv) override {
    for (int t = 0; t < nt; ++t) {
      const TargetDesc &q = td[t];
      invit_body(dcat + q.mat_off, ecat + q.mat_off, q.n, theta[t], q.tol, 3, 0, 1, x + q.x_off, fd + q.x_off,
                 fdl + q.x_off, fdu + q.x_off, fdu2 + q.x_off, piv + q.x_off);
    }
    return FST_OK;
  }
  fst_status finalize_many(const TargetDesc *td, int nt, const double *x) override {
    std::vector<double> sh(2 * 256);
    for (int t = 0; t < nt; ++t) {
      const TargetDesc &q = td[t];
      HostEx<NoStateH> ex(256);
      finalize_body(ex, x + q.x_off, q.n, 1, 0, q.parity, q.N, q.S, sh.data());
    }
    return FST_OK;
  }
  fst_status dot(const double *a, const double *b, int64_t N, int nvec, double *out) override {
    std::vector<double> sh(256);
    for (int v = 0; v < nvec; ++v) {
      HostEx<NoStateH> ex(256);
      dot_body(ex, a + (int64_t)v * N, b + (int64_t)v * N, N, out + v, sh.data());
    }
    return FST_OK;
  }
  fst_status sinc_embed(double *c, int64_t N, int64_t M, double W) override {
    for (int64_t k = 0; k < M; ++k) c[k] = sinc_embed_at(k, N, M, W);
    return FST_OK;
  }
  fst_status spec_store(const double2 *X, const Layout &L64, const Layout &L32, int64_t M, double scale,
                        double *spec64, float *spec32) override {
    for (int64_t k = 0; k < M; ++k) {
      const int64_t p64 = spec_pos(L64, k);
      const double v = X[p64].x * scale;
      spec64[p64] = v;
      spec32[spec_pos(L32, k)] = (float)v;
    }
    return FST_OK;
  }
  fst_status gather_ST(const double *S, int64_t N, const int *sel, int r, int rpad, double *ST64,
                       float *ST32) override {
    for (int64_t n = 0; n < N; ++n)
      for (int j = 0; j < rpad; ++j) {
        const double v = (j < r) ? S[(int64_t)sel[j] * N + n] : 0.0;
        ST64[n * rpad + j] = v;
        ST32[n * rpad + j] = (float)v;
      }
    return FST_OK;
  }
  fst_status to_f32(const double *src, float *dst, int64_t n) override {
    for (int64_t i = 0; i < n; ++i) dst[i] = (float)src[i];
    return FST_OK;
  }
  template <typename T> fst_status coef_lowrank_t(const CoefArgs<T> &a) {
    std::vector<T> red(COEF_RED_WORDS);
    for (int64_t sig = 0; sig < a.batch; ++sig)
      for (int c = 0; c < a.nchunks; ++c) {
        HostEx<CState<T>> ex(COEF_THREADS);
        coef_lowrank_body<T>(ex, a, sig, c, red.data());
      }
    return FST_OK;
  }
  template <typename T> fst_status exp_scatter_t(const ExpArgs<T> &a, int64_t nsig, c2<T> *Xs) {
    for (int64_t s = 0; s < nsig; ++s)
      for (int64_t n = 0; n < a.N; ++n) exp_scatter_body<T>(a, s, n, Xs);
    return FST_OK;
  }
  template <typename T> fst_status expand_t(const ExpArgs<T> &a, int64_t nsig) {
    const int64_t blk = EXP_E * 256;
    for (int64_t s = 0; s < nsig; ++s)
      for (int64_t b0 = 0; b0 < a.N; b0 += blk)
        for (int t = 0; t < 256; ++t) exp_samples_body<T>(a, s, b0 + t, 256);
    return FST_OK;
  }
  fst_status exp_scatter(const ExpArgs<float> &a, int64_t nsig, float2 *Xs) override { return exp_scatter_t(a, nsig, Xs); }
  fst_status exp_scatter(const ExpArgs<double> &a, int64_t nsig, double2 *Xs) override { return exp_scatter_t(a, nsig, Xs); }
  fst_status expand(const ExpArgs<float> &a, int64_t nsig) override { return expand_t(a, nsig); }
  fst_status expand(const ExpArgs<double> &a, int64_t nsig) override { return expand_t(a, nsig); }
  template <typename T> fst_status coef_st_t(const CoefArgs<T> &a) {
    std::vector<T> red((COEF_THREADS / 32) * 128);
    for (int64_t sig = 0; sig < a.batch; ++sig)
      for (int c = 0; c < a.nchunks; ++c) {
        HostEx<CState<T>> ex(COEF_THREADS);
        coef_st_body<T>(ex, a, sig, c, red.data());
      }
    return FST_OK;
  }
  template <typename T> fst_status coef_reduce_t(const T *part, int nchunks, int nout, int64_t batch, T *tot) {
    for (int64_t sig = 0; sig < batch; ++sig)
      for (int o = 0; o < nout; ++o) coef_reduce_body<T>(part, nchunks, nout, sig, o, tot);
    return FST_OK;
  }
  template <typename T>
  fst_status coef_gather_t(const c2<T> *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0, int64_t nsig,
                           int64_t h, c2<T> *out, int64_t Kp) {
    for (int64_t s = sig0; s < sig0 + nsig; ++s)
      for (int64_t k = 0; k < 2 * h + 1; ++k) {
        const int64_t pl = cplx ? (s - sig0) : (s / 2 - sig0 / 2);
        coef_gather_body<T>(X, Lf, N, cplx, s, pl, h, k, out + s * Kp);
      }
    return FST_OK;
  }
  template <typename T>
  fst_status coef_mix_t(const CoefArgs<T> &a, const T *tot, const T *totU, const T *CA, const T *CB, const T *sq,
                        c2<T> *out, int64_t Kp, int64_t nF) {
    const int nfin = 4 * a.rH + 2 * a.DA + 2 * a.DB + a.r;
    for (int64_t sig = 0; sig < a.batch; ++sig)
      for (int o = 0; o < nfin; ++o)
        out[sig * Kp + nF + o] = coef_mix_value<T>(a, tot + sig * (int64_t)a.nraw * 2,
                                                    totU + sig * (int64_t)(a.r > 0 ? a.r : 1) * 2, CA, CB, sq, o, sig);
    return FST_OK;
  }
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
    for (int64_t i = 0; i < n; ++i) {
      const float h = tf32_round(src[i]);
      hl[i] = make_float2(h, tf32_round(src[i] - h));
    }
    return FST_OK;
  }
};

Runner *make_emu_runner() { return new EmuRunner(); }

}  // namespace fst
