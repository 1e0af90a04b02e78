// fst_internal.h -- plan structure, launch layouts and the execution back-ends of
// the fast Slepian projection library.
//
// All host logic (plan construction, launch sequencing) is written once against
// the abstract Runner.  DevRunner (fst_device.cu) enqueues CUDA kernels on a
// stream and owns device memory; EmuRunner (fst_emu.cu) executes the very same
// kernel bodies on the host, one block at a time, for CPU tests.
#pragma once
#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

#include "../../include/fst.h"
#include "fst_kernels.cuh"
#include "fst_plan_kernels.cuh"
#include "fst_coeffs.cuh"

namespace fst {

Layout make_layout(int64_t N, int log2M, bool dbl, int rpad, bool allow_fast = false);
struct Runner {
  virtual ~Runner() {}
  virtual bool device() const = 0;
  virtual void set_stream(void *) {}
  virtual void *stream() const { return nullptr; }
  // CUDA-graph capture of a whole apply (device runner only).  While capturing,
  // lanes() == 2 and use_lane(i) selects one of two capture streams, so that
  // consecutive launch groups overlap.
  virtual bool graph_begin() { return false; }
  virtual fst_status graph_end(void **exec, long long *nodes) { return FST_EUNSUPPORTED; }
  virtual fst_status graph_launch(void *exec, long long nodes) { return FST_EUNSUPPORTED; }
  virtual void graph_destroy(void *exec) {}
  virtual bool user_stream_capturing() { return false; }
  virtual int lanes() const { return 1; }
  virtual void use_lane(int) {}
  // order lane 1 after everything lane 0 has issued so far
  virtual void lanes_after_first() {}
  // order lane 0 after everything lane 1 has issued so far
  virtual void lanes_join_first() {}
  // side lane (capture only): the separate correction runs there, beside the first passes
  // of the launch groups; side_done() marks its end and wait_side() orders the current lane
  // after that mark.  Without a capture all of it is one stream (no-ops).
  virtual void use_side() {}
  virtual void side_done() {}
  virtual void wait_side() {}
  virtual fst_status alloc(void **p, size_t bytes) = 0;
  virtual void release(void *p) = 0;
  virtual fst_status h2d(void *dst, const void *src, size_t bytes) = 0;
  virtual fst_status d2h(void *dst, const void *src, size_t bytes) = 0;  // synchronous
  virtual fst_status d2d(void *dst, const void *src, size_t bytes) = 0;
  virtual fst_status zero(void *p, size_t bytes) = 0;
  virtual fst_status sync() = 0;
  // device timing of the runner's stream: phase 0 records the start, phase 1 the end, waits
  // for it and writes the elapsed milliseconds
  virtual fst_status timer(int phase, double *ms) {
    if (ms) *ms = 0.0;
    return FST_OK;
  }
  // FST_ETIMEOUT (and clears it) when a bounded device wait of an earlier launch gave up;
  // with `sync`, first waits for the runner's stream
  virtual fst_status device_status(bool sync) { return sync ? this->sync() : FST_OK; }

  virtual fst_status small(const ConvArgs<float> &a, const Layout &L) = 0;
  virtual fst_status small(const ConvArgs<double> &a, const Layout &L) = 0;
  virtual fst_status passA(const ConvArgs<float> &a, const Layout &L) = 0;
  virtual fst_status passA(const ConvArgs<double> &a, const Layout &L) = 0;
  virtual fst_status reduce(const ConvArgs<float> &a, const Layout &L) = 0;
  virtual fst_status reduce(const ConvArgs<double> &a, const Layout &L) = 0;
  virtual fst_status passB(const ConvArgs<float> &a, const Layout &L) = 0;
  virtual fst_status passB(const ConvArgs<double> &a, const Layout &L) = 0;
  virtual fst_status passC(const ConvArgs<float> &a, const Layout &L) = 0;
  virtual fst_status passC(const ConvArgs<double> &a, const Layout &L) = 0;
  // ragged batch: one single-CTA transform per descriptor (all with FFT length 2^base.log2M)
  virtual fst_status small_ragged(const RaggedDesc<float> *d, int count, const ConvArgs<float> &base,
                                  const Layout &L) = 0;
  virtual fst_status small_ragged(const RaggedDesc<double> *d, int count, const ConvArgs<double> &base,
                                  const Layout &L) = 0;
  // separate correction (FP32, device): partials, reduce to a = D o c, out += S_T a
  virtual fst_status corr_c(const ConvArgs<float> &a) { return FST_EUNSUPPORTED; }
  // tcgen05 S_T^T y over every pair of a (a.pair0 = 0): partials [pair][a.nkb][2][rpad]
  virtual fst_status corr_tc(const ConvArgs<float> &a) { return FST_EUNSUPPORTED; }
  virtual fst_status tc_prep(const float *ST, int64_t N, int rpad, int r, int nB, int64_t Npad, float *STt) {
    return FST_EUNSUPPORTED;
  }
  virtual int sm_count() const { return 1; }
  virtual fst_status corr_reduce(const ConvArgs<float> &a, const float *scale) { return FST_EUNSUPPORTED; }
  virtual fst_status corr_z(const ConvArgs<float> &a) { return FST_EUNSUPPORTED; }
  // T1 c (fst_expand): scatter of the F bins of nsig signals into Xs, then the samples
  virtual fst_status exp_scatter(const ExpArgs<float> &a, int64_t nsig, float2 *Xs) = 0;
  virtual fst_status exp_scatter(const ExpArgs<double> &a, int64_t nsig, double2 *Xs) = 0;
  virtual fst_status expand(const ExpArgs<float> &a, int64_t nsig) = 0;
  virtual fst_status expand(const ExpArgs<double> &a, int64_t nsig) = 0;
  // out += S_T a on CUDA cores (FP32, r <= 64)
  virtual fst_status z_rmw(const ConvArgs<float> &a, const float *ST) { return FST_EUNSUPPORTED; }
  // ragged four-step signals (FP32 device): correction partials per item, a per signal, and
  // out += S_T a per item (descriptor arrays in runner memory)
  virtual fst_status rcorr(const RSig *sigs, int nsig, const RItem *items, int nitems, int cplx, float *part,
                           float *acoef) { return FST_EUNSUPPORTED; }
  virtual fst_status rzadd(const RSig *sigs, const RItem *items, int nitems, int cplx, const float *acoef) {
    return FST_EUNSUPPORTED;
  }
  // S_T^T y partials per CORR_BLOCK samples on CUDA cores (FP32, at most 32 signal rows, rpad <= 64)
  virtual fst_status corr_cc(const ConvArgs<float> &a) { return FST_EUNSUPPORTED; }
  // out += S_T a on CUDA cores over the whole batch (FP32, rpad <= 64, any number of rows)
  virtual fst_status zadd(const ConvArgs<float> &a) { return FST_EUNSUPPORTED; }

  // plan kernels (all pointers in runner memory)
  // batched eigen-targets of one or many plans (descriptors and data in runner memory):
  // multisection (a block of BISECT_THREADS per target) or plain bisection (a thread per target)
  virtual fst_status bisect_ms_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat,
                                    double *theta, int *flag) = 0;
  virtual fst_status bisect_many(const TargetDesc *td, int nt, const double *dcat, const double *e2cat,
                                 double *theta, int *flag) = 0;
  virtual fst_status invit_many(const TargetDesc *td, int nt, const double *dcat, const double *ecat,
                                const double *theta, double *x, double *fd, double *fdl, double *fdu, double *fdu2,
                                uint8_t *piv) = 0;
  virtual fst_status finalize_many(const TargetDesc *td, int nt, const double *x) = 0;
  virtual fst_status dot(const double *a, const double *b, int64_t N, int nvec, double *out) = 0;
  virtual fst_status sinc_embed(double *c, int64_t N, int64_t M, double W) = 0;
  virtual fst_status spec_store(const double2 *X, const Layout &L64, const Layout &L32, int64_t M, double scale,
                                double *spec64, float *spec32) = 0;
  virtual fst_status gather_ST(const double *S, int64_t N, const int *sel, int r, int rpad, double *ST64,
                               float *ST32) = 0;
  virtual fst_status to_f32(const double *src, float *dst, int64_t n) = 0;
  virtual fst_status split_tf32(const float *src, float2 *hl, int64_t n) = 0;

  // fast coefficient vector kernels (runner memory)
  virtual fst_status coef_lowrank(const CoefArgs<float> &a) = 0;
  virtual fst_status coef_lowrank(const CoefArgs<double> &a) = 0;
  virtual fst_status coef_st(const CoefArgs<float> &a) = 0;
  virtual fst_status coef_st(const CoefArgs<double> &a) = 0;
  virtual fst_status coef_reduce(const float *part, int nchunks, int nout, int64_t batch, float *tot) = 0;
  virtual fst_status coef_reduce(const double *part, int nchunks, int nout, int64_t batch, double *tot) = 0;
  virtual fst_status coef_gather(const float2 *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0,
                                 int64_t nsig, int64_t h, float2 *out, int64_t Kp) = 0;
  virtual fst_status coef_gather(const double2 *X, const Layout &Lf, int64_t N, int cplx, int64_t sig0,
                                 int64_t nsig, int64_t h, double2 *out, int64_t Kp) = 0;
  virtual fst_status coef_mix(const CoefArgs<float> &a, const float *tot, const float *totU, const float *CA,
                              const float *CB, const float *sqrtD, float2 *out, int64_t Kp, int64_t nF) = 0;
  virtual fst_status coef_mix(const CoefArgs<double> &a, const double *tot, const double *totU, const double *CA,
                              const double *CB, const double *sqrtD, double2 *out, int64_t Kp, int64_t nF) = 0;
};

Runner *make_dev_runner();
Runner *make_emu_runner();

}  // namespace fst

namespace fst {
// Lazily built data of the fast coefficient vector T2^* y (Theorem 1 construction).
struct CoefPlan {
  int64_t odd = 0, h = 0;        // 2NW' = odd = 2h + 1
  double Wp = 0;
  int rH = 0, rA = 0, rB = 0, DA = 0, DB = 0, nraw = 0, r1 = 0;
  std::vector<double> p;         // ADI shifts
  float *zfirst32 = nullptr, *zshift32 = nullptr, *CA32 = nullptr, *CB32 = nullptr, *sqrtD32 = nullptr;
  double *zfirst64 = nullptr, *zshift64 = nullptr, *CA64 = nullptr, *CB64 = nullptr, *sqrtD64 = nullptr;
  float2 *phA32 = nullptr, *phB32 = nullptr;
  double2 *phA64 = nullptr, *phB64 = nullptr;
};
}  // namespace fst

struct fst_plan_s {
  fst::Runner *R = nullptr;
  fst::CoefPlan *coef = nullptr;
  int64_t N = 0, K = 0, M = 0, r = 0, rpad = 0, win_lo = 0, win_hi = 0;
  int log2M = 0;
  double W = 0, eps = 0, alpha = 0, beta = 1;
  int op = 0;
  fst::Layout lay32, lay64;
  float *spec32 = nullptr, *ST32 = nullptr, *D32 = nullptr;
  float2 *ST32_hl = nullptr;  // TF32 (hi, lo) split of ST32, interleaved
  float *STt = nullptr;       // S_T^T, K-major FP32 [tc_nB][tc_Npad], for the tcgen05 correction
  int tc_nB = 0;
  int64_t tc_Npad = 0;
  double *spec64 = nullptr, *ST64 = nullptr, *D64 = nullptr;
  double *spec_unit = nullptr;   // plan-time only: DFT_M(c) / M for the eigenvalues
  float2 *tw32h = nullptr, *tw32l = nullptr;
  // stage twiddles of the 4096-point row FFT: [t][k] = W_256^{k t} (k < 16), then
  // W_4096^{k t} (k < 256), t < 16
  float2 *twB = nullptr;
  float2 *tw8 = nullptr;   // stage twiddles of the 8192-point row FFT (FP64 built)
  double2 *tw64h = nullptr, *tw64l = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t ws_gen = 0;   // bumped whenever ws is reallocated (recorded graphs point into it)
  std::vector<int64_t> idx;
  std::vector<double> lam, D;
  std::vector<double> lam_window;
  struct GraphEntry {
    const void *y;
    void *out;
    int64_t batch, ld;
    int dtype;
    bool full;
    void *exec;
    long long nodes;
  };
  std::vector<GraphEntry> graphs;   // cached whole-apply CUDA graphs (device plans)
};

namespace fst {
void set_error(const std::string &msg);
fst_status fail(fst_status st, const std::string &msg);
// build a plan with the given runner (takes ownership of R)
fst_status build_plan(Runner *R, fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op,
                      double alpha);
// B y (+ correction when full) for `batch` signals in runner memory
fst_status run_apply(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype, bool full);
// as run_apply with caller-provided scratch `ws` of ws_bytes (nullptr: the plan's own,
// allocated on demand); with caller scratch nothing is allocated
fst_status run_apply_ws(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype, bool full,
                        void *ws, size_t ws_bytes);
void destroy_plan(fst_plan_t p);
bool profiling_enabled();   // per-launch event timing is on (fst_profile_enable)
// Device buffers and launch choices of one ragged signature (owned by the caller): the first
// call allocates in a fixed order, later calls with the same signature reuse them in that order
struct RaggedState {
  std::vector<void *> bufs;
  size_t next = 0;                  // cursor into bufs during a call
  bool tuned = false;
  std::vector<int64_t> chunk;       // pairs per launch group of each four-step length class, by log2 M
  std::vector<double> tune_ms;      // measured time of the chosen grouping, by log2 M
};
// ragged batch on the plans' runners (buffers and tuning in st)
fst_status run_ragged(const fst_plan_t *plans, const void *const *y, void *const *out, int64_t count, int dtype,
                      RaggedState &st);
// drop every recorded ragged batch that uses plan p (before p or its workspace is freed)
void forget_ragged(fst_plan_t p);
// a test-requested stall of the tcgen05 correction is pending / consume one
bool tc_stall_pending();
bool tc_stall_take();
fst_status build_plans_many(Runner *(*mk)(), void *stream, int64_t count, const int64_t *N, const double *W,
                            const int64_t *K, const double *eps, fst_plan_t *out);
}  // namespace fst
