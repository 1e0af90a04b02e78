// fst_host.cu -- plan construction, launch sequencing and the C ABI of the fast
// Slepian projection library.  Written against the abstract Runner, so the same
// code drives the GPU (DevRunner) and the host emulator (EmuRunner).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fst_internal.h"
#include "fst_tc.cuh"
#include "../../include/fst_testing.h"

namespace fst {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
fst_status fail(fst_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

#define TRY(expr)                         \
  do {                                    \
    fst_status _s = (expr);               \
    if (_s != FST_OK) return _s;          \
  } while (0)

static int ilog2_exact(int64_t x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

// ---------------------------------------------------------------------------
// layouts
// ---------------------------------------------------------------------------

static int64_t chunk_bytes_target() {
  const char *s = getenv("FST_CHUNK_MB");
  int64_t mb = s ? atoll(s) : 128;
  if (mb < 1) mb = 1;
  return mb << 20;
}

Layout make_layout(int64_t N, int log2M, bool dbl, int rpad, bool allow_fast) {
  Layout L;
  const size_t cs = dbl ? 16 : 8;   // bytes per complex
  const size_t rs = dbl ? 8 : 4;    // bytes per real
  L.log2M = log2M;
  const int small_max = dbl ? 13 : 14;
  const int64_t M = 1LL << log2M;
  if (log2M <= small_max) {
    L.small = true;
    const int Lsz = 1 << log2M;
    int nthr = Lsz / 16;
    nthr = std::max(64, std::min(1024, nthr));
    L.nthr_small = nthr;
    const int nwarps = (nthr + 31) / 32;
    L.smem_small = padded_size(Lsz) * cs + (size_t)nwarps * 128 * rs + 2 * (size_t)std::max(rpad, 1) * rs;
    L.chunk = std::max<int64_t>(1, chunk_bytes_target() / (int64_t)(M * cs));
    return L;
  }
  L.small = false;
  if (dbl) {
    L.log2Q = std::min(13, std::max(11, log2M - 5));
  } else {
    // FP32: 4096-point rows up to M = 2^22 (P <= 1024), then P = 1024 with longer rows
    L.log2Q = log2M <= 22 ? 12 : log2M - 10;
  }
  L.log2P = log2M - L.log2Q;
  const int P = 1 << L.log2P, Q = 1 << L.log2Q;
  L.Pnz = (int)((N + Q - 1) / Q);
  L.nthr_B = std::max(32, Q / 16);
  L.smem_B = padded_size(Q) * cs;
  if (allow_fast && !dbl && P >= 8 && P <= 32) {
    // register column passes: 8 pairs x 32 columns per CTA, one thread per column
    L.fast = true;
    L.G = 8;
    L.NB = 32;
    L.ntiles = Q / L.NB;
    L.nthr_A = L.nthr_C = 256;
    L.smem_A = L.smem_C = 0;
    L.fused_reduce = (L.log2Q == 12);
  } else if (allow_fast && !dbl && P >= 64 && P <= 1024) {
    // two-stage register column passes (P = 32 P2), one pair per CTA, 256 threads; the
    // correction runs outside them
    L.big = true;
    L.split_corr = true;
    L.P2 = P / 32;
    L.G = 1;
    L.NB = 256 / L.P2;
    L.ntiles = Q / L.NB;
    L.nthr_A = L.nthr_C = 256;
    L.smem_A = L.smem_C = (size_t)big_smem_bytes(L.P2);
  } else {
    L.split_corr = allow_fast && !dbl;
    const int tile = 8192;
    const int ncols = std::max(1, tile / P);
    const int nb0 = std::min(32, ncols);
    L.G = std::min(ncols / nb0, 16);
    L.NB = ncols / L.G;
    L.ntiles = Q / L.NB;
    L.nthr_A = L.nthr_C = std::max(32, ncols * P / 16);
    const int nwarps = L.nthr_A / 32;
    L.smem_A = padded_size(P * ncols) * cs + (size_t)nwarps * 128 * rs;
    L.smem_C = padded_size(P * ncols) * cs;
  }
  int64_t ch = chunk_bytes_target() / (int64_t)(M * cs);
  ch = std::max<int64_t>(L.G, (ch / L.G) * L.G);
  L.chunk = ch;
  return L;
}

static size_t ws_need(const Layout &L, bool dbl, int rpad, bool forward) {
  const size_t cs = dbl ? 16 : 8, rs = dbl ? 8 : 4;
  const int64_t M = 1LL << L.log2M;
  if (L.small) return forward ? (size_t)L.chunk * M * cs : 0;
  size_t b = (size_t)L.chunk * M * cs;
  b += (size_t)L.chunk * L.ntiles * 2 * std::max(rpad, 1) * rs;
  b += (size_t)L.chunk * 2 * std::max(rpad, 1) * rs;
  return b + 1024;
}

// ---------------------------------------------------------------------------
// convolution driver
// ---------------------------------------------------------------------------

// bytes of one launch group's scratch (one lane)
static size_t slot_bytes(const Layout &L, bool dbl, int rpad, bool forward) { return ws_need(L, dbl, rpad, forward); }

// scratch of the separate correction for npairs pairs (partials per CORR_BLOCK rows or per
// tcgen05 slice, then a)
static size_t split_corr_bytes(int64_t N, int64_t npairs, int rpad) {
  const int64_t nK = std::max<int64_t>((N + CORR_BLOCK - 1) / CORR_BLOCK, tc_slices(N));
  return (size_t)npairs * (nK + 1) * 2 * std::max(rpad, 1) * sizeof(float) + 256;
}

static bool tc_disabled() {
  const char *s = getenv("FST_TC");
  return s && s[0] == '0';
}

// FST_PLAIN=1: the plain FP32 form the batched path is compared with -- generic four-step
// kernels with the rank-r correction on CUDA cores inside the column passes, launched
// directly (no CUDA graph, no tensor cores); read at every call
static bool plain_mode() {
  const char *s = getenv("FST_PLAIN");
  return s && s[0] == '1';
}

// the tcgen05 correction applies: FP32 device plan with K-major S_T^T tiles and signal rows
// a TMA tensor map can address (16-byte aligned base and row stride)
static bool tc_usable(const ConvArgs<float> &a) {
  if (!a.STt || tc_disabled() || plain_mode()) return false;
  const int64_t row_bytes = a.ld * (a.cplx ? 8 : 4);
  return ((uintptr_t)a.y % 16) == 0 && row_bytes % 16 == 0 && a.N < (1LL << 30) && a.batch < (1LL << 31);
}

// S_T^T y for every pair into sc.part, then a = scale o (sum of the partials) into sc.acoef
static fst_status corr_coefficients(Runner *R, ConvArgs<float> &sc, const float *scale) {
  const int64_t rows = sc.cplx ? 2 * sc.batch : sc.batch;
  const int combos = (int)((rows + 3) / 4) * (sc.rpad / 8);
  if (R->device() && sc.ST && rows <= 32 && sc.rpad <= 64 && combos <= 256 && (uintptr_t)sc.ST % 16 == 0 &&
      !plain_mode()) {
    // few signal rows: FP32 CUDA-core partials (the tensor-core tile would be mostly empty)
    sc.nkb = (int)((sc.N + CORR_BLOCK - 1) / CORR_BLOCK);
    TRY(R->corr_cc(sc));
  } else if (tc_usable(sc)) {
    sc.nkb = tc_slices(sc.N);
    TRY(R->corr_tc(sc));
  } else {
    sc.nkb = (int)((sc.N + CORR_BLOCK - 1) / CORR_BLOCK);
    TRY(R->corr_c(sc));
  }
  return R->corr_reduce(sc, scale);
}

template <typename T>
static fst_status run_conv(Runner *R, const Layout &L, ConvArgs<T> a, int64_t npairs, void *ws) {
  using C = c2<T>;
  a.log2M = L.log2M;
  a.log2P = L.log2P;
  a.log2Q = L.log2Q;
  a.Pnz = L.Pnz;
  a.NB = L.NB;
  a.G = L.G;
  if (a.mode == MODE_FORWARD && !L.small) a.Pnz = 1 << L.log2P;
  const int64_t M = 1LL << L.log2M;
  const int lanes = R->lanes();
  const size_t slot = slot_bytes(L, sizeof(T) == 8, a.rpad, a.mode == MODE_FORWARD);
  // separate correction (FP32 device): a = D o S_T^T y over every pair first (before any
  // output is written, so y == out works); on tcgen05 whenever the signal rows allow a
  // tensor map, else (P > 32) mma.sync kernels.  Then out += S_T a: in the fast column
  // pass C, or by a last kernel over the whole batch.
  const bool want = a.mode == MODE_FULL && a.r > 0 && sizeof(T) == 4 && R->device() && !L.small;
  const bool tc = want && tc_usable(*reinterpret_cast<const ConvArgs<float> *>(&a));
  const bool split = want && (L.split_corr || tc);
  ConvArgs<float> sc{};
  if (split) {
    sc = *reinterpret_cast<const ConvArgs<float> *>(&a);
    char *w = (char *)ws + (size_t)lanes * slot;
    const int64_t nK = std::max<int64_t>((a.N + CORR_BLOCK - 1) / CORR_BLOCK, tc_slices(a.N));
    sc.pair0 = 0;
    sc.npairs = npairs;
    sc.part = (float *)w;
    sc.acoef = (float *)(w + (size_t)npairs * nK * 2 * a.rpad * sizeof(float));
    // on the side lane: only the passes that write the output (pass C, or the last
    // S_T a pass) wait for the coefficients, so the correction overlaps the first passes
    R->use_side();
    TRY(corr_coefficients(R, sc, (const float *)a.D));
    R->side_done();
    a.mode = L.fast ? MODE_ZONLY : MODE_CONV;
  }
  bool waited[2] = {false, false};
  int64_t group = 0;
  for (int64_t p0 = 0; p0 < npairs; p0 += L.chunk, ++group) {
    const int lane = (int)(group % lanes);
    R->use_lane(lane);
    char *w = (char *)ws + (size_t)lane * slot;
    a.inter = (C *)w;
    if (!L.small) {
      const size_t inter_b = (size_t)L.chunk * M * sizeof(C);
      a.part = (T *)(w + inter_b);
      a.acoef = (T *)(w + inter_b + (size_t)L.chunk * L.ntiles * 2 * std::max(a.rpad, 1) * sizeof(T));
      if (a.mode == MODE_ZONLY) a.acoef = (T *)(sc.acoef + (size_t)p0 * 2 * a.rpad);
    }
    a.pair0 = p0;
    a.npairs = std::min<int64_t>(L.chunk, npairs - p0);
    if (L.small) {
      TRY(R->small(a, L));
    } else {
      TRY(R->passA(a, L));
      if (a.mode == MODE_FULL && a.r > 0 && !(L.fused_reduce && R->device())) TRY(R->reduce(a, L));
      TRY(R->passB(a, L));
      if (split && L.fast && !waited[lane]) {
        R->wait_side();
        waited[lane] = true;
      }
      if (a.mode != MODE_FORWARD) TRY(R->passC(a, L));
    }
  }
  R->use_lane(0);
  if (split && !L.fast) {
    // out += S_T a over the whole batch once both lanes have written B y
    R->lanes_join_first();
    R->wait_side();
    // CUDA-core pass with register-blocked sums (any batch, rpad <= 64), else mma.sync
    const bool za_ok = sc.ST && sc.rpad <= 64 && (!sc.cplx || (uintptr_t)sc.out % 8 == 0) &&
                       (uintptr_t)sc.ST % 16 == 0;
    if (za_ok) TRY(R->zadd(sc));
    else TRY(R->corr_z(sc));
  }
  return FST_OK;
}

template <typename T> static Tw<T> plan_tw(fst_plan_t p);
template <> Tw<float> plan_tw<float>(fst_plan_t p) { return Tw<float>{p->tw32h, p->tw32l}; }
template <> Tw<double> plan_tw<double>(fst_plan_t p) { return Tw<double>{p->tw64h, p->tw64l}; }

static bool graphs_enabled() {
  const char *s = getenv("FST_GRAPHS");
  return !(s && s[0] == '0');
}

static fst_status ensure_ws(fst_plan_t p, size_t bytes) {
  if (bytes <= p->ws_bytes) return FST_OK;
  // the cached graphs point at the old workspace (recorded ragged batches check ws_gen)
  for (auto &e : p->graphs) p->R->graph_destroy(e.exec);
  p->graphs.clear();
  ++p->ws_gen;
  if (p->ws) p->R->release(p->ws);
  p->ws = nullptr;
  p->ws_bytes = 0;
  TRY(p->R->alloc(&p->ws, bytes));
  p->ws_bytes = bytes;
  return FST_OK;
}

template <typename T>
static fst_status apply_t(fst_plan_t p, const T *y, T *out, int64_t batch, int64_t ld, bool cplx, bool full,
                          const T *spec, const T *ST, const T *D, const Layout &L0, void *ext_ws,
                          size_t ext_bytes) {
  ConvArgs<T> a{};
  a.y = y;
  a.out = out;
  a.ld = ld;
  a.batch = batch;
  a.cplx = cplx ? 1 : 0;
  a.N = p->N;
  a.spec = spec;
  a.ST = ST;
  if (sizeof(T) == 4) {
    a.ST_hl = (const c2<T> *)p->ST32_hl;
    a.STt = p->STt;
    a.tc_nB = p->tc_nB;
    a.tc_Npad = p->tc_Npad;
    a.twB = p->twB;
    a.tw8 = p->tw8;
  }
  a.r = full ? (int)p->r : 0;
  a.rpad = (int)p->rpad;
  a.D = D;
  a.tw = plan_tw<T>(p);
  a.mode = full ? MODE_FULL : MODE_CONV;
  const int64_t npairs = cplx ? batch : (batch + 1) / 2;
  const bool dbl = sizeof(T) == 8;
  const bool sep = (L0.split_corr || (p->STt && !L0.small && !dbl)) && full && p->r > 0;
  const size_t extra = sep ? split_corr_bytes(p->N, npairs, (int)p->rpad) : 0;
  if (!ext_ws) {
    Runner *R = p->R;
    // launch groups no larger than the call needs (small batches, ragged signals)
    Layout L1 = L0;
    if (!L1.small) L1.chunk = std::min<int64_t>(L0.chunk, (npairs + L0.G - 1) / L0.G * L0.G);
    const Layout &Lc = L1;
    if (plain_mode() && !dbl && R->device() && !L0.small) {
      Layout Lp = make_layout(p->N, p->log2M, false, (int)p->rpad, false);
      Lp.chunk = std::min<int64_t>(Lp.chunk, (npairs + Lp.G - 1) / Lp.G * Lp.G);
      TRY(ensure_ws(p, ws_need(Lp, false, (int)p->rpad, false)));
      return run_conv<T>(R, Lp, a, npairs, p->ws);
    }
    const size_t slot = ws_need(Lc, dbl, (int)p->rpad, false);
    const bool graphs = R->device() && graphs_enabled() && !profiling_enabled() && !tc_stall_pending() &&
                        !R->user_stream_capturing();
    if (!graphs) {
      TRY(ensure_ws(p, slot + extra));
      return run_conv<T>(R, Lc, a, npairs, p->ws);
    }
    // whole apply as one cached CUDA graph (two overlapping lanes of launch groups)
    for (auto &e : p->graphs)
      if (e.y == (const void *)y && e.out == (void *)out && e.batch == batch && e.ld == ld &&
          e.dtype == (int)(cplx ? 1 : 0) + (dbl ? 2 : 0) && e.full == full)
        return R->graph_launch(e.exec, e.nodes);
    TRY(ensure_ws(p, 2 * slot + 256 + extra));
    if (!R->graph_begin()) {
      return run_conv<T>(R, Lc, a, npairs, p->ws);
    }
    fst_status st = run_conv<T>(R, Lc, a, npairs, p->ws);
    const std::string first_err = st != FST_OK ? std::string(g_err) : std::string();
    void *exec = nullptr;
    long long nodes = 0;
    fst_status st2 = R->graph_end(&exec, &nodes);
    if (st != FST_OK) {
      if (exec) R->graph_destroy(exec);
      return fail(st, first_err);   // the failure inside the recording, not its consequence
    }
    TRY(st2);
    if (p->graphs.size() >= 8) {
      R->graph_destroy(p->graphs.front().exec);
      p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back({(const void *)y, (void *)out, batch, ld, (int)(cplx ? 1 : 0) + (dbl ? 2 : 0), full, exec,
                         nodes});
    return R->graph_launch(exec, nodes);
  }
  // caller-provided scratch: shrink the launch group until it fits
  Layout L = L0;
  if (!L.small) {
    int64_t ch = L.chunk;
    while (ch > L.G) {
      L.chunk = ch;
      if (ws_need(L, dbl, (int)p->rpad, false) + extra <= ext_bytes) break;
      ch = std::max<int64_t>(L.G, ((ch / 2) / L.G) * L.G);
    }
    L.chunk = ch;
    if (ws_need(L, dbl, (int)p->rpad, false) + extra > ext_bytes)
      return fail(FST_EINVAL, "signal too long for the fixed scratch buffer");
  }
  return run_conv<T>(p->R, L, a, npairs, ext_ws);
}

fst_status run_apply_ws(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype, bool full,
                        void *ws, size_t ws_bytes) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FST_EINVAL, "batch < 0");
  if (batch == 0) return FST_OK;
  if (!y || !out) return fail(FST_EINVAL, "NULL signal pointer");
  if (ld == 0) ld = p->N;
  if (ld < p->N) return fail(FST_EINVAL, "ld < N");
  TRY(p->R->device_status(false));
  switch (dtype) {
    case FST_F32:
      return apply_t<float>(p, (const float *)y, (float *)out, batch, ld, false, full, p->spec32, p->ST32, p->D32,
                            p->lay32, ws, ws_bytes);
    case FST_C64:
      return apply_t<float>(p, (const float *)y, (float *)out, batch, ld, true, full, p->spec32, p->ST32, p->D32,
                            p->lay32, ws, ws_bytes);
    case FST_F64:
      return apply_t<double>(p, (const double *)y, (double *)out, batch, ld, false, full, p->spec64, p->ST64,
                             p->D64, p->lay64, ws, ws_bytes);
    case FST_C128:
      return apply_t<double>(p, (const double *)y, (double *)out, batch, ld, true, full, p->spec64, p->ST64,
                             p->D64, p->lay64, ws, ws_bytes);
    default:
      return fail(FST_EINVAL, "unknown dtype");
  }
}

fst_status run_apply(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype, bool full) {
  return run_apply_ws(p, y, out, batch, ld, dtype, full, nullptr, 0);
}

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------

static double cospi_host(double x) {
  // cos(pi x) for x in [0, 1] with exact zero at 1/2 (the differences are exact)
  if (x <= 0.25) return cos(M_PI * x);
  if (x <= 0.75) return sin(M_PI * (0.5 - x));
  return -cos(M_PI * (1.0 - x));
}

struct Reduced {
  int n = 0;
  std::vector<double> d, e, e2;  // e[i] couples i-1 and i (e[0] = 0)
};

static Reduced reduced_tridiagonal(int64_t N, double W, int parity) {
  Reduced R;
  const double cw = cospi_host(2.0 * W);
  auto dfull = [&](int64_t i) {
    const double c = 0.5 * (double)(N - 1) - (double)i;
    return c * c * cw;
  };
  auto efull = [&](int64_t i) { return 0.5 * (double)i * (double)(N - i); };
  const int64_t m = N / 2;
  const bool odd = (N & 1) != 0;
  int64_t n;
  if (!odd) n = m;
  else n = (parity == 0) ? m + 1 : m;
  R.n = (int)n;
  R.d.resize(n);
  R.e.assign(n, 0.0);
  R.e2.assign(n, 0.0);
  for (int64_t i = 0; i < n; ++i) R.d[i] = dfull(i);
  for (int64_t i = 1; i < n; ++i) R.e[i] = efull(i);
  if (!odd && n > 0) R.d[n - 1] += (parity == 0 ? 1.0 : -1.0) * efull(m);
  if (odd && parity == 0 && n > 1) R.e[n - 1] = sqrt(2.0) * efull(m);
  for (int64_t i = 1; i < n; ++i) R.e2[i] = R.e[i] * R.e[i];
  return R;
}

static void build_twiddles(std::vector<double2> &hi, std::vector<double2> &lo) {
  hi.resize(TW_HI_SIZE);
  lo.resize(TW_LO_SIZE);
  // exp(-2 pi i k / 2^24); the angle fraction k / 2^24 is exact in double
  for (int a = 0; a < TW_HI_SIZE; ++a) {
    const double f = (double)((int64_t)a << TW_SPLIT) / (double)(1 << TW_LOG2);
    hi[a] = make_double2(cos(2.0 * M_PI * f), -sin(2.0 * M_PI * f));
  }
  for (int b = 0; b < TW_LO_SIZE; ++b) {
    const double f = (double)b / (double)(1 << TW_LOG2);
    lo[b] = make_double2(cos(2.0 * M_PI * f), -sin(2.0 * M_PI * f));
  }
}

static double asymptotic_transition(int64_t N, double eps) {
  const double n = (double)std::max<int64_t>(N, 2);
  return 2.0 / (M_PI * M_PI) * log(n) * log(1.0 / eps - 1.0);
}
static double cor1_bound(int64_t N, double eps) {
  return (8.0 / (M_PI * M_PI) * log(8.0 * (double)N) + 12.0) * log(15.0 / eps);
}

struct Scoped {
  Runner *R;
  std::vector<void *> ptrs;
  explicit Scoped(Runner *r) : R(r) {}
  ~Scoped() { for (void *q : ptrs) R->release(q); }
  template <typename P> fst_status alloc(P **p, size_t n) {
    void *q = nullptr;
    fst_status s = R->alloc(&q, std::max<size_t>(n, 1) * sizeof(P));
    if (s != FST_OK) return s;
    ptrs.push_back(q);
    *p = (P *)q;
    return FST_OK;
  }
};

static bool in_T(double lam, int64_t l, int64_t K, double eps, int op, double alpha) {
  if (op == FST_OP_TIKHONOV) return lam > alpha * (1.0 + alpha) * eps && lam < 1.0 - eps / 3.0;
  const double one = (l < K) ? 1.0 : 0.0;
  return fabs(one - lam) > eps;
}
static double D_of(double lam, int64_t l, int64_t K, int op, double alpha) {
  if (op == FST_OP_PROJECT) return (l < K) ? 1.0 - lam : -lam;                 // U1 U2^*, Corollary 2
  if (op == FST_OP_PINV) return (l < K) ? 1.0 / lam - lam : -lam;              // U3 U4^*, Corollary 3
  return lam / (lam * lam + alpha) - lam / (1.0 + alpha);                      // U5 U5^*, Corollary 4
}

// lambda_l = s_l^T (B s_l) for the nwin window vectors (rows of S), FP64 convolution
// with the unit-scaled spectrum
static fst_status window_eigenvalues(fst_plan_t p, double *S, int nwin, double *lam_host, const double *spec_unit) {
  Runner *R = p->R;
  const int64_t N = p->N;
  Scoped sc(R);
  double *BS, *lamd;
  TRY(sc.alloc(&BS, (size_t)nwin * N));
  TRY(sc.alloc(&lamd, nwin));
  {
    ConvArgs<double> a{};
    a.y = S;
    a.out = BS;
    a.ld = N;
    a.batch = nwin;
    a.cplx = 0;
    a.N = N;
    a.spec = spec_unit;
    a.r = 0;
    a.rpad = 0;
    a.tw = plan_tw<double>(p);
    a.mode = MODE_CONV;
    const Layout L = make_layout(N, p->log2M, true, 0);
    void *ws = nullptr;
    const size_t need = ws_need(L, true, 0, false);
    if (need) {
      char *w;
      TRY(sc.alloc(&w, need));
      ws = w;
    }
    TRY(run_conv<double>(R, L, a, (nwin + 1) / 2, ws));
  }
  TRY(R->dot(S, BS, N, nwin, lamd));
  TRY(R->d2h(lam_host, lamd, nwin * sizeof(double)));
  return FST_OK;
}

// Slepian vectors s^(l), lo <= l <= hi, as rows S[l - lo][0..N), and their
// eigenvalues lambda_l = s^T B s (FP64 FFT convolution with spec64 = DFT_M(c)/M).
struct PendingWin {
  fst_plan_t p;
  int64_t centre, Rw, lo, hi;
  double *S;
  bool done;
};

// The window vectors of a group of plans: both parities of every plan's window as one batch of
// independent targets (bisection, inverse iteration one thread per target, expansion).
static fst_status batched_window_vectors(std::vector<PendingWin *> &grp) {
  if (grp.empty()) return FST_OK;
  Runner *R0 = grp[0]->p->R;
  Scoped sc(R0);
  // concatenated reduced matrices and one descriptor per target
  std::vector<double> dcat, ecat, e2cat;
  std::vector<TargetDesc> td;
  for (PendingWin *pw : grp) {
    fst_plan_t p = pw->p;
    for (int parity = 0; parity < 2; ++parity) {
      Reduced red = reduced_tridiagonal(p->N, p->W, parity);
      if (red.n == 0) continue;
      double glo = 1e300, ghi = -1e300, tnorm = 0.0, emax2 = 0.0;
      for (int i = 0; i < red.n; ++i) {
        const double el = fabs(red.e[i]), er = (i + 1 < red.n) ? fabs(red.e[i + 1]) : 0.0;
        glo = std::min(glo, red.d[i] - el - er);
        ghi = std::max(ghi, red.d[i] + el + er);
        tnorm = std::max(tnorm, fabs(red.d[i]) + el + er);
        emax2 = std::max(emax2, red.e2[i]);
      }
      const double pivmin = 2.2250738585072014e-308 * std::max(1.0, emax2);
      const double widen = 2.220446049250313e-16 * tnorm * 4.0 + 4.0 * pivmin;
      const int64_t off = (int64_t)dcat.size();
      dcat.insert(dcat.end(), red.d.begin(), red.d.end());
      ecat.insert(ecat.end(), red.e.begin(), red.e.end());
      e2cat.insert(e2cat.end(), red.e2.begin(), red.e2.end());
      for (int64_t l = pw->lo; l <= pw->hi; ++l) {
        if ((l & 1) != parity) continue;
        TargetDesc q{};
        q.mat_off = off;
        q.x_off = 0;
        q.S = pw->S + (size_t)(l - pw->lo) * p->N;
        q.N = p->N;
        q.n = red.n;
        q.target = red.n - 1 - (int)(l >> 1);
        q.parity = parity;
        q.glo = glo - widen;
        q.ghi = ghi + widen;
        q.pivmin = pivmin;
        // pivot lift of the inverse iteration and absolute floor of the bisection's stopping
        // test; > 0 also for a zero matrix (N = 1)
        q.tol = 2.220446049250313e-16 * tnorm + pivmin;
        td.push_back(q);
      }
    }
  }
  const int nt = (int)td.size();
  double *dd, *de, *de2, *theta;
  int *flag;
  TargetDesc *dtd;
  TRY(sc.alloc(&dd, dcat.size()));
  TRY(sc.alloc(&de, ecat.size()));
  TRY(sc.alloc(&de2, e2cat.size()));
  TRY(sc.alloc(&theta, nt));
  TRY(sc.alloc(&flag, 1));
  TRY(sc.alloc(&dtd, nt));
  TRY(R0->h2d(dd, dcat.data(), dcat.size() * sizeof(double)));
  TRY(R0->h2d(de, ecat.data(), ecat.size() * sizeof(double)));
  TRY(R0->h2d(de2, e2cat.data(), e2cat.size() * sizeof(double)));
  TRY(R0->zero(flag, sizeof(int)));
  TRY(R0->h2d(dtd, td.data(), td.size() * sizeof(TargetDesc)));
  // few targets: multisection, one block each (fewer rounds; the GPU has room for the extra
  // Sturm counts); many: plain bisection, one thread each (less arithmetic in all)
  if (nt <= BISECT_MS_MAX_TARGETS) TRY(R0->bisect_ms_many(dtd, nt, dd, de2, theta, flag));
  else TRY(R0->bisect_many(dtd, nt, dd, de2, theta, flag));
  int hflag = 0;
  TRY(R0->d2h(&hflag, flag, sizeof(int)));
  if (hflag) return fail(FST_ENOCONVERGE, "bisection did not converge");
  // inverse iteration and expansion in groups bounded by the factor storage
  const int64_t budget = 192LL << 20;   // elements per factor array (41 bytes each in all)
  for (int t0 = 0; t0 < nt;) {
    int t1 = t0;
    int64_t tot = 0;
    while (t1 < nt && (tot + td[t1].n <= budget || t1 == t0)) {
      td[t1].x_off = tot;
      tot += td[t1].n;
      ++t1;
    }
    Scoped g(R0);
    double *x, *fd, *fdl, *fdu, *fdu2;
    uint8_t *piv;
    TargetDesc *gtd;
    TRY(g.alloc(&x, tot));
    TRY(g.alloc(&fd, tot));
    TRY(g.alloc(&fdl, tot));
    TRY(g.alloc(&fdu, tot));
    TRY(g.alloc(&fdu2, tot));
    TRY(g.alloc(&piv, tot));
    TRY(g.alloc(&gtd, t1 - t0));
    TRY(R0->h2d(gtd, td.data() + t0, (size_t)(t1 - t0) * sizeof(TargetDesc)));
    TRY(R0->invit_many(gtd, t1 - t0, dd, de, theta + t0, x, fd, fdl, fdu, fdu2, piv));
    TRY(R0->finalize_many(gtd, t1 - t0, x));
    TRY(R0->sync());
    t0 = t1;
  }
  return FST_OK;
}

static fst_status window_vectors(fst_plan_t p, int64_t lo, int64_t hi, double *S, double *lam_host,
                                 const double *spec_unit) {
  PendingWin pw{p, 0, 0, lo, hi, S, false};
  std::vector<PendingWin *> grp{&pw};
  TRY(batched_window_vectors(grp));
  return window_eigenvalues(p, S, (int)(hi - lo + 1), lam_host, spec_unit);
}

static fst_status plan_fill(fst_plan_t p) {
  Runner *R = p->R;
  const int64_t N = p->N, M = p->M;
  const double W = p->W;
  // errors return straight away: the caller destroys the plan once every scoped buffer here
  // has been released (they need the plan's runner)
  auto bail = [](fst_status s) { return s; };

  // twiddle tables (FP64, rounded copy for FP32)
  {
    std::vector<double2> hi, lo;
    build_twiddles(hi, lo);
    std::vector<float2> hi32(hi.size()), lo32(lo.size());
    for (size_t i = 0; i < hi.size(); ++i) hi32[i] = make_float2((float)hi[i].x, (float)hi[i].y);
    for (size_t i = 0; i < lo.size(); ++i) lo32[i] = make_float2((float)lo[i].x, (float)lo[i].y);
    fst_status s;
    if ((s = R->alloc((void **)&p->tw64h, hi.size() * sizeof(double2))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->tw64l, lo.size() * sizeof(double2))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->tw32h, hi.size() * sizeof(float2))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->tw32l, lo.size() * sizeof(float2))) != FST_OK) return bail(s);
    if ((s = R->h2d(p->tw64h, hi.data(), hi.size() * sizeof(double2))) != FST_OK) return bail(s);
    if ((s = R->h2d(p->tw64l, lo.data(), lo.size() * sizeof(double2))) != FST_OK) return bail(s);
    if ((s = R->h2d(p->tw32h, hi32.data(), hi32.size() * sizeof(float2))) != FST_OK) return bail(s);
    if ((s = R->h2d(p->tw32l, lo32.data(), lo32.size() * sizeof(float2))) != FST_OK) return bail(s);
    std::vector<float2> tb(TWB_WORDS);
    for (int t = 0; t < 16; ++t) {
      for (int k = 0; k < 16; ++k) {
        const double ang = -2.0 * M_PI * (double)(k * t) / 256.0;
        tb[t * 16 + k] = make_float2((float)cos(ang), (float)sin(ang));
      }
      for (int k = 0; k < 256; ++k) {
        const double ang = -2.0 * M_PI * (double)(k * t) / 4096.0;
        tb[256 + t * 256 + k] = make_float2((float)cos(ang), (float)sin(ang));
      }
    }
    for (int t = 0; t < 1024; ++t) {
      const double ang = -2.0 * M_PI * (double)t / 1024.0;
      tb[TWB_P_OFF + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
    if ((s = R->alloc((void **)&p->twB, tb.size() * sizeof(float2))) != FST_OK) return bail(s);
    if ((s = R->h2d(p->twB, tb.data(), tb.size() * sizeof(float2))) != FST_OK) return bail(s);
    if (R->device()) {
      // the 8192-point row FFT: W_8192^j (j < 4096), then [t][k] W_32^{kt}, W_512^{kt}, W_8192^{kt}
      std::vector<float2> t8(TW8_WORDS);
      auto w = [](double num, double den) {
        const double ang = -2.0 * M_PI * num / den;
        return make_float2((float)cos(ang), (float)sin(ang));
      };
      for (int j = 0; j < 4096; ++j) t8[TW8_R2 + j] = w(j, 8192.0);
      for (int t = 0; t < 16; ++t) {
        for (int k = 0; k < 2; ++k) t8[TW8_32 + t * 2 + k] = w(k * t, 32.0);
        for (int k = 0; k < 32; ++k) t8[TW8_512 + t * 32 + k] = w(k * t, 512.0);
        for (int k = 0; k < 512; ++k) t8[TW8_8192 + t * 512 + k] = w(k * t, 8192.0);
      }
      if ((s = R->alloc((void **)&p->tw8, t8.size() * sizeof(float2))) != FST_OK) return bail(s);
      if ((s = R->h2d(p->tw8, t8.data(), t8.size() * sizeof(float2))) != FST_OK) return bail(s);
    }
  }

  Scoped sc(R);
  sc.ptrs.clear();
  const Layout L64 = make_layout(N, p->log2M, true, 0);
  const Layout L32 = make_layout(N, p->log2M, false, 0);   // FP32 P, Q do not depend on the kernels

  // sinc spectrum: forward FFT (FP64) of the even embedding c of the first row of B
  double *cvec, *spec_unit;
  double2 *X;
  {
    fst_status s;
    if ((s = sc.alloc(&cvec, (size_t)M)) != FST_OK) return bail(s);
    if ((s = sc.alloc(&X, (size_t)M)) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&spec_unit, (size_t)M * sizeof(double))) != FST_OK) return bail(s);
    p->spec_unit = spec_unit;
    if ((s = R->alloc((void **)&p->spec64, (size_t)M * sizeof(double))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->spec32, (size_t)M * sizeof(float))) != FST_OK) return bail(s);
    if ((s = R->sinc_embed(cvec, N, M, W)) != FST_OK) return bail(s);
    ConvArgs<double> a{};
    a.y = cvec;
    a.out = nullptr;
    a.ld = M;
    a.batch = 1;
    a.cplx = 0;
    a.N = M;
    a.r = 0;
    a.tw = plan_tw<double>(p);
    a.mode = MODE_FORWARD;
    Layout Lf = L64;
    Lf.chunk = std::max<int64_t>(1, Lf.G);
    if (!Lf.small) Lf.Pnz = 1 << Lf.log2P;
    // forward output goes straight into X ([k1][k2] order for 3-pass, natural for small)
    if (Lf.small) {
      a.inter = X;
      a.pair0 = 0;
      a.npairs = 1;
      a.log2M = Lf.log2M;
      if ((s = R->small(a, Lf)) != FST_OK) return bail(s);
    } else {
      const size_t need = (size_t)Lf.chunk * M * sizeof(double2) + (size_t)Lf.chunk * Lf.ntiles * 2 * 8 +
                          (size_t)Lf.chunk * 2 * 8 + 1024;
      char *w;
      if ((s = sc.alloc(&w, need)) != FST_OK) return bail(s);
      if ((s = run_conv<double>(R, Lf, a, 1, w)) != FST_OK) return bail(s);
      if ((s = R->d2d(X, w, (size_t)M * sizeof(double2))) != FST_OK) return bail(s);
    }
    // unit-scaled spectrum (for the eigenvalues) in the FP64 layout, then the
    // operator's spectrum beta/M in both layouts
    float *dummy32;
    if ((s = sc.alloc(&dummy32, (size_t)M)) != FST_OK) return bail(s);
    if ((s = R->spec_store(X, L64, L32, M, 1.0 / (double)M, spec_unit, dummy32)) != FST_OK) return bail(s);
    if ((s = R->spec_store(X, L64, L32, M, p->beta / (double)M, p->spec64, p->spec32)) != FST_OK) return bail(s);
  }

  return FST_OK;
}

static fst_status plan_begin(Runner *R, fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op,
                             double alpha) {
  if (!out) { delete R; return fail(FST_EINVAL, "out is NULL"); }
  *out = nullptr;
  if (!(N >= 1 && N <= (1LL << 23))) { delete R; return fail(FST_EINVAL, "need 1 <= N <= 2^23"); }
  if (!(W > 0.0 && W < 0.5)) { delete R; return fail(FST_EINVAL, "need 0 < W < 1/2"); }
  if (!(eps > 0.0 && eps < 0.5)) { delete R; return fail(FST_EINVAL, "need 0 < eps < 1/2"); }
  if (op < 0 || op > 2) { delete R; return fail(FST_EINVAL, "unknown operator"); }
  if (op == FST_OP_TIKHONOV && !(alpha > 0.0)) { delete R; return fail(FST_EINVAL, "Tikhonov needs alpha > 0"); }
  const int64_t Kdef = (int64_t)floor(2.0 * (double)N * W + 0.5);
  if (K < 0) K = Kdef;
  if (K > N) { delete R; return fail(FST_EINVAL, "need 0 <= K <= N"); }

  fst_plan_t p = new fst_plan_s();
  p->R = R;
  p->N = N;
  p->W = W;
  p->K = K;
  p->eps = eps;
  p->op = op;
  p->alpha = (op == FST_OP_TIKHONOV) ? alpha : 0.0;
  p->beta = (op == FST_OP_TIKHONOV) ? 1.0 / (1.0 + alpha) : 1.0;
  int64_t M = 2;
  while (M < 2 * N) M *= 2;
  p->M = M;
  p->log2M = ilog2_exact(M);

  fst_status fs = plan_fill(p);
  if (fs != FST_OK) {
    destroy_plan(p);
    return fs;
  }
  *out = p;
  return FST_OK;
}

static fst_status plan_end(fst_plan_t p, double *S, const std::vector<double> &lamw, int64_t lo, int64_t hi) {
  Runner *R = p->R;
  const int64_t N = p->N, K = p->K;
  const double eps = p->eps;
  const int op = p->op;
  auto bail = [&](fst_status s) { return s; };
  Scoped sc(R);
  p->win_lo = lo;
  p->win_hi = hi;
  p->lam_window = lamw;

  std::vector<int> sel;
  for (int64_t l = lo; l <= hi; ++l) {
    const double lam = lamw[l - lo];
    if (in_T(lam, l, K, eps, op, p->alpha)) {
      sel.push_back((int)(l - lo));
      p->idx.push_back(l);
      p->lam.push_back(lam);
      p->D.push_back(D_of(lam, l, K, op, p->alpha));
    }
  }
  p->r = (int64_t)sel.size();
  p->rpad = std::max<int64_t>(8, (p->r + 7) / 8 * 8);
  {
    fst_status s;
    const size_t nst = (size_t)N * p->rpad;
    if ((s = R->alloc((void **)&p->ST64, nst * sizeof(double))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->ST32, nst * sizeof(float))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->D64, (size_t)p->rpad * sizeof(double))) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->D32, (size_t)p->rpad * sizeof(float))) != FST_OK) return bail(s);
    if ((s = R->zero(p->D64, (size_t)p->rpad * sizeof(double))) != FST_OK) return bail(s);
    if (p->r > 0) {
      int *dsel;
      if ((s = sc.alloc(&dsel, sel.size())) != FST_OK) return bail(s);
      if ((s = R->h2d(dsel, sel.data(), sel.size() * sizeof(int))) != FST_OK) return bail(s);
      if ((s = R->gather_ST(S, N, dsel, (int)p->r, (int)p->rpad, p->ST64, p->ST32)) != FST_OK) return bail(s);
      if ((s = R->h2d(p->D64, p->D.data(), p->D.size() * sizeof(double))) != FST_OK) return bail(s);
    } else {
      if ((s = R->zero(p->ST64, nst * sizeof(double))) != FST_OK) return bail(s);
      if ((s = R->zero(p->ST32, nst * sizeof(float))) != FST_OK) return bail(s);
    }
    if ((s = R->to_f32(p->D64, p->D32, p->rpad)) != FST_OK) return bail(s);
    if ((s = R->alloc((void **)&p->ST32_hl, nst * sizeof(float2))) != FST_OK) return bail(s);
    if ((s = R->split_tf32(p->ST32, p->ST32_hl, (int64_t)nst)) != FST_OK) return bail(s);
    if ((s = R->sync()) != FST_OK) return bail(s);
  }
  p->lay32 = make_layout(N, p->log2M, false, (int)p->rpad, R->device());
  p->lay64 = make_layout(N, p->log2M, true, (int)p->rpad, false);
  if (R->device() && !p->lay32.small && p->r > 0 && p->r <= 128) {
    // K-major FP32 S_T^T for the tcgen05 correction
    fst_status s;
    p->tc_nB = (int)((p->r + 31) / 32 * 32);
    p->tc_Npad = (N + 3) / 4 * 4;
    const size_t nt = (size_t)p->tc_nB * p->tc_Npad;
    if ((s = R->alloc((void **)&p->STt, nt * sizeof(float))) != FST_OK) return bail(s);
    if ((s = R->tc_prep(p->ST32, N, (int)p->rpad, (int)p->r, p->tc_nB, p->tc_Npad, p->STt)) != FST_OK)
      return bail(s);
    if ((s = R->sync()) != FST_OK) return bail(s);
  }
  if (p->lay32.small && p->lay32.smem_small > 227 * 1024)
    return bail(fail(FST_EUNSUPPORTED, "transition rank too large for the single-CTA path"));
  if (p->lay64.small && p->lay64.smem_small > 227 * 1024)
    return bail(fail(FST_EUNSUPPORTED, "transition rank too large for the single-CTA path"));
  if (p->spec_unit) {
    R->release(p->spec_unit);
    p->spec_unit = nullptr;
  }
  return FST_OK;
}

static void free_coef(fst_plan_t p);
// eigen stage of one plan: window search, vectors, eigenvalues, transition set
static fst_status plan_eigen(fst_plan_t p) {
  const int64_t N = p->N;
  const double W = p->W, eps = p->eps;
  const int op = p->op;
  Runner *R = p->R;
  const int64_t K = p->K;
  const int64_t Kdef = (int64_t)floor(2.0 * (double)N * W + 0.5);
  // errors return straight away: the caller destroys the plan after the scoped buffers here
  // are released
  auto bail = [](fst_status s) { return s; };
  const double *spec_unit = p->spec_unit;
  Scoped sc(R);
  // eigen-window around the centre, widened until both edges are outside T
  const int64_t centre = (op == FST_OP_TIKHONOV) ? Kdef : K;
  int64_t Rw = (int64_t)std::min(ceil(cor1_bound(N, eps)), ceil(0.6 * asymptotic_transition(N, eps)) + 6.0);
  Rw = std::max<int64_t>(Rw, 2);
  std::vector<double> lamw;
  double *S = nullptr;
  int64_t lo = 0, hi = 0;
  for (int attempt = 0;; ++attempt) {
    lo = std::max<int64_t>(0, centre - Rw);
    hi = std::min<int64_t>(N - 1, centre + Rw);
    const int nwin = (int)(hi - lo + 1);
    Scoped win(R);
    double *Sw;
    fst_status s;
    if ((s = win.alloc(&Sw, (size_t)nwin * N)) != FST_OK) return bail(s);
    lamw.assign(nwin, 0.0);
    if ((s = window_vectors(p, lo, hi, Sw, lamw.data(), spec_unit)) != FST_OK) return bail(s);
    const bool lo_ok = (lo == 0) || !in_T(lamw[0], lo, K, eps, op, p->alpha);
    const bool hi_ok = (hi == N - 1) || !in_T(lamw[nwin - 1], hi, K, eps, op, p->alpha);
    if (lo_ok && hi_ok) {
      // keep the window's vectors: move ownership of Sw to sc
      win.ptrs.erase(std::find(win.ptrs.begin(), win.ptrs.end(), (void *)Sw));
      sc.ptrs.push_back(Sw);
      S = Sw;
      break;
    }
    if (attempt > 12) return bail(fail(FST_ENOCONVERGE, "eigen-window search did not terminate"));
    Rw *= 2;
  }
  return plan_end(p, S, lamw, lo, hi);
}

fst_status build_plan(Runner *R, fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op,
                      double alpha) {
  if (!out) { delete R; return fail(FST_EINVAL, "out is NULL"); }
  *out = nullptr;
  fst_plan_t p = nullptr;
  TRY(plan_begin(R, &p, N, W, K, eps, op, alpha));
  const fst_status st = plan_eigen(p);
  if (st != FST_OK) {
    destroy_plan(p);
    return st;
  }
  *out = p;
  return FST_OK;
}

void destroy_plan(fst_plan_t p) {
  if (!p) return;
  forget_ragged(p);
  if (p->R) free_coef(p);
  Runner *R = p->R;
  if (R) {
    R->sync();
    for (auto &e : p->graphs) R->graph_destroy(e.exec);
    p->graphs.clear();
    void *bufs[] = {p->spec32, p->ST32, p->D32, p->spec64, p->ST64, p->D64, p->ST32_hl, p->STt, p->spec_unit,
                    p->tw32h, p->tw32l, p->tw64h, p->tw64l, p->twB, p->tw8, p->ws};
    for (void *b : bufs)
      if (b) R->release(b);
    delete R;
  }
  delete p;
}

}  // namespace fst

using namespace fst;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *fst_last_error(void) { return g_err.c_str(); }
const char *fst_version(void) { return "fst-gb300 0.1"; }

fst_status fst_plan_op(fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op, double alpha,
                       void *stream) {
  Runner *R = make_dev_runner();
  if (!R) return fail(FST_ECUDA, "no CUDA device");
  R->set_stream(stream);
  return build_plan(R, out, N, W, K, eps, op, alpha);
}

fst_status fst_plan(fst_plan_t *out, int64_t N, double W, int64_t K, double eps, void *stream) {
  return fst_plan_op(out, N, W, K, eps, FST_OP_PROJECT, 0.0, stream);
}

fst_status fst_plan_info(fst_plan_t p, int64_t *K, int64_t *r, int64_t *M, int64_t *wlo, int64_t *whi) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (K) *K = p->K;
  if (r) *r = p->r;
  if (M) *M = p->M;
  if (wlo) *wlo = p->win_lo;
  if (whi) *whi = p->win_hi;
  return FST_OK;
}

fst_status fst_plan_export(fst_plan_t p, int64_t *idx, double *lam, double *D, double *S_T) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  const int64_t r = p->r;
  if (idx) memcpy(idx, p->idx.data(), r * sizeof(int64_t));
  if (lam) memcpy(lam, p->lam.data(), r * sizeof(double));
  if (D) memcpy(D, p->D.data(), r * sizeof(double));
  if (S_T && r > 0) {
    std::vector<double> rows((size_t)p->N * p->rpad);
    fst_status s = p->R->d2h(rows.data(), p->ST64, rows.size() * sizeof(double));
    if (s != FST_OK) return s;
    for (int64_t j = 0; j < r; ++j)
      for (int64_t n = 0; n < p->N; ++n) S_T[j * p->N + n] = rows[n * p->rpad + j];
  }
  return FST_OK;
}

fst_status fst_project(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype,
                       void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  p->R->set_stream(stream);
  return run_apply(p, y, out, batch, ld, dtype, true);
}

fst_status fst_apply_prolate(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype,
                             void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  p->R->set_stream(stream);
  return run_apply(p, y, out, batch, ld, dtype, false);
}

fst_status fst_destroy(fst_plan_t p) {
  destroy_plan(p);
  return FST_OK;
}

fst_status fst_sync(fst_plan_t p, void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  p->R->set_stream(stream);
  return p->R->device_status(true);
}

fst_status fst_reduced_tridiagonal(int64_t N, double W, int parity, int64_t *n, double *d, double *e) {
  if (N < 1 || !(W > 0.0 && W < 0.5) || (parity != 0 && parity != 1) || !n)
    return fail(FST_EINVAL, "bad arguments");
  Reduced R = reduced_tridiagonal(N, W, parity);
  *n = R.n;
  if (d) memcpy(d, R.d.data(), R.n * sizeof(double));
  if (e && R.n > 1) memcpy(e, R.e.data() + 1, (R.n - 1) * sizeof(double));
  return FST_OK;
}

// ---- host emulation (tests) ----
fst_status fst_emu_plan_op(fst_plan_t *out, int64_t N, double W, int64_t K, double eps, int op, double alpha) {
  return build_plan(make_emu_runner(), out, N, W, K, eps, op, alpha);
}

int fst_plan_is_emulated(fst_plan_t p) { return (p && p->R && !p->R->device()) ? 1 : 0; }

}  // extern "C"

// ===========================================================================
// Fast coefficient vector T2^* y (Theorem 1 construction, Section 2; Section 1.3)
// ===========================================================================
namespace fst {

// Complete elliptic integral K and Jacobi dn for parameter m = 1 - m1, by the
// arithmetic-geometric mean (Abramowitz & Stegun 17.6 and 16.4).
static double agm_K(double m1) {
  double a = 1.0, b = sqrt(m1);
  for (int i = 0; i < 64 && fabs(a - b) > 1e-16 * a; ++i) {
    const double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return M_PI / (2.0 * a);
}
static double jacobi_dn(double u, double m1) {
  double a[80], c[80];
  a[0] = 1.0;
  double b = sqrt(m1);
  c[0] = sqrt(1.0 - m1);
  int n = 0;
  while (n < 78 && fabs(c[n]) > 1e-17) {
    a[n + 1] = 0.5 * (a[n] + b);
    c[n + 1] = 0.5 * (a[n] - b);
    b = sqrt(a[n] * b);
    ++n;
  }
  double phi = ldexp(1.0, n) * a[n] * u;
  double phi_next = phi;
  for (int i = n; i >= 1; --i) {
    phi_next = phi;
    phi = 0.5 * (phi + asin(c[i] / a[i] * sin(phi)));
  }
  // phi = phi_0, phi_next = phi_1
  return cos(phi) / cos(phi_next - phi);
}

// optimal CF-ADI shifts for A = diag(n + 1/2): p_k = b dn((2k-1)/(2r) K, m), m = 1 - (a/b)^2
static std::vector<double> adi_shifts(int64_t N, int r) {
  const double a = 0.5, b = (double)N - 0.5;
  const double m1 = (a / b) * (a / b);
  const double K = agm_K(m1);
  std::vector<double> p(r);
  for (int k = 1; k <= r; ++k) p[k - 1] = (N == 1) ? 0.5 : b * jacobi_dn((2.0 * k - 1.0) / (2.0 * r) * K, m1);
  return p;
}
static double adi_error_bound(int64_t N, const std::vector<double> &p) {
  double mx = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    const double x = (double)n + 0.5;
    double phi = 1.0;
    for (double pj : p) phi *= (x - pj) / (x + pj);
    mx = std::max(mx, phi * phi);
  }
  return mx;
}

static fst_status build_coef(fst_plan_t p) {
  if (p->coef) return FST_OK;
  Runner *R = p->R;
  const int64_t N = p->N;
  const double eps = p->eps, W = p->W;
  CoefPlan *cp = new CoefPlan();
  cp->odd = 2 * (int64_t)floor((double)N * W) + 1;
  cp->h = (cp->odd - 1) / 2;
  cp->Wp = (double)cp->odd / (2.0 * (double)N);
  const double dH = 4.0 * M_PI * eps / 15.0, dA = 7.0 * eps / 30.0, dB = 7.0 * eps / 30.0;
  int rH = (int)ceil(log(8.0 * (double)N - 4.0) * log(4.0 * M_PI / dH) / (M_PI * M_PI));
  rH = std::max(rH, 1);
  for (;;) {
    cp->p = adi_shifts(N, rH);
    if (adi_error_bound(N, cp->p) <= dH / M_PI || rH > 400) break;
    ++rH;
  }
  cp->rH = rH;
  cp->rA = std::max(1, (int)ceil(log(2.0 / (3.0 * M_PI * dA)) / (2.0 * log(2.0))));
  cp->rB = std::max(1, (int)ceil(log(3.0 / (2.0 * dB)) / (2.0 * log(6.0 / M_PI))));
  cp->DA = 2 * cp->rA;
  cp->DB = 2 * cp->rB - 1;
  cp->nraw = 4 * cp->rH + 2 * cp->DA + 2 * cp->DB;
  cp->r1 = 4 * cp->rH + 2 * cp->DA + 2 * cp->DB;
  // ADI recurrence factors
  std::vector<double> zfirst(rH), zshift(rH);
  for (int k = 0; k < rH; ++k) {
    zshift[k] = cp->p[k];
    zfirst[k] = (k == 0) ? sqrt(2.0 * cp->p[0]) : sqrt(cp->p[k] / cp->p[k - 1]);
  }
  // Taylor coefficients: alpha_k = 1 - (1 - 2^{1-2k}) zeta(2k) = sum_{n>=2} (-1)^n n^{-2k}
  // (k = 1: 1 - pi^2/12), beta_k = (-1)^k t^{2k+1} / (2k+1)!, t = pi (W - W') N
  std::vector<double> alpha(cp->rA + 1, 0.0), beta(cp->rB, 0.0);
  for (int k = 1; k <= cp->rA; ++k) {
    if (k == 1) { alpha[k] = 1.0 - M_PI * M_PI / 12.0; continue; }
    double s = 0.0;
    for (int n = 20000; n >= 2; --n) s += ((n & 1) ? -1.0 : 1.0) * pow((double)n, -2.0 * k);
    alpha[k] = s;
  }
  const double t = M_PI * (W - cp->Wp) * (double)N;
  {
    double term = t;   // t^{2k+1} / (2k+1)! for k = 0
    for (int k = 0; k < cp->rB; ++k) {
      beta[k] = ((k & 1) ? -1.0 : 1.0) * term;
      term *= t * t / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
  }
  // C_A, C_B on centred monomials: (u_m - u_n)^d = sum_i C(d,i) u_m^i (-u_n)^{d-i}
  const int Dmax = std::max(cp->DA, cp->DB) + 1;
  std::vector<std::vector<double>> binom(Dmax, std::vector<double>(Dmax, 0.0));
  for (int d = 0; d < Dmax; ++d) {
    binom[d][0] = binom[d][d] = 1.0;
    for (int i = 1; i < d; ++i) binom[d][i] = binom[d - 1][i - 1] + binom[d - 1][i];
  }
  const double sc = 2.0 / ((double)N * M_PI);
  std::vector<double> CA((size_t)cp->DA * cp->DA, 0.0), CB((size_t)cp->DB * cp->DB, 0.0);
  for (int k = 1; k <= cp->rA; ++k) {
    const int d = 2 * k - 1;
    for (int i = 0; i <= d; ++i) CA[(size_t)i * cp->DA + (d - i)] += sc * alpha[k] * binom[d][i] * (((d - i) & 1) ? -1.0 : 1.0);
  }
  for (int k = 0; k < cp->rB; ++k) {
    const int d = 2 * k;
    for (int i = 0; i <= d; ++i) CB[(size_t)i * cp->DB + (d - i)] += sc * beta[k] * binom[d][i] * (((d - i) & 1) ? -1.0 : 1.0);
  }
  std::vector<double> sqrtD(std::max<int64_t>(p->r, 1), 0.0);
  for (int64_t j = 0; j < p->r; ++j) sqrtD[j] = sqrt(fabs(p->D[j]));
  // phase ramps exp(-j 2 pi W' n) (exact reduction: W' n = odd n / 2N) and
  // exp(-j pi (W + W') n) (product split exactly with fma before reducing mod 2)
  std::vector<double2> phA(N), phB(N);
  const double sW = W + cp->Wp;
  for (int64_t n = 0; n < N; ++n) {
    const int64_t m = (int64_t)(((__int128)cp->odd * n) % (2 * N));   // W' n = m / (2N) cycles
    const double ang = M_PI * ((double)m / (double)N);
    phA[n] = make_double2(cos(ang), -sin(ang));
    const double hi = sW * (double)n, lo = fma(sW, (double)n, -hi);
    double r = fmod(hi, 2.0) + lo;
    phB[n] = make_double2(cos(M_PI * r), -sin(M_PI * r));
  }
  auto up64 = [&](double **dst, const std::vector<double> &v) -> fst_status {
    TRY(R->alloc((void **)dst, v.size() * sizeof(double)));
    return R->h2d(*dst, v.data(), v.size() * sizeof(double));
  };
  auto up32 = [&](float **dst, const std::vector<double> &v) -> fst_status {
    std::vector<float> f(v.begin(), v.end());
    TRY(R->alloc((void **)dst, f.size() * sizeof(float)));
    return R->h2d(*dst, f.data(), f.size() * sizeof(float));
  };
  fst_status st = FST_OK;
  if ((st = up64(&cp->zfirst64, zfirst)) || (st = up64(&cp->zshift64, zshift)) || (st = up64(&cp->CA64, CA)) ||
      (st = up64(&cp->CB64, CB)) || (st = up64(&cp->sqrtD64, sqrtD)) || (st = up32(&cp->zfirst32, zfirst)) ||
      (st = up32(&cp->zshift32, zshift)) || (st = up32(&cp->CA32, CA)) || (st = up32(&cp->CB32, CB)) ||
      (st = up32(&cp->sqrtD32, sqrtD))) {
    p->coef = cp;
    return st;
  }
  {
    std::vector<float2> a32(N), b32(N);
    for (int64_t n = 0; n < N; ++n) {
      a32[n] = make_float2((float)phA[n].x, (float)phA[n].y);
      b32[n] = make_float2((float)phB[n].x, (float)phB[n].y);
    }
    p->coef = cp;
    TRY(R->alloc((void **)&cp->phA64, N * sizeof(double2)));
    TRY(R->alloc((void **)&cp->phB64, N * sizeof(double2)));
    TRY(R->alloc((void **)&cp->phA32, N * sizeof(float2)));
    TRY(R->alloc((void **)&cp->phB32, N * sizeof(float2)));
    TRY(R->h2d(cp->phA64, phA.data(), N * sizeof(double2)));
    TRY(R->h2d(cp->phB64, phB.data(), N * sizeof(double2)));
    TRY(R->h2d(cp->phA32, a32.data(), N * sizeof(float2)));
    TRY(R->h2d(cp->phB32, b32.data(), N * sizeof(float2)));
  }
  return FST_OK;
}

static void free_coef(fst_plan_t p) {
  CoefPlan *cp = p->coef;
  if (!cp) return;
  void *bufs[] = {cp->zfirst32, cp->zshift32, cp->CA32, cp->CB32, cp->sqrtD32, cp->zfirst64, cp->zshift64,
                  cp->CA64, cp->CB64, cp->sqrtD64, cp->phA32, cp->phB32, cp->phA64, cp->phB64};
  for (void *b : bufs)
    if (b) p->R->release(b);
  delete cp;
  p->coef = nullptr;
}

template <typename T> struct CoefPtrs;
template <> struct CoefPtrs<float> {
  static void fill(const CoefPlan *c, CoefArgs<float> &a, const float *&CA, const float *&CB, const float *&sq) {
    a.zfirst = c->zfirst32; a.zshift = c->zshift32; a.phA = c->phA32; a.phB = c->phB32;
    CA = c->CA32; CB = c->CB32; sq = c->sqrtD32;
  }
};
template <> struct CoefPtrs<double> {
  static void fill(const CoefPlan *c, CoefArgs<double> &a, const double *&CA, const double *&CB, const double *&sq) {
    a.zfirst = c->zfirst64; a.zshift = c->zshift64; a.phA = c->phA64; a.phB = c->phB64;
    CA = c->CA64; CB = c->CB64; sq = c->sqrtD64;
  }
};

template <typename T>
static fst_status coeffs_t(fst_plan_t p, const T *y, c2<T> *out, int64_t batch, int64_t ld, bool cplx) {
  using C = c2<T>;
  Runner *R = p->R;
  TRY(build_coef(p));
  const CoefPlan *cp = p->coef;
  const int64_t N = p->N;
  const int64_t nF = cp->odd;
  const int64_t Kp = nF + cp->r1 + p->r;
  const bool dbl = sizeof(T) == 8;
  int log2N = 0;
  while ((1LL << log2N) < N) ++log2N;
  // ---- F^* y: forward DFT of length N, chunk by chunk of pairs, then the bins
  Layout Lf = make_layout(N, log2N, dbl, 0, false);
  if (!Lf.small) Lf.Pnz = 1 << Lf.log2P;
  const int64_t npairs = cplx ? batch : (batch + 1) / 2;
  const size_t ws_f = ws_need(Lf, dbl, 0, true) + 4096;
  const int nchunks = (int)((N + COEF_CHUNK - 1) / COEF_CHUNK);
  const size_t part_b = (size_t)batch * nchunks * cp->nraw * 2 * sizeof(T);
  const size_t partU_b = std::max((size_t)batch * nchunks * std::max<int64_t>(p->r, 1) * 2 * sizeof(T),
                                  split_corr_bytes(N, npairs, (int)p->rpad));
  const size_t tot_b = (size_t)batch * cp->nraw * 2 * sizeof(T);
  const size_t totU_b = (size_t)batch * std::max<int64_t>(p->r, 1) * 2 * sizeof(T);
  TRY(ensure_ws(p, std::max(ws_f, part_b + partU_b + tot_b + totU_b + 4096)));
  {
    ConvArgs<T> a{};
    a.y = y;
    a.ld = ld;
    a.batch = batch;
    a.cplx = cplx ? 1 : 0;
    a.N = N;
    a.r = 0;
    a.rpad = 0;
    a.tw = plan_tw<T>(p);
    a.mode = MODE_FORWARD;
    a.log2M = Lf.log2M;
    a.log2P = Lf.log2P;
    a.log2Q = Lf.log2Q;
    a.Pnz = Lf.Pnz;
    a.NB = Lf.NB;
    a.G = Lf.G;
    char *w = (char *)p->ws;
    a.inter = (C *)w;
    if (!Lf.small) {
      a.part = (T *)(w + (size_t)Lf.chunk * N * sizeof(C));
      a.acoef = a.part;
    }
    for (int64_t p0 = 0; p0 < npairs; p0 += Lf.chunk) {
      a.pair0 = p0;
      a.npairs = std::min<int64_t>(Lf.chunk, npairs - p0);
      if (Lf.small) {
        TRY(R->small(a, Lf));
      } else {
        TRY(R->passA(a, Lf));
        TRY(R->passB(a, Lf));
      }
      const int64_t sig0 = cplx ? p0 : 2 * p0;
      const int64_t nsig = cplx ? a.npairs : std::min<int64_t>(2 * a.npairs, batch - sig0);
      TRY(R->coef_gather(a.inter, Lf, N, a.cplx, sig0, nsig, cp->h, out, Kp));
    }
  }
  // ---- L2^* y and U2^* y
  CoefArgs<T> c{};
  c.y = y;
  c.ld = ld;
  c.batch = batch;
  c.cplx = cplx ? 1 : 0;
  c.N = N;
  c.rH = cp->rH;
  c.DA = cp->DA;
  c.DB = cp->DB;
  c.nraw = cp->nraw;
  c.nchunks = nchunks;
  char *w = (char *)p->ws;
  c.part = (T *)w;
  c.partU = (T *)(w + part_b);
  T *tot = (T *)(w + part_b + partU_b);
  T *totU = (T *)(w + part_b + partU_b + tot_b);
  c.ST = (const T *)(dbl ? (const void *)p->ST64 : (const void *)p->ST32);
  c.r = (int)p->r;
  c.rpad = (int)p->rpad;
  const T *CA, *CB, *sq;
  CoefPtrs<T>::fill(cp, c, CA, CB, sq);
  TRY(R->coef_lowrank(c));
  const bool mma_u = !dbl && R->device() && p->r > 0;
  if (mma_u) {
    // U2^* y on the tensor cores: S_T^T y per pair, scaled by sqrt|D| in the reduce
    ConvArgs<float> ca{};
    ca.y = (const float *)y;
    ca.ld = ld;
    ca.batch = batch;
    ca.cplx = cplx ? 1 : 0;
    ca.N = N;
    ca.r = (int)p->r;
    ca.rpad = (int)p->rpad;
    ca.ST = p->ST32;
    ca.ST_hl = p->ST32_hl;
    ca.pair0 = 0;
    ca.npairs = npairs;
    ca.STt = p->STt;
    ca.tc_nB = p->tc_nB;
    ca.tc_Npad = p->tc_Npad;
    const int64_t nK = std::max<int64_t>((N + CORR_BLOCK - 1) / CORR_BLOCK, tc_slices(N));
    ca.part = (float *)c.partU;
    ca.acoef = (float *)c.partU + (size_t)npairs * nK * 2 * p->rpad;
    TRY(corr_coefficients(R, ca, (const float *)sq));
    c.upairs = 1;
    c.acoefU = (const T *)ca.acoef;
  } else if (p->r > 0) {
    TRY(R->coef_st(c));
  }
  TRY(R->coef_reduce(c.part, nchunks, cp->nraw, batch, tot));
  if (p->r > 0 && !mma_u) TRY(R->coef_reduce(c.partU, nchunks, (int)p->r, batch, totU));
  TRY(R->coef_mix(c, tot, totU, CA, CB, sq, out, Kp, nF));
  return FST_OK;
}

// T1 c for `batch` coefficient vectors (Section 1.3, the fast factorization S_K S_K^* ~ T1 T2^*):
// per launch group of signals, the F bins are scattered and transformed by the forward DFT,
// then one pass over the samples adds the L1 and U1 parts
template <typename T> struct ExpPtrs;
template <> struct ExpPtrs<float> {
  static void fill(fst_plan_t p, ExpArgs<float> &e) {
    const CoefPlan *c = p->coef;
    e.zfirst = c->zfirst32; e.zshift = c->zshift32; e.phA = c->phA32; e.phB = c->phB32;
    e.ST = p->ST32; e.D = p->D32; e.sqrtD = c->sqrtD32;
  }
};
template <> struct ExpPtrs<double> {
  static void fill(fst_plan_t p, ExpArgs<double> &e) {
    const CoefPlan *c = p->coef;
    e.zfirst = c->zfirst64; e.zshift = c->zshift64; e.phA = c->phA64; e.phB = c->phB64;
    e.ST = p->ST64; e.D = p->D64; e.sqrtD = c->sqrtD64;
  }
};

template <typename T>
static fst_status expand_t(fst_plan_t p, const c2<T> *coef, c2<T> *out, int64_t batch) {
  using C = c2<T>;
  Runner *R = p->R;
  TRY(build_coef(p));
  const CoefPlan *cp = p->coef;
  const int64_t N = p->N;
  const bool dbl = sizeof(T) == 8;
  int log2N = 0;
  while ((1LL << log2N) < N) ++log2N;
  Layout Lf = make_layout(N, log2N, dbl, 0, false);
  if (!Lf.small) Lf.Pnz = 1 << Lf.log2P;
  // scratch: the scattered rows of one launch group, then the forward transform's own
  const size_t xs_b = ((size_t)Lf.chunk * N * sizeof(C) + 255) / 256 * 256;
  TRY(ensure_ws(p, xs_b + ws_need(Lf, dbl, 0, true) + 4096));
  C *Xs = (C *)p->ws;
  char *wf = (char *)p->ws + xs_b;
  ExpArgs<T> e{};
  e.coef = coef;
  e.Kp = cp->odd + cp->r1 + p->r;
  e.h = cp->h;
  e.N = N;
  e.rH = cp->rH;
  e.DA = cp->DA;
  e.DB = cp->DB;
  e.r = (int)p->r;
  e.rpad = (int)p->rpad;
  ExpPtrs<T>::fill(p, e);
  e.Lf = Lf;
  e.out = out;
  ConvArgs<T> a{};
  a.y = (const T *)Xs;
  a.ld = N;
  a.cplx = 1;
  a.N = N;
  a.tw = plan_tw<T>(p);
  a.mode = MODE_FORWARD;
  a.log2M = Lf.log2M;
  a.log2P = Lf.log2P;
  a.log2Q = Lf.log2Q;
  a.Pnz = Lf.Pnz;
  a.NB = Lf.NB;
  a.G = Lf.G;
  a.inter = (C *)wf;
  if (!Lf.small) {
    a.part = (T *)(wf + (size_t)Lf.chunk * N * sizeof(C));
    a.acoef = a.part;
  }
  for (int64_t s0 = 0; s0 < batch; s0 += Lf.chunk) {
    const int64_t nsig = std::min<int64_t>(Lf.chunk, batch - s0);
    e.sig0 = s0;
    TRY(R->exp_scatter(e, nsig, Xs));
    a.batch = nsig;
    a.pair0 = 0;
    a.npairs = nsig;
    if (Lf.small) {
      TRY(R->small(a, Lf));
    } else {
      TRY(R->passA(a, Lf));
      TRY(R->passB(a, Lf));
    }
    e.X = (const C *)a.inter;
    TRY(R->expand(e, nsig));
  }
  return FST_OK;
}

static fst_status run_coeffs(fst_plan_t p, const void *y, void *out, int64_t batch, int64_t ld, int dtype) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FST_EINVAL, "batch < 0");
  if (batch == 0) return FST_OK;
  if (!y || !out) return fail(FST_EINVAL, "NULL pointer");
  if (ld == 0) ld = p->N;
  if (ld < p->N) return fail(FST_EINVAL, "ld < N");
  if (p->op != FST_OP_PROJECT) return fail(FST_EINVAL, "coefficients need a projection plan");
  if ((p->N & (p->N - 1)) != 0) return fail(FST_EUNSUPPORTED, "coefficients need N a power of two");
  TRY(p->R->device_status(false));
  switch (dtype) {
    case FST_F32: return coeffs_t<float>(p, (const float *)y, (float2 *)out, batch, ld, false);
    case FST_C64: return coeffs_t<float>(p, (const float *)y, (float2 *)out, batch, ld, true);
    case FST_F64: return coeffs_t<double>(p, (const double *)y, (double2 *)out, batch, ld, false);
    case FST_C128: return coeffs_t<double>(p, (const double *)y, (double2 *)out, batch, ld, true);
    default: return fail(FST_EINVAL, "unknown dtype");
  }
}

}  // namespace fst

extern "C" {

fst_status fst_coeffs(fst_plan_t p, const void *y, void *coeffs, int64_t batch, int64_t ld, int dtype,
                      void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  p->R->set_stream(stream);
  return run_coeffs(p, y, coeffs, batch, ld, dtype);
}

fst_status fst_expand(fst_plan_t p, const void *coeffs, void *out, int64_t batch, int dtype, void *stream) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if (batch < 0) return fail(FST_EINVAL, "batch < 0");
  if (batch == 0) return FST_OK;
  if (!coeffs || !out) return fail(FST_EINVAL, "NULL pointer");
  if (p->op != FST_OP_PROJECT) return fail(FST_EINVAL, "expansion needs a projection plan");
  if ((p->N & (p->N - 1)) != 0) return fail(FST_EUNSUPPORTED, "expansion needs N a power of two");
  p->R->set_stream(stream);
  switch (dtype) {
    case FST_C64: return fst::expand_t<float>(p, (const float2 *)coeffs, (float2 *)out, batch);
    case FST_C128: return fst::expand_t<double>(p, (const double2 *)coeffs, (double2 *)out, batch);
    default: return fail(FST_EINVAL, "coefficients are complex: dtype FST_C64 or FST_C128");
  }
}

fst_status fst_coeffs_info(fst_plan_t p, int64_t *Kprime, int64_t *nF, int64_t *r1, int64_t *rH, int64_t *rA,
                           int64_t *rB) {
  if (!p) return fail(FST_EINVAL, "plan is NULL");
  if ((p->N & (p->N - 1)) != 0) return fail(FST_EUNSUPPORTED, "coefficients need N a power of two");
  fst_status s = build_coef(p);
  if (s != FST_OK) return s;
  const CoefPlan *cp = p->coef;
  if (Kprime) *Kprime = cp->odd + cp->r1 + p->r;
  if (nF) *nF = cp->odd;
  if (r1) *r1 = cp->r1;
  if (rH) *rH = cp->rH;
  if (rA) *rA = cp->rA;
  if (rB) *rB = cp->rB;
  return FST_OK;
}

fst_status fst_adi_shifts(int64_t N, int r, double *out) {
  if (N < 1 || r < 1 || !out) return fail(FST_EINVAL, "bad arguments");
  std::vector<double> p = fst::adi_shifts(N, r);
  memcpy(out, p.data(), r * sizeof(double));
  return FST_OK;
}

}  // extern "C"

// ===========================================================================
// Many plans at once (ragged batches): the eigen stage of every plan's window
// runs as one batch of independent targets (bisection and inverse iteration one
// thread per target), the rest per plan.
// ===========================================================================
namespace fst {

fst_status build_plans_many(Runner *(*mk)(), void *stream, int64_t count, const int64_t *N, const double *W,
                            const int64_t *K, const double *eps, fst_plan_t *out) {
  if (!out || count < 0 || (count > 0 && (!N || !W || !eps))) return fail(FST_EINVAL, "bad arguments");
  for (int64_t i = 0; i < count; ++i) out[i] = nullptr;
  auto cleanup = [&](fst_status s) {
    for (int64_t i = 0; i < count; ++i) {
      destroy_plan(out[i]);
      out[i] = nullptr;
    }
    return s;
  };
  std::vector<PendingWin> pw(count);
  for (int64_t i = 0; i < count; ++i) {
    Runner *R = mk();
    if (!R) return cleanup(fail(FST_ECUDA, "no CUDA device"));
    R->set_stream(stream);
    fst_status s = plan_begin(R, &out[i], N[i], W[i], K ? K[i] : -1, eps[i], FST_OP_PROJECT, 0.0);
    if (s != FST_OK) return cleanup(s);
    fst_plan_t p = out[i];
    pw[i].p = p;
    pw[i].centre = p->K;
    pw[i].Rw = std::max<int64_t>(
        2, (int64_t)std::min(ceil(cor1_bound(p->N, p->eps)), ceil(0.6 * asymptotic_transition(p->N, p->eps)) + 6.0));
    pw[i].S = nullptr;
    pw[i].done = false;
  }
  for (int attempt = 0; attempt < 14; ++attempt) {
    std::vector<PendingWin *> pend;
    for (auto &q : pw)
      if (!q.done) pend.push_back(&q);
    if (pend.empty()) break;
    // groups bounded by the device size of the window vectors (2^31 doubles, 16 GiB): large
    // enough that the batched bisection has targets for every SM
    size_t gi = 0;
    while (gi < pend.size()) {
      std::vector<PendingWin *> grp;
      int64_t elems = 0;
      while (gi < pend.size() && (grp.empty() || elems < (2048LL << 20))) {
        PendingWin *q = pend[gi++];
        fst_plan_t p = q->p;
        q->lo = std::max<int64_t>(0, q->centre - q->Rw);
        q->hi = std::min<int64_t>(p->N - 1, q->centre + q->Rw);
        const int64_t nwin = q->hi - q->lo + 1;
        fst_status s = p->R->alloc((void **)&q->S, (size_t)nwin * p->N * sizeof(double));
        if (s != FST_OK) return cleanup(s);
        elems += nwin * p->N;
        grp.push_back(q);
      }
      fst_status s = batched_window_vectors(grp);
      if (s != FST_OK) return cleanup(s);
      for (PendingWin *q : grp) {
        fst_plan_t p = q->p;
        const int nwin = (int)(q->hi - q->lo + 1);
        std::vector<double> lamw(nwin);
        s = window_eigenvalues(p, q->S, nwin, lamw.data(), p->spec_unit);
        if (s != FST_OK) return cleanup(s);
        const bool lo_ok = (q->lo == 0) || !in_T(lamw[0], q->lo, p->K, p->eps, p->op, p->alpha);
        const bool hi_ok = (q->hi == p->N - 1) || !in_T(lamw[nwin - 1], q->hi, p->K, p->eps, p->op, p->alpha);
        if (lo_ok && hi_ok) {
          s = plan_end(p, q->S, lamw, q->lo, q->hi);
          q->done = true;
        } else {
          q->Rw *= 2;
        }
        p->R->release(q->S);
        q->S = nullptr;
        if (s != FST_OK) return cleanup(s);
      }
    }
  }
  for (auto &q : pw)
    if (!q.done) return cleanup(fail(FST_ENOCONVERGE, "eigen-window search did not terminate"));
  return FST_OK;
}

}  // namespace fst

extern "C" {

fst_status fst_plan_many(fst_plan_t *out, int64_t count, const int64_t *N, const double *W, const int64_t *K,
                         const double *eps, void *stream) {
  return build_plans_many(make_dev_runner, stream, count, N, W, K, eps, out);
}

fst_status fst_emu_plan_many(fst_plan_t *out, int64_t count, const int64_t *N, const double *W, const int64_t *K,
                             const double *eps) {
  return build_plans_many(make_emu_runner, nullptr, count, N, W, K, eps, out);
}

}  // extern "C"

// ===========================================================================
// Ragged batches: signal i with its own plan plans[i]
// ===========================================================================
namespace fst {

// next buffer of the signature's state: allocated (and filled from `init`) on the first call,
// reused in the same order afterwards (same signature, same sizes and contents)
static fst_status ragged_buf(Runner *R, RaggedState &st, size_t bytes, const void *init, void **out) {
  if (st.next < st.bufs.size()) {
    *out = st.bufs[st.next++];
    return FST_OK;
  }
  void *b = nullptr;
  TRY(R->alloc(&b, std::max<size_t>(bytes, 16)));
  st.bufs.push_back(b);
  st.next = st.bufs.size();
  if (init) TRY(R->h2d(b, init, bytes));
  *out = b;
  return FST_OK;
}

static bool autotune_enabled() {
  const char *s = getenv("FST_AUTOTUNE");
  return !(s && s[0] == '0');
}

// The four-step signals of a ragged batch (FP32 device plans), by FFT length class M:
//   1. the correction coefficients a_i = D_i o S_T,i^T y_i of every signal (one launch over
//      (signal, 2048-sample chunk) items, one reduction launch);
//   2. per class, launch groups of transform slots through the batched column / row / column
//      passes, B y only: a complex signal takes a slot of its own, real signals share one two at
//      a time (re, im), each with its own data, length and spectrum (4096-point rows: the row
//      pass applies both spectra; other row lengths: one real signal per slot);
//   3. out_i += S_T,i a_i over all items (one launch).
// The pairs per launch group of each class are picked on the first call (autotuner: the
// candidate groupings of 16 .. 256 MiB of intermediate are timed with device events and the
// fastest kept; the grouping does not change the arithmetic, so results do not depend on it).
static fst_status ragged_fourstep_f32(const fst_plan_t *plans, const void *const *y, void *const *out,
                                      const std::vector<int64_t> &idx, bool cplx, RaggedState &st) {
  Runner *R = plans[idx[0]]->R;
  const int nsig = (int)idx.size();
  // correction descriptors and items
  std::vector<RSig> sig(nsig);
  std::vector<RItem> items;
  int64_t poff = 0;
  for (int i = 0; i < nsig; ++i) {
    fst_plan_t p = plans[idx[i]];
    RSig &q = sig[i];
    q.y = (const float *)y[idx[i]];
    q.out = (float *)out[idx[i]];
    q.ST = p->ST32;
    q.D = p->D32;
    q.N = p->N;
    q.r = (int)p->r;
    q.rpad = (int)p->rpad;
    q.nK = (int)(((p->N + 1) / 2 + CORR_BLOCK - 1) / CORR_BLOCK);   // chunks of the folded half
    q.part = poff;
    for (int w = 0; w < 4; ++w) q.odd[w] = 0;
    for (int j = 0; j < (int)p->r; ++j)
      if (p->idx[j] & 1) q.odd[j >> 5] |= 1u << (j & 31);
    poff += (int64_t)q.nK * 2 * q.rpad;
    if (p->r > 0)
      for (int c = 0; c < q.nK; ++c) items.push_back({i, c});
  }
  void *dsig, *ditems, *dpart, *dacoef;
  TRY(ragged_buf(R, st, sig.size() * sizeof(RSig), sig.data(), &dsig));
  TRY(ragged_buf(R, st, std::max<size_t>(1, items.size()) * sizeof(RItem), items.empty() ? nullptr : items.data(),
                 &ditems));
  TRY(ragged_buf(R, st, (size_t)std::max<int64_t>(poff, 1) * sizeof(float), nullptr, &dpart));
  TRY(ragged_buf(R, st, (size_t)nsig * 2 * RC_RMAX * sizeof(float), nullptr, &dacoef));
  TRY(R->rcorr((const RSig *)dsig, nsig, (const RItem *)ditems, (int)items.size(), cplx ? 1 : 0, (float *)dpart,
               (float *)dacoef));

  // length classes
  std::vector<std::vector<int>> cls(32);
  for (int i = 0; i < nsig; ++i) cls[plans[idx[i]]->log2M].push_back(i);
  if (st.chunk.empty()) {
    st.chunk.assign(32, 0);
    st.tune_ms.assign(32, 0.0);
  }
  // one intermediate workspace for every class (they run one after the other): 256 MiB at most
  size_t ws_max = 0;
  for (int lg = 0; lg < 32; ++lg)
    if (!cls[lg].empty())
      ws_max = std::max(ws_max, std::min<size_t>((size_t)cls[lg].size(), std::max<size_t>(1, (256u << 20) >> (lg + 3))) *
                                    ((size_t)8 << lg));
  void *dws;
  TRY(ragged_buf(R, st, ws_max, nullptr, &dws));
  for (int lg = 0; lg < 32; ++lg) {
    if (cls[lg].empty()) continue;
    const std::vector<int> &c = cls[lg];
    const int64_t cnt = (int64_t)c.size();
    fst_plan_t p0 = plans[idx[c[0]]];
    int64_t Nmax = 0;
    for (int k : c) Nmax = std::max(Nmax, plans[idx[k]]->N);
    const Layout L = make_layout(Nmax, lg, false, 8, true);
    // real signals of the class travel two to a slot (re, im) when the row pass can apply two
    // spectra (4096-point rows); otherwise one per slot
    const bool two = !cplx && (L.fast || L.big) && L.log2Q == 12;
    const int64_t nslot = two ? (cnt + 1) / 2 : cnt;
    std::vector<RPair<float>> rp(nslot);
    for (int64_t k = 0; k < nslot; ++k) {
      const int i0 = two ? c[2 * k] : c[k];
      fst_plan_t p = plans[idx[i0]];
      RPair<float> &q = rp[k];
      q = RPair<float>{};
      q.y = (const float *)y[idx[i0]];
      q.out = (float *)out[idx[i0]];
      q.spec = p->spec32;
      q.N = p->N;
      if (two && 2 * k + 1 < cnt) {
        const int i1 = c[2 * k + 1];
        fst_plan_t p1 = plans[idx[i1]];
        q.y2 = (const float *)y[idx[i1]];
        q.out2 = (float *)out[idx[i1]];
        q.spec2 = p1->spec32;
        q.N2 = p1->N;
      }
    }
    void *drp;
    TRY(ragged_buf(R, st, rp.size() * sizeof(RPair<float>), rp.data(), &drp));
    ConvArgs<float> a{};
    a.rp = (const RPair<float> *)drp;
    a.two_spec = two ? 1 : 0;
    a.batch = nslot;
    a.cplx = cplx ? 1 : 0;
    a.N = Nmax;
    a.log2M = L.log2M;
    a.log2P = L.log2P;
    a.log2Q = L.log2Q;
    a.Pnz = L.Pnz;
    a.NB = L.NB;
    a.G = L.G;
    a.r = 0;
    a.rpad = 8;
    a.tw = plan_tw<float>(p0);
    a.twB = p0->twB;
    a.tw8 = p0->tw8;
    a.inter = (float2 *)dws;
    a.mode = MODE_CONV;
    auto run_groups = [&](int64_t chunk) -> fst_status {
      for (int64_t q0 = 0; q0 < nslot; q0 += chunk) {
        a.pair0 = q0;
        a.npairs = std::min<int64_t>(chunk, nslot - q0);
        TRY(R->passA(a, L));
        TRY(R->passB(a, L));
        TRY(R->passC(a, L));
      }
      return FST_OK;
    };
    const int64_t cap = std::max<int64_t>(1, (int64_t)(ws_max >> (lg + 3)));
    if (st.chunk[lg] == 0) {
      int64_t best = std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)((128u << 20) >> (lg + 3))));
      double best_ms = 0.0;
      // in place (y == out) a second run would read its own output: no timing runs then
      bool inplace = false;
      for (int64_t k = 0; k < cnt; ++k) inplace = inplace || y[idx[c[k]]] == out[idx[c[k]]];
      if (autotune_enabled() && !inplace && !R->user_stream_capturing()) {
        for (int mb = 16; mb <= 256; mb *= 2) {
          const int64_t ch = std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)(((size_t)mb << 20) >> (lg + 3))));
          if (mb > 16 && ch == std::min<int64_t>(cap, std::max<int64_t>(1, (int64_t)(((size_t)(mb / 2) << 20) >> (lg + 3)))))
            continue;   // same grouping as the previous candidate
          TRY(run_groups(ch));   // warm
          double ms = 0.0;
          TRY(R->timer(0, nullptr));
          TRY(run_groups(ch));
          TRY(R->timer(1, &ms));
          if (best_ms == 0.0 || ms < best_ms) {
            best_ms = ms;
            best = ch;
          }
        }
      }
      st.chunk[lg] = best;
      st.tune_ms[lg] = best_ms;
    }
    TRY(run_groups(st.chunk[lg]));
  }
  return R->rzadd((const RSig *)dsig, (const RItem *)ditems, (int)items.size(), cplx ? 1 : 0, (const float *)dacoef);
}

template <typename T>
static fst_status ragged_t(const fst_plan_t *plans, const void *const *y, void *const *out, int64_t count,
                           bool cplx, RaggedState &st) {
  const bool dbl = sizeof(T) == 8;
  st.next = 0;
  // single-CTA signals by FFT length, one launch each
  std::vector<std::vector<RaggedDesc<T>>> buckets(32);
  std::vector<int> maxr(32, 0);
  std::vector<int64_t> others;
  for (int64_t i = 0; i < count; ++i) {
    fst_plan_t p = plans[i];
    const Layout &L = dbl ? p->lay64 : p->lay32;
    if (L.small) {
      RaggedDesc<T> d;
      d.y = (const T *)y[i];
      d.out = (T *)out[i];
      d.spec = (const T *)(dbl ? (const void *)p->spec64 : (const void *)p->spec32);
      d.ST = (const T *)(dbl ? (const void *)p->ST64 : (const void *)p->ST32);
      d.D = (const T *)(dbl ? (const void *)p->D64 : (const void *)p->D32);
      d.N = p->N;
      d.r = (int)p->r;
      d.rpad = (int)p->rpad;
      buckets[p->log2M].push_back(d);
      maxr[p->log2M] = std::max(maxr[p->log2M], (int)p->rpad);
    } else {
      others.push_back(i);
    }
  }
  for (int lg = 0; lg < 32; ++lg) {
    if (buckets[lg].empty()) continue;
    fst_plan_t p0 = nullptr;
    for (int64_t i = 0; i < count && !p0; ++i)
      if (plans[i]->log2M == lg && (dbl ? plans[i]->lay64 : plans[i]->lay32).small) p0 = plans[i];
    Runner *R = p0->R;
    Layout L = make_layout(p0->N, lg, dbl, maxr[lg], false);
    void *dd = nullptr;
    TRY(ragged_buf(R, st, buckets[lg].size() * sizeof(RaggedDesc<T>), buckets[lg].data(), &dd));
    ConvArgs<T> base{};
    base.batch = 1;
    base.cplx = cplx ? 1 : 0;
    base.log2M = lg;
    base.tw = plan_tw<T>(p0);
    base.mode = MODE_FULL;
    base.pair0 = 0;
    base.npairs = 1;
    TRY(R->small_ragged((const RaggedDesc<T> *)dd, (int)buckets[lg].size(), base, L));
  }
  if (others.empty()) return FST_OK;
  // FP32 device plans: batched four-step path; otherwise one call per signal
  bool batched = !dbl;
  for (int64_t i : others) {
    fst_plan_t p = plans[i];
    batched = batched && p->R->device() && p->lay32.log2Q >= 12 && p->rpad <= RC_RMAX && p->twB && p->ST32 &&
              (p->lay32.fast || p->lay32.big) && (!cplx || (uintptr_t)out[i] % 8 == 0) &&
              (!cplx || (uintptr_t)y[i] % 8 == 0);
  }
  if (batched) return ragged_fourstep_f32(plans, y, out, others, cplx, st);
  for (int64_t i : others)
    TRY(run_apply(plans[i], y[i], out[i], 1, 0, cplx ? (dbl ? FST_C128 : FST_C64) : (dbl ? FST_F64 : FST_F32), true));
  return FST_OK;
}

fst_status run_ragged(const fst_plan_t *plans, const void *const *y, void *const *out, int64_t count, int dtype,
                      RaggedState &desc_bufs) {
  if (count < 0 || (count > 0 && (!plans || !y || !out))) return fail(FST_EINVAL, "bad arguments");
  for (int64_t i = 0; i < count; ++i)
    if (!plans[i] || !y[i] || !out[i]) return fail(FST_EINVAL, "NULL plan or signal pointer");
  if (count == 0) return FST_OK;
  switch (dtype) {
    case FST_F32: return ragged_t<float>(plans, y, out, count, false, desc_bufs);
    case FST_C64: return ragged_t<float>(plans, y, out, count, true, desc_bufs);
    case FST_F64: return ragged_t<double>(plans, y, out, count, false, desc_bufs);
    case FST_C128: return ragged_t<double>(plans, y, out, count, true, desc_bufs);
    default: return fail(FST_EINVAL, "unknown dtype");
  }
}

}  // namespace fst
