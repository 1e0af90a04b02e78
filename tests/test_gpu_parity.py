"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (per signal, 2-norm, relative to ||y||):
  * against the oracle's fast projection at the same eps (same method, FP64):
    FP64 path 1e-12, FP32 path 1e-5 (FP32 FFT of length M ~ 2^17..2^23 rounds at
    ~1e-7 per element; 1e-5 is the stated FP32 budget);
  * against the plain definition S_K S_K^T y: eps + 1e-12 (FP64) and eps + 1e-5
    (FP32), the Corollary 2 bound plus the rounding budget.
The transition set T is an integer decision taken from FP64 eigenvalues on both
sides; it must agree exactly.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_04950_gb300 import fst as F  # noqa: E402
from paper_1611_04950_gb300 import workloads  # noqa: E402
from oracle import fst_oracle as O  # noqa: E402


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@functools.lru_cache(maxsize=None)
def oplan(N, W, K, eps, op="project", alpha=0.0):
    return O.make_plan(N, W, K, eps, op=op, alpha=alpha)


def rel_err(out, ref, y):
    out = np.asarray(out, dtype=np.complex128 if np.iscomplexobj(out) else np.float64)
    return np.linalg.norm(out - ref, axis=1) / np.linalg.norm(y, axis=1)


# ---------------------------------------------------------------- plan ------------

@pytest.mark.parametrize("N,W,eps", [(4096, 1 / 16, 1e-6), (65536, 1 / 8, 1e-4), (1000, 1 / 64, 1e-8),
                                     (12345, 0.3, 1e-3), (777, 0.45, 1e-12), (1, 0.3, 1e-6), (2, 0.1, 1e-6),
                                     (3001, 0.25, 1e-6), (40000, 0.25, 1e-8)])   # W = 1/4: zero diagonal
def test_plan_matches_oracle(N, W, eps):
    _cuda()
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    ex = p.export()
    assert p.K == O.default_K(N, W)
    assert p.r == o.r
    assert np.array_equal(ex["idx"], o.idx)
    assert np.max(np.abs(ex["lam"] - o.lam), initial=0) < 1e-12
    if p.r:
        assert np.max(np.abs(ex["S_T"] - o.S_T)) < 1e-9


# ---------------------------------------------------------------- tiny (FP64 + FP32) ----

@functools.lru_cache(maxsize=None)
def tiny_exact():
    wl = workloads.tiny()
    y = wl.y.numpy()
    return wl, y, O.exact_project(wl.N, wl.W, O.default_K(wl.N, wl.W), y.T).T


def test_tiny_fp64_and_fp32_against_exact_and_fast():
    dev = _cuda()
    wl, y, exact = tiny_exact()
    p = F.Plan(wl.N, wl.W, eps=wl.eps)
    o = oplan(wl.N, wl.W, p.K, wl.eps)
    fast = O.fast_project(o, y.T).T
    yd = torch.as_tensor(y, device=dev)
    out64 = p.project(yd).cpu().numpy()
    out32 = p.project(yd.float()).cpu().numpy()
    assert np.all(rel_err(out64, fast, y) < 1e-12)
    assert np.all(rel_err(out32, fast, y) < 1e-5)
    assert np.all(rel_err(out64, exact, y) <= wl.eps + 1e-12)
    assert np.all(rel_err(out32, exact, y) <= wl.eps + 1e-5)


# ---------------------------------------------------------------- N = 65536 -------------

def test_c65k_small_batch():
    dev = _cuda()
    wl = workloads.c65k(batch=6)
    p = F.Plan(wl.N, wl.W, eps=wl.eps)
    o = oplan(wl.N, wl.W, p.K, wl.eps)
    y = wl.y.numpy().astype(np.float64)
    fast = O.fast_project(o, y.T).T
    out = p.project(wl.y.to(dev)).cpu().numpy()
    assert np.all(rel_err(out, fast, y) < 1e-5)
    ref = O.fast_project(oplan(wl.N, wl.W, p.K, O.EPS_REF), y.T).T   # within 1e-13 of S_K S_K^T y
    assert np.all(rel_err(out, ref, y) <= wl.eps + 1e-5)


def _fast_rows(o, y, chunk=128):
    """Oracle fast projection of the rows of y (FP64), in chunks of rows."""
    out = np.empty(y.shape, dtype=np.complex128 if np.iscomplexobj(y) else np.float64)
    for i in range(0, y.shape[0], chunk):
        out[i:i + chunk] = O.fast_project(o, y[i:i + chunk].T).T
    return out


def test_c65k_full_batch_every_row():
    # the benchmark's launch configuration: 1024 signals in one call (every tcgen05 row block,
    # launch group and column tile), every row against the FP64 oracle
    _cuda()
    wl = workloads.c65k(batch=1024, device="cuda")
    p = F.Plan(wl.N, wl.W, eps=wl.eps)
    out = p.project(wl.y)
    torch.cuda.synchronize()
    F.fst_sync(p.h, 0)
    o = oplan(wl.N, wl.W, p.K, wl.eps)
    y = wl.y.double().cpu().numpy()
    e = rel_err(out.cpu().numpy(), _fast_rows(o, y), y)
    assert e.shape == (1024,)
    assert np.all(e < 1e-5), (np.argmax(e), e.max())


# ---------------------------------------------------------------- edge cases ------------

@pytest.mark.parametrize("N,W,eps", [(1, 0.3, 1e-6), (3, 0.2, 1e-6), (17, 0.05, 1e-3), (1000, 1 / 64, 1e-8),
                                     (4097, 0.2, 1e-6), (8192, 0.25, 1e-8), (8193, 0.1, 1e-6),
                                     (30001, 0.17, 1e-6), (131072, 1 / 64, 1e-3)])
def test_ragged_lengths_fp32_fp64(N, W, eps):
    dev = _cuda()
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    y = workloads.gaussian(3, N, seed=N)          # odd batch
    fast = O.fast_project(o, y.numpy().T).T
    out64 = p.project(y.to(dev)).cpu().numpy()
    out32 = p.project(y.float().to(dev)).cpu().numpy()
    assert np.all(rel_err(out64, fast, y.numpy()) < 1e-12)
    assert np.all(rel_err(out32, fast, y.numpy()) < 1e-5)


@pytest.mark.parametrize("N,W,eps,cplx", [(150001, 0.1, 1e-6, False),     # M = 2^19: P = 128 (P2 = 4)
                                           (300000, 0.02, 1e-4, True),      # M = 2^20: P = 256 (P2 = 8)
                                           (1048577, 0.01, 1e-3, False)])   # M = 2^22: P = 1024 (P2 = 32)
def test_two_stage_column_passes(N, W, eps, cplx):
    # the FP32 four-step path with P = 32 P2 column rows (two register stages), odd batches,
    # every row against the FP64 oracle
    dev = _cuda()
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    assert p.r == o.r
    y = workloads.gaussian(3, N, seed=N % 1000, complex_=cplx)
    fast = O.fast_project(o, y.numpy().T).T
    out = p.project(y.to(torch.complex64 if cplx else torch.float32).to(dev)).cpu().numpy()
    e = rel_err(out, fast, y.numpy())
    assert np.all(e < 1e-5), e


def test_complex_signals():
    dev = _cuda()
    N, W, eps = 20000, 0.05, 1e-6
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    y = workloads.gaussian(4, N, seed=3, complex_=True)
    fast = O.fast_project(o, y.numpy().T).T
    out128 = p.project(y.to(dev)).cpu().numpy()
    out64 = p.project(y.to(torch.complex64).to(dev)).cpu().numpy()
    assert np.all(rel_err(out128, fast, y.numpy()) < 1e-12)
    assert np.all(rel_err(out64, fast, y.numpy()) < 1e-5)


def test_wide_transition_band_real_and_complex():
    # r ~ 69 > 64: the tcgen05 correction's wide-S variant (nB = 96, one accumulator for the
    # three TF32 products), 300 real signals (three 128-row blocks, odd count) and 70 complex
    # ones (two 64-signal blocks); sampled rows against the FP64 oracle's fast projection
    dev = _cuda()
    N, W, eps = 32768, 0.25, 1e-14
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    # at eps = 1e-14 an eigenvalue within rounding of the 1 - eps threshold may fall on either
    # side in the two FP64 solvers; such a vector has |D| ~ eps and moves the result by ~1e-14
    assert p.r > 64 and abs(p.r - o.r) <= 1
    g = np.random.default_rng(21)
    yr = torch.from_numpy(g.standard_normal((301, N))).float()
    yc = torch.complex(torch.from_numpy(g.standard_normal((70, N))).float(),
                       torch.from_numpy(g.standard_normal((70, N))).float())
    outr = p.project(yr.to(dev)).cpu().numpy()
    outc = p.project(yc.to(dev)).cpu().numpy()
    for y, out, rows in ((yr, outr, [0, 1, 127, 128, 255, 256, 300]), (yc, outc, [0, 63, 64, 69])):
        ys = y[rows].numpy().astype(np.complex128 if y.is_complex() else np.float64)
        fast = O.fast_project(o, ys.T).T
        assert np.all(rel_err(out[rows], fast, ys) < 1e-5)


def test_apply_prolate_direct_sum():
    dev = _cuda()
    N, W = 2049, 0.21
    p = F.Plan(N, W, eps=1e-6)
    y = workloads.gaussian(2, N, seed=1)
    out = p.apply_prolate(y.to(dev)).cpu().numpy()
    ref = O.apply_prolate_direct(y.numpy().T, W).T
    assert np.max(np.abs(out - ref)) < 1e-12 * np.sqrt(N)


@pytest.mark.parametrize("op,alpha,mul", [("pinv", 0.0, 3.0), ("tikhonov", 1e-3, 1.0)])
def test_other_operators(op, alpha, mul):
    dev = _cuda()
    N, W, eps = 600, 0.2, 1e-5
    p = F.Plan(N, W, eps=eps, op=op, alpha=alpha)
    o = oplan(N, W, p.K, eps, op, alpha)
    assert p.r == o.r
    y = workloads.gaussian(2, N, seed=8)
    out = p.project(y.to(dev)).cpu().numpy()
    assert np.max(np.abs(out - O.fast_apply(o, y.numpy().T).T)) < 1e-10
    exact = O.exact_operator_dense(N, W, p.K, op, alpha)
    assert np.all(rel_err(out, (exact @ y.numpy().T).T, y.numpy()) <= mul * eps + 1e-10)


@pytest.mark.parametrize("op,alpha", [("pinv", 0.0), ("tikhonov", 1e-3)])
@pytest.mark.parametrize("cplx", [False, True])
def test_other_operators_four_step(op, alpha, cplx):
    # N = 65536: the four-step kernels with the pseudoinverse D (1/lambda - lambda on l < K) and
    # with the Tikhonov scaling of the Toeplitz part (beta = 1/(1 + alpha) = 0.999, visible far
    # above the tolerance), against the FP64 oracle
    dev = _cuda()
    N, W, eps = 65536, 1 / 8, 1e-5
    p = F.Plan(N, W, eps=eps, op=op, alpha=alpha)
    o = oplan(N, W, p.K, eps, op, alpha)
    assert p.r == o.r
    y = workloads.gaussian(6, N, seed=31, complex_=cplx)
    ref = O.fast_apply(o, y.numpy().T).T
    out = p.project(y.to(torch.complex64 if cplx else torch.float32).to(dev)).cpu().numpy()
    assert np.all(rel_err(out, ref, y.numpy()) < 1e-5 * max(1.0, np.abs(o.D).max()))
    if op == "tikhonov":
        # without the 1/(1 + alpha) scaling the result would be off by ~alpha ||B y||
        plain = O.fast_apply(oplan(N, W, p.K, eps), y.numpy().T).T
        assert np.all(rel_err(out, plain, y.numpy()) > 1e-4)


def _threshold_K(N, W, lam_min=1e-4):
    # eigenvalues above lam_min (Section 4.2's truncation): Rayleigh quotients of a window of
    # the oracle's Slepian vectors beyond round(2NW)
    K0 = O.default_K(N, W)
    lo, hi = max(0, K0 - 8), min(N - 1, K0 + 120)
    lam = O.rayleigh_eigenvalues(O.dpss_window(N, W, lo, hi), W)
    assert lam[0] > lam_min > lam[-1]
    return lo + int(np.sum(lam > lam_min))


@pytest.mark.parametrize("M", [448, 4096])
def test_fourier_extension_pinv(M):
    # Section 4.2: the normal equations B g = F y of the Fourier extension (T = 1.5), solved with
    # the fast truncated pseudoinverse (eigenvalues below 1e-4 truncated, eps = 1e-5) on the GPU,
    # FP64 and FP32, against the oracle; for M = 448 also the paper's claim that the extension's
    # RMS error is at least 10 times below the truncated Fourier series'
    from tests.test_oracle_fext import rel_rms, synth
    dev = _cuda()
    fe = workloads.fourier_extension(M)
    K = _threshold_K(fe.N, fe.W)
    p = F.Plan(fe.N, fe.W, K=K, eps=1e-5, op="pinv")
    o = oplan(fe.N, fe.W, K, 1e-5, "pinv")
    assert p.r == o.r
    ref = O.fast_apply(o, fe.yhat)
    gain = max(1.0, np.abs(o.D).max())
    nrm = np.linalg.norm(fe.yhat)
    g64 = p.project(torch.from_numpy(fe.yhat[None, :]).to(dev)).cpu().numpy()[0]
    g32 = p.project(torch.from_numpy(fe.yhat[None, :].astype(np.complex64)).to(dev)).cpu().numpy()[0]
    assert np.linalg.norm(g64 - ref) <= 1e-12 * gain * nrm
    assert np.linalg.norm(g32 - ref) <= 1e-5 * gain * nrm
    if M <= 1024:
        t = np.linspace(-1.0, 1.0, 4097)
        ft = fe.f(t)
        e_ref = rel_rms(synth(ref, t, fe.T), ft, t)
        e32 = rel_rms(synth(g32.astype(np.complex128), t, fe.T), ft, t)
        e_ser = rel_rms(synth(fe.fhat, t, 1.0), ft, t)
        assert abs(e32 - e_ref) <= 0.02 * e_ref
        assert e32 * 10 <= e_ser


def test_degenerate_K_and_batch_zero():
    dev = _cuda()
    N, W = 200, 0.1
    y = workloads.gaussian(2, N, seed=2).to(dev)
    for K, want in ((0, torch.zeros_like(y)), (N, y)):
        p = F.Plan(N, W, K=K, eps=1e-6)
        out = p.project(y)
        assert torch.all(torch.linalg.vector_norm(out - want, dim=1) <= 1e-6 * torch.linalg.vector_norm(y, dim=1) + 1e-12)
    p = F.Plan(N, W, eps=1e-6)
    F.fst_project(p.h, y.data_ptr(), y.data_ptr(), 0, N, F.FST_F64, 0)


def test_strided_inplace_and_host_entry_point():
    dev = _cuda()
    N, W = 40000, 0.125
    p = F.Plan(N, W, eps=1e-4)
    y = workloads.gaussian(5, N + 7, seed=4).float().to(dev)
    view = y[:, :N]
    out = torch.zeros_like(y)
    F.fst_project(p.h, view.data_ptr(), out.data_ptr(), 5, N + 7, F.FST_F32,
                  torch.cuda.current_stream().cuda_stream)
    dense = p.project(view.contiguous())
    torch.cuda.synchronize()
    # rows N + 7 floats apart are not 16-byte aligned, so no TMA tensor map can address them:
    # that call sums S_T^T y on the mma.sync kernels instead of tcgen05 (another summation
    # order, same FP32 accuracy)
    scale = dense.abs().max().item()
    assert (out[:, :N] - dense).abs().max().item() <= 2e-6 * scale
    assert torch.all(out[:, N:] == 0)
    host = view.contiguous().cpu().pin_memory()
    hout = p.project_host(host)
    assert torch.equal(hout, dense.cpu())
    z = view.contiguous().clone()
    F.fst_project(p.h, z.data_ptr(), z.data_ptr(), 5, N, F.FST_F32, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(z, dense)


def test_repeatable_bit_for_bit():
    dev = _cuda()
    N, W = 65536, 0.25
    p = F.Plan(N, W, eps=1e-8)
    y = workloads.gaussian(8, N, seed=12).float().to(dev)
    a = p.project(y)
    b = p.project(y)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# ---------------------------------------------------------------- fast coefficient vector

@pytest.mark.parametrize("N,W,eps", [(4096, 1 / 16, 1e-6), (65536, 0.25, 1e-8)])
def test_coeffs_against_oracle(N, W, eps):
    from oracle import thm1 as T
    dev = _cuda()
    p = F.Plan(N, W, eps=eps)
    t = T.thm1(N, W, eps)
    o = oplan(N, W, p.K, eps)
    y = workloads.gaussian(3, N, seed=21)
    ref = T.coeffs(t, o, y.numpy().T).T
    nrm = np.linalg.norm(y.numpy(), axis=1)[:, None]
    c64 = p.coeffs(y.to(dev)).cpu().numpy()
    c32 = p.coeffs(y.float().to(dev)).cpu().numpy()
    assert c64.shape == ref.shape
    assert np.all(np.abs(c64 - ref) <= 1e-11 * nrm)
    assert np.all(np.abs(c32 - ref) <= 1e-5 * nrm)
    if N <= 8192:
        back = T.expand(t, o, c32[0].astype(np.complex128))
        ex = O.exact_project(N, W, p.K, y.numpy()[0])
        assert np.linalg.norm(back - ex) <= (2 * eps + 1e-5) * nrm[0, 0]


def test_expand_against_dense_T1_and_roundtrip():
    # T1 c on the GPU (FP64 and FP32) against the oracle's dense T1 on random coefficients,
    # and T1 T2^* y against the exact projection (within 2 eps of it, Section 1.3)
    from oracle import thm1 as T
    dev = _cuda()
    N, W, eps = 4096, 1 / 16, 1e-6
    p = F.Plan(N, W, eps=eps)
    t = T.thm1(N, W, eps)
    o = oplan(N, W, p.K, eps)
    Kp = F.fst_coeffs_info(p.h)["Kprime"]
    g = np.random.default_rng(8)
    c = g.standard_normal((3, Kp)) + 1j * g.standard_normal((3, Kp))
    ref = np.stack([T.expand(t, o, ci) for ci in c])
    scale = np.abs(ref).max()
    e128 = p.expand(torch.from_numpy(c).to(dev)).cpu().numpy()
    e64 = p.expand(torch.from_numpy(c.astype(np.complex64)).to(dev)).cpu().numpy()
    assert np.max(np.abs(e128 - ref)) <= 1e-12 * scale
    assert np.max(np.abs(e64 - ref)) <= 2e-5 * scale
    y = workloads.gaussian(2, N, seed=22)
    ex = O.exact_project(N, W, p.K, y.numpy().T).T
    nrm = np.linalg.norm(y.numpy(), axis=1)
    back64 = p.expand(p.coeffs(y.to(dev))).cpu().numpy()
    back32 = p.expand(p.coeffs(y.float().to(dev))).cpu().numpy()
    assert np.all(np.linalg.norm(back64 - ex, axis=1) <= 2 * eps * nrm)
    assert np.all(np.linalg.norm(back32 - ex, axis=1) <= (2 * eps + 1e-5) * nrm)


def test_expand_roundtrip_large_N():
    # N = 65536, eps = 1e-8: T1 T2^* y against the oracle's fast projection (each within a
    # few eps of S_K S_K^T y), FP32 end to end on the device
    dev = _cuda()
    N, W, eps = 65536, 0.25, 1e-8
    p = F.Plan(N, W, eps=eps)
    o = oplan(N, W, p.K, eps)
    y = workloads.gaussian(2, N, seed=23)
    fast = O.fast_project(o, y.numpy().T).T
    back = p.expand(p.coeffs(y.float().to(dev))).cpu().numpy()
    nrm = np.linalg.norm(y.numpy(), axis=1)
    assert np.all(np.linalg.norm(back - fast, axis=1) <= (3 * eps + 2e-5) * nrm)


def test_coeffs_complex_input():
    from oracle import thm1 as T
    dev = _cuda()
    N, W, eps = 8192, 0.05, 1e-6
    p = F.Plan(N, W, eps=eps)
    t = T.thm1(N, W, eps)
    o = oplan(N, W, p.K, eps)
    y = workloads.gaussian(2, N, seed=5, complex_=True)
    ref = T.coeffs(t, o, y.numpy().T).T
    got = p.coeffs(y.to(torch.complex64).to(dev)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.linalg.norm(y.numpy(), axis=1)[:, None])


# ---------------------------------------------------------------- full-size workloads, sampled

def test_c1m_complex_full_batch_every_row():
    # N = 2^20, W = 0.05, eps = 1e-6, 64 complex64 signals (half band-limited), one call
    _cuda()
    wl = workloads.c1m(batch=64, device="cuda")
    p = F.Plan(wl.N, wl.W, eps=wl.eps)
    out = p.project(wl.y)
    torch.cuda.synchronize()
    o = oplan(wl.N, wl.W, p.K, wl.eps)
    assert p.r == o.r
    y = wl.y.to(torch.complex128).cpu().numpy()
    e = rel_err(out.cpu().numpy(), _fast_rows(o, y, chunk=8), y)
    assert e.shape == (64,)
    assert np.all(e < 1e-5), (np.argmax(e), e.max())


@functools.lru_cache(maxsize=None)
def _c4m():
    wl = workloads.c4m(batch=16, device="cuda")
    p = F.Plan(wl.N, wl.W, eps=wl.eps)
    return wl, p


def test_c4m_full_batch_projection_every_row_and_coeffs():
    # N = 2^22, W = 1/4, eps = 1e-8, 16 real FP32 signals: every projected row, and the
    # coefficient vector of two rows (one from each half of the workload)
    from oracle import thm1 as T
    _cuda()
    wl, p = _c4m()
    out = p.project(wl.y)
    coef = p.coeffs(wl.y)
    torch.cuda.synchronize()
    o = oplan(wl.N, wl.W, p.K, wl.eps)
    assert p.r == o.r
    y = wl.y.double().cpu().numpy()
    e = rel_err(out.cpu().numpy(), _fast_rows(o, y, chunk=4), y)
    assert e.shape == (16,)
    assert np.all(e < 1e-5), (np.argmax(e), e.max())
    idx = [0, 15]
    t = T.thm1(wl.N, wl.W, wl.eps)
    ref = T.coeffs(t, o, y[idx].T).T
    c = coef[idx].cpu().numpy()
    assert c.shape == ref.shape
    assert np.all(np.abs(c - ref) <= 1e-5 * np.linalg.norm(y[idx], axis=1)[:, None])


def test_c4m_repeatable_bit_for_bit():
    # the large tight-tolerance workload: projection and coefficient vector, run twice
    _cuda()
    wl, p = _c4m()
    a, ca = p.project(wl.y), p.coeffs(wl.y)
    b, cb = p.project(wl.y), p.coeffs(wl.y)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(ca, cb)


# ---------------------------------------------------------------- ragged batches

def test_ragged_batch_against_oracle_and_replay():
    dev = _cuda()
    params = workloads.ragged_params(48, seed=3)          # N log-uniform in [1000, 262144]
    ps = F.PlanSet(params)
    rng = np.random.default_rng(7)
    ys64 = [rng.standard_normal(N) for (N, W, e) in params]
    ys = [torch.as_tensor(y, dtype=torch.float32, device=dev) for y in ys64]
    outs = [torch.empty_like(v) for v in ys]
    ps.project(ys, outs)                 # direct
    first = [o.clone() for o in outs]
    ps.project(ys, outs)                 # recorded into a graph
    ps.project(ys, outs)                 # replayed
    torch.cuda.synchronize()
    for a, b in zip(first, outs):
        assert torch.equal(a, b)
    order = np.argsort([N for (N, W, e) in params])
    check = list(order[:3]) + list(order[len(order) // 2:len(order) // 2 + 2]) + list(order[-2:])
    for i in check:
        N, W, e = params[i]
        op = oplan(N, W, O.default_K(N, W), e)
        assert ps.info(i)["r"] == op.r
        ref = O.fast_project(op, ys64[i])
        err = np.linalg.norm(outs[i].double().cpu().numpy() - ref) / np.linalg.norm(ys64[i])
        assert err < 1e-5, (i, N, err)


@pytest.mark.parametrize("inplace", [False, True])
def test_ragged_paired_real_slots(inplace):
    # real signals of one FFT-length class share a complex transform two at a time, each with
    # its own spectrum (different N, W, eps); an odd count leaves one slot with a single signal.
    # M = 2^18 (P = 64, two-stage column passes) and M = 2^16 (P = 16): every signal against
    # the FP64 oracle, and the in-place call equal to the out-of-place one
    dev = _cuda()
    params = [(70001, 0.3, 1e-6), (90000, 0.05, 1e-4), (100003, 0.12, 1e-8), (120000, 0.2, 1e-6),
              (131072, 0.01, 1e-3), (20000, 0.25, 1e-6), (30001, 0.1, 1e-8), (32768, 0.03, 1e-4)]
    ps = F.PlanSet(params)
    rng = np.random.default_rng(21)
    ys64 = [rng.standard_normal(N) for (N, W, e) in params]
    ys = [torch.as_tensor(y, dtype=torch.float32, device=dev) for y in ys64]
    outs = [torch.empty_like(v) for v in ys]
    ps.project(ys, outs)
    if inplace:
        io = [v.clone() for v in ys]
        ps.project(io, io)
        torch.cuda.synchronize()
        for a, b in zip(outs, io):
            assert torch.equal(a, b)
    torch.cuda.synchronize()
    for i, (N, W, e) in enumerate(params):
        op = oplan(N, W, O.default_K(N, W), e)
        ref = O.fast_project(op, ys64[i])
        err = np.linalg.norm(outs[i].double().cpu().numpy() - ref) / np.linalg.norm(ys64[i])
        assert err < 1e-5, (i, N, err)


def test_ragged_4096_every_signal():
    # the ragged workload at full size (4096 signals, N log-uniform in [1000, 262144], own W and
    # eps each): every signal of the batched call against the one-signal-per-call path, a
    # stratified sample of 48 against the FP64 oracle (spawn pool), and repeated calls (direct
    # with tuning, recorded, replayed) bit for bit
    import concurrent.futures as cf
    import multiprocessing as mp
    from tests._oracle_pool import oracle_fast
    _cuda()
    params = workloads.ragged_params(4096, seed=3)
    ps = F.PlanSet(params)
    lens = [N for (N, W, e) in params]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    gen = torch.Generator(device="cuda").manual_seed(11)
    yall = torch.randn(int(offs[-1]), device="cuda", generator=gen)
    oall = torch.empty_like(yall)
    ys = [yall[offs[i]:offs[i + 1]] for i in range(len(params))]
    outs = [oall[offs[i]:offs[i + 1]] for i in range(len(params))]
    ps.project(ys, outs)
    first = oall.clone()
    ps.project(ys, outs)
    ps.project(ys, outs)
    torch.cuda.synchronize()
    assert torch.equal(first, oall)
    # one fst_project call per signal (the plans' own paths)
    single = torch.empty_like(yall)
    stream = torch.cuda.current_stream().cuda_stream
    for i, h in enumerate(ps.h):
        F.fst_project(h, ys[i].data_ptr(), single[offs[i]:offs[i + 1]].data_ptr(), 1, 0, F.FST_F32, stream)
    torch.cuda.synchronize()
    d = (oall - single).double()
    num = torch.zeros(len(params), dtype=torch.float64, device="cuda")
    den = torch.zeros_like(num)
    seg = torch.repeat_interleave(torch.arange(len(params), device="cuda"),
                                  torch.as_tensor(lens, device="cuda"))
    num.index_add_(0, seg, d * d)
    den.index_add_(0, seg, yall.double() ** 2)
    rel = torch.sqrt(num / den).cpu().numpy()
    assert np.all(rel < 2e-6), (int(np.argmax(rel)), float(rel.max()))
    # stratified sample against the oracle (48 signals spread over the sorted lengths)
    order = np.argsort(lens)
    pick = [int(order[k]) for k in np.linspace(0, len(order) - 1, 48).round().astype(int)]
    jobs = [(params[i][0], params[i][1], params[i][2], ys[i].double().cpu().numpy()) for i in pick]
    with cf.ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=mp.get_context("spawn")) as ex:
        refs = list(ex.map(oracle_fast, jobs))
    for i, ref, job in zip(pick, refs, jobs):
        err = np.linalg.norm(outs[i].double().cpu().numpy() - ref) / np.linalg.norm(job[3])
        assert err < 1e-5, (i, params[i], err)
