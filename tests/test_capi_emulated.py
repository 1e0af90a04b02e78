"""CPU tests of the C ABI library: it loads and exports every declared symbol, it
rejects bad arguments, and -- through the host emulator, which runs the library's
own kernel bodies on the CPU -- its plan and apply paths agree with the FP64 oracle."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest
import scipy.linalg as sla

import paper_1611_04950_gb300 as P
from paper_1611_04950_gb300 import fst as F
from oracle import fst_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in ("fst.h", "fst_testing.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(fst_[a-z_0-9]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(F.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(F.EXPORTED)


def test_version_and_error_string():
    assert P.fst_version().startswith("fst-gb300")
    with pytest.raises(F.FSTError) as ei:
        F.fst_emu_plan_op(0, 0.1, -1, 1e-6)
    assert ei.value.status == F.FST_EINVAL
    assert "N" in P.fst_last_error()


@pytest.mark.parametrize("args", [(10, 0.0, -1, 1e-6), (10, 0.5, -1, 1e-6), (10, 0.1, -1, 0.0),
                                  (10, 0.1, -1, 0.5), (10, 0.1, 11, 1e-6), (1 << 24, 0.1, -1, 1e-6)])
def test_invalid_arguments(args):
    with pytest.raises(F.FSTError) as ei:
        F.fst_emu_plan_op(*args)
    assert ei.value.status == F.FST_EINVAL


def test_tikhonov_needs_alpha():
    with pytest.raises(F.FSTError):
        F.fst_emu_plan_op(100, 0.1, -1, 1e-6, F.FST_OP_TIKHONOV, 0.0)


@pytest.mark.parametrize("N", [1, 2, 3, 8, 9, 64, 101])
@pytest.mark.parametrize("W", [0.07, 0.25, 0.4])
def test_reduced_tridiagonal_split(N, W):
    # the parity split reproduces the spectrum of Slepian's full tridiagonal matrix,
    # with the l-th largest eigenvalue in parity l mod 2 at position l div 2
    d, e = O.slepian_tridiagonal(N, W)
    full = np.sort(sla.eigvalsh_tridiagonal(d, e) if N > 1 else d)[::-1]
    parts = []
    for p in (0, 1):
        dd, ee = P.fst_reduced_tridiagonal(N, W, p)
        if dd.size == 0:
            parts.append(np.zeros(0))
            continue
        ev = sla.eigvalsh_tridiagonal(dd, ee) if dd.size > 1 else dd.copy()
        parts.append(np.sort(ev)[::-1])
    assert parts[0].size == (N + 1) // 2 and parts[1].size == N // 2
    for l in range(N):
        got = parts[l % 2][l // 2]
        assert abs(got - full[l]) <= 1e-9 * max(1.0, abs(full).max())


EMU_CASES = [(1, 0.3, 1e-6), (2, 0.3, 1e-6), (5, 0.2, 1e-3), (64, 0.2, 1e-3), (257, 0.11, 1e-6),
             (1000, 1 / 64, 1e-8), (4096, 1 / 16, 1e-6), (9000, 0.05, 1e-6), (20000, 0.2, 1e-4),
             # W = 1/4: the tridiagonal's diagonal vanishes (cos 2 pi W = 0); W > 1/4: it is negative
             (3001, 0.25, 1e-6), (777, 0.45, 1e-8)]


@pytest.mark.parametrize("N,W,eps", EMU_CASES)
def test_emulated_plan_matches_oracle(N, W, eps):
    p = P.Plan(N, W, eps=eps, emulate=True)
    op = O.make_plan(N, W, None, eps)
    ex = p.export()
    assert p.K == op.K and p.M == op.M
    assert p.r == op.r
    assert np.array_equal(ex["idx"], op.idx)
    assert np.max(np.abs(ex["lam"] - op.lam), initial=0) < 1e-12
    assert np.max(np.abs(ex["D"] - op.D), initial=0) < 1e-12
    if p.r:
        assert np.max(np.abs(ex["S_T"] - op.S_T)) < 1e-10


@pytest.mark.parametrize("N,W,eps", EMU_CASES)
def test_emulated_projection_matches_oracle(N, W, eps):
    p = P.Plan(N, W, eps=eps, emulate=True)
    op = O.make_plan(N, W, None, eps)
    rng = np.random.default_rng(N)
    y = rng.standard_normal((3, N))        # odd batch: last pair has one signal
    ref = O.fast_project(op, y.T).T
    nrm = np.linalg.norm(y, axis=1)
    out64 = p.project(y)
    assert np.all(np.linalg.norm(out64 - ref, axis=1) <= 1e-12 * nrm)
    out32 = p.project(y.astype(np.float32))
    assert np.all(np.linalg.norm(out32 - ref, axis=1) <= 1e-6 * nrm)
    yc = (rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N)))
    refc = O.fast_project(op, yc.T).T
    nc = np.linalg.norm(yc, axis=1)
    assert np.all(np.linalg.norm(p.project(yc) - refc, axis=1) <= 1e-12 * nc)
    assert np.all(np.linalg.norm(p.project(yc.astype(np.complex64)) - refc, axis=1) <= 1e-6 * nc)


def test_emulated_against_exact_projection():
    # end to end: library (emulated) vs the plain definition S_K S_K^T y, Corollary 2 bound
    N, W, eps = 1500, 0.2, 1e-6
    p = P.Plan(N, W, eps=eps, emulate=True)
    y = np.random.default_rng(9).standard_normal((2, N))
    ex = O.exact_project(N, W, p.K, y.T).T
    out = p.project(y)
    assert np.all(np.linalg.norm(out - ex, axis=1) <= eps * np.linalg.norm(y, axis=1))


@pytest.mark.parametrize("op,alpha,tolmul", [("pinv", 0.0, 3), ("tikhonov", 1e-3, 1)])
def test_emulated_other_operators(op, alpha, tolmul):
    N, W, eps = 400, 0.2, 1e-4
    p = P.Plan(N, W, eps=eps, op=op, alpha=alpha, emulate=True)
    oop = O.make_plan(N, W, None, eps, op=op, alpha=alpha)
    assert p.r == oop.r
    y = np.random.default_rng(2).standard_normal((2, N))
    ref = O.fast_apply(oop, y.T).T
    assert np.max(np.abs(p.project(y) - ref)) < 1e-11
    exact = O.exact_operator_dense(N, W, p.K, op, alpha)
    assert np.all(np.linalg.norm(p.project(y) - (exact @ y.T).T, axis=1)
                  <= tolmul * eps * np.linalg.norm(y, axis=1) + 1e-10)


def test_emulated_apply_prolate_and_degenerate_K():
    N, W = 300, 0.1
    y = np.random.default_rng(4).standard_normal((2, N))
    p = P.Plan(N, W, eps=1e-6, emulate=True)
    assert np.max(np.abs(p.apply_prolate(y) - (O.prolate_matrix(N, W) @ y.T).T)) < 1e-12
    for K in (0, N):
        pk = P.Plan(N, W, K=K, eps=1e-6, emulate=True)
        want = np.zeros_like(y) if K == 0 else y
        assert np.all(np.linalg.norm(pk.project(y) - want, axis=1) <= 1e-6 * np.linalg.norm(y, axis=1) + 1e-12)


def test_emulated_strided_and_inplace():
    N, W = 777, 0.15
    p = P.Plan(N, W, eps=1e-6, emulate=True)
    op = O.make_plan(N, W, None, 1e-6)
    rng = np.random.default_rng(5)
    big = rng.standard_normal((3, N + 13))
    out = np.zeros_like(big)
    F.fst_project(p.h, big.ctypes.data, out.ctypes.data, 3, N + 13, F.FST_F64)
    ref = O.fast_project(op, big[:, :N].T).T
    assert np.max(np.abs(out[:, :N] - ref)) < 1e-12
    assert np.all(out[:, N:] == 0)
    y = rng.standard_normal((2, N))
    ref = O.fast_project(op, y.T).T
    F.fst_project(p.h, y.ctypes.data, y.ctypes.data, 2, N, F.FST_F64)
    assert np.max(np.abs(y - ref)) < 1e-12


def test_emulated_bad_apply_arguments():
    p = P.Plan(50, 0.1, eps=1e-6, emulate=True)
    y = np.zeros((2, 50))
    with pytest.raises(F.FSTError):
        F.fst_project(p.h, y.ctypes.data, y.ctypes.data, 2, 10, F.FST_F64)   # ld < N
    with pytest.raises(F.FSTError):
        F.fst_project(p.h, 0, y.ctypes.data, 2, 50, F.FST_F64)
    with pytest.raises(F.FSTError):
        F.fst_project(p.h, y.ctypes.data, y.ctypes.data, 2, 50, 9)
    F.fst_project(p.h, y.ctypes.data, y.ctypes.data, 0, 50, F.FST_F64)      # batch 0: no-op


def test_repeatability_bit_for_bit():
    N, W = 20000, 0.25
    p = P.Plan(N, W, eps=1e-6, emulate=True)
    y = np.random.default_rng(6).standard_normal((4, N)).astype(np.float32)
    a = p.project(y)
    b = p.project(y)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- fast coefficient vector

def test_adi_shifts_match_scipy():
    from oracle import thm1 as T
    for N, r in [(1, 2), (64, 7), (4096, 18), (65536, 16), (1 << 22, 38)]:
        got = F.fst_adi_shifts(N, r)
        ref = T.adi_shifts(N, r)
        assert np.max(np.abs(got - ref) / ref) < 1e-6


@pytest.mark.parametrize("N,W,eps", [(256, 1 / 16, 1e-6), (1024, 0.2, 1e-4), (4096, 1 / 16, 1e-6),
                                     (32768, 0.25, 1e-8), (2, 0.3, 1e-3)])
def test_emulated_coeffs_match_oracle(N, W, eps):
    from oracle import thm1 as T
    p = P.Plan(N, W, eps=eps, emulate=True)
    t = T.thm1(N, W, eps)
    op = O.make_plan(N, W, None, eps)
    info = F.fst_coeffs_info(p.h)
    assert (info["rH"], info["rA"], info["rB"], info["r1"]) == (t.r_H, t.r_A, t.r_B, t.r1)
    assert info["Kprime"] == t.nF + t.r1 + op.r
    rng = np.random.default_rng(N)
    y = rng.standard_normal((3, N))
    ref = T.coeffs(t, op, y.T).T
    nrm = np.linalg.norm(y, axis=1)[:, None]
    assert np.all(np.abs(p.coeffs(y) - ref) <= 1e-12 * nrm)
    assert np.all(np.abs(p.coeffs(y.astype(np.float32)) - ref) <= 1e-6 * nrm)
    yc = rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N))
    refc = T.coeffs(t, op, yc.T).T
    assert np.all(np.abs(p.coeffs(yc) - refc) <= 1e-12 * np.linalg.norm(yc, axis=1)[:, None])


def test_emulated_coeffs_expand_to_projection():
    from oracle import thm1 as T
    N, W, eps = 512, 0.2, 1e-6
    p = P.Plan(N, W, eps=eps, emulate=True)
    t = T.thm1(N, W, eps)
    op = O.make_plan(N, W, None, eps)
    y = np.random.default_rng(3).standard_normal(N)
    c = p.coeffs(y)[0]
    back = T.expand(t, op, c)
    assert np.linalg.norm(back - O.exact_project(N, W, p.K, y)) <= 2 * eps * np.linalg.norm(y)


@pytest.mark.parametrize("N,W,eps", [(256, 0.2, 1e-6), (1024, 1 / 16, 1e-8)])
def test_emulated_expand_matches_dense_T1(N, W, eps):
    # T1 c of the library (matrix-free, emulated kernels) against the oracle's dense
    # T1 = [F  L1  U1] on random complex coefficient vectors
    from oracle import thm1 as T
    p = P.Plan(N, W, eps=eps, emulate=True)
    t = T.thm1(N, W, eps)
    op = O.make_plan(N, W, None, eps)
    Kp = F.fst_coeffs_info(p.h)["Kprime"]
    rng = np.random.default_rng(N + 1)
    c = rng.standard_normal((2, Kp)) + 1j * rng.standard_normal((2, Kp))
    ref = np.stack([T.expand(t, op, ci) for ci in c])
    scale = np.abs(ref).max()
    assert np.max(np.abs(p.expand(c) - ref)) <= 1e-12 * scale
    assert np.max(np.abs(p.expand(c.astype(np.complex64)) - ref)) <= 2e-5 * scale


def test_emulated_expand_of_coeffs_is_the_projection():
    # T1 T2^* y is within 2 eps ||y|| of S_K S_K^T y (Section 1.3), through both entry points
    N, W, eps = 512, 0.2, 1e-6
    p = P.Plan(N, W, eps=eps, emulate=True)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((2, N))
    exact = O.exact_project(N, W, p.K, y.T).T
    back = p.expand(p.coeffs(y))
    nrm = np.linalg.norm(y, axis=1)
    assert np.all(np.linalg.norm(back - exact, axis=1) <= 2 * eps * nrm)
    back32 = p.expand(p.coeffs(y.astype(np.float32)))
    assert np.all(np.linalg.norm(back32 - exact, axis=1) <= 2 * eps * nrm + 1e-5 * nrm)
    yc = y + 1j * rng.standard_normal((2, N))
    exc = O.exact_project(N, W, p.K, yc.T).T
    assert np.all(np.linalg.norm(p.expand(p.coeffs(yc)) - exc, axis=1) <= 2 * eps * np.linalg.norm(yc, axis=1))


def test_emulated_coeffs_and_expand_across_launch_groups(monkeypatch):
    # 1 MiB launch groups of 8 (N = 8192, FP64): 18 real signals are 9 pairs, two groups for the
    # coefficients, and 18 coefficient rows, three groups for the expansion; rows from every group
    # against the oracle
    from oracle import thm1 as T
    monkeypatch.setenv("FST_CHUNK_MB", "1")
    N, W, eps = 8192, 1 / 16, 1e-6
    p = P.Plan(N, W, eps=eps, emulate=True)
    t = T.thm1(N, W, eps)
    op = O.make_plan(N, W, None, eps)
    rng = np.random.default_rng(11)
    y = rng.standard_normal((18, N))
    c = p.coeffs(y)
    rows = [0, 15, 16, 17]
    ref = T.coeffs(t, op, y[rows].T).T
    nrm = np.linalg.norm(y[rows], axis=1)[:, None]
    # FP64 rounding of the ADI column sums grows with N: ~2e-12 ||y|| at N = 8192 (the GPU FP64
    # coefficient test uses the same 1e-11 bound)
    assert np.all(np.abs(c[rows] - ref) <= 1e-11 * nrm)
    back = p.expand(c)
    dense = np.stack([T.expand(t, op, c[i]) for i in rows])
    assert np.max(np.abs(back[rows] - dense)) <= 1e-11 * np.abs(dense).max()


def test_expand_argument_errors():
    p = P.Plan(128, 0.1, eps=1e-6, emulate=True)
    Kp = F.fst_coeffs_info(p.h)["Kprime"]
    c = np.zeros((1, Kp), np.complex128)
    out = np.zeros((1, 128), np.complex128)
    with pytest.raises(F.FSTError) as ei:
        F.fst_expand(p.h, c.ctypes.data, out.ctypes.data, 1, F.FST_F64)
    assert ei.value.status == F.FST_EINVAL
    with pytest.raises(F.FSTError) as ei:
        F.fst_expand(p.h, 0, out.ctypes.data, 1, F.FST_C128)
    assert ei.value.status == F.FST_EINVAL
    F.fst_expand(p.h, c.ctypes.data, out.ctypes.data, 0, F.FST_C128)     # batch 0: no-op
    q = P.Plan(100, 0.1, eps=1e-6, emulate=True)
    with pytest.raises(F.FSTError) as ei:
        q.expand(np.zeros((1, 10), np.complex128))
    assert ei.value.status == F.FST_EUNSUPPORTED


def test_coeffs_need_power_of_two_and_projection():
    p = P.Plan(100, 0.1, eps=1e-6, emulate=True)
    with pytest.raises(F.FSTError) as ei:
        p.coeffs(np.zeros((1, 100)))
    assert ei.value.status == F.FST_EUNSUPPORTED
    q = P.Plan(128, 0.1, eps=1e-6, op="pinv", emulate=True)
    with pytest.raises(F.FSTError) as ei:
        q.coeffs(np.zeros((1, 128)))
    assert ei.value.status == F.FST_EINVAL


# ---------------------------------------------------------------- ragged batches

def test_emulated_plan_many_and_ragged_projection():
    from paper_1611_04950_gb300 import workloads
    params = workloads.ragged_params(10, seed=3, n_lo=100, n_hi=20000)
    ps = F.PlanSet(params, emulate=True)
    rng = np.random.default_rng(0)
    ys = [rng.standard_normal(N) for (N, W, e) in params]
    plans = [O.make_plan(N, W, None, e) for (N, W, e) in params]
    for i, ((N, W, e), op) in enumerate(zip(params, plans)):
        ex = F.fst_plan_export(ps.h[i], N)
        assert ps.info(i)["r"] == op.r
        assert np.array_equal(ex["idx"], op.idx)
        assert np.max(np.abs(ex["S_T"] - op.S_T)) < 1e-9
    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-6)):
        outs = ps.project([y.astype(dt) for y in ys])
        for y, o, op in zip(ys, outs, plans):
            assert np.linalg.norm(o - O.fast_project(op, y)) <= tol * np.linalg.norm(y)


def test_emulated_ragged_small_signals_one_length_class():
    # five single-CTA signals of one FFT length (M = 4096) with their own plans and ranks,
    # against the oracle, and the in-place call equal to the out-of-place one
    params = [(1100, 0.05, 1e-3), (1500, 0.2, 1e-8), (2048, 0.1, 1e-6), (1025, 0.3, 1e-4), (1800, 0.02, 1e-6)]
    ps = F.PlanSet(params, emulate=True)
    rng = np.random.default_rng(4)
    ys = [rng.standard_normal(N) for (N, W, e) in params]
    plans = [O.make_plan(N, W, None, e) for (N, W, e) in params]
    assert len({ps.info(i)["r"] for i in range(len(params))}) > 1
    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-6)):
        outs = ps.project([y.astype(dt) for y in ys])
        for y, o, op in zip(ys, outs, plans):
            assert np.linalg.norm(o - O.fast_project(op, y)) <= tol * np.linalg.norm(y)
        io = [y.astype(dt) for y in ys]
        ps.project(io, io)                      # in place
        for a, b in zip(outs, io):
            assert np.array_equal(a, b)


def test_plan_many_rejects_bad_arguments():
    with pytest.raises(F.FSTError):
        F.fst_plan_many([100, 0], [0.1, 0.1], [1e-6, 1e-6], emulate=True)
