"""Planted mistakes in the oracle (on the CPU, through monkeypatch) must be caught by
the pins: a dropped term, a wrong sign, an off-by-one index, a transposed operand."""
import math

import numpy as np
import pytest

from oracle import fst_oracle as O


def cor2_error(N=400, W=1 / 8, eps=1e-3):
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    Pex = O.exact_operator_dense(N, W, K)
    Pfast = O.prolate_matrix(N, W) + plan.S_T @ np.diag(plan.D) @ plan.S_T.T
    return np.linalg.norm(Pex - Pfast, 2), eps


def fast_vs_exact_error(N=300, W=0.11, eps=1e-6):
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    y = np.random.default_rng(1).standard_normal(N)
    return np.linalg.norm(O.fast_project(plan, y) - O.exact_project(N, W, K, y)) / np.linalg.norm(y), eps


def test_unmutated_passes():
    e, tol = cor2_error()
    assert e <= tol
    e, tol = fast_vs_exact_error()
    assert e <= tol


def test_wrong_sign_of_D_is_caught(monkeypatch):
    orig = O._D_of
    monkeypatch.setattr(O, "_D_of", lambda *a: -orig(*a))
    e, tol = cor2_error()
    assert e > 10 * tol


def test_dropped_one_minus_lambda_is_caught(monkeypatch):
    # D = -lambda everywhere (forgets the 1 on l < K)
    monkeypatch.setattr(O, "_D_of", lambda lam, l, K, op, alpha: -lam)
    e, tol = fast_vs_exact_error()
    assert e > 10 * tol


def test_off_by_one_in_K_is_caught(monkeypatch):
    orig = O._D_of
    monkeypatch.setattr(O, "_D_of", lambda lam, l, K, op, alpha: orig(lam, l, K + 1, op, alpha))
    orig_T = O._in_T
    monkeypatch.setattr(O, "_in_T", lambda lam, l, K, eps, op, alpha: orig_T(lam, l, K + 1, eps, op, alpha))
    e, tol = fast_vs_exact_error()
    assert e > 10 * tol


def test_missing_cos_in_tridiagonal_is_caught():
    N, W = 64, 0.2
    n = np.arange(N, dtype=np.float64)
    d = ((N - 1) / 2.0 - n) ** 2          # cos(2 pi W) dropped
    e = n[1:] * (N - n[1:]) / 2.0
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    B = O.prolate_matrix(N, W)
    rel = np.linalg.norm(T @ B - B @ T) / (np.linalg.norm(T) * np.linalg.norm(B))
    assert rel > 1e-3


def test_one_sided_sinc_embedding_is_caught(monkeypatch):
    def bad_spectrum(N, W, M):
        c = np.zeros(M)
        c[:N] = O.sinc_row(N, W)      # the mirrored half c[M-k] is missing
        return np.fft.fft(c).real
    monkeypatch.setattr(O, "sinc_spectrum", bad_spectrum)
    y = np.random.default_rng(2).standard_normal(200)
    err = np.linalg.norm(O.apply_prolate(y, 0.2) - O.apply_prolate_direct(y, 0.2))
    assert err > 1e-3 * np.linalg.norm(y)


def test_transposed_correction_is_caught(monkeypatch):
    # ascending instead of descending eigen-index (l <-> N-1-l) picks the wrong vectors
    def bad_window(N, W, lo, hi):
        import scipy.linalg as sla
        d, e = O.slepian_tridiagonal(N, W)
        _, V = sla.eigh_tridiagonal(d, e, select="i", select_range=(lo, hi), lapack_driver="stebz")
        return V / np.linalg.norm(V, axis=0, keepdims=True)
    monkeypatch.setattr(O, "dpss_window", bad_window)
    e, tol = fast_vs_exact_error()
    assert e > 10 * tol


def test_wrong_fft_length_rule_is_caught():
    # an FFT shorter than 2N-1 wraps the convolution around
    N, W = 256, 0.2
    y = np.random.default_rng(3).standard_normal(N)
    ref = O.apply_prolate_direct(y, W)
    M = N  # too short
    C = np.fft.fft(np.concatenate([O.sinc_row(N, W)[: M // 2 + 1],
                                   O.sinc_row(N, W)[1: M // 2][::-1]])).real
    got = np.fft.ifft(np.fft.fft(y, n=M) * C)[:N].real
    assert np.linalg.norm(got - ref) > 1e-3 * math.sqrt(N)
