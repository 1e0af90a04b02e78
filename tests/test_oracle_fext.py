"""Pins of the oracle's fast truncated pseudoinverse (Corollary 3) on the Fourier-extension
problem of Section 4.2 (synthetic stand-in for its random test function, see workloads):
  * Corollary 3: the fast pseudoinverse is within 3 eps of the rank-K truncated pseudoinverse
    of B (dense eigensolve) applied to the right-hand side;
  * Section 4.2: for M >= 448 the 2M+1-term Fourier extension (T = 1.5, eigenvalues below
    1e-4 truncated, fast pseudoinverse at eps = 1e-5) has a relative RMS error at least 10
    times lower than the 2M+1-term truncated Fourier series.
"""
import numpy as np
import pytest

from oracle import fst_oracle as O
from paper_1611_04950_gb300 import workloads


def synth(coef, t, period_half):
    """sum_m coef[m] exp(j pi m t / period_half) / sqrt(2 period_half), m = -M..M."""
    M = (len(coef) - 1) // 2
    m = np.arange(-M, M + 1)
    return (np.exp(1j * np.pi * np.outer(t, m) / period_half) @ coef) / np.sqrt(2.0 * period_half)


def rel_rms(x, ref, t):
    return np.sqrt(np.trapezoid(np.abs(x - ref) ** 2, t) / np.trapezoid(np.abs(ref) ** 2, t))


def threshold_K(N, W, lam_min=1e-4):
    """Number of eigenvalues of B_{N,W} above lam_min (the paper's truncation in Section 4.2)."""
    lam, _ = O.dpss_dense(N, W)
    return int(np.sum(lam > lam_min))


@pytest.mark.parametrize("M", [448, 512])
def test_fourier_extension_pinv(M):
    fe = workloads.fourier_extension(M)
    K = threshold_K(fe.N, fe.W)
    plan = O.make_plan(fe.N, fe.W, K, 1e-5, op=O.OP_PINV)
    g_fast = O.fast_apply(plan, fe.yhat)
    lam, S = O.dpss_dense(fe.N, fe.W)
    SK = S[:, :K]
    g_exact = (SK / lam[:K]) @ (SK.T @ fe.yhat)
    # Corollary 3: || B_K^dagger - fast || <= 3 eps
    assert np.linalg.norm(g_fast - g_exact) <= 3 * 1e-5 * np.linalg.norm(fe.yhat)
    t = np.linspace(-1.0, 1.0, 4097)
    ft = fe.f(t)
    e_ext = rel_rms(synth(g_fast, t, fe.T), ft, t)
    e_ser = rel_rms(synth(fe.fhat, t, 1.0), ft, t)
    assert e_ext * 10 <= e_ser, (e_ext, e_ser)


def test_fourier_extension_needs_the_threshold_truncation():
    # planted mistake: the rank-round(2NW) truncation loses the advantage (the paper truncates
    # the eigenvalues below 1e-4, not at K = 2NW)
    fe = workloads.fourier_extension(448)
    K = O.default_K(fe.N, fe.W)
    g = O.fast_apply(O.make_plan(fe.N, fe.W, K, 1e-5, op=O.OP_PINV), fe.yhat)
    t = np.linspace(-1.0, 1.0, 4097)
    ft = fe.f(t)
    assert rel_rms(synth(g, t, fe.T), ft, t) * 10 > rel_rms(synth(fe.fhat, t, 1.0), ft, t)
