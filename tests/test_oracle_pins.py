"""Pins for the FP64 oracle against facts the paper and the mathematics fix,
independent of the oracle's own formulas: dense eigensolves of B, the O(N^2)
Toeplitz sum, closed forms (eigenvectors map to themselves or to zero), the
Corollary 1 and 2 bounds, the trace identity and the W <-> 1/2 - W symmetry."""
import functools
import math

import numpy as np
import pytest

from oracle import fst_oracle as O


@functools.lru_cache(maxsize=None)
def dense(N, W):
    return O.dpss_dense(N, W)


# --- Slepian's tridiagonal matrix commutes with B (reading: it is not written in the paper)
@pytest.mark.parametrize("N,W", [(16, 0.1), (33, 0.25), (128, 0.37), (257, 1 / 64)])
def test_tridiagonal_commutes_with_prolate(N, W):
    d, e = O.slepian_tridiagonal(N, W)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    B = O.prolate_matrix(N, W)
    rel = np.linalg.norm(T @ B - B @ T) / (np.linalg.norm(T) * np.linalg.norm(B))
    assert rel < 1e-13


# --- Section 1.2: S contains the eigenvectors of B, eigenvalues in (0,1), descending
@pytest.mark.parametrize("N,W", [(256, 1 / 8), (301, 0.3), (200, 1 / 64)])
def test_dpss_match_dense_eigensolve(N, W):
    lam_d, S_d = dense(N, W)
    S = O.dpss_window(N, W, 0, N - 1)
    lam = O.rayleigh_eigenvalues(S, W)
    # eigenvalues of B agree with the dense solve (Rayleigh quotients of tridiagonal vectors)
    assert np.max(np.abs(lam - lam_d)) < 1e-12
    assert np.all(lam_d > -1e-13) and np.all(lam_d < 1 + 1e-13)
    # vectors agree up to sign wherever the dense eigenvalue is well separated
    gaps = np.minimum(np.abs(np.diff(lam_d, prepend=np.inf)), np.abs(np.diff(lam_d, append=-np.inf)))
    ok = gaps > 1e-6
    assert ok.sum() > 10
    dots = np.abs(np.einsum("ij,ij->j", S, S_d))
    assert np.all(dots[ok] > 1 - 1e-9)


def test_eigenvalues_strictly_decreasing_in_transition():
    N, W = 1024, 1 / 16
    K = O.default_K(N, W)
    S = O.dpss_window(N, W, K - 30, K + 30)
    lam = O.rayleigh_eigenvalues(S, W)
    # strictly decreasing wherever FP64 resolves lambda away from 0 and 1
    mid = (lam > 1e-10) & (lam < 1 - 1e-10)
    assert mid.sum() > 10
    assert np.all(np.diff(lam[mid]) < 0)
    assert lam[0] > 1 - 1e-8 and lam[-1] < 1e-8


# --- Eq. dpssorth / dpssnorm: the Slepian basis is orthonormal
def test_orthonormal_window():
    S = O.dpss_window(2000, 0.2, 700, 900)
    assert np.max(np.abs(S.T @ S - np.eye(S.shape[1]))) < 1e-12


# --- trace(B) = N * 2W = sum of all eigenvalues (diag of the prolate matrix is 2W)
@pytest.mark.parametrize("N,W", [(300, 0.11), (512, 0.25)])
def test_trace_identity(N, W):
    S = O.dpss_window(N, W, 0, N - 1)
    lam = O.rayleigh_eigenvalues(S, W)
    assert abs(lam.sum() - 2 * N * W) < 1e-10


# --- Section 1.2, Figure 1 discussion: lambda_{N,1/2-W}^(l) = 1 - lambda_{N,W}^(N-1-l)
def test_eigenvalue_symmetry_W_half_minus_W():
    N, W = 240, 0.13
    lam1, _ = dense(N, W)
    lam2, _ = dense(N, 0.5 - W)
    assert np.max(np.abs(lam2 - (1 - lam1[::-1]))) < 1e-12


# --- centro-symmetry: J s^(l) = (-1)^l s^(l)
def test_parity_of_slepian_vectors():
    N, W = 501, 0.07
    S = O.dpss_window(N, W, 0, 80)
    for l in range(S.shape[1]):
        assert np.max(np.abs(S[::-1, l] - (-1) ** l * S[:, l])) < 1e-12


# --- B y by FFT (Section 4.1's zero-padded convolution) against the O(N^2) Toeplitz sum
@pytest.mark.parametrize("N", [1, 2, 3, 17, 100, 1000, 2049])
@pytest.mark.parametrize("W", [1 / 64, 0.25, 0.41])
def test_apply_prolate_fft_vs_direct(N, W):
    rng = np.random.default_rng(N)
    y = rng.standard_normal(N)
    ref = O.apply_prolate_direct(y, W)
    for M in {O.fft_length(N), 2 * N - 1 if N > 1 else 1, 3 * N + 5}:
        got = O.apply_prolate(y, W, M)
        assert np.linalg.norm(got - ref) <= 1e-13 * max(1.0, np.linalg.norm(y)) * math.sqrt(N)


def test_apply_prolate_complex_and_batch():
    N, W = 300, 0.2
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    got = O.apply_prolate(Y, W)
    B = O.prolate_matrix(N, W)
    assert np.max(np.abs(got - B @ Y)) < 1e-12


# --- Corollary 1: transition count below the bound; close to Eq. (asymptotic);
#     equal to the count from a dense eigensolve
@pytest.mark.parametrize("N,W,eps", [(512, 0.25, 1e-3), (1024, 1 / 16, 1e-6), (2048, 0.1, 1e-9),
                                     (777, 0.3, 1e-12)])
def test_transition_count(N, W, eps):
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    lam_d, _ = dense(N, W)
    dense_count = int(np.sum((lam_d > eps) & (lam_d < 1 - eps)))
    assert plan.r == dense_count
    assert plan.r <= O.cor1_bound(N, eps)
    assert abs(plan.r - O.asymptotic_transition(N, eps)) < 0.5 * O.asymptotic_transition(N, eps) + 6


def test_transition_count_tiny_workload():
    # N=4096, W=1/16, eps=1e-6: the window search and the Rayleigh quotients give r=24,
    # against 23.3 from Eq. (asymptotic) and 337.5 from Corollary 1
    plan = O.make_plan(4096, 1 / 16, 512, 1e-6)
    assert plan.r == 24
    assert 337 < O.cor1_bound(4096, 1e-6) < 338
    lo, hi = plan.window
    assert lo < plan.idx.min() and hi > plan.idx.max()


# --- Corollary 2 as a matrix statement: || S_K S_K^* - (B + U1 U2^*) ||_2 <= eps
@pytest.mark.parametrize("N,W,eps", [(400, 1 / 8, 1e-3), (512, 0.25, 1e-6), (640, 0.05, 1e-9)])
def test_cor2_operator_bound(N, W, eps):
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    Pex = O.exact_operator_dense(N, W, K)
    Pfast = O.prolate_matrix(N, W) + plan.S_T @ np.diag(plan.D) @ plan.S_T.T
    err = np.linalg.norm(Pex - Pfast, 2)
    assert err <= eps
    # and the correction is needed: without it the error is O(1)
    assert np.linalg.norm(Pex - O.prolate_matrix(N, W), 2) > 0.1


# --- Corollaries 3 and 4 (next rows): same machinery with a different D
def test_cor3_pinv_bound():
    N, W, eps = 400, 0.2, 1e-4
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps, op=O.OP_PINV)
    ex = O.exact_operator_dense(N, W, K, O.OP_PINV)
    fast = O.prolate_matrix(N, W) + plan.S_T @ np.diag(plan.D) @ plan.S_T.T
    assert np.linalg.norm(ex - fast, 2) <= 3 * eps


def test_cor4_tikhonov_bound():
    N, W, eps, alpha = 400, 0.2, 1e-4, 1e-3
    plan = O.make_plan(N, W, None, eps, op=O.OP_TIKHONOV, alpha=alpha)
    ex = O.exact_operator_dense(N, W, 0, O.OP_TIKHONOV, alpha)
    fast = O.prolate_matrix(N, W) / (1 + alpha) + plan.S_T @ np.diag(plan.D) @ plan.S_T.T
    assert np.linalg.norm(ex - fast, 2) <= eps


# --- the fast projection on vectors (Section 1.3): error <= eps ||y||
@pytest.mark.parametrize("N,W,eps", [(64, 0.2, 1e-3), (257, 0.11, 1e-6), (1000, 1 / 64, 1e-8),
                                     (2048, 0.25, 1e-12), (1500, 0.45, 1e-6)])
def test_fast_projection_vs_exact(N, W, eps):
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    rng = np.random.default_rng(11)
    Y = rng.standard_normal((N, 4))
    ex = O.exact_project(N, W, K, Y)
    got = O.fast_project(plan, Y)
    for j in range(Y.shape[1]):
        assert np.linalg.norm(got[:, j] - ex[:, j]) <= eps * np.linalg.norm(Y[:, j]) + 1e-13 * math.sqrt(N)


# --- closed forms: Slepian vectors with l < K are kept, the others removed
def test_projection_of_slepian_vectors():
    N, W, eps = 700, 0.15, 1e-9
    K = O.default_K(N, W)
    plan = O.make_plan(N, W, K, eps)
    ls = [0, K // 2, K - 3, K - 1, K, K + 1, K + 5, N - 1]
    lam_d, S_d = dense(N, W)
    for l in ls:
        s = S_d[:, l]
        got = O.fast_project(plan, s)
        want = s if l < K else np.zeros(N)
        assert np.linalg.norm(got - want) <= eps + 1e-12


# --- degenerate K: K = 0 (projection is 0) and K = N (identity)
@pytest.mark.parametrize("K", [0, 60])
def test_degenerate_K(K):
    N, W, eps = 60, 0.05, 1e-6
    plan = O.make_plan(N, W, K, eps)
    y = np.random.default_rng(3).standard_normal(N)
    want = np.zeros(N) if K == 0 else y
    assert np.linalg.norm(O.fast_project(plan, y) - want) <= eps * np.linalg.norm(y) + 1e-12


def test_small_N_edge_cases():
    for N in (1, 2, 3, 5):
        W = 0.3
        K = O.default_K(N, W)
        plan = O.make_plan(N, W, K, 1e-6)
        y = np.arange(1.0, N + 1)
        ex = O.exact_project(N, W, K, y)
        assert np.linalg.norm(O.fast_project(plan, y) - ex) <= 1e-6 * np.linalg.norm(y) + 1e-13


def test_exact_reference_above_dense_limit_agrees():
    # the eps_ref = 1e-13 reference used above N = 8192 agrees with the dense one below it
    N, W = 1200, 0.19
    K = O.default_K(N, W)
    y = np.random.default_rng(5).standard_normal(N)
    ref = O.fast_project(O.make_plan(N, W, K, O.EPS_REF), y)
    ex = O.exact_project(N, W, K, y)
    assert np.linalg.norm(ref - ex) <= 1e-12 * np.linalg.norm(y)


def test_sign_convention():
    N, W = 128, 0.1
    S = O.dpss_window(N, W, 0, 20)
    n = np.arange(N)
    for l in range(S.shape[1]):
        if l % 2 == 0:
            assert S[:, l].sum() > 0
        else:
            assert np.dot(N - 1 - 2 * n, S[:, l]) > 0
