"""Pins for the Theorem 1 / fast factorization oracle (oracle/thm1.py): every identity
of the constructive proof checked on dense matrices, the error budgets of each low-rank
piece, Theorem 1 and the 2 eps bound of the fast factorization, the rank formulas, the
matrix-free coefficients against the dense T2^* y, and planted mistakes."""
import math

import numpy as np
import pytest

from oracle import fst_oracle as O
from oracle import thm1 as T

CASES = [(64, 0.2, 1e-3), (256, 1 / 16, 1e-6), (300, 0.25, 1e-8), (512, 0.31, 1e-6), (128, 0.05, 1e-12),
         (100, 0.4, 1e-4)]


def test_nearest_odd_reading():
    assert T.nearest_odd_2NW(4096, 1 / 16) == 513     # 2NW = 512 even: tie rounds up
    assert T.nearest_odd_2NW(100, 0.016) == 3         # 2NW = 3.2
    assert T.nearest_odd_2NW(100, 0.0245) == 5        # 2NW = 4.9
    for N, W in [(77, 0.13), (1000, 0.3), (64, 0.2)]:
        odd = T.nearest_odd_2NW(N, W)
        assert odd % 2 == 1 and abs(odd - 2 * N * W) <= 1


@pytest.mark.parametrize("N,W", [(64, 0.2), (101, 0.07), (256, 0.31)])
def test_FFstar_is_dirichlet(N, W):
    F = T.partial_fourier_matrix(N, W)
    assert np.max(np.abs(F @ F.conj().T - T.dirichlet_FFstar(N, W))) < 1e-12
    # orthonormal columns, 2NW' of them
    assert F.shape[1] == T.nearest_odd_2NW(N, W)
    assert np.max(np.abs(F.conj().T @ F - np.eye(F.shape[1]))) < 1e-12


@pytest.mark.parametrize("N,W", [(64, 0.2), (99, 0.07), (256, 0.31)])
def test_eq_BA0_and_A0A1(N, W):
    t = T.thm1(N, W, 1e-6)
    B = O.prolate_matrix(N, W)
    F = T.partial_fourier_matrix(N, W)
    DA = np.diag(T.phase_A(t))
    DB = np.diag(T.phase_B(t))
    A0, B0 = T.A0_matrix(N), T.B0_matrix(N, W)
    rhs = (DA @ A0 @ DA.conj().T - DA.conj().T @ A0 @ DA) / 2j + (DB @ B0 @ DB.conj().T + DB.conj().T @ B0 @ DB) / 2
    assert np.max(np.abs((B - F @ F.conj().T) - rhs)) < 1e-12
    H = T.hilbert(N)
    J = np.eye(N)[::-1]
    assert np.max(np.abs(A0 - ((H @ J - J @ H) / math.pi + T.A1_matrix(N)))) < 1e-12
    # H solves the Lyapunov equation A X + X A = 1 1^T with A = diag(n + 1/2)
    A = np.diag(np.arange(N) + 0.5)
    assert np.max(np.abs(A @ H + H @ A - np.ones((N, N)))) < 1e-12


@pytest.mark.parametrize("N,W,eps", CASES)
def test_low_rank_pieces_within_budget(N, W, eps):
    t = T.thm1(N, W, eps)
    dH, dA, dB = T.deltas(eps)
    Z = T.adi_Z(N, t.r_H)
    assert np.linalg.norm(T.hilbert(N) - Z @ Z.T, 2) <= dH
    VA = T.monomials(N, 2 * t.r_A)
    assert np.linalg.norm(T.A1_matrix(N) - VA @ t.CA @ VA.T, 2) <= dA
    VB = T.monomials(N, 2 * t.r_B - 1)
    assert np.linalg.norm(T.B0_matrix(N, W) - VB @ t.CB @ VB.T, 2) <= dB


@pytest.mark.parametrize("N,W,eps", CASES)
def test_theorem1_and_fast_factorization(N, W, eps):
    t = T.thm1(N, W, eps)
    L1, L2 = T.L_factors(t)
    B = O.prolate_matrix(N, W)
    F = T.partial_fourier_matrix(N, W)
    assert np.linalg.norm(B - F @ F.conj().T - L1 @ L2.conj().T, 2) <= eps            # Theorem 1
    assert t.r1 <= (4 / math.pi ** 2 * math.log(8 * N) + 6) * math.log(15 / eps)       # its rank bound
    assert t.r_H == T.rank_H_formula(N, eps)
    plan = O.make_plan(N, W, None, eps)
    T1, T2 = T.T_factors(t, plan)
    Pex = O.exact_operator_dense(N, W, plan.K)
    assert np.linalg.norm(Pex - T1 @ T2.conj().T, 2) <= 2 * eps                        # Section 1.3
    Kp = t.nF + t.r1 + plan.r
    assert Kp <= math.ceil(2 * N * W) + (12 / math.pi ** 2 * math.log(8 * N) + 18) * math.log(15 / eps) + 1


@pytest.mark.parametrize("N,W,eps", CASES[:4])
def test_matrix_free_coefficients(N, W, eps):
    t = T.thm1(N, W, eps)
    plan = O.make_plan(N, W, None, eps)
    _, T2 = T.T_factors(t, plan)
    rng = np.random.default_rng(N)
    Y = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    assert np.max(np.abs(T.coeffs(t, plan, Y) - T2.conj().T @ Y)) < 1e-12
    y = rng.standard_normal(N)
    c = T.coeffs(t, plan, y)
    assert np.linalg.norm(T.expand(t, plan, c) - O.exact_project(N, W, plan.K, y)) <= 2 * eps * np.linalg.norm(y)


def test_optimal_shifts_beat_logspaced():
    N, eps = 4096, 1e-6
    r = T.rank_H_formula(N, eps)
    dH = T.deltas(eps)[0]
    assert T.adi_error_bound(N, T.adi_shifts(N, r)) <= dH / math.pi
    assert T.adi_error_bound(N, T.adi_shifts_logspaced(N, r)) > dH / math.pi


def test_planted_mistakes_are_caught(monkeypatch):
    N, W, eps = 128, 0.2, 1e-6
    B = O.prolate_matrix(N, W)
    F = T.partial_fourier_matrix(N, W)
    base = B - F @ F.conj().T
    # D_B without the pi of the cosine identity
    t = T.thm1(N, W, eps)
    monkeypatch.setattr(T, "phase_B", lambda tt: np.exp(1j * (tt.W + tt.Wp) * np.arange(tt.N)))
    L1, L2 = T.L_factors(t)
    assert np.linalg.norm(base - L1 @ L2.conj().T, 2) > 100 * eps
    monkeypatch.undo()
    # W' rounded to the nearest even integer instead of odd
    monkeypatch.setattr(T, "nearest_odd_2NW", lambda n, w: 2 * int(round(n * w)))
    F2 = T.partial_fourier_matrix(N, W)
    assert np.max(np.abs(F2 @ F2.conj().T - T.dirichlet_FFstar(N, W))) > 1e-3
