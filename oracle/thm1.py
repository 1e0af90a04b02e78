"""FP64 CPU oracle for the fast factorization of S_K S_K^* (Section 1.3, "A fast
factorization of S_K S_K^*") built from the constructive proof of Theorem 1
(Section 2) and of Corollary 2 (Section 3.2).

TEST INFRASTRUCTURE ONLY (same rules as fst_oracle.py): only the tests, the smoke
check and the benchmark's CPU leg use it.

    B_{N,W} - F F^* = L1 L2^* + E1,   ||E1|| <= eps                      (Theorem 1)
    S_K S_K^*       = B_{N,W} + U1 U2^* + E2,   ||E2|| <= eps             (Corollary 2)
    S_K S_K^*       = T1 T2^* + E1 + E2,  T1 = [F L1 U1], T2 = [F L2 U2]  (Section 1.3)

The coefficient vector of a signal y is T2^* y = [F^* y; L2^* y; U2^* y] (length
K' = 2NW' + r1 + r2), and T1 (T2^* y) is within 2 eps ||y|| of S_K S_K^* y.

Readings of the paper taken here:
  * "2NW' is the nearest odd integer to W" is read as nearest odd integer to 2NW;
    ties (2NW an even integer) round up: 2NW' = 2 floor(NW) + 1.
  * D_B[n,n] = exp(j pi (W + W') n): the pi is needed for the cosine identity
    the proof uses (D_B B0 D_B^* + D_B^* B0 D_B = 2 cos(pi (W+W')(m-n)) B0).
  * B0's diagonal is its limit 2 (W - W') (the proof writes only the m != n form).
  * V_A, V_B use centred, scaled monomials u_m^k, u_m = (m - (N-1)/2) / N, instead
    of m^k: (m - n)/N = u_m - u_n, so V C V^T is the same matrix, but the FP64
    entries stay bounded (m^k overflows for N = 2^22, k ~ 27).
  * CF-ADI shifts: the optimal choice of the appendix's remarks,
    p_k = b dn((2k-1)/(2r) I(sqrt(1 - kappa^-2)), sqrt(1 - kappa^-2)), a = 1/2,
    b = N - 1/2, kappa = b/a, with r_H from the lemma's formula; r_H grows only if
    the exact ADI error bound max_n |phi(n + 1/2)|^2 <= delta_H / pi fails
    (it holds at the formula's value for every case tested).
  * The expanded expression of L (the line after "Putting it all together") has
    a sign slip in its fourth term; L1 and L2 follow Eq. (BFF), and L1 L2^* is
    checked against B - F F^* directly.
  * U1, U2 use the transition set of fst_oracle (|1[l<K] - lambda_l| > eps):
    U2 column = sqrt|D_l| s_l, U1 column = sign(D_l) sqrt|D_l| s_l, so that
    U1 U2^* = S_T diag(D) S_T^T.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import comb, ellipj, ellipkm1, zeta

from . import fst_oracle as O


def nearest_odd_2NW(N: int, W: float) -> int:
    """2NW' (see module docstring)."""
    return 2 * int(math.floor(N * W)) + 1


def partial_fourier_matrix(N: int, W: float) -> np.ndarray:
    """F_{N,W} (Eq. PartialFourierMatrix): columns e_{k/N}/sqrt(N), k = -h..h, 2h+1 = 2NW'."""
    h = (nearest_odd_2NW(N, W) - 1) // 2
    n = np.arange(N)[:, None]
    k = np.arange(-h, h + 1)[None, :]
    return np.exp(2j * np.pi * n * k / N) / math.sqrt(N)


def dirichlet_FFstar(N: int, W: float) -> np.ndarray:
    """Closed form of F F^* (Eq. FFstar): sin(2 pi W'(m-n)) / (N sin(pi (m-n)/N)), diagonal 2W'."""
    Wp = nearest_odd_2NW(N, W) / (2.0 * N)
    d = np.arange(N)[:, None] - np.arange(N)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.sin(2 * np.pi * Wp * d) / (N * np.sin(np.pi * d / N))
    out[d == 0] = 2 * Wp
    return out


# --------------------------------------------------------------------------- ranks

def deltas(eps: float):
    """delta_H = 4 pi eps / 15, delta_A = delta_B = 7 eps / 30 (Section 2, putting it together)."""
    return 4 * math.pi * eps / 15, 7 * eps / 30, 7 * eps / 30


def rank_H_formula(N: int, eps: float) -> int:
    dH, _, _ = deltas(eps)
    return int(math.ceil(math.log(8 * N - 4) * math.log(4 * math.pi / dH) / math.pi ** 2))


def rank_A(eps: float) -> int:
    _, dA, _ = deltas(eps)
    return int(math.ceil(math.log(2 / (3 * math.pi * dA)) / (2 * math.log(2))))


def rank_B(eps: float) -> int:
    _, _, dB = deltas(eps)
    return int(math.ceil(math.log(3 / (2 * dB)) / (2 * math.log(6 / math.pi))))


# --------------------------------------------------------------------------- H ~ Z Z^*

def adi_shifts_logspaced(N: int, r: int) -> np.ndarray:
    """The appendix's fallback: shifts evenly spaced on a log scale in [a, b]."""
    a, b = 0.5, N - 0.5
    k = np.arange(1, r + 1)
    return a ** ((2 * k - 1) / (2 * r)) * b ** ((2 * r - 2 * k + 1) / (2 * r))


def adi_shifts(N: int, r: int) -> np.ndarray:
    """Optimal shifts p_k = b dn((2k-1)/(2r) K, m), m = 1 - kappa^-2 (appendix, remark)."""
    a, b = 0.5, N - 0.5
    m1 = (a / b) ** 2                  # 1 - m
    K = ellipkm1(m1)                   # complete elliptic integral I(sqrt(m))
    k = np.arange(1, r + 1)
    _, _, dn, _ = ellipj((2 * k - 1) / (2.0 * r) * K, 1.0 - m1)
    return b * dn


def adi_error_bound(N: int, p: np.ndarray) -> float:
    """max over the spectrum {n + 1/2} of |phi|^2, phi(x) = prod (x - p_j)/(x + p_j)."""
    x = np.arange(N) + 0.5
    phi = np.ones(N)
    for pj in p:
        phi *= (x - pj) / (x + pj)
    return float(np.max(phi ** 2))


def rank_H(N: int, eps: float) -> int:
    """The lemma's formula value, grown only if the shifts miss ||H - ZZ^*|| <= delta_H."""
    dH, _, _ = deltas(eps)
    r = max(1, rank_H_formula(N, eps))
    while adi_error_bound(N, adi_shifts(N, r)) > dH / math.pi:
        r += 1
    return r


def adi_Z(N: int, r: int) -> np.ndarray:
    """CF-ADI factor of H (appendix) with A = diag(n + 1/2), B = ones, x = n + 1/2:
    Z_1 = sqrt(2 p_1)/(x + p_1), Z_k = sqrt(p_k/p_{k-1}) (x - p_{k-1})/(x + p_k) Z_{k-1}."""
    p = adi_shifts(N, r)
    x = np.arange(N) + 0.5
    Z = np.empty((N, r))
    Z[:, 0] = math.sqrt(2 * p[0]) / (x + p[0])
    for k in range(1, r):
        Z[:, k] = math.sqrt(p[k] / p[k - 1]) * (x - p[k - 1]) / (x + p[k]) * Z[:, k - 1]
    return Z


def hilbert(N: int) -> np.ndarray:
    i = np.arange(N)
    return 1.0 / (i[:, None] + i[None, :] + 1.0)


# --------------------------------------------------------------------------- A1, B0

def alpha_A(r_A: int) -> np.ndarray:
    """alpha_k = 1 - (1 - 2^{-(2k-1)}) zeta(2k), k = 1..r_A (Taylor series of A1)."""
    k = np.arange(1, r_A + 1)
    return 1.0 - (1.0 - 2.0 ** (-(2 * k - 1))) * zeta(2 * k)


def beta_B(r_B: int, N: int, W: float) -> np.ndarray:
    """beta_k = (-1)^k (pi (W - W') N)^{2k+1} / (2k+1)!, k = 0..r_B-1 (Taylor series of B0)."""
    Wp = nearest_odd_2NW(N, W) / (2.0 * N)
    t = math.pi * (W - Wp) * N
    k = np.arange(r_B)
    return np.array([(-1) ** kk * t ** (2 * kk + 1) / math.factorial(2 * kk + 1) for kk in k])


def centred(N: int) -> np.ndarray:
    return (np.arange(N) - (N - 1) / 2.0) / N


def poly_CA(r_A: int, N: int) -> np.ndarray:
    """C_A with A1~[m,n] = (2/(N pi)) sum_k alpha_k (u_m - u_n)^{2k-1} = sum_{i,l} C[i,l] u_m^i u_n^l."""
    D = 2 * r_A
    al = alpha_A(r_A)
    C = np.zeros((D, D))
    for kk in range(1, r_A + 1):
        d = 2 * kk - 1
        for i in range(d + 1):
            C[i, d - i] += 2.0 / (N * math.pi) * al[kk - 1] * comb(d, i, exact=True) * (-1) ** (d - i)
    return C


def poly_CB(r_B: int, N: int, W: float) -> np.ndarray:
    """C_B with B0~[m,n] = (2/(N pi)) sum_k beta_k (u_m - u_n)^{2k} = sum_{i,l} C[i,l] u_m^i u_n^l."""
    D = 2 * r_B - 1
    be = beta_B(r_B, N, W)
    C = np.zeros((D, D))
    for kk in range(r_B):
        d = 2 * kk
        for i in range(d + 1):
            C[i, d - i] += 2.0 / (N * math.pi) * be[kk] * comb(d, i, exact=True) * (-1) ** (d - i)
    return C


def monomials(N: int, D: int) -> np.ndarray:
    u = centred(N)
    return u[:, None] ** np.arange(D)[None, :]


def A0_matrix(N: int) -> np.ndarray:
    d = np.arange(N)[:, None] - np.arange(N)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        A0 = 1.0 / (np.pi * d) - 1.0 / (N * np.sin(np.pi * d / N))
    A0[d == 0] = 0.0
    return A0


def A1_matrix(N: int) -> np.ndarray:
    d = np.arange(N)[:, None] - np.arange(N)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        A1 = A0_matrix(N) - 1.0 / (np.pi * (d + N)) - 1.0 / (np.pi * (d - N))
    A1[d == 0] = 0.0
    return A1


def B0_matrix(N: int, W: float) -> np.ndarray:
    Wp = nearest_odd_2NW(N, W) / (2.0 * N)
    d = np.arange(N)[:, None] - np.arange(N)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        B0 = 2 * np.sin(np.pi * (W - Wp) * d) / (np.pi * d)
    B0[d == 0] = 2 * (W - Wp)
    return B0


# --------------------------------------------------------------------------- factors

@dataclass
class Thm1:
    N: int
    W: float
    eps: float
    Wp: float
    h: int
    r_H: int
    r_A: int
    r_B: int
    p: np.ndarray         # ADI shifts
    CA: np.ndarray
    CB: np.ndarray

    @property
    def r1(self) -> int:
        return 4 * self.r_H + 4 * self.r_A + 2 * (2 * self.r_B - 1)

    @property
    def nF(self) -> int:
        return 2 * self.h + 1


def thm1(N: int, W: float, eps: float) -> Thm1:
    odd = nearest_odd_2NW(N, W)
    rH, rA, rB = rank_H(N, eps), rank_A(eps), rank_B(eps)
    return Thm1(N=N, W=W, eps=eps, Wp=odd / (2.0 * N), h=(odd - 1) // 2, r_H=rH, r_A=rA, r_B=rB,
                p=adi_shifts(N, rH), CA=poly_CA(rA, N), CB=poly_CB(rB, N, W))


def phase_A(t: Thm1) -> np.ndarray:
    """diag of D_A: exp(j 2 pi W' n)."""
    return np.exp(2j * np.pi * t.Wp * np.arange(t.N))


def phase_B(t: Thm1) -> np.ndarray:
    """diag of D_B: exp(j pi (W + W') n)."""
    return np.exp(1j * np.pi * (t.W + t.Wp) * np.arange(t.N))


def L_factors(t: Thm1):
    """Dense L1, L2 (N x r1), block order of Section 2 (putting it all together)."""
    N = t.N
    Z = adi_Z(N, t.r_H)
    JZ = Z[::-1]
    VA = monomials(N, 2 * t.r_A)
    VB = monomials(N, 2 * t.r_B - 1)
    dA = phase_A(t)[:, None]
    dB = phase_B(t)[:, None]
    c = 1.0 / (2j * np.pi)
    L1 = np.hstack([c * dA * Z, -c * dA * JZ, -c * np.conj(dA) * Z, c * np.conj(dA) * JZ,
                    dA * VA / 2j, -np.conj(dA) * VA / 2j, dB * VB / 2, np.conj(dB) * VB / 2])
    L2 = np.hstack([dA * JZ, dA * Z, np.conj(dA) * JZ, np.conj(dA) * Z,
                    dA * (VA @ t.CA.T), np.conj(dA) * (VA @ t.CA.T),
                    dB * (VB @ t.CB.T), np.conj(dB) * (VB @ t.CB.T)])
    return L1, L2


def U_factors(plan: O.Plan):
    """U1, U2 of Corollary 2's proof on the oracle's transition set."""
    sq = np.sqrt(np.abs(plan.D))
    U2 = plan.S_T * sq[None, :]
    U1 = plan.S_T * (np.sign(plan.D) * sq)[None, :]
    return U1, U2


def T_factors(t: Thm1, plan: O.Plan):
    F = partial_fourier_matrix(t.N, t.W)
    L1, L2 = L_factors(t)
    U1, U2 = U_factors(plan)
    return np.hstack([F, L1, U1]), np.hstack([F, L2, U2])


# --------------------------------------------------------------------------- matrix-free coefficients

def coeffs(t: Thm1, plan: O.Plan | None, y: np.ndarray) -> np.ndarray:
    """T2^* y without forming T2 (any N).  y: (N,) or (N, batch), real or complex.
    Order: F^* y (frequencies -h..h), then the eight L2 blocks, then U2^* y
    (left out when plan is None)."""
    y = np.asarray(y)
    one = y.ndim == 1
    Y = y[:, None] if one else y
    N = t.N
    # F^* y: length-N DFT bins k = -h..h, divided by sqrt(N)
    Yf = np.fft.fft(Y, axis=0) / math.sqrt(N)
    kk = np.arange(-t.h, t.h + 1) % N
    cF = Yf[kk]
    # L2^* y: conj(column) . y for every column, generated column by column
    dA = phase_A(t)
    dB = phase_B(t)
    x = np.arange(N) + 0.5
    p = t.p
    ZY = []      # block 1..4 sums for each k
    z = math.sqrt(2 * p[0]) / (x + p[0])
    zs = [z]
    for k in range(1, t.r_H):
        z = math.sqrt(p[k] / p[k - 1]) * (x - p[k - 1]) / (x + p[k]) * z
        zs.append(z)
    yA = np.conj(dA)[:, None] * Y        # D_A^* y
    yAc = dA[:, None] * Y                # D_A y
    yB = np.conj(dB)[:, None] * Y
    yBc = dB[:, None] * Y
    b1 = np.array([zz[::-1] @ yA for zz in zs])      # (D_A J Z)^* y = Z^T J D_A^* y
    b2 = np.array([zz @ yA for zz in zs])            # (D_A Z)^* y
    b3 = np.array([zz[::-1] @ yAc for zz in zs])     # (D_A^* J Z)^* y
    b4 = np.array([zz @ yAc for zz in zs])           # (D_A^* Z)^* y
    u = centred(N)
    DA, DB = 2 * t.r_A, 2 * t.r_B - 1
    qA = np.array([(u ** i) @ yA for i in range(DA)])
    qAc = np.array([(u ** i) @ yAc for i in range(DA)])
    qB = np.array([(u ** i) @ yB for i in range(DB)])
    qBc = np.array([(u ** i) @ yBc for i in range(DB)])
    # (D V C^T)^* y = C V^T D^* y  (C real)
    b5, b6 = t.CA @ qA, t.CA @ qAc
    b7, b8 = t.CB @ qB, t.CB @ qBc
    cL = np.vstack([b1, b2, b3, b4, b5, b6, b7, b8])
    if plan is None:
        c = np.vstack([cF, cL])
    else:
        _, U2 = U_factors(plan)
        c = np.vstack([cF, cL, U2.T @ Y])
    return c[:, 0] if one else c


def expand(t: Thm1, plan: O.Plan, c: np.ndarray) -> np.ndarray:
    """T1 c (dense T1; small N)."""
    T1, _ = T_factors(t, plan)
    return T1 @ c
