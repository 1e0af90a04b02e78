"""FP64 CPU oracle for the Fast Slepian Transform projection (Karnik, Zhu, Wakin,
Romberg, Davenport, "The Fast Slepian Transform", arXiv:1611.04950).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
It is deliberately plain and slow: every function follows the paper's definitions
in its own notation, with numpy / scipy primitives (FFT, dense and tridiagonal
symmetric eigensolvers) as the only building blocks, so a reader can check it
against the paper by eye.  It shares no code, tables or constants with the CUDA
library.

Notation: N signal length, W half-bandwidth in (0, 1/2), K number of Slepian
vectors kept, eps tolerance, M FFT length, B the prolate matrix, S_{N,W} the
Slepian basis (columns s^(l), eigenvalues lambda_l in descending order).

Readings taken where the paper is silent:
  * The commuting tridiagonal matrix used to compute the DPSS is Slepian's (1978),
    which the paper cites for the DPSS but does not write out (Section 1.1).
  * "log" in every bound is the natural logarithm.
  * K defaults to round(2NW) with halves rounded away from zero (Section 4.1).
  * The transition set is T = {l : |1[l<K] - lambda_l| > eps}; it equals the
    paper's {eps < lambda_l < 1 - eps} whenever K meets the band condition of
    Corollary 2, and it stays a valid (larger) set otherwise.
  * DPSS sign convention: symmetric vectors have positive sum, antisymmetric ones
    have positive first moment sum((N-1-2n) s[n]) (Slepian's convention).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Scalars: K, the Corollary 1 bound, the asymptotic transition count
# ---------------------------------------------------------------------------


def default_K(N: int, W: float) -> int:
    """K = round(2NW), halves away from zero (Section 4.1 uses round(2NW))."""
    x = 2.0 * N * W
    return int(math.floor(x + 0.5))


def cor1_bound(N: int, eps: float) -> float:
    """Corollary 1: #{l : eps < lambda_l < 1-eps} <= (8/pi^2 log 8N + 12) log(15/eps)."""
    return (8.0 / math.pi ** 2 * math.log(8.0 * N) + 12.0) * math.log(15.0 / eps)


def asymptotic_transition(N: int, eps: float) -> float:
    """Eq. (asymptotic): #{eps <= lambda <= 1-eps} ~ (2/pi^2) log N log(1/eps - 1)."""
    return 2.0 / math.pi ** 2 * math.log(N) * math.log(1.0 / eps - 1.0)


# ---------------------------------------------------------------------------
# Definitions: prolate matrix, sinc kernel, B y
# ---------------------------------------------------------------------------


def prolate_matrix(N: int, W: float) -> np.ndarray:
    """Dense B_{N,W}[m,n] = sin(2 pi W (m-n)) / (pi (m-n)), diagonal 2W (Eq. Prolate matrix)."""
    k = np.arange(N)
    diff = k[:, None] - k[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        B = np.sin(2.0 * np.pi * W * diff) / (np.pi * diff)
    B[diff == 0] = 2.0 * W
    return B


def sinc_row(N: int, W: float) -> np.ndarray:
    """First row of the Toeplitz matrix B_{N,W}: b[k] = sin(2 pi W k)/(pi k), b[0] = 2W."""
    k = np.arange(1, N, dtype=np.float64)
    b = np.empty(N)
    b[0] = 2.0 * W
    b[1:] = np.sin(2.0 * np.pi * W * k) / (np.pi * k)
    return b


def fft_length(N: int) -> int:
    """Smallest power of 2 that is at least 2N (Section 4.1)."""
    M = 1
    while M < 2 * N:
        M *= 2
    return M


def sinc_spectrum(N: int, W: float, M: int) -> np.ndarray:
    """DFT_M of the circulant embedding of B_{N,W}: c[k] = c[M-k] = b[k] for 0 <= k < N,
    zero elsewhere.  c is even, so its DFT is real; the real part is returned."""
    assert M >= 2 * N - 1
    b = sinc_row(N, W)
    c = np.zeros(M)
    c[:N] = b
    c[M - N + 1:] = b[1:][::-1]
    return np.fft.fft(c).real


def apply_prolate(y: np.ndarray, W: float, M: int | None = None) -> np.ndarray:
    """B_{N,W} y by a zero-padded length-M FFT convolution (Section 1.3, fast
    projection; Section 4.1 for M).  y has shape (N,) or (N, batch); real or complex."""
    y = np.asarray(y)
    N = y.shape[0]
    if M is None:
        M = fft_length(N)
    C = sinc_spectrum(N, W, M)
    shape = (M,) + (1,) * (y.ndim - 1)
    Y = np.fft.fft(y, n=M, axis=0)
    out = np.fft.ifft(Y * C.reshape(shape), axis=0)[:N]
    if not np.iscomplexobj(y):
        out = out.real
    return out


def apply_prolate_direct(y: np.ndarray, W: float) -> np.ndarray:
    """B_{N,W} y by the O(N^2) Toeplitz sum (the definition, no FFT)."""
    y = np.asarray(y)
    N = y.shape[0]
    b = sinc_row(N, W)
    out = np.zeros_like(y, dtype=np.result_type(y, np.float64))
    for m in range(N):
        row = np.concatenate([b[m:0:-1], b[: N - m]])  # B[m, n] = b[|m - n|]
        out[m] = row @ y
    return out


# ---------------------------------------------------------------------------
# Slepian basis
# ---------------------------------------------------------------------------


def slepian_tridiagonal(N: int, W: float):
    """Slepian's tridiagonal matrix that commutes with B_{N,W} (not written in the
    paper; Slepian 1978, which Section 1.1 cites for the DPSS):
    diag[n] = ((N-1)/2 - n)^2 cos(2 pi W), offdiag[n-1] = n (N - n) / 2, n = 1..N-1.
    Its l-th largest eigenvector is the DPSS s^(l)."""
    n = np.arange(N, dtype=np.float64)
    d = ((N - 1) / 2.0 - n) ** 2 * math.cos(2.0 * math.pi * W)
    e = n[1:] * (N - n[1:]) / 2.0
    return d, e


def _fix_sign(S: np.ndarray) -> np.ndarray:
    N = S.shape[0]
    n = np.arange(N)
    out = S.copy()
    for j in range(S.shape[1]):
        s = S[:, j]
        sym = np.dot(s, s[::-1]) > 0.0  # J s = +s or -s
        ref = s.sum() if sym else np.dot(N - 1 - 2 * n, s)
        if ref < 0:
            out[:, j] = -s
    return out


def dpss_window(N: int, W: float, l_lo: int, l_hi: int) -> np.ndarray:
    """Slepian basis vectors s^(l) for l_lo <= l <= l_hi (descending-lambda index),
    as columns of an N x (l_hi - l_lo + 1) array, unit 2-norm (Eq. dpssnorm),
    sign convention as in the module docstring.  LAPACK bisection + inverse
    iteration (stebz / stein) on Slepian's tridiagonal matrix."""
    assert 0 <= l_lo <= l_hi <= N - 1
    d, e = slepian_tridiagonal(N, W)
    if N == 1:
        return np.ones((1, 1))
    # l-th largest eigenvalue = ascending index N-1-l
    _, V = sla.eigh_tridiagonal(d, e, select="i",
                                select_range=(N - 1 - l_hi, N - 1 - l_lo),
                                lapack_driver="stebz")
    S = V[:, ::-1]
    S = S / np.linalg.norm(S, axis=0, keepdims=True)
    return _fix_sign(S)


def dpss_dense(N: int, W: float):
    """All N Slepian vectors and eigenvalues from a dense eigensolve of B_{N,W}
    (B = S Lambda S^*, Section 1.2).  Small N only.  Returns (lambda desc, S)."""
    lam, V = np.linalg.eigh(prolate_matrix(N, W))
    return lam[::-1].copy(), V[:, ::-1].copy()


def rayleigh_eigenvalues(S: np.ndarray, W: float, M: int | None = None) -> np.ndarray:
    """lambda_l = s_l^T B s_l for each column (s_l unit norm eigenvectors of B);
    columns in groups of 8 to bound the FFT's memory at large N."""
    lam = np.empty(S.shape[1])
    for j0 in range(0, S.shape[1], 8):
        blk = S[:, j0:j0 + 8]
        lam[j0:j0 + 8] = np.einsum("ij,ij->j", blk, apply_prolate(blk, W, M))
    return lam


# ---------------------------------------------------------------------------
# The plan: transition set, D, and the fast operators
# ---------------------------------------------------------------------------

OP_PROJECT = "project"      # S_K S_K^*            (Corollary 2, Section 1.3)
OP_PINV = "pinv"            # rank-K truncated pseudoinverse of B (Corollary 3)
OP_TIKHONOV = "tikhonov"    # (B^2 + alpha I)^{-1} B            (Corollary 4)


@dataclass
class Plan:
    N: int
    W: float
    K: int
    eps: float
    M: int
    op: str
    alpha: float
    window: tuple              # (l_lo, l_hi) eigen-window searched
    idx: np.ndarray            # transition indices T (ascending l)
    lam: np.ndarray            # lambda_l for l in T
    S_T: np.ndarray            # N x r, columns s^(l), l in T
    D: np.ndarray              # diagonal of the correction, one per l in T
    beta: float                # scale of the Toeplitz part (1, or 1/(1+alpha))
    lam_window: np.ndarray = field(repr=False, default=None)

    @property
    def r(self) -> int:
        return int(self.idx.size)


def window_halfwidth(N: int, eps: float) -> int:
    """Initial half-width of the eigen-window searched around K: a little more than
    half the asymptotic transition count (Eq. asymptotic), never more than the
    Corollary 1 bound.  make_plan doubles it until both edges fall outside T."""
    a = asymptotic_transition(max(N, 2), eps)
    return int(min(math.ceil(cor1_bound(N, eps)), math.ceil(0.6 * a) + 6))


def _in_T(lam: np.ndarray, l: np.ndarray, K: int, eps: float, op: str, alpha: float):
    if op == OP_TIKHONOV:
        # Lemma for Corollary 4: alpha(1+alpha) eps < lambda < 1 - eps/3
        return (lam > alpha * (1.0 + alpha) * eps) & (lam < 1.0 - eps / 3.0)
    # Corollaries 2 and 3: I_2 u I_3, read as |1[l<K] - lambda_l| > eps
    return np.abs((l < K).astype(np.float64) - lam) > eps


def _D_of(lam: np.ndarray, l: np.ndarray, K: int, op: str, alpha: float):
    if op == OP_PROJECT:
        # U1 U2^* = V2 (I - Lambda2) V2^* - V3 Lambda3 V3^*  (proof of Corollary 2)
        return np.where(l < K, 1.0 - lam, -lam)
    if op == OP_PINV:
        # U3 U4^* = V2 (Lambda2^{-1} - Lambda2) V2^* - V3 Lambda3 V3^*  (proof of Corollary 3)
        return np.where(l < K, 1.0 / lam - lam, -lam)
    if op == OP_TIKHONOV:
        # U5 U5^* = V1 [(Lambda1^2 + alpha)^{-1} Lambda1 - Lambda1/(1+alpha)] V1^*  (Corollary 4)
        return lam / (lam ** 2 + alpha) - lam / (1.0 + alpha)
    raise ValueError(op)


def make_plan(N: int, W: float, K: int | None = None, eps: float = 1e-6,
              op: str = OP_PROJECT, alpha: float = 0.0, M: int | None = None) -> Plan:
    """Precomputation (Section 1.3, last paragraph; Section 4.1): the transition
    Slepian vectors S_T, their eigenvalues, the diagonal D, and the FFT length."""
    if not (N >= 1 and 0.0 < W < 0.5 and 0.0 < eps < 0.5):
        raise ValueError("need N >= 1, 0 < W < 1/2, 0 < eps < 1/2")
    if K is None:
        K = default_K(N, W)
    if not (0 <= K <= N):
        raise ValueError("need 0 <= K <= N")
    if op == OP_TIKHONOV and not alpha > 0.0:
        raise ValueError("Tikhonov needs alpha > 0")
    if M is None:
        M = fft_length(N)
    # the window is centred on K for the projection / pseudoinverse and on
    # 2NW for Tikhonov (its set does not depend on K)
    centre = K if op != OP_TIKHONOV else default_K(N, W)
    R = window_halfwidth(N, eps)
    while True:
        lo, hi = max(0, centre - R), min(N - 1, centre + R)
        S = dpss_window(N, W, lo, hi)
        lam = rayleigh_eigenvalues(S, W, M)
        l = np.arange(lo, hi + 1)
        inT = _in_T(lam, l, K, eps, op, alpha)
        edge_ok = (lo == 0 or not inT[0]) and (hi == N - 1 or not inT[-1])
        if edge_ok:
            break
        R *= 2
    sel = np.nonzero(inT)[0]
    D = _D_of(lam[sel], l[sel], K, op, alpha)
    beta = 1.0 / (1.0 + alpha) if op == OP_TIKHONOV else 1.0
    return Plan(N=N, W=W, K=K, eps=eps, M=M, op=op, alpha=alpha, window=(lo, hi),
                idx=l[sel], lam=lam[sel], S_T=S[:, sel].copy(), D=D, beta=beta,
                lam_window=lam)


def fast_apply(plan: Plan, y: np.ndarray) -> np.ndarray:
    """The fast operator: beta * B_{N,W} y + S_T (D o (S_T^T y)).  For the projection
    this is B y + U1 U2^* y (Section 1.3, fast projections); y is (N,) or (N, batch),
    real or complex (B and S_T are real, so real and imaginary parts separate)."""
    y = np.asarray(y)
    By = apply_prolate(y, plan.W, plan.M)
    c = plan.S_T.T @ y
    Dc = plan.D.reshape((-1,) + (1,) * (y.ndim - 1)) * c
    return plan.beta * By + plan.S_T @ Dc


def fast_project(plan: Plan, y: np.ndarray) -> np.ndarray:
    assert plan.op == OP_PROJECT
    return fast_apply(plan, y)


# ---------------------------------------------------------------------------
# Exact operators (the plain definitions the fast method approximates)
# ---------------------------------------------------------------------------

EXACT_DENSE_MAX_N = 8192
EPS_REF = 1e-13


def exact_operator_dense(N: int, W: float, K: int, op: str = OP_PROJECT,
                         alpha: float = 0.0) -> np.ndarray:
    """The N x N matrix the fast operator approximates, from a dense eigensolve of B:
    S_K S_K^* (projection), S_K Lambda_K^{-1} S_K^* (truncated pseudoinverse), or
    (B^2 + alpha I)^{-1} B (Tikhonov).  Small N only."""
    lam, S = dpss_dense(N, W)
    if op == OP_PROJECT:
        SK = S[:, :K]
        return SK @ SK.T
    if op == OP_PINV:
        SK = S[:, :K]
        return (SK / lam[:K]) @ SK.T
    if op == OP_TIKHONOV:
        return (S * (lam / (lam ** 2 + alpha))) @ S.T
    raise ValueError(op)


def exact_project(N: int, W: float, K: int, y: np.ndarray) -> np.ndarray:
    """P y = S_K S_K^* y.  Dense eigensolve for N <= 8192; above that the fast
    projection at eps_ref = 1e-13, whose distance to S_K S_K^* y is at most
    1e-13 ||y|| by Corollary 2."""
    y = np.asarray(y)
    if N <= EXACT_DENSE_MAX_N:
        lam, S = dpss_dense(N, W)
        SK = S[:, :K]
        return SK @ (SK.T @ y)
    ref = make_plan(N, W, K, EPS_REF)
    return fast_project(ref, y)
