"""Seeded synthetic workloads for the fast Slepian projection.

This module only draws random numbers and assembles signals; it holds none of the
method's arithmetic.  Both the CUDA path (through the tests and the benchmark) and
the FP64 oracle are fed from here.  Every parameter (tone frequencies, amplitudes,
phases, noise) is drawn on the host with numpy's PCG64 generator from a fixed
seed; tone sums are evaluated in float64 with torch on the requested device, so
large batches can be assembled on the GPU without changing their definition.

The five workloads follow the paper's own test signals (random vectors,
Section 4.1) at the sizes of the benchmark configurations:

  tiny     N=4096,  W=1/16, eps=1e-6, one N(0,1) signal and one 64-tone signal (FP64)
  c65k     N=65536, W=1/8,  eps=1e-4, B signals, half N(0,1), half 256-tone (FP32)
  ragged   4096 signals, N log-uniform in [1000, 262144], W ~ U[1/64, 1/4],
           eps from {1e-3, 1e-6, 1e-8}, N(0,1) entries (FP32)
  c1m      N=2^20,  W=0.05, eps=1e-6, 64 complex signals, CN(0,1), half of them
           band-limited to |f| <= W (complex64)
  c4m      N=2^22,  W=1/4,  eps=1e-8, 8 N(0,1) + 8 1024-tone signals (FP32)

and the Fourier-extension problem of Section 4.2 (the right-hand side of the normal
equations B g = F y for a continuous, non-smooth, non-periodic test function; the paper's
random parameters are not given, so they are drawn here):

  fourier_extension  f(t) = 5 t + sum_{l<500} a_l exp(-|t - mu_l| / sigma_l) on [-1, 1],
                     a_l ~ N(0, 1/4), mu_l ~ U[-1, 1], sigma_l ~ U[0.02, 0.5] (seed 6),
                     extension to [-T, T], T = 1.5: N = 2M + 1 coefficients, W = 1/(2T)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _torch():
    import torch
    return torch


def tone_sum(N: int, freqs: np.ndarray, amps: np.ndarray, phases: np.ndarray | None = None,
             device: str = "cpu", complex_out: bool = False, chunk: int = 1 << 16):
    """x[n] = sum_k amps[k] exp(j (2 pi freqs[k] n + phases[k])) for n < N, in float64.
    Returns the real part unless complex_out.  torch tensor on `device`."""
    torch = _torch()
    f = torch.as_tensor(np.asarray(freqs, dtype=np.float64), device=device)
    a = torch.as_tensor(np.asarray(amps, dtype=np.complex128), device=device)
    ph = torch.zeros_like(f) if phases is None else torch.as_tensor(
        np.asarray(phases, dtype=np.float64), device=device)
    out = torch.empty(N, dtype=torch.complex128 if complex_out else torch.float64, device=device)
    for n0 in range(0, N, chunk):
        n = torch.arange(n0, min(N, n0 + chunk), dtype=torch.float64, device=device)
        # phase in cycles, reduced mod 1 before the trig call
        cyc = torch.remainder(n[:, None] * f[None, :] + ph[None, :] / (2 * math.pi), 1.0)
        ang = 2.0 * math.pi * cyc
        z = torch.complex(torch.cos(ang), torch.sin(ang)) @ a
        out[n0:n0 + n.numel()] = z if complex_out else z.real
    return out


@dataclass
class Workload:
    name: str
    N: int                 # signal length (0 for ragged)
    W: float
    eps: float
    dtype: str             # "f64", "f32", "c64"
    y: object              # torch tensor (batch, N) or list of tensors (ragged)
    params: list | None = None   # ragged: list of (N, W, eps)

    @property
    def batch(self) -> int:
        return len(self.y) if isinstance(self.y, list) else int(self.y.shape[0])


def tiny(device: str = "cpu") -> Workload:
    """Two FP64 signals, N=4096, W=1/16: y ~ N(0,1) (seed 0) and a sum of 64
    random-phase unit cosines with frequencies uniform in [-W, W] (seed 1)."""
    torch = _torch()
    N, W = 4096, 1.0 / 16
    g0 = np.random.default_rng(0)
    y0 = torch.as_tensor(g0.standard_normal(N), device=device)
    g1 = np.random.default_rng(1)
    f = g1.uniform(-W, W, 64)
    ph = g1.uniform(0.0, 2 * math.pi, 64)
    y1 = tone_sum(N, f, np.ones(64), ph, device=device)
    return Workload("tiny", N, W, 1e-6, "f64", torch.stack([y0, y1]))


def multitone_batch(N: int, W: float, count: int, ntones: int, rng, device: str):
    torch = _torch()
    rows = []
    for _ in range(count):
        f = rng.uniform(-W, W, ntones)
        a = (rng.standard_normal(ntones) + 1j * rng.standard_normal(ntones)) / math.sqrt(2.0)
        rows.append(tone_sum(N, f, a, device=device))
    return torch.stack(rows) if rows else torch.empty(0, N, dtype=torch.float64, device=device)


def c65k(batch: int = 1024, device: str = "cpu", N: int = 65536) -> Workload:
    """N=65536, W=1/8, eps=1e-4, FP32: the first half of the batch N(0,1), the
    second half real parts of 256-tone sums with CN(0,1) amplitudes (seed 2)."""
    torch = _torch()
    W = 1.0 / 8
    rng = np.random.default_rng(2)
    half = batch // 2
    noise = torch.as_tensor(rng.standard_normal((batch - half, N)), device=device)
    tones = multitone_batch(N, W, half, 256, rng, device)
    y = torch.cat([noise, tones]).to(torch.float32)
    return Workload("c65k", N, W, 1e-4, "f32", y)


def c1m(batch: int = 64, device: str = "cpu", N: int = 1 << 20) -> Workload:
    """N=2^20, W=0.05, eps=1e-6, complex64: CN(0,1) i.i.d.; the second half of
    the batch is band-limited to |f| <= W (length-N DFT, zero the bins with
    |k/N| > W, inverse DFT, rescale to unit mean power) (seed 4)."""
    torch = _torch()
    W = 0.05
    rng = np.random.default_rng(4)
    re = rng.standard_normal((batch, N))
    im = rng.standard_normal((batch, N))
    y = torch.complex(torch.as_tensor(re, device=device),
                      torch.as_tensor(im, device=device)) / math.sqrt(2.0)
    half = batch // 2
    if batch - half > 0:
        k = torch.fft.fftfreq(N, device=device, dtype=torch.float64)
        keep = (k.abs() <= W).to(torch.complex128)
        Yb = torch.fft.fft(y[half:], dim=1) * keep
        yb = torch.fft.ifft(Yb, dim=1)
        yb = yb / torch.sqrt((yb.abs() ** 2).mean(dim=1, keepdim=True))
        y = torch.cat([y[:half], yb])
    return Workload("c1m", N, W, 1e-6, "c64", y.to(torch.complex64))


def c4m(batch: int = 16, device: str = "cpu", N: int = 1 << 22) -> Workload:
    """N=2^22, W=1/4, eps=1e-8, FP32: first half N(0,1), second half real parts of
    1024-tone sums with CN(0,1) amplitudes (seed 5)."""
    torch = _torch()
    W = 0.25
    rng = np.random.default_rng(5)
    half = batch // 2
    noise = torch.as_tensor(rng.standard_normal((batch - half, N)), device=device)
    tones = multitone_batch(N, W, half, 1024, rng, device)
    y = torch.cat([noise, tones]).to(torch.float32)
    return Workload("c4m", N, W, 1e-8, "f32", y)


RAGGED_EPS = (1e-3, 1e-6, 1e-8)


def ragged_params(count: int = 4096, seed: int = 3, n_lo: int = 1000, n_hi: int = 262144):
    """(N, W, eps) per signal: N = floor(exp(U[ln n_lo, ln n_hi])), W ~ U[1/64, 1/4],
    eps uniform over {1e-3, 1e-6, 1e-8}."""
    rng = np.random.default_rng(seed)
    Ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(np.int64)
    Ws = rng.uniform(1.0 / 64, 1.0 / 4, count)
    es = np.asarray(RAGGED_EPS)[rng.integers(0, len(RAGGED_EPS), count)]
    return [(int(n), float(w), float(e)) for n, w, e in zip(Ns, Ws, es)]


def ragged(count: int = 4096, device: str = "cpu", seed: int = 3,
           n_lo: int = 1000, n_hi: int = 262144) -> Workload:
    """Ragged batch: per-signal (N, W, eps) from ragged_params, y ~ N(0,1), FP32."""
    torch = _torch()
    params = ragged_params(count, seed, n_lo, n_hi)
    rng = np.random.default_rng(seed + 1000)
    ys = [torch.as_tensor(rng.standard_normal(n), device=device).to(torch.float32)
          for (n, _, _) in params]
    return Workload("ragged", 0, 0.0, 0.0, "f32", ys, params)


def gaussian(batch: int, N: int, seed: int, device: str = "cpu", complex_: bool = False):
    """Plain N(0,1) (or CN(0,1)) test signals, float64 / complex128."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    if complex_:
        z = (rng.standard_normal((batch, N)) + 1j * rng.standard_normal((batch, N))) / math.sqrt(2)
        return torch.as_tensor(z, device=device)
    return torch.as_tensor(rng.standard_normal((batch, N)), device=device)


@dataclass
class FourierExtension:
    M: int
    T: float
    N: int              # 2M + 1
    W: float            # 1 / (2T)
    yhat: np.ndarray    # (F_{N''} f)[m], m = -M..M (complex128): right-hand side of B g = yhat
    fhat: np.ndarray    # Fourier series coefficients of f on [-1, 1], m = -M..M (complex128)
    f: object           # callable: f(t) for an array of t in [-1, 1]


def fourier_extension(M: int, T: float = 1.5, L: int = 500, seed: int = 6, nquad: int = 1 << 17):
    """Section 4.2's Fourier-extension set-up with a seeded stand-in for its random test
    function.  Both coefficient vectors are integrals over [-1, 1] approximated by an
    FFT of length nquad (the paper likewise uses an FFT):
      yhat[m] = 1/sqrt(2T) int_{-1}^{1} f(t) exp(-j pi m t / T) dt   (t on a grid of [-T, T))
      fhat[m] = 1/sqrt(2)  int_{-1}^{1} f(t) exp(-j pi m t) dt       (t on a grid of [-1, 1))
    for |m| <= M.  (The paper prints + in the exponent of the coefficient formula of
    Section 4.2 and - in the operator F_{N''} of Section 1.4; - is taken for both.)"""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(L) * 0.5
    mu = rng.uniform(-1.0, 1.0, L)
    sig = rng.uniform(0.02, 0.5, L)

    def f(t):
        t = np.asarray(t, dtype=np.float64)
        out = 5.0 * t
        for i in range(0, t.size, 8192):
            tc = t[i:i + 8192]
            out[i:i + 8192] += (a[None, :] * np.exp(-np.abs(tc[:, None] - mu[None, :]) / sig[None, :])).sum(1)
        return out

    m = np.arange(-M, M + 1)
    tk = -T + 2.0 * T * np.arange(nquad) / nquad
    fk = np.zeros(nquad)
    inside = np.abs(tk) <= 1.0
    fk[inside] = f(tk[inside])
    Fk = np.fft.fft(fk)
    yhat = (2.0 * T / nquad) / math.sqrt(2.0 * T) * np.exp(1j * np.pi * m) * Fk[m % nquad]
    t1 = -1.0 + 2.0 * np.arange(nquad) / nquad
    F1 = np.fft.fft(f(t1))
    fhat = (2.0 / nquad) / math.sqrt(2.0) * np.exp(1j * np.pi * m) * F1[m % nquad]
    return FourierExtension(M=M, T=T, N=2 * M + 1, W=1.0 / (2.0 * T), yhat=yhat, fhat=fhat, f=f)
