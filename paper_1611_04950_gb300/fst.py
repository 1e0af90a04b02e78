"""GB300-native fast Slepian projection (Karnik, Zhu, Wakin, Romberg, Davenport,
"The Fast Slepian Transform", arXiv:1611.04950).

Thin Python binding of the C ABI in include/fst.h (libfst_gb300.so): argument
marshalling only.  Every step of the computation runs in the library's CUDA
kernels; there is no Python or CPU fallback.  If the shared library has not been
built, importing the binding raises -- build it with
``python -m paper_1611_04950_gb300.build``.

The functions carry the C names (fst_plan, fst_plan_op, fst_plan_info,
fst_plan_export, fst_project, fst_project_host, fst_apply_prolate, fst_destroy,
fst_last_error); ``Plan`` wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfst_gb300.so")

FST_OK, FST_EINVAL, FST_ENOMEM, FST_ECUDA, FST_ENOCONVERGE, FST_ETIMEOUT, FST_EUNSUPPORTED = range(7)
FST_F32, FST_F64, FST_C64, FST_C128 = range(4)
FST_OP_PROJECT, FST_OP_PINV, FST_OP_TIKHONOV = range(3)
_OPS = {"project": FST_OP_PROJECT, "pinv": FST_OP_PINV, "tikhonov": FST_OP_TIKHONOV}
_STATUS = {0: "FST_OK", 1: "FST_EINVAL", 2: "FST_ENOMEM", 3: "FST_ECUDA", 4: "FST_ENOCONVERGE",
           5: "FST_ETIMEOUT", 6: "FST_EUNSUPPORTED"}

# every symbol include/fst.h and include/fst_testing.h declare
EXPORTED = ["fst_plan", "fst_plan_op", "fst_plan_info", "fst_plan_export", "fst_project",
            "fst_project_host", "fst_apply_prolate", "fst_destroy", "fst_last_error", "fst_version",
            "fst_reduced_tridiagonal", "fst_emu_plan_op", "fst_plan_is_emulated",
            "fst_launch_count", "fst_profile_enable", "fst_profile_count", "fst_profile_read",
            "fst_project_noalloc", "fst_noalloc_scratch_bytes", "fst_coeffs", "fst_coeffs_info",
            "fst_adi_shifts", "fst_plan_many", "fst_emu_plan_many", "fst_project_ragged", "fst_expand",
            "fst_sync", "fst_test_tc_stall", "fst_ragged_tuning"]


class FSTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1611_04950_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P, i64, d, vp, I = C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_int
    sig = {
        "fst_plan": ([C.POINTER(P), i64, d, i64, d, vp], I),
        "fst_plan_op": ([C.POINTER(P), i64, d, i64, d, I, d, vp], I),
        "fst_plan_info": ([P] + [C.POINTER(i64)] * 5, I),
        "fst_plan_export": ([P, C.POINTER(i64), C.POINTER(d), C.POINTER(d), C.POINTER(d)], I),
        "fst_project": ([P, vp, vp, i64, i64, I, vp], I),
        "fst_project_host": ([P, vp, vp, i64, I, vp], I),
        "fst_apply_prolate": ([P, vp, vp, i64, i64, I, vp], I),
        "fst_destroy": ([P], I),
        "fst_sync": ([P, vp], I),
        "fst_ragged_tuning": ([C.POINTER(P), C.POINTER(vp), C.POINTER(vp), i64, I, C.POINTER(i64), C.POINTER(d)], I),
        "fst_test_tc_stall": ([I, d], I),
        "fst_last_error": ([], C.c_char_p),
        "fst_version": ([], C.c_char_p),
        "fst_reduced_tridiagonal": ([i64, d, I, C.POINTER(i64), C.POINTER(d), C.POINTER(d)], I),
        "fst_emu_plan_op": ([C.POINTER(P), i64, d, i64, d, I, d], I),
        "fst_plan_is_emulated": ([P], I),
        "fst_launch_count": ([], C.c_longlong),
        "fst_project_noalloc": ([P, vp, vp, i64, i64, I, vp], I),
        "fst_coeffs": ([P, vp, vp, i64, i64, I, vp], I),
        "fst_coeffs_info": ([P] + [C.POINTER(i64)] * 6, I),
        "fst_expand": ([P, vp, vp, i64, I, vp], I),
        "fst_adi_shifts": ([i64, I, C.POINTER(d)], I),
        "fst_plan_many": ([C.POINTER(P), i64, C.POINTER(i64), C.POINTER(d), C.POINTER(i64), C.POINTER(d), vp], I),
        "fst_emu_plan_many": ([C.POINTER(P), i64, C.POINTER(i64), C.POINTER(d), C.POINTER(i64), C.POINTER(d)], I),
        "fst_project_ragged": ([C.POINTER(P), C.POINTER(vp), C.POINTER(vp), i64, I, vp], I),
        "fst_noalloc_scratch_bytes": ([], C.c_ulonglong),
        "fst_profile_enable": ([I], I),
        "fst_profile_count": ([], I),
        "fst_profile_read": ([I, C.POINTER(C.c_char_p), C.POINTER(d), C.POINTER(C.c_longlong)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def _check(st: int):
    if st != FST_OK:
        raise FSTError(st, _lib.fst_last_error().decode())


# ---- C-named functions -------------------------------------------------------

def fst_last_error() -> str:
    return _lib.fst_last_error().decode()


def fst_version() -> str:
    return _lib.fst_version().decode()


def fst_plan(N: int, W: float, K: int = -1, eps: float = 1e-6, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(_lib.fst_plan(C.byref(h), N, W, K, eps, C.c_void_p(stream)))
    return h.value


def fst_plan_op(N: int, W: float, K: int, eps: float, op: int, alpha: float = 0.0, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(_lib.fst_plan_op(C.byref(h), N, W, K, eps, op, alpha, C.c_void_p(stream)))
    return h.value


def fst_emu_plan_op(N: int, W: float, K: int, eps: float, op: int = FST_OP_PROJECT, alpha: float = 0.0) -> int:
    h = C.c_void_p()
    _check(_lib.fst_emu_plan_op(C.byref(h), N, W, K, eps, op, alpha))
    return h.value


def fst_plan_info(h: int) -> dict:
    v = [C.c_int64() for _ in range(5)]
    _check(_lib.fst_plan_info(C.c_void_p(h), *[C.byref(x) for x in v]))
    return {"K": v[0].value, "r": v[1].value, "M": v[2].value, "window": (v[3].value, v[4].value)}


def fst_plan_export(h: int, N: int, with_vectors: bool = True) -> dict:
    r = fst_plan_info(h)["r"]
    idx = np.zeros(max(r, 1), np.int64)
    lam = np.zeros(max(r, 1))
    D = np.zeros(max(r, 1))
    S = np.zeros((max(r, 1), N)) if with_vectors else None
    ptr = lambda a, t: a.ctypes.data_as(C.POINTER(t)) if a is not None else None
    _check(_lib.fst_plan_export(C.c_void_p(h), ptr(idx, C.c_int64), ptr(lam, C.c_double), ptr(D, C.c_double),
                                ptr(S, C.c_double)))
    out = {"idx": idx[:r], "lam": lam[:r], "D": D[:r]}
    if with_vectors:
        out["S_T"] = S[:r].T.copy()
    return out


def fst_project(h: int, y_ptr: int, out_ptr: int, batch: int, ld: int, dtype: int, stream: int = 0):
    _check(_lib.fst_project(C.c_void_p(h), C.c_void_p(y_ptr), C.c_void_p(out_ptr), batch, ld, dtype,
                            C.c_void_p(stream)))


def fst_apply_prolate(h: int, y_ptr: int, out_ptr: int, batch: int, ld: int, dtype: int, stream: int = 0):
    _check(_lib.fst_apply_prolate(C.c_void_p(h), C.c_void_p(y_ptr), C.c_void_p(out_ptr), batch, ld, dtype,
                                  C.c_void_p(stream)))


def fst_project_host(h: int, y_ptr: int, out_ptr: int, batch: int, dtype: int, stream: int = 0):
    _check(_lib.fst_project_host(C.c_void_p(h), C.c_void_p(y_ptr), C.c_void_p(out_ptr), batch, dtype,
                                 C.c_void_p(stream)))


def fst_project_noalloc(h: int, y_ptr: int, out_ptr: int, batch: int, ld: int, dtype: int, stream: int = 0):
    """fst_project without any device allocation (fixed library-owned scratch)."""
    _check(_lib.fst_project_noalloc(C.c_void_p(h), C.c_void_p(y_ptr), C.c_void_p(out_ptr), batch, ld, dtype,
                                    C.c_void_p(stream)))


def fst_noalloc_scratch_bytes() -> int:
    return int(_lib.fst_noalloc_scratch_bytes())


def fst_coeffs(h: int, y_ptr: int, out_ptr: int, batch: int, ld: int, dtype: int, stream: int = 0):
    _check(_lib.fst_coeffs(C.c_void_p(h), C.c_void_p(y_ptr), C.c_void_p(out_ptr), batch, ld, dtype,
                           C.c_void_p(stream)))


def fst_expand(h: int, c_ptr: int, out_ptr: int, batch: int, dtype: int, stream: int = 0):
    _check(_lib.fst_expand(C.c_void_p(h), C.c_void_p(c_ptr), C.c_void_p(out_ptr), batch, dtype, C.c_void_p(stream)))


def fst_coeffs_info(h: int) -> dict:
    v = [C.c_int64() for _ in range(6)]
    _check(_lib.fst_coeffs_info(C.c_void_p(h), *[C.byref(x) for x in v]))
    return dict(zip(["Kprime", "nF", "r1", "rH", "rA", "rB"], [x.value for x in v]))


def fst_adi_shifts(N: int, r: int) -> np.ndarray:
    out = np.zeros(r)
    _check(_lib.fst_adi_shifts(N, r, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def fst_plan_many(Ns, Ws, epss, Ks=None, stream=None, emulate: bool = False) -> list:
    """Handles of len(Ns) projection plans built together (fst_plan_many)."""
    n = len(Ns)
    out = (C.c_void_p * n)()
    Na = (C.c_int64 * n)(*[int(v) for v in Ns])
    Wa = (C.c_double * n)(*[float(v) for v in Ws])
    Ea = (C.c_double * n)(*[float(v) for v in epss])
    Ka = None if Ks is None else (C.c_int64 * n)(*[int(v) for v in Ks])
    cast = lambda a, t: C.cast(a, C.POINTER(t)) if a is not None else None
    if emulate:
        _check(_lib.fst_emu_plan_many(cast(out, C.c_void_p), n, cast(Na, C.c_int64), cast(Wa, C.c_double),
                                      cast(Ka, C.c_int64), cast(Ea, C.c_double)))
    else:
        _check(_lib.fst_plan_many(cast(out, C.c_void_p), n, cast(Na, C.c_int64), cast(Wa, C.c_double),
                                  cast(Ka, C.c_int64), cast(Ea, C.c_double), C.c_void_p(_stream_handle(stream))))
    return [out[i] for i in range(n)]


def fst_project_ragged(handles, y_ptrs, out_ptrs, dtype: int, stream: int = 0):
    n = len(handles)
    Pa = (C.c_void_p * n)(*handles)
    Ya = (C.c_void_p * n)(*y_ptrs)
    Oa = (C.c_void_p * n)(*out_ptrs)
    _check(_lib.fst_project_ragged(C.cast(Pa, C.POINTER(C.c_void_p)), C.cast(Ya, C.POINTER(C.c_void_p)),
                                   C.cast(Oa, C.POINTER(C.c_void_p)), n, dtype, C.c_void_p(stream)))


def fst_ragged_tuning(handles, y_ptrs, out_ptrs, dtype: int) -> dict:
    """{log2 M: (signals per launch group, measured ms)} chosen for an earlier ragged call."""
    n = len(handles)
    Pa = (C.c_void_p * n)(*handles)
    Ya = (C.c_void_p * n)(*y_ptrs)
    Oa = (C.c_void_p * n)(*out_ptrs)
    pairs = (C.c_int64 * 32)()
    ms = (C.c_double * 32)()
    _check(_lib.fst_ragged_tuning(C.cast(Pa, C.POINTER(C.c_void_p)), C.cast(Ya, C.POINTER(C.c_void_p)),
                                  C.cast(Oa, C.POINTER(C.c_void_p)), n, dtype, pairs, ms))
    return {lg: (int(pairs[lg]), float(ms[lg])) for lg in range(32) if pairs[lg]}


class PlanSet:
    """Plans of a ragged batch (one per signal), built with fst_plan_many."""

    def __init__(self, params, stream=None, emulate: bool = False):
        Ns, Ws, es = zip(*params) if params else ((), (), ())
        self.params = list(params)
        self.emulated = emulate
        self.h = fst_plan_many(Ns, Ws, es, stream=stream, emulate=emulate)

    def close(self):
        for h in getattr(self, "h", []) or []:
            fst_destroy(h)
        self.h = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, i: int) -> dict:
        return fst_plan_info(self.h[i])

    def tuning(self, ys, outs) -> dict:
        """The autotuned launch grouping of an earlier project(ys, outs) call."""
        return fst_ragged_tuning(self.h, [v.data_ptr() for v in ys], [o.data_ptr() for o in outs],
                                 _dtype_code(ys[0].dtype))

    def project(self, ys, outs=None, stream=None):
        """ys: list of (N_i,) device tensors (numpy arrays for an emulated set)."""
        if self.emulated:
            outs = [np.empty_like(v) for v in ys] if outs is None else outs
            fst_project_ragged(self.h, [v.ctypes.data for v in ys], [o.ctypes.data for o in outs],
                               _dtype_code(ys[0].dtype), 0)
            return outs
        import torch
        outs = [torch.empty_like(v) for v in ys] if outs is None else outs
        fst_project_ragged(self.h, [v.data_ptr() for v in ys], [o.data_ptr() for o in outs],
                           _dtype_code(ys[0].dtype), _stream_handle(stream))
        return outs


def fst_destroy(h: int):
    _check(_lib.fst_destroy(C.c_void_p(h)))


def fst_sync(h: int, stream: int = 0):
    """Waits for `stream`; raises FSTError(FST_ETIMEOUT) if a bounded device wait of an
    earlier call on the plan gave up."""
    _check(_lib.fst_sync(C.c_void_p(h), C.c_void_p(stream)))


def fst_test_tc_stall(launches: int, limit_s: float = 0.02):
    """Test hook: the next `launches` tensor-core correction launches give up on a wait that
    nothing completes, after limit_s seconds, before issuing any work."""
    _check(_lib.fst_test_tc_stall(launches, limit_s))


def fst_launch_count() -> int:
    return int(_lib.fst_launch_count())


def fst_profile_enable(on: bool = True):
    _check(_lib.fst_profile_enable(1 if on else 0))


def fst_profile_records() -> list:
    """[(kernel name, ms, pairs)] of the launches recorded since fst_profile_enable."""
    out = []
    for i in range(_lib.fst_profile_count()):
        nm, ms, un = C.c_char_p(), C.c_double(), C.c_longlong()
        _check(_lib.fst_profile_read(i, C.byref(nm), C.byref(ms), C.byref(un)))
        out.append((nm.value.decode(), ms.value, un.value))
    return out


def fst_plan_is_emulated(h: int) -> bool:
    return bool(_lib.fst_plan_is_emulated(C.c_void_p(h)))


def fst_reduced_tridiagonal(N: int, W: float, parity: int):
    n = C.c_int64()
    _check(_lib.fst_reduced_tridiagonal(N, W, parity, C.byref(n), None, None))
    d = np.zeros(max(n.value, 1))
    e = np.zeros(max(n.value - 1, 1))
    _check(_lib.fst_reduced_tridiagonal(N, W, parity, C.byref(n),
                                        d.ctypes.data_as(C.POINTER(C.c_double)),
                                        e.ctypes.data_as(C.POINTER(C.c_double))))
    return d[: n.value], e[: max(n.value - 1, 0)]


# ---- torch / numpy convenience -------------------------------------------------

def _dtype_code(dt) -> int:
    import torch
    m = {torch.float32: FST_F32, torch.float64: FST_F64, torch.complex64: FST_C64,
         torch.complex128: FST_C128,
         np.dtype(np.float32): FST_F32, np.dtype(np.float64): FST_F64,
         np.dtype(np.complex64): FST_C64, np.dtype(np.complex128): FST_C128}
    if dt not in m:
        raise TypeError(f"unsupported dtype {dt}")
    return m[dt]


class Plan:
    """Owns an fst plan.  ``emulate=True`` builds it on the host emulator (CPU tests:
    signals are then numpy arrays or CPU tensors)."""

    def __init__(self, N: int, W: float, K: int | None = None, eps: float = 1e-6, op: str = "project",
                 alpha: float = 0.0, stream=None, emulate: bool = False):
        self.N, self.W, self.eps, self.op, self.alpha = int(N), float(W), float(eps), op, float(alpha)
        k = -1 if K is None else int(K)
        self.emulated = emulate
        if emulate:
            self.h = fst_emu_plan_op(self.N, self.W, k, self.eps, _OPS[op], self.alpha)
        else:
            self.h = fst_plan_op(self.N, self.W, k, self.eps, _OPS[op], self.alpha, _stream_handle(stream))
        info = fst_plan_info(self.h)
        self.K, self.r, self.M, self.window = info["K"], info["r"], info["M"], info["window"]

    def close(self):
        if getattr(self, "h", None):
            fst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, with_vectors: bool = True) -> dict:
        return fst_plan_export(self.h, self.N, with_vectors)

    def _run(self, fn, y, out, stream):
        if self.emulated:
            y = np.ascontiguousarray(np.asarray(y))
            if y.ndim == 1:
                y = y[None]
            out = np.empty_like(y) if out is None else out
            fn(self.h, y.ctypes.data, out.ctypes.data, y.shape[0], y.shape[1], _dtype_code(y.dtype), 0)
            return out
        import torch
        if y.dim() == 1:
            y = y.unsqueeze(0)
        if y.shape[-1] != self.N or y.stride(-1) != 1:
            raise ValueError("signals must be (batch, N) with unit stride along N")
        if out is None:
            out = torch.empty_like(y)
        ld = y.stride(0) if y.shape[0] > 1 else self.N
        if out.stride(0) != ld and out.shape[0] > 1:
            raise ValueError("out must have the same row stride as y")
        fn(self.h, y.data_ptr(), out.data_ptr(), y.shape[0], ld, _dtype_code(y.dtype), _stream_handle(stream))
        return out

    def project(self, y, out=None, stream=None):
        """P_fast y (B y + S_T (D o S_T^T y)) for a (batch, N) device tensor."""
        return self._run(fst_project, y, out, stream)

    def apply_prolate(self, y, out=None, stream=None):
        """B_{N,W} y alone."""
        return self._run(fst_apply_prolate, y, out, stream)

    def coeffs(self, y, stream=None):
        """Fast coefficient vector T2^* y, (batch, K') complex (Section 1.3, fast factorization)."""
        info = fst_coeffs_info(self.h)
        Kp = info["Kprime"]
        if self.emulated:
            y = np.ascontiguousarray(np.asarray(y))
            if y.ndim == 1:
                y = y[None]
            ct = np.complex128 if y.dtype in (np.float64, np.complex128) else np.complex64
            out = np.zeros((y.shape[0], Kp), ct)
            fst_coeffs(self.h, y.ctypes.data, out.ctypes.data, y.shape[0], y.shape[1], _dtype_code(y.dtype), 0)
            return out
        import torch
        if y.dim() == 1:
            y = y.unsqueeze(0)
        ct = torch.complex128 if y.dtype in (torch.float64, torch.complex128) else torch.complex64
        out = torch.zeros((y.shape[0], Kp), dtype=ct, device=y.device)
        ld = y.stride(0) if y.shape[0] > 1 else self.N
        fst_coeffs(self.h, y.data_ptr(), out.data_ptr(), y.shape[0], ld, _dtype_code(y.dtype), _stream_handle(stream))
        return out

    def expand(self, c, stream=None):
        """T1 c for a (batch, K') complex coefficient array: (batch, N) complex (Section 1.3)."""
        if self.emulated:
            c = np.ascontiguousarray(np.asarray(c))
            if c.ndim == 1:
                c = c[None]
            out = np.zeros((c.shape[0], self.N), c.dtype)
            fst_expand(self.h, c.ctypes.data, out.ctypes.data, c.shape[0], _dtype_code(c.dtype), 0)
            return out
        import torch
        if c.dim() == 1:
            c = c.unsqueeze(0)
        c = c.contiguous()
        out = torch.zeros((c.shape[0], self.N), dtype=c.dtype, device=c.device)
        fst_expand(self.h, c.data_ptr(), out.data_ptr(), c.shape[0], _dtype_code(c.dtype), _stream_handle(stream))
        return out

    def project_host(self, y, out=None, stream=None):
        """P_fast y for a (batch, N) HOST array / tensor (copies inside the call)."""
        import torch
        if isinstance(y, np.ndarray):
            y = torch.from_numpy(y)
        if y.dim() == 1:
            y = y.unsqueeze(0)
        y = y.contiguous()
        if out is None:
            out = torch.empty_like(y)
        fst_project_host(self.h, y.data_ptr(), out.data_ptr(), y.shape[0], _dtype_code(y.dtype),
                         _stream_handle(stream))
        return out


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream
