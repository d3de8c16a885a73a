"""ctypes binding of libttm.so (include/ttm.h): argument marshalling only.

Every step of the product runs in the library's CUDA kernels; this module only
turns lists of torch tensors (device, float64, shape (D_l, d, D_r)) or numpy arrays
(host) into the C descriptors and back. There is no fallback: if the shared
library is missing or fails to load, every call raises.
"""

import ctypes
import os

import numpy as np

from . import _build

TTM_OK = 0
PREC = {"fp64": 0, "bf16_split": 2}
LOSS = {"inner": 0, "sqdist": 1}
STATUS = {0: "TTM_OK", 1: "TTM_WARN_NOT_CONVERGED", -1: "TTM_ERR_INVALID_ARG", -2: "TTM_ERR_SHAPE", -3: "TTM_ERR_NOMEM",
          -4: "TTM_ERR_WORKSPACE", -5: "TTM_ERR_NONFINITE", -6: "TTM_ERR_CUDA",
          -7: "TTM_ERR_TIMEOUT", -8: "TTM_ERR_RANK_CAP", -9: "TTM_ERR_UNSUPPORTED"}

# Every symbol include/ttm.h declares (checked by the CPU test suite).
EXPORTED = ["ttm_create", "ttm_destroy", "ttm_set_options", "ttm_multiply", "ttm_multiply_batched",
            "ttm_output_capacity", "ttm_backward", "ttm_inner", "ttm_inner3", "ttm_synchronize",
            "ttm_tt_free", "ttm_last_error", "ttm_version", "ttm_multiply_noalloc", "ttm_gemm"]


class TTMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class c_tt(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("d", ctypes.c_int32), ("on_host", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("bonds", ctypes.POINTER(ctypes.c_int64)),
                ("cores", ctypes.POINTER(ctypes.c_void_p))]


class c_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("eps", ctypes.c_double), ("chi_max", ctypes.c_int64),
                ("chi_out", ctypes.c_int64), ("max_sweeps", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("check_finite", ctypes.c_int32), ("profile_kernels", ctypes.c_int32),
                ("f32_passes", ctypes.c_int32), ("jacobi_kernel", ctypes.c_int32),
                ("newton_steps", ctypes.c_int32), ("split_digits", ctypes.c_int32),
                ("reserved1", ctypes.c_int32), ("env_budget_bytes", ctypes.c_int64)]


class c_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("jacobi_sweeps_max", ctypes.c_int32),
                ("max_bond", ctypes.c_int64), ("n_swaps", ctypes.c_int64), ("n_contracts", ctypes.c_int64),
                ("n_qr", ctypes.c_int64), ("discarded_weight", ctypes.c_double), ("err_bound", ctypes.c_double),
                ("norm_out", ctypes.c_double), ("flops_counted", ctypes.c_double), ("seconds", ctypes.c_double),
                ("peak_workspace_bytes", ctypes.c_int64), ("bond_trace", ctypes.POINTER(ctypes.c_int64)),
                ("bond_trace_len", ctypes.c_int64), ("n_kernel_launches", ctypes.c_int64),
                ("jacobi_launches", ctypes.c_int64), ("gemm_ms", ctypes.c_double),
                ("newton_residual", ctypes.c_double), ("jacobi32_ms", ctypes.c_double),
                ("jacobi32_flops", ctypes.c_double), ("n_nonconverged", ctypes.c_int64),
                ("n_frozen_pairs", ctypes.c_int64), ("gemm_flops", ctypes.c_double),
                ("gemm_launches", ctypes.c_int64), ("qr_ms", ctypes.c_double), ("n_fallback", ctypes.c_int64),
                ("jacobi32_sweeps", ctypes.c_int64), ("svd_trace", ctypes.POINTER(ctypes.c_int32)),
                ("svd_trace_len", ctypes.c_int64), ("jacobi64_ms", ctypes.c_double)]


_LIB = None


def library_path():
    return _build.LIB


def load_library(build_if_missing=False):
    """Load libttm.so (building it first only if asked). Raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise TTMError(-9, "libttm.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    lib.ttm_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, P(c_options)]
    lib.ttm_destroy.argtypes = [ctypes.c_void_p]
    lib.ttm_set_options.argtypes = [ctypes.c_void_p, P(c_options)]
    lib.ttm_multiply.argtypes = [ctypes.c_void_p, P(c_tt), P(c_tt), P(c_tt), P(c_report)]
    lib.ttm_multiply_batched.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(c_tt), P(c_tt), P(c_tt), P(c_report)]
    lib.ttm_output_capacity.argtypes = [P(c_tt), P(c_tt), P(c_options)]
    lib.ttm_output_capacity.restype = ctypes.c_int64
    lib.ttm_backward.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(c_tt), P(c_tt), P(c_tt),
                                 P(ctypes.c_double), P(c_tt), P(c_tt)]
    lib.ttm_inner.argtypes = [ctypes.c_void_p, P(c_tt), P(c_tt), P(ctypes.c_double)]
    lib.ttm_inner3.argtypes = [ctypes.c_void_p, P(c_tt), P(c_tt), P(c_tt), P(ctypes.c_double)]
    lib.ttm_multiply_noalloc.argtypes = [P(c_tt), P(c_tt), P(c_tt), P(c_options), ctypes.c_void_p]
    lib.ttm_multiply_noalloc.restype = ctypes.c_int
    lib.ttm_gemm.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_int64]
    lib.ttm_gemm.restype = ctypes.c_int
    lib.ttm_synchronize.argtypes = [ctypes.c_void_p]
    lib.ttm_tt_free.argtypes = [ctypes.c_void_p, P(c_tt)]
    lib.ttm_last_error.restype = ctypes.c_char_p
    lib.ttm_version.restype = ctypes.c_char_p
    for name in ("ttm_create", "ttm_destroy", "ttm_set_options", "ttm_multiply", "ttm_multiply_batched",
                 "ttm_backward", "ttm_inner", "ttm_inner3", "ttm_synchronize", "ttm_tt_free"):
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(status):
    """Raises on an error status; a warning status (positive) is returned to the caller, and
    the report of the call carries the details."""
    if status < TTM_OK:
        raise TTMError(status, _LIB.ttm_last_error().decode())
    return status


def make_options(prec="fp64", eps=0.0, chi_max=0, chi_out=0, max_sweeps=0, use_graph=0, profile=0,
                 f32_passes=0, jacobi_kernel=0, newton_steps=0, split_digits=0, env_budget_bytes=0):
    return c_options(PREC[prec] if isinstance(prec, str) else int(prec), float(eps), int(chi_max),
                     int(chi_out), int(max_sweeps), int(use_graph), 0, int(profile), int(f32_passes),
                     int(jacobi_kernel), int(newton_steps), int(split_digits), 0, int(env_budget_bytes))


class TTDesc:
    """Keeps a C descriptor and the arrays it points to alive."""

    def __init__(self, cores, on_host=None, writable=False):
        import torch  # noqa: F401  (tensors are the device container)
        self.cores = list(cores)
        L = len(self.cores)
        first = self.cores[0]
        self.is_numpy = isinstance(first, np.ndarray)
        self.is_cpu_tensor = (not self.is_numpy) and (not first.is_cuda)
        if on_host is None:
            on_host = self.is_numpy or self.is_cpu_tensor
        d = int(first.shape[1])
        bonds = [int(first.shape[0])] + [int(c.shape[2]) for c in self.cores]
        self.bonds = (ctypes.c_int64 * (L + 1))(*bonds)
        ptrs = []
        for c in self.cores:
            if self.is_numpy:
                assert c.dtype == np.float64 and c.flags["C_CONTIGUOUS"], "cores must be C-contiguous float64"
                ptrs.append(c.ctypes.data)
            else:
                assert c.dtype.is_floating_point and c.element_size() == 8 and c.is_contiguous(), \
                    "cores must be contiguous float64 tensors"
                ptrs.append(c.data_ptr())
        self.ptrs = (ctypes.c_void_p * L)(*ptrs)
        self.c = c_tt(L, d, 1 if on_host else 0, 0, self.bonds, self.ptrs)


class Handle:
    """ttm_create / ttm_destroy on a device and stream (torch's current stream by default)."""

    def __init__(self, device=0, stream=None, **opts):
        lib = load_library()
        self.lib = lib
        self.device = device
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        self.h = ctypes.c_void_p()
        o = make_options(**opts)
        _check(lib.ttm_create(ctypes.byref(self.h), int(device), ctypes.c_void_p(stream), ctypes.byref(o)))

    def set_options(self, **opts):
        o = make_options(**opts)
        _check(self.lib.ttm_set_options(self.h, ctypes.byref(o)))

    def close(self):
        if self.h:
            self.lib.ttm_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def report_dict(r, trace=None, svd=None):
    out = {f: getattr(r, f) for f, _ in c_report._fields_ if f not in ("bond_trace", "svd_trace")}
    if svd is not None:
        out["svd_trace"] = [tuple(svd[8 * i + j] for j in range(7)) for i in range(r.svd_trace_len)]
    out["status_name"] = STATUS.get(r.status, r.status)
    if trace is not None:
        out["bond_trace"] = [int(trace[i]) for i in range(r.bond_trace_len)]
    return out


def output_capacity(A, B, **opts):
    lib = load_library()
    a, b = TTDesc(A, on_host=True), TTDesc(B, on_host=True)
    o = make_options(**opts)
    return int(lib.ttm_output_capacity(ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(o)))


def _alloc_out(like, L, cap, n_items):
    import torch
    outs, keep = [], []
    for _ in range(n_items):
        if like == "numpy":
            bufs = [np.empty(cap, dtype=np.float64) for _ in range(L)]
            ptrs = [b.ctypes.data for b in bufs]
            on_host = 1
        elif like == "pinned":
            bufs = [torch.empty(cap, dtype=torch.float64).pin_memory() for _ in range(L)]
            ptrs = [b.data_ptr() for b in bufs]
            on_host = 1
        else:
            bufs = [torch.empty(cap, dtype=torch.float64, device=like) for _ in range(L)]
            ptrs = [b.data_ptr() for b in bufs]
            on_host = 0
        bonds = (ctypes.c_int64 * (L + 1))()
        cptrs = (ctypes.c_void_p * L)(*ptrs)
        outs.append(c_tt(L, 0, on_host, 0, bonds, cptrs))
        keep.append(bufs)
    return outs, keep


def _shape_out(o, bufs, d):
    L = o.L
    cores = []
    for k in range(L):
        n = int(o.bonds[k]) * d * int(o.bonds[k + 1])
        cores.append(bufs[k][:n].reshape(int(o.bonds[k]), d, int(o.bonds[k + 1])))
    return cores


def ttm_multiply_batched(handle, pairs, eps=0.0, chi_max=0, chi_out=0, prec="fp64", max_sweeps=0, profile=0,
                         f32_passes=0, jacobi_kernel=0, newton_steps=0, split_digits=0, use_graph=0):
    """[(A_i, B_i)] -> ([Omega_i], [report_i]) with one batched launch sequence (ttm_multiply_batched)."""
    lib = handle.lib
    handle.set_options(prec=prec, eps=eps, chi_max=chi_max, chi_out=chi_out, max_sweeps=max_sweeps,
                       profile=profile, f32_passes=f32_passes, jacobi_kernel=jacobi_kernel,
                       newton_steps=newton_steps, split_digits=split_digits, use_graph=use_graph)
    n = len(pairs)
    da = [TTDesc(A) for A, _ in pairs]
    db = [TTDesc(B) for _, B in pairs]
    L = da[0].c.L
    d = da[0].c.d
    cap = 0
    o = make_options(prec=prec, eps=eps, chi_max=chi_max, chi_out=chi_out)
    for a, b in zip(da, db):
        cap = max(cap, int(lib.ttm_output_capacity(ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(o))))
    if cap <= 0:
        raise TTMError(-1, "ttm_output_capacity failed: " + lib.ttm_last_error().decode())
    like = "numpy" if da[0].is_numpy else ("pinned" if da[0].is_cpu_tensor else pairs[0][0][0].device)
    outs, keep = _alloc_out(like, L, cap, n)
    arrA = (c_tt * n)(*[a.c for a in da])
    arrB = (c_tt * n)(*[b.c for b in db])
    arrO = (c_tt * n)(*outs)
    traces = [(ctypes.c_int64 * L)() for _ in range(n)]
    reps = (c_report * n)()
    for i in range(n):
        reps[i].bond_trace = ctypes.cast(traces[i], ctypes.POINTER(ctypes.c_int64))
        reps[i].bond_trace_len = L
    _check(lib.ttm_multiply_batched(handle.h, n, arrA, arrB, arrO, reps))
    results = [_shape_out(arrO[i], keep[i], d) for i in range(n)]
    return results, [report_dict(reps[i], traces[i]) for i in range(n)]


def ttm_multiply(handle, A, B, eps=0.0, chi_max=0, chi_out=0, prec="fp64", max_sweeps=0, profile=0,
                 f32_passes=0, jacobi_kernel=0, newton_steps=0, split_digits=0, use_graph=0):
    """Omega = A o B through ttm_multiply. Returns (cores, report)."""
    lib = handle.lib
    handle.set_options(prec=prec, eps=eps, chi_max=chi_max, chi_out=chi_out, max_sweeps=max_sweeps,
                       profile=profile, f32_passes=f32_passes, jacobi_kernel=jacobi_kernel,
                       newton_steps=newton_steps, split_digits=split_digits, use_graph=use_graph)
    a, b = TTDesc(A), TTDesc(B)
    o = make_options(prec=prec, eps=eps, chi_max=chi_max, chi_out=chi_out)
    cap = int(lib.ttm_output_capacity(ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(o)))
    if cap <= 0:
        raise TTMError(-1, "ttm_output_capacity failed: " + lib.ttm_last_error().decode())
    like = "numpy" if a.is_numpy else ("pinned" if a.is_cpu_tensor else A[0].device)
    outs, keep = _alloc_out(like, a.c.L, cap, 1)
    out = outs[0]
    trace = (ctypes.c_int64 * a.c.L)()
    nsvd = a.c.L * a.c.L
    svd = (ctypes.c_int32 * (8 * nsvd))()
    rep = c_report()
    rep.bond_trace = ctypes.cast(trace, ctypes.POINTER(ctypes.c_int64))
    rep.bond_trace_len = a.c.L
    rep.svd_trace = ctypes.cast(svd, ctypes.POINTER(ctypes.c_int32))
    rep.svd_trace_len = nsvd
    _check(lib.ttm_multiply(handle.h, ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(out), ctypes.byref(rep)))
    return _shape_out(out, keep[0], a.c.d), report_dict(rep, trace, svd)


def ttm_inner(handle, X, Y):
    x, y = TTDesc(X), TTDesc(Y)
    v = ctypes.c_double()
    _check(handle.lib.ttm_inner(handle.h, ctypes.byref(x.c), ctypes.byref(y.c), ctypes.byref(v)))
    return v.value


def ttm_inner3(handle, W, A, B):
    w, a, b = TTDesc(W), TTDesc(A), TTDesc(B)
    v = ctypes.c_double()
    _check(handle.lib.ttm_inner3(handle.h, ctypes.byref(w.c), ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(v)))
    return v.value


def ttm_backward(handle, kind, A, B, WC, want_a=True, want_b=True):
    """Loss and gradients w.r.t. every core of A and B (device tensors). Returns (loss, gA, gB)."""
    import torch
    a, b, w = TTDesc(A), TTDesc(B), TTDesc(WC)
    gA = [torch.empty_like(c) for c in A] if want_a else None
    gB = [torch.empty_like(c) for c in B] if want_b else None
    ga = TTDesc(gA) if want_a else None
    gb = TTDesc(gB) if want_b else None
    v = ctypes.c_double()
    _check(handle.lib.ttm_backward(handle.h, LOSS[kind] if isinstance(kind, str) else int(kind),
                                   ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(w.c), ctypes.byref(v),
                                   ctypes.byref(ga.c) if ga else None, ctypes.byref(gb.c) if gb else None))
    return v.value, gA, gB


def ttm_gemm(handle, A, B, prec="fp64"):
    """C = A B through ttm_gemm for 2-D float64 CUDA tensors (any strides with a unit row
    stride are passed as column-major views; other layouts are made contiguous first)."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    a = A.t().contiguous().t() if A.stride(0) != 1 else A     # column-major views
    b = B.t().contiguous().t() if B.stride(0) != 1 else B
    C = torch.empty((N, M), dtype=torch.float64, device=A.device).t()
    _check(handle.lib.ttm_gemm(handle.h, PREC[prec] if isinstance(prec, str) else int(prec), M, N, K,
                               a.data_ptr(), max(a.stride(1), M), b.data_ptr(), max(b.stride(1), K),
                               C.data_ptr(), M))
    return C
