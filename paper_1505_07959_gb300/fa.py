"""Thin ctypes binding of libfa (declared in include/fa.h).

Module-level functions carry the C names and only marshal arguments; every
step of the computation runs in the library's CUDA kernels.  `Plan` is a
convenience wrapper that allocates the workspace with PyTorch (the library
itself never allocates device memory) and passes raw device pointers and the
stream handle.  If the library has not been built, every call raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfa.so")

FA_OK = 0
FA_ERR_NOT_CONVERGED = 5
FA_FLOW_INV, FA_FLOW_EXP, FA_FLOW_SQRT, FA_FLOW_COS = 0, 1, 2, 3
FA_F64, FA_BF16, FA_BF16X3, FA_BF16X4, FA_BF16X6, FA_FP8E4M3 = 0, 1, 2, 3, 4, 5
DTYPES = {"f64": FA_F64, "bf16": FA_BF16, "bf16x3": FA_BF16X3, "bf16x4": FA_BF16X4,
          "bf16x6": FA_BF16X6, "fp8e4m3": FA_FP8E4M3}
SYMBOLS = ["fa_plan", "fa_plan_bind_workspace", "fa_plan_set_matrix", "fa_fine_sweep",
           "fa_coarse_sweep", "fa_refine", "fa_parareal_solve", "fa_parareal_solve_host",
           "fa_debug_product", "fa_debug_set_profile", "fa_debug_set_wait_fault", "fa_product_noalloc", "fa_plan_destroy", "fa_status_string", "fa_last_error",
           "fa_launch_count", "fa_launch_count_reset", "fa_batch_plan", "fa_batch_bind_workspace",
           "fa_batch_solve", "fa_batch_destroy", "fa_plan_set_learned", "fa_plan_learned_coefs",
           "fa_learned_records_scratch", "fa_learned_records", "fa_plan_set_recorder",
           "fa_plan_set_learned_check", "fa_aima_plan", "fa_aima",
           "fa_mlp_forward", "fa_mlp_scratch_bytes", "fa_mlp_loss_grad", "fa_mlp_adam",
           "fa_batch_autotune", "fa_batch_tuning", "fa_plan_autotune", "fa_plan_tuning"]
FA_COARSE_EULER, FA_COARSE_LEARNED = 0, 1
FA_METHOD_CLASSICAL, FA_METHOD_MODIFIED = 0, 1
FA_SCHEME_DEFAULT, FA_SCHEME_RK4, FA_SCHEME_EULER, FA_SCHEME_CN = 0, 1, 2, 3
SCHEMES = {"default": FA_SCHEME_DEFAULT, "rk4": FA_SCHEME_RK4, "euler": FA_SCHEME_EULER,
           "cn": FA_SCHEME_CN}
FA_MLP_FEATURES, FA_MLP_HIDDEN, FA_MLP_COEFS, FA_MLP_PARAMS = 8, 128, 4, 18196
FA_RECORD_DOUBLES = 32
FA_PROBES, FA_PROBE_SEED = 8, 0x150507959


class fa_problem_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("flow", ctypes.c_int), ("T", ctypes.c_double),
                ("N", ctypes.c_int), ("coarse_steps", ctypes.c_int), ("fine_steps", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("fine_dtype", ctypes.c_int), ("coarse_dtype", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("coarse_kind", ctypes.c_int),
                ("method", ctypes.c_int), ("span_drop", ctypes.c_double),
                ("max_basis", ctypes.c_int), ("fine_scheme", ctypes.c_int),
                ("coarse_scheme", ctypes.c_int)]


class fa_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("last_dx", ctypes.c_double),
                ("t_init_ms", ctypes.c_double), ("t_fine_ms", ctypes.c_double),
                ("t_coarse_ms", ctypes.c_double), ("t_refine_ms", ctypes.c_double),
                ("dx_history", ctypes.POINTER(ctypes.c_double)), ("g_fallback_iter", ctypes.c_int),
                ("coef_fallbacks", ctypes.c_int), ("records", ctypes.c_int),
                ("basis_dim", ctypes.c_int), ("double_angle_steps", ctypes.c_int),
                ("fine_blocks", ctypes.c_int)]


class FaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libfa status {status}: {msg}")
        self.status = status


_LIB = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfa.so and declare the C signatures (raises if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1505_07959_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, sz, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
    sigs = {
        "fa_plan": [ctypes.POINTER(vp), ctypes.POINTER(fa_problem_desc), vp, ctypes.POINTER(sz)],
        "fa_plan_bind_workspace": [vp, vp, sz],
        "fa_plan_set_matrix": [vp, dp],
        "fa_fine_sweep": [vp, dp, dp],
        "fa_coarse_sweep": [vp, dp, dp, dp, dp, dp, dp],
        "fa_refine": [vp, dp],
        "fa_parareal_solve": [vp, dp, dp, dp, ctypes.POINTER(fa_report)],
        "fa_parareal_solve_host": [vp, dp, dp, dp, ctypes.POINTER(fa_report)],
        "fa_debug_product": [vp, dp, dp, dp],
        "fa_debug_set_profile": [dp],
        "fa_debug_set_wait_fault": [ctypes.c_longlong, ctypes.c_int],
        "fa_product_noalloc": [ctypes.c_int, ctypes.c_int, dp, dp, dp, vp],
        "fa_plan_destroy": [vp],
        "fa_batch_plan": [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_double, ctypes.c_int, vp, ctypes.POINTER(sz)],
        "fa_batch_bind_workspace": [vp, vp, sz],
        "fa_batch_solve": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_double)],
        "fa_batch_destroy": [vp],
        "fa_plan_set_learned": [vp, dp],
        "fa_plan_learned_coefs": [vp, dp],
        "fa_learned_records_scratch": [vp, ctypes.POINTER(sz)],
        "fa_learned_records": [vp, dp, dp, dp, dp, sz],
        "fa_plan_set_recorder": [vp, dp, ctypes.c_int, dp, sz],
        "fa_plan_set_learned_check": [vp, ctypes.c_int],
        "fa_mlp_forward": [dp, ctypes.c_int, dp, ctypes.c_int, dp, vp],
        "fa_mlp_scratch_bytes": [ctypes.c_int, ctypes.POINTER(sz)],
        "fa_mlp_loss_grad": [dp, ctypes.c_int, dp, dp, dp, dp, sz, vp],
        "fa_mlp_adam": [dp, dp, dp, dp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                        ctypes.c_float, ctypes.c_float, vp],
        "fa_batch_autotune": [vp, ctypes.POINTER(vp), ctypes.c_char_p],
        "fa_plan_autotune": [vp],
        "fa_aima_plan": [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(sz)],
        "fa_aima": [vp, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp,
                    ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fa_status_string.argtypes = [ctypes.c_int]
    lib.fa_status_string.restype = ctypes.c_char_p
    lib.fa_last_error.argtypes = []
    lib.fa_last_error.restype = ctypes.c_char_p
    for name in ("fa_batch_tuning", "fa_plan_tuning"):
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = ctypes.c_char_p
    lib.fa_launch_count.argtypes = []
    lib.fa_launch_count.restype = ctypes.c_ulonglong
    lib.fa_launch_count_reset.argtypes = []
    lib.fa_launch_count_reset.restype = None
    _LIB = lib
    return lib


def _check(status: int, allow=(FA_OK,)) -> int:
    if status not in allow:
        lib = load_library()
        raise FaError(status, lib.fa_last_error().decode())
    return status


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# --- the C names ----------------------------------------------------------------------------

def fa_plan(desc: fa_problem_desc, stream_handle: int):
    lib = load_library()
    h, ws = ctypes.c_void_p(), ctypes.c_size_t()
    _check(lib.fa_plan(ctypes.byref(h), ctypes.byref(desc), ctypes.c_void_p(stream_handle),
                       ctypes.byref(ws)))
    return h, ws.value


def fa_plan_bind_workspace(h, ws_ptr: int, nbytes: int):
    _check(load_library().fa_plan_bind_workspace(h, ctypes.c_void_p(ws_ptr), nbytes))


def fa_plan_set_matrix(h, dA):
    _check(load_library().fa_plan_set_matrix(h, _ptr(dA)))


def fa_fine_sweep(h, dU, dF):
    _check(load_library().fa_fine_sweep(h, _ptr(dU), _ptr(dF)))


def fa_coarse_sweep(h, dU0, dD, dUnew, dGnew, dNorms, dUold):
    _check(load_library().fa_coarse_sweep(h, _ptr(dU0), _ptr(dD), _ptr(dUnew), _ptr(dGnew),
                                          _ptr(dNorms), _ptr(dUold)))


def fa_refine(h, dX):
    _check(load_library().fa_refine(h, _ptr(dX)))


def fa_parareal_solve(h, dA, dX0, dXout, report: fa_report):
    return _check(load_library().fa_parareal_solve(h, _ptr(dA), _ptr(dX0), _ptr(dXout),
                                                   ctypes.byref(report)),
                  allow=(FA_OK, FA_ERR_NOT_CONVERGED))


def fa_parareal_solve_host(h, hA: np.ndarray, hX0, hXout: np.ndarray, report: fa_report):
    dp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    return _check(load_library().fa_parareal_solve_host(h, dp(hA), dp(hX0), dp(hXout),
                                                        ctypes.byref(report)),
                  allow=(FA_OK, FA_ERR_NOT_CONVERGED))


def fa_debug_product(h, dL, dR, dC):
    _check(load_library().fa_debug_product(h, _ptr(dL), _ptr(dR), _ptr(dC)))


def fa_debug_set_profile(d_counters):
    _check(load_library().fa_debug_set_profile(_ptr(d_counters)))


def fa_debug_set_wait_fault(wait_cycles: int, skip_loads_cta: int):
    _check(load_library().fa_debug_set_wait_fault(wait_cycles, skip_loads_cta))


def fa_product_noalloc(n: int, dtype: int, dL, dR, dC, stream_handle: int):
    """dC = dL @ dR through the library's fixed scratch array (no device allocation)."""
    _check(load_library().fa_product_noalloc(n, dtype, _ptr(dL), _ptr(dR), _ptr(dC),
                                             ctypes.c_void_p(stream_handle)))


def fa_plan_destroy(h):
    if _LIB is not None and h:
        _LIB.fa_plan_destroy(h)


def fa_status_string(status: int) -> str:
    return load_library().fa_status_string(status).decode()


def fa_last_error() -> str:
    return load_library().fa_last_error().decode()


def fa_launch_count() -> int:
    return int(load_library().fa_launch_count())


def fa_launch_count_reset() -> None:
    load_library().fa_launch_count_reset()


def fa_batch_plan(ns, flows, Ts, coarse_steps, N, fine_steps, max_iters, tol, dtype, stream_handle):
    lib = load_library()
    cnt = len(ns)
    arr = lambda t, xs: (t * cnt)(*xs)
    h, ws = ctypes.c_void_p(), ctypes.c_size_t()
    _check(lib.fa_batch_plan(ctypes.byref(h), cnt, arr(ctypes.c_int, ns), arr(ctypes.c_int, flows),
                             arr(ctypes.c_double, Ts), arr(ctypes.c_int, coarse_steps), N,
                             fine_steps, max_iters, float(tol), int(dtype),
                             ctypes.c_void_p(stream_handle), ctypes.byref(ws)))
    return h, ws.value


def fa_batch_bind_workspace(h, ws_ptr: int, nbytes: int):
    _check(load_library().fa_batch_bind_workspace(h, ctypes.c_void_p(ws_ptr), nbytes))


def fa_batch_solve(h, dAs, dXs, iters, last_dx):
    cnt = len(dAs)
    pa = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in dAs])
    px = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in dXs])
    return _check(load_library().fa_batch_solve(h, pa, px, iters, last_dx),
                  allow=(FA_OK, FA_ERR_NOT_CONVERGED))


def fa_batch_autotune(h, dAs, cache_path=None):
    cnt = len(dAs)
    pa = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in dAs])
    _check(load_library().fa_batch_autotune(h, pa, None if cache_path is None else cache_path.encode()))
    return load_library().fa_batch_tuning(h).decode()


def fa_plan_autotune(h):
    _check(load_library().fa_plan_autotune(h))
    return load_library().fa_plan_tuning(h).decode()


def fa_batch_destroy(h):
    if _LIB is not None and h:
        _LIB.fa_batch_destroy(h)


def fa_plan_set_learned(h, d_params):
    _check(load_library().fa_plan_set_learned(h, _ptr(d_params)))


def fa_plan_learned_coefs(h, d_coef):
    _check(load_library().fa_plan_learned_coefs(h, _ptr(d_coef)))


def fa_learned_records_scratch(h) -> int:
    b = ctypes.c_size_t()
    _check(load_library().fa_learned_records_scratch(h, ctypes.byref(b)))
    return b.value


def fa_learned_records(h, dU, dF, d_records, d_scratch, scratch_bytes: int):
    _check(load_library().fa_learned_records(h, _ptr(dU), _ptr(dF), _ptr(d_records),
                                             _ptr(d_scratch), scratch_bytes))


def fa_plan_set_learned_check(h, enable: bool):
    _check(load_library().fa_plan_set_learned_check(h, 1 if enable else 0))


def fa_plan_set_recorder(h, d_records, capacity: int, d_scratch, scratch_bytes: int):
    _check(load_library().fa_plan_set_recorder(h, _ptr(d_records), int(capacity), _ptr(d_scratch),
                                               scratch_bytes))


def fa_mlp_forward(d_params, batch: int, d_feat, feat_stride: int, d_coef, stream_handle: int):
    _check(load_library().fa_mlp_forward(_ptr(d_params), batch, _ptr(d_feat), feat_stride,
                                         _ptr(d_coef), ctypes.c_void_p(stream_handle)))


def fa_mlp_scratch_bytes(batch: int) -> int:
    b = ctypes.c_size_t()
    _check(load_library().fa_mlp_scratch_bytes(batch, ctypes.byref(b)))
    return b.value


def fa_mlp_loss_grad(d_params, batch: int, d_records, d_grad, d_loss, d_scratch,
                     scratch_bytes: int, stream_handle: int):
    _check(load_library().fa_mlp_loss_grad(_ptr(d_params), batch, _ptr(d_records), _ptr(d_grad),
                                           _ptr(d_loss), _ptr(d_scratch), scratch_bytes,
                                           ctypes.c_void_p(stream_handle)))


def fa_mlp_adam(d_params, d_grad, d_m, d_v, step: int, lr: float, beta1: float, beta2: float,
                eps: float, stream_handle: int):
    _check(load_library().fa_mlp_adam(_ptr(d_params), _ptr(d_grad), _ptr(d_m), _ptr(d_v), step,
                                      lr, beta1, beta2, eps, ctypes.c_void_p(stream_handle)))


# --- convenience wrapper ----------------------------------------------------------------------

class Plan:
    """A plan plus its PyTorch-allocated workspace, on the current CUDA stream."""

    def __init__(self, n, flow, T, N, fine_steps, coarse_steps=1, max_iters=None, tol=0.0,
                 fine_dtype="f64", coarse_dtype=None, refine_steps=0, stream=None,
                 coarse_kind=FA_COARSE_EULER, method=FA_METHOD_CLASSICAL, span_drop=0.0,
                 max_basis=0, fine_scheme="default", coarse_scheme="default"):
        import torch

        self.torch = torch
        fd = DTYPES[fine_dtype] if isinstance(fine_dtype, str) else int(fine_dtype)
        cd = fd if coarse_dtype is None else (DTYPES[coarse_dtype] if isinstance(coarse_dtype, str)
                                              else int(coarse_dtype))
        self.desc = fa_problem_desc(n=n, flow=flow, T=float(T), N=N, coarse_steps=coarse_steps,
                                    fine_steps=fine_steps,
                                    max_iters=N if max_iters is None else max_iters,
                                    tol=float(tol), fine_dtype=fd, coarse_dtype=cd,
                                    refine_steps=refine_steps, coarse_kind=int(coarse_kind),
                                    method=int(method), span_drop=float(span_drop),
                                    max_basis=int(max_basis),
                                    fine_scheme=SCHEMES[fine_scheme] if isinstance(fine_scheme, str)
                                    else int(fine_scheme),
                                    coarse_scheme=SCHEMES[coarse_scheme]
                                    if isinstance(coarse_scheme, str) else int(coarse_scheme))
        self.n, self.N = n, N
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle, self.ws_bytes = fa_plan(self.desc, self.stream.cuda_stream)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device="cuda")
        fa_plan_bind_workspace(self.handle, self.ws.data_ptr(), self.ws_bytes)

    def _f64(self, x, shape):
        t = self.torch.as_tensor(x, dtype=self.torch.float64)
        if t.device.type != "cuda":
            t = t.cuda()
        t = t.contiguous()
        assert tuple(t.shape) == tuple(shape), (tuple(t.shape), shape)
        return t

    def set_matrix(self, A):
        self.A = self._f64(A, (self.n, self.n))
        fa_plan_set_matrix(self.handle, self.A)

    def fine_sweep(self, U):
        U = self._f64(U, (self.N, self.n, self.n))
        F = self.torch.empty_like(U)
        fa_fine_sweep(self.handle, U, F)
        return F

    def coarse_sweep(self, U0, D=None, Uold=None):
        n, N = self.n, self.N
        U0 = self._f64(U0, (n, n))
        D = None if D is None else self._f64(D, (N, n, n))
        Unew = self.torch.empty((N + 1, n, n), dtype=self.torch.float64, device="cuda")
        Gnew = self.torch.empty((N, n, n), dtype=self.torch.float64, device="cuda")
        norms = None
        if Uold is not None:
            Uold = self._f64(Uold, (N + 1, n, n))
            norms = self.torch.empty((N, 2), dtype=self.torch.float64, device="cuda")
        fa_coarse_sweep(self.handle, U0, D, Unew, Gnew, norms, Uold)
        return Unew, Gnew, norms

    def refine(self, X):
        X = self._f64(X, (self.n, self.n)).clone()
        fa_refine(self.handle, X)
        return X

    def debug_product(self, L, R):
        L = self._f64(L, (self.n, self.n))
        R = self._f64(R, (self.n, self.n))
        C = self.torch.empty_like(L)
        fa_debug_product(self.handle, L, R, C)
        return C

    def solve(self, A, X0=None, out=None):
        """Returns (X, report dict).  Not converging within max_iters is reported, not raised."""
        A = self._f64(A, (self.n, self.n))
        X0 = None if X0 is None else self._f64(X0, (self.n, self.n))
        X = out if out is not None else self.torch.empty_like(A)
        hist = (ctypes.c_double * max(self.desc.max_iters, 1))()
        rep = fa_report()
        rep.dx_history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        st = fa_parareal_solve(self.handle, A, X0, X, rep)
        return X, _report(rep, hist, st)

    def solve_host(self, A: np.ndarray, X0=None, out=None):
        """The same solve on host arrays (float64, C-contiguous); copies happen inside the call."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        X0 = None if X0 is None else np.ascontiguousarray(X0, dtype=np.float64)
        X = out if out is not None else np.empty_like(A)
        hist = (ctypes.c_double * max(self.desc.max_iters, 1))()
        rep = fa_report()
        rep.dx_history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        st = fa_parareal_solve_host(self.handle, A, X0, X, rep)
        return X, _report(rep, hist, st)

    def autotune(self):
        """Tune the tensor-core launch schedule (the matrix must be set); returns the account."""
        return fa_plan_autotune(self.handle)

    def set_learned(self, params):
        """Install the coefficient network (float32 blob of FA_MLP_PARAMS values)."""
        self.params = self.torch.as_tensor(params, dtype=self.torch.float32).cuda().contiguous()
        assert self.params.numel() == FA_MLP_PARAMS
        fa_plan_set_learned(self.handle, self.params)

    def set_learned_check(self, enable=True):
        """Opt-in fallback: Euler G for the rest of a solve whose first convergence measure
        exceeds Euler G's (costs one extra fine sweep per solve)."""
        fa_plan_set_learned_check(self.handle, enable)

    def learned_coefs(self):
        c = self.torch.empty((self.N, FA_MLP_COEFS), dtype=self.torch.float32, device="cuda")
        fa_plan_learned_coefs(self.handle, c)
        return c

    def _records_scratch(self):
        if getattr(self, "rec_scratch", None) is None:
            nb = fa_learned_records_scratch(self.handle)
            self.rec_scratch = self.torch.empty(nb, dtype=self.torch.uint8, device="cuda")
        return self.rec_scratch

    def records(self, U, F):
        """Pair records (N, FA_RECORD_DOUBLES) of the states U[b] and their fine images F[b]."""
        U = self._f64(U, (self.N, self.n, self.n))
        F = self._f64(F, (self.N, self.n, self.n))
        out = self.torch.empty((self.N, FA_RECORD_DOUBLES), dtype=self.torch.float64, device="cuda")
        sc = self._records_scratch()
        fa_learned_records(self.handle, U, F, out, sc, sc.numel())
        return out

    def set_recorder(self, capacity):
        """Record up to `capacity` training pairs during the next solves (None: off)."""
        if capacity is None:
            fa_plan_set_recorder(self.handle, None, 0, None, 0)
            self.rec_buf = None
            return None
        self.rec_buf = self.torch.zeros((capacity, FA_RECORD_DOUBLES), dtype=self.torch.float64,
                                        device="cuda")
        sc = self._records_scratch()
        fa_plan_set_recorder(self.handle, self.rec_buf, capacity, sc, sc.numel())
        return self.rec_buf

    def close(self):
        if getattr(self, "handle", None):
            fa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Aima:
    """Algorithm 8 (accelerated inverse-matrix approximation) through fa_aima_plan / fa_aima, with
    a PyTorch-allocated workspace on the current CUDA stream."""

    def __init__(self, n, dtype="f64", stream=None):
        import torch

        self.torch = torch
        self.n = n
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        _check(load_library().fa_aima_plan(ctypes.byref(h), n,
                                           DTYPES[dtype] if isinstance(dtype, str) else int(dtype),
                                           ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(nb)))
        self.handle = h
        self.ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
        fa_plan_bind_workspace(self.handle, self.ws.data_ptr(), nb.value)

    def run(self, A, X0, E, dt, steps):
        """Returns (X^(steps), [||I - A X^(k)||_F for k = 0..steps])."""
        t = lambda x: self.torch.as_tensor(x, dtype=self.torch.float64).cuda().contiguous()
        A, X0, E = t(A), t(X0), t(E)
        X = self.torch.empty_like(A)
        res = (ctypes.c_double * (steps + 1))()
        _check(load_library().fa_aima(self.handle, _ptr(A), _ptr(X0), _ptr(E), float(dt), steps,
                                      _ptr(X), res))
        return X, list(res)

    def close(self):
        if getattr(self, "handle", None):
            fa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The coefficient network's kernels on one parameter blob (training state on the device)."""

    def __init__(self, params, stream=None):
        import torch

        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = torch.as_tensor(params, dtype=torch.float32).cuda().contiguous().clone()
        assert self.params.numel() == FA_MLP_PARAMS
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.step = 0
        self.scratch = None

    def forward(self, feat, stride=None):
        """feat: (B, >= 8) float64 CUDA tensor (e.g. records) -> (B, 4) float32 coefficients."""
        feat = feat.contiguous()
        B = feat.shape[0]
        out = self.torch.empty((B, FA_MLP_COEFS), dtype=self.torch.float32, device="cuda")
        fa_mlp_forward(self.params, B, feat, feat.shape[1] if stride is None else stride, out,
                       self.stream.cuda_stream)
        return out

    def loss_grad(self, records):
        """Mean loss and gradient of a batch of records (float64 CUDA (B, FA_RECORD_DOUBLES))."""
        records = records.contiguous()
        B = records.shape[0]
        need = fa_mlp_scratch_bytes(B)
        if self.scratch is None or self.scratch.numel() < need:
            self.scratch = self.torch.empty(need, dtype=self.torch.uint8, device="cuda")
        fa_mlp_loss_grad(self.params, B, records, self.grad, self.loss, self.scratch,
                         self.scratch.numel(), self.stream.cuda_stream)
        return self.loss, self.grad

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        fa_mlp_adam(self.params, self.grad, self.m, self.v, self.step, lr, beta1, beta2, eps,
                    self.stream.cuda_stream)


class Batch:
    """Many independent problems (orders, flows, horizons, Euler substeps) solved together."""

    def __init__(self, ns, flows, Ts, coarse_steps, N, fine_steps, max_iters, tol=0.0,
                 dtype="bf16x6", stream=None):
        import torch

        self.torch = torch
        self.ns = list(ns)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle, self.ws_bytes = fa_batch_plan(
            self.ns, list(flows), list(Ts), list(coarse_steps), N, fine_steps, max_iters, tol,
            DTYPES[dtype] if isinstance(dtype, str) else int(dtype), self.stream.cuda_stream)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device="cuda")
        fa_batch_bind_workspace(self.handle, self.ws.data_ptr(), self.ws_bytes)

    def autotune(self, As, cache_path=None):
        """Tune the launch schedule on these matrices (see fa_batch_autotune); returns the account."""
        return fa_batch_autotune(self.handle, [a.contiguous() for a in As], cache_path)

    def solve(self, As):
        """As: list of (n_i, n_i) float64 CUDA tensors.  Returns (list of X_i, iters, last_dx, status)."""
        torch = self.torch
        As = [a.contiguous() for a in As]
        Xs = [torch.empty_like(a) for a in As]
        cnt = len(As)
        iters = (ctypes.c_int * cnt)()
        dx = (ctypes.c_double * cnt)()
        st = fa_batch_solve(self.handle, As, Xs, iters, dx)
        return Xs, list(iters), list(dx), st

    def close(self):
        if getattr(self, "handle", None):
            fa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _report(rep: fa_report, hist, status) -> dict:
    return {"iters": rep.iters, "converged": bool(rep.converged), "last_dx": rep.last_dx,
            "dx_history": [hist[i] for i in range(rep.iters)], "t_init_ms": rep.t_init_ms,
            "t_fine_ms": rep.t_fine_ms, "t_coarse_ms": rep.t_coarse_ms,
            "t_refine_ms": rep.t_refine_ms, "status": status,
            "g_fallback_iter": rep.g_fallback_iter, "coef_fallbacks": rep.coef_fallbacks,
            "records": rep.records, "basis_dim": rep.basis_dim, "fine_blocks": rep.fine_blocks,
            "double_angle_steps": rep.double_angle_steps}
