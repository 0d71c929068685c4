"""Python binding of libipt (include/ipt.h): argument marshalling only.

Every step of the solver runs inside libipt's CUDA kernels; this module turns
torch tensors into pointers, sizes and dtype codes and calls the C ABI with
ctypes.  Importing it loads ``_lib/libipt.so`` and raises ImportError when
the library is missing: there is no fallback path.

Layouts: M is row-major (n, n); Z is column-major n x k, i.e. stored as a
(k, n) tensor whose row c is the eigenvector of column c; the functions
return it as the (n, k) view ``Zt.T``.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libipt.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libipt.so is not built ({_LIB_PATH}); run __graft_entry__.build() first")
_lib = C.CDLL(_LIB_PATH)

MAX_HISTORY = 128

STATUS = {0: "OK", 1: "MAXITER", 2: "DIVERGED", 3: "DEGENERATE_THETA", 4: "INVALID_ARG",
          5: "CUDA_ERROR", 6: "DEVICE_TIMEOUT", 7: "UNSUPPORTED", 8: "INACCURATE"}
PRECISION = {"f64": 0, "f32": 1, "bf16": 2, "bf16x3": 3, "staged": 4, "fp16": 5, "fp16x3": 6,
             "f32c": 7}
PRECISION_NAME = {v: k for k, v in PRECISION.items()}
PRECISION_NAME[-1] = "none"  # product-free first evaluation (Z = E, P = Delta E)
STOP = {"increment": 0, "residual": 1}
DTYPE = {torch.float64: 0, torch.float32: 1}


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("stop", C.c_int), ("diverge_bound", C.c_double),
                ("stage_switch", C.c_double), ("staged_bf16", C.c_int), ("verify_fp64", C.c_int),
                ("record_timing", C.c_int), ("z0", C.c_void_p), ("product_kernel", C.c_int),
                ("accel", C.c_int), ("acx_sigma", C.c_int), ("damping_model", C.c_void_p),
                ("csr_window", C.c_int), ("epilogue_operand", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("stage_iters", C.c_int * 2),
                ("increment", C.c_double), ("rho", C.c_double), ("rho_fp64", C.c_double),
                ("r0", C.c_double), ("kernel_launches", C.c_int),
                ("product_launches", C.c_int * 2), ("product_ms", C.c_double * 2),
                ("prepass_ms", C.c_double), ("setup_ms", C.c_double),
                ("finalize_ms", C.c_double), ("wall_ms", C.c_double), ("history_len", C.c_int),
                ("hist_increment", C.c_double * MAX_HISTORY),
                ("hist_rho", C.c_double * MAX_HISTORY),
                ("hist_stage", C.c_int * MAX_HISTORY), ("rows_evaluated", C.c_longlong),
                ("acc_launches", C.c_int), ("acc_ms", C.c_double), ("rho_error", C.c_double),
                ("epilogue_operands", C.c_int)]

    def to_dict(self) -> dict:
        h = self.history_len
        return {"status": STATUS.get(self.status, str(self.status)), "status_code": self.status,
                "iterations": self.iterations, "stage_iters": list(self.stage_iters),
                "increment": self.increment, "rho": self.rho, "rho_fp64": self.rho_fp64,
                "r0": self.r0, "kernel_launches": self.kernel_launches,
                "product_launches": list(self.product_launches),
                "product_ms": list(self.product_ms), "prepass_ms": self.prepass_ms,
                "setup_ms": self.setup_ms, "finalize_ms": self.finalize_ms,
                "wall_ms": self.wall_ms,
                "hist_increment": list(self.hist_increment[:h]),
                "hist_rho": list(self.hist_rho[:h]),
                "hist_stage": [PRECISION_NAME.get(s, s) for s in self.hist_stage[:h]],
                "rows_evaluated": self.rows_evaluated, "acc_launches": self.acc_launches,
                "acc_ms": self.acc_ms, "rho_error": self.rho_error,
                "epilogue_operands": self.epilogue_operands}


_vp, _i64, _i32, _d = C.c_void_p, C.c_int64, C.c_int, C.c_double
_lib.ipt_options_default.argtypes = [C.POINTER(Options)]
_lib.ipt_options_default.restype = None
_lib.ipt_status_string.argtypes = [_i32]
_lib.ipt_status_string.restype = C.c_char_p
_lib.ipt_create.argtypes = [C.POINTER(_vp), _vp]
_lib.ipt_create.restype = _i32
_lib.ipt_destroy.argtypes = [_vp]
_lib.ipt_destroy.restype = _i32
_SOLVE_ARGS = [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _vp, _d, _i32, C.POINTER(Options), _vp, _vp,
               _i64, _i32, C.POINTER(Result)]
_lib.ipt_solve_dense.argtypes = _SOLVE_ARGS
_lib.ipt_solve_dense.restype = _i32
_lib.ipt_solve_dense_host.argtypes = _SOLVE_ARGS
_lib.ipt_solve_dense_host.restype = _i32
_lib.ipt_step_dense.argtypes = [_vp, _i64, _vp, _i64, _i32, _vp, _i64, _vp, _i32, _vp, _vp, _i64,
                                _i32, _vp, C.POINTER(_d)]
_lib.ipt_step_dense.restype = _i32
_lib.ipt_solve_csr.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _d, _i32,
                               C.POINTER(Options), _vp, _vp, _i64, _i32, C.POINTER(Result)]
_lib.ipt_solve_csr.restype = _i32

_lib.ipt_residual_dense_noalloc.argtypes = [_i64, _vp, _i64, _i32, _i64, _vp, _i64, _i32, _vp,
                                           _vp, _vp]
_lib.ipt_residual_dense_noalloc.restype = _i32

LIB_PATH = _LIB_PATH
lib = _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        t = t.to(dtype)
    return t.contiguous()


PRODUCT_KERNEL = {"auto": 0, "single": 1, "pair": 2}
ACCEL = {None: 0, "none": 0, "acx": 1, "damped": 2, "anderson": 3, "mixing": 4}


def make_options(precision="staged", stop="residual", diverge_bound=1e8, stage_switch=0.1,
                 verify_fp64=False, z0=None, staged_bf16=False, record_timing=False,
                 product_kernel="auto") -> Options:
    o = Options()
    _lib.ipt_options_default(C.byref(o))
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.stop = STOP[stop] if isinstance(stop, str) else int(stop)
    o.diverge_bound = diverge_bound
    o.stage_switch = stage_switch
    o.verify_fp64 = 1 if verify_fp64 else 0
    o.staged_bf16 = 1 if staged_bf16 else 0
    o.record_timing = 1 if record_timing else 0
    o.z0 = None if z0 is None else z0.data_ptr()
    o.product_kernel = (PRODUCT_KERNEL[product_kernel] if isinstance(product_kernel, str)
                        else int(product_kernel))
    return o


class Solver:
    """A libipt handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = _lib.ipt_create(C.byref(h), C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise RuntimeError(f"ipt_create failed: {STATUS.get(st, st)}")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.ipt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ dense
    def solve_dense(self, M, theta=None, cols=None, tol=1e-6, max_iter=100, precision="staged",
                    stop="residual", z_dtype=torch.float32, verify_fp64=False, z0=None,
                    diverge_bound=1e8, stage_switch=0.1, staged_bf16=False,
                    record_timing=False, product_kernel="auto", accel=None,
                    acx_sigma="column", damping_model=None, epilogue_operand=True):
        """Alg. 2 / Alg. 1 on the GPU.  Returns (lam [k] f64, Z (n, k) view, info dict).

        product_kernel: "auto", "single" (one CTA per tile) or "pair" (two CTAs
        per 256-row tile); selects the tensor-core product kernel only.
        accel: None (Picard update), "acx" (Alg. 3, with acx_sigma "column" —
        one step length per column — or "global"), "damped" (learned damping,
        damping_model = the model's FP16 parameters as a CUDA tensor),
        "anderson" (depth-one Anderson mixing per column) or "mixing" (learned
        damping and mixing, damping_model = the mixing model's parameters).
        epilogue_operand: staged solves only; False makes the pre-pass write
        every product's operand (the epilogue writes it by default)."""
        M = _dev(M, name="M")
        n = M.shape[0]
        if M.dim() != 2 or M.shape[1] != n or M.dtype not in DTYPE:
            raise ValueError("M must be a square float32/float64 CUDA matrix")
        theta = _dev(theta, torch.float64, "theta")
        cols = _dev(cols, torch.int32, "cols")
        k = n if cols is None else cols.numel()
        lam = torch.empty(k, dtype=torch.float64, device=M.device)
        Zt = torch.empty((k, n), dtype=z_dtype, device=M.device)
        if z0 is not None:
            z0 = _dev(z0, z_dtype, "z0")
            z0t = z0.t().contiguous() if z0.shape == (n, k) else z0
        else:
            z0t = None
        o = make_options(precision, stop, diverge_bound, stage_switch, verify_fp64, z0t,
                         staged_bf16, record_timing, product_kernel)
        if accel not in ACCEL or acx_sigma not in ("column", "global"):
            raise ValueError("accel must be None, 'acx', 'damped', 'anderson' or 'mixing'; "
                             "acx_sigma 'column' or 'global'")
        o.accel = ACCEL[accel]
        o.acx_sigma = 1 if acx_sigma == "global" else 0
        o.epilogue_operand = 1 if epilogue_operand else 0
        if damping_model is not None:
            damping_model = _dev(damping_model, torch.float16, "damping_model")
            o.damping_model = damping_model.data_ptr()
        r = Result()
        _lib.ipt_solve_dense(self._h, n, _ptr(M), M.stride(0), DTYPE[M.dtype], _ptr(theta), k,
                             _ptr(cols), float(tol), int(max_iter), C.byref(o), _ptr(lam),
                             _ptr(Zt), n, DTYPE[z_dtype], C.byref(r))
        return lam, Zt.t(), r.to_dict()

    def solve_dense_host(self, M, theta=None, cols=None, tol=1e-6, max_iter=100,
                         precision="staged", stop="residual", z_dtype=torch.float32,
                         lam_out=None, zt_out=None, record_timing=False, accel=None,
                         acx_sigma="column", damping_model=None):
        """The same solve from host tensors (pinned for speed); copies are inside the call.
        accel / acx_sigma / damping_model as in solve_dense (the model stays a CUDA tensor)."""
        if M.is_cuda:
            raise ValueError("solve_dense_host takes host tensors")
        M = M.contiguous()
        n = M.shape[0]
        theta = None if theta is None else theta.to(torch.float64).contiguous()
        cols = None if cols is None else cols.to(torch.int32).contiguous()
        k = n if cols is None else cols.numel()
        lam = lam_out if lam_out is not None else torch.empty(k, dtype=torch.float64)
        Zt = zt_out if zt_out is not None else torch.empty((k, n), dtype=z_dtype)
        o = make_options(precision, stop, record_timing=record_timing)
        if accel not in ACCEL:
            raise ValueError("accel must be None, 'acx', 'damped', 'anderson' or 'mixing'")
        o.accel = ACCEL[accel]
        o.acx_sigma = 1 if acx_sigma == "global" else 0
        if damping_model is not None:
            o.damping_model = damping_model.data_ptr()
        r = Result()
        _lib.ipt_solve_dense_host(self._h, n, _ptr(M), M.stride(0), DTYPE[M.dtype], _ptr(theta),
                                  k, _ptr(cols), float(tol), int(max_iter), C.byref(o), _ptr(lam),
                                  _ptr(Zt), n, DTYPE[Zt.dtype], C.byref(r))
        return lam, Zt.t(), r.to_dict()

    def solve_batched(self, sizes, M, theta=None, tol=1e-6, max_iter=100, stop="residual",
                      diverge_bound=1e8, record_timing=False, precision="f32"):
        """Many dense problems in one launch (Alg. 2 on each, all eigenpairs).

        sizes: the problem orders (host sequence); M: CUDA float32 tensor with the
        problems packed row-major back to back; theta: packed CUDA float64 or None.
        precision: "f32" (FP32 SIMT product), "bf16x3" (split-BF16 tensor-core
        product, three passes) or "bf16" (one BF16 pass).
        Returns (lam packed f64, Z packed f32 (each block column-major), status
        int32[count], iterations int32[count], info dict)."""
        sizes = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
        M = _dev(M, torch.float32, "M").reshape(-1)
        theta = _dev(theta, torch.float64, "theta")
        count = len(sizes)
        if M.numel() != int(np.sum(sizes * sizes)):
            raise ValueError("M does not hold the packed problems of the given sizes")
        lam = torch.empty(int(np.sum(sizes)), dtype=torch.float64, device=M.device)
        Z = torch.empty(M.numel(), dtype=torch.float32, device=M.device)
        status = torch.empty(count, dtype=torch.int32, device=M.device)
        iters = torch.empty(count, dtype=torch.int32, device=M.device)
        if precision not in ("f32", "bf16x3", "bf16"):
            raise ValueError("batched precision must be 'f32', 'bf16x3' or 'bf16'")
        o = make_options(precision, stop, diverge_bound, record_timing=record_timing)
        r = Result()
        _lib.ipt_solve_batched(self._h, count,
                               sizes.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(M),
                               _ptr(theta), float(tol), int(max_iter), C.byref(o), _ptr(lam),
                               _ptr(Z), _ptr(status), _ptr(iters), C.byref(r))
        return lam, Z, status, iters, r.to_dict()

    @property
    def batched_tiles(self):
        """Output tile per size class (n <= 64, <= 256, <= 1024) of solve_batched;
        0 = not tuned yet.  Assign a 3-sequence of 32/64/0 to fix or re-tune them."""
        t = (C.c_int32 * 3)()
        if _lib.ipt_get_batched_tiles(self._h, t) != 0:
            raise RuntimeError("ipt_get_batched_tiles failed")
        return tuple(t)

    @batched_tiles.setter
    def batched_tiles(self, tiles):
        t = (C.c_int32 * 3)(*[int(x) for x in tiles])
        if _lib.ipt_set_batched_tiles(self._h, t) != 0:
            raise ValueError(f"batched tiles must be 32, 64 or 0, got {tuple(tiles)}")

    def step_dense(self, M, Z, theta=None, cols=None, precision="f32"):
        """One evaluation of F (Eq. dyn) at Z (n, k).  Returns (F (n, k), lam, norms)."""
        M = _dev(M, name="M")
        n = M.shape[0]
        theta = _dev(theta, torch.float64, "theta")
        cols = _dev(cols, torch.int32, "cols")
        k = n if cols is None else cols.numel()
        Zt = _dev(Z, name="Z").t().contiguous()
        Ft = torch.empty_like(Zt)
        lam = torch.empty(k, dtype=torch.float64, device=M.device)
        norms = (C.c_double * 3)()
        p = PRECISION[precision] if isinstance(precision, str) else int(precision)
        st = _lib.ipt_step_dense(self._h, n, _ptr(M), M.stride(0), DTYPE[M.dtype], _ptr(theta), k,
                                 _ptr(cols), p, _ptr(Zt), _ptr(Ft), n, DTYPE[Zt.dtype], _ptr(lam),
                                 norms)
        if st != 0:
            raise RuntimeError(f"ipt_step_dense: {STATUS.get(st, st)}")
        return Ft.t(), lam, {"increment_abs": norms[0], "z_norm": norms[1],
                             "residual_abs": norms[2]}

    # ------------------------------------------------------------------ sparse
    def solve_csr(self, rowptr, colind, vals, n, theta=None, cols=None, tol=1e-6, max_iter=100,
                  precision="f32", stop="residual", z_dtype=torch.float32, diverge_bound=1e8,
                  record_timing=False, window=True, verify_fp64=False, accel=None,
                  acx_sigma="column"):
        """Sparse M (CSR, all stored entries of M).  Returns (lam, Z (n, k) view, info).

        window: evaluate only the rows that can be nonzero (exact); False = all rows.
        verify_fp64: info["rho_fp64"] = the result's residual recomputed in FP64.
        accel: None (Picard update) or "acx" (Alg. 3, acx_sigma "column" or "global")."""
        if accel not in (None, "none", "acx") or acx_sigma not in ("column", "global"):
            raise ValueError("sparse accel must be None or 'acx'; acx_sigma 'column' or "
                             "'global'")
        rowptr = _dev(rowptr, torch.int32, "rowptr")
        colind = _dev(colind, torch.int32, "colind")
        vals = _dev(vals, name="vals")
        theta = _dev(theta, torch.float64, "theta")
        cols = _dev(cols, torch.int32, "cols")
        k = n if cols is None else cols.numel()
        lam = torch.empty(k, dtype=torch.float64, device=vals.device)
        Zt = torch.empty((k, n), dtype=z_dtype, device=vals.device)
        o = make_options(precision, stop, diverge_bound, record_timing=record_timing,
                         verify_fp64=verify_fp64)
        o.csr_window = 1 if window else 0
        o.accel = 1 if accel == "acx" else 0
        o.acx_sigma = 1 if acx_sigma == "global" else 0
        r = Result()
        _lib.ipt_solve_csr(self._h, n, colind.numel(), _ptr(rowptr), _ptr(colind), _ptr(vals),
                           DTYPE[vals.dtype], _ptr(theta), k, _ptr(cols), float(tol),
                           int(max_iter), C.byref(o), _ptr(lam), _ptr(Zt), n, DTYPE[z_dtype],
                           C.byref(r))
        return lam, Zt.t(), r.to_dict()


_lib.ipt_check_map_division.argtypes = [_i64, _vp, _vp, _vp, _vp]
_lib.ipt_check_map_division.restype = _i32


_lib.ipt_check_conversions.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.ipt_check_conversions.restype = _i32


def check_conversions(x, stream=None):
    """The integer-ALU conversions of the sparse setup for a CUDA float64 vector:
    returns (hi, lo, f, back, ok) as ipt_check_conversions defines them
    (synchronises the stream)."""
    x = _dev(x, torch.float64, "x").contiguous()
    hi = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
    lo = torch.empty_like(hi)
    f = torch.empty_like(hi)
    back = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
    ok = torch.empty(x.numel(), dtype=torch.int32, device=x.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = _lib.ipt_check_conversions(x.numel(), _ptr(x), _ptr(hi), _ptr(lo), _ptr(f), _ptr(back),
                                    _ptr(ok), C.c_void_p(s.cuda_stream))
    if st != 0:
        raise RuntimeError(f"ipt_check_conversions: {STATUS.get(st, st)}")
    s.synchronize()
    return hi, lo, f, back, ok


def check_map_division(gap, u, stream=None):
    """u / gap as the FP32 map computes it (refined reciprocal), for CUDA float32
    vectors of equal length; returns the quotients (synchronises the stream)."""
    gap = _dev(gap, torch.float32, "gap").contiguous()
    u = _dev(u, torch.float32, "u").contiguous()
    if gap.numel() != u.numel():
        raise ValueError("gap and u must have the same length")
    q = torch.empty_like(gap)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = _lib.ipt_check_map_division(gap.numel(), _ptr(gap), _ptr(u), _ptr(q),
                                     C.c_void_p(s.cuda_stream))
    if st != 0:
        raise RuntimeError(f"ipt_check_map_division: {STATUS.get(st, st)}")
    s.synchronize()
    return q


def check_bounded_wait(arrive, limit_s=0.2, stream=None):
    """Run the product kernel's bounded barrier wait in a one-CTA kernel (see
    ipt_check_bounded_wait): returns (succeeded, seconds waited)."""
    ok = C.c_int32()
    waited = C.c_double()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    st = _lib.ipt_check_bounded_wait(int(arrive), float(limit_s), C.c_void_p(s), C.byref(ok),
                                     C.byref(waited))
    if st != 0:
        raise RuntimeError(f"ipt_check_bounded_wait: {STATUS.get(st, st)}")
    return bool(ok.value), waited.value


def _batched_argtypes():
    _lib.ipt_solve_batched.argtypes = [_vp, _i64, C.POINTER(C.c_int64), _vp, _vp, _d, _i32,
                                       C.POINTER(Options), _vp, _vp, _vp, _vp,
                                       C.POINTER(Result)]
    _lib.ipt_solve_batched.restype = _i32
    _lib.ipt_check_bounded_wait.argtypes = [C.c_int, _d, _vp, C.POINTER(C.c_int32),
                                            C.POINTER(C.c_double)]
    _lib.ipt_check_bounded_wait.restype = _i32
    for name in ("ipt_set_batched_tiles", "ipt_get_batched_tiles"):
        getattr(_lib, name).argtypes = [_vp, C.POINTER(C.c_int32)]
        getattr(_lib, name).restype = _i32


_batched_argtypes()


_lib.ipt_damping_forward.argtypes = [_i64, _vp, _vp, _vp, _vp]
_lib.ipt_damping_forward.restype = _i32
_lib.ipt_damping_grad.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.ipt_damping_grad.restype = _i32
_lib.ipt_damping_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float,
                                  C.c_float, _i32, _vp]
_lib.ipt_damping_adam.restype = _i32
DAMPING_PARAMS = 4673


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def damping_forward(params, X, alpha=None, stream=None):
    """alpha (B,) float32 of the damping model (params: CUDA float16 [4673]) at
    feature rows X (B, 6) float32; runs on ``stream`` without synchronising."""
    X = _dev(X, torch.float32, "X").contiguous()
    params = _dev(params, torch.float16, "params")
    if alpha is None:
        alpha = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    st = _lib.ipt_damping_forward(X.shape[0], _ptr(params), _ptr(X), _ptr(alpha),
                                  _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_damping_forward: {STATUS.get(st, st)}")
    return alpha


def damping_grad(params, X, target, grad, loss, stream=None):
    """Adds the mean-squared-error gradient (and the loss) of the model over (X, target)."""
    X = _dev(X, torch.float32, "X").contiguous()
    st = _lib.ipt_damping_grad(X.shape[0], _ptr(params), _ptr(X), _ptr(target), _ptr(grad),
                               _ptr(loss), _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_damping_grad: {STATUS.get(st, st)}")


def damping_adam(master, params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None):
    """One Adam step on the FP32 master parameters; writes the FP16 params, zeroes grad."""
    st = _lib.ipt_damping_adam(_ptr(master), _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                               float(lr), float(beta1), float(beta2), float(eps), int(step),
                               _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_damping_adam: {STATUS.get(st, st)}")


_lib.ipt_mixing_forward.argtypes = [_i64, _vp, _vp, _vp, _vp]
_lib.ipt_mixing_forward.restype = _i32
_lib.ipt_mixing_grad.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.ipt_mixing_grad.restype = _i32
_lib.ipt_mixing_adam.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float,
                                 C.c_float, _i32, _vp]
_lib.ipt_mixing_adam.restype = _i32
MIXING_PARAMS = 4802


def mixing_forward(params, X, out=None, stream=None):
    """(B, 2) float32 rows (alpha, gamma) of the mixing model (params: CUDA float16
    [4802]) at feature rows X (B, 7) float32; runs on ``stream`` without synchronising."""
    X = _dev(X, torch.float32, "X").contiguous()
    params = _dev(params, torch.float16, "params")
    if out is None:
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
    st = _lib.ipt_mixing_forward(X.shape[0], _ptr(params), _ptr(X), _ptr(out),
                                 _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_mixing_forward: {STATUS.get(st, st)}")
    return out


def mixing_grad(params, X, target, grad, loss, stream=None):
    """Adds the mean-squared-error gradient (and the loss) of the mixing model over
    (X, target (B, 2))."""
    X = _dev(X, torch.float32, "X").contiguous()
    target = _dev(target, torch.float32, "target").contiguous()
    st = _lib.ipt_mixing_grad(X.shape[0], _ptr(params), _ptr(X), _ptr(target), _ptr(grad),
                              _ptr(loss), _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_mixing_grad: {STATUS.get(st, st)}")


def mixing_adam(master, params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8,
                stream=None):
    """One Adam step on the mixing model's FP32 master parameters."""
    st = _lib.ipt_mixing_adam(_ptr(master), _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                              float(lr), float(beta1), float(beta2), float(eps), int(step),
                              _stream_ptr(stream))
    if st != 0:
        raise RuntimeError(f"ipt_mixing_adam: {STATUS.get(st, st)}")


def residual_dense_noalloc(M, Z, lam, out=None, stream=None):
    """||M Z - Z Lambda||_F in FP64 through the allocation-free C entry point.

    M (n, n) row-major CUDA float32/float64 matrix (unit stride along a row),
    Z (n, k) CUDA float32/float64 given as the (n, k) view the solvers return
    (column-major storage), lam (k,) contiguous CUDA float64.  Writes the norm
    into ``out`` (a CUDA float64 tensor of one element, created here when not
    given) without synchronising; returns (status code, out).  The C call
    itself allocates nothing on the device.  Any other layout or dtype raises
    ValueError: the C call would read it as a different matrix.
    """
    if M.dim() != 2 or not M.is_cuda or M.dtype not in DTYPE or M.shape[0] != M.shape[1]:
        raise ValueError("M must be a square CUDA float32/float64 matrix")
    if M.stride(1) != 1 or M.stride(0) < M.shape[0]:
        raise ValueError("M must be row-major with unit stride along a row")
    n = M.shape[0]
    if Z.dim() != 2 or not Z.is_cuda or Z.dtype not in DTYPE or Z.shape[0] != n:
        raise ValueError("Z must be an (n, k) CUDA float32/float64 matrix")
    k = Z.shape[1]
    Zt = Z.t()
    if Zt.stride(1) != 1 or Zt.stride(0) < n:
        raise ValueError("Z must be column-major (the (n, k) view of a (k, n) tensor)")
    if (not lam.is_cuda or lam.dtype != torch.float64 or lam.dim() != 1 or lam.numel() != k
            or not lam.is_contiguous()):
        raise ValueError("lam must be a contiguous CUDA float64 vector of k entries")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=M.device)
    elif not out.is_cuda or out.dtype != torch.float64 or out.numel() < 1 or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA float64 tensor")
    s = stream if stream is not None else torch.cuda.current_stream()
    st = _lib.ipt_residual_dense_noalloc(n, _ptr(M), M.stride(0), DTYPE[M.dtype], k, _ptr(Zt),
                                         Zt.stride(0), DTYPE[Zt.dtype], _ptr(lam), _ptr(out),
                                         C.c_void_p(s.cuda_stream))
    return st, out


_default: Solver | None = None


def default_solver() -> Solver:
    global _default
    if _default is None:
        _default = Solver()
    return _default


def solve_dense(M, **kw):
    return default_solver().solve_dense(M, **kw)


def step_dense(M, Z, **kw):
    return default_solver().step_dense(M, Z, **kw)


def solve_csr(rowptr, colind, vals, n, **kw):
    return default_solver().solve_csr(rowptr, colind, vals, n, **kw)
