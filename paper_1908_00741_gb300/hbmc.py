"""Python binding of libhbmc.so (ctypes): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  Function names follow the C ABI in include/hbmc.h.

If libhbmc.so has not been built, the first call raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libhbmc.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = 1
ERR_NOT_SPD_PIVOT = 2
ERR_BREAKDOWN = 3
NOT_CONVERGED = 4
ERR_TIMEOUT = 5
ERR_CUDA = 6
ERR_OOM = 7
ERR_NOT_FACTORED = 8
ERR_NO_DEVICE = 9

BLOCK_ALGEBRAIC = 0
BLOCK_BOXES = 1
PREC_F64 = 0
PREC_F32 = 1
LOOP_GRAPH = 0
LOOP_HOST = 1
LOOP_PERSISTENT = 2

EXPORTED = [
    "hbmc_default_options", "hbmc_build", "hbmc_destroy", "hbmc_last_error",
    "hbmc_status_string", "hbmc_info", "hbmc_get_ordering", "hbmc_get_matrix", "hbmc_get_split", "hbmc_get_vslice",
    "hbmc_get_dag_deps",
    "hbmc_set_stream", "hbmc_set_precision", "hbmc_ic0", "hbmc_get_factor",
    "hbmc_precond", "hbmc_iccg", "hbmc_iccg_host", "hbmc_residual_history",
    "hbmc_fwd_bar", "hbmc_bwd_bar", "hbmc_spmv_bar", "hbmc_profile_kernels",
    "hbmc_debug_stall", "hbmc_debug_convert", "hbmc_spmv_dot_static", "hbmc_sor", "hbmc_sor_bar", "hbmc_ilu0", "hbmc_get_factor_u", "hbmc_bicgstab",
    "hbmc_batch_build", "hbmc_batch_build_w", "hbmc_batch_destroy", "hbmc_batch_last_error", "hbmc_batch_info",
    "hbmc_batch_set_stream", "hbmc_batch_set_precision", "hbmc_batch_ic0", "hbmc_batch_iccg",
    "hbmc_batch_autotune", "hbmc_batch_autotune_w", "hbmc_batch_features",
    "hbmc_features", "hbmc_shift_grid", "hbmc_mlp_num_params", "hbmc_mlp_create", "hbmc_mlp_destroy",
    "hbmc_mlp_last_error", "hbmc_mlp_set_params", "hbmc_mlp_get_params", "hbmc_mlp_forward",
    "hbmc_mlp_gradient", "hbmc_mlp_train", "hbmc_predict_shift", "hbmc_ic0_auto",
]


class Options(ctypes.Structure):
    _fields_ = [("blocking", ctypes.c_int32), ("grid", ctypes.c_int64 * 3),
                ("box", ctypes.c_int32 * 3), ("precision", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("device", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("sweep_tpb", ctypes.c_int32), ("sweep_kernel", ctypes.c_int32),
                ("nonsymmetric", ctypes.c_int32), ("sell_split", ctypes.c_int32),
                ("sell_split_cost", ctypes.c_int32), ("sell_vslice", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("nnz_lower", ctypes.c_int64), ("bs", ctypes.c_int32), ("w", ctypes.c_int32),
                ("nc", ctypes.c_int32), ("nblocks", ctypes.c_int64), ("ntiles", ctypes.c_int64),
                ("sell_entries_a", ctypes.c_int64), ("sell_entries_l", ctypes.c_int64),
                ("sell_entries_u", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("factored", ctypes.c_int32), ("device_bytes", ctypes.c_size_t),
                ("last_iters", ctypes.c_int64), ("last_launches", ctypes.c_int64),
                ("split_rows", ctypes.c_int64), ("split_pieces", ctypes.c_int64),
                ("sell_entries_split", ctypes.c_int64), ("sell_entries_vslice", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HbmcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libhbmc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(_LIB_PATH)
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        sigs = {
            "hbmc_default_options": (None, [P]),
            "hbmc_build": (I32, [I64, P, P, P, I32, I32, P, P]),
            "hbmc_destroy": (None, [P]),
            "hbmc_last_error": (ctypes.c_char_p, [P]),
            "hbmc_status_string": (ctypes.c_char_p, [I32]),
            "hbmc_info": (I32, [P, P]),
            "hbmc_get_ordering": (I32, [P, P, P, P, P]),
            "hbmc_get_matrix": (I32, [P, P, P, P]),
            "hbmc_get_split": (I32, [P, P]),
            "hbmc_get_vslice": (I32, [P, P]),
            "hbmc_get_dag_deps": (I32, [P, I32, P, P, I64, P]),
            "hbmc_set_stream": (I32, [P, P]),
            "hbmc_set_precision": (I32, [P, I32]),
            "hbmc_ic0": (I32, [P, D, P]),
            "hbmc_get_factor": (I32, [P, P, P]),
            "hbmc_precond": (I32, [P, P, P]),
            "hbmc_iccg": (I32, [P, P, P, D, I64, P, P, P]),
            "hbmc_iccg_host": (I32, [P, P, P, D, I64, P, P, P]),
            "hbmc_residual_history": (I32, [P, P, I64, P]),
            "hbmc_fwd_bar": (I32, [P, P, P]),
            "hbmc_bwd_bar": (I32, [P, P, P]),
            "hbmc_spmv_bar": (I32, [P, P, P]),
            "hbmc_profile_kernels": (I32, [P, I32, P]),
            "hbmc_debug_stall": (I32, [P, I64, D]),
            "hbmc_debug_convert": (I32, [P, P, P, P, I64, P]),
            "hbmc_spmv_dot_static": (I32, [P, P, P, P]),
            "hbmc_sor": (I32, [P, P, P, D, I32, I32, P]),
            "hbmc_sor_bar": (I32, [P, P, P, D, I32, I32]),
            "hbmc_ilu0": (I32, [P, D, P]),
            "hbmc_get_factor_u": (I32, [P, P]),
            "hbmc_bicgstab": (I32, [P, P, P, D, I64, P, P, P]),
            "hbmc_batch_build": (I32, [I32, P, I32, P, P]),
            "hbmc_batch_build_w": (I32, [I32, P, I32, I32, P, P]),
            "hbmc_batch_destroy": (None, [P]),
            "hbmc_batch_last_error": (ctypes.c_char_p, [P]),
            "hbmc_batch_info": (I32, [P, P, P, P, P]),
            "hbmc_batch_set_stream": (I32, [P, P]),
            "hbmc_batch_set_precision": (I32, [P, I32]),
            "hbmc_batch_ic0": (I32, [P, P, P]),
            "hbmc_batch_iccg": (I32, [P, P, P, D, I64, P, P, P, P, P]),
            "hbmc_batch_autotune": (I32, [I32, P, P, I32, P, P, D, I64, ctypes.c_char_p, P, P]),
            "hbmc_batch_autotune_w": (I32, [I32, P, P, I32, P, I32, P, I32, P, P, D, I64, ctypes.c_char_p, P, P, P,
                                            P]),
            "hbmc_batch_features": (I32, [P, P]),
            "hbmc_features": (I32, [P, P]),
            "hbmc_shift_grid": (D, [I32]),
            "hbmc_mlp_num_params": (I32, [I32]),
            "hbmc_mlp_create": (I32, [I32, P]),
            "hbmc_mlp_destroy": (None, [P]),
            "hbmc_mlp_last_error": (ctypes.c_char_p, [P]),
            "hbmc_mlp_set_params": (I32, [P, P, P, P]),
            "hbmc_mlp_get_params": (I32, [P, P]),
            "hbmc_mlp_forward": (I32, [P, P, I32, P]),
            "hbmc_mlp_gradient": (I32, [P, P, P, I32, P, P]),
            "hbmc_mlp_train": (I32, [P, P, P, I32, I32, ctypes.c_float, P]),
            "hbmc_predict_shift": (I32, [P, P, P, P]),
            "hbmc_ic0_auto": (I32, [P, P, P, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _status_name(s):
    try:
        return load().hbmc_status_string(s).decode()
    except Exception:  # library not loadable while formatting an error
        return f"status {s}"


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, n, name):
    """Device pointer of a contiguous float64 CUDA tensor of length n."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous float64 tensor of length {n}")
    return ctypes.c_void_p(t.data_ptr())


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    relres: float
    true_relres: float

    @property
    def converged(self):
        return self.status == OK


class Context:
    """An hbmc_ctx handle; frees the context when garbage collected."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n
        self._lib = load()

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("context destroyed")
        return self._h

    def close(self):
        if self._h:
            self._lib.hbmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status, allowed=(OK,)):
        if status not in allowed:
            raise HbmcError(status, self._lib.hbmc_last_error(self._h).decode())
        return status

    def info(self) -> dict:
        inf = Info()
        self.check(self._lib.hbmc_info(self.handle, ctypes.byref(inf)))
        return inf.as_dict()


def hbmc_build(A, bs: int, w: int, *, box=None, grid=None, precision=PREC_F64,
               loop_mode=LOOP_GRAPH, host_only=False, device=-1, check_every=16,
               sweep_tpb=0, sweep_kernel=0, nonsymmetric=False, sell_split=0,
               sell_split_cost=0, sell_vslice=0) -> Context:
    """hbmc_build on a CSR (workloads.CSR or any object with n, row_ptr, col, val).
    sell_split = P > 0 splits the SpMV's long rows into a head and pieces of P;
    sell_vslice = K > 0 gives every SpMV slice its own sub-slice height
    (cost K entries per sub-slice)."""
    lib = load()
    opt = Options()
    lib.hbmc_default_options(ctypes.byref(opt))
    if box is not None:
        grid = grid if grid is not None else A.grid
        if grid is None:
            raise ValueError("box blocking needs the grid dimensions")
        opt.blocking = BLOCK_BOXES
        opt.grid[:] = [int(g) for g in grid]
        opt.box[:] = [int(b) for b in box]
    opt.precision = precision
    opt.loop_mode = loop_mode
    opt.host_only = 1 if host_only else 0
    opt.device = device
    opt.check_every = check_every
    opt.sweep_tpb = sweep_tpb
    opt.sweep_kernel = sweep_kernel
    opt.nonsymmetric = 1 if nonsymmetric else 0
    opt.sell_split = int(sell_split)
    opt.sell_split_cost = int(sell_split_cost)
    opt.sell_vslice = int(sell_vslice)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    h = ctypes.c_void_p()
    s = lib.hbmc_build(int(A.n), _np_ptr(rp), _np_ptr(ci), _np_ptr(v), int(bs), int(w),
                       ctypes.byref(opt), ctypes.byref(h))
    if s != OK:
        raise HbmcError(s, lib.hbmc_last_error(None).decode())
    return Context(h, int(A.n))


def hbmc_info(ctx: Context) -> dict:
    return ctx.info()


def hbmc_get_ordering(ctx: Context):
    """Returns (pi[n], color_ptr[nc+1], block_of[n], block_color[nblocks])."""
    inf = ctx.info()
    pi = np.empty(inf["n"], dtype=np.int64)
    cp = np.empty(inf["nc"] + 1, dtype=np.int64)
    bo = np.empty(inf["n"], dtype=np.int64)
    bc = np.empty(max(inf["nblocks"], 1), dtype=np.int32)
    ctx.check(ctx._lib.hbmc_get_ordering(ctx.handle, _np_ptr(pi), _np_ptr(cp), _np_ptr(bo), _np_ptr(bc)))
    return pi, cp, bo, bc[: inf["nblocks"]]


def hbmc_get_matrix(ctx: Context):
    """Abar on the padded index space: (row_ptr, col, val)."""
    inf = ctx.info()
    nnz = inf["nnz"] + inf["n_pad"] - inf["n"]
    rp = np.empty(inf["n_pad"] + 1, dtype=np.int64)
    ci = np.empty(max(nnz, 1), dtype=np.int32)
    v = np.empty(max(nnz, 1), dtype=np.float64)
    ctx.check(ctx._lib.hbmc_get_matrix(ctx.handle, _np_ptr(rp), _np_ptr(ci), _np_ptr(v)))
    return rp, ci[:nnz], v[:nnz]


def hbmc_get_split(ctx: Context):
    """Head width of every slice of w rows of the row-split SpMV layout."""
    inf = ctx.info()
    head = np.empty(max(inf["n_pad"] // max(inf["w"], 1), 1), dtype=np.int32)
    ctx.check(ctx._lib.hbmc_get_split(ctx.handle, _np_ptr(head)))
    return head[: inf["n_pad"] // max(inf["w"], 1)]


def hbmc_get_vslice(ctx: Context):
    """Sub-slice height C of every slice of w rows of the variable-height SpMV layout."""
    inf = ctx.info()
    h = np.empty(max(inf["n_pad"] // max(inf["w"], 1), 1), dtype=np.int32)
    ctx.check(ctx._lib.hbmc_get_vslice(ctx.handle, _np_ptr(h)))
    return h[: inf["n_pad"] // max(inf["w"], 1)]


def hbmc_get_dag_deps(ctx: Context, direction: int):
    """What each level-1 block of the dependency-driven forward (0) or
    backward (1) sweep waits for: (ptr[ntiles + 1], dep[count]); entries >= 0
    are level-1 blocks, -(c + 1) the completion counter of color c."""
    count = ctypes.c_int64(0)
    ctx.check(ctx._lib.hbmc_get_dag_deps(ctx.handle, direction, None, None, 0, ctypes.byref(count)))
    inf = ctx.info()
    ptr = np.empty(inf["ntiles"] + 1, dtype=np.int64)
    dep = np.empty(max(count.value, 1), dtype=np.int32)
    ctx.check(ctx._lib.hbmc_get_dag_deps(ctx.handle, direction, _np_ptr(ptr), _np_ptr(dep), count.value,
                                         ctypes.byref(count)))
    return ptr, dep[: count.value]


def hbmc_set_stream(ctx: Context, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = None if stream is None else getattr(stream, "cuda_stream", stream)
    ctx.check(ctx._lib.hbmc_set_stream(ctx.handle, ctypes.c_void_p(raw) if raw else None))


def hbmc_set_precision(ctx: Context, precision: int) -> None:
    ctx.check(ctx._lib.hbmc_set_precision(ctx.handle, int(precision)))


def hbmc_ic0(ctx: Context, shift: float = 0.0):
    """Returns (status, bad_row); raises on errors other than a bad pivot."""
    bad = ctypes.c_int64(-1)
    s = ctx._lib.hbmc_ic0(ctx.handle, float(shift), ctypes.byref(bad))
    ctx.check(s, (OK, ERR_NOT_SPD_PIVOT))
    return s, int(bad.value)


def hbmc_get_factor(ctx: Context):
    """(lower values aligned with hbmc_get_matrix, diagonal l_ii)."""
    inf = ctx.info()
    nnz = inf["nnz"] + inf["n_pad"] - inf["n"]
    lo = np.empty(max(nnz, 1))
    dg = np.empty(max(inf["n_pad"], 1))
    ctx.check(ctx._lib.hbmc_get_factor(ctx.handle, _np_ptr(lo), _np_ptr(dg)))
    return lo[:nnz], dg[: inf["n_pad"]]


def hbmc_precond(ctx: Context, r, z) -> None:
    ctx.check(ctx._lib.hbmc_precond(ctx.handle, _dev_ptr(r, ctx.n, "r"), _dev_ptr(z, ctx.n, "z")))


def hbmc_iccg(ctx: Context, b, x, tol=1e-8, maxit=10000) -> SolveResult:
    """Device tensors b, x (x: initial guess in, solution out)."""
    it, rr, tr = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
    s = ctx._lib.hbmc_iccg(ctx.handle, _dev_ptr(b, ctx.n, "b"), _dev_ptr(x, ctx.n, "x"),
                           float(tol), int(maxit), ctypes.byref(it), ctypes.byref(rr), ctypes.byref(tr))
    ctx.check(s, (OK, NOT_CONVERGED, ERR_BREAKDOWN))
    return SolveResult(s, int(it.value), float(rr.value), float(tr.value))


def hbmc_iccg_host(ctx: Context, b: np.ndarray, x: np.ndarray, tol=1e-8, maxit=10000) -> SolveResult:
    """Host numpy arrays b, x (float64, length n); x is overwritten."""
    for name, a in (("b", b), ("x", x)):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != ctx.n:
            raise ValueError(f"{name} must be a contiguous float64 array of length {ctx.n}")
    it, rr, tr = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
    s = ctx._lib.hbmc_iccg_host(ctx.handle, _np_ptr(b), _np_ptr(x), float(tol), int(maxit),
                                ctypes.byref(it), ctypes.byref(rr), ctypes.byref(tr))
    ctx.check(s, (OK, NOT_CONVERGED, ERR_BREAKDOWN))
    return SolveResult(s, int(it.value), float(rr.value), float(tr.value))


def hbmc_ilu0(ctx: Context, shift: float = 0.0):
    """ILU(0) of a context built with nonsymmetric=True; returns (status,
    bad_row in the original numbering or -1)."""
    bad = ctypes.c_int64(-1)
    s = ctx._lib.hbmc_ilu0(ctx.handle, float(shift), ctypes.byref(bad))
    ctx.check(s, (OK, ERR_NOT_SPD_PIVOT))
    return s, int(bad.value)


def hbmc_get_factor_u(ctx: Context) -> np.ndarray:
    """U's strict upper triangle on Abar's positions (see hbmc_get_matrix)."""
    nnz = len(hbmc_get_matrix(ctx)[1])
    out = np.empty(nnz)
    ctx.check(ctx._lib.hbmc_get_factor_u(ctx.handle, _np_ptr(out)))
    return out


def hbmc_bicgstab(ctx: Context, b, x, tol=1e-8, maxit=10000) -> SolveResult:
    """ILU(0)-preconditioned BiCGStab; device tensors b, x (x: initial guess
    in, solution out)."""
    it, rr, tr = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
    s = ctx._lib.hbmc_bicgstab(ctx.handle, _dev_ptr(b, ctx.n, "b"), _dev_ptr(x, ctx.n, "x"), float(tol), int(maxit),
                               ctypes.byref(it), ctypes.byref(rr), ctypes.byref(tr))
    ctx.check(s, (OK, NOT_CONVERGED, ERR_BREAKDOWN))
    return SolveResult(s, int(it.value), float(rr.value), float(tr.value))


def hbmc_sor(ctx: Context, b, x, omega=1.0, sweeps=1, symmetric=False) -> float:
    """SOR (symmetric SOR) sweeps on device tensors b, x of length n in the
    original ordering (x: initial guess in, result out); returns
    ||b - A x|| / ||b|| after the sweeps."""
    rr = ctypes.c_double(0)
    ctx.check(ctx._lib.hbmc_sor(ctx.handle, _dev_ptr(b, ctx.n, "b"), _dev_ptr(x, ctx.n, "x"), float(omega),
                                int(sweeps), 1 if symmetric else 0, ctypes.byref(rr)))
    return float(rr.value)


def hbmc_sor_bar(ctx: Context, b, x, omega=1.0, sweeps=1, symmetric=False) -> None:
    """The same on reordered device vectors of length n_pad (no residual)."""
    n_pad = ctx.info()["n_pad"]
    ctx.check(ctx._lib.hbmc_sor_bar(ctx.handle, _dev_ptr(b, n_pad, "b"), _dev_ptr(x, n_pad, "x"), float(omega),
                                    int(sweeps), 1 if symmetric else 0))


def hbmc_residual_history(ctx: Context, cap: int = 100000) -> np.ndarray:
    h = np.empty(max(cap, 1))
    cnt = ctypes.c_int64(0)
    ctx.check(ctx._lib.hbmc_residual_history(ctx.handle, _np_ptr(h), int(cap), ctypes.byref(cnt)))
    return h[: cnt.value].copy()


def _bar(fn, ctx, a, b):
    n_pad = ctx.info()["n_pad"]
    ctx.check(fn(ctx.handle, _dev_ptr(a, n_pad, "input"), _dev_ptr(b, n_pad, "output")))


def hbmc_fwd_bar(ctx: Context, r, y) -> None:
    _bar(ctx._lib.hbmc_fwd_bar, ctx, r, y)


def hbmc_bwd_bar(ctx: Context, y, z) -> None:
    _bar(ctx._lib.hbmc_bwd_bar, ctx, y, z)


def hbmc_spmv_bar(ctx: Context, p, q) -> None:
    _bar(ctx._lib.hbmc_spmv_bar, ctx, p, q)


PROFILE_PHASES = ("fwd", "bwd", "spmv", "update_xr", "update_p")


def hbmc_profile_kernels(ctx: Context, reps: int = 20) -> dict:
    """Average device ms per call of each phase of one CG iteration."""
    out = np.zeros(5)
    ctx.check(ctx._lib.hbmc_profile_kernels(ctx.handle, int(reps), _np_ptr(out)))
    return dict(zip(PROFILE_PHASES, out.tolist()))


def hbmc_debug_stall(ctx: Context, unit: int = -1, wait_s: float = 0.0) -> None:
    """Test hook of the dependency-driven sweeps: level-1 block `unit` never
    publishes its completion, and every wait gives up after wait_s seconds
    (unit = -1, wait_s = 0: normal operation)."""
    ctx.check(ctx._lib.hbmc_debug_stall(ctx.handle, int(unit), float(wait_s)))


def hbmc_debug_convert(d_in, f_in):
    """Test hook: the integer-operation conversions of the FP32 substitutions
    on device tensors d_in (float64) and f_in (float32) of equal length;
    returns (d_in narrowed to float32, f_in widened to float64)."""
    import torch
    lib = load()
    if not (d_in.is_cuda and f_in.is_cuda and d_in.dtype == torch.float64 and f_in.dtype == torch.float32
            and d_in.is_contiguous() and f_in.is_contiguous() and d_in.numel() == f_in.numel()):
        raise ValueError("d_in: contiguous CUDA float64, f_in: contiguous CUDA float32, equal lengths")
    f_out = torch.empty_like(f_in)
    d_out = torch.empty_like(d_in)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    st = lib.hbmc_debug_convert(vp(d_in), vp(f_out), vp(f_in), vp(d_out), int(d_in.numel()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != OK:
        raise HbmcError(st, "hbmc_debug_convert failed")
    return f_out, d_out


def hbmc_spmv_dot_static(ctx: Context, p, q, pq) -> None:
    """q = Abar p and pq[0] = p.q (device tensors; p, q of length n_pad, pq of
    length 1) using only the library's static scratch: for callers that must
    not allocate device memory.  Asynchronous on the context's stream."""
    n_pad = ctx.info()["n_pad"]
    ctx.check(ctx._lib.hbmc_spmv_dot_static(ctx.handle, _dev_ptr(p, n_pad, "p"), _dev_ptr(q, n_pad, "q"),
                                            _dev_ptr(pq, 1, "pq")))


# --------------------------------------------------------------------------
# Batched solver
# --------------------------------------------------------------------------

class System(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("blocking", ctypes.c_int32), ("grid", ctypes.c_int64 * 3)]


def _systems(mats, use_boxes):
    """ctypes array of hbmc_system for CSR matrices (box blocking on grid
    matrices when use_boxes); returns (array, keep-alive list)."""
    keep = []
    arr = (System * len(mats))()
    for k, A in enumerate(mats):
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.col, dtype=np.int32)
        v = np.ascontiguousarray(A.val, dtype=np.float64)
        keep += [rp, ci, v]
        arr[k].n = int(A.n)
        arr[k].row_ptr = rp.ctypes.data
        arr[k].col = ci.ctypes.data
        arr[k].val = v.ctypes.data
        if use_boxes and getattr(A, "grid", None) is not None:
            arr[k].blocking = BLOCK_BOXES
            arr[k].grid[:] = [int(g) for g in A.grid]
        else:
            arr[k].blocking = BLOCK_ALGEBRAIC
    return arr, keep


def _box_opts(bs, precision, loop_mode, device, check_every=16):
    lib = load()
    opt = Options()
    lib.hbmc_default_options(ctypes.byref(opt))
    shapes = {1: (1, 1, 1), 2: (1, 1, 2), 4: (1, 2, 2), 8: (2, 2, 2), 16: (2, 2, 4), 32: (2, 4, 4),
              64: (4, 4, 4)}
    opt.box[:] = list(shapes.get(bs, (1, 1, bs)))
    opt.precision = precision
    opt.loop_mode = loop_mode
    opt.device = device
    opt.check_every = check_every
    return opt


@dataclasses.dataclass
class BatchResult:
    status: int
    iters: np.ndarray
    relres: np.ndarray
    true_relres: np.ndarray
    statuses: np.ndarray
    solve_ms: np.ndarray


class Batch:
    """An hbmc_batch handle (many independent systems solved together)."""

    def __init__(self, handle, nsys, n_total, sizes):
        self._h = handle
        self.nsys = nsys
        self.n_total = n_total
        self.sizes = sizes
        self._lib = load()

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("batch destroyed")
        return self._h

    def close(self):
        if self._h:
            self._lib.hbmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status, allowed=(OK,)):
        if status not in allowed:
            raise HbmcError(status, self._lib.hbmc_batch_last_error(self._h).decode())
        return status

    def info(self):
        n, npad, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        nc = ctypes.c_int32()
        self.check(self._lib.hbmc_batch_info(self.handle, ctypes.byref(n), ctypes.byref(npad), ctypes.byref(nc),
                                             ctypes.byref(nu)))
        return {"n": n.value, "n_pad": npad.value, "nc": nc.value, "units": nu.value}


def hbmc_batch_build(mats, bs, *, w=32, vslice=0, use_boxes=True, precision=PREC_F64, loop_mode=LOOP_GRAPH,
                     device=-1, check_every=16) -> Batch:
    """Batch of CSR systems (box blocking for grid matrices when use_boxes);
    w = 32 or 16 BMC blocks per level-1 block; vslice = K > 0: the SpMV's
    variable-slice-height layout."""
    lib = load()
    arr, keep = _systems(mats, use_boxes)
    opt = _box_opts(bs, precision, loop_mode, device, check_every)
    opt.sell_vslice = int(vslice)
    h = ctypes.c_void_p()
    s = lib.hbmc_batch_build_w(len(mats), ctypes.cast(arr, ctypes.c_void_p), int(bs), int(w), ctypes.byref(opt),
                               ctypes.byref(h))
    if s != OK:
        raise HbmcError(s, lib.hbmc_batch_last_error(None).decode())
    del keep
    sizes = [int(A.n) for A in mats]
    return Batch(h, len(mats), sum(sizes), sizes)


def hbmc_batch_set_stream(batch: Batch, stream) -> None:
    raw = None if stream is None else getattr(stream, "cuda_stream", stream)
    batch.check(batch._lib.hbmc_batch_set_stream(batch.handle, ctypes.c_void_p(raw) if raw else None))


def hbmc_batch_set_precision(batch: Batch, precision: int) -> None:
    batch.check(batch._lib.hbmc_batch_set_precision(batch.handle, int(precision)))


def hbmc_batch_ic0(batch: Batch, shifts=None):
    """Returns (status, bad_rows[nsys]); bad_rows[s] = -1 when system s factored."""
    bad = np.full(batch.nsys, -1, dtype=np.int64)
    sh = None if shifts is None else np.ascontiguousarray(shifts, dtype=np.float64)
    s = batch._lib.hbmc_batch_ic0(batch.handle, _np_ptr(sh) if sh is not None else None, _np_ptr(bad))
    batch.check(s, (OK, ERR_NOT_SPD_PIVOT))
    return s, bad


def hbmc_batch_iccg(batch: Batch, b, x, tol=1e-8, maxit=10000) -> BatchResult:
    """Device tensors b, x (the systems' vectors concatenated)."""
    k = batch.nsys
    it = np.zeros(k, dtype=np.int64)
    rr = np.zeros(k)
    tr = np.zeros(k)
    st = np.zeros(k, dtype=np.int32)
    ms = np.zeros(k)
    s = batch._lib.hbmc_batch_iccg(batch.handle, _dev_ptr(b, batch.n_total, "b"), _dev_ptr(x, batch.n_total, "x"),
                                   float(tol), int(maxit), _np_ptr(it), _np_ptr(rr), _np_ptr(tr), _np_ptr(st),
                                   _np_ptr(ms))
    batch.check(s, (OK, NOT_CONVERGED, ERR_BREAKDOWN))
    return BatchResult(s, it, rr, tr, st, ms)


def hbmc_batch_autotune(mats, b, bs_candidates=(4, 8, 16, 32), *, use_boxes=True, precision=PREC_F32,
                        tol=1e-8, maxit=10000, cache_path=None, device=-1):
    """Pick the block size that solves the batch fastest; returns (best_bs, ms per candidate)."""
    lib = load()
    arr, keep = _systems(mats, use_boxes)
    opt = _box_opts(8, precision, LOOP_GRAPH, device)
    cand = np.ascontiguousarray(bs_candidates, dtype=np.int32)
    ms = np.zeros(len(cand))
    best = ctypes.c_int32(-1)
    n_total = sum(int(A.n) for A in mats)
    s = lib.hbmc_batch_autotune(len(mats), ctypes.cast(arr, ctypes.c_void_p), _np_ptr(cand), len(cand),
                                ctypes.byref(opt), _dev_ptr(b, n_total, "b"), float(tol), int(maxit),
                                cache_path.encode() if cache_path else None, ctypes.byref(best), _np_ptr(ms))
    if s != OK:
        raise HbmcError(s, lib.hbmc_batch_last_error(None).decode())
    del keep
    return int(best.value), ms


def hbmc_batch_autotune_w(mats, b, bs_candidates=(4, 8, 16, 32), w_candidates=(16, 32), vslice_candidates=(0,),
                          *, use_boxes=True, precision=PREC_F32, tol=1e-8, maxit=10000, cache_path=None, device=-1):
    """Pick the (bs, w, vslice) triple that solves the batch fastest (vslice 0:
    SELL slices of height w; K > 0: per-slice heights from {w, w/2, w/4});
    returns (best_bs, best_w, best_vslice, ms[nbs, nw, nv])."""
    lib = load()
    arr, keep = _systems(mats, use_boxes)
    opt = _box_opts(8, precision, LOOP_GRAPH, device)
    cb = np.ascontiguousarray(bs_candidates, dtype=np.int32)
    cw = np.ascontiguousarray(w_candidates, dtype=np.int32)
    cv = np.ascontiguousarray(vslice_candidates, dtype=np.int32)
    ms = np.zeros(len(cb) * len(cw) * len(cv))
    best_bs, best_w, best_v = ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int32(-1)
    n_total = sum(int(A.n) for A in mats)
    s = lib.hbmc_batch_autotune_w(len(mats), ctypes.cast(arr, ctypes.c_void_p), _np_ptr(cb), len(cb), _np_ptr(cw),
                                  len(cw), _np_ptr(cv), len(cv), ctypes.byref(opt), _dev_ptr(b, n_total, "b"),
                                  float(tol), int(maxit), cache_path.encode() if cache_path else None,
                                  ctypes.byref(best_bs), ctypes.byref(best_w), ctypes.byref(best_v), _np_ptr(ms))
    if s != OK:
        raise HbmcError(s, lib.hbmc_batch_last_error(None).decode())
    del keep
    return int(best_bs.value), int(best_w.value), int(best_v.value), ms.reshape(len(cb), len(cw), len(cv))


# --------------------------------------------------------------------------
# Learned IC(0) shift
# --------------------------------------------------------------------------

NUM_FEATURES = 12
SHIFT_GRID = 13


def shift_grid():
    """The shift grid: 0, then 1e-3 * 2^k for k = 0..11."""
    lib = load()
    return np.array([lib.hbmc_shift_grid(c) for c in range(SHIFT_GRID)])


def hbmc_features(ctx: Context) -> np.ndarray:
    f = np.zeros(NUM_FEATURES, dtype=np.float32)
    ctx.check(ctx._lib.hbmc_features(ctx.handle, _np_ptr(f)))
    return f


def hbmc_batch_features(batch: Batch) -> np.ndarray:
    f = np.zeros((batch.nsys, NUM_FEATURES), dtype=np.float32)
    batch.check(batch._lib.hbmc_batch_features(batch.handle, _np_ptr(f)))
    return f


class Mlp:
    """hbmc_mlp handle: D -> 32 -> 32 -> 1 network with device-side training."""

    def __init__(self, in_dim: int):
        self._lib = load()
        h = ctypes.c_void_p()
        s = self._lib.hbmc_mlp_create(int(in_dim), ctypes.byref(h))
        if s != OK:
            raise HbmcError(s, self._lib.hbmc_mlp_last_error(None).decode())
        self._h = h
        self.in_dim = int(in_dim)
        self.num_params = int(self._lib.hbmc_mlp_num_params(int(in_dim)))

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("network destroyed")
        return self._h

    def close(self):
        if self._h:
            self._lib.hbmc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status):
        if status != OK:
            raise HbmcError(status, self._lib.hbmc_mlp_last_error(self._h).decode())

    def set_params(self, params=None, mean=None, std=None):
        def fp(a, n):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size != n:
                raise ValueError(f"expected {n} values")
            return a, _np_ptr(a)
        p, pp = fp(params, self.num_params)
        m, mp = fp(mean, self.in_dim)
        s, sp = fp(std, self.in_dim)
        self.check(self._lib.hbmc_mlp_set_params(self.handle, pp, mp, sp))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        self.check(self._lib.hbmc_mlp_get_params(self.handle, _np_ptr(out)))
        return out

    @staticmethod
    def _fptr(t, n, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or \
                not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {n} elements")
        return ctypes.c_void_p(t.data_ptr())

    def forward(self, X):
        import torch
        B = X.shape[0]
        out = torch.empty(B, dtype=torch.float32, device=X.device)
        self.check(self._lib.hbmc_mlp_forward(self.handle, self._fptr(X, B * self.in_dim, "X"), int(B),
                                              self._fptr(out, B, "out")))
        return out

    def gradient(self, X, T):
        import torch
        B = X.shape[0]
        g = torch.empty(self.num_params, dtype=torch.float32, device=X.device)
        loss = ctypes.c_float(0)
        self.check(self._lib.hbmc_mlp_gradient(self.handle, self._fptr(X, B * self.in_dim, "X"),
                                               self._fptr(T, B, "T"), int(B), self._fptr(g, self.num_params, "g"),
                                               ctypes.byref(loss)))
        return g, float(loss.value)

    def train(self, X, T, steps, lr=1e-3):
        B = X.shape[0]
        loss = ctypes.c_float(0)
        self.check(self._lib.hbmc_mlp_train(self.handle, self._fptr(X, B * self.in_dim, "X"), self._fptr(T, B, "T"),
                                            int(B), int(steps), ctypes.c_float(lr), ctypes.byref(loss)))
        return float(loss.value)


def hbmc_predict_shift(ctx: Context, net: Mlp):
    """(learned shift, predicted log2 iterations per grid shift)."""
    sh = ctypes.c_double(0)
    pred = np.zeros(SHIFT_GRID, dtype=np.float32)
    ctx.check(ctx._lib.hbmc_predict_shift(ctx.handle, net.handle, ctypes.byref(sh), _np_ptr(pred)))
    return float(sh.value), pred


def hbmc_ic0_auto(ctx: Context, net: Mlp | None = None):
    """Factor with the learned shift (net) or the plain rule (None).
    Returns (status, shift_used, fallback_used)."""
    sh = ctypes.c_double(0)
    fb = ctypes.c_int32(0)
    s = ctx._lib.hbmc_ic0_auto(ctx.handle, net.handle if net is not None else None, ctypes.byref(sh),
                               ctypes.byref(fb))
    ctx.check(s, (OK, ERR_NOT_SPD_PIVOT))
    return s, float(sh.value), bool(fb.value)
