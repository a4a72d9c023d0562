"""Plain FP64 CPU oracle for HBMC-ordered IC(0)-CG (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use it; the CUDA solver never does.  The
arithmetic lives in ``hbmc_oracle.c`` (single-threaded C, compiled with
``-ffp-contract=off``); this module only marshals numpy arrays and chains the
steps in the paper's order:

  blocking (Section 4.1 / 5.1) -> greedy block coloring (Section 5.1)
  -> BMC order + dummy padding + HBMC secondary reordering (Section 4.2)
  -> Abar = P A P^T (Section 3, Eq. "AB") -> shifted IC(0) (Section 2, 5.1)
  -> PCG with forward/backward substitution (Section 2, Eqs. "for", "back").
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hbmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DOT_SEQUENTIAL = 0
DOT_EXACT = 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int64
            D = ctypes.c_double
            C = ctypes.c_int
            sig = {
                "orc_blocks_boxes": (I, [I, I, I, I, I, I, P]),
                "orc_blocks_greedy": (I, [I, P, P, I, P]),
                "orc_color_blocks": (I, [I, P, P, I, P, P]),
                "orc_ordering": (I, [I, I, P, P, I, I, I, C, P, P]),
                "orc_permute": (None, [I, P, P, P, P, I, P, P, P]),
                "orc_ic0": (I, [I, P, P, P, D, P, P, P]),
                "orc_fwd": (None, [I, P, P, P, P, P, P]),
                "orc_transpose_pos": (C, [I, P, P, P]),
                "orc_bwd": (None, [I, P, P, P, P, P, P, P]),
                "orc_spmv": (None, [I, P, P, P, P, P]),
                "orc_dot": (D, [I, P, P, P, C]),
                "orc_pcg": (C, [I, P, P, P, P, P, P, P, I, P, C, D, I, P, P, P]),
                "orc_split_plan": (I, [I, P, C, C, C, P, P, P]),
                "orc_spmv_split": (None, [I, P, P, P, C, P, C, P, P]),
                "orc_pcg_split": (C, [I, P, P, P, P, P, P, P, I, P, C, D, I, P, P, P, C, P, C]),
                "orc_sor": (C, [I, P, P, P, P, P, D, I, C]),
                "orc_ilu0": (I, [I, P, P, P, P, D, P, P, P, P]),
                "orc_bwd_u": (None, [I, P, P, P, P, P, P]),
                "orc_bicgstab": (C, [I, P, P, P, P, P, P, P, P, I, P, C, D, I, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Steps
# --------------------------------------------------------------------------

def blocks_boxes(grid, box):
    """Geometric blocks of a lexicographic grid; returns (block_of[n], nblocks)."""
    nx, ny, nz = grid
    bx, by, bz = box
    out = np.empty(nx * ny * nz, dtype=np.int64)
    nb = _load().orc_blocks_boxes(nx, ny, nz, bx, by, bz, _p(out))
    return out, int(nb)


def blocks_greedy(row_ptr, col, bs):
    """Minimal-number-seeded algebraic blocks; returns (block_of[n], nblocks)."""
    rp, ci = _i64(row_ptr), _i32(col)
    n = len(rp) - 1
    out = np.empty(n, dtype=np.int64)
    nb = _load().orc_blocks_greedy(n, _p(rp), _p(ci), bs, _p(out))
    return out, int(nb)


def color_blocks(row_ptr, col, block_of, nblocks):
    """Greedy first-fit block colors; returns (color[nblocks], n_c)."""
    rp, ci, bo = _i64(row_ptr), _i32(col), _i64(block_of)
    color = np.empty(nblocks, dtype=np.int64)
    nc = _load().orc_color_blocks(len(rp) - 1, _p(rp), _p(ci), nblocks, _p(bo), _p(color))
    return color, int(nc)


def ordering(block_of, nblocks, color, nc, bs, w, hbmc=True):
    """BMC or HBMC permutation; returns (pi[n], color_ptr[nc+1], n_pad)."""
    bo, co = _i64(block_of), _i64(color)
    pi = np.empty(len(bo), dtype=np.int64)
    cp = np.empty(nc + 1, dtype=np.int64)
    n_pad = _load().orc_ordering(len(bo), nblocks, _p(bo), _p(co), nc, bs, w, int(bool(hbmc)),
                                 _p(pi), _p(cp))
    return pi, cp, int(n_pad)


def permute(row_ptr, col, val, pi, n_pad):
    """Abar = P A P^T with identity dummy rows; returns (row_ptr, col, val)."""
    rp, ci, v, p = _i64(row_ptr), _i32(col), _f64(val), _i64(pi)
    n = len(rp) - 1
    nnz = int(rp[-1]) + (n_pad - n)
    rpo = np.empty(n_pad + 1, dtype=np.int64)
    cio = np.empty(nnz, dtype=np.int32)
    vo = np.empty(nnz, dtype=np.float64)
    _load().orc_permute(n, _p(rp), _p(ci), _p(v), _p(p), n_pad, _p(rpo), _p(cio), _p(vo))
    return rpo, cio, vo


def ic0(row_ptr, col, val, shift=0.0):
    """Shifted IC(0); returns (lval[nnz], ldiag[n], dinv[n], bad_row) (bad_row -1 if ok)."""
    rp, ci, v = _i64(row_ptr), _i32(col), _f64(val)
    n = len(rp) - 1
    lval = np.empty(len(v))
    ldiag = np.zeros(n)
    dinv = np.zeros(n)
    bad = _load().orc_ic0(n, _p(rp), _p(ci), _p(v), float(shift), _p(lval), _p(ldiag), _p(dinv))
    return lval, ldiag, dinv, int(bad)


def fwd(row_ptr, col, lval, dinv, r):
    rp, ci = _i64(row_ptr), _i32(col)
    y = np.empty(len(rp) - 1)
    _load().orc_fwd(len(rp) - 1, _p(rp), _p(ci), _p(_f64(lval)), _p(_f64(dinv)), _p(_f64(r)), _p(y))
    return y


def transpose_pos(row_ptr, col):
    rp, ci = _i64(row_ptr), _i32(col)
    t = np.empty(len(ci), dtype=np.int64)
    if _load().orc_transpose_pos(len(rp) - 1, _p(rp), _p(ci), _p(t)):
        raise ValueError("matrix is not structurally symmetric")
    return t


def bwd(row_ptr, col, lval, dinv, y, tpos=None):
    rp, ci = _i64(row_ptr), _i32(col)
    if tpos is None:
        tpos = transpose_pos(rp, ci)
    z = np.empty(len(rp) - 1)
    _load().orc_bwd(len(rp) - 1, _p(rp), _p(ci), _p(_i64(tpos)), _p(_f64(lval)), _p(_f64(dinv)),
                    _p(_f64(y)), _p(z))
    return z


def spmv(row_ptr, col, val, p):
    rp, ci = _i64(row_ptr), _i32(col)
    q = np.empty(len(rp) - 1)
    _load().orc_spmv(len(rp) - 1, _p(rp), _p(ci), _p(_f64(val)), _p(_f64(p)), _p(q))
    return q


SplitPlan = collections.namedtuple("SplitPlan", "w piece cost head processed nsplit npieces")


def split_plan(row_ptr, w, piece=64, cost=2):
    """Head width per slice of w rows for the row-splitting SELL SpMV
    (Section 5.2.2's remedy), pieces of at most `piece` entries, `cost` per
    piece in the plan's cost model; see orc_split_plan."""
    rp = _i64(row_ptr)
    n = len(rp) - 1
    if n % w:
        raise ValueError("the row count must be a multiple of w")
    head = np.zeros(n // w, dtype=np.int32)
    nsplit = ctypes.c_int64(0)
    npieces = ctypes.c_int64(0)
    processed = _load().orc_split_plan(n, _p(rp), int(w), int(piece), int(cost), _p(head),
                                       ctypes.byref(nsplit), ctypes.byref(npieces))
    return SplitPlan(int(w), int(piece), int(cost), head, int(processed), int(nsplit.value),
                     int(npieces.value))


def spmv_split(row_ptr, col, val, plan: SplitPlan, p):
    """q = A p with every row cut by `plan`: parts summed from zero, then added in order."""
    rp, ci = _i64(row_ptr), _i32(col)
    q = np.empty(len(rp) - 1)
    _load().orc_spmv_split(len(rp) - 1, _p(rp), _p(ci), _p(_f64(val)), plan.w, _p(_i32(plan.head)),
                           plan.piece, _p(_f64(p)), _p(q))
    return q


def sor(row_ptr, col, val, b, x0, omega=1.0, sweeps=1, symmetric=False):
    """SOR (symmetric SOR when `symmetric`) sweeps on a CSR matrix in its own
    index order, from x0; returns the new x (orc_sor: Section 2, Eq. "xj")."""
    rp, ci = _i64(row_ptr), _i32(col)
    x = _f64(x0).copy()
    if _load().orc_sor(len(rp) - 1, _p(rp), _p(ci), _p(_f64(val)), _p(_f64(b)), _p(x), float(omega), int(sweeps),
                       1 if symmetric else 0):
        raise ValueError("a row has no nonzero diagonal entry")
    return x


def sor_solve(an, b, x0=None, omega=1.0, sweeps=1, symmetric=False):
    """SOR sweeps on Abar with b and x0 in the original ordering; returns x in
    the original ordering (dummy rows stay 0)."""
    bbar = np.zeros(an.n_pad)
    bbar[an.pi] = b
    xbar = np.zeros(an.n_pad)
    if x0 is not None:
        xbar[an.pi] = x0
    xbar = sor(an.row_ptr, an.col, an.val, bbar, xbar, omega, sweeps, symmetric)
    return xbar[an.pi].copy()


def ilu0(row_ptr, col, val, shift=0.0, tpos=None):
    """ILU(0) of a CSR matrix with a symmetric pattern (orc_ilu0): returns
    (lval, uval, udiag, uinv, bad_row) with lval / uval at the positions of
    the strict lower / upper entries."""
    rp, ci, v = _i64(row_ptr), _i32(col), _f64(val)
    if tpos is None:
        tpos = transpose_pos(rp, ci)
    n = len(rp) - 1
    lval, uval = np.zeros(len(ci)), np.zeros(len(ci))
    udiag, uinv = np.zeros(n), np.zeros(n)
    bad = _load().orc_ilu0(n, _p(rp), _p(ci), _p(v), _p(_i64(tpos)), float(shift), _p(lval), _p(uval),
                           _p(udiag), _p(uinv))
    return lval, uval, udiag, uinv, int(bad)


def bwd_u(row_ptr, col, uval, uinv, y):
    rp, ci = _i64(row_ptr), _i32(col)
    z = np.empty(len(rp) - 1)
    _load().orc_bwd_u(len(rp) - 1, _p(rp), _p(ci), _p(_f64(uval)), _p(_f64(uinv)), _p(_f64(y)), _p(z))
    return z


def factor_ilu(an, shift=0.0):
    return ilu0(an.row_ptr, an.col, an.val, shift)


def bicgstab(an, lval, uval, uinv, b, tol=1e-8, maxit=10000, x0=None, dot_mode=DOT_SEQUENTIAL):
    """ILU(0)-preconditioned BiCGStab on Abar (orc_bicgstab); b and x0 in the
    original ordering.  status: 0 converged, 1 maxit, 2 breakdown."""
    bbar = np.zeros(an.n_pad)
    bbar[an.pi] = b
    xbar = np.zeros(an.n_pad)
    if x0 is not None:
        xbar[an.pi] = x0
    hist = np.zeros(maxit + 1)
    iters = ctypes.c_int64(0)
    relres = ctypes.c_double(0.0)
    order = _i64(an.pi)
    st = _load().orc_bicgstab(an.n_pad, _p(an.row_ptr), _p(an.col), _p(an.val), _p(_f64(lval)), _p(_f64(uval)),
                              _p(_f64(uinv)), _p(bbar), _p(xbar), len(order), _p(order), int(dot_mode), float(tol),
                              int(maxit), ctypes.byref(iters), ctypes.byref(relres), _p(hist))
    return Solve(xbar[an.pi].copy(), int(iters.value), float(relres.value), int(st),
                 hist[: iters.value + 1].copy(), -1, xbar)


def dot(a, b, idx=None, mode=DOT_EXACT):
    a, b = _f64(a), _f64(b)
    ii = None if idx is None else _i64(idx)
    m = len(a) if idx is None else len(ii)
    return float(_load().orc_dot(m, _p(ii), _p(a), _p(b), int(mode)))


# --------------------------------------------------------------------------
# Whole pipeline
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Analysis:
    """Everything the oracle derives from (A, bs, w) before a solve."""
    n: int
    bs: int
    w: int
    block_of: np.ndarray
    nblocks: int
    color: np.ndarray     # per block
    nc: int
    pi: np.ndarray        # original index -> padded reordered index
    color_ptr: np.ndarray
    n_pad: int
    row_ptr: np.ndarray   # Abar
    col: np.ndarray
    val: np.ndarray


def analyse(A, bs, w, box=None, hbmc=True, block_of=None):
    """Blocking (geometric boxes when `box` is given and A has a grid, else the
    algebraic rule), coloring, ordering and Abar, as the oracle defines them."""
    if block_of is None:
        if box is not None:
            if A.grid is None:
                raise ValueError("geometric blocking needs a grid matrix")
            block_of, nblocks = blocks_boxes(A.grid, box)
        else:
            block_of, nblocks = blocks_greedy(A.row_ptr, A.col, bs)
    else:
        nblocks = int(block_of.max()) + 1 if len(block_of) else 0
    color, nc = color_blocks(A.row_ptr, A.col, block_of, nblocks)
    pi, cp, n_pad = ordering(block_of, nblocks, color, nc, bs, w, hbmc)
    rp, ci, v = permute(A.row_ptr, A.col, A.val, pi, n_pad)
    return Analysis(A.n, bs, w, block_of, nblocks, color, nc, pi, cp, n_pad, rp, ci, v)


@dataclasses.dataclass
class Solve:
    x: np.ndarray      # original ordering
    iters: int
    relres: float
    status: int        # 0 converged, 1 maxit, 2 breakdown
    hist: np.ndarray
    bad_row: int       # IC(0) failure row in Abar numbering (-1 if none)
    xbar: np.ndarray   # reordered (padded) solution


def factor(an: Analysis, shift=0.0):
    return ic0(an.row_ptr, an.col, an.val, shift)


def pcg(an: Analysis, lval, dinv, b, tol=1e-8, maxit=10000, x0=None, dot_mode=DOT_SEQUENTIAL,
        split: SplitPlan | None = None):
    """IC(0)-PCG on Abar; b and x0 in original ordering.  With `split`, the
    iteration's q = A p is the row-splitting product (spmv_split)."""
    bbar = np.zeros(an.n_pad)
    bbar[an.pi] = b
    xbar = np.zeros(an.n_pad)
    if x0 is not None:
        xbar[an.pi] = x0
    hist = np.zeros(maxit + 1)
    iters = ctypes.c_int64(0)
    relres = ctypes.c_double(0.0)
    order = _i64(an.pi)
    args = (an.n_pad, _p(an.row_ptr), _p(an.col), _p(an.val), _p(_f64(lval)), _p(_f64(dinv)),
            _p(bbar), _p(xbar), len(order), _p(order), int(dot_mode), float(tol), int(maxit),
            ctypes.byref(iters), ctypes.byref(relres), _p(hist))
    if split is None:
        st = _load().orc_pcg(*args)
    else:
        if split.w != an.w:
            raise ValueError("the split plan's slice height must be the analysis' w")
        head = _i32(split.head)
        st = _load().orc_pcg_split(*args, split.w, _p(head), split.piece)
    if st == 3:
        raise ValueError("matrix is not structurally symmetric")
    return Solve(xbar[an.pi].copy(), int(iters.value), float(relres.value), int(st),
                 hist[: iters.value + 1].copy(), -1, xbar)


def iccg(A, b, bs, w, box=None, hbmc=True, shift=0.0, tol=1e-8, maxit=10000, x0=None,
         dot_mode=DOT_SEQUENTIAL, an=None, split=None):
    """Full pipeline: analyse, factor, solve.  Returns (Solve, Analysis).
    `split` = (piece, cost) solves with the row-splitting SpMV of that plan."""
    if an is None:
        an = analyse(A, bs, w, box=box, hbmc=hbmc)
    plan = None if split is None else split_plan(an.row_ptr, an.w, *split)
    lval, ldiag, dinv, bad = factor(an, shift)
    if bad >= 0:
        return Solve(np.zeros(A.n), 0, float("nan"), 2, np.zeros(0), bad, np.zeros(an.n_pad)), an
    return pcg(an, lval, dinv, b, tol, maxit, x0, dot_mode, split=plan), an
