"""Host side of the C ABI, no GPU needed: the library loads and exports every
function include/hbmc.h declares, and hbmc_build's host-only mode produces
exactly the oracle's blocks, colors, HBMC permutation and Abar."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "hbmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hbmc_\w+)\s*\(", src)))


def test_library_exports_every_declared_function(lib):
    declared = _declared_functions()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(H.EXPORTED) == declared


def test_status_strings(lib):
    assert lib.hbmc_status_string(0) == b"HBMC_OK"
    assert lib.hbmc_status_string(2) == b"HBMC_ERR_NOT_SPD_PIVOT"


CASES = [
    ("poisson7_8_boxes", lambda: W.poisson7(8), 8, 4, (2, 2, 2)),
    ("poisson7_7_boxes", lambda: W.poisson7(7), 8, 32, (2, 2, 2)),
    ("poisson7_9_bs16", lambda: W.poisson7(9), 16, 8, (2, 2, 4)),
    ("poisson7_8_bs32", lambda: W.poisson7(8), 32, 2, (2, 4, 4)),
    ("poisson7_6_alg", lambda: W.poisson7(6), 8, 32, None),
    ("hetero27_7_rand", lambda: W.permute_input(W.heterogeneous_stencil(7, 27, 2.0, 1),
                                                W.random_order(2, 343)), 8, 16, None),
    ("veclap_4_rand", lambda: W.permute_input(W.vector_laplacian(4, 3), W.random_order(4, 192)), 4, 32, None),
    ("hetero7_5_bs1", lambda: W.heterogeneous_stencil(5, 7, 1.0, 3), 1, 1, None),
    ("poisson7_4_bs64", lambda: W.poisson7(4), 64, 1, None),
]


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
def test_host_ordering_matches_oracle(lib, orc, name, mk, bs, w, box):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box, host_only=True)
    inf = ctx.info()
    an = orc.analyse(A, bs, w, box=box)
    pi, cp, bo, bc = H.hbmc_get_ordering(ctx)
    assert inf["nc"] == an.nc and inf["n_pad"] == an.n_pad and inf["nblocks"] == an.nblocks
    np.testing.assert_array_equal(bo, an.block_of)
    np.testing.assert_array_equal(bc, an.color)
    np.testing.assert_array_equal(pi, an.pi)
    np.testing.assert_array_equal(cp, an.color_ptr)
    rp, ci, v = H.hbmc_get_matrix(ctx)
    np.testing.assert_array_equal(rp, an.row_ptr)
    np.testing.assert_array_equal(ci, an.col)
    np.testing.assert_array_equal(v, an.val)
    assert inf["ntiles"] * bs * w == inf["n_pad"]
    assert inf["nnz_lower"] == (A.nnz - A.n) // 2
    # SELL stores at least every nonzero (plus padding)
    assert inf["sell_entries_a"] >= A.nnz + (an.n_pad - A.n)
    assert inf["sell_entries_l"] >= inf["nnz_lower"] and inf["sell_entries_u"] >= inf["nnz_lower"]
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_ic0(ctx, 0.0)
    assert e.value.status == H.ERR_NO_DEVICE
    ctx.close()


def test_empty_system(lib):
    A = W.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    ctx = H.hbmc_build(A, 8, 32, host_only=True)
    inf = ctx.info()
    assert inf["n"] == 0 and inf["n_pad"] == 0 and inf["nc"] == 0


def _bad(A, bs=8, w=32, **kw):
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_build(A, bs, w, host_only=True, **kw)
    assert e.value.status == H.ERR_INVALID_ARG
    return str(e.value)


def test_invalid_inputs_are_rejected(lib):
    A = W.poisson7(3)
    assert "not symmetric" in _bad(W.CSR(A.n, A.row_ptr, A.col, np.where(np.arange(A.nnz) == 1, -2.0, A.val)))
    col = A.col.copy(); col[[0, 1]] = col[[1, 0]]
    assert "ascending" in _bad(W.CSR(A.n, A.row_ptr, col, A.val))
    # drop the diagonal of row 0
    keep = np.ones(A.nnz, bool); keep[0] = False
    rp = A.row_ptr.copy(); rp[1:] -= 1
    assert "diagonal" in _bad(W.CSR(A.n, rp, A.col[keep], A.val[keep]))
    neg = A.val.copy(); neg[0] = -6.0
    assert "diagonal" in _bad(W.CSR(A.n, A.row_ptr, A.col, neg))
    nan = A.val.copy(); nan[1] = np.nan
    _bad(W.CSR(A.n, A.row_ptr, A.col, nan))
    _bad(A, bs=0)
    _bad(A, bs=65)
    _bad(A, w=3)
    _bad(A, w=64)
    _bad(A, bs=8, box=(2, 2, 1))  # box volume != bs
    _bad(A, bs=8, box=(2, 2, 2), grid=(3, 3, 2))  # grid != n
    oob = A.col.copy(); oob[-1] = A.n
    _bad(W.CSR(A.n, A.row_ptr, oob, A.val))


def test_last_error_thread_message(lib):
    A = W.poisson7(3)
    try:
        H.hbmc_build(A, 8, 3, host_only=True)
    except H.HbmcError:
        pass
    assert b"w must be" in lib.hbmc_last_error(None)
