"""The host build's variable-slice-height SpMV plan (hbmc_build host_only
with sell_vslice; the other SELL remedy of Section 5.2.2 and the
conclusions): the sub-slice height of every slice of w rows against a
direct evaluation of the cost over the three candidate heights, the stored
entries, and argument checks."""
import numpy as np
import pytest

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def expected_plan(row_ptr, w, cost):
    """Per slice of w rows: C in {w, w/2, w/4} (C >= 1) minimising
    sum over sub-slices of C * longest row + cost * (w / C), the largest C on
    ties; and the stored entries of the resulting layout."""
    lens = np.diff(np.asarray(row_ptr, dtype=np.int64))
    ns = len(lens) // w
    heights, stored = [], 0
    cands = [c for c in (w, w // 2, w // 4) if c >= 1]
    cands = list(dict.fromkeys(cands))  # w < 4 repeats candidates
    for s in range(ns):
        L = lens[s * w:(s + 1) * w]
        best_c, best = None, None
        for C in cands:
            val = cost * (w // C) + sum(C * int(L[k * C:(k + 1) * C].max()) for k in range(w // C))
            if best is None or val < best:
                best, best_c = val, C
        heights.append(best_c)
        stored += sum(best_c * int(L[k * best_c:(k + 1) * best_c].max()) for k in range(w // best_c))
    return np.array(heights, dtype=np.int32), stored


CASES = [
    ("structural_8_bs8_w32_K8", lambda: W.irregular_structural(8, 7), 8, 32, None, 8),
    ("structural_7_bs4_w16_K1", lambda: W.irregular_structural(7, 2), 4, 16, None, 1),
    ("hetero27_9_rand_w8_K4", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                      W.random_order(2, 729)), 8, 8, None, 4),
    ("poisson7_9_box_w32_K2", lambda: W.poisson7(9), 8, 32, (2, 2, 2), 2),
    ("curlcurl_5_rand_w32_K16", lambda: W.permute_input(W.curl_curl(5, 0.01, 3, 0.5), W.random_order(5, 540)),
     8, 32, None, 16),
    ("veclap_5_rand_w2_K3", lambda: W.permute_input(W.vector_laplacian(5, 3), W.random_order(4, 375)), 8, 2, None, 3),
    ("veclap_4_rand_w1_K3", lambda: W.permute_input(W.vector_laplacian(4, 3), W.random_order(4, 192)), 4, 1, None, 3),
]


@pytest.mark.parametrize("name,mk,bs,w,box,K", CASES)
def test_host_vslice_plan(lib, orc, name, mk, bs, w, box, K):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box, host_only=True, sell_vslice=K)
    an = orc.analyse(A, bs, w, box=box)
    heights, stored = expected_plan(an.row_ptr, w, K)
    np.testing.assert_array_equal(H.hbmc_get_vslice(ctx), heights)
    inf = ctx.info()
    assert inf["sell_entries_vslice"] == stored
    # never more than the plain layout's padded entries, never fewer than the nonzeros
    assert an.row_ptr[-1] <= stored <= inf["sell_entries_a"]


def test_host_vslice_large_cost_keeps_full_slices(lib, orc):
    """With a per-sub-slice charge larger than any saving, every slice keeps
    C = w and the layout is the plain one's size."""
    A = W.irregular_structural(6, 3)
    ctx = H.hbmc_build(A, 8, 32, host_only=True, sell_vslice=10 ** 6)
    assert np.all(H.hbmc_get_vslice(ctx) == 32)
    inf = ctx.info()
    assert inf["sell_entries_vslice"] == inf["sell_entries_a"]


def test_host_vslice_argument_checks(lib):
    A = W.poisson7(4)
    with pytest.raises(H.HbmcError):
        H.hbmc_build(A, 8, 32, host_only=True, sell_vslice=-1)
    ctx = H.hbmc_build(A, 8, 32, host_only=True)
    assert ctx.info()["sell_entries_vslice"] == 0
    with pytest.raises(H.HbmcError):
        H.hbmc_get_vslice(ctx)
    E = W.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    ctx = H.hbmc_build(E, 8, 32, host_only=True, sell_vslice=4)
    assert ctx.info()["sell_entries_vslice"] == 0 and H.hbmc_get_vslice(ctx).size == 0
