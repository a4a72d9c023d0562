"""The variable-slice-height SpMV (hbmc_options.sell_vslice) on the GPU:
the product bit-equal to the oracle's SpMV (same terms, same order; only
the padding differs), and a solve with it taking the plain layout's
iteration count with iterates within 1e-12 (its p.q is reduced in its own
kernel's order, like every SpMV variant's)."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return H.load()


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


CASES = [
    ("structural_8_bs8_w32_K8", lambda: W.irregular_structural(8, 7), 8, 32, None, 8),
    ("structural_7_bs4_w16_K1", lambda: W.irregular_structural(7, 2), 4, 16, None, 1),
    ("hetero27_9_rand_w8_K4", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                      W.random_order(2, 729)), 8, 8, None, 4),
    ("poisson7_9_box_w32_K2", lambda: W.poisson7(9), 8, 32, (2, 2, 2), 2),
    ("curlcurl_6_rand_w32_K4", lambda: W.permute_input(W.curl_curl(6, 0.05, 3, 0.5), W.random_order(5, 882)),
     8, 32, None, 4),
]


@pytest.mark.parametrize("name,mk,bs,w,box,K", CASES)
def test_vslice_spmv_bitwise_and_solve(lib, orc, name, mk, bs, w, box, K):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box, sell_vslice=K)
    an = orc.analyse(A, bs, w, box=box)
    r = np.random.default_rng(3).standard_normal(an.n_pad)
    q = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    H.hbmc_spmv_bar(ctx, dev(r), q)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(q.cpu().numpy(), orc.spmv(an.row_ptr, an.col, an.val, r))
    assert np.any(H.hbmc_get_vslice(ctx) < w) or "poisson" in name
    # the solve with it: the plain layout's iteration count, iterates within 1e-12
    shift = 0.3 if "curlcurl" in name else 0.0
    b, _ = W.rhs_from_solution(A, 0)
    xs = []
    for c in (ctx, H.hbmc_build(A, bs, w, box=box)):
        assert H.hbmc_ic0(c, shift)[0] == H.OK
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(c, dev(b), x, tol=1e-8, maxit=5000)
        assert res.status == H.OK
        xs.append((res.iters, x.cpu().numpy()))
    assert xs[0][0] == xs[1][0]
    assert np.max(np.abs(xs[0][1] - xs[1][1])) <= 1e-12 * np.max(np.abs(xs[1][1]))


def test_vslice_full_size_structural(lib, orc):
    """The Audikw_1-shaped matrix at full size (943,296 unknowns): the
    variable-height product bit-equal to the oracle's on a random vector,
    with fewer stored entries than the plain SELL layout."""
    A = W.irregular_structural(68, 7)
    ctx = H.hbmc_build(A, 8, 32, sell_vslice=8)
    inf = ctx.info()
    assert inf["sell_entries_vslice"] < inf["sell_entries_a"]
    an = orc.analyse(A, 8, 32)
    r = np.random.default_rng(4).standard_normal(an.n_pad)
    q = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    H.hbmc_spmv_bar(ctx, dev(r), q)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(q.cpu().numpy(), orc.spmv(an.row_ptr, an.col, an.val, r))
