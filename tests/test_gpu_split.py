"""GPU row-split SpMV (hbmc_options.sell_split; Section 5.2.2's remedy for
SELL slices whose rows differ much in length) against the oracle: the split
product bit-identical to orc_spmv_split on the reordered system, the IC(0)-CG
solve with the oracle's split PCG iteration count and x within 1e-12, graph
and host loop bit-identical, the layout counts equal to the host build's,
edge cases, and the full-size structural workload."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("structural_8_bs8_w32_P64", lambda: W.irregular_structural(8, 7), 8, 32, None, 64, 0),
    ("structural_9_bs8_w32_P16", lambda: W.irregular_structural(9, 4), 8, 32, None, 16, 2),
    ("structural_7_bs4_w16_P16_c1", lambda: W.irregular_structural(7, 2), 4, 16, None, 16, 1),
    ("hetero27_9_rand_w8_P4_c3", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                         W.random_order(2, 729)), 8, 8, None, 4, 3),
    ("poisson7_9_box_w32_P2", lambda: W.poisson7(9), 8, 32, (2, 2, 2), 2, 1),
    ("veclap_5_rand_w1_P8", lambda: W.permute_input(W.vector_laplacian(5, 3), W.random_order(4, 375)),
     8, 1, None, 8, 2),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("name,mk,bs,w,box,P,cost", CASES)
def test_split_spmv_bitwise(lib, orc, name, mk, bs, w, box, P, cost):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box, sell_split=P, sell_split_cost=cost)
    an = orc.analyse(A, bs, w, box=box)
    plan = orc.split_plan(an.row_ptr, w, P, cost if cost > 0 else 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    inf = ctx.info()
    assert (inf["split_rows"], inf["split_pieces"], inf["sell_entries_split"]) == \
        (plan.nsplit, plan.npieces, plan.processed)
    rng = np.random.default_rng(5)
    for trial in range(2):
        p = rng.standard_normal(an.n_pad)
        q = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
        H.hbmc_spmv_bar(ctx, dev(p), q)
        np.testing.assert_array_equal(host(q), orc.spmv_split(an.row_ptr, an.col, an.val, plan, p))


@pytest.mark.parametrize("name,mk,bs,w,box,P,cost", CASES)
def test_split_iccg_matches_oracle(lib, orc, name, mk, bs, w, box, P, cost):
    A = mk()
    b, _ = W.rhs_from_solution(A, 0)
    an = orc.analyse(A, bs, w, box=box)
    lval, _, dinv, bad = orc.factor(an, 0.0)
    assert bad == -1
    plan = orc.split_plan(an.row_ptr, w, P, cost if cost > 0 else 2)
    ref = orc.pcg(an, lval, dinv, b, tol=1e-8, split=plan)
    xs = []
    for loop_mode in (H.LOOP_GRAPH, H.LOOP_HOST):
        ctx = H.hbmc_build(A, bs, w, box=box, loop_mode=loop_mode, sell_split=P, sell_split_cost=cost)
        assert H.hbmc_ic0(ctx, 0.0) == (H.OK, -1)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8, maxit=10000)
        assert res.status == H.OK and ref.status == 0
        assert res.iters == ref.iters
        assert _rel(host(x), ref.x) <= 1e-12
        assert res.true_relres < 1.1e-8
        xs.append(host(x))
    np.testing.assert_array_equal(xs[0], xs[1])


def test_split_persistent_falls_back_to_graph(lib, orc):
    """The persistent loop has no split SpMV: a split context solves through
    the graph, with the graph's bits."""
    A = W.irregular_structural(8, 7)
    b, _ = W.rhs_from_solution(A, 1)
    out = []
    for mode in (H.LOOP_GRAPH, H.LOOP_PERSISTENT):
        ctx = H.hbmc_build(A, 8, 32, loop_mode=mode, sell_split=64)
        H.hbmc_ic0(ctx, 0.0)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
        assert res.status == H.OK
        out.append((res.iters, host(x)))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_split_edge_cases(lib, orc):
    """Zero right-hand side, maxit 0 and 3, FP32 substitutions with the split
    SpMV, and a plan that cuts nothing (the unsplit product's bits)."""
    A = W.irregular_structural(8, 3)
    b, _ = W.rhs_from_solution(A, 2)
    ctx = H.hbmc_build(A, 8, 32, sell_split=32)
    H.hbmc_ic0(ctx, 0.0)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, dev(np.zeros(A.n)), x)
    assert r.status == H.OK and r.iters == 0 and not host(x).any()
    x.zero_()
    r = H.hbmc_iccg(ctx, dev(b), x, maxit=0)
    assert r.status == H.NOT_CONVERGED and r.iters == 0
    an = orc.analyse(A, 8, 32)
    lval, _, dinv, _ = orc.factor(an, 0.0)
    plan = orc.split_plan(an.row_ptr, 32, 32, 2)
    ref3 = orc.pcg(an, lval, dinv, b, tol=1e-30, maxit=3, split=plan)
    x.zero_()
    r = H.hbmc_iccg(ctx, dev(b), x, tol=1e-30, maxit=3)
    assert r.status == H.NOT_CONVERGED and r.iters == 3
    assert _rel(host(x), ref3.x) <= 1e-12
    H.hbmc_set_precision(ctx, H.PREC_F32)
    x.zero_()
    r32 = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
    assert r32.status == H.OK and r32.true_relres < 1.1e-8
    # a cost that forbids every cut: the split layout gives the plain product
    P = W.poisson7(10)
    ctxp = H.hbmc_build(P, 8, 32, box=(2, 2, 2), sell_split=8, sell_split_cost=1000)
    assert ctxp.info()["split_rows"] == 0
    anp = orc.analyse(P, 8, 32, box=(2, 2, 2))
    p = np.random.default_rng(3).standard_normal(anp.n_pad)
    q = torch.empty(anp.n_pad, dtype=torch.float64, device="cuda")
    H.hbmc_spmv_bar(ctxp, dev(p), q)
    np.testing.assert_array_equal(host(q), orc.spmv(anp.row_ptr, anp.col, anp.val, p))


def test_split_full_size_structural(lib, orc):
    """The Audikw_1-shaped stand-in at full size (68^3 nodes x 3 DOF =
    943,296 unknowns, about 78M nonzeros), in the benchmark's launch
    configuration (bs = 8, w = 32, P = 64): the plan and layout counts equal
    the oracle's, the split product is bit-identical to orc_spmv_split, and
    the split ICCG solve reaches the FP64 tolerance with the unsplit solve's
    iteration count within 2 (both measured on the GPU)."""
    A = W.irregular_structural(68, 7)
    b, _ = W.rhs_from_solution(A, 0)
    ctx = H.hbmc_build(A, 8, 32, sell_split=64)
    an = orc.analyse(A, 8, 32)
    plan = orc.split_plan(an.row_ptr, 32, 64, 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    inf = ctx.info()
    assert inf["sell_entries_split"] == plan.processed
    assert inf["sell_entries_split"] < 0.7 * inf["sell_entries_a"]
    p = np.random.default_rng(23).standard_normal(an.n_pad)
    q = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    H.hbmc_spmv_bar(ctx, dev(p), q)
    np.testing.assert_array_equal(host(q), orc.spmv_split(an.row_ptr, an.col, an.val, plan, p))
    assert H.hbmc_ic0(ctx, 0.0) == (H.OK, -1)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
    assert res.status == H.OK and res.true_relres < 1.1e-8
    ctx0 = H.hbmc_build(A, 8, 32)
    H.hbmc_ic0(ctx0, 0.0)
    x0 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res0 = H.hbmc_iccg(ctx0, dev(b), x0, tol=1e-8)
    assert res0.status == H.OK and abs(res.iters - res0.iters) <= 2
