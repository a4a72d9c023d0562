"""Dependency-driven sweeps (sweep_kernel 8): every color of a substitution
in one launch, each level-1 block waiting only for the level-1 blocks of
other colors whose rows it reads (Section 4.3.3's synchronizations done per
block instead of per color).

Checked through the C ABI against the CPU oracle: the substitutions bit for
bit (the per-row term order is the oracle's), the solve with the oracle's
iteration count; that the epoch-numbered flags stay consistent over many
launches in both loop modes; and that a wait that runs out -- forced with
the test hook hbmc_debug_stall, which makes one level-1 block withhold its
completion flag -- ends the solve with HBMC_ERR_TIMEOUT and leaves the
context usable."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("poisson7_8_bs8", lambda: W.poisson7(8), 8, (2, 2, 2)),
    ("poisson7_9_bs4", lambda: W.poisson7(9), 4, (1, 2, 2)),
    ("poisson7_10_bs16", lambda: W.poisson7(10), 16, (2, 2, 4)),
    ("hetero27_12_rand", lambda: W.permute_input(W.heterogeneous_stencil(12, 27, 2.0, 1),
                                                 W.random_order(2, 1728)), 8, None),
    ("veclap_7_rand", lambda: W.permute_input(W.vector_laplacian(7, 3), W.random_order(4, 1029)), 8, None),
    ("hetero27_10_rand_bs32", lambda: W.permute_input(W.heterogeneous_stencil(10, 27, 1.0, 5),
                                                      W.random_order(6, 1000)), 32, None),
    # about 37 level-1 blocks per color: a level-1 block reads more than 16
    # level-1 blocks of a color and waits on that color's counter instead
    ("hetero27_60_rand", lambda: W.permute_input(W.heterogeneous_stencil(60, 27, 2.0, 1),
                                                 W.random_order(2, 216000)), 8, None),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return H.load()


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name,mk,bs,box", CASES)
def test_dag_sweeps_bitwise_and_solve(lib, orc, name, mk, bs, box):
    A = mk()
    ctx = H.hbmc_build(A, bs, 32, box=box, sweep_kernel=8)
    assert H.hbmc_ic0(ctx, 0.05) == (H.OK, -1)
    an = orc.analyse(A, bs, 32, box=box)
    lval, _, dinv, bad = orc.factor(an, 0.05)
    assert bad == -1
    r = np.random.default_rng(21).standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z_ref = orc.bwd(an.row_ptr, an.col, lval, dinv, y_ref)
    y = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    z = torch.empty_like(y)
    # several launches in a row: the epochs advance, the bits stay the oracle's
    for _ in range(3):
        H.hbmc_fwd_bar(ctx, dev(r), y)
        H.hbmc_bwd_bar(ctx, dev(y_ref), z)
        np.testing.assert_array_equal(host(y), y_ref)
        np.testing.assert_array_equal(host(z), z_ref)
    b, _ = W.rhs_from_solution(A, 0)
    ref = orc.pcg(an, lval, dinv, b, tol=1e-8)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
    assert res.status == H.OK and res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-12
    # the preconditioner on original-order vectors (dummy rows have no
    # couplings, so their entries of r do not reach the real rows)
    pi = np.asarray(an.pi)
    zr = orc.bwd(an.row_ptr, an.col, lval, dinv, orc.fwd(an.row_ptr, an.col, lval, dinv, r))
    zo = torch.empty(A.n, dtype=torch.float64, device="cuda")
    H.hbmc_precond(ctx, dev(r[pi]), zo)
    np.testing.assert_array_equal(host(zo), zr[pi])


@pytest.mark.parametrize("name,mk,bs,box", CASES[:5])
def test_dag_fp32_matches_per_color_kernels(lib, name, mk, bs, box):
    """FP32 substitutions: the same bits as the per-color kernels (the
    bulk-copy warp kernels for bs 4 and 8, else the automatic choice)."""
    A = mk()
    outs = []
    for sk in (5 if bs in (4, 8) else 0, 8):
        ctx = H.hbmc_build(A, bs, 32, box=box, sweep_kernel=sk, precision=H.PREC_F32)
        assert H.hbmc_ic0(ctx, 0.0)[0] == H.OK
        n_pad = ctx.info()["n_pad"]
        r = np.random.default_rng(5).standard_normal(n_pad)
        y = torch.empty(n_pad, dtype=torch.float64, device="cuda")
        z = torch.empty_like(y)
        H.hbmc_fwd_bar(ctx, dev(r), y)
        H.hbmc_bwd_bar(ctx, y, z)
        b, _ = W.rhs_from_solution(A, 1)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
        assert res.status == H.OK
        outs.append((host(y), host(z), res.iters, host(x)))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]
    assert _rel(outs[1][3], outs[0][3]) <= 1e-12


def test_dag_graph_and_host_loop_agree_bitwise(lib):
    A = W.permute_input(W.heterogeneous_stencil(12, 27, 2.0, 1), W.random_order(2, 1728))
    b, _ = W.rhs_from_solution(A, 0)
    xs = []
    for mode in (H.LOOP_GRAPH, H.LOOP_HOST, H.LOOP_GRAPH):
        ctx = H.hbmc_build(A, 8, 32, sweep_kernel=8, loop_mode=mode, check_every=3)
        assert H.hbmc_ic0(ctx)[0] == H.OK
        for _ in range(2):  # a second solve on the same flags and counters
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-10)
            assert res.status == H.OK
            xs.append((res.iters, host(x)))
    for it, x in xs[1:]:
        assert it == xs[0][0]
        np.testing.assert_array_equal(x, xs[0][1])


@pytest.mark.parametrize("m,loop_mode,last", [(10, H.LOOP_GRAPH, False), (10, H.LOOP_HOST, False),
                                               (60, H.LOOP_GRAPH, False), (60, H.LOOP_GRAPH, True),
                                               (60, H.LOOP_HOST, True)])
def test_dag_wait_runs_out_and_context_recovers(lib, m, loop_mode, last):
    """A level-1 block withholds its completion: the level-1 blocks that
    gather from it (through its flag at 10^3, through its color's counter at
    60^3) wait 0.2 s, give up, and the solve returns HBMC_ERR_TIMEOUT.  A
    block of the first color stalls the forward sweep; a block of the last
    color (last = True) is read by nobody in the forward sweep, so the wait
    runs out in the backward sweep, the one that reduces r.z.  With the hook
    cleared the same context solves again, to the same bits as an
    undisturbed context (the reduction counters start clean)."""
    A = W.permute_input(W.heterogeneous_stencil(m, 27, 2.0, 1), W.random_order(2, m ** 3))
    b, _ = W.rhs_from_solution(A, 0)
    ref_ctx = H.hbmc_build(A, 8, 32, sweep_kernel=8)
    assert H.hbmc_ic0(ref_ctx)[0] == H.OK
    x_ref = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    ref = H.hbmc_iccg(ref_ctx, dev(b), x_ref)
    assert ref.status == H.OK
    ctx = H.hbmc_build(A, 8, 32, sweep_kernel=8, loop_mode=loop_mode)
    assert H.hbmc_ic0(ctx)[0] == H.OK
    assert ctx.info()["nc"] > 2
    H.hbmc_debug_stall(ctx, ctx.info()["ntiles"] - 1 if last else 0, 0.2)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_iccg(ctx, dev(b), x)
    assert e.value.status == H.ERR_TIMEOUT
    torch.cuda.synchronize()  # the context and the device are still usable
    H.hbmc_debug_stall(ctx, -1, 0.0)
    x.zero_()
    res = H.hbmc_iccg(ctx, dev(b), x)
    assert res.status == H.OK and res.iters == ref.iters
    np.testing.assert_array_equal(host(x), host(x_ref))


def test_dag_stall_hook_rejects_bad_unit(lib):
    A = W.poisson7(6)
    ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2), sweep_kernel=8)
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_debug_stall(ctx, 10 ** 9, 0.1)
    assert e.value.status == H.ERR_INVALID_ARG
