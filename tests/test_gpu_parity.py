"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

The oracle and the kernels sum every row in the same term order with fused
multiply-adds (forward and IC(0): ascending columns; backward: descending;
SpMV: ascending from zero), so IC(0), the substitutions and SpMV are compared
bit for bit.  Dot products are summed in a different order on the two sides
(deterministic tree on the GPU, sequential on the CPU), so the full solve is
compared by iteration count and by iterates within 1e-12 relative.
"""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("poisson7_8_bs8_w32", lambda: W.poisson7(8), 8, 32, (2, 2, 2)),
    ("poisson7_7_ragged", lambda: W.poisson7(7), 8, 32, (2, 2, 2)),
    ("poisson7_9_bs4_w32", lambda: W.poisson7(9), 4, 32, (1, 2, 2)),
    ("poisson7_10_bs16_w8", lambda: W.poisson7(10), 16, 8, (2, 2, 4)),
    ("poisson7_9_bs32_w4", lambda: W.poisson7(9), 32, 4, (2, 4, 4)),
    ("hetero27_9_rand", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                W.random_order(2, 729)), 8, 32, None),
    ("veclap_5_rand", lambda: W.permute_input(W.vector_laplacian(5, 3), W.random_order(4, 375)), 8, 16, None),
    ("hetero7_6_bs1_w1", lambda: W.heterogeneous_stencil(6, 7, 1.5, 3), 1, 1, None),
    ("poisson7_6_bs64_w2", lambda: W.poisson7(6), 64, 2, None),
    ("poisson7_5_bs3_w2", lambda: W.poisson7(5), 3, 2, None),
    # rows of 40-190 entries: the loader-thread sweeps stage the other-color
    # runs (about 25k entries a level-1 block) in groups of steps
    ("structural_8_bs8_w32", lambda: W.irregular_structural(8, 7), 8, 32, None),
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


def _setup(orc, A, bs, w, box, shift=0.0, precision=H.PREC_F64, loop_mode=H.LOOP_GRAPH):
    ctx = H.hbmc_build(A, bs, w, box=box, precision=precision, loop_mode=loop_mode)
    st, bad = H.hbmc_ic0(ctx, shift)
    assert st == H.OK and bad == -1
    an = orc.analyse(A, bs, w, box=box)
    lval, ldiag, dinv, obad = orc.factor(an, shift)
    assert obad == -1
    return ctx, an, lval, ldiag, dinv


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("shift", [0.0, 0.25])
def test_ic0_bitwise(lib, orc, name, mk, bs, w, box, shift):
    A = mk()
    ctx, an, lval, ldiag, _ = _setup(orc, A, bs, w, box, shift)
    glo, gdiag = H.hbmc_get_factor(ctx)
    rows = np.repeat(np.arange(an.n_pad), np.diff(an.row_ptr))
    low = an.col < rows
    np.testing.assert_array_equal(glo[low], lval[low])
    np.testing.assert_array_equal(gdiag, ldiag)


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
def test_substitutions_and_spmv_bitwise(lib, orc, name, mk, bs, w, box):
    A = mk()
    ctx, an, lval, ldiag, dinv = _setup(orc, A, bs, w, box, 0.1)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z_ref = orc.bwd(an.row_ptr, an.col, lval, dinv, y_ref)
    q_ref = orc.spmv(an.row_ptr, an.col, an.val, r)
    y, z, q = (torch.empty(an.n_pad, dtype=torch.float64, device="cuda") for _ in range(3))
    H.hbmc_fwd_bar(ctx, dev(r), y)
    H.hbmc_bwd_bar(ctx, dev(y_ref), z)
    H.hbmc_spmv_bar(ctx, dev(r), q)
    np.testing.assert_array_equal(host(y), y_ref)
    np.testing.assert_array_equal(host(z), z_ref)
    np.testing.assert_array_equal(host(q), q_ref)


@pytest.mark.parametrize("name,mk,bs,w,box", CASES[:6])
def test_fp32_substitutions_within_fp32_error(lib, orc, name, mk, bs, w, box):
    """FP32 factor and accumulation: the error against the FP64 oracle stays at
    FP32 rounding level (relative 1e-4 in the max norm)."""
    A = mk()
    ctx, an, lval, ldiag, dinv = _setup(orc, A, bs, w, box, 0.0, precision=H.PREC_F32)
    rng = np.random.default_rng(8)
    r = rng.standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z_ref = orc.bwd(an.row_ptr, an.col, lval, dinv, y_ref)
    y = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    z = torch.empty_like(y)
    H.hbmc_fwd_bar(ctx, dev(r), y)
    H.hbmc_bwd_bar(ctx, dev(y_ref), z)
    yh, zh = host(y), host(z)
    assert np.max(np.abs(yh - y_ref)) <= 1e-4 * np.max(np.abs(y_ref))
    assert np.max(np.abs(zh - z_ref)) <= 1e-4 * np.max(np.abs(z_ref))
    assert not np.array_equal(yh, y_ref)  # it really ran in FP32


@pytest.mark.parametrize("name,mk,bs,w,box", CASES[:6])
def test_precond_original_order_bitwise(lib, orc, name, mk, bs, w, box):
    A = mk()
    ctx, an, lval, ldiag, dinv = _setup(orc, A, bs, w, box)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(A.n)
    rbar = np.zeros(an.n_pad)
    rbar[an.pi] = r
    zbar = orc.bwd(an.row_ptr, an.col, lval, dinv, orc.fwd(an.row_ptr, an.col, lval, dinv, rbar))
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    H.hbmc_precond(ctx, dev(r), z)
    np.testing.assert_array_equal(host(z), zbar[an.pi])


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("loop_mode", [H.LOOP_GRAPH, H.LOOP_HOST, H.LOOP_PERSISTENT])
def test_iccg_matches_oracle(lib, orc, name, mk, bs, w, box, loop_mode):
    A = mk()
    b, _ = W.rhs_from_solution(A, 0)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, bs, w, box, loop_mode=loop_mode)
    ref = orc.pcg(an, lval, dinv, b, tol=1e-8)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8, maxit=10000)
    assert res.status == H.OK and ref.status == 0
    assert res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-12
    hist = H.hbmc_residual_history(ctx)
    np.testing.assert_allclose(hist, ref.hist, rtol=1e-10)
    assert abs(res.relres - ref.relres) <= 1e-10 * ref.relres
    true = np.linalg.norm(b - A.to_scipy() @ host(x)) / np.linalg.norm(b)
    assert abs(res.true_relres - true) <= 1e-6 * true


def test_graph_and_host_loop_agree_bitwise(lib, orc):
    A = W.poisson7(12)
    b, _ = W.rhs_from_solution(A, 0)
    xs = []
    for mode in (H.LOOP_GRAPH, H.LOOP_HOST):
        ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2), loop_mode=mode, check_every=5)
        H.hbmc_ic0(ctx)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = H.hbmc_iccg(ctx, dev(b), x)
        xs.append((r.iters, host(x)))
    assert xs[0][0] == xs[1][0]
    np.testing.assert_array_equal(xs[0][1], xs[1][1])


def test_repeated_solves_are_deterministic(lib, orc):
    A = W.permute_input(W.heterogeneous_stencil(10, 27, 2.0, 1), W.random_order(2, 1000))
    ctx = H.hbmc_build(A, 8, 32)
    H.hbmc_ic0(ctx)
    outs = []
    for seed in (0, 1, 0):
        b, _ = W.rhs_from_solution(A, seed)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = H.hbmc_iccg(ctx, dev(b), x)
        outs.append((r.iters, host(x)))
    assert outs[0][0] == outs[2][0]
    np.testing.assert_array_equal(outs[0][1], outs[2][1])
    assert not np.array_equal(outs[0][1], outs[1][1])


def test_fp32_preconditioner_reaches_fp64_tolerance(lib, orc):
    A = W.poisson7(24)
    b, _ = W.rhs_from_solution(A, 0)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, 8, 32, (2, 2, 2), precision=H.PREC_F32)
    ref = orc.pcg(an, lval, dinv, b, tol=1e-8)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
    assert res.status == H.OK
    assert abs(res.iters - ref.iters) <= max(2, ref.iters // 20)
    assert res.true_relres < 2e-8
    assert _rel(host(x), ref.x) < 1e-6


def test_initial_guess_and_restart(lib, orc):
    A = W.poisson7(10)
    b, xs = W.rhs_from_solution(A, 3)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, 8, 32, (2, 2, 2))
    x0 = 0.5 * xs
    ref = orc.pcg(an, lval, dinv, b, tol=1e-9, x0=x0)
    x = dev(x0)
    res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-9)
    assert res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-12
    # restarting from the converged x: already below the tolerance -> 0 iterations
    res2 = H.hbmc_iccg(ctx, dev(b), x, tol=1e-7)
    assert res2.status == H.OK and res2.iters == 0


@pytest.mark.parametrize("precision", [H.PREC_F64, H.PREC_F32])
def test_single_color_fused_preconditioner(lib, orc, precision):
    """A system of one color: the last color is also the first, so the fused
    forward-backward pass is the whole preconditioner and its own launch
    reduces r.z.  Bulk-copy warp kernels forced (sweep_kernel 5) against the
    block-per-level-1-block kernels (1), and FP64 against the oracle."""
    A = W.poisson7(2)  # 8 unknowns, one 2x2x2 box, one color
    b, _ = W.rhs_from_solution(A, 0)
    outs = []
    for sk in (5, 1):
        ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2), sweep_kernel=sk, precision=precision)
        assert ctx.info()["nc"] == 1
        assert H.hbmc_ic0(ctx, 0.0)[0] == H.OK
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-10)
        z = torch.empty(A.n, dtype=torch.float64, device="cuda")
        H.hbmc_precond(ctx, dev(b), z)
        outs.append((res.iters, host(x), host(z)))
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])
    if precision == H.PREC_F64:
        an = orc.analyse(A, 8, 32, box=(2, 2, 2))
        lval, _, dinv, _ = orc.factor(an, 0.0)
        ref = orc.pcg(an, lval, dinv, b, tol=1e-10)
        assert outs[0][0] == ref.iters and _rel(outs[0][1], ref.x) <= 1e-12


def test_edge_cases(lib, orc):
    A = W.poisson7(6)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, 8, 32, (2, 2, 2))
    # zero right-hand side: x = 0, no iterations
    x = dev(np.ones(A.n))
    r = H.hbmc_iccg(ctx, dev(np.zeros(A.n)), x)
    assert r.status == H.OK and r.iters == 0 and np.all(host(x) == 0)
    # maxit = 0 and maxit = 3
    b, _ = W.rhs_from_solution(A, 0)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, dev(b), x, maxit=0)
    assert r.status == H.NOT_CONVERGED and r.iters == 0
    ref = orc.pcg(an, lval, dinv, b, maxit=3)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, dev(b), x, maxit=3)
    assert r.status == H.NOT_CONVERGED and r.iters == 3 and ref.status == 1
    assert _rel(host(x), ref.x) <= 1e-12
    # solve before factorization
    ctx2 = H.hbmc_build(A, 8, 32, box=(2, 2, 2))
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_iccg(ctx2, dev(b), x)
    assert e.value.status == H.ERR_NOT_FACTORED
    # bad arguments
    with pytest.raises(ValueError):
        H.hbmc_iccg(ctx, dev(b[:-1]), x)
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_ic0(ctx, -1.0)
    assert e.value.status == H.ERR_INVALID_ARG


@pytest.mark.parametrize("opts", [{}, {"sell_split": 16}, {"sweep_kernel": 7}, {"sweep_kernel": 5}])
def test_empty_system_on_device(lib, opts):
    A = W.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    ctx = H.hbmc_build(A, 8, 32, **opts)
    assert H.hbmc_ic0(ctx)[0] == H.OK
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, e, e)
    assert r.status == H.OK and r.iters == 0


def _indefinite(n=40, seed=3):
    """Symmetric tridiagonal-plus matrix with a negative eigenvalue but a
    positive diagonal."""
    rng = np.random.default_rng(seed)
    M = np.diag(np.full(n, 1.0)) + np.diag(np.full(n - 1, 0.9), 1) + np.diag(np.full(n - 1, 0.9), -1)
    import scipy.sparse as sp
    S = sp.csr_matrix(M)
    S.sort_indices()
    return W.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def test_not_spd_pivot_reports_oracle_row(lib, orc):
    A = _indefinite()
    for bs, w in ((4, 2), (1, 1), (8, 4)):
        ctx = H.hbmc_build(A, bs, w)
        st, bad = H.hbmc_ic0(ctx, 0.0)
        an = orc.analyse(A, bs, w)
        _, _, _, obad = orc.factor(an, 0.0)
        assert obad >= 0 and st == H.ERR_NOT_SPD_PIVOT
        inv = np.full(an.n_pad, -1)
        inv[an.pi] = np.arange(A.n)
        assert bad == inv[obad]
        with pytest.raises(H.HbmcError):
            H.hbmc_iccg(ctx, dev(np.ones(A.n)), torch.zeros(A.n, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("bs,w", [(4, 2), (4, 32), (8, 32)])
def test_cg_breakdown_matches_oracle(lib, orc, bs, w):
    """Indefinite A with a shift large enough for IC(0): CG breaks down on a
    non-positive p.q, at the same iteration as the oracle, for the plain
    and the bulk-copy-fed kernels."""
    A = _indefinite()
    ctx = H.hbmc_build(A, bs, w)
    assert H.hbmc_ic0(ctx, 2.0)[0] == H.OK
    an = orc.analyse(A, bs, w)
    lval, _, dinv, _ = orc.factor(an, 2.0)
    b = np.cos(np.arange(A.n))
    ref = orc.pcg(an, lval, dinv, b, tol=1e-12, maxit=500)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, dev(b), x, tol=1e-12, maxit=500)
    assert ref.status == 2 and r.status == H.ERR_BREAKDOWN
    assert r.iters == ref.iters


def test_host_buffer_entry_point(lib, orc):
    A = W.poisson7(16)
    b, _ = W.rhs_from_solution(A, 0)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, 8, 32, (2, 2, 2))
    ref = orc.pcg(an, lval, dinv, b)
    x = np.zeros(A.n)
    r = H.hbmc_iccg_host(ctx, b, x)
    assert r.iters == ref.iters and _rel(x, ref.x) <= 1e-12


def test_stream_binding(lib, orc):
    A = W.poisson7(12)
    b, _ = W.rhs_from_solution(A, 0)
    ctx, an, lval, ldiag, dinv = _setup(orc, A, 8, 32, (2, 2, 2))
    s = torch.cuda.Stream()
    H.hbmc_set_stream(ctx, s)
    with torch.cuda.stream(s):
        bd = dev(b)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    s.synchronize()
    r = H.hbmc_iccg(ctx, bd, x)
    ref = orc.pcg(an, lval, dinv, b)
    assert r.iters == ref.iters and _rel(host(x), ref.x) <= 1e-12


@pytest.mark.parametrize("bs", [8, 16, 32])
def test_full_size_poisson128(lib, orc, bs):
    """The 7-point 128^3 workload in the configuration the benchmark times
    (geometric bs-boxes, w = 32, FP64), against the full oracle solve."""
    P = W.poisson_problem(128, bs=bs)
    ctx, an, lval, ldiag, dinv = _setup(orc, P.A, bs, 32, P.box)
    assert ctx.info()["nc"] == 2
    x = torch.zeros(P.A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_iccg(ctx, dev(P.b), x, tol=1e-8)
    ref = orc.pcg(an, lval, dinv, P.b, tol=1e-8)
    assert res.status == H.OK and res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-12
    assert res.true_relres < 1.1e-8


@pytest.mark.parametrize("tpb,w,bs", [(1, 32, 8), (2, 32, 8), (4, 32, 8), (8, 32, 8), (2, 32, 16),
                                      (8, 8, 8), (32, 8, 4), (1, 16, 16), (4, 4, 2)])
def test_sweep_geometry_variants_bitwise(lib, orc, tpb, w, bs):
    """Any number of level-1 blocks per CUDA block gives the same bits."""
    box = W.box_for_bs(bs)
    A = W.poisson7(11)
    ctx = H.hbmc_build(A, bs, w, box=box, sweep_tpb=tpb)
    assert H.hbmc_ic0(ctx, 0.05)[0] == H.OK
    an = orc.analyse(A, bs, w, box=box)
    lval, ldiag, dinv, _ = orc.factor(an, 0.05)
    r = np.random.default_rng(tpb).standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z_ref = orc.bwd(an.row_ptr, an.col, lval, dinv, y_ref)
    y = torch.empty(an.n_pad, dtype=torch.float64, device="cuda")
    z = torch.empty_like(y)
    H.hbmc_fwd_bar(ctx, dev(r), y)
    H.hbmc_bwd_bar(ctx, dev(y_ref), z)
    np.testing.assert_array_equal(host(y), y_ref)
    np.testing.assert_array_equal(host(z), z_ref)


@pytest.mark.parametrize("name,mk,bs,w,box", [c for c in CASES if c[3] == 32])
@pytest.mark.parametrize("precision", [H.PREC_F64, H.PREC_F32])
def test_sweep_kernel_variants_agree(lib, orc, name, mk, bs, w, box, precision):
    """Every substitution kernel computes the same bits, in both precisions,
    and FP64 matches the oracle: 0 automatic (loader-thread blocks for these
    small colors), 1 block per level-1 block, 3 warp
    per level-1 block with plain loads, 4 loader-thread blocks staged by bulk
    copy, 5 warp per level-1 block staged by bulk copy (bs 4 and 8), 6
    loader-thread blocks with plain loads, 7 loader-thread sweeps split over
    bs CUDA blocks per level-1 block, 8 dependency-driven (every color in one
    launch)."""
    A = mk()
    outs = []
    for sk in (0, 1, 3, 4, 5, 6, 7, 8):
        ctx = H.hbmc_build(A, bs, w, box=box, sweep_kernel=sk, precision=precision)
        assert H.hbmc_ic0(ctx, 0.1)[0] == H.OK
        n_pad = ctx.info()["n_pad"]
        r = np.random.default_rng(11).standard_normal(n_pad)
        y = torch.empty(n_pad, dtype=torch.float64, device="cuda")
        z = torch.empty_like(y)
        q = torch.empty_like(y)
        H.hbmc_fwd_bar(ctx, dev(r), y)
        H.hbmc_bwd_bar(ctx, y, z)
        H.hbmc_spmv_bar(ctx, dev(r), q)
        b, _ = W.rhs_from_solution(A, 0)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x)
        outs.append((host(y), host(z), res.iters, host(x), host(q)))
    assert all(o[2] > 0 for o in outs)
    for o in outs[1:]:
        for k in (0, 1, 4):  # substitutions and SpMV: identical term order, identical bits
            np.testing.assert_array_equal(outs[0][k], o[k])
        # the dot products reduce in kernel-specific orders: equal counts, x to 1e-12
        assert outs[0][2] == o[2]
        assert _rel(o[3], outs[0][3]) <= 1e-12
    if precision == H.PREC_F64:
        an = orc.analyse(A, bs, w, box=box)
        lval, _, dinv, _ = orc.factor(an, 0.1)
        np.testing.assert_array_equal(outs[0][0], orc.fwd(an.row_ptr, an.col, lval, dinv, r))
        np.testing.assert_array_equal(outs[0][4], orc.spmv(an.row_ptr, an.col, an.val, r))


def test_mc_bmc_hbmc_orderings(lib, orc):
    """The paper's comparison with the library's kernels (Section 5): BMC
    (w = 1, pi_HBMC = pi_BMC) and HBMC (w = 32) with the same blocks and
    colors take the same number of iterations (Section 4.2.1's equivalence)
    and agree with the oracle; nodal MC (bs = 1) needs more iterations than
    either on the 7-point stencil."""
    A = W.poisson7(16)
    b, _ = W.rhs_from_solution(A, 0)
    out = {}
    for name, bs, w in (("MC", 1, 32), ("BMC", 8, 1), ("HBMC", 8, 32)):
        box = W.box_for_bs(bs)
        ctx, an, lval, ldiag, dinv = _setup(orc, A, bs, w, box)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(b), x, tol=1e-8)
        ref = orc.pcg(an, lval, dinv, b, tol=1e-8)
        assert res.status == H.OK and res.iters == ref.iters
        assert _rel(host(x), ref.x) <= 1e-12
        out[name] = (res.iters, host(x))
    assert out["BMC"][0] == out["HBMC"][0]
    assert _rel(out["BMC"][1], out["HBMC"][1]) <= 1e-12
    assert out["MC"][0] > out["HBMC"][0]


@pytest.mark.parametrize("which", ["hetero27_96", "veclap_100"])
def test_full_size_algebraic(lib, orc, which):
    """The random-order configurations at full size, in the launch
    configuration of the benchmark (bs = 8, w = 32, algebraic blocking), with
    the automatic choice (the dependency-driven sweeps for these many-color
    matrices) and with the per-color loader-thread kernels (sweep_kernel 4):
    IC(0), both substitutions and SpMV bit-equal to the
    oracle, the FP64 solve with the oracle's iteration count and x within
    1e-12, and the FP32-substitution solve to the FP64 tolerance."""
    P = W.heterogeneous27_problem(96) if which == "hetero27_96" else W.vector_laplacian_problem(100)
    an = orc.analyse(P.A, 8, 32)
    lval, ldiag, dinv, obad = orc.factor(an, 0.0)
    assert obad == -1
    r = np.random.default_rng(17).standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z_ref = orc.bwd(an.row_ptr, an.col, lval, dinv, y_ref)
    q_ref = orc.spmv(an.row_ptr, an.col, an.val, r)
    ref = orc.pcg(an, lval, dinv, P.b, tol=1e-8)
    rows = np.repeat(np.arange(an.n_pad), np.diff(an.row_ptr))
    low = an.col < rows
    for sk in (0, 4):
        ctx = H.hbmc_build(P.A, 8, 32, sweep_kernel=sk)
        assert H.hbmc_ic0(ctx, 0.0) == (H.OK, -1)
        assert ctx.info()["nc"] > 10
        glo, gdiag = H.hbmc_get_factor(ctx)
        np.testing.assert_array_equal(glo[low], lval[low])
        np.testing.assert_array_equal(gdiag, ldiag)
        y, z, q = (torch.empty(an.n_pad, dtype=torch.float64, device="cuda") for _ in range(3))
        H.hbmc_fwd_bar(ctx, dev(r), y)
        H.hbmc_bwd_bar(ctx, dev(y_ref), z)
        H.hbmc_spmv_bar(ctx, dev(r), q)
        np.testing.assert_array_equal(host(y), y_ref)
        np.testing.assert_array_equal(host(z), z_ref)
        np.testing.assert_array_equal(host(q), q_ref)
        x = torch.zeros(P.A.n, dtype=torch.float64, device="cuda")
        res = H.hbmc_iccg(ctx, dev(P.b), x, tol=1e-8)
        assert res.status == H.OK and res.iters == ref.iters, (sk, res.iters, ref.iters)
        assert _rel(host(x), ref.x) <= 1e-12
        H.hbmc_set_precision(ctx, H.PREC_F32)
        x.zero_()
        res32 = H.hbmc_iccg(ctx, dev(P.b), x, tol=1e-8)
        assert res32.status == H.OK and res32.true_relres < 1.1e-8
        assert abs(res32.iters - ref.iters) <= max(2, ref.iters // 20)
        del ctx


@pytest.mark.parametrize("precision", [H.PREC_F64, H.PREC_F32])
def test_persistent_solve_edge_cases(lib, orc, precision):
    """The persistent cooperative solve: zero right-hand side, maxit 0 and 3,
    restart from the solution, the FP32 substitutions, the 32^3 system."""
    A = W.poisson7(6)
    ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2), loop_mode=H.LOOP_PERSISTENT, precision=precision)
    assert H.hbmc_ic0(ctx)[0] == H.OK
    x = dev(np.ones(A.n))
    r = H.hbmc_iccg(ctx, dev(np.zeros(A.n)), x)
    assert r.status == H.OK and r.iters == 0 and np.all(host(x) == 0)
    b, _ = W.rhs_from_solution(A, 0)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(ctx, dev(b), x, maxit=0)
    assert r.status == H.NOT_CONVERGED and r.iters == 0
    an = orc.analyse(A, 8, 32, box=(2, 2, 2))
    lval, _, dinv, _ = orc.factor(an, 0.0)
    r = H.hbmc_iccg(ctx, dev(b), x, maxit=3)
    ref = orc.pcg(an, lval, dinv, b, maxit=3)
    assert r.status == H.NOT_CONVERGED and r.iters == 3
    if precision == H.PREC_F64:
        assert _rel(host(x), ref.x) <= 1e-12
    P = W.poisson_problem(32, bs=8)
    c32 = H.hbmc_build(P.A, 8, 32, box=P.box, loop_mode=H.LOOP_PERSISTENT, precision=precision)
    assert H.hbmc_ic0(c32)[0] == H.OK
    an = orc.analyse(P.A, 8, 32, box=P.box)
    lval, _, dinv, _ = orc.factor(an, 0.0)
    ref = orc.pcg(an, lval, dinv, P.b, tol=1e-8)
    x = torch.zeros(P.A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_iccg(c32, dev(P.b), x, tol=1e-8)
    assert r.status == H.OK and r.true_relres < 1.1e-8
    if precision == H.PREC_F64:
        assert r.iters == ref.iters and _rel(host(x), ref.x) <= 1e-12
    x2 = x.clone()
    r2 = H.hbmc_iccg(c32, dev(P.b), x2, tol=1e-7)
    assert r2.status == H.OK and r2.iters == 0
