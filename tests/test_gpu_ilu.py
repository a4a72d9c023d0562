"""GPU ILU(0) and ILU(0)-preconditioned BiCGStab for nonsymmetric values on a
symmetric pattern, against the oracle (orc_ilu0, orc_bwd_u, orc_bicgstab):
L and U bit-equal, both substitutions bit-equal, BiCGStab with the oracle's
iteration count and x within 1e-10, in graph and host-loop modes and with
FP32 substitutions, edge cases, and the 128^3 convection-diffusion system."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("convdiff_8_bs8_w32", lambda: W.convection_diffusion(8), 8, 32, (2, 2, 2)),
    ("convdiff_7_ragged", lambda: W.convection_diffusion(7, (1.0, 0.5, 2.0)), 8, 32, (2, 2, 2)),
    ("convdiff_9_bs4_w32", lambda: W.convection_diffusion(9), 4, 32, (1, 2, 2)),
    ("convdiff_10_bs16_w8", lambda: W.convection_diffusion(10), 16, 8, (2, 2, 4)),
    ("convdiff_9_rand", lambda: W.permute_input(W.convection_diffusion(9, (3.0, 0.0, 1.0)),
                                                W.random_order(6, 729)), 8, 32, None),
    ("convdiff_6_bs1_w1", lambda: W.convection_diffusion(6), 1, 1, None),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _setup(orc, A, bs, w, box, shift=0.0, **kw):
    ctx = H.hbmc_build(A, bs, w, box=box, nonsymmetric=True, **kw)
    st, bad = H.hbmc_ilu0(ctx, shift)
    assert st == H.OK and bad == -1
    an = orc.analyse(A, bs, w, box=box)
    lval, uval, udiag, uinv, obad = orc.factor_ilu(an, shift)
    assert obad == -1
    return ctx, an, lval, uval, udiag, uinv


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("shift", [0.0, 0.2])
def test_ilu0_factor_and_substitutions_bitwise(lib, orc, name, mk, bs, w, box, shift):
    A = mk()
    ctx, an, lval, uval, udiag, uinv = _setup(orc, A, bs, w, box, shift)
    glo, gdiag = H.hbmc_get_factor(ctx)
    gup = H.hbmc_get_factor_u(ctx)
    rows = np.repeat(np.arange(an.n_pad), np.diff(an.row_ptr))
    low, up = an.col < rows, an.col > rows
    np.testing.assert_array_equal(glo[low], lval[low])
    np.testing.assert_array_equal(gup[up], uval[up])
    np.testing.assert_array_equal(gdiag, udiag)
    r = np.random.default_rng(5).standard_normal(an.n_pad)
    y_ref = orc.fwd(an.row_ptr, an.col, lval, np.ones(an.n_pad), r)
    z_ref = orc.bwd_u(an.row_ptr, an.col, uval, uinv, y_ref)
    y, z = (torch.empty(an.n_pad, dtype=torch.float64, device="cuda") for _ in range(2))
    H.hbmc_fwd_bar(ctx, dev(r), y)
    H.hbmc_bwd_bar(ctx, dev(y_ref), z)
    np.testing.assert_array_equal(host(y), y_ref)
    np.testing.assert_array_equal(host(z), z_ref)


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("loop_mode", [H.LOOP_GRAPH, H.LOOP_HOST])
def test_bicgstab_matches_oracle(lib, orc, name, mk, bs, w, box, loop_mode):
    A = mk()
    b, _ = W.rhs_from_solution(A, 0)
    ctx, an, lval, uval, udiag, uinv = _setup(orc, A, bs, w, box, loop_mode=loop_mode, check_every=3)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_bicgstab(ctx, dev(b), x, tol=1e-10)
    ref = orc.bicgstab(an, lval, uval, uinv, b, tol=1e-10)
    assert ref.status == 0 and res.status == H.OK
    assert res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-10
    assert res.true_relres < 1.1e-10


def test_bicgstab_fp32_substitutions_reach_the_tolerance(lib, orc):
    A = W.convection_diffusion(12, (2.0, 1.0, 0.5))
    b, xstar = W.rhs_from_solution(A, 0)
    ctx, an, lval, uval, udiag, uinv = _setup(orc, A, 8, 32, (2, 2, 2))
    ref = orc.bicgstab(an, lval, uval, uinv, b, tol=1e-9)
    H.hbmc_set_precision(ctx, H.PREC_F32)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_bicgstab(ctx, dev(b), x, tol=1e-9)
    assert res.status == H.OK and res.true_relres < 1.1e-9
    assert abs(res.iters - ref.iters) <= 2


def test_nonsymmetric_edge_cases(lib, orc):
    A = W.convection_diffusion(6)
    ctx, an, lval, uval, udiag, uinv = _setup(orc, A, 8, 32, (2, 2, 2))
    x = dev(np.ones(A.n))
    r = H.hbmc_bicgstab(ctx, dev(np.zeros(A.n)), x)
    assert r.status == H.OK and r.iters == 0 and np.all(host(x) == 0)
    b, _ = W.rhs_from_solution(A, 1)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_bicgstab(ctx, dev(b), x, maxit=0)
    assert r.status == H.NOT_CONVERGED and r.iters == 0
    ref = orc.bicgstab(an, lval, uval, uinv, b, maxit=2)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = H.hbmc_bicgstab(ctx, dev(b), x, maxit=2)
    assert r.status == H.NOT_CONVERGED and r.iters == 2 and ref.status == 1
    assert _rel(host(x), ref.x) <= 1e-12
    # IC(0) and CG are refused on nonsymmetric contexts, ILU(0) on symmetric ones
    with pytest.raises(H.HbmcError):
        H.hbmc_ic0(ctx)
    with pytest.raises(H.HbmcError):
        H.hbmc_iccg(ctx, dev(b), x)
    sym = H.hbmc_build(W.poisson7(6), 8, 32, box=(2, 2, 2))
    with pytest.raises(H.HbmcError):
        H.hbmc_ilu0(sym)
    # a nonsymmetric value set without the option is refused at build time
    with pytest.raises(H.HbmcError):
        H.hbmc_build(A, 8, 32, box=(2, 2, 2))


def test_zero_pivot_matches_oracle_row(lib, orc):
    """A row with a tiny diagonal and huge couplings: whichever of it and its
    neighbours comes first in the ordering, a later pivot overflows."""
    import scipy.sparse as sp
    n = 40
    M = sp.diags([np.full(n - 1, -1.0), np.full(n, 4.0), np.full(n - 1, -1.0)], [-1, 0, 1]).tolil()
    M[17, 17] = 1e-300
    for a, c in ((17, 16), (16, 17), (17, 18), (18, 17)):
        M[a, c] = 1e200
    M = M.tocsr()
    M.sort_indices()
    A = W.CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))
    ctx = H.hbmc_build(A, 4, 2, nonsymmetric=True)
    st, bad = H.hbmc_ilu0(ctx)
    an = orc.analyse(A, 4, 2)
    *_, obad = orc.factor_ilu(an)
    assert obad >= 0 and st == H.ERR_NOT_SPD_PIVOT
    inv = np.full(an.n_pad, -1)
    inv[an.pi] = np.arange(n)
    assert bad == inv[obad]


def test_bicgstab_full_size_convection_diffusion128(lib, orc):
    P = W.convection_diffusion_problem(128, bs=8)
    ctx, an, lval, uval, udiag, uinv = _setup(orc, P.A, 8, 32, P.box)
    x = torch.zeros(P.A.n, dtype=torch.float64, device="cuda")
    res = H.hbmc_bicgstab(ctx, dev(P.b), x, tol=1e-8)
    ref = orc.bicgstab(an, lval, uval, uinv, P.b, tol=1e-8)
    assert res.status == H.OK and ref.status == 0 and res.iters == ref.iters
    assert _rel(host(x), ref.x) <= 1e-10
    assert res.true_relres < 1.1e-8
