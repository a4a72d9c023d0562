"""GPU SOR / symmetric SOR sweeps (hbmc_sor, hbmc_sor_bar) against the
oracle's orc_sor: bit-identical iterates on the reordered system for several
block sizes, level-1 widths and blockings, the original-ordering entry point
with its residual, argument checks, and the 128^3 workload."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("poisson7_8_bs8_w32", lambda: W.poisson7(8), 8, 32, (2, 2, 2)),
    ("poisson7_7_ragged_bs8_w32", lambda: W.poisson7(7), 8, 32, (2, 2, 2)),
    ("poisson7_9_bs4_w32", lambda: W.poisson7(9), 4, 32, (1, 2, 2)),
    ("poisson7_10_bs16_w8", lambda: W.poisson7(10), 16, 8, (2, 2, 4)),
    ("hetero27_9_rand", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                W.random_order(2, 729)), 8, 32, None),
    ("veclap_5_rand_w16", lambda: W.permute_input(W.vector_laplacian(5, 3), W.random_order(4, 375)), 8, 16, None),
    ("hetero7_6_bs1_w1", lambda: W.heterogeneous_stencil(6, 7, 1.5, 3), 1, 1, None),
    ("poisson7_6_bs64_w2", lambda: W.poisson7(6), 64, 2, None),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("omega,sweeps,symmetric", [(1.0, 1, False), (1.3, 3, True), (0.8, 2, False)])
def test_sor_bar_bitwise(lib, orc, name, mk, bs, w, box, omega, sweeps, symmetric):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box)
    an = orc.analyse(A, bs, w, box=box)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(an.n_pad)
    x0 = rng.standard_normal(an.n_pad)
    ref = orc.sor(an.row_ptr, an.col, an.val, b, x0, omega, sweeps, symmetric)
    x = dev(x0)
    H.hbmc_sor_bar(ctx, dev(b), x, omega, sweeps, symmetric)
    np.testing.assert_array_equal(x.cpu().numpy(), ref)


def test_sor_original_ordering_and_residual(lib, orc):
    A = W.poisson7(12)
    b, _ = W.rhs_from_solution(A, 0)
    ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2))
    an = orc.analyse(A, 8, 32, box=(2, 2, 2))
    x0 = np.random.default_rng(4).standard_normal(A.n)
    ref = orc.sor_solve(an, b, x0=x0, omega=1.2, sweeps=4, symmetric=True)
    x = dev(x0)
    rel = H.hbmc_sor(ctx, dev(b), x, 1.2, 4, True)
    np.testing.assert_array_equal(x.cpu().numpy(), ref)
    r = b - orc.spmv(A.row_ptr, A.col, A.val, ref)
    assert abs(rel - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-12 * rel


def test_sor_converges_and_arguments(lib):
    A = W.poisson7(16)
    b, xstar = W.rhs_from_solution(A, 0)
    ctx = H.hbmc_build(A, 8, 32, box=(2, 2, 2))
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    rels = [H.hbmc_sor(ctx, dev(b), x, 1.6, 10, True) for _ in range(5)]
    assert all(rels[k + 1] < rels[k] for k in range(4))
    # zero sweeps leave x unchanged
    before = x.clone()
    H.hbmc_sor(ctx, dev(b), x, 1.0, 0, False)
    assert torch.equal(before, x)
    for omega in (0.0, 2.0, -1.0):
        with pytest.raises(H.HbmcError) as e:
            H.hbmc_sor(ctx, dev(b), x, omega, 1, False)
        assert e.value.status == H.ERR_INVALID_ARG


def test_sor_full_size_poisson128(lib, orc):
    """The 128^3 workload of the benchmark (bs 8, w 32): two symmetric sweeps
    bit-identical to the oracle."""
    P = W.poisson_problem(128, bs=8)
    ctx = H.hbmc_build(P.A, 8, 32, box=P.box)
    an = orc.analyse(P.A, 8, 32, box=P.box)
    ref = orc.sor_solve(an, P.b, omega=1.5, sweeps=2, symmetric=True)
    x = torch.zeros(P.A.n, dtype=torch.float64, device="cuda")
    H.hbmc_sor(ctx, dev(P.b), x, 1.5, 2, True)
    np.testing.assert_array_equal(x.cpu().numpy(), ref)
