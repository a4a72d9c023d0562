"""The host build's row-split SpMV plan (hbmc_build host_only with
sell_split; Section 5.2.2's remedy) against the oracle's plan: head widths,
split rows, pieces and processed entries equal; argument checks."""
import numpy as np
import pytest

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


HOST_CASES = [
    ("structural_8_bs8_w32_P64", lambda: W.irregular_structural(8, 7), 8, 32, None, 64, 0),
    ("structural_7_bs4_w16_P16_c1", lambda: W.irregular_structural(7, 2), 4, 16, None, 16, 1),
    ("hetero27_9_rand_w8_P4_c3", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                         W.random_order(2, 729)), 8, 8, None, 4, 3),
    ("poisson7_9_box_w32_P2", lambda: W.poisson7(9), 8, 32, (2, 2, 2), 2, 1),
    ("veclap_5_rand_w1_P8", lambda: W.permute_input(W.vector_laplacian(5, 3), W.random_order(4, 375)),
     8, 1, None, 8, 2),
]


@pytest.mark.parametrize("name,mk,bs,w,box,P,cost", HOST_CASES)
def test_host_split_plan_matches_oracle(lib, orc, name, mk, bs, w, box, P, cost):
    A = mk()
    ctx = H.hbmc_build(A, bs, w, box=box, host_only=True, sell_split=P, sell_split_cost=cost)
    an = orc.analyse(A, bs, w, box=box)
    plan = orc.split_plan(an.row_ptr, w, P, cost if cost > 0 else 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    inf = ctx.info()
    assert (inf["split_rows"], inf["split_pieces"], inf["sell_entries_split"]) == \
        (plan.nsplit, plan.npieces, plan.processed)


def test_host_split_argument_checks(lib):
    A = W.poisson7(4)
    with pytest.raises(H.HbmcError):
        H.hbmc_build(A, 8, 32, host_only=True, sell_split=-1)
    with pytest.raises(H.HbmcError):
        H.hbmc_build(A, 8, 32, host_only=True, sell_split=4, sell_split_cost=-2)
    ctx = H.hbmc_build(A, 8, 32, host_only=True)
    assert ctx.info()["sell_entries_split"] == 0
    with pytest.raises(H.HbmcError, match="without row splitting"):
        H.hbmc_get_split(ctx)


def test_host_split_empty_and_single_row(lib, orc):
    """An empty system gets an empty plan; a one-unknown system one slice
    (the unknown and its dummies) with no cut."""
    E = W.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    ctx = H.hbmc_build(E, 8, 32, host_only=True, sell_split=8)
    inf = ctx.info()
    assert (inf["n_pad"], inf["split_rows"], inf["split_pieces"], inf["sell_entries_split"]) == (0, 0, 0, 0)
    assert H.hbmc_get_split(ctx).size == 0
    one = W.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.0]))
    ctx = H.hbmc_build(one, 8, 32, host_only=True, sell_split=8)
    an = orc.analyse(one, 8, 32)
    plan = orc.split_plan(an.row_ptr, 32, 8, 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    assert ctx.info()["split_rows"] == 0 and (plan.head == 1).all()


@pytest.mark.parametrize("seed", range(6))
def test_host_split_plan_random_matrices(lib, orc, seed):
    """Random symmetric patterns with a few dense rows and columns (hubs), random
    w, piece length and cost: the host plan equals the oracle's."""
    import scipy.sparse as sp
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(50, 400))
    M = sp.random(n, n, density=float(rng.uniform(0.005, 0.05)), random_state=int(rng.integers(1 << 30)))
    hubs = rng.choice(n, size=max(1, n // 50), replace=False)
    H_ = sp.lil_matrix((n, n))
    for h in hubs:
        cols = rng.choice(n, size=min(n, int(rng.integers(n // 4, n))), replace=False)
        H_[h, cols] = 1.0
    S = (M + M.T + H_ + H_.T).tocsr()
    S.setdiag(0.0)
    S.eliminate_zeros()
    S = S + sp.identity(n) * (abs(S).sum(axis=1).max() + 1.0)
    S = S.tocsr()
    S.sort_indices()
    A = W.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))
    bs = int(rng.choice([1, 2, 4, 8]))
    w = int(rng.choice([4, 8, 16, 32]))
    P = int(rng.choice([2, 8, 32]))
    cost = int(rng.integers(0, 4))
    ctx = H.hbmc_build(A, bs, w, host_only=True, sell_split=P, sell_split_cost=cost)
    an = orc.analyse(A, bs, w)
    plan = orc.split_plan(an.row_ptr, w, P, cost if cost > 0 else 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    inf = ctx.info()
    assert (inf["split_rows"], inf["split_pieces"], inf["sell_entries_split"]) == \
        (plan.nsplit, plan.npieces, plan.processed)

