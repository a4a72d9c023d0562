"""Property tests over random sparse symmetric patterns (no GPU): the host
build (hbmc_build host_only) equals the oracle's blocking, coloring, HBMC
permutation, Abar and row-split plan bit for bit, and the oracle's ordering
has the structure Sections 4.1-4.2 define (blocks of at most bs unknowns, no
coupled pair of blocks in one color, a bijective permutation, colors padded to
whole level-1 blocks)."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from paper_1908_00741_gb300 import hbmc as H  # noqa: E402
from paper_1908_00741_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    return H.load()


def _random_spd(n, density, seed, hubs):
    """A random symmetric pattern (plus a few dense rows) with a strictly
    dominant diagonal, in CSR with sorted columns."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=seed)
    if hubs:
        rows = rng.choice(n, size=min(n, hubs), replace=False)
        Hm = sp.lil_matrix((n, n))
        for h in rows:
            Hm[h, rng.choice(n, size=max(1, n // 3), replace=False)] = 1.0
        M = M + Hm
    S = (M + M.T).tocsr()
    S.setdiag(0.0)
    S.eliminate_zeros()
    S.data = -np.abs(S.data) - 0.1
    S = (S + sp.identity(n) * (abs(S).sum(axis=1).max() + 1.0)).tocsr()
    S.sort_indices()
    return W.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


systems = st.fixed_dictionaries({
    "n": st.integers(1, 160),
    "density": st.floats(0.0, 0.08),
    "seed": st.integers(0, 2**31 - 1),
    "hubs": st.integers(0, 3),
    "bs": st.sampled_from([1, 2, 3, 4, 8, 16]),
    "w": st.sampled_from([1, 2, 4, 8, 16, 32]),
    "piece": st.sampled_from([1, 4, 16, 64]),
    "cost": st.integers(0, 4),
})


@settings(max_examples=40, deadline=None)
@given(systems)
def test_host_build_equals_oracle(lib, orc, p):
    A = _random_spd(p["n"], p["density"], p["seed"], p["hubs"])
    bs, w = p["bs"], p["w"]
    ctx = H.hbmc_build(A, bs, w, host_only=True, sell_split=p["piece"], sell_split_cost=p["cost"])
    an = orc.analyse(A, bs, w)
    pi, cp, bo, bc = H.hbmc_get_ordering(ctx)
    inf = ctx.info()
    assert (inf["nc"], inf["n_pad"], inf["nblocks"]) == (an.nc, an.n_pad, an.nblocks)
    np.testing.assert_array_equal(bo, an.block_of)
    np.testing.assert_array_equal(bc, an.color)
    np.testing.assert_array_equal(pi, an.pi)
    np.testing.assert_array_equal(cp, an.color_ptr)
    rp, ci, v = H.hbmc_get_matrix(ctx)
    np.testing.assert_array_equal(rp, an.row_ptr)
    np.testing.assert_array_equal(ci, an.col)
    np.testing.assert_array_equal(v, an.val)
    plan = orc.split_plan(an.row_ptr, w, p["piece"], p["cost"] if p["cost"] > 0 else 2)
    np.testing.assert_array_equal(H.hbmc_get_split(ctx), plan.head)
    assert (inf["split_rows"], inf["split_pieces"], inf["sell_entries_split"]) == \
        (plan.nsplit, plan.npieces, plan.processed)
    ctx.close()


@settings(max_examples=40, deadline=None)
@given(systems)
def test_oracle_ordering_structure(orc, p):
    A = _random_spd(p["n"], p["density"], p["seed"], p["hubs"])
    bs, w = p["bs"], p["w"]
    an = orc.analyse(A, bs, w)
    block_of = np.asarray(an.block_of)
    # blocks of at most bs unknowns, every unknown in one block
    assert np.bincount(block_of, minlength=an.nblocks).max() <= bs
    # no two coupled blocks share a color (Section 4.1)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    bi, bj = block_of[rows], block_of[A.col]
    cross = bi != bj
    color = np.asarray(an.color)
    assert not np.any(color[bi[cross]] == color[bj[cross]])
    # pi is injective into [0, n_pad) and keeps each color contiguous
    pi = np.asarray(an.pi)
    assert len(np.unique(pi)) == A.n and (pi >= 0).all() and (pi < an.n_pad).all()
    cp = np.asarray(an.color_ptr)
    assert cp[0] == 0 and cp[-1] == an.n_pad
    assert np.all(np.diff(cp) % (bs * w) == 0)
    pos_color = np.searchsorted(cp, pi, side="right") - 1
    np.testing.assert_array_equal(pos_color, color[block_of])
    # Abar = P A P^T: same values at permuted positions
    rp, ci, v = np.asarray(an.row_ptr), np.asarray(an.col), np.asarray(an.val)
    for i in range(min(A.n, 40)):
        e0, e1 = A.row_ptr[i], A.row_ptr[i + 1]
        k = pi[i]
        got = dict(zip(ci[rp[k]:rp[k + 1]].tolist(), v[rp[k]:rp[k + 1]].tolist()))
        want = dict(zip(pi[A.col[e0:e1]].tolist(), A.val[e0:e1].tolist()))
        assert got == want
