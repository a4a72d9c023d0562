"""Pins for the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form,
a textbook routine (dense Cholesky, dense triangular solve, dense solve), an
invariant stated in the paper (ER condition, Eqs. "HBMC1", "reorder1",
"BAMC1", "BAMC-level-2", the 2*bs-1 diagonals of Section 4.3.3) or a
hand-worked fixture under tests/golden/.
"""
import fractions
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_1908_00741_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = np.array([int(v) for v in vals], dtype=np.int64)
    return out


def _csr_from_dense(M):
    S = sp.csr_matrix(M)
    S.sort_indices()
    return W.CSR(M.shape[0], S.indptr.astype(np.int64), S.indices.astype(np.int32),
                 S.data.astype(np.float64))


def _chain(n, diag=2.0, off=-1.0):
    M = np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, off), 1) + np.diag(np.full(n - 1, off), -1)
    return _csr_from_dense(M)


def _grid2d(m):
    """2D 5-point Laplacian on an m x m grid, i = x + m*y."""
    T = np.diag(np.full(m, 2.0)) - np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1)
    M = np.kron(np.eye(m), T) + np.kron(T, np.eye(m))
    return _csr_from_dense(M)


def _dense(rp, ci, v, n):
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def _lower_dense(an, lval, ldiag):
    n = an.n_pad
    rows = np.repeat(np.arange(n), np.diff(an.row_ptr))
    low = an.col < rows
    L = np.zeros((n, n))
    L[rows[low], an.col[low]] = lval[low]
    L[np.arange(n), np.arange(n)] = ldiag
    return L


# --------------------------------------------------------------------------
# Blocking and coloring
# --------------------------------------------------------------------------

def test_hand_worked_algebraic_blocking(orc):
    g = _read_golden("grid3x3_bs4_blocks.txt")
    A = _grid2d(3)
    block_of, nb = orc.blocks_greedy(A.row_ptr, A.col, 4)
    assert nb == 3
    np.testing.assert_array_equal(block_of, g["block_of"])
    color, nc = orc.color_blocks(A.row_ptr, A.col, block_of, nb)
    np.testing.assert_array_equal(color, g["color"])
    assert nc == 2


def test_hand_worked_chain_blocking(orc):
    g = _read_golden("chain16_bs2_w2.txt")
    A = _chain(16)
    block_of, nb = orc.blocks_greedy(A.row_ptr, A.col, 2)
    np.testing.assert_array_equal(block_of, g["block_of"])
    color, nc = orc.color_blocks(A.row_ptr, A.col, block_of, nb)
    np.testing.assert_array_equal(color, g["color"])


@pytest.mark.parametrize("grid,box", [((4, 4, 4), (2, 2, 2)), ((5, 3, 7), (2, 2, 2)),
                                      ((6, 8, 8), (2, 4, 4)), ((8, 8, 8), (2, 2, 4))])
def test_geometric_boxes_are_boxes(orc, grid, box):
    nx, ny, nz = grid
    block_of, nb = orc.blocks_boxes(grid, box)
    i = np.arange(nx * ny * nz)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    mx, my, mz = [math.ceil(g / b) for g, b in zip(grid, box)]
    assert nb == mx * my * mz
    seen_corners = []
    for b in range(nb):
        m = block_of == b
        assert m.any()
        # the members of one block fill one axis-aligned box of the box grid
        cx, cy, cz = x[m].min(), y[m].min(), z[m].min()
        assert cx % box[0] == 0 and cy % box[1] == 0 and cz % box[2] == 0
        ex = min(box[0], nx - cx); ey = min(box[1], ny - cy); ez = min(box[2], nz - cz)
        assert m.sum() == ex * ey * ez
        assert x[m].max() - cx == ex - 1 and y[m].max() - cy == ey - 1 and z[m].max() - cz == ez - 1
        seen_corners.append((cz, cy, cx))
    # ids run lexicographically over boxes (x fastest, z slowest)
    assert seen_corners == sorted(seen_corners)


def _block_graph_edges(A, block_of):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    bi, bj = block_of[rows], block_of[A.col]
    keep = bi != bj
    return set(zip(bi[keep].tolist(), bj[keep].tolist()))


@pytest.mark.parametrize("m,box", [(8, (2, 2, 2)), (10, (2, 2, 2)), (8, (2, 2, 4)), (8, (2, 4, 4))])
def test_7pt_boxes_give_two_colors_by_parity(orc, m, box):
    """A 7-point stencil with box blocking has a bipartite box graph; first-fit
    in lexicographic box order gives exactly 2 colors, color = parity of the
    box coordinates' sum (closed form)."""
    A = W.poisson7(m)
    block_of, nb = orc.blocks_boxes(A.grid, box)
    color, nc = orc.color_blocks(A.row_ptr, A.col, block_of, nb)
    assert nc == 2
    mx, my = math.ceil(m / box[0]), math.ceil(m / box[1])
    b = np.arange(nb)
    bx, by, bz = b % mx, (b // mx) % my, b // (mx * my)
    np.testing.assert_array_equal(color, (bx + by + bz) % 2)


def test_27pt_boxes_give_eight_colors(orc):
    """27-point coupling joins every box to all 26 neighbouring boxes; the
    first-fit coloring is the 2x2x2 parity class (closed form)."""
    A = W.heterogeneous_stencil(8, 27, 1.0, 7)
    block_of, nb = orc.blocks_boxes(A.grid, (2, 2, 2))
    color, nc = orc.color_blocks(A.row_ptr, A.col, block_of, nb)
    assert nc == 8
    b = np.arange(nb)
    bx, by, bz = b % 4, (b // 4) % 4, b // 16
    np.testing.assert_array_equal(color, (bx % 2) + 2 * (by % 2) + 4 * (bz % 2))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_greedy_blocks_and_colors_are_valid(orc, seed):
    """Random input order (algebraic blocking): blocks partition the unknowns,
    hold at most bs members, are seeded by the minimal unassigned unknown,
    short blocks have no unassigned neighbour left, and no edge joins two
    blocks of one color."""
    A = W.permute_input(W.heterogeneous_stencil(6, 7, 1.0, seed), W.random_order(seed + 10, 216))
    bs = 8
    block_of, nb = orc.blocks_greedy(A.row_ptr, A.col, bs)
    assert block_of.min() == 0 and block_of.max() == nb - 1
    sizes = np.bincount(block_of, minlength=nb)
    assert sizes.max() <= bs and sizes.min() >= 1
    assigned_before = np.zeros(A.n, dtype=bool)
    for b in range(nb):
        members = np.flatnonzero(block_of == b)
        assert members.min() == np.flatnonzero(~assigned_before).min()  # seed rule
        if len(members) < bs:  # closed short: every neighbour belongs to an earlier or this block
            for i in members:
                nbrs = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
                assert np.all(block_of[nbrs] <= b)
        assigned_before[members] = True
    color, nc = orc.color_blocks(A.row_ptr, A.col, block_of, nb)
    for bi, bj in _block_graph_edges(A, block_of):
        assert color[bi] != color[bj]
    # first fit: every color below a block's own is taken by an earlier adjacent block
    adj = {}
    for bi, bj in _block_graph_edges(A, block_of):
        adj.setdefault(bi, set()).add(bj)
    for b in range(nb):
        below = {color[o] for o in adj.get(b, ()) if o < b}
        assert all(c in below for c in range(color[b]))


# --------------------------------------------------------------------------
# Orderings (Section 4.2)
# --------------------------------------------------------------------------

def test_hand_worked_bmc_hbmc_permutations(orc):
    g = _read_golden("chain16_bs2_w2.txt")
    A = _chain(16)
    for hbmc, key in ((False, "bmc_sequence"), (True, "hbmc_sequence")):
        an = orc.analyse(A, 2, 2, hbmc=hbmc)
        assert an.n_pad == 16
        np.testing.assert_array_equal(an.color_ptr, g["color_ptr"])
        seq = np.empty(16, dtype=np.int64)
        seq[an.pi] = np.arange(16)
        np.testing.assert_array_equal(seq, g[key])


def _orderings(A, bs, w, box):
    import oracle
    an_h = oracle.analyse(A, bs, w, box=box, hbmc=True)
    an_b = oracle.analyse(A, bs, w, box=box, hbmc=False)
    return an_h, an_b


CASES = [
    ("poisson7_8", lambda: W.poisson7(8), 8, 4, (2, 2, 2)),
    ("poisson7_7", lambda: W.poisson7(7), 8, 4, (2, 2, 2)),
    ("poisson7_8_bs16", lambda: W.poisson7(8), 16, 2, (2, 2, 4)),
    ("hetero27_6_rand", lambda: W.permute_input(W.heterogeneous_stencil(6, 27, 2.0, 1),
                                                W.random_order(2, 216)), 8, 4, None),
    ("veclap_4_rand", lambda: W.permute_input(W.vector_laplacian(4, 3), W.random_order(4, 192)),
     4, 8, None),
]


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
def test_permutation_structure(orc, name, mk, bs, w, box):
    A = mk()
    an_h, an_b = _orderings(A, bs, w, box)
    for an in (an_h, an_b):
        # injective into the padded space; every color segment is a multiple of bs*w
        assert len(np.unique(an.pi)) == A.n and an.pi.min() >= 0 and an.pi.max() < an.n_pad
        assert np.all(np.diff(an.color_ptr) % (bs * w) == 0)
    # ER condition (Eq. "equivalence") between BMC and HBMC on every coupled pair
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    cols = A.col.astype(np.int64)
    s_b = np.sign(an_b.pi[rows] - an_b.pi[cols])
    s_h = np.sign(an_h.pi[rows] - an_h.pi[cols])
    np.testing.assert_array_equal(s_b, s_h)
    # Eq. "HBMC1": order across different level-1 blocks is kept;
    # Eq. "reorder1": order inside one BMC block is kept.
    lev1 = an_b.pi // (bs * w)  # level-1 block of each unknown (same in both orders)
    np.testing.assert_array_equal(lev1, an_h.pi // (bs * w))
    o = np.argsort(an_b.pi)
    rng = np.random.default_rng(0)
    i1, i2 = rng.integers(0, A.n, 4000), rng.integers(0, A.n, 4000)
    diff_l1 = lev1[i1] != lev1[i2]
    np.testing.assert_array_equal(np.sign(an_b.pi[i1] - an_b.pi[i2])[diff_l1],
                                  np.sign(an_h.pi[i1] - an_h.pi[i2])[diff_l1])
    same_blk = an_b.pi[i1] // bs == an_b.pi[i2] // bs
    np.testing.assert_array_equal(np.sign(an_b.pi[i1] - an_b.pi[i2])[same_blk],
                                  np.sign(an_h.pi[i1] - an_h.pi[i2])[same_blk])
    del o


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
def test_hbmc_block_structure(orc, name, mk, bs, w, box):
    """Eq. "BAMC1": each diagonal color block C_cc is block diagonal in level-1
    blocks; Eq. "BAMC-level-2": inside a level-1 block the w x w blocks D_l on
    the diagonal are diagonal; Section 4.3.3: all nonzeros of a level-1 block
    lie on 2*bs-1 diagonals (offsets m*w, |m| < bs)."""
    A = mk()
    an, _ = _orderings(A, bs, w, box)
    rows = np.repeat(np.arange(an.n_pad), np.diff(an.row_ptr))
    cols = an.col.astype(np.int64)
    c_of = np.searchsorted(an.color_ptr, np.arange(an.n_pad), side="right") - 1
    same_color = c_of[rows] == c_of[cols]
    l1 = rows // (bs * w) == cols // (bs * w)
    assert np.all(l1[same_color]), "coupling between two level-1 blocks of one color"
    inside = l1 & (rows != cols)
    step_r, step_c = (rows % (bs * w)) // w, (cols % (bs * w)) // w
    assert np.all(step_r[inside] != step_c[inside]), "D_l is not diagonal"
    offs = np.unique(rows[l1] - cols[l1])
    assert np.all(offs % w == 0) and np.all(np.abs(offs) < bs * w)
    assert len(offs) <= 2 * bs - 1


# --------------------------------------------------------------------------
# IC(0)
# --------------------------------------------------------------------------

def _random_spd_dense(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return G @ G.T + n * np.eye(n)


@pytest.mark.parametrize("n,bs,w", [(12, 2, 2), (30, 3, 4), (64, 8, 4)])
def test_ic0_full_pattern_is_cholesky(orc, n, bs, w):
    """With a full pattern nothing is dropped, so IC(0) of Abar must equal the
    textbook dense Cholesky factor of Abar."""
    A = _csr_from_dense(_random_spd_dense(n, n))
    an = orc.analyse(A, bs, w)
    lval, ldiag, dinv, bad = orc.factor(an)
    assert bad == -1
    Ad = _dense(an.row_ptr, an.col, an.val, an.n_pad)
    Lref = np.linalg.cholesky(Ad)
    L = _lower_dense(an, lval, ldiag)
    np.testing.assert_allclose(L, Lref, rtol=0, atol=1e-13 * np.abs(Lref).max())
    np.testing.assert_allclose(dinv, 1.0 / np.diag(Lref), rtol=1e-14)


@pytest.mark.parametrize("n", [5, 17, 64])
def test_tridiagonal_single_block_is_exact_and_pcg_one_step(orc, n):
    """A tridiagonal matrix in natural order has no fill, so with one block
    holding every unknown IC(0) is the exact Cholesky factor and PCG
    converges in one iteration."""
    A = _chain(n, 2.5, -1.0)
    an = orc.analyse(A, n, 1)
    lval, ldiag, dinv, bad = orc.factor(an)
    L = _lower_dense(an, lval, ldiag)
    Ad = _dense(an.row_ptr, an.col, an.val, an.n_pad)
    np.testing.assert_allclose(L, np.linalg.cholesky(Ad), atol=1e-14)
    b = np.sin(np.arange(n) + 1.0)
    s = orc.pcg(an, lval, dinv, b, tol=1e-12, maxit=10)
    assert s.status == 0 and s.iters == 1
    np.testing.assert_allclose(s.x, np.linalg.solve(A.to_scipy().toarray(), b), rtol=1e-12)


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
@pytest.mark.parametrize("shift", [0.0, 0.3])
def test_ic0_matches_A_on_pattern(orc, name, mk, bs, w, box, shift):
    """IC(0) property: (L L^T)_ij equals the shifted Abar on Abar's pattern."""
    A = mk()
    an, _ = _orderings(A, bs, w, box)
    lval, ldiag, dinv, bad = orc.factor(an, shift)
    assert bad == -1
    n = an.n_pad
    rows = np.repeat(np.arange(n), np.diff(an.row_ptr))
    low = an.col < rows
    L = sp.csr_matrix((np.concatenate([lval[low], ldiag]),
                       (np.concatenate([rows[low], np.arange(n)]),
                        np.concatenate([an.col[low], np.arange(n)]))), shape=(n, n))
    LLt = (L @ L.T).tocsr()
    target = an.val.copy()
    target[rows == an.col] *= (1.0 + shift)
    got = np.asarray(LLt[rows, an.col]).ravel()
    np.testing.assert_allclose(got, target, rtol=1e-13, atol=1e-13 * np.abs(target).max())
    # outside the pattern L L^T may differ (dropped fill), which is what makes it incomplete
    np.testing.assert_allclose(dinv * ldiag, 1.0, rtol=1e-15)


def test_ic0_reports_first_bad_pivot(orc):
    """[[1,2],[2,1]] is indefinite: l_11 = 1, l_21 = 2, pivot 1 - 4 < 0 at row 1."""
    A = _csr_from_dense(np.array([[1.0, 2.0], [2.0, 1.0]]))
    an = orc.analyse(A, 2, 1)
    _, _, _, bad = orc.factor(an)
    assert bad == 1
    # a large enough diagonal shift makes it positive: (1+a)^2 > 4  <=>  a > 1
    _, _, _, bad = orc.factor(an, 1.5)
    assert bad == -1


# --------------------------------------------------------------------------
# Substitutions, SpMV, dots
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk,bs,w,box", CASES[:4])
def test_substitutions_match_dense_triangular_solves(orc, name, mk, bs, w, box):
    A = mk()
    an, _ = _orderings(A, bs, w, box)
    lval, ldiag, dinv, bad = orc.factor(an, 0.1)
    if an.n_pad > 800:
        pytest.skip("dense check only for small n")
    L = _lower_dense(an, lval, ldiag)
    r = np.cos(np.arange(an.n_pad) * 0.37)
    y = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z = orc.bwd(an.row_ptr, an.col, lval, dinv, y)
    np.testing.assert_allclose(y, sla.solve_triangular(L, r, lower=True), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(z, sla.solve_triangular(L.T, y, lower=False), rtol=1e-13, atol=1e-14)


def test_spmv_matches_scipy(orc):
    A = W.heterogeneous_stencil(9, 27, 2.0, 3)
    p = np.sin(np.arange(A.n) * 0.1)
    np.testing.assert_allclose(orc.spmv(A.row_ptr, A.col, A.val, p), A.to_scipy() @ p, rtol=1e-14,
                               atol=1e-14 * np.abs(A.val).max())


def test_exact_dot_is_correctly_rounded(orc):
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = 1000
        a = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
        b = rng.standard_normal(n)
        if trial % 2:  # heavy cancellation
            b[n // 2:] = -b[: n // 2] * a[: n // 2] / a[n // 2:] * (1 + 1e-15 * rng.standard_normal(n // 2))
        exact = sum((fractions.Fraction(x) * fractions.Fraction(y) for x, y in zip(a, b)),
                    fractions.Fraction(0))
        assert orc.dot(a, b, mode=orc.DOT_EXACT) == float(exact)
    # order independence
    perm = rng.permutation(1000)
    assert orc.dot(a, b, mode=orc.DOT_EXACT) == orc.dot(a[perm], b[perm], mode=orc.DOT_EXACT)


def test_sequential_dot_error_bound(orc):
    rng = np.random.default_rng(6)
    a, b = rng.standard_normal(5000), rng.standard_normal(5000)
    exact = float(sum((fractions.Fraction(x) * fractions.Fraction(y) for x, y in zip(a, b)),
                      fractions.Fraction(0)))
    bound = 5000 * 2.0 ** -53 * float(np.abs(a) @ np.abs(b))
    assert abs(orc.dot(a, b, mode=orc.DOT_SEQUENTIAL) - exact) <= bound


# --------------------------------------------------------------------------
# PCG and the equivalence claim (Section 4.2.1, Table "number-ite")
# --------------------------------------------------------------------------

def test_pcg_small_spd_matches_dense_solve(orc):
    A = _grid2d(9)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(A.n)
    s, an = orc.iccg(A, b, 4, 4, tol=1e-13, maxit=500)
    assert s.status == 0
    xd = np.linalg.solve(A.to_scipy().toarray(), b)
    np.testing.assert_allclose(s.x, xd, rtol=1e-10, atol=1e-11 * np.abs(xd).max())
    true = np.linalg.norm(b - A.to_scipy() @ s.x) / np.linalg.norm(b)
    assert true < 1e-12


def test_pcg_zero_rhs_and_maxit(orc):
    A = W.poisson7(6)
    s, an = orc.iccg(A, np.zeros(A.n), 8, 4, box=(2, 2, 2))
    assert s.status == 0 and s.iters == 0 and np.all(s.x == 0)
    b, _ = W.rhs_from_solution(A, 0)
    s, _ = orc.iccg(A, b, 8, 4, box=(2, 2, 2), maxit=2, an=an)
    assert s.status == 1 and s.iters == 2


@pytest.mark.parametrize("name,mk,bs,w,box", CASES)
def test_bmc_and_hbmc_converge_identically(orc, name, mk, bs, w, box):
    """Paper's central claim (Section 4.2.1, Table "number-ite"): HBMC and BMC
    with the same blocks and colors give the same ICCG convergence.  Rounding
    differs only through the order of terms inside a row, so the iteration
    counts are equal and the iterates agree to rounding level."""
    A = mk()
    b, _ = W.rhs_from_solution(A, 0)
    sh, _ = orc.iccg(A, b, bs, w, box=box, hbmc=True, tol=1e-10)
    sb, _ = orc.iccg(A, b, bs, w, box=box, hbmc=False, tol=1e-10)
    assert sh.status == 0 and sb.status == 0
    assert sh.iters == sb.iters
    np.testing.assert_allclose(sh.hist, sb.hist, rtol=1e-9)
    np.testing.assert_allclose(sh.x, sb.x, rtol=0, atol=1e-12 * np.abs(sb.x).max())


def test_equivalence_independent_of_w(orc):
    """The secondary reordering is equivalent for every w at fixed BMC blocks
    and colors, so the convergence does not depend on w."""
    A = W.poisson7(8)
    b, _ = W.rhs_from_solution(A, 0)
    runs = [orc.iccg(A, b, 8, w, box=(2, 2, 2), tol=1e-10)[0] for w in (1, 2, 4, 8, 32)]
    for s in runs[1:]:
        assert s.iters == runs[0].iters
        np.testing.assert_allclose(s.x, runs[0].x, rtol=0, atol=1e-12 * np.abs(runs[0].x).max())


def test_orderings_with_other_blockings_converge_differently(orc):
    """Sanity check that the equivalence tests can fail: a different blocking is
    a genuinely different preconditioner (not equivalent), so its iteration
    history differs."""
    A = W.poisson7(8)
    b, _ = W.rhs_from_solution(A, 0)
    s1, _ = orc.iccg(A, b, 8, 4, box=(2, 2, 2), tol=1e-10)
    s2, _ = orc.iccg(A, b, 8, 4, box=None, tol=1e-10)
    assert not np.allclose(s1.hist[:5], s2.hist[:5], rtol=1e-9)


def test_dot_order_does_not_change_the_solve(orc):
    """Exactly rounded and sequential dot products give the same iteration count
    and iterates within 1e-13: the solve is not sensitive to the dot's
    summation order at these sizes."""
    A = W.poisson7(12)
    b, _ = W.rhs_from_solution(A, 0)
    s0, an = orc.iccg(A, b, 8, 32, box=(2, 2, 2), dot_mode=orc.DOT_SEQUENTIAL)
    s1, _ = orc.iccg(A, b, 8, 32, box=(2, 2, 2), dot_mode=orc.DOT_EXACT, an=an)
    assert s0.iters == s1.iters
    np.testing.assert_allclose(s1.x, s0.x, rtol=0, atol=1e-13 * np.abs(s0.x).max())
