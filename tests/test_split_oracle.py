"""Row-splitting SELL SpMV (Section 5.2.2: SELL pads a slice's rows to its
longest row; the remedy splits the long rows).  Oracle pins -- the plan
against a cost computed from explicitly cut rows and hand-worked cases, the
split product against exact integer arithmetic, exact rationals within the
rounding bound, a case where the cut changes the rounding, and the no-cut
case against the plain product -- plus the split PCG and the structural
stand-in generator."""
import fractions

import numpy as np
import pytest

from paper_1908_00741_gb300 import workloads as W


def _csr_from_lengths(lengths, n_cols, seed, integer=False):
    """Rows of the given lengths with sorted distinct random columns."""
    rng = np.random.default_rng(seed)
    rp = np.zeros(len(lengths) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lengths)
    cols, vals = [], []
    for L in lengths:
        cols.append(np.sort(rng.choice(n_cols, size=L, replace=False)))
        vals.append(rng.integers(-9, 10, size=L).astype(np.float64) if integer else rng.standard_normal(L))
    ci = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    v = np.concatenate(vals) if vals else np.zeros(0)
    return rp, ci, v


def _explicit_plan(lengths, w, P, cost):
    """The plan from rows cut one by one: for every t the head entries are
    counted as w * t, every piece is built as a list of entry positions, and
    the cost adds the pieces' entries and `cost` per piece."""
    heads, pieces = [], []
    for s in range(len(lengths) // w):
        L = lengths[s * w:(s + 1) * w]
        best = None
        for t in range(1, max(L) + 1):
            cut = [list(range(t, l))[k:k + P] for l in L for k in range(0, max(l - t, 0), P)]
            c = w * t + sum(len(x) for x in cut) + cost * len(cut)
            if best is None or c <= best[0]:
                best = (c, t, [len(x) for x in cut])
        heads.append(best[1])
        pieces += best[2]
    pieces.sort(reverse=True)
    processed = w * sum(heads) + sum(w * pieces[k] for k in range(0, len(pieces), w))
    return np.array(heads), processed, len(pieces)


def test_plan_uniform_rows_cut_nothing(orc):
    rp = np.arange(0, 65 * 7, 7, dtype=np.int64)  # 64 rows of 7
    for w in (1, 4, 32):
        plan = orc.split_plan(rp, w, piece=3, cost=1)
        assert (plan.head == 7).all()
        assert plan.nsplit == 0 and plan.npieces == 0
        assert plan.processed == 64 * 7


def test_plan_hand_example(orc):
    # slice 0 = lengths 3, 3, 3, 20 (w = 4, P = 8, cost 2):
    #   t = 3: 12 + 17 + 2 * 3 = 35, every other t costs more (t = 20: 80)
    #   -> head 3, row 3 cut into pieces of 8, 8, 1;
    # slice 1 = 5, 5, 5, 5 -> head 5.  Processed: 4*3 + 4*5 + one slice of
    # pieces (8, 8, 1, pad) of width 8 = 12 + 20 + 32.
    lengths = [3, 3, 3, 20, 5, 5, 5, 5]
    rp = np.zeros(9, dtype=np.int64)
    rp[1:] = np.cumsum(lengths)
    plan = orc.split_plan(rp, 4, piece=8, cost=2)
    assert list(plan.head) == [3, 5]
    assert (plan.nsplit, plan.npieces, plan.processed) == (1, 3, 64)
    # a high piece cost keeps the row whole: t = 20 costs 80 < 12 + 17 + 100 * 3
    plan = orc.split_plan(rp, 4, piece=8, cost=100)
    assert list(plan.head) == [20, 5] and plan.nsplit == 0 and plan.processed == 80 + 20


@pytest.mark.parametrize("w,P,cost,seed", [(4, 3, 1, 0), (8, 5, 2, 1), (32, 16, 2, 2), (2, 1, 0, 3),
                                           (16, 64, 4, 4)])
def test_plan_against_explicit_cuts(orc, w, P, cost, seed):
    rng = np.random.default_rng(seed)
    n = 8 * w
    lengths = rng.integers(1, 12, size=n)
    lengths[rng.choice(n, size=max(1, n // 10), replace=False)] += rng.integers(10, 60)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lengths)
    plan = orc.split_plan(rp, w, piece=P, cost=cost)
    head, processed, npieces = _explicit_plan(list(lengths), w, P, cost)
    np.testing.assert_array_equal(plan.head, head)
    assert plan.processed == processed and plan.npieces == npieces
    # every entry is processed once as head or piece entry
    t = np.repeat(plan.head, w)
    assert int(np.minimum(lengths, t).sum() + np.maximum(lengths - t, 0).sum()) == int(lengths.sum())
    assert plan.nsplit == int((lengths > t).sum())


@pytest.mark.parametrize("w,P,cost", [(4, 2, 1), (8, 3, 0), (32, 8, 2)])
def test_spmv_split_integer_values_exact(orc, w, P, cost):
    rng = np.random.default_rng(7)
    n = 4 * w
    lengths = rng.integers(1, 9, size=n)
    lengths[::5] += 20
    rp, ci, v = _csr_from_lengths(lengths, 64, 8, integer=True)
    p = rng.integers(-9, 10, size=64).astype(np.float64)
    plan = orc.split_plan(rp, w, piece=P, cost=cost)
    assert plan.nsplit > 0
    dense = np.zeros((n, 64), dtype=np.int64)
    for i in range(n):
        dense[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]].astype(np.int64)
    q = orc.spmv_split(rp, ci, v, plan, p)
    np.testing.assert_array_equal(q, (dense @ p.astype(np.int64)).astype(np.float64))


def test_spmv_split_without_cuts_is_the_plain_product(orc):
    rng = np.random.default_rng(9)
    rp, ci, v = _csr_from_lengths([6] * 64, 100, 10)
    p = rng.standard_normal(100)
    plan = orc.split_plan(rp, 8, piece=2, cost=1)
    assert plan.nsplit == 0
    np.testing.assert_array_equal(orc.spmv_split(rp, ci, v, plan, p), orc.spmv(rp, ci, v, p))


def test_spmv_split_cut_changes_rounding(orc):
    # w = 4, lengths 2, 2, 2, 4 with P = 2, cost 2: t = 2 costs 8 + 2 + 2 = 12,
    # t = 3 costs 15, t = 4 costs 16, t = 1 costs 20 -> row 3 is cut after 2.
    # Row 3 = (1e16, 1, -1e16, 1) against p = 1: the head is fl(1e16 + 1) =
    # 1e16 (a tie, to even), the piece fl(-1e16 + 1) = -1e16, so q_3 = 0;
    # the unsplit sum is 1e16, 1e16, 0, 1 -> 1.
    rp = np.array([0, 2, 4, 6, 10], dtype=np.int64)
    ci = np.array([0, 1, 0, 1, 0, 1, 0, 1, 2, 3], dtype=np.int32)
    v = np.array([1, 1, 1, 1, 1, 1, 1e16, 1, -1e16, 1], dtype=np.float64)
    p = np.ones(4)
    plan = orc.split_plan(rp, 4, piece=2, cost=2)
    assert list(plan.head) == [2]
    assert orc.spmv_split(rp, ci, v, plan, p)[3] == 0.0
    assert orc.spmv(rp, ci, v, p)[3] == 1.0


def test_spmv_split_within_rounding_bound(orc):
    rng = np.random.default_rng(11)
    lengths = rng.integers(1, 10, size=32)
    lengths[[3, 17, 30]] = [40, 33, 25]
    rp, ci, v = _csr_from_lengths(lengths, 80, 12)
    p = rng.standard_normal(80)
    plan = orc.split_plan(rp, 8, piece=6, cost=1)
    assert plan.nsplit >= 3
    q = orc.spmv_split(rp, ci, v, plan, p)
    u = 2.0 ** -53
    for i in range(32):
        e = slice(rp[i], rp[i + 1])
        exact = sum(fractions.Fraction(a) * fractions.Fraction(b) for a, b in zip(v[e], p[ci[e]]))
        k = int(lengths[i]) + int(np.ceil(max(lengths[i] - plan.head[i // 8], 0) / 6))
        gamma = k * u / (1 - k * u)
        bound = gamma * float(np.sum(np.abs(v[e] * p[ci[e]])))
        assert abs(fractions.Fraction(q[i]) - exact) <= fractions.Fraction(bound)


def test_pcg_split_solves_and_reduces_without_cuts(orc):
    A = W.irregular_structural(6, 5)
    b, _ = W.rhs_from_solution(A, 0)
    plain, an = orc.iccg(A, b, 8, 32)
    split, _ = orc.iccg(A, b, 8, 32, split=(16, 2), an=an)
    plan = orc.split_plan(an.row_ptr, 32, 16, 2)
    assert plan.nsplit > 0
    assert split.status == 0 and abs(split.iters - plain.iters) <= 2
    r = b - A.matvec(split.x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-7
    # uniform rows: no cut, so the split solve is the plain solve bit for bit
    P = W.poisson7(6)
    bp, _ = W.rhs_from_solution(P, 1)
    s0, anp = orc.iccg(P, bp, 8, 32, box=(2, 2, 2))
    if orc.split_plan(anp.row_ptr, 32, 64, 1000).nsplit == 0:
        s1, _ = orc.iccg(P, bp, 8, 32, an=anp, split=(64, 1000))
        assert s1.iters == s0.iters
        np.testing.assert_array_equal(s1.x, s0.x)


def test_structural_generator_shape():
    A = W.irregular_structural(6, 3)
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0.0
    assert np.linalg.eigvalsh(S.toarray())[0] > 0.0
    A = W.irregular_structural(16, 7)
    L = np.diff(A.row_ptr)
    assert A.n == 3 * 16 ** 3
    assert 60 < L.mean() < 85 and 0.2 < L.std() / L.mean() < 0.4
    assert L.max() > 2 * L.mean()


def test_structural_sell_padding_like_audikw(orc):
    """The paper reports 28% (slice 4) and 40% (slice 8) more processed
    elements in SELL than in CRS on Audikw_1; the stand-in lands near both."""
    A = W.irregular_structural(20, 7)
    out = {}
    for w in (4, 8):
        an = orc.analyse(A, 8, w)
        ln = np.diff(np.asarray(an.row_ptr))
        out[w] = (ln.reshape(-1, w).max(1) * w).sum() / ln.sum() - 1.0
    assert 0.15 < out[4] < 0.40 and 0.25 < out[8] < 0.55 and out[8] > out[4]


@pytest.mark.parametrize("seed", range(12))
def test_plan_random_length_mixes(orc, seed):
    """Many random row-length mixes (uniform, heavy-tailed, a few very long
    rows, empty-ish slices of length-1 rows) against the explicitly cut plan."""
    rng = np.random.default_rng(100 + seed)
    w = int(rng.choice([1, 2, 4, 8, 16, 32]))
    ns = int(rng.integers(1, 6))
    kind = seed % 4
    n = ns * w
    if kind == 0:
        lengths = rng.integers(1, 20, size=n)
    elif kind == 1:
        lengths = np.minimum(1 + rng.pareto(1.5, size=n) * 5, 300).astype(np.int64)
    elif kind == 2:
        lengths = np.full(n, 5)
        lengths[rng.choice(n, size=max(1, n // 16), replace=False)] = rng.integers(50, 200)
    else:
        lengths = np.ones(n, dtype=np.int64)
        lengths[::3] = rng.integers(1, 40, size=len(lengths[::3]))
    P = int(rng.choice([1, 3, 8, 64]))
    cost = int(rng.integers(0, 5))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lengths)
    plan = orc.split_plan(rp, w, piece=P, cost=cost)
    head, processed, npieces = _explicit_plan(list(lengths), w, P, cost)
    np.testing.assert_array_equal(plan.head, head)
    assert (plan.processed, plan.npieces) == (processed, npieces)
