"""Property tests of the oracle's numerics over random inputs (hypothesis, no
GPU): IC(0) reproduces A on its pattern (Section 2, Eq. "ILU") for random
M-matrices; the substitutions equal dense triangular solves; SpMV and the
row-split SpMV equal exact integer products; the sequential dot stays within
its rounding bound of the exactly rounded one."""
import fractions

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402
import scipy.linalg as sla  # noqa: E402
import scipy.sparse as sp  # noqa: E402

from paper_1908_00741_gb300 import workloads as W  # noqa: E402


def _m_matrix(n, density, seed, integer=False):
    """Symmetric, negative off-diagonals, strictly dominant positive diagonal:
    an M-matrix, for which IC(0) exists without a shift."""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=seed)
    S = (M + M.T).tocsr()
    S.setdiag(0.0)
    S.eliminate_zeros()
    if integer:
        S.data = -rng.integers(1, 5, size=S.data.size).astype(np.float64)
        S = ((S + S.T) * 0.5).tocsr()
        S.data = np.round(S.data)
    else:
        S.data = -np.abs(S.data) - 0.05
    d = np.asarray(abs(S).sum(axis=1)).ravel() + (1.0 if integer else 0.5)
    S = (S + sp.diags(d)).tocsr()
    S.eliminate_zeros()
    S.sort_indices()
    return W.CSR(n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


cases = st.fixed_dictionaries({
    "n": st.integers(2, 90),
    "density": st.floats(0.01, 0.2),
    "seed": st.integers(0, 2**31 - 1),
    "bs": st.sampled_from([1, 2, 4, 8]),
    "w": st.sampled_from([1, 2, 4, 8, 32]),
})


@settings(max_examples=30, deadline=None)
@given(cases, st.sampled_from([0.0, 0.2]))
def test_ic0_reproduces_a_on_pattern(orc, p, shift):
    A = _m_matrix(p["n"], p["density"], p["seed"])
    an = orc.analyse(A, p["bs"], p["w"])
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
    np.testing.assert_allclose(got, target, rtol=1e-12, atol=1e-12 * np.abs(target).max())


@settings(max_examples=30, deadline=None)
@given(cases)
def test_substitutions_are_triangular_solves(orc, p):
    A = _m_matrix(p["n"], p["density"], p["seed"])
    an = orc.analyse(A, p["bs"], p["w"])
    lval, ldiag, dinv, bad = orc.factor(an, 0.0)
    assert bad == -1
    n = an.n_pad
    Ld = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(an.row_ptr))
    low = an.col < rows
    Ld[rows[low], an.col[low]] = lval[low]
    Ld[np.arange(n), np.arange(n)] = ldiag
    r = np.random.default_rng(p["seed"] % 1000).standard_normal(n)
    y = orc.fwd(an.row_ptr, an.col, lval, dinv, r)
    z = orc.bwd(an.row_ptr, an.col, lval, dinv, y)
    np.testing.assert_allclose(y, sla.solve_triangular(Ld, r, lower=True), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(z, sla.solve_triangular(Ld.T, y, lower=False), rtol=1e-11, atol=1e-12)


@settings(max_examples=30, deadline=None)
@given(cases, st.sampled_from([1, 2, 5, 64]), st.integers(0, 4))
def test_spmv_and_split_spmv_exact_on_integers(orc, p, piece, cost):
    A = _m_matrix(p["n"], p["density"], p["seed"], integer=True)
    an = orc.analyse(A, p["bs"], p["w"])
    rng = np.random.default_rng(p["seed"] % 997)
    x = rng.integers(-7, 8, size=an.n_pad).astype(np.float64)
    n = an.n_pad
    dense = np.zeros((n, n), dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(an.row_ptr))
    dense[rows, an.col] = an.val.astype(np.int64)
    exact = (dense @ x.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(orc.spmv(an.row_ptr, an.col, an.val, x), exact)
    plan = orc.split_plan(an.row_ptr, p["w"], piece, cost)
    np.testing.assert_array_equal(orc.spmv_split(an.row_ptr, an.col, an.val, plan, x), exact)


@settings(max_examples=40, deadline=None)
@given(st.lists(st.floats(-1e6, 1e6, allow_nan=False, allow_infinity=False), min_size=1, max_size=60),
       st.integers(0, 2**31 - 1))
def test_sequential_dot_within_bound_of_exact(orc, a, seed):
    a = np.array(a)
    b = np.random.default_rng(seed).standard_normal(len(a))
    idx = np.arange(len(a), dtype=np.int64)
    exact = orc.dot(a, b, idx, mode=orc.DOT_EXACT)
    seq = orc.dot(a, b, idx, mode=orc.DOT_SEQUENTIAL)
    true = sum(fractions.Fraction(float(x)) * fractions.Fraction(float(y)) for x, y in zip(a, b))
    assert abs(fractions.Fraction(exact) - true) <= abs(true) * fractions.Fraction(2.0 ** -53) + \
        fractions.Fraction(2.0 ** -1074)
    u = 2.0 ** -53
    k = len(a)
    # recursive summation of k products: relative error gamma_k = k u / (1 - k u)
    # of sum |a_i b_i|, plus, where products or partial sums fall below the
    # normal range, an absolute error of at most half the smallest subnormal
    # (2^-1075) per rounding, 2k roundings
    # (2^-1075 as an exact rational: the float literal 2.0 ** -1075 is half
    # the smallest subnormal and rounds to zero)
    bound = fractions.Fraction(k * u / (1 - k * u)) * sum(abs(fractions.Fraction(float(x)) * fractions.Fraction(float(y)))
                                                         for x, y in zip(a, b)) + 2 * k * fractions.Fraction(1, 2 ** 1075)
    assert abs(fractions.Fraction(seq) - true) <= bound
