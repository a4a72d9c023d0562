"""Property tests of the oracle's SOR and ILU(0) over random inputs
(hypothesis, no GPU).  SOR (Section 2): one forward Gauss-Seidel sweep is
the lower-triangular solve (D + L) x1 = b - U x0, and omega scales the step
from x0.  ILU(0) (Section 2, Eq. "ILU"): L U equals A on A's pattern for
random nonsymmetric values on a symmetric pattern, and the two triangular
solves equal dense ones."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402
import scipy.linalg as sla  # noqa: E402
import scipy.sparse as sp  # noqa: E402


def _dominant(n, density, seed, symmetric_values):
    """Random symmetric pattern, values symmetric or not, strictly dominant
    diagonal; CSR with sorted columns."""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=seed)
    P = ((M + M.T) != 0).astype(np.float64).tocsr()
    P.setdiag(0.0)
    P.eliminate_zeros()
    P = P.tocoo()
    vals = -rng.uniform(0.1, 1.0, size=P.nnz)
    if symmetric_values:
        key = np.minimum(P.row, P.col) * n + np.maximum(P.row, P.col)
        _, inv = np.unique(key, return_inverse=True)
        vals = -rng.uniform(0.1, 1.0, size=inv.max() + 1)[inv] if P.nnz else vals
    S = sp.csr_matrix((vals, (P.row, P.col)), shape=(n, n))
    rowsum = np.asarray(abs(S).sum(axis=1)).ravel()
    colsum = np.asarray(abs(S).sum(axis=0)).ravel()
    S = (S + sp.diags(np.maximum(rowsum, colsum) + 0.5)).tocsr()
    S.sort_indices()
    return S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64), S.toarray()


mats = st.fixed_dictionaries({
    "n": st.integers(1, 70),
    "density": st.floats(0.0, 0.2),
    "seed": st.integers(0, 2**31 - 1),
})


@settings(max_examples=40, deadline=None)
@given(mats, st.floats(0.2, 1.8))
def test_sor_sweep_is_the_splitting_step(orc, p, omega):
    rp, ci, v, Ad = _dominant(p["n"], p["density"], p["seed"], True)
    n = p["n"]
    rng = np.random.default_rng(p["seed"] % 1009)
    b, x0 = rng.standard_normal(n), rng.standard_normal(n)
    D = np.diag(np.diag(Ad))
    Lo, Up = np.tril(Ad, -1), np.triu(Ad, 1)
    # omega = 1: (D + L) x1 = b - U x0
    gs = sla.solve_triangular(D + Lo, b - Up @ x0, lower=True)
    np.testing.assert_allclose(orc.sor(rp, ci, v, b, x0, 1.0, 1, False), gs, rtol=1e-11, atol=1e-12)
    # general omega: (D + omega L) x1 = omega b - (omega U + (omega - 1) D) x0
    rhs = omega * b - (omega * Up + (omega - 1.0) * D) @ x0
    so = sla.solve_triangular(D + omega * Lo, rhs, lower=True)
    np.testing.assert_allclose(orc.sor(rp, ci, v, b, x0, omega, 1, False), so, rtol=1e-10, atol=1e-11)


@settings(max_examples=40, deadline=None)
@given(mats, st.sampled_from([0.0, 0.25]))
def test_ilu0_reproduces_a_on_pattern(orc, p, shift):
    rp, ci, v, Ad = _dominant(p["n"], p["density"], p["seed"], False)
    n = p["n"]
    lval, uval, udiag, uinv, bad = orc.ilu0(rp, ci, v, shift)
    assert bad == -1
    rows = np.repeat(np.arange(n), np.diff(rp))
    Ld = np.eye(n)
    Ud = np.diag(udiag)
    low, up = ci < rows, ci > rows
    Ld[rows[low], ci[low]] = lval[low]
    Ud[rows[up], ci[up]] = uval[up]
    LU = Ld @ Ud
    target = Ad.copy()
    target[np.arange(n), np.arange(n)] *= (1.0 + shift)
    np.testing.assert_allclose(LU[rows, ci], target[rows, ci], rtol=1e-12, atol=1e-12 * np.abs(target).max())
    r = np.random.default_rng(p["seed"] % 1013).standard_normal(n)
    ones = np.ones(n)
    y = orc.fwd(rp, ci, lval, ones, r)
    z = orc.bwd_u(rp, ci, uval, uinv, y)
    np.testing.assert_allclose(y, sla.solve_triangular(Ld, r, lower=True, unit_diagonal=True),
                               rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(z, sla.solve_triangular(Ud, y, lower=False), rtol=1e-11, atol=1e-12)
