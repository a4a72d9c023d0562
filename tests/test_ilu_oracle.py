"""Pins for the oracle's ILU(0), U-substitution and BiCGStab (orc_ilu0,
orc_bwd_u, orc_bicgstab): the exact LU when the pattern has no fill, L U = A
on the pattern, the IC(0) relation for a symmetric matrix, the triangular
solve against a dense one, one-step convergence with the exact factorization,
convergence to the dense solution, and the HBMC / BMC equivalence of
iteration counts (Section 3.1)."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1908_00741_gb300 import workloads as W


def _dense(rp, ci, v, n):
    M = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            M[i, ci[e]] = v[e]
    return M


def _factors(rp, ci, lval, uval, udiag, n):
    L, U = np.eye(n), np.diag(udiag)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = ci[e]
            if j < i:
                L[i, j] = lval[e]
            elif j > i:
                U[i, j] = uval[e]
    return L, U


def _tridiag(n=30, seed=1):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j, a in ((i - 1, -1.0 - rng.random()), (i, 4.0 + rng.random()), (i + 1, -1.0 + 0.5 * rng.random())):
            if 0 <= j < n:
                rows.append(i); cols.append(j); vals.append(a)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return rp, np.array(cols, dtype=np.int32), np.array(vals), n


def test_ilu_is_exact_lu_without_fill():
    """A tridiagonal matrix in natural order has no fill: ILU(0) = LU, L U = A."""
    rp, ci, v, n = _tridiag()
    lval, uval, udiag, uinv, bad = oracle.ilu0(rp, ci, v)
    assert bad == -1
    L, U = _factors(rp, ci, lval, uval, udiag, n)
    A = _dense(rp, ci, v, n)
    assert np.max(np.abs(L @ U - A)) <= 1e-14 * np.max(np.abs(A))
    np.testing.assert_allclose(uinv, 1.0 / udiag, rtol=0, atol=0)


def test_ilu_matches_a_on_its_pattern():
    """The defining property of ILU(0): (L U)_ij = a_ij wherever a_ij != 0."""
    A = W.convection_diffusion(5)
    an = oracle.analyse(A, 8, 4, box=(2, 2, 2))
    lval, uval, udiag, uinv, bad = oracle.factor_ilu(an, 0.0)
    assert bad == -1
    n = an.n_pad
    L, U = _factors(an.row_ptr, an.col, lval, uval, udiag, n)
    Ab = _dense(an.row_ptr, an.col, an.val, n)
    LU = L @ U
    mask = Ab != 0
    assert np.max(np.abs(LU[mask] - Ab[mask])) <= 1e-13 * np.max(np.abs(Ab))
    assert np.max(np.abs(LU[~mask])) > 1e-6  # there is fill outside the pattern


def test_symmetric_matrix_relates_to_ic0():
    """For symmetric A, ILU(0) = (L_c D^-1)(D L_c^T) with the IC(0) factor L_c
    and D = diag(L_c): u_ii = l_ii^2, u_ij = l_ii l_ji, l_ij = l_ij / l_jj."""
    A = W.poisson7(5)
    an = oracle.analyse(A, 8, 4, box=(2, 2, 2))
    lc, ldiag, _, bad_c = oracle.factor(an, 0.1)
    lval, uval, udiag, uinv, bad = oracle.factor_ilu(an, 0.1)
    assert bad_c == -1 and bad == -1
    n = an.n_pad
    rp, ci = an.row_ptr, an.col
    np.testing.assert_allclose(udiag, ldiag ** 2, rtol=1e-13)
    tpos = oracle.transpose_pos(rp, ci)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = ci[e]
            if j < i:
                assert abs(lval[e] - lc[e] / ldiag[j]) <= 1e-13 * abs(lc[e] / ldiag[j]) + 1e-300
            elif j > i:
                ref = ldiag[i] * lc[tpos[e]]
                assert abs(uval[e] - ref) <= 1e-13 * abs(ref) + 1e-300


def test_backward_substitution_with_u():
    A = W.convection_diffusion(4)
    an = oracle.analyse(A, 8, 4, box=(2, 2, 2))
    lval, uval, udiag, uinv, _ = oracle.factor_ilu(an)
    n = an.n_pad
    _, U = _factors(an.row_ptr, an.col, lval, uval, udiag, n)
    y = np.random.default_rng(2).standard_normal(n)
    z = oracle.bwd_u(an.row_ptr, an.col, uval, uinv, y)
    ref = sl.solve_triangular(U, y, lower=False)
    assert np.max(np.abs(z - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_bicgstab_with_exact_factor_takes_one_step():
    """No fill (tridiagonal, natural order, one block): M = A, so the first
    half step solves the system."""
    rp, ci, v, n = _tridiag(24, 3)
    A = W.CSR(n, rp, ci, v)
    an = oracle.analyse(A, n, 1)  # one block holding every unknown: the natural order
    lval, uval, udiag, uinv, bad = oracle.factor_ilu(an)
    assert bad == -1
    b = np.cos(np.arange(n))
    s = oracle.bicgstab(an, lval, uval, uinv, b, tol=1e-12)
    assert s.status == 0 and s.iters == 1
    xs = np.linalg.solve(_dense(rp, ci, v, n), b)
    assert np.max(np.abs(s.x - xs)) <= 1e-12 * np.max(np.abs(xs))


def test_bicgstab_converges_to_the_solution():
    A = W.convection_diffusion(8, (2.0, 1.0, 0.5))
    b, xstar = W.rhs_from_solution(A, 0)
    an = oracle.analyse(A, 8, 32, box=(2, 2, 2))
    lval, uval, udiag, uinv, _ = oracle.factor_ilu(an)
    s = oracle.bicgstab(an, lval, uval, uinv, b, tol=1e-11)
    assert s.status == 0 and 1 < s.iters < 60
    assert np.max(np.abs(s.x - xstar)) <= 1e-8 * np.max(np.abs(xstar))
    assert s.relres < 1e-11


def test_hbmc_and_bmc_take_the_same_iterations():
    A = W.convection_diffusion(8)
    b, _ = W.rhs_from_solution(A, 0)
    res = []
    for hbmc in (True, False):
        an = oracle.analyse(A, 8, 4, box=(2, 2, 2), hbmc=hbmc)
        lval, uval, udiag, uinv, _ = oracle.factor_ilu(an)
        res.append(oracle.bicgstab(an, lval, uval, uinv, b, tol=1e-10))
    assert res[0].iters == res[1].iters
    assert np.max(np.abs(res[0].x - res[1].x)) <= 1e-10 * np.max(np.abs(res[0].x))


def test_zero_pivot_reported():
    rp = np.array([0, 2, 4], dtype=np.int64)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    v = np.array([1.0, 2.0, 0.5, 1.0])  # u_11 = 1 - 0.5 * 2 = 0
    *_, bad = oracle.ilu0(rp, ci, v)
    assert bad == 1
