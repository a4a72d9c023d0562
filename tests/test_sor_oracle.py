"""Pins for the oracle's SOR / symmetric SOR sweeps (orc_sor): one sweep
against the closed forms of the splitting A = L + D + U (dense triangular
solves), the symmetric sweep against the SSOR preconditioner, the equivalence
of the HBMC and BMC orderings for SOR iterates (Section 3.1, Eq. "xj"), and
convergence to the dense solution."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1908_00741_gb300 import workloads as W


def _dense(an):
    n = an.n_pad
    M = np.zeros((n, n))
    for i in range(n):
        for e in range(an.row_ptr[i], an.row_ptr[i + 1]):
            M[i, an.col[e]] = an.val[e]
    return M


def _small():
    A = W.permute_input(W.heterogeneous_stencil(4, 27, 1.0, 3), W.random_order(5, 64))
    return oracle.analyse(A, 4, 4)


@pytest.mark.parametrize("omega", [1.0, 0.7, 1.6])
def test_forward_sweep_closed_form(omega):
    """x1 = (D + w L)^-1 (w b - (w U + (w - 1) D) x0) on Abar."""
    an = _small()
    M = _dense(an)
    D, L, U = np.diag(np.diag(M)), np.tril(M, -1), np.triu(M, 1)
    rng = np.random.default_rng(1)
    b, x0 = rng.standard_normal(an.n_pad), rng.standard_normal(an.n_pad)
    x1 = oracle.sor(an.row_ptr, an.col, an.val, b, x0, omega, 1, False)
    ref = sl.solve_triangular(D + omega * L, omega * b - (omega * U + (omega - 1.0) * D) @ x0, lower=True)
    assert np.max(np.abs(x1 - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("omega", [1.0, 1.4])
def test_symmetric_sweep_from_zero_is_ssor_preconditioner(omega):
    """From x0 = 0 one symmetric sweep gives M^-1 b with
    M = (D + w L) D^-1 (D + w U) / (w (2 - w))."""
    an = _small()
    M = _dense(an)
    D, L, U = np.diag(np.diag(M)), np.tril(M, -1), np.triu(M, 1)
    b = np.random.default_rng(2).standard_normal(an.n_pad)
    x = oracle.sor(an.row_ptr, an.col, an.val, b, np.zeros(an.n_pad), omega, 1, True)
    y = sl.solve_triangular(D + omega * L, b, lower=True)
    ref = omega * (2.0 - omega) * sl.solve_triangular(D + omega * U, D @ y, lower=False)
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_hbmc_and_bmc_orderings_give_the_same_iterates():
    """Section 3.1: an equivalent reordering gives the same SOR iterates
    (Eq. "xj"); HBMC and BMC with the same blocks and colors satisfy the ER
    condition, so after k sweeps x agrees up to the rounding of the row sums."""
    A = W.poisson7(8)
    b, _ = W.rhs_from_solution(A, 0)
    xs = []
    for hbmc in (True, False):
        an = oracle.analyse(A, 8, 4, box=(2, 2, 2), hbmc=hbmc)
        xs.append(oracle.sor_solve(an, b, omega=1.3, sweeps=3, symmetric=True))
    assert np.max(np.abs(xs[0] - xs[1])) <= 1e-13 * np.max(np.abs(xs[0]))


def test_natural_order_is_not_equivalent():
    """The original (lexicographic) order is not an equivalent reordering of the
    multi-color one: the iterates differ by far more than rounding."""
    A = W.poisson7(8)
    b, _ = W.rhs_from_solution(A, 0)
    an = oracle.analyse(A, 8, 4, box=(2, 2, 2))
    x_hbmc = oracle.sor_solve(an, b, omega=1.0, sweeps=2)
    x_nat = oracle.sor(A.row_ptr, A.col, A.val, b, np.zeros(A.n), 1.0, 2, False)
    assert np.max(np.abs(x_hbmc - x_nat)) > 1e-6


def test_sor_converges_to_the_solution():
    A = W.poisson7(6)
    b, xstar = W.rhs_from_solution(A, 0)
    an = oracle.analyse(A, 8, 32, box=(2, 2, 2))
    x = oracle.sor_solve(an, b, omega=1.5, sweeps=300, symmetric=False)
    assert np.max(np.abs(x - xstar)) <= 1e-10 * np.max(np.abs(xstar))


def test_zero_diagonal_is_refused():
    rp = np.array([0, 2, 4], dtype=np.int64)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    v = np.array([1.0, 2.0, 2.0, 0.0])
    with pytest.raises(ValueError):
        oracle.sor(rp, ci, v, np.ones(2), np.zeros(2), 1.0, 1, False)
