"""Host logic of the learned IC shift, no GPU needed: which shift the plain
rule takes, the best shift, the training targets and the fallback, on
hand-built sweep results.

The shift alpha enters IC(0) as the diagonal (1 + alpha) a_ii (Section 5.1
uses alpha = 0.3 for one of its models).  The plain rule takes the smallest
grid shift whose IC(0) pivots are all positive and finite: it is defined on
the pivots alone, so a shift whose IC(0) succeeds but whose CG does not
converge is still its choice, and costs FAIL_FACTOR times maxit."""
import numpy as np
import pytest

from paper_1908_00741_gb300 import learned_shift as LS


def _sweep(iters, ic_ok, maxit=100):
    iters = np.asarray(iters, dtype=np.int64)
    ic_ok = np.asarray(ic_ok, dtype=bool)
    feats = np.arange(iters.shape[0] * 12, dtype=np.float32).reshape(iters.shape[0], 12)
    return LS.Sweep(feats, iters, ic_ok, np.full(iters.shape, np.nan), maxit)


def test_plain_choice_uses_pivots_only():
    assert LS.plain_choice(np.array([False, False, True, True])) == 2
    assert LS.plain_choice(np.array([True, True])) == 0
    assert LS.plain_choice(np.array([False, False])) == -1
    # IC(0) works at shift 1 but CG fails there: still the plain rule's shift
    sw = _sweep([[-1, -1, 30]], [[False, True, True]])
    assert LS.plain_choice(sw.ic_ok[0]) == 1
    assert sw.cost(0, 1) == int(LS.FAIL_FACTOR * sw.maxit)


def test_best_choice_least_cost_ties_to_smaller_shift():
    sw = _sweep([[50, 40, 40, 45], [-1, 20, 10, 10], [-1, -1, -1, -1]],
                [[True, True, True, True], [False, True, True, True], [False, False, False, False]])
    assert LS.best_choice(sw, 0) == 1   # 40 at shifts 1 and 2: the smaller
    assert LS.best_choice(sw, 1) == 2   # 10 at 2 and 3
    assert LS.best_choice(sw, 2) == -1  # no shift factors
    # a failed shift is never best while a converged one exists
    sw = _sweep([[-1, 399]], [[True, True]], maxit=100)
    assert LS.best_choice(sw, 0) == 1


def test_dataset_targets_relative_to_least_cost():
    g = 4
    sw = _sweep([[80, 40, -1, 20], [-1, -1, -1, -1], [-1, 25, 50, 100]],
                [[True, True, True, True], [False, False, False, False], [True, True, True, True]], maxit=100)
    X, T = LS.dataset(sw)
    # the system with no converged shift is left out
    assert X.shape == (2 * g, 13) and T.shape == (2 * g,)
    np.testing.assert_array_equal(X[:g, :12], np.repeat(sw.features[:1], g, axis=0))
    np.testing.assert_array_equal(X[g:, :12], np.repeat(sw.features[2:3], g, axis=0))
    np.testing.assert_allclose(X[:g, 12], np.arange(g) / (g - 1))
    fail = LS.FAIL_FACTOR * sw.maxit
    np.testing.assert_allclose(T[:g], np.log2(np.array([80, 40, fail, 20]) / 20), rtol=1e-6)
    np.testing.assert_allclose(T[g:], np.log2(np.array([fail, 25, 50, 100]) / 25), rtol=1e-6)
    # the target is zero exactly at each system's best shift
    assert T[:g].argmin() == LS.best_choice(sw, 0) and T[:g].min() == 0.0
    assert T[g:].argmin() == LS.best_choice(sw, 2) and T[g:].min() == 0.0


def test_dataset_least_cost_among_factoring_shifts():
    # shift 0's IC(0) fails: its (converged) count is not the reference
    sw = _sweep([[10, 40, 20]], [[False, True, True]])
    _, T = LS.dataset(sw)
    np.testing.assert_allclose(T, np.log2(np.array([10, 40, 20]) / 20), rtol=1e-6)


@pytest.mark.parametrize("ic,c,plain,expect", [
    ([True, True, True], 1, 0, (1, False)),
    ([False, False, True, True], 1, 2, (2, True)),
    ([True, False, False, True], 1, 0, (3, True)),
    ([True, True, False, False], 2, 0, (0, True)),   # nothing larger factors: the plain rule
    ([False, True, False], 2, 1, (1, True)),
])
def test_fallback_choice(ic, c, plain, expect):
    assert LS.fallback_choice(np.array(ic), c, plain) == expect


def test_evaluate_with_given_choices(monkeypatch):
    """evaluate() with the network's choices given: the plain, learned (with
    fallback) and best costs per system whose IC(0) works somewhere."""
    sw = _sweep([[-1, 30, 20, 25], [50, 40, 45, 60], [-1, -1, -1, -1], [-1, -1, 35, 30]],
                [[False, True, True, True], [True, True, True, True], [False, False, False, False],
                 [False, False, True, True]], maxit=100)
    choice = np.array([0, 2, 1, 1])
    monkeypatch.setattr(LS, "predicted_choice", lambda net, feats: (choice, None))
    plain, learned, best, fallback = LS.evaluate(None, sw)
    # system 2 factors at no shift and is left out
    np.testing.assert_array_equal(plain, [30, 50, 35])
    np.testing.assert_array_equal(learned, [30, 45, 35])   # 0 -> 1 (fallback), 2, 1 -> 2 (fallback)
    np.testing.assert_array_equal(best, [20, 40, 30])
    np.testing.assert_array_equal(fallback, [True, False, True])
