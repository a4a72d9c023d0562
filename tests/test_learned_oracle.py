"""Pins for the learned-shift reference (oracle/learned.py): the MLP gradient
against central finite differences, features against closed forms, and the
plain rule on a matrix whose admissible shifts are known exactly."""
import numpy as np
import pytest

from oracle import learned as L
from paper_1908_00741_gb300 import workloads as W


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    D, B = 5, 17
    p = rng.standard_normal(L.n_params(D)) * 0.5
    X = rng.standard_normal((B, D))
    T = rng.standard_normal(B)
    mean, std = X.mean(0), X.std(0) + 0.1
    g = L.gradient(p, mean, std, X, T)
    num = np.zeros_like(p)
    h = 1e-6
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        num[k] = (L.loss(p + e, mean, std, X, T) - L.loss(p - e, mean, std, X, T)) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_mlp_forward_shapes_and_relu():
    D = 3
    p = np.zeros(L.n_params(D))
    W1, b1, W2, b2, w3, b3 = L.unpack(p, D)
    assert W1.shape == (32, 3) and W2.shape == (32, 32)
    p[-1] = 2.5  # only the output bias: every output equals it
    out, _ = L.forward(p, np.zeros(D), np.ones(D), np.ones((4, D)))
    np.testing.assert_array_equal(out, 2.5)


@pytest.mark.parametrize("m", [4, 7])
def test_features_closed_form_poisson(m):
    A = W.poisson7(m)
    f = L.features(A, nc=2, bs=8)
    n = m ** 3
    assert f[0] == pytest.approx(np.log10(n))
    assert f[1] == pytest.approx((7 * m ** 3 - 6 * m ** 2) / n)
    assert f[2] == 7
    assert f[3] == pytest.approx(1.0)           # interior rows: 6 / (6 * 1)
    assert f[5] == 0.0 and f[6] == 0.0           # no weak rows, no positive off-diagonals
    assert f[7] == pytest.approx(np.log(6.0)) and f[8] == pytest.approx(0.0, abs=1e-12)
    assert f[9] == 2 and f[10] == 8
    assert f[11] == L.DOM_CAP or f[11] == pytest.approx(6.0 / 3.0)  # corner rows: 6 / 3


def test_features_closed_form_vector_laplacian():
    A = W.vector_laplacian(4, 3, dominance=1.05)
    f = L.features(A, nc=3, bs=4)
    assert f[3] == pytest.approx(1.05) and f[4] == pytest.approx(1.05) and f[11] == pytest.approx(1.05)
    assert f[5] == 0.0


def test_plain_rule_exact_threshold(orc):
    """[[1,2],[2,1]]: IC(0) needs (1+a)^2 > 4, i.e. a > 1; the first grid shift
    above 1 is 1e-3 * 2^10 = 1.024."""
    import scipy.sparse as sp
    S = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    A = W.CSR(2, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data)
    an = orc.analyse(A, 2, 1)
    assert L.plain_rule(an) == pytest.approx(1.024)
    P = W.poisson7(4)
    assert L.plain_rule(orc.analyse(P, 8, 4, box=(2, 2, 2))) == 0.0


def test_shift_grid():
    g = L.shift_grid()
    assert len(g) == 13 and g[0] == 0 and g[1] == 1e-3 and g[-1] == pytest.approx(2.048)
