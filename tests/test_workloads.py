"""The synthetic generators produce what their docstrings promise: the stencil
sizes from the closed-form nonzero counts, symmetric matrices, SPD by
diagonal dominance, and a reproducible random stream."""
import numpy as np
import pytest

from paper_1908_00741_gb300 import workloads as W


def _sym_ok(A):
    S = A.to_scipy()
    return abs(S - S.T).max() == 0.0


@pytest.mark.parametrize("m", [3, 5, 8])
def test_poisson7_counts_and_symmetry(m):
    A = W.poisson7(m)
    assert A.n == m ** 3 and A.nnz == 7 * m ** 3 - 6 * m ** 2
    assert _sym_ok(A)
    d = A.to_scipy().diagonal()
    assert np.all(d == 6.0)


@pytest.mark.parametrize("m", [3, 6])
def test_hetero27_counts_and_dominance(m):
    A = W.heterogeneous_stencil(m, 27, 2.0, 1)
    assert A.nnz == (3 * m - 2) ** 3
    assert _sym_ok(A)
    S = A.to_scipy().tocsr()
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - d
    assert np.all(d >= off - 1e-12 * d) and np.any(d > off * (1 + 1e-12))
    assert np.all(S.data[S.indices != np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))] < 0)


def test_veclap_counts_dominance():
    m = 4
    A = W.vector_laplacian(m, 3, 1.05)
    assert A.n == 3 * m ** 3 and A.nnz == 9 * (7 * m ** 3 - 6 * m ** 2)
    assert _sym_ok(A)
    S = A.to_scipy().tocsr()
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - d
    np.testing.assert_allclose(d, 1.05 * off, rtol=1e-14)
    assert np.linalg.eigvalsh(S.toarray()).min() > 0


def test_random_order_is_permutation_and_permute_input_preserves_spectrum():
    A = W.heterogeneous_stencil(4, 7, 1.0, 2)
    o = W.random_order(9, A.n)
    assert np.array_equal(np.sort(o), np.arange(A.n))
    B = W.permute_input(A, o)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(B.to_scipy().toarray())),
                               np.sort(np.linalg.eigvalsh(A.to_scipy().toarray())), rtol=1e-12)
    # row k of B is natural row o[k]
    k = 5
    np.testing.assert_allclose(np.sort(B.val[B.row_ptr[k]:B.row_ptr[k + 1]]),
                               np.sort(A.val[A.row_ptr[o[k]]:A.row_ptr[o[k] + 1]]))


def test_splitmix64_reference_values():
    # splitmix64 seeded with 0: published first outputs of the reference generator
    z = W.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = W.uniform(0, 1000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.05


def _edge_gradient(m):
    """Discrete gradient of a node potential on the m^3 cell grid, in
    curl_curl's edge numbering (x-, then y-, then z-edges, lexicographic)."""
    n1 = m + 1
    node = lambda i, j, k: i + n1 * (j + n1 * k)  # noqa: E731
    rows, cols, vals = [], [], []
    e = 0
    for (di, dj, dk), (ni, nj, nk) in (((1, 0, 0), (m, n1, n1)), ((0, 1, 0), (n1, m, n1)), ((0, 0, 1), (n1, n1, m))):
        for k in range(nk):
            for j in range(nj):
                for i in range(ni):
                    rows += [e, e]
                    cols += [node(i + di, j + dj, k + dk), node(i, j, k)]
                    vals += [1.0, -1.0]
                    e += 1
    G = np.zeros((e, n1 ** 3))
    G[rows, cols] = vals
    return G


@pytest.mark.parametrize("hetero", [0.0, 0.7])
def test_curl_curl_gradients_are_its_null_space(hetero):
    """The curl of a gradient is zero, so A = C^T W C + sigma I maps every
    gradient field g to sigma g: sigma is an eigenvalue of multiplicity
    (m+1)^3 - 1 (potentials up to a constant), and every other eigenvalue is
    larger.  A wrong sign on any face of the discrete curl breaks this."""
    m, sigma = 3, 0.01
    A = W.curl_curl(m, sigma, 6, hetero)
    assert A.n == 3 * m * (m + 1) ** 2
    assert _sym_ok(A)
    S = A.to_scipy().toarray()
    G = _edge_gradient(m)
    phi = np.random.default_rng(0).standard_normal(G.shape[1])
    g = G @ phi
    np.testing.assert_allclose(S @ g, sigma * g, atol=1e-12 * np.abs(S).max() * np.abs(g).max())
    ev = np.linalg.eigvalsh(S)
    at_sigma = np.abs(ev - sigma) < 1e-9
    assert at_sigma.sum() == (m + 1) ** 3 - 1
    assert ev[~at_sigma].min() > sigma + 1e-3
    # off-diagonal entries of both signs: not an M-matrix
    off = S[~np.eye(A.n, dtype=bool)]
    assert (off > 0).any() and (off < 0).any()


def test_convection_diffusion_consistency():
    """Upwind differences are exact on linear functions: on interior rows A
    annihilates constants and maps the coordinate x_d to c_d.  The pattern is
    symmetric, the values are not, and A is a diagonally dominant M-matrix."""
    m, c = 5, (0.5, 0.3, 0.2)
    A = W.convection_diffusion(m, c)
    S = A.to_scipy().tocsr()
    idx = np.arange(m ** 3)
    x, y, z = idx % m, (idx // m) % m, idx // (m * m)
    interior = (x > 0) & (x < m - 1) & (y > 0) & (y < m - 1) & (z > 0) & (z < m - 1)
    np.testing.assert_allclose((S @ np.ones(m ** 3))[interior], 0.0, atol=1e-13)
    for d, coord in enumerate((x, y, z)):
        np.testing.assert_allclose((S @ coord.astype(float))[interior], c[d], rtol=1e-13)
    assert (abs(S - S.T) > 0).nnz > 0
    assert ((S != 0).astype(int) - (S.T != 0).astype(int)).nnz == 0
    d = S.diagonal()
    off = S - np.diag(d)
    assert off.max() <= 0
    assert np.all(d >= np.asarray(abs(off).sum(axis=1)).ravel())


def test_irregular_structural_translations():
    """A = sum_e (e_u - e_v)(e_u - e_v)^T (x) S_e plus SPD blocks on boundary
    nodes: a rigid translation of all nodes is felt only at the boundary, so
    interior nodes' rows annihilate it; A is symmetric positive definite."""
    m = 6
    A = W.irregular_structural(m, 7)
    assert A.n == 3 * m ** 3
    assert _sym_ok(A)
    S = A.to_scipy().toarray()
    node = np.arange(m ** 3)
    x, y, z = node % m, (node // m) % m, node // (m * m)
    inner = (x > 0) & (x < m - 1) & (y > 0) & (y < m - 1) & (z > 0) & (z < m - 1)
    rows = (3 * node[inner][:, None] + np.arange(3)).ravel()
    for t in np.eye(3):
        np.testing.assert_allclose((S @ np.tile(t, m ** 3))[rows], 0.0, atol=1e-12 * np.abs(S).max())
    assert np.linalg.eigvalsh(S).min() > 0
    # with a dominance factor every diagonal entry is that factor times its row's off-diagonal sum
    B = W.irregular_structural(m, 7, dominance=1.1).to_scipy().toarray()
    offsum = np.abs(B).sum(axis=1) - np.abs(np.diag(B))
    np.testing.assert_allclose(np.diag(B), 1.1 * offsum, rtol=1e-13)


def test_hetero27_dirichlet_surplus():
    """a_ij = -(k_i + k_j)/2 between neighbouring cells, and the diagonal sums
    (k_i + k_j)/2 over all 26 neighbour slots with k_j = k_i outside the
    domain.  k_i is recovered from the matrix itself (three mutually adjacent
    cells i, j, l give k_i = -a_ij - a_il + a_jl), and each row's diagonal
    exceeds its off-diagonal sum by exactly k_i per slot outside the domain."""
    m = 5
    A = W.heterogeneous_stencil(m, 27, 2.0, 1)
    S = A.to_scipy().toarray()
    n = m ** 3
    idx = np.arange(n)
    x, y, z = idx % m, (idx // m) % m, idx // (m * m)
    sx = np.where(x < m - 1, 1, -1)  # a neighbour inside the domain along x, and along y
    sy = np.where(y < m - 1, 1, -1)
    j = idx + sx
    l_ = idx + m * sy
    kappa = -S[idx, j] - S[idx, l_] + S[j, l_]
    assert np.all(kappa > 0)
    inside_slots = np.zeros(n)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx, dy, dz) != (0, 0, 0):
                    inside_slots += ((x + dx >= 0) & (x + dx < m) & (y + dy >= 0) & (y + dy < m)
                                     & (z + dz >= 0) & (z + dz < m))
    surplus = np.diag(S) - (np.abs(S).sum(axis=1) - np.abs(np.diag(S)))
    np.testing.assert_allclose(surplus, (26 - inside_slots) * kappa, rtol=1e-10, atol=1e-12 * np.abs(S).max())
    # and the recovered k reproduces every coupling
    rows, cols = np.nonzero(S)
    offd = rows != cols
    np.testing.assert_allclose(S[rows[offd], cols[offd]], -(kappa[rows[offd]] + kappa[cols[offd]]) / 2, rtol=1e-12)


def test_batch_problems_contract():
    """Each system of the uneven batch is a 7- or 27-point stencil on an m^3
    grid with nmin <= m <= nmax, symmetric, with b = A x*; both stencils occur
    and the draws are reproducible."""
    items = W.batch_problems(16, seed0=1000, nmin=3, nmax=7)
    kinds = set()
    for A, b, xs in items:
        m = round(A.n ** (1 / 3))
        assert m ** 3 == A.n and 3 <= m <= 7
        if A.nnz == 7 * m ** 3 - 6 * m ** 2:
            kinds.add(7)
        else:
            assert A.nnz == (3 * m - 2) ** 3
            kinds.add(27)
        assert _sym_ok(A)
        np.testing.assert_allclose(A.to_scipy() @ xs, b, rtol=1e-12, atol=1e-12)
        assert np.all(np.abs(xs) <= 1)
    assert kinds == {7, 27}
    again = W.batch_problems(16, seed0=1000, nmin=3, nmax=7)
    assert all(np.array_equal(a[1], c[1]) for a, c in zip(items, again))


def test_learned_family_contract():
    """The learned-shift family mixes curl-curl (3 m (m+1)^2 edges), 3-DOF
    vector Laplacian (3 m^3) and 27-point (m^3, (3m - 2)^3 nonzeros) systems,
    each symmetric, in a random input order."""
    fam = W.learned_family(24, 5000, cc_m=(2, 3), vl_m=(2, 3), st_m=(3, 4))
    kinds = set()
    for A, b in fam:
        assert _sym_ok(A) and len(b) == A.n
        if A.n in (3 * 2 * 9, 3 * 3 * 16):
            kinds.add("curl")
        elif A.n in (3 * 8, 3 * 27):
            kinds.add("veclap")
        else:
            m = round(A.n ** (1 / 3))
            assert m ** 3 == A.n and A.nnz == (3 * m - 2) ** 3
            kinds.add("stencil27")
    assert kinds == {"curl", "veclap", "stencil27"}
