"""Seeded synthetic inputs for the HBMC-ICCG solver.

This module only *generates* test systems (sparse SPD matrices in CSR form,
right-hand sides, random input orderings).  It holds none of the solver's
arithmetic: no blocking, coloring, reordering, factorization, substitution or
CG step.  Both the CUDA path and the CPU oracle consume what it produces.

The paper measures on SuiteSparse matrices (Thermal2, Parabolic_fem,
G3_circuit, Audikw_1) and the IEEJ eddy-current model (Section 5.1, Table
"matInfo").  Those data sets are not available here, so these generators stand
in for them with stencil matrices of the same shape class: 7-point stencils
(about 7 nonzeros per row, like Thermal2 and Parabolic_fem), a heterogeneous
27-point stencil and a 3-DOF vector Laplacian (denser rows, like Ieej and
Audikw_1).

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the k-th output of stream
``seed`` (k = 1, 2, ...) is ``mix(seed + k * 0x9E3779B97F4A7C15)``.  Uniforms
are ``(out >> 11) * 2**-53`` in [0, 1).

CSR conventions: ``row_ptr`` int64 of length n+1, ``col`` int32 sorted
ascending within each row, ``val`` float64; both triangles stored.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset+1 .. offset+count`` of the splitmix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): 53 high bits of splitmix64 times 2**-53."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, sigma: float = 1.0) -> np.ndarray:
    """N(0, sigma^2) by Box-Muller on consecutive uniform pairs (cosine branch)."""
    u = uniform(seed, 2 * count).reshape(count, 2)
    u1 = 1.0 - u[:, 0]  # in (0, 1], keeps log finite
    return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[:, 1])


def random_order(seed: int, n: int) -> np.ndarray:
    """A uniformly random permutation: ``order[k]`` is the natural index placed at
    input position k (stable argsort of splitmix64 keys)."""
    return np.argsort(splitmix64(seed, n), kind="stable").astype(np.int64)


@dataclasses.dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]
    grid: tuple | None = None  # (nx, ny, nz) when rows are a lexicographic grid, x fastest

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """Plain CSR product, used only to build right-hand sides b = A x*."""
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.n)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def _assemble(n, rows, cols, vals, grid=None) -> CSR:
    """Sort (row, col) pairs and pack them as CSR (no duplicate pairs expected)."""
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    o = np.argsort(key, kind="stable")
    rows, cols, vals = rows[o], cols[o], vals[o]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), vals.astype(np.float64), grid)


def _stencil_offsets(points: int):
    if points == 7:
        return [(dz, dy, dx) for dz, dy, dx in
                [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]]
    if points == 27:
        return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    raise ValueError("points must be 7 or 27")


def _grid_stencil(nx, ny, nz, points, kappa=None) -> CSR:
    """Stencil matrix on an nx*ny*nz grid, natural lexicographic order (x fastest).

    kappa=None: unit-coefficient Poisson (7-point: diagonal 6, -1 per face
    neighbour; 27-point: diagonal 26, -1 per neighbour), Dirichlet boundary.
    kappa given (per cell): a_ij = -(k_i+k_j)/2 for each neighbour j, and
    a_ii = sum over every neighbour slot, in or out of the domain, of
    (k_i+k_j)/2 with k_j = k_i outside.  That is a symmetric, weakly
    diagonally dominant, irreducible M-matrix with strict dominance on the
    boundary, hence SPD.
    """
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for dz, dy, dx in _stencil_offsets(points):
        if (dz, dy, dx) == (0, 0, 0):
            continue
        xx, yy, zz = x + dx, y + dy, z + dz
        inside = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        j = xx + nx * (yy + ny * zz)
        if kappa is None:
            diag += 1.0
            rows.append(idx[inside]); cols.append(j[inside]); vals.append(-np.ones(int(inside.sum())))
        else:
            kj = np.where(inside, kappa[np.where(inside, j, 0)], kappa)
            c = 0.5 * (kappa + kj)
            diag += c
            rows.append(idx[inside]); cols.append(j[inside]); vals.append(-c[inside])
    rows.append(idx); cols.append(idx); vals.append(diag)
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     grid=(nx, ny, nz))


def poisson7(m: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """3D 7-point Poisson, unit coefficients, Dirichlet: diagonal 6, -1 per face
    neighbour, natural lexicographic order with x fastest."""
    ny = m if ny is None else ny
    nz = m if nz is None else nz
    return _grid_stencil(m, ny, nz, 7)


def smoothed_lognormal_kappa(nx, ny, nz, sigma: float, seed: int) -> np.ndarray:
    """Per-cell coefficient exp(g~): g ~ N(0, sigma^2) per cell (Box-Muller,
    splitmix64 stream `seed`), g~ = mean of g over the 3x3x3 window around the
    cell with indices clamped to the grid."""
    g = normal(seed, nx * ny * nz, sigma).reshape(nz, ny, nx)
    acc = np.zeros_like(g)
    for dz in (-1, 0, 1):
        iz = np.clip(np.arange(nz) + dz, 0, nz - 1)
        for dy in (-1, 0, 1):
            iy = np.clip(np.arange(ny) + dy, 0, ny - 1)
            for dx in (-1, 0, 1):
                ix = np.clip(np.arange(nx) + dx, 0, nx - 1)
                acc += g[np.ix_(iz, iy, ix)]
    return np.exp(acc.reshape(-1) / 27.0)


def heterogeneous_stencil(m: int, points: int, sigma: float, seed: int) -> CSR:
    """7- or 27-point stencil with smoothed lognormal coefficients on an m^3 grid."""
    kappa = smoothed_lognormal_kappa(m, m, m, sigma, seed)
    return _grid_stencil(m, m, m, points, kappa)


def convection_diffusion(m: int, velocity=(0.5, 0.3, 0.2)) -> CSR:
    """Nonsymmetric 7-point convection-diffusion on m^3 (natural order, x
    fastest, Dirichlet): -Laplace(u) + c . grad(u) with first-order upwind
    differences for c >= 0 (grid units): the neighbour at -e_d gets
    -(1 + c_d), the one at +e_d gets -1, the diagonal 6 + sum_d c_d.  The
    pattern is symmetric, the values are not; an irreducibly diagonally
    dominant M-matrix."""
    n = m ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % m, (idx // m) % m, idx // (m * m)
    rows, cols, vals = [idx], [idx], [np.full(n, 6.0 + float(sum(velocity)))]
    for d, (dz, dy, dx) in enumerate([(0, 0, 1), (0, 1, 0), (1, 0, 0)]):
        c = float(velocity[d])  # d = 0: x, 1: y, 2: z
        for sgn in (-1, 1):
            xx, yy, zz = x + sgn * dx, y + sgn * dy, z + sgn * dz
            inside = (xx >= 0) & (xx < m) & (yy >= 0) & (yy < m) & (zz >= 0) & (zz < m)
            j = xx + m * (yy + m * zz)
            rows.append(idx[inside])
            cols.append(j[inside])
            vals.append(np.full(int(inside.sum()), -(1.0 + c) if sgn < 0 else -1.0))
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), grid=(m, m, m))


def permute_input(A: CSR, order: np.ndarray) -> CSR:
    """Relabel unknowns: input row k is natural row order[k] (A_in = Q A Q^T)."""
    n = A.n
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.row_ptr))
    return _assemble(n, inv[rows], inv[A.col.astype(np.int64)], A.val.copy(), grid=None)


def _random_spd3(seed: int, count: int) -> np.ndarray:
    """`count` random SPD 3x3 matrices Q diag(lam) Q^T with lam ~ U[0.1, 1] and Q
    from the QR factorization of a Gaussian 3x3 (splitmix64 stream `seed`)."""
    g = normal(seed, 9 * count).reshape(count, 3, 3)
    q, _ = np.linalg.qr(g)
    lam = 0.1 + 0.9 * uniform(seed ^ 0x5DEECE66D, 3 * count).reshape(count, 3)
    S = np.einsum("eij,ej,ekj->eik", q, lam, q)
    return 0.5 * (S + np.transpose(S, (0, 2, 1)))  # exactly symmetric in floating point


def vector_laplacian(m: int, seed: int, dominance: float = 1.05) -> CSR:
    """3 DOF per node, 7-point node coupling on an m^3 grid (unknown 3*node+d).

    Each node-to-node edge e carries a random SPD 3x3 block S_e; the off-node
    block is -S_e and the node block is the sum of S_e over the node's six
    edge slots (Dirichlet slots outside the domain get their own random S_e),
    intra-node off-diagonals kept.  Finally every scalar diagonal entry is
    replaced by dominance * (sum of |a_kl| over the rest of its row), which for
    dominance > 1 gives a strictly diagonally dominant, hence SPD, matrix.
    """
    nn = m * m * m
    idx = np.arange(nn, dtype=np.int64)
    x = idx % m
    y = (idx // m) % m
    z = idx // (m * m)
    # Edge slots: +x, +y, +z from every node (out-of-domain ones are Dirichlet
    # slots), plus the -x, -y, -z slots that leave the domain.
    S_plus = _random_spd3(seed, 3 * nn).reshape(3, nn, 3, 3)
    S_minus_bnd = _random_spd3(seed + 0x9E37, 3 * nn).reshape(3, nn, 3, 3)
    node_block = np.zeros((nn, 3, 3))
    brow, bcol, bval = [], [], []
    for a, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        xx, yy, zz = x + dx, y + dy, z + dz
        inside = (xx < m) & (yy < m) & (zz < m)
        j = xx + m * (yy + m * zz)
        S = S_plus[a]
        node_block += S  # this node's +slot
        # neighbour's -slot is the same edge
        np.add.at(node_block, j[inside], S[inside])
        brow.append(idx[inside]); bcol.append(j[inside]); bval.append(-S[inside])
        brow.append(j[inside]); bcol.append(idx[inside]); bval.append(-np.transpose(S[inside], (0, 2, 1)))
        # -slot that leaves the domain: x - dx < 0
        xm, ym, zm = x - dx, y - dy, z - dz
        outside = (xm < 0) | (ym < 0) | (zm < 0)
        node_block[outside] += S_minus_bnd[a][outside]
    brow.append(idx); bcol.append(idx); bval.append(node_block)
    br = np.concatenate(brow); bc = np.concatenate(bcol); bv = np.concatenate(bval)
    d = np.arange(3)
    rows = (3 * br[:, None, None] + d[None, :, None]) + 0 * d[None, None, :]
    cols = (3 * bc[:, None, None] + d[None, None, :]) + 0 * d[None, :, None]
    A = _assemble(3 * nn, rows.reshape(-1), cols.reshape(-1), bv.reshape(-1))
    rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    is_diag = rows_of == A.col
    offsum = np.bincount(rows_of, weights=np.where(is_diag, 0.0, np.abs(A.val)), minlength=A.n)
    A.val[is_diag] = dominance * offsum
    return A


def irregular_structural(m: int, seed: int, mean_refine: float = 0.11, keep_near: float = 0.65,
                         dominance: float | None = None) -> CSR:
    """3 DOF per node on an m^3 grid of nodes with an irregular, widely spread
    number of couplings per node (unknown 3*node+d), shaped like a structural
    FEM matrix such as Audikw_1: about 80 nonzeros per row on average, row
    lengths spread with a coefficient of variation near 0.27.

    Node u draws a refinement level rho_u = min(1, -mean_refine * ln(1 - U_u))
    (exponential, stream `seed`).  Node pairs at Chebyshev distance 1 are
    coupled with probability keep_near, pairs at distance 2 with probability
    (rho_u + rho_v) / 2 (one uniform per pair, stream seed + 1 + k for the k-th
    of the 62 forward offsets).  Each coupled pair e carries a random SPD 3x3
    block S_e (stream seed + 1000 + k): A = sum_e (e_u - e_v)(e_u - e_v)^T (x) S_e,
    plus a random SPD block on every node of the domain boundary (stream
    seed + 999), so A is SPD and has the conditioning of a vector Laplacian.
    With `dominance`, every scalar diagonal entry is then replaced by dominance
    times the sum of |a_kl| over the rest of its row instead.
    """
    nn = m * m * m
    idx = np.arange(nn, dtype=np.int64)
    x = idx % m
    y = (idx // m) % m
    z = idx // (m * m)
    rho = np.minimum(1.0, -mean_refine * np.log1p(-uniform(seed, nn)))
    node_block = np.zeros((nn, 3, 3))
    brow, bcol, bval = [], [], []
    offsets = [(dz, dy, dx) for dz in range(-2, 3) for dy in range(-2, 3) for dx in range(-2, 3)
               if (dz, dy, dx) > (0, 0, 0)]
    for k, (dz, dy, dx) in enumerate(offsets):
        xx, yy, zz = x + dx, y + dy, z + dz
        inside = (xx >= 0) & (xx < m) & (yy >= 0) & (yy < m) & (zz >= 0) & (zz < m)
        j = np.where(inside, xx + m * (yy + m * zz), 0)
        u = uniform(seed + 1 + k, nn)
        if max(abs(dx), abs(dy), abs(dz)) == 1:
            keep = inside & (u < keep_near)
        else:
            keep = inside & (u < 0.5 * (rho + rho[j]))
        a, b = idx[keep], j[keep]
        S = _random_spd3(seed + 1000 + k, len(a))
        np.add.at(node_block, a, S)
        np.add.at(node_block, b, S)
        brow.append(a); bcol.append(b); bval.append(-S)
        brow.append(b); bcol.append(a); bval.append(-S)  # S_e is symmetric
    bnd = (x == 0) | (x == m - 1) | (y == 0) | (y == m - 1) | (z == 0) | (z == m - 1)
    node_block[bnd] += _random_spd3(seed + 999, int(bnd.sum()))
    brow.append(idx); bcol.append(idx); bval.append(node_block)
    br = np.concatenate(brow); bc = np.concatenate(bcol); bv = np.concatenate(bval)
    d = np.arange(3)
    rows = (3 * br[:, None, None] + d[None, :, None]) + 0 * d[None, None, :]
    cols = (3 * bc[:, None, None] + d[None, None, :]) + 0 * d[None, :, None]
    A = _assemble(3 * nn, rows.reshape(-1), cols.reshape(-1), bv.reshape(-1))
    if dominance is not None:
        rows_of = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        is_diag = rows_of == A.col
        offsum = np.bincount(rows_of, weights=np.where(is_diag, 0.0, np.abs(A.val)), minlength=A.n)
        A.val[is_diag] = dominance * offsum
    return A


def curl_curl(m: int, sigma: float, seed: int, hetero: float = 0.0) -> CSR:
    """Edge unknowns of an m^3 cell grid (3 m (m+1)^2 edges; unknown order:
    x-edges, then y-, then z-edges, each lexicographic) with
    A = C^T W C + sigma I: C is the discrete curl (face <- its four edges,
    signs by the face's orientation), W = diag(w_f) with w_f = exp(N(0,
    hetero^2)) per face (stream `seed`), sigma > 0 a mass-like shift.  The
    shape of an edge-element eddy-current system such as the paper's IEEJ
    model: symmetric positive definite but nearly singular for small sigma
    (the gradients are in the null space of the curl), off-diagonal entries
    of both signs, and an IC(0) that breaks down without a diagonal shift.
    """
    n1 = m + 1
    nx, ny = m * n1 * n1, n1 * m * n1

    def ex(i, j, k):
        return i + m * (j + n1 * k)

    def ey(i, j, k):
        return nx + i + n1 * (j + m * k)

    def ez(i, j, k):
        return nx + ny + i + n1 * (j + n1 * k)

    faces = []
    g = np.arange
    # xy faces (i < m, j < m, k <= m): +ex(i,j,k) +ey(i+1,j,k) -ex(i,j+1,k) -ey(i,j,k)
    k, j, i = np.meshgrid(g(n1), g(m), g(m), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    faces.append(np.stack([ex(i, j, k), ey(i + 1, j, k), ex(i, j + 1, k), ey(i, j, k)], 1))
    # yz faces (i <= m, j < m, k < m): +ey(i,j,k) +ez(i,j+1,k) -ey(i,j,k+1) -ez(i,j,k)
    k, j, i = np.meshgrid(g(m), g(m), g(n1), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    faces.append(np.stack([ey(i, j, k), ez(i, j + 1, k), ey(i, j, k + 1), ez(i, j, k)], 1))
    # zx faces (i < m, j <= m, k < m): +ez(i,j,k) +ex(i,j,k+1) -ez(i+1,j,k) -ex(i,j,k)
    k, j, i = np.meshgrid(g(m), g(n1), g(m), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    faces.append(np.stack([ez(i, j, k), ex(i, j, k + 1), ez(i + 1, j, k), ex(i, j, k)], 1))
    F = np.concatenate(faces).astype(np.int64)
    sign = np.array([1.0, 1.0, -1.0, -1.0])
    w = np.exp(normal(seed, len(F), hetero)) if hetero > 0 else np.ones(len(F))
    n = nx + ny + n1 * n1 * m
    rows = np.repeat(F, 4, axis=1).ravel()
    cols = np.tile(F, (1, 4)).ravel()
    vals = (w[:, None, None] * sign[None, :, None] * sign[None, None, :]).reshape(-1)
    # sum the faces' contributions per (row, col) pair, then add sigma on the diagonal
    key = rows * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    acc = np.bincount(inv, weights=vals, minlength=len(uk))
    r, c = uk // n, uk % n
    acc[r == c] += sigma
    return _assemble(n, r, c, acc)


def learned_family(count: int, seed0: int, cc_m=(8, 24), vl_m=(8, 20), st_m=(12, 32),
                   mix=(0.5, 0.25, 0.25)):
    """Systems for the learned IC shift: `count` pairs (A, b), system k from
    stream seed0 + k, drawn with probabilities `mix` from
      - curl-curl systems (curl_curl with m ~ U{cc_m}, sigma = 10^U(-3, 0),
        face heterogeneity ~ U(0, 1.2)): IC(0) needs a shift, and the best
        grid shift is the first one that works or the next;
      - 3-DOF vector Laplacians (m ~ U{vl_m} nodes per side, dominance
        ~ U[0.9, 1.2]);
      - heterogeneous 27-point stencils (m ~ U{st_m}, sigma ~ U[0, 2]);
    the last two with the plain rule's 0 as the best shift.  Random input
    order; b = A x*, x* ~ U(-1, 1).  Curl-curl grids of 8 to 24 cells: small
    grids are dominated by their boundary edges, whose features (row
    lengths, dominance, diagonal spread) differ from a large grid's, and a
    network trained on 6-12 cells chose 2.048 on a 70^3 system where one
    trained on 8-24 chooses 0.512."""
    out = []
    for k in range(count):
        seed = seed0 + k
        u = uniform(seed, 5)

        def pick(lo_hi):
            return lo_hi[0] + min(int(u[1] * (lo_hi[1] - lo_hi[0] + 1)), lo_hi[1] - lo_hi[0])

        if u[0] < mix[0]:
            A = curl_curl(pick(cc_m), 10.0 ** (-3.0 + 3.0 * u[2]), seed, 1.2 * u[3])
        elif u[0] < mix[0] + mix[1]:
            A = vector_laplacian(pick(vl_m), seed, 0.9 + 0.3 * u[2])
        else:
            A = heterogeneous_stencil(pick(st_m), 27, 2.0 * u[2], seed)
        A = permute_input(A, random_order(seed ^ 0x5BD1E995, A.n))
        b, _ = rhs_from_solution(A, seed + 77777)
        out.append((A, b))
    return out


@dataclasses.dataclass
class Problem:
    """A linear system with its right-hand side and the blocking hint it asks for."""
    name: str
    A: CSR
    b: np.ndarray
    x_star: np.ndarray
    bs: int
    w: int
    box: tuple | None  # (bx, by, bz) geometric blocking on A.grid, else None (algebraic)


def rhs_from_solution(A: CSR, seed: int):
    """x* ~ U(-1, 1) per unknown (stream `seed`), b = A x*."""
    x_star = 2.0 * uniform(seed, A.n) - 1.0
    return A.matvec(x_star), x_star


def box_for_bs(bs: int) -> tuple:
    """Geometric block shape (bx, by, bz) for a block size: x extent smallest,
    z varying slowest (8 = 2x2x2, 16 = 2x2x4, 32 = 2x4x4, 4 = 1x2x2, 2 = 1x1x2)."""
    shapes = {1: (1, 1, 1), 2: (1, 1, 2), 4: (1, 2, 2), 8: (2, 2, 2), 16: (2, 2, 4),
              32: (2, 4, 4), 64: (4, 4, 4)}
    if bs not in shapes:
        raise ValueError(f"no box shape for bs={bs}")
    return shapes[bs]


def poisson_problem(m: int, bs: int = 8, w: int = 32, seed: int = 0) -> Problem:
    """7-point Poisson on m^3, geometric bs-cubes, b = A x* with x* ~ U(-1,1)."""
    A = poisson7(m)
    b, xs = rhs_from_solution(A, seed)
    return Problem(f"poisson7_{m}^3_bs{bs}", A, b, xs, bs, w, box_for_bs(bs))


def heterogeneous27_problem(m: int, bs: int = 8, w: int = 32, sigma: float = 2.0,
                            kappa_seed: int = 1, order_seed: int = 2, rhs_seed: int = 0) -> Problem:
    """Heterogeneous 27-point stencil on m^3 in a random input order (algebraic blocking)."""
    A = heterogeneous_stencil(m, 27, sigma, kappa_seed)
    A = permute_input(A, random_order(order_seed, A.n))
    b, xs = rhs_from_solution(A, rhs_seed)
    return Problem(f"hetero27_{m}^3_bs{bs}", A, b, xs, bs, w, None)


def vector_laplacian_problem(m: int, bs: int = 8, w: int = 32, seed: int = 3,
                             order_seed: int = 4, rhs_seed: int = 0, dominance: float = 1.05) -> Problem:
    """3-DOF vector Laplacian on m^3 nodes in a random input order."""
    A = vector_laplacian(m, seed, dominance)
    A = permute_input(A, random_order(order_seed, A.n))
    b, xs = rhs_from_solution(A, rhs_seed)
    return Problem(f"veclap_{m}^3_bs{bs}", A, b, xs, bs, w, None)


def structural_problem(m: int = 68, bs: int = 8, w: int = 32, seed: int = 7, rhs_seed: int = 0) -> Problem:
    """The irregular 3-DOF structural matrix on m^3 nodes (Audikw_1-shaped at
    m = 68: 943,296 unknowns, about 78M nonzeros), natural order, algebraic
    blocking, b = A x* with x* ~ U(-1, 1)."""
    A = irregular_structural(m, seed)
    b, xs = rhs_from_solution(A, rhs_seed)
    return Problem(f"structural_{m}^3x3_bs{bs}", A, b, xs, bs, w, None)


def curl_curl_problem(m: int, sigma: float = 0.01, seed: int = 6, hetero: float = 0.3, bs: int = 8,
                      w: int = 32, order_seed: int = 8, rhs_seed: int = 0) -> Problem:
    """curl_curl on an m^3 cell grid in a random input order (algebraic
    blocking); m = 70 gives 1,058,610 unknowns, about the size of the paper's IEEJ
    eddy-current system."""
    A = curl_curl(m, sigma, seed, hetero)
    A = permute_input(A, random_order(order_seed, A.n))
    b, xs = rhs_from_solution(A, rhs_seed)
    return Problem(f"curlcurl_{m}^3_bs{bs}", A, b, xs, bs, w, None)


def convection_diffusion_problem(m: int, bs: int = 8, w: int = 32, velocity=(0.5, 0.3, 0.2),
                                 seed: int = 0) -> Problem:
    """Nonsymmetric convection-diffusion on m^3, geometric bs-cubes, b = A x*."""
    A = convection_diffusion(m, velocity)
    b, xs = rhs_from_solution(A, seed)
    return Problem(f"convdiff_{m}^3_bs{bs}", A, b, xs, bs, w, box_for_bs(bs))


def batch_problems(nsys: int = 256, seed0: int = 1000, nmin: int = 16, nmax: int = 64):
    """Uneven batch of SPD systems: system s (stream seed0 + s) draws a stencil
    in {7, 27} with probability 1/2 each, an edge m ~ U{nmin..nmax} and sigma ~
    U[0, 2]; its coefficients are smoothed lognormal (kappa stream
    2*(seed0+s)+1), natural lexicographic order, b = A x* with x* ~ U(-1, 1)
    (stream 2*(seed0+s)+2).  Returns a list of (A, b, x*)."""
    out = []
    for s in range(nsys):
        seed = seed0 + s
        u = uniform(seed, 3)
        points = 7 if u[0] < 0.5 else 27
        m = nmin + min(int(u[1] * (nmax - nmin + 1)), nmax - nmin)
        sigma = 2.0 * u[2]
        A = heterogeneous_stencil(m, points, sigma, 2 * seed + 1)
        b, xs = rhs_from_solution(A, 2 * seed + 2)
        out.append((A, b, xs))
    return out
