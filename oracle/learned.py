"""Plain FP64 reference for the learned-shift part (numpy).

TEST INFRASTRUCTURE ONLY: the tests use it to check the library's feature
kernel, MLP forward/backward kernels and shift rules; the library never calls
it.

- features(A, nc, bs): the 12 matrix features, from the CSR rows directly.
- the MLP D -> 32 -> 32 -> 1 with ReLU and standardized inputs: forward,
  loss L = mean (out - t)^2 and its exact gradient by backpropagation.
- plain_rule: the first shift of the grid (0, then 1e-3 * 2^k) whose IC(0)
  has only positive pivots (the oracle's own IC(0)).
"""
from __future__ import annotations

import numpy as np

H = 32
DOM_CAP = 10.0


def shift_grid(count=13):
    return np.array([0.0] + [1e-3 * 2.0 ** k for k in range(count - 1)])


def features(A, nc, bs):
    """Features 0..11 as defined for hbmc_features, over the rows of A."""
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    is_d = A.col == rows
    d = np.zeros(n)
    d[rows[is_d]] = A.val[is_d]
    nnz = np.diff(A.row_ptr).astype(np.float64)
    off = np.bincount(rows, weights=np.where(is_d, 0.0, np.abs(A.val)), minlength=n)
    npos = np.bincount(rows, weights=np.where(~is_d & (A.val > 0), 1.0, 0.0), minlength=n)
    dom = np.where(off > 0, np.minimum(d / np.where(off > 0, off, 1.0), DOM_CAP), DOM_CAP)
    lg = np.log(d)
    return np.array([
        np.log10(n), nnz.mean(), nnz.max(), dom.min(), dom.mean(), np.mean(dom < 1.0 - 1e-9),
        npos.sum() / max((nnz - 1).sum(), 1.0), lg.mean(), lg.std(), float(nc), float(bs), dom.max(),
    ])


def n_params(D):
    return H * D + 3 * H + H * H + 1


def unpack(p, D):
    o = 0
    W1 = p[o:o + H * D].reshape(H, D); o += H * D
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, mean, std, X):
    """Returns (out, cache) for inputs X [B, D]."""
    D = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), D)
    xn = (X - mean) / std
    z1 = xn @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    out = a2 @ w3 + b3
    return out, (xn, z1, a1, z2, a2)


def loss(p, mean, std, X, T):
    out, _ = forward(p, mean, std, X)
    return float(np.mean((out - T) ** 2))


def gradient(p, mean, std, X, T):
    """Exact gradient of the mean squared error with respect to p (same layout)."""
    D = X.shape[1]
    B = X.shape[0]
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), D)
    out, (xn, z1, a1, z2, a2) = forward(p, mean, std, X)
    dout = 2.0 * (out - T) / B
    g_w3 = a2.T @ dout
    g_b3 = dout.sum()
    dz2 = np.outer(dout, w3) * (z2 > 0)
    g_W2 = dz2.T @ a1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g_W1 = dz1.T @ xn
    g_b1 = dz1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def plain_rule(an, grid=None):
    """First grid shift whose IC(0) of the analysed matrix succeeds, or None."""
    import oracle
    for a in (shift_grid() if grid is None else grid):
        _, _, _, bad = oracle.factor(an, a)
        if bad < 0:
            return float(a)
    return None
