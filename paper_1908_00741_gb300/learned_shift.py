"""Learned IC(0) shift: data from shift sweeps, training and use.

Orchestration only: the sweeps are batched HBMC-ICCG solves, the features
come from the library's feature kernel, and training is the library's
forward/backward/Adam kernels (hbmc_mlp_train).  The network predicts,
from [features, shift code], log2 of the CG iterations at that shift over
the system's least over the grid; the shift it recommends is the grid shift
with the lowest prediction.  The plain positive-pivot rule
(hbmc_ic0_auto without a network) remains the fallback when the predicted
shift's factorization fails, and the yardstick the learned choice is
measured against.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import hbmc as H

FAIL_FACTOR = 4.0  # a failed shift (pivot or no convergence) counts as 4 * maxit iterations


@dataclasses.dataclass
class Sweep:
    features: np.ndarray   # [nsys, 12]
    iters: np.ndarray      # [nsys, grid]; -1 = IC(0) failed or CG did not converge
    ic_ok: np.ndarray      # [nsys, grid]; IC(0) had only positive, finite pivots
    true_relres: np.ndarray
    maxit: int

    def cost(self, s, c):
        """CG iterations of system s at grid shift c; a shift whose IC(0) or CG
        failed costs FAIL_FACTOR * maxit."""
        it = self.iters[s, c]
        return int(it) if it >= 0 else int(FAIL_FACTOR * self.maxit)


def sweep(mats, bvecs, bs=8, tol=1e-8, maxit=2000, precision=H.PREC_F32, use_boxes=False) -> Sweep:
    """Iterations of every system at every grid shift (one batched solve per shift)."""
    import torch
    grid = H.shift_grid()
    batch = H.hbmc_batch_build(mats, bs, use_boxes=use_boxes, precision=precision)
    feats = H.hbmc_batch_features(batch)
    b = torch.tensor(np.concatenate(bvecs), device="cuda")
    x = torch.zeros_like(b)
    iters = np.full((len(mats), len(grid)), -1, dtype=np.int64)
    ic_ok = np.zeros((len(mats), len(grid)), dtype=bool)
    tr = np.full((len(mats), len(grid)), np.nan)
    for c, a in enumerate(grid):
        st, bad = H.hbmc_batch_ic0(batch, shifts=np.full(len(mats), a))
        x.zero_()
        res = H.hbmc_batch_iccg(batch, b, x, tol=tol, maxit=maxit)
        ic_ok[:, c] = bad == -1
        ok = ic_ok[:, c] & (res.statuses == H.OK)
        iters[ok, c] = res.iters[ok]
        tr[ok, c] = res.true_relres[ok]
    batch.close()
    return Sweep(feats, iters, ic_ok, tr, maxit)


def plain_choice(ic_row):
    """Index of the plain rule's shift: the first grid shift whose IC(0) has
    only positive, finite pivots (whatever CG then does with it), -1 if none."""
    ok = np.flatnonzero(ic_row)
    return int(ok[0]) if len(ok) else -1


def fallback_choice(ic_row, c, plain):
    """The shift actually used when the network chooses grid index c: c if
    its IC(0) works, else the first larger grid shift whose IC(0) works (as
    hbmc_ic0_auto continues), else the plain rule's index.  Returns (index,
    whether the fallback was taken)."""
    if ic_row[c]:
        return int(c), False
    nxt = np.flatnonzero(ic_row[c + 1:])
    return (int(c + 1 + nxt[0]) if len(nxt) else int(plain)), True


def best_choice(sw: Sweep, s):
    """argmin of the cost over the shifts whose IC(0) works, ties to the
    smaller shift; -1 if none works."""
    ok = np.flatnonzero(sw.ic_ok[s])
    if not len(ok):
        return -1
    return int(ok[np.argmin([sw.cost(s, c) for c in ok])])


def dataset(sw: Sweep):
    """Inputs [features, shift code] and targets for every (system, shift)
    pair of systems with at least one converged shift: log2 of the shift's
    cost over the system's least cost among the shifts whose IC(0) works.
    The choice only needs the shape of each system's cost curve; a target
    relative to its minimum spares the network from predicting the absolute
    iteration count, which the features capture poorly (measured on 40
    validation systems of the learned family over three seeds: gains of 3.7
    to 5.2% over the plain rule with this target, 0 to 5.1% with log2 of the
    iterations themselves)."""
    g = sw.iters.shape[1]
    keep = (sw.iters >= 0).any(axis=1)
    X, T = [], []
    for s in np.flatnonzero(keep):
        costs = np.array([sw.cost(s, c) for c in range(g)], dtype=np.float64)
        ok = sw.ic_ok[s]
        least = costs[ok].min() if ok.any() else costs.min()
        for c in range(g):
            X.append(np.concatenate([sw.features[s], [c / (g - 1)]]))
            T.append(np.log2(costs[c] / least))
    return np.asarray(X, np.float32), np.asarray(T, np.float32)


def init_params(D, seed=0):
    """Glorot-uniform weights, zero biases (numpy, seeded)."""
    rng = np.random.default_rng(seed)
    h = 32

    def glorot(fan_out, fan_in):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    return np.concatenate([glorot(h, D).ravel(), np.zeros(h), glorot(h, h).ravel(), np.zeros(h),
                           glorot(1, h).ravel(), [0.0]]).astype(np.float32)


# Features the network does not see: log10 n (0) and the color count (9)
# describe the system's size and ordering, not what the shift acts on, and a
# network trained on small systems extrapolates them badly (measured: on the
# 96^3 27-point and 70^3 curl-curl systems, with them, it chose 2.048 and
# lost 70% and 34% against the plain rule).  They are masked by standardizing
# them to 0 whatever their value.
MASKED_FEATURES = (0, 9)
MASK_STD = 1e30


def train(X, T, steps=3000, lr=3e-3, seed=0) -> H.Mlp:
    """Network trained on the GPU by the library's kernels."""
    import torch
    D = X.shape[1]
    net = H.Mlp(D)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std = np.where(std > 1e-6, std, 1.0).astype(np.float32)
    for f in MASKED_FEATURES:
        mean[f] = 0.0
        std[f] = MASK_STD
    net.set_params(init_params(D, seed), mean, std)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    net.train(Xd, Td, steps, lr)
    return net


def predicted_choice(net: H.Mlp, feats):
    """Grid index with the lowest predicted iterations, per system."""
    import torch
    g = H.SHIFT_GRID
    X = np.concatenate([np.repeat(feats, g, axis=0),
                        np.tile(np.arange(g) / (g - 1), len(feats))[:, None]], axis=1).astype(np.float32)
    out = net.forward(torch.tensor(X, device="cuda")).cpu().numpy().reshape(len(feats), g)
    return np.argmin(out, axis=1), out


def evaluate(net: H.Mlp, sw: Sweep):
    """Per system whose IC(0) works at some grid shift: the cost (CG
    iterations) with the plain rule, with the learned choice (when its IC(0)
    fails, the plain rule continues from the next larger grid shift, as
    hbmc_ic0_auto does) and with the best grid shift, and whether the
    fallback was taken."""
    choice, _ = predicted_choice(net, sw.features)
    plain, learned, best, fallback = [], [], [], []
    for s in range(len(sw.iters)):
        pc = plain_choice(sw.ic_ok[s])
        if pc < 0:
            continue
        lc, fb = fallback_choice(sw.ic_ok[s], int(choice[s]), pc)
        plain.append(sw.cost(s, pc))
        learned.append(sw.cost(s, lc))
        best.append(sw.cost(s, best_choice(sw, s)))
        fallback.append(fb)
    return np.array(plain), np.array(learned), np.array(best), np.array(fallback)
