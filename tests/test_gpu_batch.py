"""Batched solver (many independent SPD systems swept together) against the
oracle solving each system alone."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H
from paper_1908_00741_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return H.load()


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _small_batch(nsys=10, seed0=1000):
    return W.batch_problems(nsys, seed0=seed0, nmin=4, nmax=11)


def _concat(items):
    return np.concatenate([b for _, b, _ in items])


@pytest.mark.parametrize("bs", [4, 8, 16])
@pytest.mark.parametrize("w,vslice", [(32, 0), (16, 0), (32, 2), (16, 1)])
@pytest.mark.parametrize("loop_mode", [H.LOOP_GRAPH, H.LOOP_HOST])
def test_batch_fp64_matches_oracle_per_system(lib, orc, bs, w, vslice, loop_mode):
    """Every system of the batch, with w = 32 or 16 BMC blocks per level-1
    block (two level-1 blocks per warp at 16), with the SpMV's slices at
    height w or of variable height, takes its own oracle solve's iteration
    count and iterates."""
    items = _small_batch()
    mats = [A for A, _, _ in items]
    batch = H.hbmc_batch_build(mats, bs, w=w, vslice=vslice, loop_mode=loop_mode, check_every=3)
    st, bad = H.hbmc_batch_ic0(batch)
    assert st == H.OK and np.all(bad == -1)
    b = torch.tensor(_concat(items), device="cuda")
    x = torch.zeros_like(b)
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-8)
    assert res.status == H.OK and np.all(res.statuses == H.OK)
    xh = x.cpu().numpy()
    off = 0
    box = W.box_for_bs(bs)
    for k, (A, bk, _) in enumerate(items):
        ref, _ = orc.iccg(A, bk, bs, w, box=box, tol=1e-8)
        assert ref.status == 0
        assert res.iters[k] == ref.iters, (k, res.iters[k], ref.iters)
        assert _rel(xh[off:off + A.n], ref.x) <= 1e-12
        true = np.linalg.norm(bk - A.to_scipy() @ xh[off:off + A.n]) / np.linalg.norm(bk)
        assert abs(res.true_relres[k] - true) <= 1e-6 * true
        off += A.n
    assert np.all(res.solve_ms > 0)


@pytest.mark.parametrize("w", [32, 16])
def test_batch_fp32_reaches_fp64_tolerance(lib, orc, w):
    items = _small_batch(12, seed0=1100)
    mats = [A for A, _, _ in items]
    batch = H.hbmc_batch_build(mats, 8, w=w, precision=H.PREC_F32)
    assert H.hbmc_batch_ic0(batch)[0] == H.OK
    b = torch.tensor(_concat(items), device="cuda")
    x = torch.zeros_like(b)
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-8)
    assert res.status == H.OK
    assert np.all(res.true_relres < 3e-8)
    xh = x.cpu().numpy()
    off = 0
    for k, (A, bk, _) in enumerate(items):
        ref, _ = orc.iccg(A, bk, 8, w, box=(2, 2, 2), tol=1e-8)
        assert abs(int(res.iters[k]) - ref.iters) <= max(2, ref.iters // 10)
        assert _rel(xh[off:off + A.n], ref.x) < 1e-6
        off += A.n


def test_single_system_batch_matches_single_solver(lib, orc):
    P = W.poisson_problem(12, bs=8)
    batch = H.hbmc_batch_build([P.A], 8)
    H.hbmc_batch_ic0(batch)
    ctx = H.hbmc_build(P.A, 8, 32, box=P.box)
    H.hbmc_ic0(ctx)
    b = torch.tensor(P.b, device="cuda")
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    r1 = H.hbmc_batch_iccg(batch, b, x1)
    r2 = H.hbmc_iccg(ctx, b, x2)
    assert r1.iters[0] == r2.iters
    assert _rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-12


def test_batch_shifts_failures_and_edge_cases(lib, orc):
    items = _small_batch(5, seed0=1200)
    mats = [A for A, _, _ in items]
    # an indefinite 1D system with positive diagonal, natural order
    import scipy.sparse as sp
    n = 40
    M = sp.diags([np.full(n - 1, 0.9), np.ones(n), np.full(n - 1, 0.9)], [-1, 0, 1]).tocsr()
    M.sort_indices()
    bad_sys = W.CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.copy())
    mats.insert(2, bad_sys)
    bvecs = [b for _, b, _ in items]
    bvecs.insert(2, np.cos(np.arange(n)))
    bvecs[0] = np.zeros_like(bvecs[0])  # zero right-hand side: x = 0 at once
    batch = H.hbmc_batch_build(mats, 8)
    st, bad = H.hbmc_batch_ic0(batch, shifts=[0.0, 0.3, 0.0, 0.0, 0.1, 0.0])
    assert st == H.ERR_NOT_SPD_PIVOT
    assert bad[2] >= 0 and np.all(np.delete(bad, 2) == -1)
    an = orc.analyse(bad_sys, 8, 32)
    _, _, _, obad = orc.factor(an, 0.0)
    inv = np.full(an.n_pad, -1)
    inv[an.pi] = np.arange(n)
    assert bad[2] == inv[obad]
    b = torch.tensor(np.concatenate(bvecs), device="cuda")
    x = torch.ones_like(b)
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-9)
    assert res.statuses[2] == H.ERR_BREAKDOWN
    assert res.statuses[0] == H.OK and res.iters[0] == 0
    assert np.all(x[: mats[0].n].cpu().numpy() == 0)
    for k in (1, 3, 4, 5):
        assert res.statuses[k] == H.OK
    # shifted systems against the oracle with the same shift
    xh = x.cpu().numpy()
    offs = np.cumsum([0] + [A.n for A in mats])
    ref, _ = orc.iccg(mats[1], bvecs[1], 8, 32, box=(2, 2, 2), shift=0.3, tol=1e-9, x0=np.ones(mats[1].n))
    assert res.iters[1] == ref.iters and _rel(xh[offs[1]:offs[2]], ref.x) <= 1e-12
    # maxit
    x.zero_()
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-9, maxit=2)
    assert res.statuses[1] == H.NOT_CONVERGED and res.iters[1] == 2


def test_batch_autotune_and_cache(lib, tmp_path):
    items = _small_batch(8, seed0=1300)
    mats = [A for A, _, _ in items]
    b = torch.tensor(_concat(items), device="cuda")
    cache = str(tmp_path / "tune.txt")
    best, ms = H.hbmc_batch_autotune(mats, b, (4, 8, 16), cache_path=cache)
    assert best in (4, 8, 16) and np.all(ms > 0)
    assert ms[[4, 8, 16].index(best)] == ms.min()
    best2, ms2 = H.hbmc_batch_autotune(mats, b, (4, 8, 16), cache_path=cache)
    assert best2 == best and np.all(ms2 == -1)


def test_batch_full_size_sampled(lib, orc):
    """The 256-system batch at full size (n^3 with n in [16, 64], 7- or
    27-point, 23.35 M unknowns) in the benchmark's launch configuration
    (bs = 4, FP32 substitutions, FP64 CG): every system reaches the FP64
    tolerance; then the same batch in FP64 gives, on the six smallest
    systems, the oracle's iteration counts and x within 1e-12."""
    items = W.batch_problems(256)
    mats = [A for A, _, _ in items]
    b = torch.tensor(_concat(items), device="cuda")
    x = torch.zeros_like(b)
    batch = H.hbmc_batch_build(mats, 4, precision=H.PREC_F32)
    assert H.hbmc_batch_ic0(batch)[0] == H.OK
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-8)
    assert res.status == H.OK and np.all(res.statuses == H.OK)
    assert np.all(res.true_relres < 1.1e-8)
    del batch
    batch = H.hbmc_batch_build(mats, 4, precision=H.PREC_F64)
    assert H.hbmc_batch_ic0(batch)[0] == H.OK
    x.zero_()
    res = H.hbmc_batch_iccg(batch, b, x, tol=1e-8)
    assert res.status == H.OK and np.all(res.statuses == H.OK)
    xh = x.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([A.n for A in mats])])
    for k in np.argsort([A.n for A in mats], kind="stable")[:6]:
        A, bk, _ = items[k]
        ref, _ = orc.iccg(A, bk, 4, 32, box=W.box_for_bs(4), tol=1e-8)
        assert res.iters[k] == ref.iters, (k, res.iters[k], ref.iters)
        assert _rel(xh[offs[k]:offs[k] + A.n], ref.x) <= 1e-12


def test_batch_autotune_over_bs_and_w(lib, tmp_path):
    """The (bs, w) autotuner times every pair, picks the fastest, and a
    cached choice comes back without timing."""
    items = _small_batch(16, seed0=1300)
    mats = [A for A, _, _ in items]
    b = torch.tensor(_concat(items), device="cuda")
    cache = str(tmp_path / "tune.txt")
    bs, w, v, ms = H.hbmc_batch_autotune_w(mats, b, (4, 8), (16, 32), (0, 8), cache_path=cache)
    assert ms.shape == (2, 2, 2) and np.all(ms > 0)
    i, j, k = (4, 8).index(bs), (16, 32).index(w), (0, 8).index(v)
    assert ms[i, j, k] == ms.min()
    bs2, w2, v2, ms2 = H.hbmc_batch_autotune_w(mats, b, (4, 8), (16, 32), (0, 8), cache_path=cache)
    assert (bs2, w2, v2) == (bs, w, v) and np.all(ms2 == -1)
    # the chosen triple solves the batch
    batch = H.hbmc_batch_build(mats, bs, w=w, vslice=v, precision=H.PREC_F32)
    assert H.hbmc_batch_ic0(batch)[0] == H.OK
    x = torch.zeros_like(b)
    assert H.hbmc_batch_iccg(batch, b, x, tol=1e-8).status == H.OK
