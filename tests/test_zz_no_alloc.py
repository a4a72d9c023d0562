"""hbmc_spmv_dot_static: the SpMV with fused p.q for callers that cannot
allocate device memory (a device whose memory another allocator owns, loops
that must not allocate after start-up).  Its scratch is a static
array inside the library; these tests check it against the solver's own
SpMV entry point, twice in a row (the array is reused and must be cleared
between calls), and that oversized systems are refused.

This file is named so that pytest collects it last."""
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


CASES = [
    ("poisson7_16_bs8", lambda: W.poisson7(16), 8, (2, 2, 2)),
    ("poisson7_13_ragged_bs16", lambda: W.poisson7(13), 16, (2, 2, 4)),
    ("hetero27_9_rand_bs8", lambda: W.permute_input(W.heterogeneous_stencil(9, 27, 2.0, 1),
                                                    W.random_order(2, 729)), 8, None),
]


@pytest.mark.parametrize("name,mk,bs,box", CASES)
def test_static_scratch_spmv_matches_spmv_bar(lib, name, mk, bs, box):
    A = mk()
    ctx = H.hbmc_build(A, bs, 32, box=box)
    n_pad = ctx.info()["n_pad"]
    for call in range(2):
        p = torch.tensor(np.random.default_rng(call).standard_normal(n_pad), device="cuda")
        q_ref = torch.empty_like(p)
        H.hbmc_spmv_bar(ctx, p, q_ref)
        q = torch.full_like(p, float("nan"))
        pq = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        H.hbmc_spmv_dot_static(ctx, p, q, pq)
        torch.cuda.synchronize()
        # same entries, same order, same fused multiply-adds: same bits
        assert torch.equal(q, q_ref)
        # the dot is reduced in a different order than a host sum: 1e-12 relative
        ref = float(np.dot(p.cpu().numpy(), q_ref.cpu().numpy()))
        assert abs(pq.item() - ref) <= 1e-12 * abs(ref)


def test_static_scratch_empty_system_sets_pq_to_zero(lib):
    A = W.CSR(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    ctx = H.hbmc_build(A, 8, 32)
    p = torch.zeros(0, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(p)
    pq = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    H.hbmc_spmv_dot_static(ctx, p, q, pq)
    torch.cuda.synchronize()
    assert pq.item() == 0.0


def test_static_scratch_refuses_oversized_systems(lib):
    A = W.poisson7(104)  # bs = 1: 1,124,864 rows = 35,152 level-1 blocks > 32,768
    ctx = H.hbmc_build(A, 1, 32)
    n_pad = ctx.info()["n_pad"]
    p = torch.zeros(n_pad, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(p)
    pq = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HbmcError) as e:
        H.hbmc_spmv_dot_static(ctx, p, q, pq)
    assert e.value.status == H.ERR_INVALID_ARG and "static scratch limit" in str(e.value)
