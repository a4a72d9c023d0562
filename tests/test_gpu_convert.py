"""The FP32 substitutions convert between binary64 and binary32 with integer
operations (widen_f32 / narrow_f64 in csrc/device_util.cuh) instead of
conversion instructions, which issue on this GPU's slow FP64 pipe.  Their
results must equal the casts bit for bit: widening exactly, narrowing to
nearest with ties to even.  Checked through the C ABI (hbmc_debug_convert)
against torch's casts on the same device, over random bit patterns across
the whole exponent range, exact halfway cases, the float subnormal range and
the boundaries (largest float, overflow, smallest normal and subnormal)."""
import numpy as np
import pytest
import torch

from paper_1908_00741_gb300 import hbmc as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00741_gb300 import _build
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return H.load()


def _doubles(rng, count):
    """Bit patterns of doubles: random exponents around the float range,
    ties (29 dropped bits exactly one half), float-subnormal results and
    edge values; no NaN."""
    u64 = np.uint64
    sign = rng.integers(0, 2, count, dtype=np.uint64) << u64(63)
    mant = rng.integers(0, 2 ** 52, count, dtype=np.uint64)
    wide = sign | mant | (rng.integers(1, 2047, count // 4, dtype=np.uint64).repeat(4)[:count] << u64(52))
    near = sign | mant | (rng.integers(820, 1160, count, dtype=np.uint64) << u64(52))
    ties = sign | (rng.integers(0, 2 ** 23, count, dtype=np.uint64) << u64(29)) | u64(0x10000000) | \
        (rng.integers(860, 1152, count, dtype=np.uint64) << u64(52))
    sub = sign | mant | (rng.integers(860, 898, count, dtype=np.uint64) << u64(52))
    edges = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 3.4028234663852886e38, 3.4028235677973366e38,
                      -3.4028235677973366e38, 3.4028236e38, 2.0 ** 128, 2.0 ** -126, 2.0 ** -149, 2.0 ** -150,
                      1.5 * 2.0 ** -150, 2.0 ** -151, 2.0 ** -1070, 5e-324, 1e300, -1e-300,
                      1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52])
    bits = np.concatenate([wide, near, ties, sub, edges.view(np.uint64)])
    return bits.view(np.float64)


def _floats(rng, count):
    bits = rng.integers(0, 2 ** 32, count, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0, 0x80000000, 1, 0x80000001, 0x007fffff, 0x00800000, 0x7f7fffff, 0x7f800000, 0xff800000,
                      0x00400000, 0x3f800000], dtype=np.uint32)
    bits = np.concatenate([bits, rng.integers(1, 2 ** 23, count // 4, dtype=np.uint64).astype(np.uint32), extra])
    f = bits.view(np.float32)
    return f[~np.isnan(f)]


@pytest.mark.parametrize("seed", [0, 1])
def test_integer_conversions_equal_the_casts(lib, seed):
    rng = np.random.default_rng(seed)
    d = _doubles(rng, 100000)
    f = _floats(rng, len(d))
    n = min(len(d), len(f))
    d_dev = torch.tensor(d[:n], device="cuda")
    f_dev = torch.tensor(f[:n], device="cuda")
    narrowed, widened = H.hbmc_debug_convert(d_dev, f_dev)
    torch.cuda.synchronize()
    ref_n = d_dev.to(torch.float32)
    ref_w = f_dev.to(torch.float64)
    assert torch.equal(narrowed.view(torch.int32), ref_n.view(torch.int32))
    assert torch.equal(widened.view(torch.int64), ref_w.view(torch.int64))


def test_convert_hook_rejects_bad_arguments(lib):
    assert lib.hbmc_debug_convert(None, None, None, None, -1, None) == H.ERR_INVALID_ARG
    assert lib.hbmc_debug_convert(None, None, None, None, 5, None) == H.ERR_INVALID_ARG
    assert lib.hbmc_debug_convert(None, None, None, None, 0, None) == H.OK
