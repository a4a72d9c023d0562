"""Algorithmic bytes behind the bench's roofline fractions, no GPU needed.

Compulsory traffic of one substitution (Section 4.2.2's Eqs. "y2-2" /
"y2-3"): every stored coefficient of L once with its int32 column, dinv, the
input vector and the result; the backward sweep also reads r for the fused
r.z.  SpMV: every nonzero of A with its column, p in and q out.  The
expected figures are worked out by hand from the stencils' closed-form
nonzero counts (7-point m^3 grid: 7m^3 - 6m^2; 27-point: (3m - 2)^3; 3-DOF
vector Laplacian on a 7-point node stencil: 9 (7m^3 - 6m^2)) and rounded to
0.1 MB."""
import pytest

import bench

MB = 1e6

CONFIGS = {
    # name: (n, nnz)
    "poisson7_128": (128 ** 3, 7 * 128 ** 3 - 6 * 128 ** 2),
    "stencil27_96": (96 ** 3, (3 * 96 - 2) ** 3),
    "veclap_100": (3 * 100 ** 3, 9 * (7 * 100 ** 3 - 6 * 100 ** 2)),
}


@pytest.mark.parametrize("name,s,fwd_mb", [
    ("poisson7_128", 8, 125.2), ("poisson7_128", 4, 83.5),
    ("stencil27_96", 8, 156.3), ("stencil27_96", 4, 104.2),
    ("veclap_100", 8, 428.8), ("veclap_100", 4, 285.8),
])
def test_forward_substitution_bytes(name, s, fwd_mb):
    n, nnz = CONFIGS[name]
    fwd, bwd = bench.subst_bytes(n, (nnz - n) // 2, s)
    assert round(fwd / MB, 1) == fwd_mb
    # the backward sweep reads y (s bytes) and writes z in FP64 where the
    # forward reads r in FP64 and writes y: the same, plus r for the fused r.z
    assert bwd - fwd == n * 8


def test_poisson128_iteration_bytes():
    """One FP64 CG iteration at 128^3: both substitutions, SpMV and the nine
    vector passes of the updates come to about 627 MB (78 us at 8 TB/s)."""
    n, nnz = CONFIGS["poisson7_128"]
    fwd, bwd = bench.subst_bytes(n, (nnz - n) // 2, 8)
    spmv = bench.spmv_bytes(n, nnz)
    assert round(spmv / MB, 1) == 208.5
    total = fwd + bwd + spmv + 9 * n * 8
    assert round(total / MB) == 627
    assert round(total / (bench.HBM_NOMINAL_GBS * 1e9) * 1e6) == 78


def test_fractions():
    f = bench.fracs(4000.0, 5000.0)
    assert f == {"frac": 0.8, "frac_nominal": 0.5}


def test_clock_summary_from_sampled_lines():
    """The clocks key: median SM clock under load, the highest max clock, and
    every throttle reason seen active in any sample."""
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    assert cs.summary() == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.lines.append("0, 1200, 2070, 700.0, 0x48, Active, Not Active, Active, Not Active")
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                               "samples": 0}


def test_spmv_traffic_record_matches_the_kernel_source():
    """The ncu traffic the bench reports belongs to the SpMV kernel as it is
    now: the committed record names the sha1 of its source, and a changed
    source turns the figure into null."""
    t = bench.measured_traffic()
    assert t is not None and t > 0
    n, nnz = CONFIGS["poisson7_128"]
    assert 1.0 <= t / bench.spmv_bytes(n, nnz) < 1.1
