"""Pins for the oracle's number formats (Table 2) against library casts.

The oracle rounds by definition (RN-even to t significand bits within the
format's exponent range).  These tests compare it with independent
implementations: numpy's direct float64->float16/float32 casts and torch's
float32->bfloat16/float8_e4m3fn casts (single roundings only; torch's
float64->half goes through float32 and double-rounds, so it is not used).
"""
import numpy as np
import pytest


def test_unit_roundoffs_match_table2(orc):
    # Table 2 prints half 2^-11 ~ 4.9e-4, single 2^-24 ~ 6.0e-8, double 2^-53 ~ 1.1e-16
    assert orc.unit_roundoff("fp16") == 2.0 ** -11
    assert orc.unit_roundoff("fp32") == 2.0 ** -24
    assert orc.unit_roundoff("fp64") == 2.0 ** -53
    assert f"{orc.unit_roundoff('fp16'):.1e}" == "4.9e-04"
    assert f"{orc.unit_roundoff('fp32'):.1e}" == "6.0e-08"
    assert f"{orc.unit_roundoff('fp64'):.1e}" == "1.1e-16"
    # u_q = 1 means the element is dropped (Section 4)
    assert orc.unit_roundoff("drop") == 1.0
    assert orc.round_to([3.5, -1e-30], "drop").tolist() == [0.0, 0.0]
    assert [orc.fmt_bits(f) for f in ("fp64", "fp32", "fp16", "bf16", "e4m3", "drop")] == \
        [64, 32, 16, 16, 8, 0]


def _hard_doubles(rng, n, lo, hi):
    """Random doubles over [2^lo, 2^hi) in magnitude plus constructed near-ties."""
    e = rng.integers(lo, hi, size=n)
    m = rng.random(n) + 1.0
    x = np.ldexp(m, e) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return x


def test_fp16_exhaustive_fixed_points_and_midpoints(orc):
    h = np.arange(1 << 16, dtype=np.uint16).view(np.float16)
    h = h[np.isfinite(h)]
    x = h.astype(np.float64)
    assert np.array_equal(orc.round_to(x, "fp16"), x)  # representable values are fixed
    xs = np.sort(np.unique(x))
    mids = (xs[:-1] + xs[1:]) / 2.0  # exact in fp64: ties between neighbours
    ref = mids.astype(np.float16).astype(np.float64)
    assert np.array_equal(orc.round_to(mids, "fp16"), ref)
    # just above / below each tie
    up = np.nextafter(mids, np.inf)
    dn = np.nextafter(mids, -np.inf)
    assert np.array_equal(orc.round_to(up, "fp16"), up.astype(np.float16).astype(np.float64))
    assert np.array_equal(orc.round_to(dn, "fp16"), dn.astype(np.float16).astype(np.float64))


def test_fp16_random_doubles_vs_numpy(orc):
    rng = np.random.default_rng(1)
    x = _hard_doubles(rng, 1_000_000, -30, 17)  # subnormal, normal and overflow range
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(orc.round_to(x, "fp16"), ref)


def test_fp32_random_doubles_vs_numpy(orc):
    rng = np.random.default_rng(2)
    x = _hard_doubles(rng, 1_000_000, -155, 129)
    # constructed ties at fp32 precision, and ties plus/minus one fp64 ulp
    t = np.ldexp(rng.integers(1 << 23, 1 << 24, size=10000).astype(np.float64) + 0.5,
                 rng.integers(-100, 100, size=10000))
    x = np.concatenate([x, t, np.nextafter(t, np.inf), np.nextafter(t, -np.inf)])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(orc.round_to(x, "fp32"), ref)


def test_bf16_vs_torch_from_fp32(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    b = np.arange(1 << 16, dtype=np.uint32) << 16
    v = b.view(np.float32)
    v = v[np.isfinite(v)].astype(np.float64)
    vs = np.sort(np.unique(v))
    mids = (vs[:-1] + vs[1:]) / 2.0  # 9 significant bits: exact in fp32
    x32 = np.concatenate([
        _hard_doubles(rng, 500_000, -133, 127).astype(np.float32),
        mids.astype(np.float32), v.astype(np.float32)])
    x32 = x32[np.isfinite(x32)]
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    got = orc.round_to(x32.astype(np.float64), "bf16")
    assert np.array_equal(got, ref)


def test_e4m3_vs_torch_from_fp32_in_range(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    codes = np.arange(256, dtype=np.uint8)
    v = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    v = np.unique(v[np.isfinite(v)])
    mids = (v[:-1] + v[1:]) / 2.0
    x = np.concatenate([v, mids, np.nextafter(mids, np.inf), np.nextafter(mids, -np.inf),
                        rng.uniform(-448, 448, 200_000),
                        np.ldexp(rng.random(100_000) + 1, rng.integers(-12, 8, 100_000))])
    x32 = x.astype(np.float32)
    x32 = x32[np.abs(x32) <= 448]
    ref = torch.from_numpy(x32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = orc.round_to(x32.astype(np.float64), "e4m3")
    assert np.array_equal(got, ref)


def test_e4m3_saturates(orc):
    # OCP e4m3 "satfinite": magnitudes beyond 448 clamp to 448; 464 is the tie
    # between 448 (even significand) and 480 and rounds to 448.
    got = orc.round_to([464.0, 470.0, 1e6, -1e6, np.inf], "e4m3")
    assert got.tolist() == [448.0, 448.0, 448.0, -448.0, 448.0]
