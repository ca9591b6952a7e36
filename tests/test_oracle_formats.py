"""Pins for the oracle's rounding (Section 4 rounding model, Table 1) and its Philox generator.

Every expected value here comes from something other than the oracle's own formula:
the numbers printed in Table 1 (tests/golden/table1.txt), the bit layouts of the formats
enumerated exhaustively, numpy's float16/float32 conversions (library routines that round
once from fp64), and numpy's Philox4x64-10 bit generator."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")
PARAMS = {O.FP16: (11, -14, 15), O.BF16: (8, -126, 127), O.TF32: (11, -126, 127), O.FP32: (24, -126, 127),
          O.Q52: (3, -14, 15)}


def _table1():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, u, xmin, xmax, t, emin, emax = line.split()
        rows[name] = dict(u=float(u), xmin=float(xmin), xmax=float(xmax), t=int(t), emin=int(emin), emax=int(emax))
    return rows


def _sig3(x):
    return float(f"{x:.2e}")


@pytest.mark.parametrize("name,fmt", [("bf16", O.BF16), ("fp16", O.FP16), ("fp32", O.FP32), ("q52", O.Q52)])
def test_table1_constants(name, fmt):
    """u = 2^-t, x_min = 2^e_min and x_max = 2^e_max (2 - 2^(1-t)) reproduce Table 1."""
    row = _table1()[name]
    t, emin, emax = PARAMS[fmt]
    assert (emin, emax) == (row["emin"], row["emax"])
    if name != "q52":
        assert t == row["t"]
    assert _sig3(2.0 ** -t) == row["u"]
    assert _sig3(2.0 ** emin) == row["xmin"]
    xmax = 2.0 ** emax * (2 - 2.0 ** (1 - t))
    assert _sig3(xmax) == row["xmax"]
    # the rounding keeps x_min and x_max, and |fl(x) - x| <= u |x| on normal numbers
    assert O.chop(np.array([2.0 ** emin, xmax]), fmt).tolist() == [2.0 ** emin, xmax]
    x = np.random.default_rng(1).uniform(1.0, 2.0, 10000) * 2.0 ** np.random.default_rng(2).integers(emin, emax, 10000)
    y = O.chop(x, fmt)
    assert np.all(np.abs(y - x) <= 2.0 ** -t * np.abs(x))


def _rand_doubles(n, rng, lo=-40, hi=40):
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return mant * 2.0 ** rng.integers(lo, hi, n).astype(np.float64)


def test_fp16_matches_numpy_float16():
    """numpy converts fp64 -> float16 with one round-to-nearest-even (library routine)."""
    rng = np.random.default_rng(3)
    x = np.concatenate([_rand_doubles(400000, rng, -30, 18), rng.standard_normal(100000) * 1e-6,
                        [65504.0, 65519.99, 65520.0, 65536.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, -0.0]])
    ref = x.astype(np.float16).astype(np.float64)
    got = O.chop(x, O.FP16)
    assert np.array_equal(np.isinf(ref), np.isinf(got))
    fin = np.isfinite(ref)
    assert np.array_equal(ref[fin], got[fin])


def test_fp32_matches_numpy_float32():
    rng = np.random.default_rng(4)
    x = np.concatenate([_rand_doubles(400000, rng, -160, 130), [3.4028235677973366e38, 3.4028235e38 * 1.0000001,
                                                                 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151]])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    got = O.chop(x, O.FP32)
    assert np.array_equal(np.isinf(ref), np.isinf(got))
    fin = np.isfinite(ref)
    assert np.array_equal(ref[fin], got[fin])


def _enumerate(fmt):
    """All finite non-negative values of a format from its bit layout, ascending."""
    if fmt == O.FP16:
        bits = np.arange(0, 0x7C00, dtype=np.uint16)
        return bits.view(np.float16).astype(np.float64), bits.astype(np.int64)
    if fmt == O.Q52:  # E5M2 is the high byte of an fp16 pattern
        b8 = np.arange(0, 0x7C, dtype=np.uint16)
        return (b8 << 8).view(np.float16).astype(np.float64), b8.astype(np.int64)
    if fmt == O.BF16:  # bf16 is the high half of an fp32 pattern
        b16 = np.arange(0, 0x7F80, dtype=np.uint32)
        return (b16 << 16).view(np.float32).astype(np.float64), b16.astype(np.int64)
    if fmt == O.TF32:  # tf32 keeps 10 fraction bits: fp32 patterns with the low 13 bits clear
        b19 = np.arange(0, 0x7F80 << 3, dtype=np.uint32)
        return (b19 << 13).view(np.float32).astype(np.float64), b19.astype(np.int64)
    raise ValueError(fmt)


@pytest.mark.parametrize("fmt", [O.FP16, O.Q52, O.BF16, O.TF32])
def test_exhaustive_roundtrip_and_midpoints(fmt):
    """Every representable value is kept; every midpoint between neighbours rounds to the
    neighbour with the even bit pattern; points just off a midpoint round to the nearer one;
    one half-ulp above x_max overflows to infinity."""
    v, bits = _enumerate(fmt)
    for sign in (1.0, -1.0):
        assert np.array_equal(O.chop(sign * v, fmt), sign * v)
        lo, hi = v[:-1], v[1:]
        mid = 0.5 * (lo + hi)  # exact in fp64
        even = np.where(bits[:-1] % 2 == 0, lo, hi)
        assert np.array_equal(O.chop(sign * mid, fmt), sign * even)
        gap = hi - lo
        assert np.array_equal(O.chop(sign * (mid - gap / 64), fmt), sign * lo)
        assert np.array_equal(O.chop(sign * (mid + gap / 64), fmt), sign * hi)
    t, emin, emax = PARAMS[fmt]
    xmax = v[-1]
    ulp = 2.0 ** (emax - t + 1)
    assert xmax == 2.0 ** emax * (2 - 2.0 ** (1 - t))
    assert O.chop(np.array([xmax + ulp / 2]), fmt)[0] == math.inf
    assert O.chop(np.array([-(xmax + ulp / 2)]), fmt)[0] == -math.inf
    assert O.chop(np.array([xmax + ulp / 2 - ulp / 64]), fmt)[0] == xmax


def test_special_values_pass_through():
    x = np.array([0.0, -0.0, math.inf, -math.inf, math.nan])
    for fmt in range(8):
        y = O.chop(x, fmt)
        assert y[0] == 0 and y[1] == 0 and math.copysign(1, y[1]) == -1
        assert y[2] == math.inf and y[3] == -math.inf and math.isnan(y[4])


def test_fp64_identity():
    x = _rand_doubles(1000, np.random.default_rng(5), -1000, 1000)
    assert np.array_equal(O.chop(x, O.FP64), x)


def test_chop_is_single_rounding_from_fp64():
    """A value just above a bf16 midpoint that is itself rounded onto the midpoint by an fp32
    conversion must still round up: the oracle rounds once from fp64, never through fp32."""
    lo = 1.0
    hi = 1.0 + 2.0 ** -7
    x = 0.5 * (lo + hi) + 2.0 ** -40  # fp32 rounding would land exactly on the midpoint
    assert float(np.float32(x)) == 0.5 * (lo + hi)
    assert O.chop(np.array([x]), O.BF16)[0] == hi


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_philox_matches_numpy(seed):
    """numpy.random.Philox is Philox4x64-10; it pre-increments its 256-bit counter."""
    rng = np.random.default_rng(seed)
    for _ in range(20):
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        c = rng.integers(1, 2 ** 63, 4, dtype=np.uint64)
        bg = np.random.Philox(key=int(key[0]) | (int(key[1]) << 64),
                              counter=[int(c[0]) - 1, int(c[1]), int(c[2]), int(c[3])])
        ref = bg.random_raw(4)
        got = O.philox4x64(c, key)
        assert np.array_equal(ref, got)


def test_exploration_draw_statistics():
    """u is uniform on [0,1) and the random action is uniform over |P| = 5 (chi-square)."""
    us, picks = [], []
    for k in range(4000):
        u, p = O.draw(7, 3, 1, k, k % 4)
        us.append(u)
        picks.append(p % 5)
    us = np.array(us)
    assert np.all((us >= 0) & (us < 1))
    assert abs(np.mean(us < 0.3) - 0.3) < 0.03
    cnt = np.bincount(picks, minlength=5)
    chi2 = np.sum((cnt - 800) ** 2 / 800)
    assert chi2 < 20.5  # p ~ 0.0004 for 4 degrees of freedom
