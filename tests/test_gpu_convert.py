"""The fixed-point outer loop's conversions (binary64 / binary32 to and from
64-bit integers, round to nearest with ties to even) are computed in integer
arithmetic; they must give the correctly rounded IEEE 754 result, i.e. the
same bits as the hardware conversions torch uses, on every input of their
range: ties, the edges of the significand, subnormals, saturation."""
import numpy as np
import pytest
import torch

import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(20230227)


def doubles(n, lo_exp, hi_exp):
    """Random doubles with uniformly spread exponents and random significands."""
    e = RNG.integers(lo_exp, hi_exp, n)
    m = RNG.random(n) + 1.0
    s = RNG.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def ties(n, scale_exp):
    """Values exactly halfway between two integers (or two representable
    values after a scale by 2^scale_exp)."""
    k = RNG.integers(-2**40, 2**40, n).astype(np.float64)
    return np.ldexp(k + 0.5, scale_exp)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    if a.dtype == torch.float64:
        return torch.equal(a.view(torch.int64), b.view(torch.int64))
    if a.dtype == torch.float32:
        return torch.equal(a.view(torch.int32), b.view(torch.int32))
    return torch.equal(a, b)


def first_mismatch(a, b, x):
    bad = (a != b).nonzero()
    k = int(bad[0]) if len(bad) else 0
    return f"input {x.flatten()[k].item()!r}: got {a.flatten()[k].item()!r}, want {b.flatten()[k].item()!r}"


def test_double_to_int64():
    x = np.concatenate([
        doubles(200000, -1080, 62), ties(20000, 0), ties(5000, -3),
        np.array([0.0, -0.0, 0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 2.0**52 + 0.5, 2.0**52 - 0.5,
                  2.0**53, 2.0**62, -2.0**62, -(2.0**63), 5e-324, -5e-324, 2.0**-1022,
                  0.49999999999999994, 4503599627370495.5]),
    ])
    xd = cuda(x)
    got = mg.op_convert(0, xd)
    want = torch.round(xd).to(torch.int64)
    assert same_bits(got, want), first_mismatch(got, want, xd)
    big = mg.op_convert(0, cuda(np.array([1e19, -1e19, np.inf, -np.inf, 2.0**63])))
    assert big.tolist() == [2**63 - 1, -2**63, 2**63 - 1, -2**63, 2**63 - 1]


def test_int64_to_double():
    r = RNG.integers(-2**63, 2**63 - 1, 200000, dtype=np.int64, endpoint=True)
    shifts = RNG.integers(0, 63, r.size)
    x = np.concatenate([
        r >> shifts,  # every magnitude
        np.array([0, 1, -1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 2, 2**53 + 3, 2**54 + 2,
                  2**54 + 6, -(2**53 + 1), 2**63 - 1, -2**63, -2**63 + 1, 2**62 + 2**9,
                  2**62 + 2**10, 2**62 + 3 * 2**9], dtype=np.int64),
    ])
    xd = cuda(x)
    got = mg.op_convert(1, xd)
    want = xd.to(torch.float64)
    assert same_bits(got, want), first_mismatch(got, want, xd)


def test_double_to_float():
    f32_ties = np.ldexp(RNG.integers(2**23, 2**24, 20000).astype(np.float64) + 0.5,
                        RNG.integers(-140, 100, 20000))  # halfway between binary32 neighbours
    sub_ties = np.ldexp(RNG.integers(0, 2**23, 5000).astype(np.float64) + 0.5, -149)
    x = np.concatenate([
        doubles(200000, -160, 129), doubles(20000, -1074, -140), f32_ties, sub_ties,
        np.array([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                  3.402823669209385e38, 1e39, -1e39, np.inf, -np.inf, 1.1754943508222875e-38,
                  1.1754942807573643e-38, 1.401298464324817e-45, 7.006492321624085e-46,
                  7.006492321624087e-46, 2.1019476964872256e-45, 5e-324, 1e-300]),
    ])
    xd = cuda(x)
    got = mg.op_convert(2, xd)
    want = xd.to(torch.float32)
    assert same_bits(got, want), first_mismatch(got, want, xd)


def test_float_to_int64():
    x = np.concatenate([
        doubles(200000, -150, 63), ties(20000, 0) / 2**20, np.ldexp(RNG.integers(
            -2**22, 2**22, 5000).astype(np.float64) + 0.5, 0),
        np.array([0.0, -0.0, 0.5, -0.5, 1.5, 2.5, -2.5, 8388607.5, 8388608.0, 2.0**62, -(2.0**63),
                  1e-45]),
    ]).astype(np.float32)
    xd = cuda(x)
    got = mg.op_convert(3, xd)
    want = torch.round(xd).to(torch.int64)
    assert same_bits(got, want), first_mismatch(got, want, xd)
    big = mg.op_convert(3, cuda(np.array([1e19, -1e19, 2.0**63], dtype=np.float32)))
    assert big.tolist() == [2**63 - 1, -2**63, 2**63 - 1]


def test_int64_to_float():
    r = RNG.integers(-2**63, 2**63 - 1, 200000, dtype=np.int64, endpoint=True)
    shifts = RNG.integers(0, 63, r.size)
    x = np.concatenate([
        r >> shifts,
        np.array([0, 1, -1, 2**24 - 1, 2**24, 2**24 + 1, 2**24 + 2, 2**24 + 3, 2**25 + 2, 2**25 + 6,
                  -(2**24 + 1), 2**63 - 1, -2**63, 2**40 + 2**16, 2**40 + 2**17, 2**40 + 3 * 2**16,
                  2**40 + 2**16 + 1], dtype=np.int64),
    ])
    xd = cuda(x)
    got = mg.op_convert(4, xd)
    want = xd.to(torch.float32)
    assert same_bits(got, want), first_mismatch(got, want, xd)
