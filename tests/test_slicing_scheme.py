"""CPU checks of the exact-splitting arithmetic used by the tensor-core FP64
products (Ozaki scheme): FP64 values cut into eight balanced 7-bit digits from
their bit patterns, level sums of digit products, and the integer combination of
the levels.  Written in plain Python integers from the scheme's definition (not
from the CUDA sources) so that a wrong bias, shift or level weight fails here:

  M_s = sign(x) trunc(|x| 2^(1078 - E_r)),  M_s = sum_s a_s 2^(49 - 7 s),
  |a_0| <= 128, a_s in [-64, 63]; the level sums T_d = sum_{s+t=d} sum_k a_s b_t
  stay below 2^22 in magnitude for K = 64, so FP32 accumulates them exactly.
"""
import math
import struct

import numpy as np

BIAS = 64 * sum(1 << (49 - 7 * s) for s in range(1, 8)) + (1 << 57)


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def exp_class(x):
    b = bits(x)
    E = (b >> 52) & 0x7FF
    if E:
        return E
    return 1 if (b & ((1 << 52) - 1)) else 0


def digits(x, Er):
    """Balanced digits of one value against the row's exponent class Er."""
    b = bits(x)
    E = (b >> 52) & 0x7FF
    mant = b & ((1 << 52) - 1)
    if E:
        mant |= 1 << 52
    sh = max(E, 1) - Er + 3
    M = mant << sh if sh >= 0 else mant >> -sh
    if b >> 63:
        M = -M
    v = M + BIAS
    d = [(v >> 49) - 256] + [((v >> (49 - 7 * s)) & 127) - 64 for s in range(1, 8)]
    return d, M


def test_digits_reconstruct_and_bounds():
    rng = np.random.default_rng(11)
    for _ in range(200):
        row = rng.standard_normal(64) * 10.0 ** rng.integers(-30, 30)
        row[rng.integers(0, 64)] *= 1e-12          # entries far below the row maximum
        Er = max(exp_class(float(x)) for x in row)
        for x in row:
            d, M = digits(float(x), Er)
            assert abs(d[0]) <= 128 and all(-64 <= a <= 63 for a in d[1:])
            assert sum(a << (49 - 7 * s) for s, a in enumerate(d)) == M
            # value represented: M 2^(Er - 1078); error below 2^(Er - 1078)
            rep = math.ldexp(M, Er - 1078)
            assert abs(rep - float(x)) <= math.ldexp(1.0, Er - 1078)
            if exp_class(float(x)) >= Er - 3:                 # within 2^3 of the maximum: exact
                assert rep == float(x)


def test_level_sums_fit_fp32_and_combine_exactly():
    rng = np.random.default_rng(12)
    for _ in range(20):
        X = rng.standard_normal(64)
        F = rng.standard_normal(64) * 2.0 ** -int(rng.integers(0, 20))
        Ex = max(exp_class(float(x)) for x in X)
        Ef = max(exp_class(float(f)) for f in F)
        dx = [digits(float(x), Ex)[0] for x in X]
        df = [digits(float(f), Ef)[0] for f in F]
        T = [0] * 8
        for k in range(64):
            for s in range(8):
                for t in range(8 - s):
                    T[s + t] += dx[k][s] * df[k][t]
        assert max(abs(v) for v in T) < 2 ** 22           # exact in FP32, magic conversion valid
        # the integer combination sum_d T_d 2^(42 - 7 d), last level truncated by 2^-7
        S = sum(T[d] << (42 - 7 * d) for d in range(7)) + (T[7] >> 7)
        assert abs(S) < 2 ** 63
        exact128 = sum(T[d] << (49 - 7 * d) for d in range(8))     # 2^7 times the exact sum
        assert 0 <= exact128 - 128 * S < 128                       # floor of the last level only
        # the product it stands for: sum_k x_k f_k up to the dropped levels d >= 8
        approx = math.ldexp(S, Ex + Ef - 2100)
        ref = math.fsum(float(x) * float(f) for x, f in zip(X, F))
        bound = 64 * 2.0 ** -55 * max(abs(X)) * max(abs(F)) + abs(ref) * 2.0 ** -52
        assert abs(approx - ref) <= 4 * bound
