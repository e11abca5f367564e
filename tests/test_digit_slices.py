"""The arithmetic the tensor-core FP64 residual relies on, checked on the CPU: every FP64
value of a row, scaled by the row's power of two and rounded to a 56-bit fixed-point
integer, is exactly the sum of eight balanced base-128 digits (the first in [-128, 128],
the others in [-64, 63]) times powers of 2^-7; every partial sum of digit-pair products
over K <= 256 terms and the pairs of a diagonal d <= 7 is an integer of magnitude below
2^24, so summing them in FP32 (the tensor memory's accumulator) in any order is exact;
and the diagonals recombined as two 64-bit integers and one FP64 rounding give the dot
product to FP64 working accuracy. The digits follow the definition written out in the
GPU kernel's header; nothing here calls the library.
"""
import numpy as np
import pytest

S, BITS = 8, 7


def balanced(q):
    """Balanced base-128 digits of the integer q, most significant first."""
    r, out = int(q), [0] * S
    for j in range(S - 1, 0, -1):
        d = ((r & 127) ^ 64) - 64
        out[j] = d
        r = (r - d) >> 7
    out[0] = r
    return out


def balanced_by_bias(q):
    """The same digits from the plain base-128 digits of q + 64 sum_{j >= 1} 2^(49 - 7 j)."""
    r = int(q) + 64 * sum(1 << (49 - BITS * j) for j in range(1, S))
    return [r >> 49] + [((r >> (49 - BITS * j)) & 127) - 64 for j in range(1, S)]


def row_digits(x):
    """Digits [S][len(x)] and the row exponent e of x (|x| < 2^e)."""
    mx = np.max(np.abs(x))
    e = int(np.frexp(mx)[1]) if mx > 0 else 0
    q = [int(round(v)) for v in np.ldexp(x, 56 - e)]  # |q| <= 2^56
    dig = np.array([balanced(v) for v in q]).T
    return dig, e, q


def diagonals_fp32(sa, sb, seed=7):
    """A_d = sum_{i + j = d} sum_k sa_i[k] sb_j[k], accumulated in float32 in a random
    order, and the same sums in exact integers with the sum of their magnitudes."""
    rng = np.random.default_rng(seed)
    out32, exact, mags = [], [], []
    for d in range(S):
        prods = [int(sa[i][k]) * int(sb[d - i][k]) for i in range(d + 1) for k in range(sa.shape[1])]
        terms = np.array(prods, dtype=np.float32)[rng.permutation(len(prods))]
        acc = np.float32(0.0)
        for t in terms:
            acc = np.float32(acc + t)
        out32.append(acc)
        exact.append(sum(prods))
        mags.append(sum(abs(p) for p in prods))
    return out32, exact, mags


def test_balanced_digit_ranges_and_extremes():
    for q in (0, 1, -1, 63, 64, -64, -65, 2 ** 56, -(2 ** 56), 2 ** 56 - 1, -(2 ** 56) + 1,
              sum(64 << (7 * j) for j in range(8)), -sum(64 << (7 * j) for j in range(8))):
        d = balanced(q)
        assert d == balanced_by_bias(q)
        assert sum(v << (49 - BITS * j) for j, v in enumerate(d)) == q
        assert abs(d[0]) <= 128 and all(-64 <= v <= 63 for v in d[1:]), (q, d)


@pytest.mark.parametrize("K,seed", [(32, 0), (64, 1), (256, 2)])
def test_digits_reconstruct_the_fixed_point_value(K, seed):
    x = np.random.default_rng(seed).standard_normal(K) * np.exp(np.random.default_rng(seed + 9).uniform(-20, 20, K))
    dig, e, q = row_digits(x)
    assert np.all(np.abs(dig[0]) <= 128) and np.all((dig[1:] >= -64) & (dig[1:] <= 63))
    for k in range(K):
        assert sum(int(dig[j][k]) << (49 - BITS * j) for j in range(S)) == q[k]
        assert list(dig[:, k]) == balanced_by_bias(q[k])
    # the fixed point carries the row's entries to half a unit of 2^-56 of the row scale
    back = np.array([float(v) for v in q]) * 2.0 ** (e - 56)
    assert np.max(np.abs(back - x)) <= 2.0 ** (e - 57)


def extreme_rows(K):
    """Digits at the ends of their ranges with equal signs (largest diagonal sums)."""
    top = np.full((S, K), -64)
    top[0] = 128
    return top, top.copy()


@pytest.mark.parametrize("K", [32, 128, 256])
def test_diagonal_sums_are_exact_in_fp32_even_at_the_bounds(K):
    a, b = extreme_rows(K)
    cases = [(a, b), (a, -b)]
    rng = np.random.default_rng(K)
    for _ in range(2):
        cases.append((row_digits(rng.standard_normal(K))[0], row_digits(rng.standard_normal(K))[0]))
    for sa, sb in cases:
        out32, exact, mags = diagonals_fp32(sa, sb)
        for d in range(S):
            bound = K * (2 ** 14 if d <= 1 else (d + 3) * 2 ** 12)
            assert mags[d] <= bound <= 10 * 2 ** 20 < 2 ** 24
            assert int(out32[d]) == exact[d], (d, out32[d], exact[d])


def test_recombined_dot_product_has_fp64_accuracy():
    rng = np.random.default_rng(3)
    K = 256
    x = rng.standard_normal(K) * np.exp(rng.uniform(-5, 5, K))
    y = rng.standard_normal(K)
    sx, ex, _ = row_digits(x)
    sy, ey, _ = row_digits(y)
    out32, exact, _ = diagonals_fp32(sx, sy)
    hi = sum(int(out32[d]) << (BITS * (3 - d)) for d in range(4))
    lo = sum(int(out32[d]) << (BITS * (7 - d)) for d in range(4, S))
    assert abs(hi) < 2 ** 46 and abs(lo) < 2 ** 46
    val = (float(hi) * 2.0 ** -21 + float(lo) * 2.0 ** -49) * 2.0 ** (ex + ey - 14)
    ref = float(sum(np.longdouble(a) * np.longdouble(b) for a, b in zip(x, y)))
    scale = float(np.sum(np.abs(x) * np.abs(y)))
    assert abs(val - ref) <= 4e-16 * scale, (val, ref, abs(val - ref) / scale)
