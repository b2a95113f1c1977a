"""The arithmetic the split-precision form relies on, checked on the CPU from its definition:
balanced base-256 digits of a scaled FP64 value, each exact in bf16, exact fp32 sums of the
same-weight digit products for K <= 256, and the error of dropping products of weight above 5."""
import numpy as np
import pytest

S = 6


def balanced_digits(x, e):
    """Digits d_0..d_5 with x = 2^e sum_i d_i 2^(-8(i+1)) up to rounding of the last one:
    T = round(|x| 2^(48 - e)) written in base 256 from the least significant digit up, each digit
    moved into [-128, 127] by a carry, the leading digit what remains; the sign of x on every digit."""
    T = int(round(abs(x) * 2.0 ** (8 * S - e)))
    d = [0] * S
    for i in range(S - 1, 0, -1):
        r = T % 256
        T //= 256
        if r >= 128:
            r -= 256
            T += 1
        d[i] = r
    d[0] = T
    return [-v for v in d] if x < 0 else d


def exponent(v):
    return int(np.frexp(v)[1]) if v > 0 else 0


def test_digits_reconstruct_and_are_bounded():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        x = rng.standard_normal() * 10.0 ** rng.integers(-30, 30)
        e = exponent(abs(x))
        d = balanced_digits(x, e)
        assert 0 <= abs(d[0]) <= 256 and all(abs(v) <= 128 for v in d[1:])
        back = sum(v * 2.0 ** (e - 8 * (i + 1)) for i, v in enumerate(d))
        assert abs(back - x) <= 2.0 ** (e - 8 * S - 1) * (1 + 1e-12)


def test_scaled_digits_are_exact_in_bf16():
    torch = pytest.importorskip("torch")
    vals = [v * 2.0 ** (-8 * (i + 1)) for i in range(S) for v in range(-256, 257)]
    t = torch.tensor(vals, dtype=torch.float64)
    assert torch.equal(t.to(torch.bfloat16).to(torch.float64), t)


def test_same_weight_sums_fit_fp32_for_k_256():
    # weight w products a_i b_j (i + j = w) summed over K = 256 stay below 2^24 of their unit for
    # w <= 1, so an fp32 accumulator holds them exactly, in any order
    K = 256
    worst = {0: 256 * 256 * K, 1: 2 * 256 * 128 * K}
    assert worst[0] <= 2 ** 24 and worst[1] <= 2 ** 24
    rng = np.random.default_rng(1)
    a = rng.integers(-128, 129, (2, K)); a[0] = rng.integers(0, 257, K)
    b = rng.integers(-128, 129, (2, K)); b[0] = rng.integers(0, 257, K)
    for w, terms in ((0, [(0, 0)]), (1, [(0, 1), (1, 0)])):
        exact = sum(int(np.dot(a[i].astype(np.int64), b[j].astype(np.int64))) for i, j in terms)
        acc = np.float32(0.0)
        for k in rng.permutation(K):
            for i, j in terms:
                acc = np.float32(acc + np.float32(a[i][k] * b[j][k]))
        assert int(acc) == exact


def test_dropping_high_weights_costs_about_2_to_the_minus_48():
    # a dot product of K = 256 FP64 numbers from the 21 kept slice products (i + j <= 5), summed
    # exactly: each operand is represented to half a unit of 2^(e - 48) and the dropped products
    # (weight >= 6) are below K 2^(ea + eb - 56), so the error is bounded by
    # 2^-48 (2^ea sum |b| + 2^eb sum |a|) + K 2^(ea + eb - 56)
    rng = np.random.default_rng(2)
    K = 256
    for _ in range(20):
        a = rng.standard_normal(K) * np.exp(rng.uniform(-3, 3, K))
        b = rng.standard_normal(K) * np.exp(rng.uniform(-3, 3, K))
        ea, eb = exponent(np.abs(a).max()), exponent(np.abs(b).max())
        da = np.array([balanced_digits(v, ea) for v in a], dtype=object)
        db = np.array([balanced_digits(v, eb) for v in b], dtype=object)
        total = 0
        for i in range(S):
            for j in range(S - i):
                total += sum(int(da[k][i]) * int(db[k][j]) * 2 ** (8 * (2 * S - 2 - i - j)) for k in range(K))
        from fractions import Fraction
        approx = Fraction(total) * Fraction(2) ** (ea + eb - 16 * S)
        ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        bound = 2.0 ** -48 * (2.0 ** ea * np.abs(b).sum() + 2.0 ** eb * np.abs(a).sum()) + K * 2.0 ** (ea + eb - 56)
        assert abs(approx - ref) <= Fraction(bound)


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    e = np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))
    return s, e


def test_fold_of_the_four_weight_groups():
    # the device fold (split.cu fold4) in fp32: TwoSums bring in groups 0, 1 and 2, their two errors
    # and group 3 are added in fp32, a last TwoSum renormalises; h + l stays within
    # 2^-23 (2^-24 (|g0 + g1| + |g0 + g1 + g2|) + |g3|) of the exact sum, whatever the signs and
    # cancellation (adding group 2 in fp32 instead would cost up to 2^-24 |g2|)
    from fractions import Fraction
    rng = np.random.default_rng(3)
    for _ in range(5000):
        g0 = np.float32(rng.integers(-2 ** 24, 2 ** 24))
        g1 = np.float32(rng.integers(-2 ** 24, 2 ** 24) * 2.0 ** -8)
        if rng.random() < 0.2:
            g1 = np.float32(-g0 + rng.integers(-4, 4) * 2.0 ** -8)   # heavy cancellation
        g2 = np.float32(rng.standard_normal() * 2.0 ** (8 - rng.integers(0, 12)))
        g3 = np.float32(rng.standard_normal() * 2.0 ** (-rng.integers(0, 12)))
        s, e = _two_sum(g0, g1)
        s2, e2 = _two_sum(s, g2)
        h, l = _two_sum(s2, np.float32(np.float32(e + e2) + g3))
        F = lambda v: Fraction(float(v))
        exact = F(g0) + F(g1) + F(g2) + F(g3)
        err = abs(F(h) + F(l) - exact)
        bound = Fraction(2) ** -23 * (Fraction(2) ** -24 * Fraction(101, 100) * (abs(F(g0) + F(g1)) + abs(F(g0) + F(g1) + F(g2)))
                                      + abs(F(g3)))
        assert err <= bound, (g0, g1, g2, g3, float(err), float(bound))
