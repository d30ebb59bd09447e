"""The exact-splitting arithmetic the FP64 tensor-core kernels rely on, checked
in numpy on the CPU, independently of the kernels.

An FP64 vector x with 2^e > max|x| is scaled to integers I = rint(x 2^(beta S - e))
and written as S balanced digits in base 2^beta, most significant first (the
leading digit up to 2^beta in magnitude, the others up to 2^(beta-1)).  A dot
product of two such vectors keeps the digit-pair groups g = s + t <= S + 1:
C_g = sum_{s+t=g} sum_k A_s[k] B_t[k], and a.b ~ Y 2^(e_a + e_b - beta (S+1)) with
Y = sum_g C_g 2^(beta (S + 1 - g)).  The claims checked here:
- with K 4^(beta-1) (S+2) < 2^24 (the rule that picks beta for a contraction of
  length K), every partial sum of every C_g, in any order, is an integer an FP32
  accumulator holds exactly;
- Y combined in two int64 Horner chains (ceil(S/2) groups of largest scale, then
  the rest) keeps each chain below 2^53, so one conversion and one fused
  multiply-add round once;
- the result equals the exact dot product up to a few units of FP64 rounding of
  max|a| max|b| per term.
The digit plans are those of the fitting GEMMs ((beta, S) = (7, 8), (6, 10),
(5, 11), (4, 14)) and of the embedding layers (beta = 8, S = 7, K <= 64).
"""
from fractions import Fraction

import numpy as np
import pytest

PLANS = [(7, 8), (6, 10), (5, 11), (4, 14), (8, 7)]


def k_max(beta, S):
    """Largest contraction length the selection rule accepts for (beta, S)."""
    return (2 ** 24 - 1) // (4 ** (beta - 1) * (S + 2))


def balanced_digits(I, beta, S):
    """S digits of the int64 array I, most significant first: I = sum_s d_s 2^(beta (S - s))."""
    I = np.array(I, dtype=object)
    out = []
    base, half = 1 << beta, 1 << (beta - 1)
    for _ in range(S - 1):
        r = np.array([int(v) % base for v in I], dtype=object)
        r = np.where(r > half, r - base, r)
        out.append(r)
        I = (I - r) // base
    out.append(I)
    return [np.array(d, dtype=np.int64) for d in reversed(out)]


def split(x, beta, S):
    e = int(np.frexp(np.abs(x).max())[1])      # 2^e > max|x|
    # x 2^(beta S - e) is exact (a power-of-two scaling); rounding it to the nearest
    # integer (ties to even) is what the kernels' conversion does
    I = [int(round(float(v) * 2.0 ** (beta * S - e))) for v in x]
    return balanced_digits(I, beta, S), e


def worst_group_bound(beta, S):
    """max over g of sum_{s+t=g} |d_s|max |e_t|max, with the leading digit's larger bound."""
    b = [2 ** beta] + [2 ** (beta - 1)] * (S - 1)
    best = 0
    for g in range(2, S + 2):
        best = max(best, sum(b[s - 1] * b[g - s - 1] for s in range(1, g) if 1 <= g - s <= S))
    return best


@pytest.mark.parametrize("beta,S", PLANS)
def test_selection_rule_bounds_every_group_sum(beta, S):
    K = k_max(beta, S) if (beta, S) != (8, 7) else 64
    assert K * 4 ** (beta - 1) * (S + 2) < 2 ** 24
    assert worst_group_bound(beta, S) == (S + 2) * 4 ** (beta - 1)
    assert K * worst_group_bound(beta, S) < 2 ** 24
    # both Horner chains of the combination stay below 2^53
    H = (S + 1) // 2 if (beta, S) != (8, 7) else 3
    for n in (H, S - H):
        assert 2 ** 24 * sum(2 ** (beta * j) for j in range(n)) < 2 ** 53
    # the digits carry at least 55 bits of each operand
    assert beta * S >= 55


@pytest.mark.parametrize("beta,S", PLANS)
def test_digits_reconstruct_and_are_bounded(beta, S):
    rng = np.random.default_rng(beta * 100 + S)
    x = rng.standard_normal(64) * np.exp(rng.uniform(-20, 20, 64))
    d, e = split(x, beta, S)
    assert np.abs(d[0]).max() <= 2 ** beta
    for ds in d[1:]:
        assert np.abs(ds).max() <= 2 ** (beta - 1)
    for k in range(len(x)):
        val = sum(int(d[s][k]) << (beta * (S - 1 - s)) for s in range(S))
        assert val == int(round(float(x[k]) * 2.0 ** (beta * S - e)))


@pytest.mark.parametrize("beta,S", PLANS)
def test_split_dot_product_is_fp64_accurate(beta, S):
    rng = np.random.default_rng(7 * beta + S)
    K = min(k_max(beta, S), 1600) if (beta, S) != (8, 7) else 64
    a = rng.standard_normal(K) * np.exp(rng.uniform(-3, 3, K))
    b = rng.standard_normal(K) * 1e-3
    A, ea = split(a, beta, S)
    B, eb = split(b, beta, S)
    perm = rng.permutation(K)
    C = {}
    for g in range(2, S + 2):
        terms = []
        for s in range(1, g):
            t = g - s
            if 1 <= t <= S:
                terms.append(A[s - 1][perm] * B[t - 1][perm])
        terms = np.concatenate(terms)
        # FP32 accumulation in this order: every prefix sum exact
        acc32 = np.add.accumulate(terms.astype(np.float32), dtype=np.float32)
        acc64 = np.add.accumulate(terms.astype(np.int64))
        np.testing.assert_array_equal(acc32.astype(np.int64), acc64)
        assert np.abs(acc64).max() < 2 ** 24
        C[g] = int(acc64[-1])
    H = (S + 1) // 2
    hi = 0
    for g in range(2, H + 2):
        hi = hi * 2 ** beta + C[g]
    lo = 0
    for g in range(H + 2, S + 2):
        lo = lo * 2 ** beta + C[g]
    assert abs(hi) < 2 ** 53 and abs(lo) < 2 ** 53
    y = float(Fraction(hi) * 2 ** (beta * (S - H)) + Fraction(lo))   # one rounding
    res = y * 2.0 ** (ea + eb - beta * (S + 1))
    exact = sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(a, b))
    scale = float(np.abs(a).max() * np.abs(b).max())
    assert abs(Fraction(res) - exact) <= 4 * K * 2.0 ** -55 * scale + abs(float(exact)) * 2.0 ** -52


# The 28-bit plans of the split mixed mode's fitting net ((beta, S) = (7, 4)
# for K = 240, (6, 5) for K <= 2,048): the same exactness of every group sum
# and of the combination, and a dot product within the expansions' precision.
REDUCED = [(7, 4), (6, 5)]


@pytest.mark.parametrize("beta,S", REDUCED)
def test_reduced_plans_are_exact_to_their_precision(beta, S):
    assert beta * S >= 28
    assert k_max(beta, S) >= (240 if beta == 7 else 2048)
    assert worst_group_bound(beta, S) == (S + 2) * 4 ** (beta - 1)
    H = (S + 1) // 2
    for n in (H, S - H):
        assert 2 ** 24 * sum(2 ** (beta * j) for j in range(n)) < 2 ** 53
    rng = np.random.default_rng(11 * beta + S)
    K = 240 if beta == 7 else 2048
    a = rng.standard_normal(K) * np.exp(rng.uniform(-3, 3, K))
    b = rng.standard_normal(K) * 1e-3
    A, ea = split(a, beta, S)
    B, eb = split(b, beta, S)
    C = {}
    for g in range(2, S + 2):
        terms = np.concatenate([A[s - 1] * B[g - s - 1] for s in range(1, g) if 1 <= g - s <= S])
        acc32 = np.add.accumulate(terms.astype(np.float32), dtype=np.float32)
        acc64 = np.add.accumulate(terms.astype(np.int64))
        np.testing.assert_array_equal(acc32.astype(np.int64), acc64)
        C[g] = int(acc64[-1])
    y = 0
    for g in range(2, S + 2):
        y = y * 2 ** beta + C[g]
    res = float(Fraction(y) * Fraction(2) ** (ea + eb - beta * (S + 1)))
    exact = sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(a, b))
    scale = float(np.abs(a).max() * np.abs(b).max())
    # truncation of the operands to beta S bits plus the dropped groups g > S + 1
    assert abs(Fraction(res) - exact) <= 4 * K * 2.0 ** -(beta * S) * scale
