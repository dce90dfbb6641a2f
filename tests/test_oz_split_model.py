"""The dense true residual's error-free splitting (Ozaki, Ogita, Oishi and
Rump, Numer. Algorithms 59, 2012) on a CPU model of its integer arithmetic.

Each row of an operand is written 2^E sum_{i=1..7} d_i 2^(-6 i) with
|x| < 2^E over the row, balanced integer digits |d_1| <= 64, |d_i| <= 32,
taken from the value as a 62-bit fixed-point integer.  A slice d_i 2^(-6i)
is a BF16 value exactly.  Over one anti-diagonal s = i + j of slice pairs
and K terms, every product is an integer multiple of 2^(-6 s) and their
absolute sum is at most K 2^10 max(s + 1, 4) such units, which for K <= 1024
and s <= 8 is below 2^24: the FP32 accumulation of a diagonal is exact in any
order.  The seven diagonal sums then give the product within about 2^-42 of
K max|x| max|phi|.  The model follows those definitions in Python integers
and float64; it checks the scheme, not the kernels.
"""
import numpy as np
import pytest

S, BETA = 7, 6


def _digits(row):
    """(E, digits[S][K]) of one row, as the splitting defines them."""
    row = np.asarray(row, dtype=np.float64)
    mx = np.abs(row).max()
    if mx == 0.0:
        return 0, np.zeros((S, row.size), dtype=np.int64)
    E = int(np.frexp(mx)[1])                      # mx < 2^E, mx >= 2^(E-1)
    out = np.zeros((S, row.size), dtype=np.int64)
    for k, v in enumerate(row):
        # v / 2^E as an integer over 2^62, truncated toward zero: the 53-bit
        # significand shifted by its exponent (no overflow at any scale)
        m, e = np.frexp(abs(v))
        mi = int(m * 2.0 ** 53)
        sh = int(e) - 53 + 62 - E
        V = mi << sh if sh >= 0 else mi >> -sh
        r = V if v >= 0 else -V
        for i in range(1, S + 1):
            sh = 62 - i * BETA
            d = (r + (1 << (sh - 1))) >> sh           # balanced digit (round half up)
            r -= d << sh
            out[i - 1, k] = d
    return E, out


def _bf16_exact(v):
    """v is a BF16 value: 8 significant bits."""
    m, _ = np.frexp(v)
    return np.all(m * 256.0 == np.round(m * 256.0))


def _diagonals(dx, dp):
    """Exact integer sums over each anti-diagonal s = i + j (1-based, s = 2..S+1)
    in units of 2^(-6 s), and the absolute sums."""
    sums, abss = {}, {}
    for i in range(1, S + 1):
        for j in range(1, S + 2 - i):
            s = i + j
            prod = dx[i - 1].astype(object) * dp[j - 1].astype(object)
            sums[s] = sums.get(s, 0) + int(sum(prod))
            abss[s] = abss.get(s, 0) + int(sum(abs(t) for t in prod))
    return sums, abss


@pytest.mark.parametrize("scale", [1.0, 1e-300, 3e200])
def test_digits_are_balanced_bf16_slices_and_reconstruct_the_row(scale):
    rng = np.random.default_rng(3)
    row = scale * rng.standard_normal(200) * np.exp(rng.uniform(-20, 0, 200))
    E, d = _digits(row)
    assert np.abs(d[0]).max() <= 64 and np.abs(d[1:]).max() <= 32
    for i in range(S):
        assert _bf16_exact(d[i] * 2.0 ** (-BETA * (i + 1)))
    rec = sum(d[i].astype(np.float64) * 2.0 ** (-BETA * (i + 1)) for i in range(S)) * 2.0 ** E
    # the part below the seventh digit is at most half a unit of 2^(E - 42)
    assert np.abs(rec - row).max() <= 2.0 ** (E - 42)


def test_diagonal_sums_are_exact_in_fp32_up_to_k_1024():
    """Worst-case digits (every |d| at its bound) over K = 1024 terms: every
    diagonal's absolute sum stays below 2^24 units, so any FP32 accumulation
    order is exact; random rows reach far less."""
    K = 1024
    worst = np.full((S, K), 32, dtype=np.int64)
    worst[0] = 64
    _, abss = _diagonals(worst, worst)
    assert abss == {s: K * 2 ** 10 * max(s + 1, 4) for s in range(2, S + 2)}
    assert max(abss.values()) < 2 ** 24
    rng = np.random.default_rng(4)
    _, dx = _digits(rng.standard_normal(K))
    _, dp = _digits(rng.standard_normal(K))
    sums, abss = _diagonals(dx, dp)
    for s, v in sums.items():
        assert abss[s] < 2 ** 24
        assert float(np.float32(v)) == v            # the diagonal sum itself is an FP32 value


def test_diagonal_bound_fails_beyond_k_1024():
    """A planted mistake: twice the K the scheme allows.  The worst-case
    absolute sums pass 2^24 units, and an FP32 running sum of a diagonal's
    terms then rounds: the exactness argument needs K <= 1024."""
    K = 2048
    worst = np.full((S, K), 32, dtype=np.int64)
    worst[0] = 64
    _, abss = _diagonals(worst, worst)
    assert max(abss.values()) > 2 ** 24
    # diagonal s = 8 at worst-case digits: the pairs (1, 7) and (7, 1) give
    # 64 * 32 per term, the five inner pairs 32 * 32; summed in FP32 in order,
    # with one unit more, against the exact (odd, above 2^24) sum
    terms = [64 * 32, 32 * 32, 32 * 32, 32 * 32, 32 * 32, 32 * 32, 64 * 32] * K + [1]
    assert sum(terms) > 2 ** 24 and sum(terms) % 2 == 1
    acc = np.float32(0.0)
    for t in terms:
        acc = np.float32(acc + np.float32(t))
    assert int(acc) != sum(terms)


def test_split_product_within_its_bound():
    """The product of a row of Phi and a row of X from the seven diagonal
    sums (added smallest first) against the exact product, for rows of very
    different scales: within 2^-40 of K max|x| max|phi| (the dropped digits
    and pairs are below about 2^-41 of it) and within the GPU tests' bound
    2^-36 sum_k |phi_k| |x_k|."""
    from fractions import Fraction
    rng = np.random.default_rng(9)
    K = 300
    for sx, sp in ((1.0, 1.0), (1e-8, 3e5), (1e120, 1e-150)):
        x = sx * rng.standard_normal(K) * np.exp(rng.uniform(-10, 0, K))
        p = sp * rng.standard_normal(K)
        Ex, dx = _digits(x)
        Ep, dp = _digits(p)
        sums, _ = _diagonals(dx, dp)
        got = 0.0
        for s in sorted(sums, reverse=True):          # smallest diagonal first
            got += float(np.float32(sums[s])) * 2.0 ** (-BETA * s)
        got = got * 2.0 ** (Ex + Ep)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, p))
        err = abs(float(Fraction(got) - exact))
        assert err <= 2.0 ** -40 * K * np.abs(x).max() * np.abs(p).max()
        assert err <= 2.0 ** -36 * float(sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(x, p)))
