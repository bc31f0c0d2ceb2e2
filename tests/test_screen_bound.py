"""The error bound that certifies the screened kNN on real-valued rows (CPU).

The screened form centres the rows on the column means in FP32, splits each
centred value v into BF16 parts hi = bf16(v), lo = bf16(v - hi), and the
tensor cores contract [hi | hi | lo] with [hi | lo | hi] in FP32 (every
product of two BF16 values is exact in FP32), so the dropped terms are
lo.lo and the rounding of lo.  The tile epilogue forms s = |q|^2 + (|x|^2 -
2 <q, x>) from FP32 row norms.  A row's shortlist is accepted only when its
exact K-th distance lies below the last screened distance minus the bound, so
the bound must hold for every pair in any summation order the tensor cores
may use.  Here the arithmetic is emulated in several orders and compared
with the exact distance of the original FP32 rows (Python fractions); the
bound is restated from the kernel (2 (3 2^-16 + gamma(3d)) |x||y|, the FP32
norms d 2^-23 (|x|^2 + |y|^2), the final additions 2^-22 (|x| + |y|)^2 and
the centring's rounding), with its 1% margins.  A screen without the lo
terms breaks the bound, so the test can fail."""
from fractions import Fraction

import numpy as np
import pytest

import synthetic


def round_f32(q: Fraction) -> Fraction:
    """Exact round-to-nearest-even of a rational to FP32 (normal range)."""
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    scale = Fraction(2) ** (e - 23)  # 24-bit significand
    m = a / scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * fl * scale


def bf16(v: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP32 -> BF16, as FP32 values."""
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def screen_bound(na, nb, d, dp3):
    """The kernel's bound for a row of squared norm na against a point of
    squared norm <= nb (centred rows, L2)."""
    a, b = np.sqrt(na) * 1.0001, np.sqrt(nb) * 1.0001
    u16, u23 = 2.0 ** -16, 2.0 ** -23
    g = dp3 * u23 / (1.0 - dp3 * u23)
    e = 2.0 * (3.001 * u16 + 1.02 * g) * a * b
    dl = 2.0 ** -24 * 1.001 * (a + b)
    e += d * u23 * (a * a + b * b) + 2.0 ** -22 * 1.01 * (a + b) ** 2 + 2.0 * (a + b) * dl + dl * dl
    return e * 1.01 + 1e-12


def accumulate(terms, order):
    """FP32 sum of exact FP32 terms in one of several orders."""
    t = np.asarray(terms, np.float32)
    if order == "reverse":
        t = t[::-1]
    if order == "pairwise":
        while len(t) > 1:
            if len(t) % 2:
                t = np.append(t, np.float32(0))
            t = (t[0::2] + t[1::2]).astype(np.float32)
        return float(t[0])
    if order == "k16":  # blocks of 16 products summed, then the blocks in order
        acc = np.float32(0)
        for i in range(0, len(t), 16):
            acc = np.float32(acc + np.float32(np.sum(t[i:i + 16], dtype=np.float32)))
        return float(acc)
    acc = np.float32(0)
    for x in t:
        acc = np.float32(acc + x)
    return float(acc)


def screened(rows, with_lo=True):
    """Centred split rows and FP32 norms, as the split kernel makes them."""
    n, d = rows.shape
    colsum = np.sum(rows, axis=0, dtype=np.float32)
    mean = (colsum * np.float32(1.0 / n)).astype(np.float32)
    v = (rows - mean).astype(np.float32)
    hi = bf16(v)
    lo = bf16((v - hi).astype(np.float32)) if with_lo else np.zeros_like(v)
    norms = np.zeros(n, np.float32)
    for r in range(n):  # 32 strided lanes of fused multiply-adds, then a butterfly
        lanes = np.zeros(32, np.float32)
        for i in range(d):
            lanes[i % 32] = np.float32(float(lanes[i % 32]) + float(v[r, i]) * float(v[r, i]))
        while len(lanes) > 1:
            lanes = (lanes[: len(lanes) // 2] + lanes[len(lanes) // 2:]).astype(np.float32)
        norms[r] = lanes[0]
    return hi, lo, norms


def screened_distance(hq, lq, hx, lx, nq, nx, order):
    terms = np.concatenate([hq * hx, hq * lx, lq * hx]).astype(np.float32)  # exact products
    dot = accumulate(terms, order)
    inner = round_f32(Fraction(float(nx)) - 2 * Fraction(dot))  # fmaf(-2, dot, |x|^2)
    return float(round_f32(Fraction(float(nq)) + inner))


def exact_distance(x, y):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, y))


@pytest.mark.parametrize("kind,d,n", [("mixture", 32, 24), ("mixture", 128, 16),
                                      ("offset", 64, 16)])
def test_screen_error_within_the_bound(kind, d, n):
    if kind == "mixture":
        rows, _ = synthetic.mixture_float(n, d, 3, 7 + d)
    else:  # a large common offset: the centring carries the accuracy
        rng = np.random.default_rng(d)
        rows = (1000.0 + rng.normal(0.0, 0.05, size=(n, d))).astype(np.float32)
    rows = rows.astype(np.float32)
    hi, lo, norms = screened(rows)
    dp3 = (3 * d + 63) // 64 * 64
    nb = float(norms.max())
    worst = 0.0
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            ex = exact_distance(rows[i], rows[j])
            bound = screen_bound(float(norms[i]), nb, d, dp3)
            for order in ("sequential", "reverse", "pairwise", "k16"):
                s = screened_distance(hi[i], lo[i], hi[j], lo[j], norms[i], norms[j], order)
                err = abs(Fraction(s) - ex)
                assert err <= Fraction(bound), (i, j, order, float(err), bound)
                worst = max(worst, float(err) / bound)
    assert worst > 0.0


def test_the_lo_terms_are_needed_for_the_bound():
    rows, _ = synthetic.mixture_float(16, 128, 3, 99)
    rows = rows.astype(np.float32)
    hi, lo0, norms = screened(rows, with_lo=False)
    nb = float(norms.max())
    broke = 0
    for i in range(16):
        for j in range(16):
            if i != j:
                ex = exact_distance(rows[i], rows[j])
                s = screened_distance(hi[i], lo0[i], hi[j], lo0[j], norms[i], norms[j],
                                      "sequential")
                broke += abs(Fraction(s) - ex) > Fraction(screen_bound(float(norms[i]), nb, 128,
                                                                       384))
    assert broke > 0


@pytest.mark.parametrize("seed", range(4))
def test_chunk_lower_bound_never_exceeds_a_column(seed):
    """The kNN tile epilogue dismisses a 32-column chunk for a row when
    |q|^2 + fmaf(-2, max_j v_j, min_j |x_j|^2) exceeds the row's K-th
    distance.  Correctly rounded operations are monotone, so that bound is at
    most every column's |q|^2 + fmaf(-2, v_j, |x_j|^2): checked with exact
    roundings on random and nearly tied columns."""
    rng = np.random.default_rng(seed)
    for _ in range(200):
        nq = np.float32(rng.uniform(0, 1e7))
        base = rng.uniform(-1e6, 1e6)
        v = (base + rng.normal(0, rng.choice([1e-3, 1.0, 1e3]), 32)).astype(np.float32)
        nb = np.abs(rng.normal(5e6, rng.choice([1e-2, 10.0, 1e5]), 32)).astype(np.float32)
        fma = [round_f32(Fraction(float(b)) - 2 * Fraction(float(x))) for x, b in zip(v, nb)]
        cols = [round_f32(Fraction(float(nq)) + f) for f in fma]
        lb = round_f32(Fraction(float(nq)) +
                       round_f32(Fraction(float(nb.min())) - 2 * Fraction(float(v.max()))))
        assert lb <= min(cols)
