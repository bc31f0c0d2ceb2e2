"""The FP32 rounding bounds that decide when a kernel re-decides a
comparison in FP64 (CPU): with c = ceil(d / 8) + 8, the squared-L2
difference form is within c 2^-24 relative of the exact value, and the
unit-row chord 2 - 2<x, y> within 2 c 2^-24 |x||y| + 2^-24 (2 + 2 |x||y|)
absolute, for the kernels' summation orders (eight strided lanes of float4
chunks combined by a butterfly, 32 strided lanes and a butterfly,
pairwise) with fused multiply-adds, on random and cancellation-heavy rows.
Exact values come from Python fractions."""
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -24


def f32(v):
    return np.float32(v)


def fma32(a, b, c):
    """fmaf: a * b + c with one rounding (the float64 product of two float32
    values is exact; float64 then float32 rounding of the sum differs from
    a single rounding by far less than the bounds' 1% margin)."""
    return f32(float(a) * float(b) + float(c))


def sum_orders(terms_a, terms_b, form):
    """FP32 accumulations of sum_i f(a_i, b_i) in the kernels' orders."""
    d = len(terms_a)

    def term_acc(acc, i):
        if form == "l2":
            t = f32(terms_a[i] - terms_b[i])
            return fma32(t, t, acc)
        return fma32(terms_a[i], terms_b[i], acc)

    out = []
    lanes = [f32(0)] * 8  # eight lanes, lane li takes float4 chunks li, li + 8, ...
    for c in range(d // 4):
        for e in range(4):
            lanes[c % 8] = term_acc(lanes[c % 8], 4 * c + e)
    for o in (4, 2, 1):
        lanes = [f32(lanes[j] + lanes[j ^ o]) for j in range(8)]
    out.append(lanes[0])
    lanes = [f32(0)] * 32  # 32 strided lanes, then a butterfly
    for i in range(d):
        lanes[i % 32] = term_acc(lanes[i % 32], i)
    for o in (16, 8, 4, 2, 1):
        lanes = [f32(lanes[j] + lanes[j ^ o]) for j in range(32)]
    out.append(lanes[0])
    parts = [term_acc(f32(0), i) for i in range(d)]  # pairwise
    while len(parts) > 1:
        parts = [f32(parts[j] + parts[j + 1]) if j + 1 < len(parts) else parts[j]
                 for j in range(0, len(parts), 2)]
    out.append(parts[0])
    return out


def exact_sum(a, b, form):
    if form == "l2":
        return sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a, b))
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))


@pytest.mark.parametrize("d", [4, 36, 128, 384, 960])
def test_difference_form_bound(d):
    rs = np.random.default_rng(d)
    bound = ((d + 7) // 8 + 8) * U * 1.01
    for trial in range(60):
        scale = 10.0 ** rs.uniform(-3, 3)
        x = (rs.normal(0, 1, d) * scale).astype(np.float32)
        # near neighbours (heavy cancellation in x - y) and far pairs
        y = (x + rs.normal(0, 10.0 ** rs.uniform(-6, 0), d) * scale).astype(np.float32)
        s = exact_sum(x, y, "l2")
        if s == 0:
            continue
        for got in sum_orders(x, y, "l2"):
            assert abs(Fraction(float(got)) - s) <= Fraction(bound) * s, (d, trial)


@pytest.mark.parametrize("d", [4, 96, 384])
def test_chord_form_bound(d):
    rs = np.random.default_rng(100 + d)
    for trial in range(60):
        x = rs.normal(0, 1, d)
        x = (x / np.linalg.norm(x)).astype(np.float32)
        y = x + rs.normal(0, 10.0 ** rs.uniform(-4, 0), d)
        y = (y / np.linalg.norm(y)).astype(np.float32)
        nm = float(np.linalg.norm(x.astype(np.float64)) * np.linalg.norm(y.astype(np.float64)))
        bound = (2 * ((d + 7) // 8 + 8) * U * nm + U * (2 + 2 * nm)) * 1.01
        exact = 2 - 2 * exact_sum(x, y, "dot")
        for dot in sum_orders(x, y, "dot"):
            got = max(float(f32(2) - f32(2) * dot), 0.0)
            assert abs(Fraction(got) - exact) <= Fraction(bound), (d, trial)

