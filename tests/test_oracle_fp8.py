"""Pins of the oracle's FP8 E4M3 row format (CPU): the decoder against values
fixed by the format's bit fields, the encoder against brute force over all
finite codes (nearest value, ties to the even mantissa, saturation at 448,
sign kept), and the per-row scaling."""
import math

import numpy as np
import pytest

import oracle

FINITE = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)


def test_decoder_fixed_values():
    table = {0x00: 0.0, 0x38: 1.0, 0x40: 2.0, 0xC0: -2.0, 0xB0: -0.5, 0x7E: 448.0,
             0x08: 2.0 ** -6, 0x01: 2.0 ** -9, 0x07: 7 * 2.0 ** -9, 0x77: 240.0,
             0x3A: 1.25, 0xFE: -448.0}
    for code, value in table.items():
        assert oracle.fp8_e4m3_decode(np.uint8(code)) == value, hex(code)
    assert math.isnan(oracle.fp8_e4m3_decode(np.uint8(0x7F)))
    assert math.isnan(oracle.fp8_e4m3_decode(np.uint8(0xFF)))
    # the 126 positive finite values are distinct and ascend with the code
    pos = oracle.fp8_e4m3_decode(np.arange(0, 0x7F, dtype=np.uint8))
    assert (np.diff(pos) > 0).all() and pos[-1] == 448.0


def test_encoder_fixed_values():
    cases = [(0.0, 0x00), (1.0, 0x38), (-2.0, 0xC0), (448.0, 0x7E), (1000.0, 0x7E),
             (-1e9, 0xFE), (2.0 ** -6, 0x08), (2.0 ** -9, 0x01),
             (2.0 ** -10, 0x00),        # tie between 0 and 2^-9: even
             (3 * 2.0 ** -10, 0x02),    # tie between 1 and 2 (x 2^-9): even
             (1.0625, 0x38),            # tie between 1 and 1.125: even
             (1.1875, 0x3A),            # tie between 1.125 and 1.25: even
             (464.0, 0x7E), (-0.0, 0x80), (-1e-5, 0x80)]
    for x, code in cases:
        assert int(oracle.fp8_e4m3_encode(np.float32(x))) == code, (x, hex(code))


def test_encoder_is_nearest_with_ties_to_even_by_brute_force():
    vals = oracle.fp8_e4m3_decode(FINITE)
    rs = np.random.default_rng(3)
    xs = np.concatenate([rs.uniform(-448, 448, 3000), rs.normal(0, 0.01, 1000),
                         rs.normal(0, 2.0 ** -8, 500),
                         # exact midpoints between neighbouring positive values
                         (np.sort(vals[vals > 0])[1:] + np.sort(vals[vals > 0])[:-1]) / 2]
                        ).astype(np.float32)
    codes = oracle.fp8_e4m3_encode(xs)
    for x, c in zip(xs.astype(np.float64), codes):
        err = np.abs(vals - x)
        best = err.min()
        got = float(oracle.fp8_e4m3_decode(c))
        assert abs(got - x) == best, (x, hex(int(c)))
        ties = FINITE[err == best]
        if len(ties) > 1 and abs(x) > 0:
            # of two nearest values the one with the even mantissa
            assert (int(c) & 1) == 0, (x, hex(int(c)))


def test_every_finite_value_round_trips():
    vals = oracle.fp8_e4m3_decode(FINITE).astype(np.float32)
    back = oracle.fp8_e4m3_encode(vals)
    zero = vals == 0
    assert (back[~zero] == FINITE[~zero]).all()
    assert set(back[zero]) <= {0x00, 0x80}


def test_rows_scale_maps_the_largest_magnitude_to_448():
    rs = np.random.default_rng(4)
    D = rs.normal(0, 1, (20, 48)).astype(np.float32)
    D[3] = 0.0
    codes, scale = oracle.fp8_rows(D)
    assert scale[3] == 1.0 and (codes[3] == 0).all()
    for r in range(20):
        if r == 3:
            continue
        j = int(np.argmax(np.abs(D[r])))
        assert scale[r] == np.float32(np.abs(D[r]).max() / np.float32(448.0))
        assert abs(oracle.fp8_e4m3_decode(codes[r, j])) == 448.0
        # reconstruction error per element: half a step of E4M3, 2^-4 relative
        # for normal codes, 2^-10 absolute (x scale) below 2^-6
        rec = oracle.fp8_e4m3_decode(codes[r]) * scale[r]
        tol = np.maximum(np.abs(D[r]) * 2.0 ** -4, 2.0 ** -10 * scale[r])
        assert (np.abs(rec - D[r]) <= tol * (1 + 1e-6)).all()
