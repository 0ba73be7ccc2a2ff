"""Pins of the oracle's rate quantisation, Hill production, argument checks
and overflow rule, against exact rational arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests._util import q_exact


def test_quantize_is_round_half_even_of_x_times_2_32():
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(0, 1000, 2000)) + [0.0, 0.1, 0.01, 1.0, 5.0, 10.0, 20.0]
    # exact ties: (m + 1/2) * 2^-32 rounds to the even neighbour
    xs += [(m + 0.5) * 2.0 ** -32 for m in (0, 1, 2, 3, 12345, 98765)]
    for x in xs:
        assert O.quantize(float(x)) == q_exact(float(x)), x
    assert O.quantize(0.5 * 2.0 ** -32) == 0 and O.quantize(1.5 * 2.0 ** -32) == 2


@pytest.mark.parametrize("bad", [-1.0, float("nan"), float("inf"), 2.0 ** 20])
def test_quantize_rejects_out_of_range(bad):
    with pytest.raises(O.OracleError):
        O.quantize(bad)


def test_hill_production_within_binary64_rounding():
    m = O.Model(kD=10.0, K=20.0)
    for R in list(range(0, 300)) + [1000, 65535, 2 ** 20, 2 ** 30 - 1]:
        exact = Fraction(10) / (1 + (Fraction(R) / 20) ** 2) * 2 ** 32
        got = O.hill_q(m, R)
        # four binary64 roundings (R/K, square, +1, divide) then rounding to an integer
        assert abs(Fraction(got) - exact) <= 1 + exact * Fraction(5, 2 ** 53), R
    assert O.hill_q(m, 0) == 10 * 2 ** 32
    assert O.hill_q(m, 20) == 5 * 2 ** 32


def test_overflow_is_reported():
    d = O.Desc(2, 1, 2, seed=1, init_lambda=(0.0, 0.0, 0.0))
    m = O.Model(hopD=1000.0)
    counts = np.zeros(2 * 3 * 4, dtype=np.int32)
    counts[0] = 2 ** 30 - 1  # 1000 * 2^32 * (2^30 - 1) * 2 directions >= 2^52
    with pytest.raises(O.OracleError) as e:
        O.step(d, m, counts, 0, 1, 0.1)
    assert e.value.code == -4


def test_invalid_arguments_rejected():
    m = O.Model()
    for d in (O.Desc(0, 1, 8, 1), O.Desc(1, 1, 1, 1), O.Desc(1, 1, 33, 1),
              O.Desc(1, 1, 8, 1, tissue_id=1 << 24), O.Desc(1, 1, 8, 1, init_lambda=(701, 0, 0))):
        with pytest.raises(O.OracleError):
            O.init_counts(d)
    d = O.Desc(2, 2, 4, 1)
    c = O.init_counts(d)
    with pytest.raises(O.OracleError):
        O.step(d, O.Model(K=0.0), c, 0, 1, 0.1)
    with pytest.raises(O.OracleError):
        O.step(d, m, c, 0, 1, 0.0)
    with pytest.raises(O.OracleError):
        O.sig_face(d, m, c, 1, 0, 0, 0.1)  # cell 1 has no +x neighbour in a 2-wide tissue


def test_zero_propensity_cell_fires_nothing():
    d = O.Desc(2, 2, 4, seed=3, init_lambda=(0.0, 0.0, 0.0))
    m = O.Model(kD=0.0, kN=0.0)
    c = O.init_counts(d)
    ne, tl = O.step(d, m, c, 0, 3, 0.1)
    assert ne.sum() == 0 and tl.sum() == 0 and c.sum() == 0
