"""The sweep's curve fits (Section 3.1's x^(5/6) term, Section 3.2's
Li_{1/6} term) recover known coefficients from synthetic curves."""
import math

import numpy as np
import pytest

from paper_2507_06579_gb300 import sweep


def test_five_sixths_fit_recovers_the_coefficient():
    xs = np.geomspace(1e6, 1e11, 60)
    for c in (-0.024, 0.0, 0.05):
        curve = [(int(x), 0, int(round(x / (3 * math.pi ** 2) + c * x ** (5 / 6)))) for x in xs]
        assert sweep.fit_five_sixths(curve, x_min=1e8) == pytest.approx(c, abs=1e-6)
    # points below x_min are ignored
    bad = [(10**6, 0, 10**9)] + [(int(x), 0, int(round(x / (3 * math.pi ** 2)))) for x in xs[30:]]
    assert abs(sweep.fit_five_sixths(bad, x_min=1e8)) < 1e-6


def test_prime_fit_recovers_the_coefficient():
    quad = pytest.importorskip("scipy.integrate").quad
    xs = np.geomspace(1e8, 1e11, 12)

    def li16(x):  # int_2^x dt / (t^(1/6) log t), by adaptive quadrature in log t
        val, _ = quad(lambda u: math.exp(u) / (math.exp(u / 6) * u), math.log(2.0), math.log(x),
                      limit=200)
        return val

    c = -0.037
    curve = []
    for x in xs:
        p = int(x / (4 * math.log(x)))  # a stand-in for the primes == 5 mod 8 below x
        curve.append((int(x), p, int(round(p / 3 + c * li16(x)))))
    assert sweep.fit_prime_coefficient(curve, x_min=1e8) == pytest.approx(c, rel=2e-3)


def test_curve_from_journal_rows(tmp_path):
    j = sweep.Journal(str(tmp_path / "j.jsonl"))
    for (lo, hi), nD, nE in [((0, 16), 3, 1), ((16, 32), 4, 2), ((48, 64), 5, 5)]:
        j.add((lo, hi), nD, nE)
    # the curve stops at the first gap (block [32, 48) is missing)
    assert sweep.pi_E_curve(j, 0) == [(15, 3, 1), (31, 7, 3)]
