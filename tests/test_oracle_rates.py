"""Pins of the oracle's ionisation rates (Sec. II: step-wise ionisation from
the cell's electron density and temperature, Maxwellian EEDF).

The rate datasets [20-23] are not available; the oracle integrates the
single-term Lotz cross section over a Maxwellian by quadrature.  For that cross
section the average has the closed form
    k = sqrt(8 e/(pi m_e)) a q E1(P/T) / ((P/T) T^1.5),
with E1 the exponential integral, used here through scipy.
"""
import math

import numpy as np
import pytest
from scipy.special import exp1

from oracle import oracle as O
from paper_1507_03392_gb300 import inputs as I

QE = 1.602176634e-19
ME = 9.1093837015e-31


def closed_form(P, q, T):
    a = 4.5e-18  # m^2 eV^2
    x = P / T
    return math.sqrt(8 * QE / (math.pi * ME)) * a * q * exp1(x) / (x * T ** 1.5)


@pytest.mark.parametrize("P,q,T", [(30.6, 8, 1000.0), (30.6, 8, 5.0), (422.0, 8, 1000.0),
                                   (4400.0, 1, 3000.0), (41.7, 6, 300.0), (150.0, 2, 20.0)])
def test_lotz_quadrature_matches_closed_form(P, q, T):
    assert O.lotz_rate(P, q, T) == pytest.approx(closed_form(P, q, T), rel=2e-6)


def test_argon_neutral_rate_magnitude():
    # Sec. III B: Ar0 ionisation rate ~1e-7 cm^3/s at ~1 keV
    ip, nout = I.ARGON.ladder()
    k = O.lotz_rate(ip[0], nout[0], 1000.0) * 1e6
    assert 3e-8 < k < 3e-7


def test_rates_fall_with_charge_state():
    ip, nout = I.ARGON.ladder()
    ks = [O.lotz_rate(ip[q], nout[q], 1000.0) for q in range(18)]
    assert all(ks[i + 1] < ks[i] for i in range(17))
