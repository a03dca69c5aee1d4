"""Pins of the oracle's multiple-scattering angle (PDG Highland formula, z = 1) against the
PDG's printed constants (tests/golden/pdg_highland.txt).

The constants are recovered from the oracle's outputs, not retyped into a second copy of the
formula: at one radiation length and beta -> 1 the logarithm vanishes and theta0 * p is the
scale itself; the ratio between two thicknesses isolates the logarithm's coefficient; and at one
radiation length the remaining momentum dependence is a function of beta alone, which is solved
for beta and compared with the velocity of a charged pion of the PDG mass.  A constant typed
wrongly into both the oracle and the event generator (which agree with each other by another
test) fails here."""
import math
import os

import pytest

import oracle
from paper_2312_11728_gb300 import synth as S

P_ULTRA = 1.0e5   # GeV: beta = 1 - 1e-12 for a pion


def _golden(name):
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle(S.geometry_barrel())


@pytest.fixture(scope="module")
def pdg():
    return _golden("pdg_highland.txt")


def test_scale_at_one_radiation_length(orc, pdg):
    """t = x/X0 = 1 and beta = 1: ln(t / beta^2) = 0, so theta0 * beta * p is the scale."""
    th = orc.theta0(P_ULTRA, 1.0)
    assert abs(th * P_ULTRA / pdg["scale_gev"] - 1.0) < 1e-9


@pytest.mark.parametrize("t", [1e-3, 1e-2, 0.3, 3.0, 30.0])
def test_log_coefficient_from_thickness_ratio(orc, pdg, t):
    """At beta = 1, theta0(t) / (sqrt(t) theta0(1)) = 1 + c ln t: c from each thickness of the
    PDG's stated range."""
    assert pdg["x_over_x0_lo"] <= t <= pdg["x_over_x0_hi"]
    r = orc.theta0(P_ULTRA, t) / (math.sqrt(t) * orc.theta0(P_ULTRA, 1.0))
    c = (r - 1.0) / math.log(t)
    assert abs(c / pdg["log_coefficient"] - 1.0) < 1e-9


@pytest.mark.parametrize("p", [0.08, 0.15, 0.3, 0.7, 2.0])
def test_velocity_is_that_of_a_pdg_pion(orc, pdg, p):
    """At t = 1, theta0 * p / scale = (1 - 2 c ln beta) / beta, strictly decreasing in beta on
    (0, 1]: solve it for beta by bisection and compare with p / sqrt(p^2 + m_pi^2)."""
    from scipy.optimize import brentq
    f = orc.theta0(p, 1.0) * p / pdg["scale_gev"]
    c = pdg["log_coefficient"]
    beta = brentq(lambda b: (1.0 - 2.0 * c * math.log(b)) / b - f, 1e-3, 1.0, xtol=1e-15, rtol=1e-15)
    m = pdg["pion_mass_gev"]
    assert abs(beta / (p / math.hypot(p, m)) - 1.0) < 1e-9

