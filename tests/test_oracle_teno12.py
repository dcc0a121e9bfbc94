"""Pins of the oracle's twelve-point candidate S6 (TENO12-AA): the next member
of the family the paper builds (Sec. 3.1), which it does not print.

The oracle derives S6 with oracle/teno12_derive.py.  These tests pin that
derivation to what the paper does print and to the mathematics:
* the same routines give back every printed large-stencil scheme (Eq.
  6-point, 8-point, 10-point) and every printed indicator (Eq. TENO10_AA);
* beta_{6,12} equals an independent exact derivation of Eq. measureTENO;
* S6 is consistent (coefficients sum to one), exactly tenth order, its
  antisymmetric part is the 11th difference at the stated size, and its
  symmetric part is stationary for Eq. weighted-error_integral at nu = 7
  (checked by double-precision quadrature, not by the derivation's own
  code).
"""
from fractions import Fraction as Fr
import math
import os
import warnings

import numpy as np
import pytest

import oracle
from test_oracle_coefficients import smoothness_form, _cell_avgs

mp = pytest.importorskip("mpmath")
from oracle import teno12_derive as D  # noqa: E402  (needs mpmath)

# (L, half-width r, nu, accuracy constraint, antisymmetric coefficient on cell i)
PRINTED = [(3, 3, 6, 4, Fr(1, 80)), (4, 4, 7, 6, Fr(1, 200)), (5, 5, 7, 8, Fr(1, 200))]


@pytest.mark.parametrize("L,r,nu,order,inner", PRINTED)
def test_recipe_reproduces_printed_schemes(L, r, nu, order, inner):
    """The Sec. 4.1 recipe with these readings gives the printed S3/S4/S5 to
    within their own rounding (the printed coefficient sums miss one by up
    to 7.5e-15); a neighbouring nu or constraint does not."""
    got = [float(x) for x in D.linear_scheme(r, nu, order, inner)]
    printed = [oracle.lin_coef(L, m) for m in range(-r + 1, r + 1)]
    assert max(abs(a - b) for a, b in zip(got, printed)) <= 2e-15
    for alt in ((nu - 1, order), (nu + 1, order), (nu, order - 2)):
        other = [float(x) for x in D.linear_scheme(r, alt[0], alt[1], inner)]
        assert max(abs(a - b) for a, b in zip(other, printed)) > 1e-6, alt


@pytest.mark.parametrize("width", [6, 8, 10])
def test_indicator_routine_reproduces_printed(width):
    """indicator_form (primitive-function route) equals every printed term."""
    J = list(range(-width // 2 + 1, width // 2 + 1))
    Q = D.indicator_form(J)
    for a, b, c in oracle.beta_fractions(width):
        ia, ib = J.index(a), J.index(b)
        assert c == (Q[ia][ia] if a == b else 2 * Q[ia][ib]), (width, a, b)


def test_beta612_matches_independent_derivation():
    """The oracle's beta_{6,12} terms equal the cell-average-inversion
    derivation of Eq. measureTENO in the coefficient tests, exactly."""
    J = list(range(-5, 7))
    Q = smoothness_form(J)
    terms = oracle.beta_fractions(12)
    assert len(terms) == 78
    for a, b, c in terms:
        ia, ib = J.index(a), J.index(b)
        assert c == (Q[ia][ia] if a == b else Q[ia][ib] + Q[ib][ia]), (a, b)
        assert oracle.beta_coef(12, a, b) == float(c)


def test_tables_header_is_current():
    path = os.path.join(os.path.dirname(oracle.__file__), "teno12_tables.h")
    assert open(path).read() == D.header_text()


def _lin6():
    return np.array([oracle.lin_coef(6, m) for m in range(-5, 7)])


def test_s6_consistency_and_dissipation_part():
    c = _lin6()
    assert abs(c.sum() - 1.0) <= 2e-15
    offs = np.arange(-5, 7)
    anti = 0.5 * (c - c[::-1])            # pairs offset j with 1 - j
    want = np.array([(-1.0) ** (j % 2) * math.comb(11, j + 5) for j in offs]) / 92400.0
    # to the rounding of the doubles (an ulp of the largest coefficient, 1.1e-16)
    assert np.abs(anti - want).max() <= 1.2e-16
    assert anti[5] == pytest.approx(0.005, abs=1.2e-16)     # cell i: 1/200


def test_s6_is_exactly_tenth_order():
    p = oracle.params(1, [16], [1.0], scheme=12)
    offs = list(range(-5, 7))
    s = Fr(1, 5)
    for k in range(11):
        _, fh = oracle.betas(p, _cell_avgs(k, s, offs))
        err = abs(fh[6] - float((s / 2) ** k))
        assert (err <= 1e-14) if k < 10 else (err > 1e-12), (k, err)


def _stationarity_step(c, nu):
    """Newton step of Eq. weighted-error_integral along the one direction the
    accuracy constraints leave free, from the symmetric part of c."""
    from scipy.integrate import quad
    r = len(c) // 2
    s = [0.5 * (c[r - 1 + j] + c[r - j]) for j in range(1, r + 1)] + [0.0]
    a = np.array([2 * (s[m - 1] - s[m]) for m in range(1, r + 1)])
    ms = np.arange(1, r + 1)
    C = np.array([ms ** (2 * k + 1) for k in range(r - 1)], float)
    n = np.linalg.svd(C)[2][-1]                      # null direction
    w = lambda x: math.exp(nu * (math.pi - x))
    xr = lambda x: float(np.dot(a, np.sin(ms * x)))
    nn = lambda x: float(np.dot(n, np.sin(ms * x)))
    with warnings.catch_warnings():        # quad notes its own roundoff limit
        warnings.simplefilter("ignore")
        g = quad(lambda x: w(x) * (xr(x) - x) * nn(x), 0, math.pi, limit=400, epsabs=0,
                 epsrel=1e-12)[0]
        h = quad(lambda x: w(x) * nn(x) ** 2, 0, math.pi, limit=400, epsabs=0, epsrel=1e-12)[0]
    return abs(g / h)


def test_s6_dispersion_part_is_optimal_at_nu7():
    """E is stationary at the derived S6 for nu = 7 (to the rounding of the
    doubles, which the tenth-order constraints amplify) and is not for
    nu = 6, 8 (steps of 0.03-0.04)."""
    c = _lin6()
    assert _stationarity_step(c, 7.0) < 1e-9
    assert _stationarity_step(c, 6.0) > 1e-3
    assert _stationarity_step(c, 8.0) > 1e-3


@pytest.mark.parametrize("L,r,nu", [(3, 3, 6.0), (4, 4, 7.0), (5, 5, 7.0)])
def test_printed_schemes_are_optimal_for_their_nu(L, r, nu):
    """The same stationarity check on the printed schemes, and its failure
    one unit of nu away."""
    c = [oracle.lin_coef(L, m) for m in range(-r + 1, r + 1)]
    assert _stationarity_step(c, nu) < 1e-9
    assert _stationarity_step(c, nu + 1.0) > 1e-3


def test_fallback_never_writes_the_s6_pattern():
    """S6 is written with bits 0-4 zero; a fallback keeps at least one small
    stencil, so its cut-off bits are never all zero.  Every byte read as S6
    carries exactly the S6 value (a fallback with no stencil kept would give
    NaN), over random, step and smooth data of magnitudes 1e-30 .. 1e30."""
    p = oracle.params(1, [16], [1.0], scheme=12)
    g = np.random.Generator(np.random.PCG64(1201))
    offs = np.arange(-5, 7)
    seen_s6 = seen_fb = 0
    for t in range(3000):
        scale = 10.0 ** g.uniform(-30, 30)
        v = g.normal(size=12) * scale
        if t % 3 == 1:
            v = np.where(offs >= g.integers(-5, 7), 1.0, 0.0) * scale + 1e-3 * scale * g.normal(size=12)
        if t % 3 == 2:
            v = np.sin(g.uniform(0.05, 1.5) * offs) * scale
        val, fl = oracle.recon(p, v)
        sel, dl, _ = oracle.decode_flag(fl)
        if sel == 6:
            seen_s6 += 1
            assert val == oracle.betas(p, v)[1][6]
        if sel == 0:
            seen_fb += 1
            assert dl != (0, 0, 0)
    assert seen_s6 > 100 and seen_fb > 100
