"""Pins of the oracle's coefficient tables and scalar reconstruction against what
the paper fixes (arXiv 2109.14340, Sec. 3-4): exact rational re-derivation of
every smoothness indicator from Eq. measureTENO, the stated orders of the
candidate schemes, the small-stencil weights, the C_T map endpoints (Sec. 3.4)
and hand-checkable ENO-like selections (Sec. 3.3)."""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

import oracle


# --------------------------------------------------------------------------
# exact rational derivation of Eq. measureTENO for a stencil of offsets J
# --------------------------------------------------------------------------

def _cell_avg_monomial(j, l):
    """Average of x^l over cell j = [j-1/2, j+1/2] (unit spacing)."""
    a, b = Fr(2 * j - 1, 2), Fr(2 * j + 1, 2)
    return (b ** (l + 1) - a ** (l + 1)) / (l + 1)


def _inverse(A):
    n = len(A)
    M = [row[:] + [Fr(int(i == k)) for k in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [x * inv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [row[n:] for row in M]


def smoothness_form(J):
    """Symmetric rational Q with beta = f^T Q f for the stencil offsets J: the
    polynomial of degree r-1 whose cell averages are f (Eq. definitionEq and
    Eq. approximatepolynomial) and beta = sum_m int_{-1/2}^{1/2} (p^(m))^2."""
    r = len(J)
    A = [[_cell_avg_monomial(j, l) for l in range(r)] for j in J]
    M = _inverse(A)                       # a = M f

    def integral(k):
        if k % 2:
            return Fr(0)
        return 2 * Fr(1, 2) ** (k + 1) / (k + 1)

    G = [[Fr(0)] * r for _ in range(r)]
    for m in range(1, r):
        for l1 in range(m, r):
            c1 = Fr(math.factorial(l1), math.factorial(l1 - m))
            for l2 in range(m, r):
                c2 = Fr(math.factorial(l2), math.factorial(l2 - m))
                G[l1][l2] += c1 * c2 * integral(l1 + l2 - 2 * m)
    Q = [[sum(M[l1][a] * G[l1][l2] * M[l2][b] for l1 in range(r) for l2 in range(r))
          for b in range(r)] for a in range(r)]
    return Q


STENCILS = {6: list(range(-2, 4)), 8: list(range(-3, 5)), 10: list(range(-4, 6))}


@pytest.mark.parametrize("width", [6, 8, 10])
def test_beta_tables_rederived_exactly(width):
    """Every printed integer of Eq. TENO10_AA equals the exact derivation."""
    J = STENCILS[width]
    Q = smoothness_form(J)
    terms, den = oracle.beta_terms(width)
    seen = set()
    for a, b, c in terms:
        ia, ib = J.index(a), J.index(b)
        want = Q[ia][ia] if a == b else Q[ia][ib] + Q[ib][ia]
        assert Fr(c, den) == want, (width, a, b)
        seen.add((min(a, b), max(a, b)))
    assert len(seen) == width * (width + 1) // 2 == len(terms)


@pytest.mark.parametrize("width", [6, 8, 10])
def test_coefficients_correctly_rounded(width):
    """Table doubles are the round-to-nearest of c/D (Python int division is
    correctly rounded)."""
    terms, den = oracle.beta_terms(width)
    for a, b, c in terms:
        assert oracle.beta_coef(width, a, b) == c / den
        assert oracle.round_ratio(c, den) == c / den


def test_round_ratio_random():
    g = np.random.Generator(np.random.PCG64(7))
    for _ in range(2000):
        num = int(g.integers(-2**62, 2**62)) * int(g.integers(1, 2**40)) + int(g.integers(0, 2**20))
        den = int(g.integers(1, 2**52))
        assert oracle.round_ratio(num, den) == num / den


def _exact_beta(Q, f):
    fr = [Fr(x) for x in f]
    return float(sum(Q[a][b] * fr[a] * fr[b] for a in range(len(f)) for b in range(len(f))))


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_beta_evaluation_matches_exact(scheme):
    """The six indicators as evaluated by the oracle agree with the exact
    rational forms (small ones derived the same way from Eq. measureTENO)."""
    p = oracle.params(1, [16], [1.0], scheme=scheme)
    H = scheme // 2
    offs = list(range(-H + 1, H + 1))
    forms = {0: ([-1, 0, 1], smoothness_form([-1, 0, 1])),
             1: ([0, 1, 2], smoothness_form([0, 1, 2])),
             2: ([-2, -1, 0], smoothness_form([-2, -1, 0])),
             3: (STENCILS[6], smoothness_form(STENCILS[6])),
             4: (STENCILS[8], smoothness_form(STENCILS[8]))}
    if scheme >= 10:
        forms[5] = (STENCILS[10], smoothness_form(STENCILS[10]))
    if scheme == 12:
        forms[6] = (list(range(-5, 7)), smoothness_form(list(range(-5, 7))))
    g = np.random.Generator(np.random.PCG64(11))
    for trial in range(60):
        v = g.uniform(-1, 1, 2 * H) * (10.0 ** g.uniform(-3, 3))
        if trial % 3 == 0:
            v = v + 1e3 * g.uniform(-1, 1)            # large common offset
        beta, _ = oracle.betas(p, v)
        for k, (J, Q) in forms.items():
            f = [v[offs.index(j)] for j in J]
            ex = _exact_beta(Q, f)
            # FP64 bound: the differences inside the form carry an absolute
            # error of a few ulps of max|v|, amplified by 2 sqrt(beta).
            vmax = float(np.max(np.abs(v)))
            tol = 1e-12 * abs(ex) + 1e-13 * vmax * math.sqrt(abs(ex)) * 100
            assert abs(beta[k] - ex) <= tol, (k, trial, beta[k], ex)


def _cell_avgs(k, s, offs):
    """Cell averages of h(x) = (s x)^k, exactly, as doubles."""
    return np.array([float(Fr(s) ** k * _cell_avg_monomial(j, k)) for j in offs])


@pytest.mark.parametrize("L,order", [(0, 3), (1, 3), (2, 3), (3, 4), (4, 6), (5, 8), (6, 10)])
def test_candidate_flux_orders(L, order):
    """f_0..f_2 are third order, S3/S4/S5 are fourth/sixth/eighth order
    (Sec. 4.1), the derived S6 tenth: exact at the face x = 1/2 for
    polynomials of degree < order, and not for degree = order."""
    scheme = 12 if L == 6 else 10
    p = oracle.params(1, [16], [1.0], scheme=scheme)
    offs = list(range(-scheme // 2 + 1, scheme // 2 + 1))
    s = Fr(1, 5)
    for k in range(order + 1):
        v = _cell_avgs(k, s, offs)
        _, fh = oracle.betas(p, v)
        exact = float((s / 2) ** k)
        err = abs(fh[L] - exact)
        if k < order:
            assert err <= 1e-14, (L, k, err)
        else:
            assert err > 1e-11, (L, k, err)


def test_small_weights():
    """d_k of Sec. 4.1 sum to one (10 printed digits); the blended five-point
    scheme is exact for quadratics only (third order)."""
    d = np.array([0.5065006634, 0.3699651429, 0.1235341937])
    assert abs(d.sum() - 1.0) < 1e-10
    p = oracle.params(1, [16], [1.0], scheme=10)
    offs = list(range(-4, 6))
    s = Fr(1, 5)
    for k in range(4):
        _, fh = oracle.betas(p, _cell_avgs(k, s, offs))
        blend = d @ fh[:3]
        err = abs(blend - float((s / 2) ** k))
        assert (err < 1e-10) if k < 3 else (err > 1e-9)


# --------------------------------------------------------------------------
# C_T map (Sec. 3.4) and ENO-like selection (Sec. 3.3) on hand-checkable data
# --------------------------------------------------------------------------

def _recon(scheme, v):
    p = oracle.params(1, [16], [1.0], scheme=scheme)
    val, fl = oracle.recon(p, np.asarray(v, float))
    return val, oracle.decode_flag(fl)


@pytest.mark.parametrize("scheme", [8, 10])
def test_ct_endpoints(scheme):
    """m = 0 (smooth: equal first differences, eta = 1) gives C_T = 1e-14;
    m = 1 (a jump next to flat data, eta ~ 0) gives C_T = 1e-7."""
    H = scheme // 2
    offs = np.arange(-H + 1, H + 1)
    _, (sel, _, ct) = _recon(scheme, 0.3 * offs + 2.0)
    assert ct == 14 and sel == H
    v = np.where(offs >= 1, 1.0, 0.0)
    _, (sel, _, ct) = _recon(scheme, v)
    assert ct == 7


def test_ct_worked_example():
    """A face whose smallest eta is 2t/(1+t^2) with t = 1/4 (first differences
    1,1,1,1/4 ... arranged so the other three etas are 1 or larger):
    eta = 8/17, r = eta/0.265 > 1 so m = 0 and C_T = 1e-14; with t = 1/20:
    eta = 40/401, m = 1 - eta/0.265 = 0.6236..., g = (1-m)^4 (1+4m) = 0.0696...,
    beta = 14 - 6.4 (1 - g) = 8.045..., C_T = 1e-8."""
    for t, want in ((0.25, 14), (0.05, 8)):
        # differences Delta_{-3/2..5/2} = 1, 1, t, t, t  ->  etas at -1,0,1,2:
        # eta_-1 = 1, eta_0 = 2t/(1+t^2), eta_1 = 1, eta_2 = 1
        d = [1.0, 1.0, t, t, t]
        v = np.zeros(10)
        offs = list(range(-4, 6))
        v[offs.index(-2)] = 0.0
        for k, m in enumerate(range(-2, 3)):
            v[offs.index(m + 1)] = v[offs.index(m)] + d[k]
        for m in (-3, -4):
            v[offs.index(m)] = v[offs.index(m + 1)] - 1.0
        for m in (4, 5):
            v[offs.index(m)] = v[offs.index(m - 1)] + t
        _, (_, _, ct) = _recon(10, v)
        assert ct == want, (t, ct)


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_selection_on_steps(scheme):
    """A unit step placed between offsets s-1 and s: the large stencils that
    straddle it are dropped (largest first) and the small-stencil cut-offs
    drop exactly the small stencils that straddle it."""
    H = scheme // 2
    offs = np.arange(-H + 1, H + 1)
    expect = {
        2: (0, (1, 0, 1)),       # step inside S1 = {0,1,2} only
        3: (0, (1, 1, 1)),       # only the large stencils straddle it
        4: (3, None),            # S3 = -2..3 is smooth
        0: (0, (0, 1, 0)),       # step between -1 and 0: S0, S2 straddle
        -1: (0, (1, 1, 0)),      # step between -2 and -1: only S2 straddles
    }
    expect[-2] = (3, None)       # step between -3 and -2: S3 smooth, S4.. not
    if scheme >= 10:
        expect[5] = (4, None)    # S4 = -3..4 smooth, S5 straddles
        expect[-3] = (4, None)   # step between -4 and -3: S4 smooth
    if scheme == 12:
        expect[6] = (5, None)    # S5 = -4..5 smooth, S6 straddles
        expect[-4] = (5, None)   # step between -5 and -4: S5 smooth
    for s, (sel_w, deltas) in expect.items():
        v = np.where(offs >= s, 1.0, 0.0)
        val, (sel, dl, ct) = _recon(scheme, v)
        assert sel == sel_w, (s, sel)
        if deltas is not None:
            assert dl == deltas, (s, dl)
        if sel_w == 0 and deltas == (1, 0, 1):
            # renormalised weights d0, d2 on the two smooth stencils
            d = np.array([0.5065006634, 0.3699651429, 0.1235341937])
            w = np.array([d[0], 0, d[2]]) / (d[0] + d[2])
            p = oracle.params(1, [16], [1.0], scheme=scheme)
            _, fh = oracle.betas(p, v)
            assert val == pytest.approx(w @ fh[:3], rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_smooth_data_selects_largest(scheme):
    """Smooth data: the largest stencil is selected and the output is exactly
    its linear scheme (TENO reverts to the linear scheme, Sec. 3.3)."""
    H = scheme // 2
    offs = np.arange(-H + 1, H + 1)
    p = oracle.params(1, [16], [1.0], scheme=scheme)
    for k in (0.1, 0.3, 0.7):
        v = np.sin(k * offs) + 0.5
        val, fl = oracle.recon(p, v)
        sel, _, _ = oracle.decode_flag(fl)
        assert sel == H
        _, fh = oracle.betas(p, v)
        assert val == fh[H]
