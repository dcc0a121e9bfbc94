"""Derivation of the twelve-point candidate S6 of TENO12-AA -- TEST
INFRASTRUCTURE ONLY (part of the oracle).

The paper builds its very-high-order family recursively (Sec. 3.1): the
three small stencils plus symmetric large stencils of growing width; it
states that the framework extends to any width but prints coefficients
only up to the ten-point stencil S5.  This script derives S6 (offsets -5..6) the
way Sec. 4.1 and Sec. 4.2 describe the printed ones:

* the smoothness indicator beta_{6,12} from Eq. measureTENO, for the
  degree-11 polynomial whose cell averages are the twelve stencil values
  (Eq. definitionEq, Eq. approximatepolynomial), here through the primitive
  function: H(x_{j+1/2}) = sum_{k<=j} f_k is interpolated at the 13 cell
  boundaries and p = H'.  Exact rational arithmetic.
* the linear scheme as a dispersion part plus a dissipation part
  (Eq. difference_decomposition):
  - dispersion: the symmetric scheme whose modified wavenumber
    sum_m a_m sin(m xi) minimises Eq. weighted-error_integral under the
    accuracy-order constraints (exact for xi^1, zero error through
    xi^(order+1)); the integrals by numerical quadrature at 60 digits.
  - dissipation: a multiple of the (2r-1)-th undivided difference (the
    part antisymmetric about the face), sized by its coefficient on cell i.

Readings (the paper does not state them; each reproduces every printed
scheme to its printed digits, which the oracle tests check):
  nu = 6 for S3 and nu = 7 for S4 and S5, so nu = 7 for S6;
  accuracy constraint 4, 6, 8 for S3, S4, S5, so 10 for S6;
  antisymmetric coefficient on cell i 1/80 for S3 and 1/200 for S4 and S5,
  so 1/200 for S6.

Run from the repository root to rewrite the oracle's table header:
    python -m oracle.teno12_derive > oracle/teno12_tables.h
"""
from __future__ import annotations

from fractions import Fraction as Fr
import math

# ----------------------------------------------------------------------------
# polynomials with rational coefficients, ascending powers
# ----------------------------------------------------------------------------


def _pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def _padd(a, b, s=Fr(1)):
    n = max(len(a), len(b))
    a = list(a) + [Fr(0)] * (n - len(a))
    b = list(b) + [Fr(0)] * (n - len(b))
    return [x + s * y for x, y in zip(a, b)]


def _pder(a):
    return [a[k] * k for k in range(1, len(a))] or [Fr(0)]


def _pint_unit(a):
    """Integral over [-1/2, 1/2]."""
    tot = Fr(0)
    for k, c in enumerate(a):
        if k % 2 == 0:
            tot += c * 2 * Fr(1, 2) ** (k + 1) / (k + 1)
    return tot


def _lagrange_basis(nodes, i):
    p = [Fr(1)]
    for j, xj in enumerate(nodes):
        if j != i:
            p = _pmul(p, [-xj / (nodes[i] - xj), 1 / (nodes[i] - xj)])
    return p


def indicator_form(offsets):
    """Symmetric rational matrix Q (rows/columns in the order of `offsets`,
    consecutive cells, unit spacing, cell i centred at 0) with
    beta = f^T Q f for Eq. measureTENO on that stencil."""
    r = len(offsets)
    lo = offsets[0]
    assert list(offsets) == list(range(lo, lo + r))
    nodes = [Fr(2 * (lo + k) - 1, 2) for k in range(r + 1)]   # x_{lo-1/2} .. x_{hi+1/2}
    basis = [_lagrange_basis(nodes, k) for k in range(r + 1)]
    # f_j = unit -> H at nodes: H(x_{k}) = sum of cell values left of node k
    polys = []
    for j in range(r):
        Hn = [Fr(0)]
        for k in range(j + 1, r + 1):        # nodes right of cell j carry f_j
            Hn = _padd(Hn, basis[k])
        polys.append(_pder(Hn))              # p = H'
    Q = [[Fr(0)] * r for _ in range(r)]
    ders = [[p] for p in polys]
    for j in range(r):
        for _ in range(1, r):
            ders[j].append(_pder(ders[j][-1]))
    for a in range(r):
        for b in range(a, r):
            s = Fr(0)
            for m in range(1, r):
                s += _pint_unit(_pmul(ders[a][m], ders[b][m]))
            Q[a][b] = Q[b][a] = s
    return Q


# ----------------------------------------------------------------------------
# linear scheme on a symmetric stencil of 2r points (offsets -r+1 .. r)
# ----------------------------------------------------------------------------


def dispersion_weights(r, nu, order, dps=60):
    """a_1..a_r of the central scheme sum_m a_m sin(m xi) that minimises
    int_0^pi exp(nu (pi - xi)) (sum_m a_m sin(m xi) - xi)^2 dxi subject to
    sum_m a_m m = 1 and sum_m a_m m^(2k+1) = 0, k = 1 .. order/2 - 1
    (the accuracy-order constraint).  Returns mpmath numbers."""
    import mpmath as mp
    mp.mp.dps = dps
    nu = mp.mpf(nu)
    w = lambda x: mp.exp(nu * (mp.pi - x))
    G = mp.matrix(r, r)
    b = mp.matrix(r, 1)
    for i in range(1, r + 1):
        b[i - 1] = mp.quad(lambda x: w(x) * x * mp.sin(i * x), [0, mp.pi / 2, mp.pi])
        for j in range(i, r + 1):
            g = mp.quad(lambda x: w(x) * mp.sin(i * x) * mp.sin(j * x), [0, mp.pi / 2, mp.pi])
            G[i - 1, j - 1] = G[j - 1, i - 1] = g
    K = order // 2
    A = mp.matrix(r + K, r + K)
    rhs = mp.matrix(r + K, 1)
    for i in range(r):
        for j in range(r):
            A[i, j] = G[i, j]
        rhs[i] = b[i]
    for k in range(K):
        for m in range(1, r + 1):
            A[r + k, m - 1] = A[m - 1, r + k] = mp.mpf(m) ** (2 * k + 1)
        rhs[r + k] = 1 if k == 0 else 0
    sol = mp.lu_solve(A, rhs)
    return [sol[i] for i in range(r)]


def linear_scheme(r, nu, order, inner, dps=60):
    """Face-(i+1/2) coefficients c_j, j = -r+1 .. r, as mpmath numbers:
    symmetric part from dispersion_weights (pair j, 1-j carries
    s_j = 1/2 sum_{m>=j} a_m), plus the antisymmetric multiple of the
    (2r-1)-th difference whose coefficient on cell i is `inner`."""
    import mpmath as mp
    mp.mp.dps = dps
    a = dispersion_weights(r, nu, order, dps)
    s = {j: sum(a[m - 1] for m in range(j, r + 1)) / 2 for j in range(1, r + 1)}
    inner = Fr(inner)
    delta = mp.mpf(inner.numerator) / (inner.denominator * math.comb(2 * r - 1, r - 1))
    out = []
    for j in range(-r + 1, r + 1):
        sym = s[j] if j >= 1 else s[1 - j]
        anti = (-1) ** (j % 2) * math.comb(2 * r - 1, j + r - 1) * delta
        out.append(sym + anti)
    return out


S6_RECIPE = dict(r=6, nu=7, order=10, inner=Fr(1, 200))


def s6_tables():
    """(terms, coefficients): beta_{6,12} as (offset a, offset b, Fraction)
    for a <= b (the coefficient of f_a f_b, doubled off the diagonal), and
    the twelve S6 coefficients rounded to doubles."""
    offs = list(range(-5, 7))
    Q = indicator_form(offs)
    terms = []
    for ia, a in enumerate(offs):
        for ib in range(ia, len(offs)):
            c = Q[ia][ib] if ia == ib else 2 * Q[ia][ib]
            terms.append((a, offs[ib], c))
    R = S6_RECIPE
    lin = [float(x) for x in linear_scheme(R["r"], R["nu"], R["order"], R["inner"])]
    return terms, lin


def header_text():
    terms, lin = s6_tables()
    lines = [
        "/* Generated by oracle/teno12_derive.py -- do not edit.",
        " * TENO12-AA candidate S6 (offsets -5..6) of the oracle:",
        " *   B612: beta_{6,12} of Eq. measureTENO as exact reduced fractions",
        " *         num/den of f_a f_b (off-diagonal terms doubled);",
        " *   LIN6: the optimised linear scheme at face i+1/2 (nu = 7, accuracy",
        " *         constraint 10, antisymmetric coefficient 1/200 on cell i). */",
        "static const qterm2 B612[] = {",
    ]
    for a, b, c in terms:
        lines.append('    {%d, %d, "%d", "%d"},' % (a, b, c.numerator, c.denominator))
    lines.append("};")
    lines.append("static const double LIN6[12] = {")
    for k, x in enumerate(lin):
        lines.append("    %s,   /* %s, offset %d */" % (repr(x), x.hex(), k - 5))
    lines.append("};")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    import sys
    sys.stdout.write(header_text())
