"""Write teno_coeffs.cuh: the smoothness-indicator quadratic forms of the
eight/ten-point TENO-AA schemes (arXiv 2109.14340, Sec. 4.2, Eq. TENO10_AA)
as doubles, each the round-to-nearest of the printed integer over the printed
denominator (Python's int / int division is correctly rounded); and the
twelve-point candidate S6 of TENO12-AA -- the next member of the family the
paper builds (Sec. 3.1), which it does not print -- derived here:
* beta_{6,12} from Eq. measureTENO (exact rationals: the degree-11
  polynomial with the stencil's cell averages, by inverting the cell-average
  moment matrix), stored like the printed forms;
* its linear scheme by the recipe of Sec. 4.1: a central part minimising
  Eq. weighted-error_integral under the accuracy-order constraint (integrals
  in closed form, 60-digit arithmetic) plus a multiple of the 11th
  undivided difference, with the parameters that give back the printed
  S3, S4, S5 (nu = 6, 7, 7; constraints 4, 6, 8; coefficient 1/80, 1/200,
  1/200 of the difference part on cell i): nu = 7, constraint 10, 1/200.
  Generation checks that the same routine reproduces the printed schemes.

Layout: upper triangle in ascending stencil offset, Q<w>[r][c] for r <= c,
offset = index + lo (lo = -2, -3, -4, -5 for widths 6, 8, 10, 12); zeros
below.  Needs mpmath (generation only; the output is committed).
Run:  python gen_coeffs.py > teno_coeffs.cuh
"""

# Printed terms: (offset a, offset b, integer) meaning integer * f_a * f_b.
W6 = (120960, -2, [
    (-2, -2, 271779), (-2, -1, -2380800), (-2, 0, 4086352), (-2, 1, -3462252),
    (-2, 2, 1458762), (-2, 3, -245620), (-1, -1, 5653317), (-1, 0, -20427884),
    (-1, 1, 17905032), (-1, 2, -7727988), (-1, 3, 1325006), (0, 0, 19510972),
    (0, 1, -35817664), (0, 2, 15929912), (0, 3, -2792660), (1, 1, 17195652),
    (1, 2, -15880404), (1, 3, 2863984), (2, 2, 3824847), (2, 3, -1429976),
    (3, 3, 139633)])

W8 = (62270208000, -3, [
    (4, 4, 75349098471), (4, 3, -1078504915264), (4, 2, 3263178215782),
    (4, 1, -5401061230160), (4, 0, 5274436892970), (4, -1, -3038037798592),
    (4, -2, 956371298594), (4, -3, -127080660272),
    (3, 3, 3944861897609), (3, 2, -24347015748304), (3, 1, 41008808432890),
    (3, 0, -40666174667520), (3, -1, 23740865961334), (3, -2, -7563868580208),
    (3, -3, 1016165721854),
    (2, 2, 38342902371231), (2, 1, -131738583368480), (2, 0, 133017910915250),
    (2, -1, -78915800051952), (2, -2, 25505661974314), (2, -3, -3471156679072),
    (1, 1, 115593819531025), (1, 0, -238366288500400), (1, -1, 144163939468910),
    (1, -2, -47407534412640), (1, -3, 6553080547830),
    (0, 0, 125743620342175), (0, -1, -155660468395520), (0, -2, 52279668813670),
    (0, -3, -7366325742800),
    (-1, -1, 49429163447121), (-1, -2, -34065661645264), (-1, -3, 4916835566842),
    (-2, -2, 6047605530599), (-2, -3, -1799848509664),
    (-3, -3, 139164877641)])

W10 = (8002967132160000, -4, [
    (5, 5, 10271226852556519), (5, 4, -188781685190428812),
    (5, 3, 763744975064517708), (5, 2, -1783557622547881452),
    (5, 1, 2647293374939748168), (5, 0, -2588349166844242788),
    (5, -1, 1666621903133989812), (5, -2, -681536822065683108),
    (5, -3, 160665441665569002), (5, -4, -16642851860701568),
    (4, 4, 878723894536476309), (4, 3, -7196903757161570412),
    (4, 2, 16998197062674090348), (4, 1, -25496314580012763492),
    (4, 0, 25171844359828276512), (4, -1, -16354640170583096868),
    (4, -2, 6744593557304053812), (4, -3, -1602760184146136448),
    (4, -4, 167317608214622742),
    (3, 3, 14917582508640112584), (3, 2, -71318426816839529952),
    (3, 1, 108212250511882175688), (3, 0, -108001260086756280408),
    (3, -1, 70886485695552144912), (3, -2, -29512192424763178368),
    (3, -3, 7076170986963512652), (3, -4, -745034101222016988),
    (2, 2, 86303482562247542424), (2, 1, -265161231242943624792),
    (2, 0, 267840170248801834152), (2, -1, -177812140823999192448),
    (2, -2, 74826544942103527152), (2, -3, -18122888431675718748),
    (2, -4, 1926367559931410892),
    (1, 1, 206327958083635665564), (1, 0, -422297341631652106368),
    (1, -1, 283934849707927541592), (1, -2, -120940245081713867688),
    (1, -3, 29628242804292093792), (1, -4, -3183420029990528028),
    (0, 0, 219076505295455164644), (0, -1, -298732736184126553512),
    (0, -2, 128985549388044842808), (0, -3, -32013238878488743452),
    (0, -4, 3482351360282643768),
    (-1, -1, 103357453544031038184), (-1, -2, -90608758883967297312),
    (-1, -3, 22823791389362998548), (-1, -4, -2518379721362611092),
    (-2, -2, 20182234533315641784), (-2, -3, -10338186802053144852),
    (-2, -4, 1159763060479463988),
    (-3, -3, 1348293007163766699), (-3, -4, -308382340247963892),
    (-4, -4, 18029727887840089)])


# Printed large-stencil schemes (Sec. 4.1, Eqs. 6-, 8-, 10-point), used here
# only to check the S6 recipe.
PRINTED_LIN = {
    3: [0.02852274270130377, -0.1714015614372447, 0.650378818735941,
        0.6253788187359414, -0.1589015614372448, 0.02602274270130375],
    4: [-0.006866688980568011, 0.05128582585522106, -0.1968478198727312,
        0.6552858258552222, 0.6452858258552218, -0.1908478198727314,
        0.04928582585522098, -0.006580974694853729],
    5: [0.001911786299492748, -0.0170332977472532, 0.07339445614860979,
        -0.221228429084247, 0.6657332621611695, 0.6557332621611695,
        -0.2145617624175796, 0.07053731329146805, -0.01631901203296621,
        0.001832421220128962],
}


def indicator_spec(lo, w):
    """(den, lo, terms) of Eq. measureTENO on cells lo .. lo+w-1: the
    polynomial p of degree w-1 whose averages over cells [j-1/2, j+1/2] are
    the stencil values, beta = sum_{m=1}^{w-1} int_{-1/2}^{1/2} (p^(m))^2 dx;
    terms (a, b, integer) as in the printed forms (off-diagonal coefficient
    of f_a f_b in full), one common denominator."""
    from fractions import Fraction as Fr
    from math import factorial, lcm
    offs = list(range(lo, lo + w))
    # moment matrix A[j][l] = average of x^l over cell j, inverted exactly
    A = [[(Fr(2 * j + 1, 2) ** (l + 1) - Fr(2 * j - 1, 2) ** (l + 1)) / (l + 1)
          for l in range(w)] + [Fr(int(k == i)) for k in range(w)] for i, j in enumerate(offs)]
    for c in range(w):
        piv = next(r for r in range(c, w) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        A[c] = [x / A[c][c] for x in A[c]]
        for r in range(w):
            if r != c and A[r][c] != 0:
                A[r] = [x - A[r][c] * y for x, y in zip(A[r], A[c])]
    Minv = [row[w:] for row in A]          # monomial coefficients = Minv f
    # Gram matrix of the derivatives in the monomial basis
    def mono_int(k):
        return Fr(0) if k % 2 else Fr(2, (k + 1) * 2 ** (k + 1))
    G = [[Fr(0)] * w for _ in range(w)]
    for m in range(1, w):
        for l1 in range(m, w):
            for l2 in range(m, w):
                G[l1][l2] += (Fr(factorial(l1), factorial(l1 - m)) * Fr(factorial(l2), factorial(l2 - m))
                              * mono_int(l1 + l2 - 2 * m))
    Q = [[sum(Minv[l1][a] * G[l1][l2] * Minv[l2][b] for l1 in range(w) for l2 in range(w))
          for b in range(w)] for a in range(w)]
    coef = {}
    for ia in range(w):
        for ib in range(ia, w):
            coef[(offs[ia], offs[ib])] = Q[ia][ia] if ia == ib else Q[ia][ib] + Q[ib][ia]
    den = 1
    for c in coef.values():
        den = lcm(den, c.denominator)
    return (den, lo, [(a, b, int(c * den)) for (a, b), c in coef.items()])


def optimised_scheme(r, nu, order, inner):
    """Face coefficients on offsets -r+1 .. r (Sec. 4.1): central part
    sum_m a_m sin(m xi) minimising int_0^pi e^(nu (pi - xi)) (sum_m a_m
    sin(m xi) - xi)^2 dxi with sum_m a_m m = 1 and sum_m a_m m^(2k+1) = 0 for
    k = 1 .. order/2 - 1; plus inner / C(2r-1, r-1) times the (2r-1)-th
    difference (-1)^j C(2r-1, j+r-1).  The integrals in closed form with
    t = pi - xi:  J0(z) = int_0^pi e^(zt) dt, J1(z) = int_0^pi t e^(zt) dt,
    z = nu - i m."""
    import mpmath as mp
    from fractions import Fraction as Fr
    from math import comb
    mp.mp.dps = 60
    nu = mp.mpf(nu)
    pi = mp.pi

    def J0(z):
        return (mp.exp(z * pi) - 1) / z

    def J1(z):
        return mp.exp(z * pi) * (pi / z - 1 / z ** 2) + 1 / z ** 2

    def Ck(k):                              # int e^(nu(pi-xi)) cos(k xi)
        return mp.re((-1) ** k * J0(mp.mpc(nu, -k))) if k else mp.re(J0(mp.mpc(nu, 0)))

    K = order // 2
    n = r + K
    A = mp.matrix(n, n)
    rhs = mp.matrix(n, 1)
    for i in range(1, r + 1):
        rhs[i - 1] = mp.im((-1) ** i * (pi * J0(mp.mpc(nu, -i)) - J1(mp.mpc(nu, -i))))
        for j in range(1, r + 1):
            A[i - 1, j - 1] = (Ck(abs(i - j)) - Ck(i + j)) / 2
        for k in range(K):
            A[i - 1, r + k] = A[r + k, i - 1] = mp.mpf(i) ** (2 * k + 1)
    rhs[r] = 1
    sol = mp.lu_solve(A, rhs)
    a = [sol[m] for m in range(r)]
    inner = Fr(inner)
    unit = mp.mpf(inner.numerator) / (inner.denominator * comb(2 * r - 1, r - 1))
    out = []
    for j in range(-r + 1, r + 1):
        pair = j if j >= 1 else 1 - j       # offsets j and 1-j share the central part
        central = sum(a[m - 1] for m in range(pair, r + 1)) / 2
        out.append(float(central + (-1) ** (j % 2) * comb(2 * r - 1, j + r - 1) * unit))
    return out


def s6_scheme():
    """S6 (offsets -5..6) after checking the recipe on the printed S3-S5 (to
    their own rounding, 2e-15)."""
    for L, nu, order, inner in ((3, 6, 4, "1/80"), (4, 7, 6, "1/200"), (5, 7, 8, "1/200")):
        got = optimised_scheme(L, nu, order, inner)
        assert max(abs(x - y) for x, y in zip(got, PRINTED_LIN[L])) <= 2e-15, L
    return optimised_scheme(6, 7, 10, "1/200")


def check_printed_indicators():
    """The indicator routine reproduces the printed forms exactly."""
    for spec in (W6, W8, W10):
        den, lo, terms = spec
        dd, _, tt = indicator_spec(lo, -2 * lo + 2)
        mine = {(min(a, b), max(a, b)): c for a, b, c in tt}
        for a, b, c in terms:
            assert c * dd == mine[(min(a, b), max(a, b))] * den, (lo, a, b)


def table(spec):
    den, lo, terms = spec
    w = -2 * lo + 2
    M = [[0.0] * w for _ in range(w)]
    seen = set()
    for a, b, c in terms:
        r, s = min(a, b) - lo, max(a, b) - lo
        assert (r, s) not in seen
        seen.add((r, s))
        M[r][s] = c / den
    assert len(seen) == w * (w + 1) // 2
    return w, M


def sym_norms(M, lo, w):
    """Spectral norms of the symmetric matrix A (beta = s^T A s) of an upper-
    triangular form M on the shifted values (offset 0 removed, since its
    shifted value is zero), and of |A|; rounded up by 1 %."""
    import numpy as np
    idx = [r for r in range(w) if r + lo != 0]
    A = np.zeros((len(idx), len(idx)))
    for a, r in enumerate(idx):
        for b, c in enumerate(idx):
            if r == c:
                A[a, b] = M[r][r]
            elif r < c:
                A[a, b] = A[b, a] = M[r][c] / 2.0
    n1 = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    n2 = float(np.max(np.abs(np.linalg.eigvalsh(np.abs(A)))))
    return n1 * 1.01, n2 * 1.01


def ldl_factors(spec):
    """Exact rational L D L^T of the indicator form on the shifted values
    (offset 0 removed), variables in DESCENDING offset: beta = sum_i D_i y_i^2
    with y_i = sum_{m >= i} L[m][i] s_{off(m)}.  Every D_i > 0 (the form is
    positive definite).  The descending order gives the smaller single-
    precision error bounds on smooth data."""
    from fractions import Fraction as Fr
    den, lo, terms = spec
    w = -2 * lo + 2
    idx = [r for r in range(w) if r + lo != 0][::-1]
    M = {}
    for a, b, c in terms:
        M[(min(a, b) - lo, max(a, b) - lo)] = Fr(c, den)
    n = len(idx)
    A = [[Fr(0)] * n for _ in range(n)]
    for i, r in enumerate(idx):
        for j, t in enumerate(idx):
            if r == t:
                A[i][j] = M[(r, r)]
            else:
                A[i][j] = M[(min(r, t), max(r, t))] / 2
    L = [[Fr(int(i == j)) for j in range(n)] for i in range(n)]
    D = [Fr(0)] * n
    for j in range(n):
        D[j] = A[j][j] - sum(L[j][k] ** 2 * D[k] for k in range(j))
        assert D[j] > 0
        for i in range(j + 1, n):
            L[i][j] = (A[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    return [r + lo for r in idx], L, D


def f32_up(x):
    """Smallest float32 >= x (x > 0)."""
    import numpy as np
    f = np.float32(x)
    if float(f) < x:
        f = np.nextafter(f, np.float32(np.inf))
    return float(f)


def sos_tables(name, spec, qnorm_abs):
    """Float tables of the sum-of-squares form and the constants of its
    error bound (scaled units, every |f_m| < 2):
      beta <= beta~ (1 + (n+3) u) + TAU2 sum_i DC_i |y~_i| + K0,
    u = 2^-24, tau = 24 u bounds |y~_i - y_i| / C_i with C_i = sum_m |L~_mi|,
    TAU2 = 2 tau (1 + 4u), DC_i >= D~_i C_i, and K0 >= tau^2 (1 + 2u)
    sum_i D~_i C_i^2 + 24 2^-53 |||A|||_2 4.01 n (the double-precision
    evaluation of the printed form on the same shifted values) + 1e-30
    (underflow)."""
    import numpy as np
    offs, L, D = ldl_factors(spec)
    n = len(offs)
    Lf = [[float(np.float32(float(L[i][j]))) for j in range(n)] for i in range(n)]
    Df = [float(np.float32(float(d))) for d in D]
    C = [sum(abs(Lf[m][i]) for m in range(i, n)) for i in range(n)]
    u = 2.0 ** -24
    tau = 24 * u
    DC = [f32_up(Df[i] * C[i] * (1 + 4 * u)) for i in range(n)]
    k0 = (tau ** 2 * (1 + 2 * u) * sum(Df[i] * C[i] ** 2 for i in range(n)) +
          24 * 2.0 ** -53 * qnorm_abs * 4.01 * n + 1e-30) * 1.01
    out = ["// %s: sum-of-squares form of the large stencil's indicator, variables"
           " at offsets %s" % (name, offs)]
    out.append("static __constant__ float %s_L[%d][%d] = {" % (name, n, n))
    for i in range(n):
        out.append("    {" + ", ".join((float.hex(Lf[i][j]) + "f") if j <= i else "0.0f"
                                       for j in range(n)) + "},")
    out.append("};")
    out.append("static __constant__ float %s_D[%d] = {" % (name, n) +
               ", ".join(float.hex(d) + "f" for d in Df) + "};")
    out.append("static __constant__ float %s_DC[%d] = {" % (name, n) +
               ", ".join(float.hex(d) + "f" for d in DC) + "};")
    out.append("#define %s_TAU2 %sf" % (name, float.hex(f32_up(2 * tau * (1 + 4 * u)))))
    out.append("#define %s_K0 %sf" % (name, float.hex(f32_up(k0))))
    out.append("")
    return out


# Optimal weights d_0, d_1, d_2 of the small stencils S0 (central), S1
# (downwind), S2 (upwind) in the fallback of Eq. renormalize (Sec. 4.1).
DK = ("0.5065006634", "0.3699651429", "0.1235341937")


def fallback_weights():
    d = [float(x) for x in DK]
    rows = []
    for mask in range(8):
        dd = [d[k] if mask >> k & 1 else 0.0 for k in range(3)]
        den = (dd[0] + dd[1]) + dd[2]
        # no candidate kept (every cut-off failed, possible only for C_T = 1):
        # Eq. renormalize is 0/0, NaN as its literal evaluation gives
        rows.append([x / den for x in dd] if den else [float("nan")] * 3)
    return rows


def fallback_table():
    """Coefficients of the small-stencil fallback as one linear scheme on
    offsets -2..2, for each pattern of the cut-off flags (delta_0, delta_1,
    delta_2) = bits 0..2 of the index: w_k = d_k delta_k / sum_j d_j delta_j
    and the 3-point candidates (Eq. reconstuction), in the operation order of
    the device's exact path (IEEE double, no contraction)."""
    d = [float(x) for x in DK]
    rows = []
    for mask in range(8):
        dd = [d[k] if mask >> k & 1 else 0.0 for k in range(3)]
        den = (dd[0] + dd[1]) + dd[2]
        if den == 0.0:
            rows.append([float("nan")] * 5)     # no candidate kept: 0/0 weights
            continue
        w0, w1, w2 = dd[0] / den, dd[1] / den, dd[2] / den
        rows.append([2.0 * w2 / 6.0, (-w0 - 7.0 * w2) / 6.0, (5.0 * w0 + 2.0 * w1 + 11.0 * w2) / 6.0,
                     (2.0 * w0 + 5.0 * w1) / 6.0, -w1 / 6.0])
    return rows


def _c(x):
    """A double as a C literal (hexadecimal, NaN as the compiler builtin)."""
    if x != x:
        return '__builtin_nan("")'
    return float.hex(x) if x else "0.0"


def emit():
    import numpy as np
    check_printed_indicators()
    W12 = indicator_spec(-5, 12)
    lin6 = s6_scheme()
    out = ["// Generated by gen_coeffs.py from the integers of Eq. TENO10_AA",
           "// (arXiv 2109.14340, Sec. 4.2) and the derived twelve-point S6; do not edit.",
           "#pragma once", ""]
    norms = {}
    for name, spec in (("TENO_Q6", W6), ("TENO_Q8", W8), ("TENO_Q10", W10), ("TENO_Q12", W12)):
        w, M = table(spec)
        out.append("static __constant__ double %s[%d][%d] = {" % (name, w, w))
        for r in range(w):
            out.append("    {" + ", ".join(float(v).hex() if v else "0.0" for v in M[r]) + "},")
        out.append("};")
        out.append("")
        norms[w] = sym_norms(M, spec[1], w)
    out.append("// Linear scheme of the twelve-point candidate S6 at face i+1/2, offsets")
    out.append("// -5..6 (Sec. 4.1 recipe with nu = 7, accuracy constraint 10, 11th-")
    out.append("// difference part 1/200 on cell i).")
    out.append("static __constant__ double TENO_LIN6[12] = {")
    out.append("    " + ", ".join(float.hex(x) for x in lin6) + "};")
    out.append("")
    out.append("static __constant__ double TENO_DK[3] = {%s};" % ", ".join(DK))
    out.append("// Renormalised fallback weights w_k = d_k delta_k / sum_j d_j delta_j (double")
    out.append("// division), by (delta_0, delta_1, delta_2) = bits 0..2 of the row index;")
    out.append("// NaN (0/0) when no candidate is kept.")
    out.append("static __constant__ double TENO_FBW[8][3] = {")
    for r in fallback_weights():
        out.append("    {" + ", ".join(_c(x) for x in r) + "},")
    out.append("};")
    out.append("// Fallback as one linear scheme on offsets -2..2, by (delta_0, delta_1,")
    out.append("// delta_2) = bits 0..2 of the row index.")
    out.append("static __constant__ double TENO_FBK[8][5] = {")
    for r in fallback_table():
        out.append("    {" + ", ".join(_c(x) for x in r) + "},")
    out.append("};")
    out.append("")
    # Sum-of-squares forms of the three large indicators (single-precision
    # decision filter).
    out += sos_tables("TENO_SOS6", W6, norms[6][1])
    out += sos_tables("TENO_SOS8", W8, norms[8][1])
    out += sos_tables("TENO_SOS10", W10, norms[10][1])
    out += sos_tables("TENO_SOS12", W12, norms[12][1])
    return "\n".join(out)


if __name__ == "__main__":
    print(emit())
