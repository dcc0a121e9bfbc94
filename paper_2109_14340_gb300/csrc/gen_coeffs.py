"""Write teno_coeffs.cuh: the smoothness-indicator quadratic forms of the
eight/ten-point TENO-AA schemes (arXiv 2109.14340, Sec. 4.2, Eq. TENO10_AA)
as doubles, each the round-to-nearest of the printed integer over the printed
denominator (Python's int / int division is correctly rounded).

Layout: upper triangle in ascending stencil offset, Q<w>[r][c] for r <= c,
offset = index + lo (lo = -2, -3, -4 for widths 6, 8, 10); zeros below.
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


def emit():
    import numpy as np
    out = ["// Generated by gen_coeffs.py from the integers of Eq. TENO10_AA",
           "// (arXiv 2109.14340, Sec. 4.2); do not edit.",
           "#pragma once", ""]
    norms = {}
    for name, spec in (("TENO_Q6", W6), ("TENO_Q8", W8), ("TENO_Q10", W10)):
        w, M = table(spec)
        out.append("static __constant__ double %s[%d][%d] = {" % (name, w, w))
        for r in range(w):
            out.append("    {" + ", ".join(float(v).hex() if v else "0.0" for v in M[r]) + "},")
        out.append("};")
        out.append("static __constant__ float %sF[%d][%d] = {" % (name, w, w))
        for r in range(w):
            out.append("    {" + ", ".join((float(np.float32(v)).hex() + "f") if v else "0.0f"
                                           for v in M[r]) + "},")
        out.append("};")
        out.append("")
        norms[w] = sym_norms(M, spec[1], w)
    # small indicators in shifted values: beta0 on (s-1, s1), beta1 on (s1, s2),
    # beta2 on (s-2, s-1)
    small = [np.array([[4 / 3, 5 / 6], [5 / 6, 4 / 3]]),
             np.array([[25 / 3, -19 / 6], [-19 / 6, 4 / 3]]),
             np.array([[4 / 3, -19 / 6], [-19 / 6, 25 / 3]])]
    sn = [(float(np.max(np.abs(np.linalg.eigvalsh(A)))) * 1.01,
           float(np.max(np.abs(np.linalg.eigvalsh(np.abs(A))))) * 1.01) for A in small]
    out.append("// Spectral norms (||A||, || |A| ||, rounded up) of the indicator forms on")
    out.append("// shifted values: small stencils S0, S1, S2, then S3, S4, S5.")
    vals = sn + [norms[6], norms[8], norms[10]]
    out.append("static __constant__ float TENO_BNORM[6][2] = {" +
               ", ".join("{%r, %r}" % (float(np.float32(a)), float(np.float32(b))) for a, b in vals)
               .replace("'", "") + "};")
    out.append("")
    return "\n".join(out)


if __name__ == "__main__":
    print(emit())
