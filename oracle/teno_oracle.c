/*
 * TENO-AA CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 restatement of the eight-, ten- and twelve-point TENO-AA schemes of
 * L. Fu, "Very-high-order TENO schemes with adaptive accuracy order and adaptive
 * dissipation control" (arXiv 2109.14340), applied to the compressible Euler
 * equations (Sec. 1, Eq. Euler) in the conservative finite-difference form of
 * Sec. 2 (Eq. approximateEq) with SSP-RK3 time stepping (Sec. 5, Eq. Runge-kutta).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path: its coefficient
 * tables are its own transcription of Sec. 4 (the twelve-point candidate S6,
 * which the paper does not print, comes from oracle/teno12_derive.py, the
 * oracle's own derivation by the Sec. 4.1 recipe), and every step is
 * recomputed per face from the conserved variables, in the order the paper
 * states it.
 *
 * Rounding is pinned: build with -ffp-contract=off; the only fused operations
 * are the explicit fma() calls (dot products and quadratic forms).  Division and
 * sqrt are IEEE round-to-nearest.
 *
 * Parity-pinned by tests/test_oracle_*.py (rational re-derivation of every
 * smoothness indicator, stencil orders, design order of accuracy, linear-scheme
 * recovery, conservation, free stream, positivity, exact Riemann solutions,
 * RK3 stability polynomial).  Parity unpinned: the positivity limiter's exact
 * formula (the paper cites it without stating it); only its invariants are
 * pinned.  The twelve-point S6 is not printed: its recipe parameters (nu = 7,
 * tenth-order constraint, 1/200 of the 11th difference on cell i) are the
 * ones that reproduce the printed S3-S5, which the tests check, together with
 * S6's order, its optimality for the weighted error integral and its
 * indicator's exact derivation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXC 5          /* conserved variables in 3D: rho, m_x, m_y, m_z, E */
#define MAXH 6          /* half-width of the twelve-point stencil             */

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_SLIPWALL = 2, BC_NOSLIP = 3, BC_DIRICHLET = 4 };
enum { SPLIT_LLF = 0, SPLIT_RUSANOV = 1 };

/* Oracle-private parameter block (its own layout; the CUDA library has another). */
typedef struct {
    int32_t ndim, scheme, split, limiter;
    int64_t n[3];
    double dx[3];
    double gamma, alpha1, alpha2, cr, eps_beta, eps_eta, lim_eps;
    int32_t bc_lo[3], bc_hi[3];
    /* BC_DIRICHLET: boundary-face primitives (rho, u..., p) of each side,
     * [ndim + 2][faces of the side, other axes x fastest]; NULL otherwise */
    const double *bc_state_lo[3], *bc_state_hi[3];
} or_params;

/* ------------------------------------------------------------------------- */
/* Coefficients of Sec. 4 (transcribed from the paper).                       */
/* ------------------------------------------------------------------------- */

/* Optimal linear schemes on the large stencils: Eq. 6-point (S3, offsets -2..3),
 * Eq. 8-point (S4, -3..4), Eq. 10-point (S5, -4..5), all at face i+1/2. */
static const double LIN3[6] = {
    0.02852274270130377, -0.1714015614372447, 0.650378818735941,
    0.6253788187359414, -0.1589015614372448, 0.02602274270130375};
static const double LIN4[8] = {
    -0.006866688980568011, 0.05128582585522106, -0.1968478198727312,
    0.6552858258552222, 0.6452858258552218, -0.1908478198727314,
    0.04928582585522098, -0.006580974694853729};
static const double LIN5[10] = {
    0.001911786299492748, -0.0170332977472532, 0.07339445614860979,
    -0.221228429084247, 0.6657332621611695, 0.6557332621611695,
    -0.2145617624175796, 0.07053731329146805, -0.01631901203296621,
    0.001832421220128962};

/* Optimal weights of the three small stencils (Sec. 4.1, after Eq. 6-point). */
static const double DK[3] = {0.5065006634, 0.3699651429, 0.1235341937};

/* Smoothness-indicator quadratic forms of Eq. TENO10_AA as printed: pairs
 * (f_a, f_b) with their integer coefficient and the common denominator.
 * Offsets are relative to cell i.  Stored as decimal strings because the
 * ten-point integers exceed 64 bits. */
typedef struct { int a, b; const char *c; } qterm;

static const char *B36_DEN = "120960";
static const qterm B36[] = {
    {-2, -2, "271779"}, {-2, -1, "-2380800"}, {-2, 0, "4086352"}, {-2, 1, "-3462252"},
    {-2, 2, "1458762"}, {-2, 3, "-245620"},
    {-1, -1, "5653317"}, {-1, 0, "-20427884"}, {-1, 1, "17905032"}, {-1, 2, "-7727988"},
    {-1, 3, "1325006"},
    {0, 0, "19510972"}, {0, 1, "-35817664"}, {0, 2, "15929912"}, {0, 3, "-2792660"},
    {1, 1, "17195652"}, {1, 2, "-15880404"}, {1, 3, "2863984"},
    {2, 2, "3824847"}, {2, 3, "-1429976"},
    {3, 3, "139633"},
};

static const char *B48_DEN = "62270208000";
static const qterm B48[] = {
    {4, 4, "75349098471"}, {4, 3, "-1078504915264"}, {4, 2, "3263178215782"},
    {4, 1, "-5401061230160"}, {4, 0, "5274436892970"}, {4, -1, "-3038037798592"},
    {4, -2, "956371298594"}, {4, -3, "-127080660272"},
    {3, 3, "3944861897609"}, {3, 2, "-24347015748304"}, {3, 1, "41008808432890"},
    {3, 0, "-40666174667520"}, {3, -1, "23740865961334"}, {3, -2, "-7563868580208"},
    {3, -3, "1016165721854"},
    {2, 2, "38342902371231"}, {2, 1, "-131738583368480"}, {2, 0, "133017910915250"},
    {2, -1, "-78915800051952"}, {2, -2, "25505661974314"}, {2, -3, "-3471156679072"},
    {1, 1, "115593819531025"}, {1, 0, "-238366288500400"}, {1, -1, "144163939468910"},
    {1, -2, "-47407534412640"}, {1, -3, "6553080547830"},
    {0, 0, "125743620342175"}, {0, -1, "-155660468395520"}, {0, -2, "52279668813670"},
    {0, -3, "-7366325742800"},
    {-1, -1, "49429163447121"}, {-1, -2, "-34065661645264"}, {-1, -3, "4916835566842"},
    {-2, -2, "6047605530599"}, {-2, -3, "-1799848509664"},
    {-3, -3, "139164877641"},
};

static const char *B510_DEN = "8002967132160000";
static const qterm B510[] = {
    {5, 5, "10271226852556519"}, {5, 4, "-188781685190428812"},
    {5, 3, "763744975064517708"}, {5, 2, "-1783557622547881452"},
    {5, 1, "2647293374939748168"}, {5, 0, "-2588349166844242788"},
    {5, -1, "1666621903133989812"}, {5, -2, "-681536822065683108"},
    {5, -3, "160665441665569002"}, {5, -4, "-16642851860701568"},
    {4, 4, "878723894536476309"}, {4, 3, "-7196903757161570412"},
    {4, 2, "16998197062674090348"}, {4, 1, "-25496314580012763492"},
    {4, 0, "25171844359828276512"}, {4, -1, "-16354640170583096868"},
    {4, -2, "6744593557304053812"}, {4, -3, "-1602760184146136448"},
    {4, -4, "167317608214622742"},
    {3, 3, "14917582508640112584"}, {3, 2, "-71318426816839529952"},
    {3, 1, "108212250511882175688"}, {3, 0, "-108001260086756280408"},
    {3, -1, "70886485695552144912"}, {3, -2, "-29512192424763178368"},
    {3, -3, "7076170986963512652"}, {3, -4, "-745034101222016988"},
    {2, 2, "86303482562247542424"}, {2, 1, "-265161231242943624792"},
    {2, 0, "267840170248801834152"}, {2, -1, "-177812140823999192448"},
    {2, -2, "74826544942103527152"}, {2, -3, "-18122888431675718748"},
    {2, -4, "1926367559931410892"},
    {1, 1, "206327958083635665564"}, {1, 0, "-422297341631652106368"},
    {1, -1, "283934849707927541592"}, {1, -2, "-120940245081713867688"},
    {1, -3, "29628242804292093792"}, {1, -4, "-3183420029990528028"},
    {0, 0, "219076505295455164644"}, {0, -1, "-298732736184126553512"},
    {0, -2, "128985549388044842808"}, {0, -3, "-32013238878488743452"},
    {0, -4, "3482351360282643768"},
    {-1, -1, "103357453544031038184"}, {-1, -2, "-90608758883967297312"},
    {-1, -3, "22823791389362998548"}, {-1, -4, "-2518379721362611092"},
    {-2, -2, "20182234533315641784"}, {-2, -3, "-10338186802053144852"},
    {-2, -4, "1159763060479463988"},
    {-3, -3, "1348293007163766699"}, {-3, -4, "-308382340247963892"},
    {-4, -4, "18029727887840089"},
};

/* The twelve-point candidate S6 (TENO12-AA): terms of beta_{6,12} as reduced
 * fractions (offset a, offset b, numerator, denominator) and the linear scheme
 * LIN6, both derived by oracle/teno12_derive.py from Eq. measureTENO and the
 * optimisation of Sec. 4.1. */
typedef struct { int a, b; const char *c, *d; } qterm2;
#include "teno12_tables.h"

/* Quadratic-form coefficient c/D rounded to the nearest double (ties to even),
 * computed exactly with 128-bit integers. */
typedef __int128 i128;
typedef unsigned __int128 u128;

static i128 parse_i128(const char *s)
{
    int neg = 0;
    i128 v = 0;
    if (*s == '-') { neg = 1; s++; }
    for (; *s; s++) v = v * 10 + (*s - '0');
    return neg ? -v : v;
}

static int bitlen(u128 x)
{
    int n = 0;
    while (x) { n++; x >>= 1; }
    return n;
}

double oracle_round_ratio(const char *num, const char *den)
{
    i128 N = parse_i128(num), D = parse_i128(den);
    if (N == 0) return 0.0;
    int neg = N < 0;
    u128 a = (u128)(neg ? -N : N), d = (u128)D;
    int s = 56 + bitlen(d) - bitlen(a);          /* quotient gets >= 55 bits */
    u128 q, r;
    if (s >= 0) {
        q = (a << s) / d;
        r = (a << s) % d;
    } else {
        u128 dd = d << (-s);
        q = a / dd;
        r = a % dd;
    }
    int k = bitlen(q) - 53;                     /* bits below the mantissa */
    u128 mant = q >> k;
    u128 rem = q & (((u128)1 << k) - 1);
    u128 half = (u128)1 << (k - 1);
    if (rem > half || (rem == half && (r != 0 || (mant & 1)))) mant += 1;
    double v = ldexp((double)(uint64_t)mant, k - s);
    return neg ? -v : v;
}

/* Upper-triangular coefficient matrices, rows and columns in ascending offset. */
static double Q36[6][6], Q48[8][8], Q510[10][10], Q612[12][12];
static int tables_ready = 0;

static void fill_table(const qterm *t, int nt, const char *den, int lo, int w, double *M)
{
    memset(M, 0, sizeof(double) * w * w);
    for (int e = 0; e < nt; e++) {
        int r = t[e].a < t[e].b ? t[e].a : t[e].b;
        int c = t[e].a < t[e].b ? t[e].b : t[e].a;
        M[(r - lo) * w + (c - lo)] = oracle_round_ratio(t[e].c, den);
    }
}

static void init_tables(void)
{
    if (tables_ready) return;
#pragma omp critical(teno_oracle_tables)
    {
        if (!tables_ready) {
            fill_table(B36, sizeof(B36) / sizeof(B36[0]), B36_DEN, -2, 6, &Q36[0][0]);
            fill_table(B48, sizeof(B48) / sizeof(B48[0]), B48_DEN, -3, 8, &Q48[0][0]);
            fill_table(B510, sizeof(B510) / sizeof(B510[0]), B510_DEN, -4, 10, &Q510[0][0]);
            memset(Q612, 0, sizeof(Q612));
            for (size_t e = 0; e < sizeof(B612) / sizeof(B612[0]); e++) {
                int r = B612[e].a < B612[e].b ? B612[e].a : B612[e].b;
                int c = B612[e].a < B612[e].b ? B612[e].b : B612[e].a;
                Q612[r + 5][c + 5] = oracle_round_ratio(B612[e].c, B612[e].d);
            }
            tables_ready = 1;
        }
    }
}

/* Exposed for the coefficient pins: the integer terms of one indicator (for
 * width 12 each term carries its own denominator). */
int oracle_beta_terms(int width, int idx, int *a, int *b, const char **c, const char **den)
{
    const qterm *t;
    int nt;
    if (width == 12) {
        nt = (int)(sizeof(B612) / sizeof(B612[0]));
        if (idx < 0) return nt;
        if (idx >= nt) return -1;
        *a = B612[idx].a; *b = B612[idx].b; *c = B612[idx].c; *den = B612[idx].d;
        return nt;
    }
    if (width == 6) { t = B36; nt = sizeof(B36) / sizeof(B36[0]); *den = B36_DEN; }
    else if (width == 8) { t = B48; nt = sizeof(B48) / sizeof(B48[0]); *den = B48_DEN; }
    else if (width == 10) { t = B510; nt = sizeof(B510) / sizeof(B510[0]); *den = B510_DEN; }
    else return -1;
    if (idx < 0) return nt;
    if (idx >= nt) return -1;
    *a = t[idx].a; *b = t[idx].b; *c = t[idx].c;
    return nt;
}

/* Table coefficient (rounded double) for the pins: width 6/8/10/12, offsets r<=s. */
double oracle_beta_coef(int width, int r, int s)
{
    init_tables();
    if (r > s) { int t = r; r = s; s = t; }
    if (width == 6) return Q36[r + 2][s + 2];
    if (width == 8) return Q48[r + 3][s + 3];
    if (width == 12) return Q612[r + 5][s + 5];
    return Q510[r + 4][s + 4];
}

/* Linear-scheme coefficient of S_L at offset off (0 outside the stencil). */
double oracle_lin_coef(int L, int off)
{
    switch (L) {
    case 3: return (off >= -2 && off <= 3) ? LIN3[off + 2] : 0.0;
    case 4: return (off >= -3 && off <= 4) ? LIN4[off + 3] : 0.0;
    case 5: return (off >= -4 && off <= 5) ? LIN5[off + 4] : 0.0;
    case 6: return (off >= -5 && off <= 6) ? LIN6[off + 5] : 0.0;
    default: return 0.0;
    }
}

/* Half-width H of the scheme: 4, 5, 6 for TENO8, TENO10, TENO12-AA. */
static int half_width(const or_params *P)
{
    return P->scheme == 12 ? 6 : (P->scheme == 10 ? 5 : 4);
}

/* Powers of ten for C_T = 10^-[beta] (Eq. CT_definition). */
static const double TENPOW[23] = {
    1e0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11,
    1e-12, 1e-13, 1e-14, 1e-15, 1e-16, 1e-17, 1e-18, 1e-19, 1e-20, 1e-21, 1e-22};

/* ------------------------------------------------------------------------- */
/* Scalar TENO-AA reconstruction at face i+1/2 (Sec. 3.2-3.4, Sec. 4.2-4.3).   */
/* v[m + H - 1] holds the value at offset m = -H+1 .. H from the upwind cell. */
/* ------------------------------------------------------------------------- */

/* Eq. measureTENO in the printed quadratic form of Eq. TENO10_AA, evaluated on
 * data shifted by the cell-i value (the indicator contains derivatives only, so
 * the shift leaves it unchanged and removes the constant's cancellation). */
static double beta_large(int L, const double *v, int H)
{
    int lo;                             /* S3: -2..3, S4: -3..4, S5: -4..5, S6: -5..6 */
    int w;
    const double *M;
    if (L == 3) { lo = -2; w = 6; M = &Q36[0][0]; }
    else if (L == 4) { lo = -3; w = 8; M = &Q48[0][0]; }
    else if (L == 5) { lo = -4; w = 10; M = &Q510[0][0]; }
    else { lo = -5; w = 12; M = &Q612[0][0]; }
    double s[12];
    double v0 = v[H - 1];
    for (int r = 0; r < w; r++) s[r] = v[lo + r + H - 1] - v0;
    double acc = 0.0;
    for (int r = 0; r < w; r++) {
        double inner = M[r * w + r] * s[r];
        for (int c = r + 1; c < w; c++) inner = fma(M[r * w + c], s[c], inner);
        acc = (r == 0) ? s[r] * inner : fma(s[r], inner, acc);
    }
    return acc;
}

/* Linear scheme of the large stencil S_L (Eqs. 6-, 8-, 10-point; S6 derived). */
static double flux_large(int L, const double *v, int H)
{
    int lo, w;
    const double *c;
    if (L == 3) { lo = -2; w = 6; c = LIN3; }
    else if (L == 4) { lo = -3; w = 8; c = LIN4; }
    else if (L == 5) { lo = -4; w = 10; c = LIN5; }
    else { lo = -5; w = 12; c = LIN6; }
    double acc = c[0] * v[lo + H - 1];
    for (int r = 1; r < w; r++) acc = fma(c[r], v[lo + r + H - 1], acc);
    return acc;
}

/* Eq. scale_separation with q = 7: gamma = 1 / (beta + eps)^7. */
static double scale_sep(double beta, double eps)
{
    double x = beta + eps;
    double x2 = x * x;
    double x4 = x2 * x2;
    double x7 = (x4 * x2) * x;
    return 1.0 / x7;
}

/* C_T exponent from the first-order undivided differences (Eq. m_definition,
 * Eq. CT_definition).  Returns [beta] clamped to the power table. */
static int ct_exponent(const or_params *P, const double *v, int H)
{
#define V(m) v[(m) + H - 1]
    double dl[5];                               /* dl[k] = Delta f_{k-2+1/2} */
    for (int m = -2; m <= 2; m++) dl[m + 2] = V(m + 1) - V(m);
    double emin = 0.0;
    for (int j = -1; j <= 2; j++) {
        double dp = dl[j + 2], dm = dl[j + 1];
        double num = fabs((2.0 * dp) * dm) + P->eps_eta;
        double den = (dp * dp + dm * dm) + P->eps_eta;
        double e = num / den;
        if (j == -1 || e < emin) emin = e;
    }
    double r = emin / P->cr;
    double m = 1.0 - (r < 1.0 ? r : 1.0);
    double om = 1.0 - m;
    double om2 = om * om;
    double g = (om2 * om2) * (1.0 + 4.0 * m);
    double bct = P->alpha1 - P->alpha2 * (1.0 - g);
    double fl = floor(bct);
    int n = fl < 0.0 ? 0 : (fl > 22.0 ? 22 : (int)fl);
    return n;
#undef V
}

/* One TENO-AA reconstruction.  flag: bits 0-1 selected large stencil (L-2) or
 * 0 for the small-stencil fallback, bits 2-4 cut-off deltas of S0..S2 (fallback
 * only), bits 5-7 C_T exponent minus 7.  S6 (twelve-point scheme) is written
 * with bits 0-4 all zero: a fallback always keeps at least one small stencil
 * (the three chi_k sum to one), so that pattern is otherwise unused. */
double oracle_teno_recon(const or_params *P, const double *v, uint8_t *flag)
{
    init_tables();
    int p = half_width(P);
    int H = p;
#define V(m) v[(m) + H - 1]
    int nexp = ct_exponent(P, v, H);
    double CT = TENPOW[nexp];
    uint8_t fct = (uint8_t)(((nexp - 7) & 7) << 5);

    /* Small-stencil indicators (Eq. TENO10_AA, first three lines). */
    double a0 = V(-1) - V(1);
    double b0 = (V(-1) - 2.0 * V(0)) + V(1);
    double beta0 = 0.25 * (a0 * a0) + (13.0 / 12.0) * (b0 * b0);
    double a1 = (3.0 * V(0) - 4.0 * V(1)) + V(2);
    double b1 = (V(0) - 2.0 * V(1)) + V(2);
    double beta1 = 0.25 * (a1 * a1) + (13.0 / 12.0) * (b1 * b1);
    double a2 = (V(-2) - 4.0 * V(-1)) + 3.0 * V(0);
    double b2 = (V(-2) - 2.0 * V(-1)) + V(0);
    double beta2 = 0.25 * (a2 * a2) + (13.0 / 12.0) * (b2 * b2);
    double g0 = scale_sep(beta0, P->eps_beta);
    double g1 = scale_sep(beta1, P->eps_beta);
    double g2 = scale_sep(beta2, P->eps_beta);

    /* Targeted ENO-like selection (Sec. 3.3): groups (S0,S1,S2,S_L), L = p..3. */
    for (int L = p; L >= 3; L--) {
        double gL = scale_sep(beta_large(L, v, H), P->eps_beta);
        double sum = ((g0 + g1) + g2) + gL;
        double chi = gL / sum;                   /* Eq. normalize */
        if (!(chi < CT)) {                       /* Eq. cutoff: delta = 1 */
            *flag = (uint8_t)((L == 6 ? 0 : L - 2) | fct);
            return flux_large(L, v, H);
        }
    }

    /* Fallback on the three small stencils, Eq. renormalize / reconstuction.
     * The normalisation runs over the small stencils only. */
    double s = (g0 + g1) + g2;
    int d0 = !(g0 / s < CT), d1 = !(g1 / s < CT), d2 = !(g2 / s < CT);
    double dd0 = d0 ? DK[0] : 0.0, dd1 = d1 ? DK[1] : 0.0, dd2 = d2 ? DK[2] : 0.0;
    double den = (dd0 + dd1) + dd2;
    double w0 = dd0 / den, w1 = dd1 / den, w2 = dd2 / den;
    double f0 = ((-V(-1) + 5.0 * V(0)) + 2.0 * V(1)) / 6.0;
    double f1 = ((2.0 * V(0) + 5.0 * V(1)) - V(2)) / 6.0;
    double f2 = ((2.0 * V(-2) - 7.0 * V(-1)) + 11.0 * V(0)) / 6.0;
    double fh = w0 * f0;
    fh = fma(w1, f1, fh);
    fh = fma(w2, f2, fh);
    *flag = (uint8_t)(((d0 | (d1 << 1) | (d2 << 2)) << 2) | fct);
    return fh;
#undef V
}

/* ------------------------------------------------------------------------- */
/* Euler: ghost cells (App. A), primitive variables and fluxes (Eq. Euler).    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double U[MAXC], F[MAXC];
    double u[3], p, c, H, sr;
} cellq;

/* Map a (possibly ghost) index along one axis to an interior index (App. A).
 * *side = -1 / +1 when the cell is a ghost of a wall or Dirichlet side (the
 * rule then applies to the returned mirror cell), 0 otherwise. */
static int64_t map_index(int64_t j, int64_t n, int bc_lo, int bc_hi, int *side)
{
    *side = 0;
    if (j < 0) {
        if (bc_lo == BC_PERIODIC) return ((j % n) + n) % n;   /* ghost -r = n-r */
        if (bc_lo == BC_TRANSMISSIVE) return 0;              /* zero-order extrapolation */
        *side = -1;
        return -j - 1;                                       /* ghost -r <- cell r-1 */
    }
    if (j >= n) {
        if (bc_hi == BC_PERIODIC) return j % n;              /* ghost n-1+r = r-1 */
        if (bc_hi == BC_TRANSMISSIVE) return n - 1;
        *side = 1;
        return 2 * n - 1 - j;                                /* ghost n-1+r <- cell n-r */
    }
    return j;
}

/* App. A.3, Dirichlet: the ghost's primitive variables are 2 phi' - phi,
 * phi those of the mirror cell (in Uc on entry) and phi' the given state of
 * the boundary face the ghost row belongs to (st, faces numbered over the
 * other axes, x fastest); the ghost is returned as conserved variables. */
static void dirichlet_ghost(const or_params *P, int d, const double *st, const int64_t x[3],
                            double *Uc)
{
    int nd = P->ndim, nc = nd + 2;
    int64_t m = 1, s = 0;
    for (int a = 0; a < 3; a++) {
        if (a == d) continue;
        s += x[a] * m;
        m *= P->n[a];
    }
    double gm1 = P->gamma - 1.0;
    /* phi of the mirror cell */
    double rho = Uc[0], E = Uc[nc - 1];
    double rinv = 1.0 / rho, u[3];
    for (int a = 0; a < nd; a++) u[a] = Uc[1 + a] * rinv;
    double t = Uc[1] * u[0];
    for (int a = 1; a < nd; a++) t = fma(Uc[1 + a], u[a], t);
    double p = gm1 * (E - 0.5 * t);
    /* reflected about phi' */
    double rg = 2.0 * st[s] - rho, ug[3];
    for (int a = 0; a < nd; a++) ug[a] = 2.0 * st[(1 + a) * m + s] - u[a];
    double pg = 2.0 * st[(nc - 1) * m + s] - p;
    /* back to conserved variables: E = p / (gamma - 1) + rho |u|^2 / 2 */
    Uc[0] = rg;
    for (int a = 0; a < nd; a++) Uc[1 + a] = rg * ug[a];
    double k2 = Uc[1] * ug[0];
    for (int a = 1; a < nd; a++) k2 = fma(Uc[1 + a], ug[a], k2);
    Uc[nc - 1] = pg / gm1 + 0.5 * k2;
}

static int64_t lin_index(const or_params *P, const int64_t x[3])
{
    return x[0] + P->n[0] * (x[1] + P->n[1] * x[2]);
}

static int64_t ncells(const or_params *P)
{
    return P->n[0] * P->n[1] * P->n[2];
}

static void load_cell(const or_params *P, const double *U, int d, const int64_t base[3],
                      int64_t j, double *out)
{
    int nc = P->ndim + 2, side;
    int64_t x[3] = {base[0], base[1], base[2]};
    x[d] = map_index(j, P->n[d], P->bc_lo[d], P->bc_hi[d], &side);
    int64_t id = lin_index(P, x), N = ncells(P);
    for (int c = 0; c < nc; c++) out[c] = U[c * N + id];
    if (side) {
        int bc = side < 0 ? P->bc_lo[d] : P->bc_hi[d];
        if (bc == BC_SLIPWALL) {                  /* App. A.1: normal velocity negated */
            out[1 + d] = -out[1 + d];
        } else if (bc == BC_NOSLIP) {             /* App. A.2: all velocity negated */
            for (int a = 0; a < P->ndim; a++) out[1 + a] = -out[1 + a];
        } else {                                  /* App. A.3 */
            dirichlet_ghost(P, d, side < 0 ? P->bc_state_lo[d] : P->bc_state_hi[d], x, out);
        }
    }
}

/* Primitive variables, sound speed, enthalpy and the physical flux along d. */
static void cell_quantities(const or_params *P, int d, const double *Uc, cellq *q)
{
    int nd = P->ndim, nc = nd + 2;
    double gm1 = P->gamma - 1.0;
    for (int c = 0; c < nc; c++) q->U[c] = Uc[c];
    double rho = Uc[0], E = Uc[nc - 1];
    double rinv = 1.0 / rho;
    for (int a = 0; a < nd; a++) q->u[a] = Uc[1 + a] * rinv;
    double t = Uc[1] * q->u[0];
    for (int a = 1; a < nd; a++) t = fma(Uc[1 + a], q->u[a], t);
    double ke = 0.5 * t;
    q->p = gm1 * (E - ke);
    q->c = sqrt((P->gamma * q->p) * rinv);
    double Ep = E + q->p;
    q->H = Ep * rinv;
    q->sr = sqrt(rho);
    double md = Uc[1 + d];
    q->F[0] = md;
    for (int a = 0; a < nd; a++) {
        q->F[1 + a] = md * q->u[a];
        if (a == d) q->F[1 + a] = q->F[1 + a] + q->p;
    }
    q->F[nc - 1] = q->u[d] * Ep;
}

static int nonphysical_cell(const cellq *q)
{
    return !(q->U[0] > 0.0) || !(q->p > 0.0) || !isfinite(q->c) || !isfinite(q->H);
}

/* ------------------------------------------------------------------------- */
/* Face flux: Roe-averaged characteristic decomposition, LLF splitting,        */
/* TENO-AA reconstruction, back-projection and the positivity limiter.         */
/* ------------------------------------------------------------------------- */

/* Roe average of cells cl, cr (Sec. 5) and the left (rows) / right (columns)
 * eigenvectors of dF_d/dU there.  Field order: u-c, entropy, shear waves
 * (tangential axes ascending), u+c.  Returns the Roe sound speed squared. */
typedef struct {
    double ut[3], Ht, q2, ct;
} roe_state;

static double roe_eigensystem(const or_params *P, int d, const cellq *cl, const cellq *cr,
                              double Lm[MAXC][MAXC], double Rm[MAXC][MAXC], roe_state *rs)
{
    int nd = P->ndim, nc = nd + 2, last = nc - 1;
    double gm1 = P->gamma - 1.0;
    double sl = cl->sr, sr = cr->sr;
    double inv = 1.0 / (sl + sr);
    double ut[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < nd; a++) ut[a] = fma(sr, cr->u[a], sl * cl->u[a]) * inv;
    double Ht = fma(sr, cr->H, sl * cl->H) * inv;
    double q2 = ut[0] * ut[0];
    for (int a = 1; a < nd; a++) q2 = fma(ut[a], ut[a], q2);
    double c2 = gm1 * (Ht - 0.5 * q2);
    double ct = sqrt(c2);
    double cinv = 1.0 / ct;
    double b1 = gm1 * (cinv * cinv);
    double b2 = (0.5 * q2) * b1;
    double un = ut[d];
    double unc = un * cinv;
    double bu = b1 * un;
    double unct = un * ct;
    memset(Lm, 0, sizeof(double) * MAXC * MAXC);
    memset(Rm, 0, sizeof(double) * MAXC * MAXC);
    Lm[0][0] = 0.5 * (b2 + unc);
    Lm[last][0] = 0.5 * (b2 - unc);
    Lm[1][0] = 1.0 - b2;
    for (int a = 0; a < nd; a++) {
        double ba = b1 * ut[a];
        if (a == d) {
            Lm[0][1 + a] = 0.5 * (-bu - cinv);
            Lm[last][1 + a] = 0.5 * (cinv - bu);
        } else {
            Lm[0][1 + a] = 0.5 * (-ba);
            Lm[last][1 + a] = 0.5 * (-ba);
        }
        Lm[1][1 + a] = ba;
    }
    Lm[0][last] = 0.5 * b1;
    Lm[last][last] = 0.5 * b1;
    Lm[1][last] = -b1;
    Rm[0][0] = 1.0; Rm[0][1] = 1.0; Rm[0][last] = 1.0;
    for (int a = 0; a < nd; a++) {
        Rm[1 + a][0] = (a == d) ? un - ct : ut[a];
        Rm[1 + a][1] = ut[a];
        Rm[1 + a][last] = (a == d) ? un + ct : ut[a];
    }
    Rm[last][0] = Ht - unct;
    Rm[last][1] = 0.5 * q2;
    Rm[last][last] = Ht + unct;
    int k = 2;
    for (int a = 0; a < nd; a++) {
        if (a == d) continue;
        Lm[k][0] = -ut[a];
        Lm[k][1 + a] = 1.0;
        Rm[1 + a][k] = 1.0;
        Rm[last][k] = ut[a];
        k++;
    }
    if (rs) {
        for (int a = 0; a < 3; a++) rs->ut[a] = ut[a];
        rs->Ht = Ht; rs->q2 = q2; rs->ct = ct;
    }
    return c2;
}

typedef struct {
    double lam;          /* effective dt/dx of this direction's sub-update */
} lim_info;

/* Pressure of a conserved state (ideal-gas EOS, Sec. 1). */
static double pressure_of(const or_params *P, const double *Uc)
{
    int nd = P->ndim, nc = nd + 2;
    double rinv = 1.0 / Uc[0];
    double t = Uc[1] * (Uc[1] * rinv);
    for (int a = 1; a < nd; a++) t = fma(Uc[1 + a], Uc[1 + a] * rinv, t);
    return (P->gamma - 1.0) * (Uc[nc - 1] - 0.5 * t);
}

/* st[0..2H-1] are cells i-H+1 .. i+H around face i+1/2. */
static void face_flux(const or_params *P, int d, const cellq *st, const lim_info *li,
                      double *Fout, uint8_t *flags, int *bad_face, int *lim_on)
{
    int nd = P->ndim, nc = nd + 2;
    int H = half_width(P), W = 2 * H;
    const cellq *cl = &st[H - 1], *cr = &st[H];
    int last = nc - 1;

    /* Roe average and eigenvectors (Sec. 5). */
    double Lm[MAXC][MAXC], Rm[MAXC][MAXC];
    double c2 = roe_eigensystem(P, d, cl, cr, Lm, Rm, NULL);
    *bad_face = !(c2 > 0.0);

    /* Splitting speeds: LLF per field, max |lambda_k| over the stencil cells;
     * Rusanov: max (|u_d| + c) for every field. */
    double am = 0.0, a0 = 0.0, ap = 0.0, aru = 0.0;
    for (int j = 0; j < W; j++) {
        double vd = st[j].u[d], cj = st[j].c;
        double em = fabs(vd - cj), e0 = fabs(vd), ep = fabs(vd + cj), er = fabs(vd) + cj;
        if (j == 0 || em > am) am = em;
        if (j == 0 || e0 > a0) a0 = e0;
        if (j == 0 || ep > ap) ap = ep;
        if (j == 0 || er > aru) aru = er;
    }

    double h[MAXC];
    for (int f = 0; f < nc; f++) {
        double alpha;
        if (P->split == SPLIT_RUSANOV) alpha = aru;
        else alpha = (f == 0) ? am : (f == last ? ap : a0);
        double fp[2 * MAXH], fm[2 * MAXH];
        for (int j = 0; j < W; j++) {
            double w = Lm[f][0] * st[j].U[0];
            double g = Lm[f][0] * st[j].F[0];
            for (int c = 1; c < nc; c++) {
                w = fma(Lm[f][c], st[j].U[c], w);
                g = fma(Lm[f][c], st[j].F[c], g);
            }
            fp[j] = 0.5 * fma(alpha, w, g);
            fm[j] = 0.5 * fma(-alpha, w, g);
        }
        /* f- is reconstructed on the mirrored stencil: offset m -> cell i+1-m. */
        double vm[2 * MAXH];
        for (int m = -H + 1; m <= H; m++) vm[m + H - 1] = fm[H - m];
        uint8_t fl_p, fl_m;
        double hp = oracle_teno_recon(P, fp, &fl_p);
        double hm = oracle_teno_recon(P, vm, &fl_m);
        if (flags) { flags[2 * f] = fl_p; flags[2 * f + 1] = fl_m; }
        h[f] = hp + hm;
    }
    for (int c = 0; c < nc; c++) {
        double acc = Rm[c][0] * h[0];
        for (int f = 1; f < nc; f++) acc = fma(Rm[c][f], h[f], acc);
        Fout[c] = acc;
    }

    *lim_on = 0;
    if (!P->limiter) return;

    /* Positivity-preserving flux limiter (cited in Sec. 5.3): blend toward the
     * first-order Lax-Friedrichs flux so that the two one-sided half updates
     * of cells i and i+1 keep rho >= eps and p >= eps. */
    double eps = P->lim_eps, lam2 = 2.0 * li->lam;
    double al = fabs(cl->u[d]) + cl->c, ar = fabs(cr->u[d]) + cr->c;
    double af = ar > al ? ar : al;
    double FL[MAXC], dF[MAXC], UL[MAXC], UR[MAXC], dUL[MAXC], dUR[MAXC];
    for (int c = 0; c < nc; c++) {
        FL[c] = 0.5 * ((cl->F[c] + cr->F[c]) - af * (cr->U[c] - cl->U[c]));
        dF[c] = Fout[c] - FL[c];
        UL[c] = cl->U[c] - lam2 * (FL[c] - cl->F[c]);
        UR[c] = cr->U[c] + lam2 * (FL[c] - cr->F[c]);
        dUL[c] = -(lam2 * dF[c]);
        dUR[c] = lam2 * dF[c];
    }
    double th = 1.0;
    const double *Us[2] = {UL, UR}, *dUs[2] = {dUL, dUR};
    for (int side = 0; side < 2; side++) {
        double r0 = Us[side][0], r1 = r0 + dUs[side][0];
        if (r1 < eps) {
            double t = (r0 - eps) / (r0 - r1);
            if (!(t > 0.0)) t = 0.0;
            if (t < th) th = t;
        }
    }
    double thp = th;
    for (int side = 0; side < 2; side++) {
        double Ut[MAXC];
        for (int c = 0; c < nc; c++) Ut[c] = Us[side][c] + th * dUs[side][c];
        double pt = pressure_of(P, Ut);
        if (pt < eps) {
            double p0 = pressure_of(P, Us[side]);
            double t = th * ((p0 - eps) / (p0 - pt));
            if (!(t > 0.0)) t = 0.0;
            if (t < thp) thp = t;
        }
    }
    if (thp < 1.0) {
        *lim_on = 1;
        for (int c = 0; c < nc; c++) Fout[c] = FL[c] + thp * dF[c];
    }
}

/* ------------------------------------------------------------------------- */
/* Right-hand side (Eq. approximateEq, dimension by dimension), CFL, SSP-RK3.  */
/* ------------------------------------------------------------------------- */

/* Per-direction maxima A_d = max_cells (|u_d| + c) of a state. */
static void wave_maxima(const or_params *P, const double *U, double *A, int64_t *bad)
{
    int nd = P->ndim, nc = nd + 2;
    int64_t N = ncells(P), nbad = 0;
    double Am[3] = {0.0, 0.0, 0.0};
    for (int64_t id = 0; id < N; id++) {
        double Uc[MAXC];
        cellq q;
        for (int c = 0; c < nc; c++) Uc[c] = U[c * N + id];
        cell_quantities(P, 0, Uc, &q);
        if (nonphysical_cell(&q)) nbad++;
        for (int a = 0; a < nd; a++) {
            double e = fabs(q.u[a]) + q.c;
            if (e > Am[a]) Am[a] = e;            /* NaN never enters the max */
        }
    }
    for (int a = 0; a < 3; a++) A[a] = Am[a];
    if (bad) *bad = nbad;
}

static void lim_lambdas(const or_params *P, const double *U, double dt, double *lam)
{
    if (P->ndim == 1) {
        lam[0] = dt * (1.0 / P->dx[0]);
        return;
    }
    double A[3];
    wave_maxima(P, U, A, NULL);
    double S = A[0] * (1.0 / P->dx[0]);
    for (int a = 1; a < P->ndim; a++) S = S + A[a] * (1.0 / P->dx[a]);
    for (int a = 0; a < P->ndim; a++) lam[a] = (dt * S) / A[a];
}

static int64_t face_grid_size(const or_params *P, int d)
{
    int64_t s = 1;
    for (int a = 0; a < 3; a++) s *= (a == d) ? P->n[a] + 1 : P->n[a];
    return s;
}

/* rhs[c*N + cell] = L(U); flags (nullable): per direction d, per face of the
 * face grid (n with n_d+1, x fastest), per field, per sign (+ then -).
 * lim_flags (nullable): one byte per face, 1 where the limiter bound.
 * Returns the non-physical count (cells with rho<=0, p<=0 or non-finite values,
 * plus faces whose Roe sound speed squared is not positive). */
int64_t oracle_rhs(const or_params *P, const double *U, double *rhs, double dt_lim,
                   uint8_t *flags, uint8_t *lim_flags, int nthreads)
{
    init_tables();
    int nd = P->ndim, nc = nd + 2;
    int H = half_width(P), W = 2 * H;
    int64_t N = ncells(P);
    double lam[3] = {0.0, 0.0, 0.0};
    if (P->limiter) lim_lambdas(P, U, dt_lim, lam);
    int64_t nbad = 0;
    for (int64_t i = 0; i < (int64_t)nc * N; i++) rhs[i] = 0.0;
    for (int64_t id = 0; id < N; id++) {
        double Uc[MAXC];
        cellq q;
        for (int c = 0; c < nc; c++) Uc[c] = U[c * N + id];
        cell_quantities(P, 0, Uc, &q);
        if (nonphysical_cell(&q)) nbad++;
    }
    int64_t foff = 0, loff = 0;
    for (int d = 0; d < nd; d++) {
        int64_t nd_ = P->n[d];
        int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
        int64_t np1 = P->n[a1], np2 = P->n[a2];
        int64_t npen = np1 * np2;
        double idx = 1.0 / P->dx[d];
        lim_info li = {lam[d]};
        int64_t fgs = face_grid_size(P, d);
        int64_t fstride[3] = {1, 0, 0};
        {
            int64_t fn[3] = {P->n[0], P->n[1], P->n[2]};
            fn[d] += 1;
            fstride[0] = 1; fstride[1] = fn[0]; fstride[2] = fn[0] * fn[1];
        }
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nbad) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t pen = 0; pen < npen; pen++) {
            int64_t base[3] = {0, 0, 0};
            base[a1] = pen % np1;
            base[a2] = pen / np1;
            double *Ff = (double *)malloc(sizeof(double) * (size_t)(nd_ + 1) * nc);
            cellq st[2 * MAXH];
            for (int64_t f = 0; f <= nd_; f++) {
                /* face f sits between cells f-1 and f; stencil cells f-H .. f+H-1 */
                for (int j = 0; j < W; j++) {
                    double Uc[MAXC];
                    load_cell(P, U, d, base, f - H + j, Uc);
                    cell_quantities(P, d, Uc, &st[j]);
                }
                int bad_face = 0, lim_on = 0;
                uint8_t *fl = NULL;
                int64_t fx[3] = {base[0], base[1], base[2]};
                fx[d] = f;
                int64_t flin = fx[0] * fstride[0] + fx[1] * fstride[1] + fx[2] * fstride[2];
                if (flags) fl = flags + foff + flin * nc * 2;
                face_flux(P, d, st, &li, &Ff[f * nc], fl, &bad_face, &lim_on);
                nbad += bad_face;
                if (lim_flags) lim_flags[loff + flin] = (uint8_t)lim_on;
            }
            for (int64_t i = 0; i < nd_; i++) {
                int64_t x[3] = {base[0], base[1], base[2]};
                x[d] = i;
                int64_t id = lin_index(P, x);
                for (int c = 0; c < nc; c++) {
                    double t = (Ff[(i + 1) * nc + c] - Ff[i * nc + c]) * idx;
                    rhs[c * N + id] = rhs[c * N + id] - t;
                }
            }
            free(Ff);
        }
        foff += fgs * nc * 2;
        loff += fgs;
    }
    return nbad;
}

/* Time step (Sec. 5: CFL number, default 0.4): dt = cfl / sum_d A_d / dx_d. */
double oracle_cfl_dt(const or_params *P, const double *U, double cfl, double *A_out,
                     int64_t *nbad)
{
    double A[3];
    wave_maxima(P, U, A, nbad);
    double S = A[0] * (1.0 / P->dx[0]);
    for (int a = 1; a < P->ndim; a++) S = S + A[a] * (1.0 / P->dx[a]);
    if (A_out) for (int a = 0; a < 3; a++) A_out[a] = A[a];
    return cfl / S;
}

/* One SSP-RK3 stage (Eq. Runge-kutta): stage 0: Uk + dt*L; stage 1:
 * 3/4 Un + 1/4 (Uk + dt*L); stage 2: 1/3 Un + 2/3 (Uk + dt*L). */
void oracle_rk3_combine(int stage, int64_t len, const double *Un, const double *Uk,
                        const double *L, double dt, double *out)
{
    for (int64_t i = 0; i < len; i++) {
        double t = Uk[i] + dt * L[i];
        if (stage == 0) out[i] = t;
        else if (stage == 1) out[i] = 0.75 * Un[i] + 0.25 * t;
        else out[i] = (1.0 / 3.0) * Un[i] + (2.0 / 3.0) * t;
    }
}

/* One SSP-RK3 step of size dt, in place.  Each stage's limiter uses dt. */
int64_t oracle_rk3_step(const or_params *P, double *U, double dt, int nthreads)
{
    int nc = P->ndim + 2;
    int64_t len = nc * ncells(P);
    double *Un = (double *)malloc(sizeof(double) * len);
    double *Uk = (double *)malloc(sizeof(double) * len);
    double *L = (double *)malloc(sizeof(double) * len);
    memcpy(Un, U, sizeof(double) * len);
    memcpy(Uk, U, sizeof(double) * len);
    int64_t nbad = 0;
    for (int s = 0; s < 3; s++) {
        nbad += oracle_rhs(P, Uk, L, dt, NULL, NULL, nthreads);
        oracle_rk3_combine(s, len, Un, Uk, L, dt, s == 2 ? U : Uk);
    }
    free(Un); free(Uk); free(L);
    return nbad;
}

/* RHS at a list of cells only (for sampled parity at full size): out[c*nsel+s]. */
void oracle_rhs_at(const or_params *P, const double *U, const int64_t *cells, int64_t nsel,
                   double dt_lim, double *out, int nthreads)
{
    init_tables();
    int nd = P->ndim, nc = nd + 2;
    int H = half_width(P), W = 2 * H;
    double lam[3] = {0.0, 0.0, 0.0};
    if (P->limiter) lim_lambdas(P, U, dt_lim, lam);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t s = 0; s < nsel; s++) {
        int64_t id = cells[s];
        int64_t x[3] = {id % P->n[0], (id / P->n[0]) % P->n[1], id / (P->n[0] * P->n[1])};
        double acc[MAXC];
        for (int c = 0; c < nc; c++) acc[c] = 0.0;
        for (int d = 0; d < nd; d++) {
            lim_info li = {lam[d]};
            double Ff[2][MAXC];
            for (int side = 0; side < 2; side++) {
                int64_t f = x[d] + side;
                cellq st[2 * MAXH];
                for (int j = 0; j < W; j++) {
                    double Uc[MAXC];
                    load_cell(P, U, d, x, f - H + j, Uc);
                    cell_quantities(P, d, Uc, &st[j]);
                }
                int bf, lo;
                face_flux(P, d, st, &li, Ff[side], NULL, &bf, &lo);
            }
            double idx = 1.0 / P->dx[d];
            for (int c = 0; c < nc; c++) acc[c] = acc[c] - (Ff[1][c] - Ff[0][c]) * idx;
        }
        for (int c = 0; c < nc; c++) out[c * nsel + s] = acc[c];
    }
}

/* Eigenvector pin: L and R at the Roe state of two cells (row-major nc x nc). */
double oracle_eigensystem(const or_params *P, int d, const double *UL, const double *UR,
                          double *Lout, double *Rout)
{
    int nc = P->ndim + 2;
    cellq a, b;
    cell_quantities(P, d, UL, &a);
    cell_quantities(P, d, UR, &b);
    double Lm[MAXC][MAXC], Rm[MAXC][MAXC];
    double c2 = roe_eigensystem(P, d, &a, &b, Lm, Rm, NULL);
    for (int r = 0; r < nc; r++)
        for (int c = 0; c < nc; c++) { Lout[r * nc + c] = Lm[r][c]; Rout[r * nc + c] = Rm[r][c]; }
    return c2;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Pins: the seven smoothness indicators beta_0..beta_6 (beta_L only for
 * L <= H) and the seven candidate fluxes f_0..f_6 of one stencil. */
void oracle_betas(const or_params *P, const double *v, double *beta, double *fhat)
{
    init_tables();
    int p = half_width(P);
    int H = p;
#define V(m) v[(m) + H - 1]
    double a0 = V(-1) - V(1);
    double b0 = (V(-1) - 2.0 * V(0)) + V(1);
    double a1 = (3.0 * V(0) - 4.0 * V(1)) + V(2);
    double b1 = (V(0) - 2.0 * V(1)) + V(2);
    double a2 = (V(-2) - 4.0 * V(-1)) + 3.0 * V(0);
    double b2 = (V(-2) - 2.0 * V(-1)) + V(0);
    beta[0] = 0.25 * (a0 * a0) + (13.0 / 12.0) * (b0 * b0);
    beta[1] = 0.25 * (a1 * a1) + (13.0 / 12.0) * (b1 * b1);
    beta[2] = 0.25 * (a2 * a2) + (13.0 / 12.0) * (b2 * b2);
    fhat[0] = ((-V(-1) + 5.0 * V(0)) + 2.0 * V(1)) / 6.0;
    fhat[1] = ((2.0 * V(0) + 5.0 * V(1)) - V(2)) / 6.0;
    fhat[2] = ((2.0 * V(-2) - 7.0 * V(-1)) + 11.0 * V(0)) / 6.0;
    for (int L = 3; L <= 6; L++) {
        if (L > p) { beta[L] = 0.0; fhat[L] = 0.0; continue; }
        beta[L] = beta_large(L, v, H);
        fhat[L] = flux_large(L, v, H);
    }
#undef V
}
