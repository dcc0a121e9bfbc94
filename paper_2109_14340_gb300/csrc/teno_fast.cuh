// Certified single-precision decision filter for the TENO-AA reconstruction.
//
// The reconstruction's result depends on the smoothness indicators only
// through discrete decisions: the C_T exponent [beta] of Eq. CT_definition and
// the cut-off tests chi >= C_T of the targeted selection (Eq. normalize, Eq.
// cutoff, Sec. 3.3).  This filter takes every decision of one reconstruction
// -- the exponent n, which large stencil is accepted (S_p first, then the
// smaller ones), or, when all are rejected, the three small-stencil cut-offs
// of the fallback -- in FP32 with rigorous error bounds, and says "uncertain"
// whenever the bounds do not exclude another outcome.  Only a certified
// answer is used; the exact FP64 path (teno_recon) decides everything else,
// so every decision equals the FP64 evaluation of the same formulas, and the
// value is then computed in FP64 with the exact path's own arithmetic.
//
// FP64 part kept: the shifted values s_m = v_m - v_0, computed with exactly
// the operations of the exact path.  FP32 parts: the three small indicators,
// the large-stencil indicators, the scale separation and normalisation (all
// the divisions), and the first-order undivided-difference measure eta -> m
// -> g -> [beta].  The printed quadratic forms of the large indicators
// cancel about six orders of magnitude on smooth data, so FP32 evaluates
// instead their exact rational L D L^T factorisations, beta = sum_i D_i y_i^2
// (sums of non-negative terms); the bound on the error includes the rounding
// of the tables, of FP32, and of the exact path's FP64 evaluation of the
// printed forms.
//
// Error model: every FP32 operation is bounded by its relative rounding
// 2^-24; conversions from FP64 truncate (relative error < 2^-23); the FP64
// evaluation of the same formulas differs from the exact value by a few 2^-53,
// covered by the widening factors.  Operands are scaled by a power of two
// (exact) so that FP32 never over- or underflows.  The epsilons of Eq.
// scale_separation and of the eta measure enter the bounds explicitly
// (x_k = beta_k + eps, eta <= |2ab|/(a^2+b^2) + eps/(a^2+b^2)); every
// x_k must reach 2^-140 (original units) and values stay below 2^51, so
// that the exact path's (beta+eps)^7 and its reciprocal are normal numbers.
//
// Values that agree to within rounding (a plateau carrying rounding noise,
// or the LLF split's near-cancelling side there): the exact path evaluates
// the small indicators on the unshifted values, so its own rounding is as
// large as the differences.  When the values' exponent exceeds the common
// scale by 30 or more, the filter takes the small indicators' inputs with
// the exact path's FP64 operations (bitwise its values) and bounds only
// their conversion to FP32.  Bit-identical stencils, and stencils whose
// differences all lie below 2^-100, are answered outright (S_p with the
// smooth exponent) where the parameters make that answer certain: C_r <= 1,
// C_T <= 0.1 at m = 0 and, for the second kind, epsilons of at least 2^-136.
#pragma once

#include <cmath>

#include "teno_dev.cuh"

namespace teno {

// Per-launch constants of the filter.
struct FastK {
    float cr_inv_lo, cr_inv_hi;  // 1 / C_r rounded down / up
    float alpha1, alpha2;
    int nexp_smooth;             // [beta] at m = 0, as the exact path computes it
    int nexp_min;                // [beta] at g = 0: no exponent the exact path computes
                                 // is smaller (g >= 0 and rounding is monotone)
    float thr[23];               // thr[n] <= 1 / (10^-n (1 + 2^-16)) - 1
    float thr_rej[23];           // thr_rej[n] >= 1 / (10^-n (1 - 2^-16)) - 1
    float eb_lo, eb_hi;          // eps_beta * 2^100 (1 -+ 1e-6) rounded down / up
    float ee_hi;                 // eps_eta * 2^100 rounded up
    int flat_ok;                 // C_r <= 1 and C_T at m = 0 at most 0.1 (the flat cases'
                                 // answer, S_p with the smooth exponent, holds)
    int tiny_ok;                 // flat_ok, and both epsilons at least 2^-136
};

// Filter switch (teno_set_decision_filter), process-wide.
extern int g_fast_filter;

// Whether the filter may decide for these epsilons.  Its bounds carry the
// epsilon of Eq. scale_separation and that of the eta measure (Sec. 3.4)
// explicitly, in units scaled by up to 2^200; eps <= 1e-40 keeps them
// below 2^67 there, inside the range of FP32 and of its approximate
// division.  The paper's value is 1e-40; larger epsilons (or a NaN) get
// every decision from the exact FP64 path.  Smaller ones, zero included,
// are safe: on bit-identical values the exact path's chi is then inf/inf =
// NaN, which the cut-off test keeps (S_p, as the shortcut answers), and
// every other certified answer needs each x_k = beta_k + eps at 2^-140 or
// above, where (beta + eps)^7 cannot underflow.
inline bool fast_filter_valid(double eps_beta, double eps_eta)
{
    return eps_beta >= 0.0 && eps_beta <= 1e-40 && eps_eta >= 0.0 && eps_eta <= 1e-40;
}

// Host: constants of the filter for given C_T parameters and epsilons.
inline FastK fastk_make(double cr, double alpha1, double alpha2, double eps_beta, double eps_eta)
{
    FastK F;
    const double s100 = 1267650600228229401496703205376.0;      // 2^100
    const double eb = eps_beta * s100, ee = eps_eta * s100;
    const double ebl = eb * (1.0 - 1.0e-6), ebh = eb * (1.0 + 1.0e-6);   // x_lower / x_upper
    F.eb_lo = (float)ebl;
    if ((double)F.eb_lo > ebl) F.eb_lo = nextafterf(F.eb_lo, 0.0f);
    F.eb_hi = (float)ebh;
    if ((double)F.eb_hi < ebh) F.eb_hi = nextafterf(F.eb_hi, INFINITY);
    F.ee_hi = (float)ee;
    if ((double)F.ee_hi < ee) F.ee_hi = nextafterf(F.ee_hi, INFINITY);
    const double inv = 1.0 / cr;
    F.cr_inv_lo = nextafterf((float)inv, 0.0f);
    F.cr_inv_hi = nextafterf((float)inv, 1e30f);
    F.alpha1 = (float)alpha1;
    F.alpha2 = (float)alpha2;
    const double bct = alpha1 - alpha2 * (1.0 - 1.0);
    const double fl = floor(bct);
    F.nexp_smooth = fl < 0.0 ? 0 : (fl > 22.0 ? 22 : (int)fl);
    F.flat_ok = (cr <= 1.0 && F.nexp_smooth >= 1) ? 1 : 0;
    F.tiny_ok = (F.flat_ok && eps_beta >= 0x1p-136 && eps_eta >= 0x1p-136) ? 1 : 0;
    const double bmin = alpha1 - alpha2 * (1.0 - 0.0);
    const double flm = floor(bmin);
    F.nexp_min = flm < 0.0 ? 0 : (flm > 22.0 ? 22 : (int)flm);
    for (int n = 0; n < 23; n++) {
        const double t = 1.0 / (pow(10.0, -n) * (1.0 + 1.0 / 65536.0)) - 1.0;
        // round down (toward -inf), then one more step: a safe lower bound
        float tf = (float)t;
        if ((double)tf > t) tf = nextafterf(tf, -INFINITY);
        F.thr[n] = nextafterf(tf, -INFINITY);
        // and an upper bound of the rejection threshold
        const double tr = 1.0 / (pow(10.0, -n) * (1.0 - 1.0 / 65536.0)) - 1.0;
        float tu = (float)tr;
        if ((double)tu < tr) tu = nextafterf(tu, INFINITY);
        F.thr_rej[n] = nextafterf(tu, INFINITY);
    }
    return F;
}

// FP64 -> FP32 with the exponent lowered by `shift` (exact power-of-two
// scaling), truncating the mantissa, for x whose exponent is at most shift
// (the caller's common scale).  Scaled magnitudes below 2^-100 become zero
// (absolute error < 2^-100, which callers add to their bounds); so do zero
// and subnormal x, which the caller's scale (shift >= -100) puts below that.
__device__ __forceinline__ float d2f_scaled(double x, int shift)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ef = ((hi >> 20) & 0x7FF) - 1023 - shift;     // unbiased scaled exponent, <= 0
    if (ef < -100) return 0.0f;
    const unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)(ef + 127) << 23) |
                          (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
    return __uint_as_float(bits);
}

__device__ __forceinline__ int dexp(double x)
{
    return ((__double2hiint(x) >> 20) & 0x7FF) - 1023;
}

__device__ __forceinline__ bool dbits_equal(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// Bounds [lo, hi] of eta = (|2ab| + eps)/(a^2 + b^2 + eps) from FP32 values
// a, b with absolute error bounds ea, eb (scaled units), and the exact-zero
// knowledge of the FP64 differences.  With N = |2ab| <= D = a^2 + b^2,
// eta - N/D = eps (D - N) / (D (D + eps)) lies in [0, eps/D]; eps_hi: an
// upper bound of the scaled epsilon.  Squares below 2^-120 give up (hi = 1).
__device__ __forceinline__ void eta_bounds(float a, float ea, bool za, float b, float eb, bool zb,
                                           float eps_hi, float &lo, float &hi)
{
    const float tiny = 7.52316385e-37f;                      // 2^-120
    if (za && zb) { lo = 1.0f; hi = 1.0f; return; }          // (0 + eps) / (0 + eps)
    if (za || zb) {                                           // eps / (d^2 + eps)
        const float d = za ? fabsf(b) - eb : fabsf(a) - ea;
        lo = 0.0f;
        hi = (d > 0.0f && d * d >= tiny)
                 ? fminf(__fdividef(eps_hi, d * d) * (1.0f + 1.0e-5f) + 1e-9f, 1.0f) : 1.0f;
        return;
    }
    const float al = fabsf(a) - ea, ah = fabsf(a) + ea;
    const float bl = fabsf(b) - eb, bh = fabsf(b) + eb;
    if (!(al > 1e-30f) || !(bl > 1e-30f)) { lo = 0.0f; hi = 1.0f; return; }
    const float t1 = __fdividef(bl, ah), t2 = __fdividef(bh, al);   // t1 <= t2
    const float e1 = __fdividef(2.0f * t1, 1.0f + t1 * t1);
    const float e2 = __fdividef(2.0f * t2, 1.0f + t2 * t2);
    lo = fminf(e1, e2) * (1.0f - 1.0e-5f);
    float h = (t1 <= 1.0f && t2 >= 1.0f) ? 1.0f : fmaxf(e1, e2) * (1.0f + 1.0e-5f);
    const float D = al * al + bl * bl;
    h = D >= tiny ? h + __fdividef(eps_hi, D) * (1.0f + 1.0e-5f) : 1.0f;
    hi = fminf(h + 1e-9f, 1.0f);
}

// g(m) = ((1-m)^2)^2 (1+4m) in FP32.
__device__ __forceinline__ float g_of_m(float m)
{
    const float om = 1.0f - m;
    const float om2 = om * om;
    return (om2 * om2) * (1.0f + 4.0f * m);
}

// Bounds of a small indicator 1/4 a^2 + 13/12 b^2 given FP32 a, b and their
// absolute error bounds.
__device__ __forceinline__ void small_beta(float a, float ea, float b, float eb, float &beta,
                                           float &err)
{
    const float c13 = 13.0f / 12.0f;
    beta = 0.25f * (a * a) + c13 * (b * b);
    const float aa = fabsf(a), ab = fabsf(b);
    err = 0.25f * (2.0f * aa * ea + ea * ea) + 1.0834f * (2.0f * ab * eb + eb * eb) +
          beta * 1.0e-6f;
}

// Bounds [lo, hi] of the indicator of S_L (scaled units, every |f_m| < 2)
// from its sum-of-squares form: y_i = sum_{m >= i} L_mi f_{off(m)} with the
// 2L - 1 variables in descending offset, off(i) = L - i for i < L and
// L - 1 - i after; beta~ = sum_i D_i y_i^2, and
//   |beta - beta~| <= E = (n+3) 2^-24 beta~ + TAU2 sum_i DC_i |y_i| + K0
// (TAU2, DC, K0 as generated with the tables).  The final factors cover the
// FP32 rounding of the bounds themselves; lo may be negative.
template <int L>
__device__ __forceinline__ float sos_l(int m, int i)
{
    if constexpr (L == 3) return TENO_SOS6_L[m][i];
    else if constexpr (L == 4) return TENO_SOS8_L[m][i];
    else if constexpr (L == 5) return TENO_SOS10_L[m][i];
    else return TENO_SOS12_L[m][i];
}
template <int L>
__device__ __forceinline__ float sos_d(int i)
{
    if constexpr (L == 3) return TENO_SOS6_D[i];
    else if constexpr (L == 4) return TENO_SOS8_D[i];
    else if constexpr (L == 5) return TENO_SOS10_D[i];
    else return TENO_SOS12_D[i];
}
template <int L>
__device__ __forceinline__ float sos_dc(int i)
{
    if constexpr (L == 3) return TENO_SOS6_DC[i];
    else if constexpr (L == 4) return TENO_SOS8_DC[i];
    else if constexpr (L == 5) return TENO_SOS10_DC[i];
    else return TENO_SOS12_DC[i];
}

template <int H, int L>
__device__ __forceinline__ void beta_large_bounds(const float (&f)[2 * H], float &lo, float &hi)
{
    constexpr int n = 2 * L - 1;
    float bt = 0.0f, eb = 0.0f;
#pragma unroll
    for (int i = 0; i < n; i++) {
        const int oi = i < L ? L - i : L - 1 - i;
        float y = f[oi + H - 1];
#pragma unroll
        for (int m = i + 1; m < n; m++) {
            const int om = m < L ? L - m : L - 1 - m;
            y = fmaf(sos_l<L>(m, i), f[om + H - 1], y);
        }
        bt = fmaf(sos_d<L>(i), y * y, bt);
        eb = fmaf(sos_dc<L>(i), fabsf(y), eb);
    }
    const float tau2 = (L == 3) ? TENO_SOS6_TAU2 : (L == 4 ? TENO_SOS8_TAU2 : (L == 5 ? TENO_SOS10_TAU2 : TENO_SOS12_TAU2));
    const float k0 = (L == 3) ? TENO_SOS6_K0 : (L == 4 ? TENO_SOS8_K0 : (L == 5 ? TENO_SOS10_K0 : TENO_SOS12_K0));
    const float E = fmaf(tau2, eb, fmaf(bt, (float)(n + 3) * 5.9604645e-8f, k0));
    hi = (bt + E) * (1.0f + 4.0e-6f);
    lo = fmaf(-E, 1.00001f, bt) * (1.0f - 1.0e-6f);
}

// sum_k (a / b_k)^7 over three denominators, each ratio and the sum widened
// by the relative error of the approximate division and of FP32 (up = true:
// an upper bound of the exact sum, else a lower bound).
__device__ __forceinline__ float pow7_sum(float a, float b0, float b1, float b2, bool up)
{
    const float w = up ? (1.0f + 5e-7f) : (1.0f - 5e-7f);
    const float r0 = __fdividef(a, b0) * w, r1 = __fdividef(a, b1) * w, r2 = __fdividef(a, b2) * w;
    const float q0 = r0 * r0, q1 = r1 * r1, q2 = r2 * r2;
    return (q0 * q0 * q0 * r0 + q1 * q1 * q1 * r1 + q2 * q2 * q2 * r2) * (up ? (1.0f + 2e-6f) : (1.0f - 2e-6f));
}

__device__ __forceinline__ float pow7_sum2(float a, float b0, float b1, bool up)
{
    const float w = up ? (1.0f + 5e-7f) : (1.0f - 5e-7f);
    const float r0 = __fdividef(a, b0) * w, r1 = __fdividef(a, b1) * w;
    const float q0 = r0 * r0, q1 = r1 * r1;
    return (q0 * q0 * q0 * r0 + q1 * q1 * q1 * r1) * (up ? (1.0f + 2e-6f) : (1.0f - 2e-6f));
}

// Bounds of x = beta + eps from bounds lo <= beta <= hi (hi >= 0) and the
// scaled epsilon's bounds with the factors 1 -+ 1e-6 already applied
// (FastK::eb_lo, eb_hi): one rounding of the fma is covered by them.
__device__ __forceinline__ float x_upper(float hi, float ehi)
{
    return fmaf(hi, 1.0f + 1.0e-6f, ehi);
}
__device__ __forceinline__ float x_lower(float lo, float elo)
{
    return fmaf(fmaxf(lo, 0.0f), 1.0f - 1.0e-6f, elo);
}

// Selection among the large stencils S_L, S_(L-1), ..., S_3, largest first:
// chi_L >= C_T  <=>  sum_k (x_L / x_k)^7 <= 1/C_T - 1.  Accept when the upper
// bound of the sum is at most thr, reject when its lower bound exceeds
// thr_rej; x_L = beta_L + eps, its lower bound required to reach tiny2 for
// a rejection.  x0..x2 / X0..X2: lower / upper bounds of the small stencils'
// x_k; lo, hi: the bounds of beta_L; elo, ehi: of the scaled epsilon.
// Returns L - 2 of the accepted stencil, 0 when all are rejected, -1 when
// uncertain.
template <int H, int L>
__device__ __forceinline__ int select_large(const float (&f)[2 * H], float lo, float hi, float tiny2,
                                            float elo, float ehi, float x0, float x1, float x2,
                                            float X0, float X1, float X2, float thr, float thr_rej)
{
    if (pow7_sum(x_upper(hi, ehi), x0, x1, x2, true) <= thr) return L - 2;
    const float xl = x_lower(lo, elo);
    if (!(xl >= tiny2) || !(pow7_sum(xl, X0, X1, X2, false) > thr_rej)) return -1;
    if constexpr (L > 3) {
        float lo1, hi1;
        beta_large_bounds<H, L - 1>(f, lo1, hi1);
        return select_large<H, L - 1>(f, lo1, hi1, tiny2, elo, ehi, x0, x1, x2, X0, X1, X2, thr,
                                      thr_rej);
    } else {
        return 0;
    }
}

// A small indicator's FP64 input as the exact path forms it, converted to
// scaled FP32 with the bound of its truncation and flush.
__device__ __forceinline__ void small_in_exact(double x, int emax, float &v, float &err)
{
    v = d2f_scaled(x, emax);
    err = 1.1920929e-7f * 1.0001f * fabsf(v) + 1.6e-30f;
}

// The filter.  v: the 2H values (FP64); s: shifted values s_m = v_m - v_0
// (s[H-1] == 0); need_ct: the caller records the decision byte, so its C_T
// exponent must be known.  Returns true with the decision byte (the exact
// path's encoding) when every decision is certain.
template <int H>
__device__ __forceinline__ bool fast_decide(const double (&v)[2 * H], const double (&s)[2 * H],
                                            const FastK &F, uint8_t &flag, bool need_ct)
{
    constexpr int W = 2 * H;
#define SV(m) s[(m) + H - 1]
#define VV(m) v[(m) + H - 1]
    // Common scale: the largest exponent among the shifted values (the
    // largest biased exponent field: zero for zeros and subnormals, 0x7FF for
    // non-finite values, which the range test below sends on).
    int efield = 0;
#pragma unroll
    for (int j = 0; j < W; j++)
        if (j != H - 1) efield = max(efield, (__double2hiint(s[j]) >> 20) & 0x7FF);
    const int emax = efield - 1023;
    if (efield == 0) {
        // No shifted value above the subnormal range.  All values bit-identical:
        // the exact path's beta_0 and beta_p are 0 and beta_1 = beta_2 (the
        // rounding of 3 v_0), so chi_p lies in [1/4, 1/2] (or is NaN for
        // eps = 0, which also keeps S_p), and eta = eps/eps = 1 (m = 0 when
        // C_r <= 1; NaN for eps = 0, m = 0 too): S_p with the smooth exponent
        // when C_T <= 0.1 there.  Anything else goes to the exact path.
        bool all_eq = F.flat_ok != 0;
#pragma unroll
        for (int j = 0; j < W; j++) all_eq = all_eq && dbits_equal(v[j], v[H - 1]);
        if (!all_eq) return false;
        flag = (uint8_t)(large_code(H) | (((F.nexp_smooth - 7) & 7) << 5));
        return true;
    }
    if (emax < -100) {
        // Every shifted value below 2^-100, not all zero: distinct doubles that
        // close are below 2^-46 in size, so every indicator the exact path
        // forms, its own rounding included, is below 2^-177 (the largest
        // form's coefficients sum to 2^23), at most 2^-41 of eps_beta >=
        // 2^-136.  The x_k = beta_k + eps then agree to 2^-40 and chi_p =
        // 1/4 (1 +- 2^-35) >= C_T; the eta measure's products (below 2^-194)
        // vanish next to eps_eta in the rounding, so eta = 1 exactly: S_p
        // with the smooth exponent.
        if (!F.tiny_ok) return false;
        flag = (uint8_t)(large_code(H) | (((F.nexp_smooth - 7) & 7) << 5));
        return true;
    }
    if (emax > 50) return false;
    float f[W];
#pragma unroll
    for (int j = 0; j < W; j++) f[j] = (j == H - 1) ? 0.0f : d2f_scaled(s[j], emax);
    // floor of every x_k: 2^-140 in original units (the exact path's
    // (beta+eps)^7 stays normal), at least 2^-120 scaled (FP32 stays normal)
    const int tb = max(-140 - 2 * emax, -120);
    const float tiny2 = __uint_as_float((unsigned)(tb + 127) << 23);
    // the epsilons in scaled units, eps 2^-2emax = (eps 2^100) 2^(-2emax-100)
    float ebl = 0.0f, ebh = 7.52316385e-37f, eeh = 7.52316385e-37f;   // 2^-120 bounds below
    {
        const int ke = -2 * emax - 100;
        if (ke >= -90) {
            const float pw = __uint_as_float((unsigned)(ke + 127) << 23);
            ebl = F.eb_lo * pw;
            ebh = F.eb_hi * pw;
            eeh = F.ee_hi * pw;
        }
    }
    const float u23 = 1.1920929e-7f * 1.0001f, u24 = 5.9604645e-8f * 1.0001f;
    const float z100 = 1.6e-30f;             // > 2^-100: flushed-value error
    // The exact path evaluates the small indicators on the unshifted values:
    // its rounding is relative to max |v| (bound 2^(ev - emax - 50) scaled).
    // |v_m| <= |v_0| + |v_m - v_0| < 2^(e_0 + 1) + 2^(emax + 1) (1 + 2^-52)
    // with e_0 the exponent of v_0, so ev = max(e_0, emax) + 1 bounds the
    // exponent of every v_m.
    const int ecell = (__double2hiint(VV(0)) & 0x7FF00000) != 0 ? dexp(VV(0)) : -1100;
    const int ev = max(ecell, emax) + 1;
    if (ev - emax > 60) return false;
    const float eo = ev < -900 ? 0.0f : __uint_as_float((unsigned)(max(ev - emax - 50, -126) + 127) << 23);
#define FF(m) f[(m) + H - 1]

    // Inputs a_k, b_k of the three small indicators with absolute error
    // bounds (scaled units).
    float sa[3], sea[3], sb[3], seb[3];
    if (ev - emax >= 30) {
        // values within 2^-30 of one another relative to their size: the
        // exact path's rounding on the unshifted values is then as large as
        // their differences, so take its own FP64 inputs (the same
        // operations: bitwise its values) and bound only their conversion
        small_in_exact(VV(-1) - VV(1), emax, sa[0], sea[0]);
        small_in_exact((VV(-1) - 2.0 * VV(0)) + VV(1), emax, sb[0], seb[0]);
        small_in_exact((3.0 * VV(0) - 4.0 * VV(1)) + VV(2), emax, sa[1], sea[1]);
        small_in_exact((VV(0) - 2.0 * VV(1)) + VV(2), emax, sb[1], seb[1]);
        small_in_exact((VV(-2) - 4.0 * VV(-1)) + 3.0 * VV(0), emax, sa[2], sea[2]);
        small_in_exact((VV(-2) - 2.0 * VV(-1)) + VV(0), emax, sb[2], seb[2]);
    } else {
        // on the shifted values (s_0 = 0); the slack holds the exact path's
        // rounding on the unshifted values
        const float sl0 = 2.0f * z100 + 4.0f * eo, sl1 = 5.0f * z100 + 8.0f * eo;
        sa[0] = FF(-1) - FF(1);
        sea[0] = u23 * (fabsf(FF(-1)) + fabsf(FF(1))) + u24 * fabsf(sa[0]) + sl0;
        sb[0] = FF(-1) + FF(1);
        seb[0] = u23 * (fabsf(FF(-1)) + fabsf(FF(1))) + u24 * fabsf(sb[0]) + sl0;
        sa[1] = FF(2) - 4.0f * FF(1);
        sea[1] = u23 * (fabsf(FF(2)) + 4.0f * fabsf(FF(1))) + u24 * fabsf(sa[1]) + sl1;
        sb[1] = FF(2) - 2.0f * FF(1);
        seb[1] = u23 * (fabsf(FF(2)) + 2.0f * fabsf(FF(1))) + u24 * fabsf(sb[1]) + sl1;
        sa[2] = FF(-2) - 4.0f * FF(-1);
        sea[2] = u23 * (fabsf(FF(-2)) + 4.0f * fabsf(FF(-1))) + u24 * fabsf(sa[2]) + sl1;
        sb[2] = FF(-2) - 2.0f * FF(-1);
        seb[2] = u23 * (fabsf(FF(-2)) + 2.0f * fabsf(FF(-1))) + u24 * fabsf(sb[2]) + sl1;
    }
    float b0, e0, b1, e1, b2, e2;
    small_beta(sa[0], sea[0], sb[0], seb[0], b0, e0);
    small_beta(sa[1], sea[1], sb[1], seb[1], b1, e1);
    small_beta(sa[2], sea[2], sb[2], seb[2], b2, e2);
    // x_k = beta_k + eps: lower and upper bounds, the lower ones at tiny2 or above
    const float x0 = x_lower(b0 - e0, ebl), x1 = x_lower(b1 - e1, ebl), x2 = x_lower(b2 - e2, ebl);
    if (!(x0 >= tiny2) || !(x1 >= tiny2) || !(x2 >= tiny2)) return false;
    const float X0 = x_upper(b0 + e0, ebh), X1 = x_upper(b1 + e1, ebh), X2 = x_upper(b2 + e2, ebh);

    // Without a decision record the exponent only matters when S_p is not
    // accepted: accept it at once when chi_p >= C_T holds for the largest
    // C_T the parameters allow (the exponent's lower bound, at g = 0), which
    // leaves the eta measure out for most reconstructions.  The C_T bits of
    // the byte are then zero (the byte is not stored).
    float blo, bhi;                           // bounds of beta_p, for both tests
    beta_large_bounds<H, H>(f, blo, bhi);
    if (!need_ct) {
        // sum_k (x_p / x_k)^7 <= 3 (x_p / min_k x_k)^7: one division for the
        // common case (a looser bound only sends borderline cases on)
        const float r = __fdividef(x_upper(bhi, ebh), fminf(x0, fminf(x1, x2))) * (1.0f + 5e-7f);
        const float q = r * r;
        if (3.0f * (q * q * q * r) * (1.0f + 4e-6f) <= F.thr[F.nexp_min]) {
            flag = (uint8_t)large_code(H);
            return true;
        }
    }

    // eta measure over cells -1..2 from the differences Delta_{m+1/2}, m=-2..2.
    float dl[5], el[5];
    bool zl[5];
#pragma unroll
    for (int m = -2; m <= 2; m++) {
        const float a = FF(m + 1), b = FF(m);
        dl[m + 2] = a - b;
        el[m + 2] = u23 * (fabsf(a) + fabsf(b)) + u24 * fabsf(dl[m + 2]) + 2.0f * z100;
        zl[m + 2] = dbits_equal(VV(m + 1), VV(m));
    }
    float emin_lo = 1.0f, emin_hi = 1.0f;
#pragma unroll
    for (int j = -1; j <= 2; j++) {
        float lo, hi;
        eta_bounds(dl[j + 2], el[j + 2], zl[j + 2], dl[j + 1], el[j + 1], zl[j + 1], eeh, lo, hi);
        emin_lo = fminf(emin_lo, lo);
        emin_hi = fminf(emin_hi, hi);
    }
    int nexp;
    const float r_lo = emin_lo * F.cr_inv_lo * (1.0f - 2.5e-7f);
    if (r_lo >= 1.0f) {
        nexp = F.nexp_smooth;                  // eta >= C_r: m = 0 exactly
    } else {
        const float r_hi = emin_hi * F.cr_inv_hi * (1.0f + 2.5e-7f);
        const float m_lo = fmaxf(1.0f - fminf(1.0f, r_hi) - 2.5e-7f, 0.0f);
        const float m_hi = fminf(1.0f - fminf(1.0f, r_lo) + 2.5e-7f, 1.0f);
        const float g_lo = g_of_m(m_hi) * (1.0f - 1.0e-6f);
        const float g_hi = g_of_m(m_lo) * (1.0f + 1.0e-6f);
        const float b_lo = F.alpha1 - F.alpha2 * (1.0f - g_lo) - 1.0e-4f;
        const float b_hi = F.alpha1 - F.alpha2 * (1.0f - g_hi) + 1.0e-4f;
        int n_lo = (int)floorf(b_lo), n_hi = (int)floorf(b_hi);
        n_lo = n_lo < 0 ? 0 : (n_lo > 22 ? 22 : n_lo);
        n_hi = n_hi < 0 ? 0 : (n_hi > 22 ? 22 : n_hi);
        if (!(b_lo == b_lo) || !(b_hi == b_hi) || n_lo != n_hi) return false;
        nexp = n_lo;
    }
    const uint8_t fct = (uint8_t)(((nexp - 7) & 7) << 5);
    const float thr = F.thr[nexp], thr_rej = F.thr_rej[nexp];

    // Targeted selection, largest group first (Sec. 3.3).
    const int sel = select_large<H, H>(f, blo, bhi, tiny2, ebl, ebh, x0, x1, x2, X0, X1, X2, thr,
                                       thr_rej);
    if (sel < 0) return false;
    if (sel > 0) {
        if constexpr (H == 6)
            flag = (uint8_t)((sel == 4 ? 0 : sel) | fct);     // S6: bits 0-4 zero
        else
            flag = (uint8_t)(sel | fct);
        return true;
    }

    // Small-stencil fallback (Eq. renormalize): delta_k = !(g_k / sum < C_T),
    // g_k / sum >= C_T  <=>  sum_{j != k} (x_k / x_j)^7 <= 1/C_T - 1.
    int d[3];
    {
        const float xl[3] = {x0, x1, x2}, xu[3] = {X0, X1, X2};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
            if (pow7_sum2(xu[k], xl[j1], xl[j2], true) <= thr) d[k] = 1;
            else if (pow7_sum2(xl[k], xu[j1], xu[j2], false) > thr_rej) d[k] = 0;
            else return false;
        }
    }
    flag = (uint8_t)(((d[0] | (d[1] << 1) | (d[2] << 2)) << 2) | fct);
    return true;
#undef FF
#undef SV
#undef VV
}

}  // namespace teno
