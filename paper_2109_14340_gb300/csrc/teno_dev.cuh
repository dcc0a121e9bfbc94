// Device building blocks of the TENO-AA Euler right-hand side (sm_103a, FP64).
//
// Every expression fixes its evaluation order; the library is compiled with
// --fmad=false so that the only fused multiply-adds are the explicit fma()
// calls.  Division and sqrt of doubles are IEEE round-to-nearest on the GPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "teno_coeffs.cuh"

namespace teno {

// Workspace header (first 256 bytes of every workspace).
struct Status {
    unsigned long long nonphys;    // non-physical cells + faces (teno_status)
    unsigned long long amax[3];    // bit patterns of A_d = max(|u_d| + c) >= 0
    double dt;                     // time step of the current call
    double lam[3];                 // limiter: effective dt/dx of each direction
    double t_accum;                // summed dt of teno_advance_host
    unsigned long long oob_count;  // debug build: out-of-range accesses skipped
    long long oob_line, oob_index, oob_extent;   // the first one's source line, index, extent
    double pad[19];
};
static_assert(sizeof(Status) == 256, "status block is 256 bytes");

// Debug build (-DTENO_DEBUG_BOUNDS): every global-memory index of the face
// sweeps, the combine and the primitives kernel, and the face sweeps'
// shared-memory queue indices, are range-checked.  An index outside its
// array is counted in the status block (with the first offender's source
// line, index and extent), and the access is skipped -- a load gives 0 --
// instead of faulting (teno_debug_bounds reads the record).  In the
// release build the checks compile away.
#ifdef TENO_DEBUG_BOUNDS
static __device__ __noinline__ void bounds_fault(Status *st, int line, long long idx, long long n)
{
    if (atomicAdd(&st->oob_count, 1ull) == 0ull) {
        st->oob_line = line;
        st->oob_index = idx;
        st->oob_extent = n;
    }
}
#define TENO_IN(st, i, n)                                                                  \
    (((long long)(i) >= 0 && (long long)(i) < (long long)(n))                              \
         ? true                                                                            \
         : (::teno::bounds_fault((st), __LINE__, (long long)(i), (long long)(n)), false))
#else
#define TENO_IN(st, i, n) true
#endif
#define TENO_LOAD(st, a, i, n) (TENO_IN(st, i, n) ? (a)[i] : 0)
#define TENO_STORE(st, a, i, n, v)                                                         \
    do {                                                                                   \
        if (TENO_IN(st, i, n)) (a)[i] = (v);                                               \
    } while (0)

// Optimal linear schemes on the large stencils (Sec. 4.1, Eqs. 6-, 8-,
// 10-point), ascending offsets -2..3, -3..4, -4..5.  The twelve-point S6
// (offsets -5..6, TENO_LIN6) is generated with the indicator tables.
static __constant__ double TENO_LIN3[6] = {
    0.02852274270130377, -0.1714015614372447, 0.650378818735941,
    0.6253788187359414, -0.1589015614372448, 0.02602274270130375};
static __constant__ double TENO_LIN4[8] = {
    -0.006866688980568011, 0.05128582585522106, -0.1968478198727312,
    0.6552858258552222, 0.6452858258552218, -0.1908478198727314,
    0.04928582585522098, -0.006580974694853729};
static __constant__ double TENO_LIN5[10] = {
    0.001911786299492748, -0.0170332977472532, 0.07339445614860979,
    -0.221228429084247, 0.6657332621611695, 0.6557332621611695,
    -0.2145617624175796, 0.07053731329146805, -0.01631901203296621,
    0.001832421220128962};
// Optimal weights of the small stencils S0, S1, S2 (Sec. 4.1).
// C_T = 10^-[beta] (Eq. CT_definition), [beta] clamped to 0..22.
static __constant__ double TENO_TENPOW[23] = {
    1e0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11,
    1e-12, 1e-13, 1e-14, 1e-15, 1e-16, 1e-17, 1e-18, 1e-19, 1e-20, 1e-21, 1e-22};

// Scheme constants passed by value to every kernel.
struct Consts {
    double gamma, gm1;
    double alpha1, alpha2, cr, eps_beta, eps_eta, lim_eps;
    int split, limiter;
};

// ---------------------------------------------------------------------------
// Scalar TENO-AA reconstruction at face i+1/2 (Sec. 3.2-3.4, Sec. 4.2-4.3).
// v[m + H - 1] holds offset m = -H+1 .. H from the upwind cell i.
// ---------------------------------------------------------------------------

// Eq. scale_separation with q = 7.
__device__ __forceinline__ double scale_sep(double beta, double eps)
{
    double x = beta + eps;
    double x2 = x * x;
    double x4 = x2 * x2;
    double x7 = (x4 * x2) * x;
    return 1.0 / x7;
}

// Decision-byte code of the large stencil S_L: L - 2 in bits 0-1 for S3..S5;
// S6 (twelve-point scheme) as bits 0-4 all zero -- a fallback always keeps at
// least one small stencil (the three chi_k sum to one), so its cut-off bits
// are never all zero.
__host__ __device__ constexpr int large_code(int L) { return L == 6 ? 0 : L - 2; }

// Table entries of the indicator form / linear scheme of S_L.
template <int L>
__device__ __forceinline__ double qcoef(int r, int c)
{
    if constexpr (L == 3) return TENO_Q6[r][c];
    else if constexpr (L == 4) return TENO_Q8[r][c];
    else if constexpr (L == 5) return TENO_Q10[r][c];
    else return TENO_Q12[r][c];
}
template <int L>
__device__ __forceinline__ double lcoef(int r)
{
    if constexpr (L == 3) return TENO_LIN3[r];
    else if constexpr (L == 4) return TENO_LIN4[r];
    else if constexpr (L == 5) return TENO_LIN5[r];
    else return TENO_LIN6[r];
}

// Smoothness indicator of the large stencil S_L (Eq. TENO10_AA quadratic
// forms; beta_{6,12} derived from Eq. measureTENO) on data shifted by the
// cell-i value, sh[m + H - 1] = v_m - v_0 for the whole 2H stencil; terms of
// the zero shifted value are skipped (they add exact zeros).
template <int H, int L>
__device__ __forceinline__ double beta_large_s(const double (&sh)[2 * H])
{
    constexpr int lo = 1 - L;                     // S_L covers offsets 1-L .. L
    constexpr int w = 2 * L;
    double s[w];
#pragma unroll
    for (int r = 0; r < w; r++) s[r] = sh[lo + r + H - 1];
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < w; r++) {
        if (r + lo == 0) continue;                // s == 0: contributes nothing
        double inner = qcoef<L>(r, r) * s[r];
#pragma unroll
        for (int c = r + 1; c < w; c++) {
            if (c + lo == 0) continue;
            inner = fma(qcoef<L>(r, c), s[c], inner);
        }
        acc = (r == 0) ? s[r] * inner : fma(s[r], inner, acc);
    }
    return acc;
}

template <int H, int L>
__device__ __forceinline__ double beta_large(const double (&v)[2 * H])
{
    double sh[2 * H];
#pragma unroll
    for (int r = 0; r < 2 * H; r++) sh[r] = v[r] - v[H - 1];
    return beta_large_s<H, L>(sh);
}

template <int H, int L>
__device__ __forceinline__ double flux_large(const double (&v)[2 * H])
{
    constexpr int lo = 1 - L;
    constexpr int w = 2 * L;
    double acc = lcoef<L>(0) * v[lo + H - 1];
#pragma unroll
    for (int r = 1; r < w; r++) acc = fma(lcoef<L>(r), v[lo + r + H - 1], acc);
    return acc;
}

// [beta] of Eq. CT_definition from the first-order undivided differences
// (Eq. m_definition), clamped to the power table.
template <int H>
__device__ __forceinline__ int ct_exponent(const double (&v)[2 * H], const Consts &K)
{
#define V(m) v[(m) + H - 1]
    double dl[5];
#pragma unroll
    for (int m = -2; m <= 2; m++) dl[m + 2] = V(m + 1) - V(m);
    double emin = 0.0;
#pragma unroll
    for (int j = -1; j <= 2; j++) {
        double dp = dl[j + 2], dm = dl[j + 1];
        double num = fabs((2.0 * dp) * dm) + K.eps_eta;
        double den = (dp * dp + dm * dm) + K.eps_eta;
        double e = num / den;
        if (j == -1 || e < emin) emin = e;
    }
    double r = emin / K.cr;
    double m = 1.0 - (r < 1.0 ? r : 1.0);
    double om = 1.0 - m;
    double om2 = om * om;
    double g = (om2 * om2) * (1.0 + 4.0 * m);
    double bct = K.alpha1 - K.alpha2 * (1.0 - g);
    double fl = floor(bct);
    return fl < 0.0 ? 0 : (fl > 22.0 ? 22 : (int)fl);
#undef V
}

// Small-stencil fallback value (Eq. renormalize, Eq. reconstuction): the
// kept candidates (bits 0..2 of mask) weighted by d_k renormalised over them
// (w_k = dd_k / den, tabulated in double), the 3-point candidates divided by
// 6 exactly as written.
template <int H>
__device__ __forceinline__ double fallback_value(const double (&v)[2 * H], int mask)
{
#define V(m) v[(m) + H - 1]
    const double w0 = TENO_FBW[mask][0], w1 = TENO_FBW[mask][1], w2 = TENO_FBW[mask][2];
    double f0 = ((-V(-1) + 5.0 * V(0)) + 2.0 * V(1)) / 6.0;
    double f1 = ((2.0 * V(0) + 5.0 * V(1)) - V(2)) / 6.0;
    double f2 = ((2.0 * V(-2) - 7.0 * V(-1)) + 11.0 * V(0)) / 6.0;
    double fh = w0 * f0;
    fh = fma(w1, f1, fh);
    fh = fma(w2, f2, fh);
    return fh;
#undef V
}

// One reconstruction; flag: bits 0-1 selected large stencil (L-2) or 0 for the
// small-stencil fallback, bits 2-4 deltas of S0..S2 (fallback), bits 5-7 C_T
// exponent minus 7; S6 as bits 0-4 zero (large_code).
template <int H>
__device__ __forceinline__ double teno_recon(const double (&v)[2 * H], const Consts &K,
                                             uint8_t &flag)
{
#define V(m) v[(m) + H - 1]
    const int nexp = ct_exponent<H>(v, K);
    const double CT = TENO_TENPOW[nexp];
    const uint8_t fct = (uint8_t)(((nexp - 7) & 7) << 5);

    double a0 = V(-1) - V(1);
    double b0 = (V(-1) - 2.0 * V(0)) + V(1);
    double beta0 = 0.25 * (a0 * a0) + (13.0 / 12.0) * (b0 * b0);
    double a1 = (3.0 * V(0) - 4.0 * V(1)) + V(2);
    double b1 = (V(0) - 2.0 * V(1)) + V(2);
    double beta1 = 0.25 * (a1 * a1) + (13.0 / 12.0) * (b1 * b1);
    double a2 = (V(-2) - 4.0 * V(-1)) + 3.0 * V(0);
    double b2 = (V(-2) - 2.0 * V(-1)) + V(0);
    double beta2 = 0.25 * (a2 * a2) + (13.0 / 12.0) * (b2 * b2);
    double g0 = scale_sep(beta0, K.eps_beta);
    double g1 = scale_sep(beta1, K.eps_beta);
    double g2 = scale_sep(beta2, K.eps_beta);
    double g012 = (g0 + g1) + g2;

    // Targeted ENO-like selection (Sec. 3.3), largest group first.
    if constexpr (H == 6) {
        double g6 = scale_sep(beta_large<H, 6>(v), K.eps_beta);
        double chi = g6 / (g012 + g6);
        if (!(chi < CT)) { flag = fct; return flux_large<H, 6>(v); }
    }
    if constexpr (H >= 5) {
        double g5 = scale_sep(beta_large<H, 5>(v), K.eps_beta);
        double chi = g5 / (g012 + g5);
        if (!(chi < CT)) { flag = (uint8_t)(3 | fct); return flux_large<H, 5>(v); }
    }
    {
        double g4 = scale_sep(beta_large<H, 4>(v), K.eps_beta);
        double chi = g4 / (g012 + g4);
        if (!(chi < CT)) { flag = (uint8_t)(2 | fct); return flux_large<H, 4>(v); }
    }
    {
        double g3 = scale_sep(beta_large<H, 3>(v), K.eps_beta);
        double chi = g3 / (g012 + g3);
        if (!(chi < CT)) { flag = (uint8_t)(1 | fct); return flux_large<H, 3>(v); }
    }

    // Small-stencil fallback (Eq. renormalize, Eq. reconstuction), normalised
    // over S0, S1, S2.
    double s = g012;
    int d0 = !(g0 / s < CT), d1 = !(g1 / s < CT), d2 = !(g2 / s < CT);
    const int mask = d0 | (d1 << 1) | (d2 << 2);
    flag = (uint8_t)((mask << 2) | fct);
    return fallback_value<H>(v, mask);
#undef V
}

// The value of a reconstruction whose decisions are known (decision byte in
// the encoding above): the selected large stencil's linear scheme or the
// small-stencil fallback, with the exact path's arithmetic.
template <int H>
__device__ __forceinline__ double decided_value(const double (&v)[2 * H], uint8_t flag)
{
    const int sel = flag & 3;
    if constexpr (H == 6) {
        if ((flag & 31) == 0) return flux_large<H, 6>(v);
        if (sel == 3) return flux_large<H, 5>(v);
    } else {
        if (sel == H - 2) return flux_large<H, H>(v);
    }
    if constexpr (H >= 5) {
        if (sel == 2) return flux_large<H, 4>(v);
    }
    if (sel == 1) return flux_large<H, 3>(v);
    return fallback_value<H>(v, (flag >> 2) & 7);
}

// Frozen reconstruction coefficient of value index m (offset m - H + 1) for a
// decision byte: the selected large stencil's linear scheme, or the
// renormalised small-stencil blend.
template <int H>
__device__ __forceinline__ double frozen_coef(uint8_t flag, int m)
{
    const int sel = flag & 3;
    const int off = m - H + 1;
    if constexpr (H == 6) {
        if ((flag & 31) == 0) return (off >= -5 && off <= 6) ? TENO_LIN6[off + 5] : 0.0;
    }
    if (sel == 3) return (off >= -4 && off <= 5) ? TENO_LIN5[off + 4] : 0.0;
    if (sel == 2) return (off >= -3 && off <= 4) ? TENO_LIN4[off + 3] : 0.0;
    if (sel == 1) return (off >= -2 && off <= 3) ? TENO_LIN3[off + 2] : 0.0;
    // small-stencil blend with the renormalised weights (tabulated by the
    // cut-off flags, the same double arithmetic as the exact path's weights)
    return (off >= -2 && off <= 2) ? TENO_FBK[(flag >> 2) & 7][off + 2] : 0.0;
}

// Reconstruction with a recorded decision: the same selection as the byte
// says, applied as a fixed linear scheme (no smoothness indicators).
template <int H>
__device__ __forceinline__ double frozen_recon(const double (&v)[2 * H], uint8_t flag)
{
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 2 * H; m++) acc = fma(frozen_coef<H>(flag, m), v[m], acc);
    return acc;
}

// ---------------------------------------------------------------------------
// Euler: primitive variables and physical flux of one cell (Eq. Euler, EOS).
// ---------------------------------------------------------------------------

template <int ND>
struct CellQ {
    double U[ND + 2], F[ND + 2];
    double u[ND];
    double p, c, H, sr, rinv;
};

// "e > a" for splitting speeds, which are +0, positive or NaN (absolute
// values and |u| + c): on such doubles the order of the IEEE bit patterns
// is the numeric order, and a NaN on either side makes the comparison false
// exactly as the FP64 comparison does.  Integer compares keep the FP64 pipe
// free.
__device__ __forceinline__ bool speed_gt(double e, double a)
{
    const unsigned long long eb = (unsigned long long)__double_as_longlong(e);
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    const unsigned long long inf = 0x7FF0000000000000ull;
    return eb > ab && eb <= inf && ab <= inf;
}

template <int ND, int D>
__device__ __forceinline__ void cell_quantities(const double (&Uc)[ND + 2], const Consts &K,
                                                CellQ<ND> &q)
{
    constexpr int nc = ND + 2;
#pragma unroll
    for (int c = 0; c < nc; c++) q.U[c] = Uc[c];
    double rho = Uc[0], E = Uc[nc - 1];
    double rinv = 1.0 / rho;
    q.rinv = rinv;
#pragma unroll
    for (int a = 0; a < ND; a++) q.u[a] = Uc[1 + a] * rinv;
    double t = Uc[1] * q.u[0];
#pragma unroll
    for (int a = 1; a < ND; a++) t = fma(Uc[1 + a], q.u[a], t);
    double ke = 0.5 * t;
    q.p = K.gm1 * (E - ke);
    q.c = sqrt((K.gamma * q.p) * rinv);
    double Ep = E + q.p;
    q.H = Ep * rinv;
    q.sr = sqrt(rho);
    double md = Uc[1 + D];
    q.F[0] = md;
#pragma unroll
    for (int a = 0; a < ND; a++) {
        q.F[1 + a] = md * q.u[a];
        if (a == D) q.F[1 + a] = q.F[1 + a] + q.p;
    }
    q.F[nc - 1] = q.u[D] * Ep;
}

// Primitive quantities of a cell kept between kernels: [NP][ncell] with
// rows u_0 .. u_{ND-1}, p, c, H, sqrt(rho) (the values cell_quantities
// computes).  Written once per right-hand-side input by prims_kernel or the
// previous stage's combine, read by every sweep of that evaluation.
template <int ND>
struct PrimRows {
    static constexpr int P = ND, C = ND + 1, H = ND + 2, SR = ND + 3, NP = ND + 4;
};

template <int ND>
__device__ __forceinline__ void store_prims(const CellQ<ND> &q, double *P, int64_t ncell, int64_t id)
{
    using R = PrimRows<ND>;
#pragma unroll
    for (int a = 0; a < ND; a++) P[a * ncell + id] = q.u[a];
    P[R::P * ncell + id] = q.p;
    P[R::C * ncell + id] = q.c;
    P[R::H * ncell + id] = q.H;
    P[R::SR * ncell + id] = q.sr;
}

// cell_quantities of a cell whose primitives were stored by store_prims: the
// flux along D is formed from them with the same operations, so every value
// is bitwise the one cell_quantities gives (rinv is not recovered).
template <int ND, int D>
__device__ __forceinline__ void cell_from_prims(const double (&Uc)[ND + 2], const double *P,
                                                int64_t ncell, int64_t id, CellQ<ND> &q)
{
    using R = PrimRows<ND>;
    constexpr int nc = ND + 2;
#pragma unroll
    for (int c = 0; c < nc; c++) q.U[c] = Uc[c];
#pragma unroll
    for (int a = 0; a < ND; a++) q.u[a] = P[a * ncell + id];
    q.p = P[R::P * ncell + id];
    q.c = P[R::C * ncell + id];
    q.H = P[R::H * ncell + id];
    q.sr = P[R::SR * ncell + id];
    q.rinv = 0.0;
    const double Ep = Uc[nc - 1] + q.p;
    const double md = Uc[1 + D];
    q.F[0] = md;
#pragma unroll
    for (int a = 0; a < ND; a++) {
        q.F[1 + a] = md * q.u[a];
        if (a == D) q.F[1 + a] = q.F[1 + a] + q.p;
    }
    q.F[nc - 1] = q.u[D] * Ep;
}

// The non-physical test of a cell (rho <= 0, p <= 0, non-finite c or H).
template <int ND>
__device__ __forceinline__ bool nonphysical_cell(double rho, const CellQ<ND> &q)
{
    return !(rho > 0.0) || !(q.p > 0.0) || !isfinite(q.c) || !isfinite(q.H);
}

// Pressure of a conserved state (used by the limiter).
template <int ND>
__device__ __forceinline__ double pressure_of(const double (&Uc)[ND + 2], double gm1)
{
    double rinv = 1.0 / Uc[0];
    double t = Uc[1] * (Uc[1] * rinv);
#pragma unroll
    for (int a = 1; a < ND; a++) t = fma(Uc[1 + a], Uc[1 + a] * rinv, t);
    return gm1 * (Uc[ND + 1] - 0.5 * t);
}

// ---------------------------------------------------------------------------
// Roe average (Sec. 5) and eigenvectors of dF_D/dU.  Field order: u-c,
// entropy, shear waves (tangential axes ascending), u+c.
// ---------------------------------------------------------------------------
// The Roe state's scalars; every eigenvector entry is one expression of
// them (l_row, r_entry), so kernels may keep these instead of the matrices.
template <int ND>
struct RoeScalars {
    double ut[ND], Ht, q2, ct, cinv, b1, b2, unc, bu, unct;
    double inv;                        // 1 / (sqrt(rho_l) + sqrt(rho_r))
};

// Roe average of two cells (velocities, enthalpies, sqrt(rho)); returns
// c~^2 (the caller counts c~^2 <= 0 as non-physical).
template <int ND, int D>
__device__ __forceinline__ double roe_state(const double (&ul)[ND], double Hl, double sl,
                                            const double (&ur)[ND], double Hr, double sr,
                                            double gm1, RoeScalars<ND> &rs)
{
    const double inv = 1.0 / (sl + sr);
#pragma unroll
    for (int a = 0; a < ND; a++) rs.ut[a] = fma(sr, ur[a], sl * ul[a]) * inv;
    rs.Ht = fma(sr, Hr, sl * Hl) * inv;
    double q2 = rs.ut[0] * rs.ut[0];
#pragma unroll
    for (int a = 1; a < ND; a++) q2 = fma(rs.ut[a], rs.ut[a], q2);
    rs.q2 = q2;
    const double c2 = gm1 * (rs.Ht - 0.5 * q2);
    rs.ct = sqrt(c2);
    rs.cinv = 1.0 / rs.ct;
    rs.b1 = gm1 * (rs.cinv * rs.cinv);
    rs.b2 = (0.5 * q2) * rs.b1;
    const double un = rs.ut[D];
    rs.unc = un * rs.cinv;
    rs.bu = rs.b1 * un;
    rs.unct = un * rs.ct;
    rs.inv = inv;
    return c2;
}

// Tangential axis of shear field k (2 <= k < ND + 1), ascending.
template <int ND, int D>
__device__ __forceinline__ int shear_axis(int k)
{
    int t = 0, kk = 2;
#pragma unroll
    for (int a = 0; a < ND; a++) {
        if (a == D) continue;
        if (kk == k) t = a;
        kk++;
    }
    return t;
}

// Row k of L = R^-1 (b1 = (gamma-1)/c^2, b2 = |u|^2 b1 / 2).
template <int ND, int D>
__device__ __forceinline__ void l_row(const RoeScalars<ND> &rs, int k, double (&l)[ND + 2])
{
    constexpr int last = ND + 1;
    if (k == 0 || k == last) {
        const bool m = (k == 0);
        l[0] = 0.5 * (m ? rs.b2 + rs.unc : rs.b2 - rs.unc);
#pragma unroll
        for (int a = 0; a < ND; a++) {
            if (a == D) l[1 + a] = 0.5 * (m ? -rs.bu - rs.cinv : rs.cinv - rs.bu);
            else l[1 + a] = 0.5 * (-(rs.b1 * rs.ut[a]));
        }
        l[last] = 0.5 * rs.b1;
    } else if (k == 1) {
        l[0] = 1.0 - rs.b2;
#pragma unroll
        for (int a = 0; a < ND; a++) l[1 + a] = rs.b1 * rs.ut[a];
        l[last] = -rs.b1;
    } else {
        const int t = shear_axis<ND, D>(k);
        l[0] = -rs.ut[t];
#pragma unroll
        for (int a = 0; a < ND; a++) l[1 + a] = (a == t) ? 1.0 : 0.0;
        l[last] = 0.0;
    }
}

// Entry (row c, column k) of R: columns (1, u - c e_D, H - u_D c),
// (1, u, |u|^2/2), shear (0, e_t, u_t), (1, u + c e_D, H + u_D c).
template <int ND, int D>
__device__ __forceinline__ double r_entry(const RoeScalars<ND> &rs, int c, int k)
{
    constexpr int last = ND + 1;
    const double un = rs.ut[D];
    if (k == 0 || k == 1 || k == last) {
        if (c == 0) return 1.0;
        if (c == last) return k == 0 ? rs.Ht - rs.unct : (k == 1 ? 0.5 * rs.q2 : rs.Ht + rs.unct);
        const int a = c - 1;
        if (a == D && k == 0) return un - rs.ct;
        if (a == D && k == last) return un + rs.ct;
        return rs.ut[a];
    }
    const int t = shear_axis<ND, D>(k);
    if (c == last) return rs.ut[t];
    return (c == 1 + t) ? 1.0 : 0.0;
}

template <int ND, int D>
__device__ __forceinline__ double roe_eigensystem(const double (&ul)[ND], double Hl, double sl,
                                                  const double (&ur)[ND], double Hr, double sr,
                                                  double gm1, double (&Lm)[ND + 2][ND + 2],
                                                  double (&Rm)[ND + 2][ND + 2],
                                                  RoeScalars<ND> *rsp = nullptr)
{
    constexpr int nc = ND + 2;
    RoeScalars<ND> rs;
    const double c2 = roe_state<ND, D>(ul, Hl, sl, ur, Hr, sr, gm1, rs);
#pragma unroll
    for (int k = 0; k < nc; k++) {
        double l[nc];
        l_row<ND, D>(rs, k, l);
#pragma unroll
        for (int c = 0; c < nc; c++) {
            Lm[k][c] = l[c];
            Rm[c][k] = r_entry<ND, D>(rs, c, k);
        }
    }
    if (rsp) *rsp = rs;
    return c2;
}

}  // namespace teno
