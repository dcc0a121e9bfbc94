// Adjoint (vector-Jacobian product) of the TENO-AA right-hand side and of the
// SSP-RK3 step, with the forward's discrete decisions frozen.
//
// With the stencil selection and the small-stencil cut-offs of every face,
// field and sign fixed (the decision record of the forward), the TENO-AA
// reconstruction (Sec. 3.3) is a fixed linear combination of the split
// characteristic fluxes, so L(U) is differentiable: the Roe average,
// eigenvectors, projection, splitting speeds (their maximising cell fixed),
// back-projection and the flux difference are smooth.  The positivity limiter
// is not differentiated (the adjoint calls reject limiter = 1).
//
// Per direction: one thread per face recomputes the face's forward values from
// the state, applies the reverse of each step and writes, for each of its 2H
// stencil positions, the adjoint of the conserved variables (direct part and
// the primitive-variable part of the Roe state and splitting speeds) and the
// adjoint of the cell's physical flux.  A gather kernel then sums, for every
// cell, the contributions of the faces whose stencils contain it (ghost
// positions mapped back by the boundary rules), applying the flux Jacobian's
// transpose once per cell.  The result is deterministic.
#include <cstring>

#include "teno.h"
#include "teno_face.cuh"

namespace teno {

struct AdjArgs {
    const double *U;        // state [nc][ncell]
    const double *lam;      // adjoint of L(U) [nc][ncell]
    const uint8_t *flags;   // decision record of this direction
    double *slots;          // [W][2 nc][nfaces]: per stencil position, the adjoint of U
                            // (direct) then of F, faces contiguous
    int64_t n[3];
    int64_t ncell, nfaces;
    int bc_lo, bc_hi;
    double inv_dx;
    Consts K;
};

template <int ND>
struct AdjSmem {
    static constexpr int nc = ND + 2;
    static constexpr int QU = 0, QF = nc, QV = 2 * nc;
    static constexpr int QP = QV + ND, QC = QP + 1, QH = QP + 2, QSR = QP + 3, QRI = QP + 4;
    static constexpr int QCI = QP + 5;                  // 1 / c
    static constexpr int QLM = QP + 6, QL0 = QLM + 1, QLP = QLM + 2, QLR = QLM + 3;
    static constexpr int NQ = QLR + 1;
};

template <int ND, int H, int TP, int TF>
constexpr size_t adj_smem_bytes()
{
    return sizeof(double) * (size_t)AdjSmem<ND>::NQ * (TF + 2 * H - 1) * TP;
}

// Reverse of cell_quantities for the primitive outputs: adjoints of the
// velocity ub, sound speed cb, enthalpy Hb and sqrt(rho) sb -> adjoint of U
// (added into Ub); cinv = 1/c and rinv = 1/rho as staged.
template <int ND, bool FULL = true>
__device__ __forceinline__ void prim_adjoint(const double (&Uc)[ND + 2], const double (&u)[ND],
                                             double p, double cinv, double sr, double rinv,
                                             const double (&ub_in)[ND], double cb, double Hb,
                                             double sb, double gamma, double gm1,
                                             double (&Ub)[ND + 2])
{
    constexpr int nc = ND + 2;
    const double E = Uc[nc - 1];
    const double Ep = E + p;
    double ub[ND];
#pragma unroll
    for (int a = 0; a < ND; a++) ub[a] = ub_in[a];
    double rb = 0.0, Eb = 0.0, mb[ND];
#pragma unroll
    for (int a = 0; a < ND; a++) mb[a] = 0.0;
    double pb = 0.0, rinvb = 0.0;
    if (FULL) {                                  // (FULL = false: Hb = sb = 0)
        rb += sb * 0.5 * (sr * rinv);            // sr = sqrt(rho): 1/sr = sr rinv
        const double Epb = Hb * rinv;            // H = Ep rinv
        rinvb = Hb * Ep;
        Eb += Epb;                               // Ep = E + p
        pb = Epb;
    }
    const double zb = cb * 0.5 * cinv;           // c = sqrt(gamma p rinv)
    pb += gamma * rinv * zb;
    rinvb += gamma * p * zb;
    Eb += gm1 * pb;                              // p = gm1 (E - ke)
    const double tb = 0.5 * (-gm1 * pb);         // ke = t / 2
#pragma unroll
    for (int a = 0; a < ND; a++) {               // t = sum m_a u_a
        mb[a] += tb * u[a];
        ub[a] += tb * Uc[1 + a];
    }
#pragma unroll
    for (int a = 0; a < ND; a++) {               // u_a = m_a rinv
        mb[a] += ub[a] * rinv;
        rinvb += ub[a] * Uc[1 + a];
    }
    rb += -rinv * rinv * rinvb;                  // rinv = 1 / rho
    Ub[0] += rb;
#pragma unroll
    for (int a = 0; a < ND; a++) Ub[1 + a] += mb[a];
    Ub[nc - 1] += Eb;
}

// Reverse of the physical flux F_D(U) (Eq. Euler) at a cell: Ub += (dF/dU)^T Fb.
template <int ND, int D>
__device__ __forceinline__ void flux_adjoint(const double (&Uc)[ND + 2], const double (&Fb)[ND + 2],
                                             double gm1, double (&Ub)[ND + 2])
{
    constexpr int nc = ND + 2;
    const double rho = Uc[0], E = Uc[nc - 1];
    const double rinv = 1.0 / rho;
    double u[ND];
#pragma unroll
    for (int a = 0; a < ND; a++) u[a] = Uc[1 + a] * rinv;
    double t = Uc[1] * u[0];
#pragma unroll
    for (int a = 1; a < ND; a++) t = fma(Uc[1 + a], u[a], t);
    const double p = gm1 * (E - 0.5 * t);
    const double Ep = E + p;
    const double md = Uc[1 + D];
    double mb[ND], ub[ND];
#pragma unroll
    for (int a = 0; a < ND; a++) { mb[a] = 0.0; ub[a] = 0.0; }
    mb[D] += Fb[0];                                  // F0 = m_D
    double pb = 0.0;
#pragma unroll
    for (int a = 0; a < ND; a++) {                   // F_{1+a} = m_D u_a (+ p)
        mb[D] += Fb[1 + a] * u[a];
        ub[a] += Fb[1 + a] * md;
    }
    pb += Fb[1 + D];
    ub[D] += Fb[nc - 1] * Ep;                        // F_E = u_D Ep
    const double Epb = Fb[nc - 1] * u[D];
    double Eb = Epb;
    pb += Epb;
    Eb += gm1 * pb;
    const double tb = 0.5 * (-gm1 * pb);
    double rinvb = 0.0;
#pragma unroll
    for (int a = 0; a < ND; a++) {
        mb[a] += tb * u[a];
        ub[a] += tb * Uc[1 + a];
    }
#pragma unroll
    for (int a = 0; a < ND; a++) {
        mb[a] += ub[a] * rinv;
        rinvb += ub[a] * Uc[1 + a];
    }
    Ub[0] += -rinv * rinv * rinvb;
#pragma unroll
    for (int a = 0; a < ND; a++) Ub[1 + a] += mb[a];
    Ub[nc - 1] += Eb;
}

template <int ND, int H, int D, int TP, int TF>
__global__ void __launch_bounds__(TP * TF) adj_face_kernel(AdjArgs a)
{
    using SL = AdjSmem<ND>;
    constexpr int nc = ND + 2, last = nc - 1, W = 2 * H;
    constexpr int NS = TF + 2 * H - 1;
    extern __shared__ double sm[];
#define SQ(q, j, p) sm[((q) * NS + (j)) * TP + (p)]
    const double gm1 = a.K.gm1, gamma = a.K.gamma;
    const int64_t n0 = a.n[0], n1 = a.n[1], nD = a.n[D];
    // TP pencils (along x for D = 1, 2; along y for D = 0) x TF faces along D.
    int64_t ps = 0, y = 0, z = 0, f0;
    if (D == 0) { f0 = (int64_t)blockIdx.x * TF; ps = (int64_t)blockIdx.y * TP; z = blockIdx.z; }
    else if (D == 1) { ps = (int64_t)blockIdx.x * TP; f0 = (int64_t)blockIdx.y * TF; z = blockIdx.z; }
    else { ps = (int64_t)blockIdx.x * TP; y = blockIdx.y; f0 = (int64_t)blockIdx.z * TF; }
    const int64_t npen = (D == 0) ? n1 : n0;

    for (int idx = threadIdx.x; idx < NS * TP; idx += TP * TF) {
        const int j = idx / TP, p = idx % TP;
        const int64_t pg = ps + p;
        if (pg >= npen) continue;
        int rule;                      // 0 copy, 1 slip-wall / 2 no-slip mirror
        const int64_t gi = map_index(f0 - H + j, nD, H, a.bc_lo, a.bc_hi, rule);
        int64_t id;
        if (D == 0) id = gi + n0 * (pg + n1 * z);
        else if (D == 1) id = pg + n0 * (gi + n1 * z);
        else id = pg + n0 * (y + n1 * gi);
        double Uc[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Uc[c] = a.U[c * a.ncell + id];
        apply_ghost_rule<ND, D>(Uc, rule, nullptr, nullptr, 0, 0, gm1);
        CellQ<ND> q;
        cell_quantities<ND, D>(Uc, a.K, q);
#pragma unroll
        for (int c = 0; c < nc; c++) { SQ(SL::QU + c, j, p) = q.U[c]; SQ(SL::QF + c, j, p) = q.F[c]; }
#pragma unroll
        for (int k = 0; k < ND; k++) SQ(SL::QV + k, j, p) = q.u[k];
        SQ(SL::QP, j, p) = q.p;
        SQ(SL::QC, j, p) = q.c;
        SQ(SL::QH, j, p) = q.H;
        SQ(SL::QSR, j, p) = q.sr;
        SQ(SL::QRI, j, p) = q.rinv;
        SQ(SL::QCI, j, p) = 1.0 / q.c;
        const double vd = q.u[D], cj = q.c;
        SQ(SL::QLM, j, p) = fabs(vd - cj);
        SQ(SL::QL0, j, p) = fabs(vd);
        SQ(SL::QLP, j, p) = fabs(vd + cj);
        SQ(SL::QLR, j, p) = fabs(vd) + cj;
    }
    __syncthreads();

    const int p = threadIdx.x % TP, fo = threadIdx.x / TP;
    const int64_t f = f0 + fo;
    if (f > nD || ps + p >= npen) return;
    const int jl = fo + H - 1, jr = fo + H;

    int64_t flin, cstride, cbase;      // face index; neighbouring cells along D
    const int64_t pg = ps + p;
    if (D == 0) { flin = f + (n0 + 1) * (pg + n1 * z); cbase = n0 * (pg + n1 * z); cstride = 1; }
    else if (D == 1) { flin = pg + n0 * (f + (n1 + 1) * z); cbase = pg + n0 * n1 * z; cstride = n0; }
    else { flin = pg + n0 * (y + n1 * f); cbase = pg + n0 * y; cstride = n0 * n1; }

    // Adjoint of this face's flux from the adjoint of L: face f is the right
    // face of cell f-1 (-F/dx) and the left face of cell f (+F/dx).
    double Fb[nc];
#pragma unroll
    for (int c = 0; c < nc; c++) {
        const double lr = (f < nD) ? a.lam[c * a.ncell + cbase + f * cstride] : 0.0;
        const double ll = (f > 0) ? a.lam[c * a.ncell + cbase + (f - 1) * cstride] : 0.0;
        Fb[c] = (lr - ll) * a.inv_dx;
    }

    // Forward Roe state and eigenvectors.
    double ul[ND], ur[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) { ul[k] = SQ(SL::QV + k, jl, p); ur[k] = SQ(SL::QV + k, jr, p); }
    const double Hl = SQ(SL::QH, jl, p), Hr = SQ(SL::QH, jr, p);
    const double sl = SQ(SL::QSR, jl, p), srr = SQ(SL::QSR, jr, p);
    double Lm[nc][nc], Rm[nc][nc];
    RoeScalars<ND> rs;
    roe_eigensystem<ND, D>(ul, Hl, sl, ur, Hr, srr, gm1, Lm, Rm, &rs);
    const double inv = rs.inv;
    double ut[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) ut[k] = rs.ut[k];
    const double Ht = rs.Ht, q2 = rs.q2, ct = rs.ct, cinv = rs.cinv, b1 = rs.b1;
    const double un = ut[D];

    // Splitting speeds and their maximising cells (first maximum, as forward).
    double am = 0.0, a0 = 0.0, ap = 0.0, ar = 0.0;
    int jm = 0, j0 = 0, jp = 0, jrr = 0;
#pragma unroll
    for (int j = 0; j < W; j++) {
        const double em = SQ(SL::QLM, fo + j, p), e0 = SQ(SL::QL0, fo + j, p);
        const double ep = SQ(SL::QLP, fo + j, p), er = SQ(SL::QLR, fo + j, p);
        if (j == 0 || speed_gt(em, am)) { am = em; jm = j; }
        if (j == 0 || speed_gt(e0, a0)) { a0 = e0; j0 = j; }
        if (j == 0 || speed_gt(ep, ap)) { ap = ep; jp = j; }
        if (j == 0 || speed_gt(er, ar)) { ar = er; jrr = j; }
    }

    // hb_k = sum_c R[c][k] Fb_c (adjoint of h_k = f+_k + f-_k).
    double hb[nc];
#pragma unroll
    for (int k = 0; k < nc; k++) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < nc; c++) s = fma(Rm[c][k], Fb[c], s);
        hb[k] = s;
    }
    const uint8_t *fl = a.flags + flin * nc * 2;

    // Adjoints of the Roe scalars.
    double b1b = 0.0, b2b = 0.0, uncb = 0.0, cinvb = 0.0, bub = 0.0, Htb = 0.0, q2b = 0.0;
    double ctb = 0.0, unb = 0.0, unctb = 0.0, utb[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) utb[k] = 0.0;
    double alphab[nc];

    // A shear field's row of L is (-u_t, e_t, 0): only its columns 0 and
    // 1 + t enter the products below (branches uniform over the warp).
    // With P_j = (c+_j + c-_j)/2 and Q_j = (c+_j - c-_j)/2 the frozen
    // reconstruction gives h_k = alpha sum_j Q_j w_j + sum_j P_j g_j; with
    // A_c = sum_j Q_j U_cj and B_c = sum_j P_j F_cj (w = l.U, g = l.F):
    // sum_j Q_j w_j = l.A, h_k = alpha l.A + l.B, and the adjoint of the
    // row l is hb_k (alpha A + B).  A and B depend on the field only through
    // its two decision bytes' low five bits (the frozen coefficients), so
    // they are formed again only when those change from the previous field
    // (in smooth regions every field has the same selection).
    double A[nc], B[nc];
    int abkey = -1;
#pragma unroll 1
    for (int k = 0; k < nc; k++) {
        const bool shear = (k >= 2 && k < last);
        const int tk = shear ? shear_axis<ND, D>(k) : 0;
        double lrow[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) {
            double lv = Lm[0][c];
#pragma unroll
            for (int kk = 1; kk < nc; kk++)
                if (k == kk) lv = Lm[kk][c];
            lrow[c] = lv;
        }
        double hbk = hb[0];
#pragma unroll
        for (int kk = 1; kk < nc; kk++)
            if (k == kk) hbk = hb[kk];
        const double alpha = a.K.split ? ar : (k == 0 ? am : (k == last ? ap : a0));
        const uint8_t flp = fl[2 * k], flm = fl[2 * k + 1];
        const int key = (flp & 31) | ((flm & 31) << 5);
        if (key != abkey) {
            // accumulated with 2 Q_j, 2 P_j, halved after
#pragma unroll
            for (int c = 0; c < nc; c++) { A[c] = 0.0; B[c] = 0.0; }
#pragma unroll
            for (int j = 0; j < W; j++) {
                const double cp = frozen_coef<H>(flp, j);          // v+ index j <-> cell j
                const double cm = frozen_coef<H>(flm, W - 1 - j);  // v- index W-1-j <-> cell j
                const double Pc = cp + cm, Qc = cp - cm;
#pragma unroll
                for (int c = 0; c < nc; c++) {
                    A[c] = fma(Qc, SQ(SL::QU + c, fo + j, p), A[c]);
                    B[c] = fma(Pc, SQ(SL::QF + c, fo + j, p), B[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < nc; c++) { A[c] *= 0.5; B[c] *= 0.5; }
            abkey = key;
        }
        double wq = lrow[0] * A[0], gp = lrow[0] * B[0];
#pragma unroll
        for (int c = 1; c < nc; c++) {
            if (shear && c != 1 + tk) continue;
            wq = fma(lrow[c], A[c], wq);
            gp = fma(lrow[c], B[c], gp);
        }
        const double hk = fma(alpha, wq, gp);
        double Lb[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Lb[c] = (shear && c != 0) ? 0.0 : fma(alpha, A[c], B[c]);
        double ab = hbk * wq;
#pragma unroll
        for (int kk = 0; kk < nc; kk++)
            if (k == kk) alphab[kk] = ab;
#pragma unroll
        for (int c = 0; c < nc; c++) Lb[c] = (shear && c != 0) ? 0.0 : Lb[c] * hbk;

        // R column k: Rb[c] = Fb_c h_k.
        if (k == 0) {
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                const double rb = Fb[1 + aa] * hk;
                if (aa == D) { unb += rb; ctb -= rb; } else utb[aa] += rb;
            }
            const double rbE = Fb[last] * hk;
            Htb += rbE;
            unctb -= rbE;
        } else if (k == 1) {
#pragma unroll
            for (int aa = 0; aa < ND; aa++) utb[aa] += Fb[1 + aa] * hk;
            q2b += 0.5 * (Fb[last] * hk);
        } else if (k == last) {
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                const double rb = Fb[1 + aa] * hk;
                if (aa == D) { unb += rb; ctb += rb; } else utb[aa] += rb;
            }
            const double rbE = Fb[last] * hk;
            Htb += rbE;
            unctb += rbE;
        } else {
            int t = 0, kk = 2;
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                if (aa == D) continue;
                if (kk == k) t = aa;
                kk++;
            }
#pragma unroll
            for (int aa = 0; aa < ND; aa++)
                if (aa == t) utb[aa] += Fb[last] * hk;
        }
        // L row k.
        if (k == 0 || k == last) {
            const double sg = (k == 0) ? 1.0 : -1.0;
            b2b += 0.5 * Lb[0];
            uncb += sg * 0.5 * Lb[0];
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                if (aa == D) {
                    bub += -0.5 * Lb[1 + aa];
                    cinvb += -sg * 0.5 * Lb[1 + aa];
                } else {
                    b1b += -0.5 * ut[aa] * Lb[1 + aa];
                    utb[aa] += -0.5 * b1 * Lb[1 + aa];
                }
            }
            b1b += 0.5 * Lb[last];
        } else if (k == 1) {
            b2b -= Lb[0];
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                b1b += ut[aa] * Lb[1 + aa];
                utb[aa] += b1 * Lb[1 + aa];
            }
            b1b -= Lb[last];
        } else {
            int t = 0, kk = 2;
#pragma unroll
            for (int aa = 0; aa < ND; aa++) {
                if (aa == D) continue;
                if (kk == k) t = aa;
                kk++;
            }
#pragma unroll
            for (int aa = 0; aa < ND; aa++)
                if (aa == t) utb[aa] -= Lb[0];
        }
    }

    // Chain through the Roe scalars to the two cells' velocity, enthalpy, sqrt(rho).
    unb += unctb * ct;
    ctb += unctb * un;
    b1b += bub * un;
    unb += bub * b1;
    unb += uncb * cinv;
    cinvb += uncb * un;
    q2b += 0.5 * b1 * b2b;
    b1b += 0.5 * q2 * b2b;
    cinvb += 2.0 * gm1 * cinv * b1b;
    ctb += -cinv * cinv * cinvb;
    const double c2b = 0.5 * ctb * cinv;
    Htb += gm1 * c2b;
    q2b += -0.5 * gm1 * c2b;
#pragma unroll
    for (int aa = 0; aa < ND; aa++) utb[aa] += 2.0 * ut[aa] * q2b;
    utb[D] += unb;
    double invb = 0.0, slb = 0.0, srb = 0.0, Hlb, Hrb, ulb[ND], urb[ND];
    {
        const double N = fma(srr, Hr, sl * Hl);
        const double Nb = Htb * inv;
        invb += N * Htb;
        Hlb = sl * Nb;
        Hrb = srr * Nb;
        slb += Hl * Nb;
        srb += Hr * Nb;
    }
#pragma unroll
    for (int aa = 0; aa < ND; aa++) {
        const double N = fma(srr, ur[aa], sl * ul[aa]);
        const double Nb = utb[aa] * inv;
        invb += N * utb[aa];
        ulb[aa] = sl * Nb;
        urb[aa] = srr * Nb;
        slb += ul[aa] * Nb;
        srb += ur[aa] * Nb;
    }
    {
        const double Sb = -inv * inv * invb;
        slb += Sb;
        srb += Sb;
    }

    // Splitting-speed adjoints onto their maximising cells.
    double udb_m = 0.0, cb_m = 0.0, udb_0 = 0.0, udb_p = 0.0, cb_p = 0.0, udb_r = 0.0, cb_r = 0.0;
    if (a.K.split) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < nc; k++) s += alphab[k];
        const double vd = SQ(SL::QV + D, fo + jrr, p);
        udb_r = (vd > 0.0 ? 1.0 : (vd < 0.0 ? -1.0 : 0.0)) * s;
        cb_r = s;
    } else {
        const double cm_ = SQ(SL::QC, fo + jm, p), vm = SQ(SL::QV + D, fo + jm, p);
        const double lmv = vm - cm_;
        const double sm_ = lmv > 0.0 ? 1.0 : (lmv < 0.0 ? -1.0 : 0.0);
        udb_m = sm_ * alphab[0];
        cb_m = -sm_ * alphab[0];
        double s0 = 0.0;
#pragma unroll
        for (int k = 1; k < nc - 1; k++) s0 += alphab[k];
        const double v0 = SQ(SL::QV + D, fo + j0, p);
        udb_0 = (v0 > 0.0 ? 1.0 : (v0 < 0.0 ? -1.0 : 0.0)) * s0;
        const double cp_ = SQ(SL::QC, fo + jp, p), vp = SQ(SL::QV + D, fo + jp, p);
        const double lpv = vp + cp_;
        const double sp_ = lpv > 0.0 ? 1.0 : (lpv < 0.0 ? -1.0 : 0.0);
        udb_p = sp_ * alphab[last];
        cb_p = sp_ * alphab[last];
    }

    // Per stencil cell: adjoint of U through the projection rows, and of the
    // cell's physical flux (the primitive-variable parts follow).
    // slot (j, q) of this face: a.slots[(j 2nc + q) nfaces + flin]
    double *out = a.slots + flin;
    const int64_t fs = a.nfaces;
    // w_j = l.U_j and g_j enter h_k with weights alpha Q_j and P_j:
    // wb = (alpha hb_k / 2)(c+ - c-), gb = (hb_k / 2)(c+ + c-).
    double sw[nc], sg[nc];
#pragma unroll
    for (int k = 0; k < nc; k++) {
        const double alpha = a.K.split ? ar : (k == 0 ? am : (k == last ? ap : a0));
        sg[k] = 0.5 * hb[k];
        sw[k] = alpha * sg[k];
    }
    // Every field with the same frozen coefficients (each sign's decision
    // bytes agree in their low five bits across the fields, as in smooth
    // regions): the sums over the fields factor out of the stencil loop,
    // Ub_c(j) = (c+_j - c-_j) sum_k L_kc sw_k and Fcb_c(j) = (c+_j + c-_j)
    // sum_k L_kc sg_k.
    bool uniform = true;
#pragma unroll
    for (int k = 1; k < nc; k++)
        uniform = uniform && ((fl[2 * k] ^ fl[0]) & 31) == 0 && ((fl[2 * k + 1] ^ fl[1]) & 31) == 0;
    if (uniform) {
        double M[nc], N[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) { M[c] = 0.0; N[c] = 0.0; }
#pragma unroll
        for (int k = 0; k < nc; k++) {
            const bool shear = (k >= 2 && k < last);
            const int tk = shear ? shear_axis<ND, D>(k) : 0;
#pragma unroll
            for (int c = 0; c < nc; c++) {
                if (shear && c != 0 && c != 1 + tk) continue;    // zeros of a shear row
                M[c] = fma(Lm[k][c], sw[k], M[c]);
                N[c] = fma(Lm[k][c], sg[k], N[c]);
            }
        }
#pragma unroll 1
        for (int j = 0; j < W; j++) {
            const double cp = frozen_coef<H>(fl[0], j);
            const double cm = frozen_coef<H>(fl[1], W - 1 - j);
            const double qd = cp - cm, qs = cp + cm;
#pragma unroll
            for (int c = 0; c < nc; c++) {
                out[(j * 2 * nc + c) * fs] = qd * M[c];
                out[(j * 2 * nc + nc + c) * fs] = qs * N[c];
            }
        }
    } else {
#pragma unroll 1
        for (int j = 0; j < W; j++) {
            double Ub[nc], Fcb[nc];
#pragma unroll
            for (int c = 0; c < nc; c++) { Ub[c] = 0.0; Fcb[c] = 0.0; }
#pragma unroll
            for (int k = 0; k < nc; k++) {
                const double cp = frozen_coef<H>(fl[2 * k], j);
                const double cm = frozen_coef<H>(fl[2 * k + 1], W - 1 - j);
                const double wb = sw[k] * (cp - cm);
                const double gb = sg[k] * (cp + cm);
                const bool shear = (k >= 2 && k < last);
                const int tk = shear ? shear_axis<ND, D>(k) : 0;
#pragma unroll
                for (int c = 0; c < nc; c++) {
                    if (shear && c != 0 && c != 1 + tk) continue;    // zeros of a shear row
                    Ub[c] = fma(Lm[k][c], wb, Ub[c]);
                    Fcb[c] = fma(Lm[k][c], gb, Fcb[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < nc; c++) {
                out[(j * 2 * nc + c) * fs] = Ub[c];
                out[(j * 2 * nc + nc + c) * fs] = Fcb[c];
            }
        }
    }

    // Primitive-variable parts, one contribution at a time (the same number
    // for every face, so no lane waits on another's): the Roe state's cells
    // i and i+1, and the splitting speeds at their maximising cells.  Each is
    // added into the slot written above.
#pragma unroll
    for (int e = 0; e < 5; e++) {
        if (a.K.split && e > 2) continue;
        int je;
        double ue[ND], ce = 0.0, He = 0.0, se = 0.0;
#pragma unroll
        for (int aa = 0; aa < ND; aa++) ue[aa] = 0.0;
        if (e == 0) {                            // cell i of the Roe average
            je = H - 1;
#pragma unroll
            for (int aa = 0; aa < ND; aa++) ue[aa] = ulb[aa];
            He = Hlb;
            se = slb;
        } else if (e == 1) {                     // cell i+1
            je = H;
#pragma unroll
            for (int aa = 0; aa < ND; aa++) ue[aa] = urb[aa];
            He = Hrb;
            se = srb;
        } else if (a.K.split) {
            je = jrr; ue[D] = udb_r; ce = cb_r;
        } else if (e == 2) {
            je = jm; ue[D] = udb_m; ce = cb_m;
        } else if (e == 3) {
            je = j0; ue[D] = udb_0;
        } else {
            je = jp; ue[D] = udb_p; ce = cb_p;
        }
        double Uc[nc], u[ND], Ub[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) { Uc[c] = SQ(SL::QU + c, fo + je, p); Ub[c] = 0.0; }
#pragma unroll
        for (int aa = 0; aa < ND; aa++) u[aa] = SQ(SL::QV + aa, fo + je, p);
        if (e < 2)
            prim_adjoint<ND, true>(Uc, u, SQ(SL::QP, fo + je, p), SQ(SL::QCI, fo + je, p),
                                   SQ(SL::QSR, fo + je, p), SQ(SL::QRI, fo + je, p), ue, ce, He,
                                   se, gamma, gm1, Ub);
        else                                     // splitting speeds: u_D and c only
            prim_adjoint<ND, false>(Uc, u, SQ(SL::QP, fo + je, p), SQ(SL::QCI, fo + je, p),
                                    SQ(SL::QSR, fo + je, p), SQ(SL::QRI, fo + je, p), ue, ce, He,
                                    se, gamma, gm1, Ub);
#pragma unroll
        for (int c = 0; c < nc; c++) out[(je * 2 * nc + c) * fs] += Ub[c];
    }
#undef SQ
}

// mu_i (+)= sum over the faces whose stencils contain cell i (directly or as a
// ghost image) of their slot adjoints; the flux part goes through the flux
// Jacobian's transpose at the (ghost) state, slip-wall images through the
// mirror.
// Sum of the slots of the faces whose stencils cover position g along D
// (a cell or one of its ghost images) at the transverse position (x, y, z):
// face f holds position g at stencil index j = g - f + H.  A position whose
// 2H faces all exist (the interior) takes an unrolled loop, so that its 4 H
// nc loads are independent.
template <int ND, int H, int D>
__device__ __forceinline__ void gather_position(const AdjArgs &a, int64_t g, int64_t x, int64_t y,
                                                int64_t z, double (&Us)[ND + 2],
                                                double (&Fm)[ND + 2])
{
    constexpr int nc = ND + 2, W = 2 * H;
    const int64_t n0 = a.n[0], n1 = a.n[1], nD = a.n[D];
    // linear face index = fb + f * fs
    int64_t fb, fs;
    if (D == 0) { fb = (n0 + 1) * (y + n1 * z); fs = 1; }
    else if (D == 1) { fb = x + n0 * (n1 + 1) * z; fs = n0; }
    else { fb = x + n0 * y; fs = n0 * n1; }
#pragma unroll
    for (int c = 0; c < nc; c++) { Us[c] = 0.0; Fm[c] = 0.0; }
    if (g - H + 1 >= 0 && g + H <= nD) {
#pragma unroll
        for (int t = 0; t < W; t++) {
            const int64_t f = g - H + 1 + t;
            const double *sl = a.slots + (size_t)(W - 1 - t) * 2 * nc * a.nfaces + fb + f * fs;
#pragma unroll
            for (int c = 0; c < nc; c++) {
                Us[c] += sl[c * a.nfaces];
                Fm[c] += sl[(nc + c) * a.nfaces];
            }
        }
    } else {
        const int64_t flo = g - H + 1 > 0 ? g - H + 1 : 0;
        const int64_t fhi = g + H < nD ? g + H : nD;
        for (int64_t f = flo; f <= fhi; f++) {
            const double *sl = a.slots + (size_t)(g - f + H) * 2 * nc * a.nfaces + fb + f * fs;
#pragma unroll
            for (int c = 0; c < nc; c++) {
                Us[c] += sl[c * a.nfaces];
                Fm[c] += sl[(nc + c) * a.nfaces];
            }
        }
    }
}

template <int ND, int H, int D>
__global__ void adj_gather_kernel(AdjArgs a, double *mu, int accumulate)
{
    constexpr int nc = ND + 2;
    const int64_t n0 = a.n[0], n1 = a.n[1], nD = a.n[D];
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < a.ncell;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = id % n0, y = (id / n0) % n1, z = id / (n0 * n1);
        const int64_t i = (D == 0) ? x : (D == 1 ? y : z);
        double Uc[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Uc[c] = a.U[c * a.ncell + id];
        // the cell itself
        double Ut[nc], Fs[nc];
        gather_position<ND, H, D>(a, i, x, y, z, Ut, Fs);
        if (i < H || i >= nD - H) {
            // ghost images that map to cell i, with the mirror rule of each
            // image (0 none, 1 slip wall, 2 no-slip)
            int64_t gs[2 * 5 + 2];
            int ms[2 * 5 + 2];
            int ng = 0;
            if (a.bc_lo == 0) { gs[ng] = i - nD; ms[ng] = 0; ng++; }
            if (a.bc_hi == 0) { gs[ng] = i + nD; ms[ng] = 0; ng++; }
            if (a.bc_lo == 1 && i == 0)
                for (int r = 1; r <= H; r++) { gs[ng] = -r; ms[ng] = 0; ng++; }
            if (a.bc_hi == 1 && i == nD - 1)
                for (int r = 0; r < H; r++) { gs[ng] = nD + r; ms[ng] = 0; ng++; }
            if ((a.bc_lo == 2 || a.bc_lo == 3) && i < H) { gs[ng] = -i - 1; ms[ng] = a.bc_lo - 1; ng++; }
            if ((a.bc_hi == 2 || a.bc_hi == 3) && i >= nD - H) {
                gs[ng] = 2 * nD - 1 - i; ms[ng] = a.bc_hi - 1; ng++;
            }
            for (int q = 0; q < ng; q++) {
                const int64_t g = gs[q];
                if (g < -H || g > nD + H - 1) continue;
                double Us[nc], Fm[nc];
                gather_position<ND, H, D>(a, g, x, y, z, Us, Fm);
                if (!ms[q]) {
#pragma unroll
                    for (int c = 0; c < nc; c++) { Ut[c] += Us[c]; Fs[c] += Fm[c]; }
                } else {
                    // the image is the mirror map M U (M diagonal, +-1): its flux
                    // Jacobian is taken at M U and M^T = M maps the adjoint back
                    double Ug[nc], Ub[nc];
#pragma unroll
                    for (int c = 0; c < nc; c++) { Ug[c] = Uc[c]; Ub[c] = Us[c]; }
                    apply_ghost_rule<ND, D>(Ug, ms[q], nullptr, nullptr, 0, 0, a.K.gm1);
                    flux_adjoint<ND, D>(Ug, Fm, a.K.gm1, Ub);
                    apply_ghost_rule<ND, D>(Ub, ms[q], nullptr, nullptr, 0, 0, a.K.gm1);
#pragma unroll
                    for (int c = 0; c < nc; c++) Ut[c] += Ub[c];
                }
            }
        }
        flux_adjoint<ND, D>(Uc, Fs, a.K.gm1, Ut);
#pragma unroll
        for (int c = 0; c < nc; c++)
            mu[c * a.ncell + id] = accumulate ? mu[c * a.ncell + id] + Ut[c] : Ut[c];
    }
}

// Elementwise combinations of the SSP-RK3 reverse sweep.
__global__ void axpby_kernel(int64_t len, double a, const double *x, double b, const double *y,
                             double *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

template <int ND, int H, int D>
cudaError_t launch_adj_direction(const AdjArgs &a, double *mu, int accumulate, cudaStream_t s)
{
    constexpr int TP = (ND == 1) ? 1 : 4;
    constexpr int TF = (ND == 1) ? 64 : 32;
    constexpr size_t smem = adj_smem_bytes<ND, H, TP, TF>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(adj_face_kernel<ND, H, D, TP, TF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    dim3 grid;
    if (D == 0) grid = dim3((unsigned)((a.n[0] + 1 + TF - 1) / TF), (unsigned)((a.n[1] + TP - 1) / TP), (unsigned)a.n[2]);
    else if (D == 1) grid = dim3((unsigned)((a.n[0] + TP - 1) / TP), (unsigned)((a.n[1] + 1 + TF - 1) / TF), (unsigned)a.n[2]);
    else grid = dim3((unsigned)((a.n[0] + TP - 1) / TP), (unsigned)a.n[1], (unsigned)((a.n[2] + 1 + TF - 1) / TF));
    adj_face_kernel<ND, H, D, TP, TF><<<grid, TP * TF, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks = (a.ncell + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    adj_gather_kernel<ND, H, D><<<(unsigned)blocks, 256, 0, s>>>(a, mu, accumulate);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_adj(int nd, int d, const AdjArgs &a, double *mu, int acc, cudaStream_t s)
{
    switch (nd * 3 + d) {
    case 3: return launch_adj_direction<1, H, 0>(a, mu, acc, s);
    case 6: return launch_adj_direction<2, H, 0>(a, mu, acc, s);
    case 7: return launch_adj_direction<2, H, 1>(a, mu, acc, s);
    case 9: return launch_adj_direction<3, H, 0>(a, mu, acc, s);
    case 10: return launch_adj_direction<3, H, 1>(a, mu, acc, s);
    case 11: return launch_adj_direction<3, H, 2>(a, mu, acc, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace teno

using namespace teno;

namespace {

int64_t cells_of(const teno_params *p) { return p->n[0] * p->n[1] * p->n[2]; }

int64_t faces_of(const teno_params *p, int d)
{
    int64_t s = 1;
    for (int a = 0; a < 3; a++) s *= (a == d) ? p->n[a] + 1 : p->n[a];
    return s;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct AdjLayout {
    size_t fwd, flags, slots, t0, t1, t2, total;
};

AdjLayout adj_layout(const teno_params *p)
{
    AdjLayout L;
    size_t fwd = 0;
    teno_workspace_bytes(p, &fwd);
    size_t fb = 0;
    teno_flags_bytes(p, &fb);
    const int nc = p->ndim + 2, W = p->scheme;
    int64_t maxf = 0;
    for (int d = 0; d < p->ndim; d++) maxf = faces_of(p, d) > maxf ? faces_of(p, d) : maxf;
    const size_t state = sizeof(double) * (size_t)nc * cells_of(p);
    size_t off = 0;
    L.fwd = off;
    off += a256(fwd);
    L.flags = off;
    off += a256(fb);
    L.slots = off;
    off += a256(sizeof(double) * (size_t)maxf * W * 2 * nc);
    L.t0 = off;
    off += a256(state);
    L.t1 = off;
    off += a256(state);
    L.t2 = off;
    off += a256(state);
    L.total = off;
    return L;
}

Consts consts_adj(const teno_params *p)
{
    Consts K;
    K.gamma = p->gamma;
    K.gm1 = p->gamma - 1.0;
    K.alpha1 = p->ct_alpha1;
    K.alpha2 = p->ct_alpha2;
    K.cr = p->ct_cr;
    K.eps_beta = p->eps_beta;
    K.eps_eta = p->eps_eta;
    K.lim_eps = p->limiter_eps;
    K.split = p->flux_split;
    K.limiter = 0;
    return K;
}

#define CUDA_TRY(x)                                   \
    do {                                              \
        if ((x) != cudaSuccess) return TENO_ECUDA;    \
    } while (0)

int check_adj(const teno_params *p, void *ws, size_t ws_bytes)
{
    size_t b;
    int r = teno_workspace_bytes(p, &b);
    if (r) return r;
    if (p->limiter) return TENO_EINVAL;
    for (int d = 0; d < p->ndim; d++)
        if (p->bc_lo[d] >= TENO_BC_DIRICHLET || p->bc_hi[d] >= TENO_BC_DIRICHLET) return TENO_EINVAL;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < adj_layout(p).total) return TENO_EINVAL;
    return TENO_OK;
}

void launch_axpby(int64_t len, double a, const double *x, double b, const double *y, double *out,
                  cudaStream_t s)
{
    int64_t blocks = (len + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    axpby_kernel<<<(unsigned)blocks, 256, 0, s>>>(len, a, x, b, y, out);
}

int rhs_vjp_impl(const teno_params *p, const double *U, const double *lam, const uint8_t *flags,
                 double *mu, char *ws, cudaStream_t s)
{
    const AdjLayout L = adj_layout(p);
    const int nc = p->ndim + 2;
    if (!flags) {
        uint8_t *fl = (uint8_t *)(ws + L.flags);
        double *scratch = (double *)(ws + L.t2);
        size_t fb;
        teno_workspace_bytes(p, &fb);
        int r = teno_rhs(p, U, scratch, 0.0, fl, ws + L.fwd, fb, s);
        if (r) return r;
        flags = fl;
    }
    const uint8_t *fl = flags;
    for (int d = 0; d < p->ndim; d++) {
        AdjArgs a;
        a.U = U;
        a.lam = lam;
        a.flags = fl;
        a.slots = (double *)(ws + L.slots);
        for (int k = 0; k < 3; k++) a.n[k] = p->n[k];
        a.ncell = cells_of(p);
        a.nfaces = faces_of(p, d);
        a.bc_lo = p->bc_lo[d];
        a.bc_hi = p->bc_hi[d];
        a.inv_dx = 1.0 / p->dx[d];
        a.K = consts_adj(p);
        cudaError_t e = (p->scheme == 8)    ? launch_adj<4>(p->ndim, d, a, mu, d > 0, s)
                        : (p->scheme == 10) ? launch_adj<5>(p->ndim, d, a, mu, d > 0, s)
                                            : launch_adj<6>(p->ndim, d, a, mu, d > 0, s);
        if (e != cudaSuccess) return TENO_ECUDA;
        fl += (size_t)faces_of(p, d) * nc * 2;
    }
    return TENO_OK;
}

}  // namespace

extern "C" {

int teno_adjoint_workspace_bytes(const teno_params *p, size_t *bytes)
{
    size_t b;
    int r = teno_workspace_bytes(p, &b);
    if (r) return r;
    if (!bytes) return TENO_EINVAL;
    *bytes = adj_layout(p).total;
    return TENO_OK;
}

int teno_rhs_vjp(const teno_params *p, const double *U, const double *lam, const uint8_t *flags,
                 double *mu, void *ws, size_t ws_bytes, void *stream)
{
    int r = check_adj(p, ws, ws_bytes);
    if (r) return r;
    if (!U || !lam || !mu || ((uintptr_t)U & 15) || ((uintptr_t)lam & 15) || ((uintptr_t)mu & 15))
        return TENO_EINVAL;
    if (mu == U || mu == lam) return TENO_EINVAL;
    return rhs_vjp_impl(p, U, lam, flags, mu, (char *)ws, (cudaStream_t)stream);
}

int teno_rk3_step_vjp(const teno_params *p, const double *Un, const double *U1, const double *U2,
                      const uint8_t *flags, double dt, double *abar, void *ws, size_t ws_bytes,
                      void *stream)
{
    int r = check_adj(p, ws, ws_bytes);
    if (r) return r;
    if (!Un || !U1 || !U2 || !abar || !flags || !(dt >= 0.0)) return TENO_EINVAL;
    const AdjLayout L = adj_layout(p);
    size_t flb;
    teno_flags_bytes(p, &flb);
    cudaStream_t s = (cudaStream_t)stream;
    char *w = (char *)ws;
    const int64_t len = (int64_t)(p->ndim + 2) * cells_of(p);
    double *t = (double *)(w + L.t0), *mu = (double *)(w + L.t1), *acc = (double *)(w + L.t2);
    // stage 3: U+ = 1/3 Un + 2/3 (U2 + dt L(U2))
    launch_axpby(len, 2.0 / 3.0, abar, 0.0, nullptr, t, s);            // t = 2/3 abar
    if ((r = rhs_vjp_impl(p, U2, t, flags + 2 * flb, mu, w, s))) return r;
    launch_axpby(len, 1.0, t, dt, mu, t, s);                             // Ubar2 = t + dt mu
    launch_axpby(len, 1.0 / 3.0, abar, 0.0, nullptr, acc, s);          // Ubar_n = 1/3 abar
    // stage 2: U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
    launch_axpby(len, 0.75, t, 1.0, acc, acc, s);                        // Ubar_n += 3/4 Ubar2
    launch_axpby(len, 0.25, t, 0.0, nullptr, t, s);                      // t = 1/4 Ubar2
    if ((r = rhs_vjp_impl(p, U1, t, flags + flb, mu, w, s))) return r;
    launch_axpby(len, 1.0, t, dt, mu, t, s);                             // Ubar1 = t + dt mu
    // stage 1: U1 = Un + dt L(Un)
    if ((r = rhs_vjp_impl(p, Un, t, flags, mu, w, s))) return r;
    launch_axpby(len, 1.0, t, 1.0, acc, acc, s);                         // Ubar_n += Ubar1
    launch_axpby(len, dt, mu, 1.0, acc, abar, s);                        // abar = Ubar_n + dt mu
    CUDA_TRY(cudaGetLastError());
    return TENO_OK;
}

}  // extern "C"
