// Face-flux sweep along one direction: for every face i+1/2 of the face grid,
// Roe average -> eigenvectors -> characteristic projection of the 2H-cell
// stencil -> LLF/Rusanov split -> TENO-AA reconstruction of f+ and f- per
// field -> back-projection -> positivity limiter (arXiv 2109.14340, Sec. 3-5).
//
// Tiling: a block owns TF consecutive faces along the sweep axis D for TP
// pencils adjacent in x.  It stages the TF + 2H - 1 cells those faces touch
// (ghost cells resolved by the boundary rules of App. A) in shared memory as
// per-cell primitive quantities, then one thread computes one face.  U and F
// are staged halved (exact: a power of two), so that the projections give
// the halved characteristic variables and fluxes w/2, g/2 directly and the
// split fluxes (g +- alpha w)/2 need no further scaling.
#pragma once

#include "teno_dev.cuh"
#include "teno_fast.cuh"

namespace teno {

struct FaceArgs {
    const double *U;       // state, [nc][ncell]
    const double *P;       // primitives of U ([PrimRows::NP][ncell], store_prims) or
                           // nullptr: computed while staging
    double *F;             // face fluxes of direction D, [nc][nfaces]
    uint8_t *flags;        // decision record of direction D or nullptr
    const uint8_t *frozen; // recorded decisions to apply instead of deciding, or nullptr
    uint16_t *argmax;      // per face: the maximising stencil cells of the splitting
                           // speeds (4 bits each: u-c, u, u+c, |u|+c), or nullptr
    const uint16_t *frozen_argmax;   // recorded maximising cells to apply, or nullptr
    uint8_t *limrec;       // per face: 1 where the positivity limiter bound, or nullptr
    Status *st;
    int64_t n[3];
    int64_t ncell, nfaces;
    int bc_lo, bc_hi;      // boundary rules at the two ends of axis D
    const double *bcs_lo, *bcs_hi;   // Dirichlet boundary-face states or halo arrays of
                                     // axis D, or nullptr
    const double *lam;     // limiter's effective dt/dx for this direction (device)
    int fast;              // 1: certified FP32 decision filter first
    int need_ct;           // 1: recorded decision bytes carry their C_T exponent; 0: only
                           // where it decided (the selection bits are exact either way)
    int count_cells;       // 1: count the non-physical cells this sweep owns (one
                           // sweep per evaluation does, so each cell is counted once)
    int skip_last;         // 1: face n of each line is not computed (periodic axis, no
                           // decision record: its flux is face 0's, bitwise)
    unsigned long long *exact_count;   // adds the exact-path reconstructions, or nullptr
    FastK FK;
    Consts K;
};

// App. A ghost-cell rules along one axis.  Returns the interior cell whose
// state defines the (possibly ghost) cell j, and the rule to apply to it:
// 0 copy, 1 slip-wall mirror (wall-normal momentum negated), 2 no-slip
// mirror (all momentum negated), 3 / 4 Dirichlet reflection about the low /
// high boundary-face state; or, for a side whose ghost cells are a
// neighbouring sub-domain's cells (TENO_BC_HALO), rule 5 / 6 and the plane of
// the side's halo array (0 .. H-1 in ascending position: cell -H + q below,
// n + q above).  The final clamps only matter for padding cells beyond the
// last face of a tile.
__device__ __forceinline__ int64_t map_index(int64_t j, int64_t n, int H, int lo, int hi, int &rule)
{
    rule = 0;
    int64_t r = j;
    if (j < 0) {
        if (lo == 0) r = ((j % n) + n) % n;
        else if (lo == 1) r = 0;
        else if (lo == 5) { rule = 5; r = j + H; return r < 0 ? 0 : r; }
        else { rule = lo == 2 ? 1 : (lo == 3 ? 2 : 3); r = -j - 1; }
    } else if (j >= n) {
        if (hi == 0) r = j % n;
        else if (hi == 1) r = n - 1;
        else if (hi == 5) { rule = 6; r = j - n; return r >= H ? H - 1 : r; }
        else { rule = hi == 2 ? 1 : (hi == 3 ? 2 : 4); r = 2 * n - 1 - j; }
    }
    return r < 0 ? 0 : (r >= n ? n - 1 : r);
}

// Ghost state of a Dirichlet side (App. A.3): the mirror cell's primitives
// phi (with the exact path's arithmetic for p) reflected about the boundary
// face's primitives phi' as 2 phi' - phi, then back to conserved variables.
// st: the side's state array, m faces per primitive, s this face.
template <int ND>
__device__ __forceinline__ void dirichlet_ghost(double (&Uc)[ND + 2], const double *st, int64_t m,
                                                int64_t s, double gm1)
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
    const double rg = 2.0 * st[s] - rho;
    double ug[ND];
#pragma unroll
    for (int a = 0; a < ND; a++) ug[a] = 2.0 * st[(1 + a) * m + s] - u[a];
    const double pg = 2.0 * st[(nc - 1) * m + s] - p;
    Uc[0] = rg;
#pragma unroll
    for (int a = 0; a < ND; a++) Uc[1 + a] = rg * ug[a];
    double k2 = Uc[1] * ug[0];
#pragma unroll
    for (int a = 1; a < ND; a++) k2 = fma(Uc[1 + a], ug[a], k2);
    Uc[nc - 1] = pg / gm1 + 0.5 * k2;
}

// Applies a ghost rule of map_index to the loaded state of the mirror cell.
template <int ND, int D>
__device__ __forceinline__ void apply_ghost_rule(double (&Uc)[ND + 2], int rule, const double *st_lo,
                                                 const double *st_hi, int64_t m, int64_t s,
                                                 double gm1)
{
    if (rule == 1) {
        Uc[1 + D] = -Uc[1 + D];
    } else if (rule == 2) {
#pragma unroll
        for (int a = 0; a < ND; a++) Uc[1 + a] = -Uc[1 + a];
    } else if (rule >= 3) {
        dirichlet_ghost<ND>(Uc, rule == 3 ? st_lo : st_hi, m, s, gm1);
    }
}

template <int ND>
struct SmemLayout {
    static constexpr int nc = ND + 2;
    static constexpr int QU = 0, QF = nc, QV = 2 * nc;           // U, F, velocity
    static constexpr int QH = QV + ND, QSR = QH + 1, QC = QH + 2;  // enthalpy, sqrt(rho), c
    static constexpr int QLM = QH + 3, QL0 = QLM + 1, QLP = QLM + 2, QLR = QLM + 3;
    static constexpr int NQ = QLR + 1;
};

// Tile of the sweeps: TP pencils x TF faces along the sweep, the exact-path
// queue's capacity in reconstructions per thread (QCAP) and the blocks per SM
// the register allocation is bounded for (MINB).  A single line (1D) uses
// 1 x 128.  Measured on GB300 with 128-thread blocks:
//   3D 256^3: TENO10 at three blocks per SM (164 registers, about 60 KB of
//   shared memory each) beats two by 8-9 % and four by 6 %; TENO8 at four
//   (128 registers) beats three by 2 %; with face n of periodic
//   lines left out (256 faces per line), 4 x 32 beats 8 x 16 and 16 x 8 by
//   0.5 % and 3 % (TENO10) and stages fewer halo cells per face;
//   2D 512^2 TENO8: 4 x 32 ahead of 8 x 16 by 4 %, a register bound (three
//   or four blocks per SM) ahead of an unbounded allocation by 3 %.
// TENO_FACE_TP/TF/QCAP/MINB, when defined, override every case (tuning).
template <int ND, int H>
struct FaceTile {
#ifdef TENO_FACE_TP
    static constexpr int TP = ND == 1 ? 1 : TENO_FACE_TP;
    static constexpr int TF = ND == 1 ? 128 : TENO_FACE_TF;
    static constexpr int QCAP = TENO_FACE_QCAP;
    static constexpr int MINB = TENO_FACE_MINB;
#else
    static constexpr int TP = ND == 1 ? 1 : 4;
    static constexpr int TF = ND == 1 ? 128 : 32;
    // 2D ten-point: four queue entries per thread still fit three blocks per
    // SM (73 KB each); noise plateaus hold about eight decided, non-S_p
    // reconstructions per thread, which otherwise diverge when done in place
    static constexpr int QCAP = (ND == 2 && H == 5) ? 4 : 2;
    static constexpr int MINB = ND >= 2 ? (H == 4 ? 4 : 3) : 1;
#endif
};

template <int ND, int H, int TP, int TF>
constexpr size_t face_smem_bytes()
{
    // staged cells + exact-path queue (values, owners) + per-thread results
    return sizeof(double) * (size_t)SmemLayout<ND>::NQ * (TF + 2 * H - 1) * TP +
           sizeof(double) * (size_t)(FaceTile<ND, H>::QCAP * TP * TF) * (2 * H) +
           sizeof(double) * (size_t)(TP * TF) * 2 * (ND + 2) +
           sizeof(int) * (size_t)(FaceTile<ND, H>::QCAP * TP * TF) +
           (size_t)(TP * TF) * 2 * (ND + 2);
}

// Sweep modes, a compile-time choice so that each kernel holds only its own
// code: a plain sweep, one that writes the decision record (flags, argmax,
// limrec), and one that applies recorded decisions (frozen, frozen_argmax).
enum { kSweepPlain = 0, kSweepRecord = 1, kSweepFrozen = 2 };

// One tile: faces f0 .. f0+TF-1 along D of the TP pencils starting at x0
// (at y, z for the axes not swept); for D = 0 the pencils run along y instead,
// starting at y (x0 unused).  Every thread of the block calls it; it
// synchronises once after staging and returns with no barrier pending, so a
// persistent caller must synchronise before reusing the shared tile.
template <int ND, int H, int D, int TP, int TF, int MODE>
__device__ __forceinline__ void face_block(const FaceArgs &a, int64_t f0, int64_t x0, int64_t y,
                                           int64_t z, double *sm)
{
    using SL = SmemLayout<ND>;
    constexpr int nc = ND + 2, last = nc - 1, W = 2 * H;
    constexpr int NS = TF + 2 * H - 1;
#define SQ(q, j, p) sm[((q) * NS + (j)) * TP + (p)]

    const int64_t n0 = a.n[0], n1 = a.n[1], nD = a.n[D];
    const int64_t pstart = (D == 0) ? y : x0;             // first pencil
    const int64_t npen = (D == 0) ? n1 : n0;              // pencils along that axis
    __shared__ int qcount[2];                  // queue lengths: exact path, decided
    if (threadIdx.x < 2) qcount[threadIdx.x] = 0;

    // Stage cells f0-H .. f0+TF+H-2 along D.
    for (int idx = threadIdx.x; idx < NS * TP; idx += TP * TF) {
        const int j = idx / TP, p = idx % TP;
        const int64_t pg = pstart + p;
        if (pg >= npen) continue;
        int rule;
        const int64_t gi = map_index(f0 - H + j, nD, H, a.bc_lo, a.bc_hi, rule);
        double Uc[nc];
        CellQ<ND> q;
        if (rule >= 5) {
            // a neighbouring sub-domain's cell from the side's halo array,
            // [nc][H planes][cells of a plane, the other axes x fastest]
            const int64_t m = a.ncell / nD;
            const int64_t sf = (D == 0) ? pg + n1 * z : (D == 1 ? pg + n0 * z : pg + n0 * y);
            const double *hb = rule == 5 ? a.bcs_lo : a.bcs_hi;
            const int64_t ih = gi * m + sf;
            const bool ok = TENO_IN(a.st, ih, H * m);
#pragma unroll
            for (int c = 0; c < nc; c++) Uc[c] = ok ? hb[(int64_t)c * H * m + ih] : 0.0;
            cell_quantities<ND, D>(Uc, a.K, q);
        } else {
            int64_t id;
            if (D == 0) id = gi + n0 * (pg + n1 * z);
            else if (D == 1) id = pg + n0 * (gi + n1 * z);
            else id = pg + n0 * (y + n1 * gi);
            const bool ok = TENO_IN(a.st, id, a.ncell);
#pragma unroll
            for (int c = 0; c < nc; c++) Uc[c] = ok ? a.U[c * a.ncell + id] : 0.0;
            if (!rule && a.P && ok) {
                cell_from_prims<ND, D>(Uc, a.P, a.ncell, id, q);      // stored for this input
            } else {
                if (rule) {
                    // boundary-face index among the faces of this side (other axes, x fastest)
                    const int64_t m = a.ncell / nD;
                    const int64_t sf = (D == 0) ? pg + n1 * z : (D == 1 ? pg + n0 * z : pg + n0 * y);
                    if (rule < 3 || TENO_IN(a.st, sf, m))
                        apply_ghost_rule<ND, D>(Uc, rule, a.bcs_lo, a.bcs_hi, m, sf, a.K.gm1);
                }
                cell_quantities<ND, D>(Uc, a.K, q);
            }
        }
        if (a.count_cells) {
            // interior cells of this tile's own face range: each cell once
            const int64_t ci = f0 - H + j;
            if (ci >= f0 && ci < f0 + TF && ci < nD && nonphysical_cell<ND>(Uc[0], q))
                atomicAdd(&a.st->nonphys, 1ull);
        }
#pragma unroll
        for (int c = 0; c < nc; c++) {
            SQ(SL::QU + c, j, p) = 0.5 * q.U[c];
            SQ(SL::QF + c, j, p) = 0.5 * q.F[c];
        }
#pragma unroll
        for (int k = 0; k < ND; k++) SQ(SL::QV + k, j, p) = q.u[k];
        SQ(SL::QH, j, p) = q.H;
        SQ(SL::QSR, j, p) = q.sr;
        SQ(SL::QC, j, p) = q.c;
        const double vd = q.u[D], cj = q.c;
        SQ(SL::QLM, j, p) = fabs(vd - cj);
        SQ(SL::QL0, j, p) = fabs(vd);
        SQ(SL::QLP, j, p) = fabs(vd + cj);
        SQ(SL::QLR, j, p) = fabs(vd) + cj;
    }
    __syncthreads();

    const int p = threadIdx.x % TP, fo = threadIdx.x / TP;
    const int64_t f = f0 + fo;
    const bool active = !(f > nD - a.skip_last || pstart + p >= npen);
    const int jl = fo + H - 1, jr = fo + H;           // cells i and i+1

    // Queue of reconstructions whose value is not computed in line (values,
    // owner), and per-thread result slots; after the staged cells.
    // Entries [0, QE) hold reconstructions for the exact path, [QE, CAP)
    // decided ones whose value is not the largest stencil's scheme (its
    // decision byte already in the owner's Qfl slot).
    constexpr int CAP = FaceTile<ND, H>::QCAP * TP * TF, QE = CAP / 4;
    double *Qv = sm + (size_t)SL::NQ * NS * TP;       // [CAP][W]
    double *Qres = Qv + (size_t)CAP * W;              // [threads][2 nc]: every value of the face
    int *Qmeta = (int *)(Qres + (size_t)TP * TF * 2 * nc);   // [CAP]
    uint8_t *Qfl = (uint8_t *)(Qmeta + CAP);          // [threads][2 nc]

    RoeScalars<ND> rs;                 // eigenvector rows / columns are built from these
    double am = 0.0, a0 = 0.0, ap = 0.0, ar = 0.0;
    int64_t flin = 0;
    if (active) {
        // Roe average and eigenvectors (Sec. 5).
        double ul[ND], ur[ND];
#pragma unroll
        for (int k = 0; k < ND; k++) { ul[k] = SQ(SL::QV + k, jl, p); ur[k] = SQ(SL::QV + k, jr, p); }
        const double c2 = roe_state<ND, D>(ul, SQ(SL::QH, jl, p), SQ(SL::QSR, jl, p), ur,
                                           SQ(SL::QH, jr, p), SQ(SL::QSR, jr, p), a.K.gm1, rs);
        if (!(c2 > 0.0)) atomicAdd(&a.st->nonphys, 1ull);
        if (D == 0) flin = f + (n0 + 1) * (pstart + p + n1 * z);
        else if (D == 1) flin = pstart + p + n0 * (f + (n1 + 1) * z);
        else flin = pstart + p + n0 * (y + n1 * f);
        if (!TENO_IN(a.st, flin, a.nfaces)) flin = 0;        // debug build: counted, redirected
        // Splitting speeds over the stencil (first maximum), or at recorded cells.
        if constexpr (MODE == kSweepFrozen) {
            unsigned w = a.frozen_argmax[flin];
            if (!TENO_IN(a.st, (int)(w & 15), W) || !TENO_IN(a.st, (int)((w >> 4) & 15), W) ||
                !TENO_IN(a.st, (int)((w >> 8) & 15), W) || !TENO_IN(a.st, (int)(w >> 12), W))
                w = 0;
            am = SQ(SL::QLM, fo + (int)(w & 15), p);
            a0 = SQ(SL::QL0, fo + (int)((w >> 4) & 15), p);
            ap = SQ(SL::QLP, fo + (int)((w >> 8) & 15), p);
            ar = SQ(SL::QLR, fo + (int)((w >> 12) & 15), p);
        } else {
            int jm = 0, j0 = 0, jp = 0, jr_ = 0;
#pragma unroll
            for (int j = 0; j < W; j++) {
                const double em = SQ(SL::QLM, fo + j, p), e0 = SQ(SL::QL0, fo + j, p);
                const double ep = SQ(SL::QLP, fo + j, p), er = SQ(SL::QLR, fo + j, p);
                if (j == 0 || speed_gt(em, am)) { am = em; jm = j; }
                if (j == 0 || speed_gt(e0, a0)) { a0 = e0; j0 = j; }
                if (j == 0 || speed_gt(ep, ap)) { ap = ep; jp = j; }
                if (j == 0 || speed_gt(er, ar)) { ar = er; jr_ = j; }
            }
            if constexpr (MODE == kSweepRecord)
                a.argmax[flin] = (uint16_t)(jm | (j0 << 4) | (jp << 8) | (jr_ << 12));
        }
    }

    // Split-flux reconstructions of every field and sign: those the filter
    // decides for the largest stencil now, the rest queued (or, if the queue
    // is full, done in place) and drained once per tile by the whole block --
    // the undecided ones with the exact path, the decided ones (fallback or a
    // smaller stencil) with their value formula, so that neither diverges
    // inside a warp.  Each value lands in the owner's Qres slot (shared
    // memory, not registers: 2 nc values held there would stay live across
    // the whole field loop and push the kernel into spills).
    unsigned pending = 0;              // bit 2k+s: value comes from the queue
#pragma unroll 1
    for (int k = 0; k < nc; k++) {
        if (!active) break;
        const bool shear = (k >= 2 && k < last);
        const int tax = shear ? shear_axis<ND, D>(k) : 0;
        double lrow[nc];
        l_row<ND, D>(rs, k, lrow);
        const double alpha = a.K.split ? ar : (k == 0 ? am : (k == last ? ap : a0));
        // hw = w/2 = l.(U/2), hg = g/2 = l.(F/2) from the halved staged values:
        // every product and sum is the unhalved one scaled by 1/2, exactly
        double hw[W], hg[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
            double wv, gv;
            if (shear) {
                wv = SQ(SL::QU + 1 + tax, fo + j, p) + lrow[0] * SQ(SL::QU, fo + j, p);
                gv = SQ(SL::QF + 1 + tax, fo + j, p) + lrow[0] * SQ(SL::QF, fo + j, p);
            } else {
                wv = lrow[0] * SQ(SL::QU, fo + j, p);
                gv = lrow[0] * SQ(SL::QF, fo + j, p);
#pragma unroll
                for (int c = 1; c < nc; c++) {
                    wv = fma(lrow[c], SQ(SL::QU + c, fo + j, p), wv);
                    gv = fma(lrow[c], SQ(SL::QF + c, fo + j, p), gv);
                }
            }
            hw[j] = wv;
            hg[j] = gv;
        }
#pragma unroll 1
        for (int s = 0; s < 2; s++) {
            // f+ on offsets m -> cell i+m; f- mirrored: offset m -> cell i+1-m.
            // v = (g +- alpha w)/2 = fma(+-alpha, w/2, g/2), rounded once.
            const double sa = s ? -alpha : alpha;
            double v[W];
#pragma unroll
            for (int kk = 0; kk < W; kk++) {
                const double wk = s ? hw[W - 1 - kk] : hw[kk];
                const double gk = s ? hg[W - 1 - kk] : hg[kk];
                v[kk] = fma(sa, wk, gk);
            }
            double val = 0.0;
            uint8_t fl = 0;
            bool done = true;
            if constexpr (MODE == kSweepFrozen) {
                fl = a.frozen[(flin * nc + k) * 2 + s];
                val = frozen_recon<H>(v, fl);
            } else {
                double sh[W];
#pragma unroll
                for (int kk = 0; kk < W; kk++) sh[kk] = v[kk] - v[H - 1];
                const bool dec = a.fast && fast_decide<H>(v, sh, a.FK, fl,
                                                          MODE == kSweepRecord && a.need_ct != 0);
                // the largest stencil accepted (S6 as bits 0-4 zero).  Kept
                // inline: the same test through a helper function made the 8-
                // and 10-point sweeps 4-14 % slower (same registers, other code).
                if (dec && (H == 6 ? (fl & 31) == 0 : (fl & 3) == H - 2)) {
                    val = flux_large<H, H>(v);
                } else {
                    int q = atomicAdd(&qcount[dec ? 1 : 0], 1);
                    const bool room = (dec ? (q < CAP - QE) : (q < QE)) &&
                                      TENO_IN(a.st, q + (dec ? QE : 0), CAP);
                    if (room) {
                        if (dec) {
                            q += QE;
                            Qfl[threadIdx.x * (2 * nc) + 2 * k + s] = fl;
                        }
#pragma unroll
                        for (int kk = 0; kk < W; kk++) Qv[(size_t)q * W + kk] = v[kk];
                        Qmeta[q] = (threadIdx.x << 4) | (2 * k + s);
                        pending |= 1u << (2 * k + s);
                        done = false;
                    } else {                                   // queue full: in place
                        val = dec ? decided_value<H>(v, fl) : teno_recon<H>(v, a.K, fl);
                    }
                }
            }
            if (done) {
                Qres[threadIdx.x * (2 * nc) + 2 * k + s] = val;
                if constexpr (MODE == kSweepRecord) a.flags[(flin * nc + k) * 2 + s] = fl;
            }
        }
    }
    if constexpr (MODE != kSweepFrozen) {
        __syncthreads();
        const int ne = min(qcount[0], QE), nd = min(qcount[1], CAP - QE);
        if (a.exact_count && threadIdx.x == 0 && qcount[0] > 0)
            atomicAdd(a.exact_count, (unsigned long long)qcount[0]);
        for (int q = threadIdx.x; q < ne; q += TP * TF) {
            double v[W];
#pragma unroll
            for (int kk = 0; kk < W; kk++) v[kk] = Qv[(size_t)q * W + kk];
            uint8_t fl;
            const double r = teno_recon<H>(v, a.K, fl);
            const int meta = Qmeta[q];
            const int slot = (meta >> 4) * (2 * nc) + (meta & 15);
            if (TENO_IN(a.st, slot, TP * TF * 2 * nc)) {
                Qres[slot] = r;
                Qfl[slot] = fl;
            }
        }
        for (int q = QE + threadIdx.x; q < QE + nd; q += TP * TF) {
            double v[W];
#pragma unroll
            for (int kk = 0; kk < W; kk++) v[kk] = Qv[(size_t)q * W + kk];
            const int meta = Qmeta[q];
            const int slot = (meta >> 4) * (2 * nc) + (meta & 15);
            if (TENO_IN(a.st, slot, TP * TF * 2 * nc)) Qres[slot] = decided_value<H>(v, Qfl[slot]);
        }
        __syncthreads();
        if constexpr (MODE == kSweepRecord) {
            if (active && pending) {
#pragma unroll
                for (int q = 0; q < 2 * nc; q++) {
                    if (pending & (1u << q))
                        a.flags[(flin * nc + (q >> 1)) * 2 + (q & 1)] = Qfl[threadIdx.x * (2 * nc) + q];
                }
            }
        }
    }

    // Back-projection F = sum_k r_k (f+_k + f-_k), fields ascending; the zero
    // and unit entries of the shear columns are skipped.
    double Fo[nc];
    if (active) {
#pragma unroll
        for (int k = 0; k < nc; k++) {
            const double hsum = Qres[threadIdx.x * (2 * nc) + 2 * k] + Qres[threadIdx.x * (2 * nc) + 2 * k + 1];
            if (k == 0) {
#pragma unroll
                for (int c = 0; c < nc; c++) Fo[c] = r_entry<ND, D>(rs, c, 0) * hsum;
            } else if (k >= 2 && k < last) {
                int tax = 0, kk = 2;
#pragma unroll
                for (int aa = 0; aa < ND; aa++) {
                    if (aa == D) continue;
                    if (kk == k) tax = aa;
                    kk++;
                }
                Fo[1 + tax] = Fo[1 + tax] + hsum;
                Fo[last] = fma(r_entry<ND, D>(rs, last, k), hsum, Fo[last]);
            } else {
#pragma unroll
                for (int c = 0; c < nc; c++) Fo[c] = fma(r_entry<ND, D>(rs, c, k), hsum, Fo[c]);
            }
        }
    }
    if (!active) return;

    if (a.K.limiter) {
        // Positivity-preserving flux limiter (cited in Sec. 5.3): blend toward
        // the Lax-Friedrichs flux so that the one-sided half updates of cells i
        // and i+1 keep rho >= eps and p >= eps.
        const double eps = a.K.lim_eps, lam2 = 2.0 * (*a.lam);
        const double al = SQ(SL::QLR, jl, p), arr = SQ(SL::QLR, jr, p);
        const double af = arr > al ? arr : al;
        double FL[nc], dF[nc], UL[nc], UR[nc], dUL[nc], dUR[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) {
            // staged halves: FL = (F_l + F_r)/2 - af (U_r - U_l)/2 exactly as
            // ((F_l + F_r) - af (U_r - U_l)) / 2
            const double hUl = SQ(SL::QU + c, jl, p), hUr = SQ(SL::QU + c, jr, p);
            const double hFl = SQ(SL::QF + c, jl, p), hFr = SQ(SL::QF + c, jr, p);
            const double Ul = 2.0 * hUl, Ur = 2.0 * hUr, Fl = 2.0 * hFl, Fr = 2.0 * hFr;
            FL[c] = (hFl + hFr) - af * (hUr - hUl);
            dF[c] = Fo[c] - FL[c];
            UL[c] = Ul - lam2 * (FL[c] - Fl);
            UR[c] = Ur + lam2 * (FL[c] - Fr);
            dUL[c] = -(lam2 * dF[c]);
            dUR[c] = lam2 * dF[c];
        }
        double th = 1.0;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const double r0 = side ? UR[0] : UL[0];
            const double r1 = r0 + (side ? dUR[0] : dUL[0]);
            if (r1 < eps) {
                double t = (r0 - eps) / (r0 - r1);
                if (!(t > 0.0)) t = 0.0;
                if (t < th) th = t;
            }
        }
        double thp = th;
#pragma unroll
        for (int side = 0; side < 2; side++) {
            double Us[nc], Ut[nc];
#pragma unroll
            for (int c = 0; c < nc; c++) {
                Us[c] = side ? UR[c] : UL[c];
                Ut[c] = Us[c] + th * (side ? dUR[c] : dUL[c]);
            }
            const double pt = pressure_of<ND>(Ut, a.K.gm1);
            if (pt < eps) {
                const double p0 = pressure_of<ND>(Us, a.K.gm1);
                double t = th * ((p0 - eps) / (p0 - pt));
                if (!(t > 0.0)) t = 0.0;
                if (t < thp) thp = t;
            }
        }
        if (thp < 1.0) {
#pragma unroll
            for (int c = 0; c < nc; c++) Fo[c] = FL[c] + thp * dF[c];
        }
        if constexpr (MODE == kSweepRecord) a.limrec[flin] = thp < 1.0 ? 1 : 0;
    } else if constexpr (MODE == kSweepRecord) {
        a.limrec[flin] = 0;
    }

#pragma unroll
    for (int c = 0; c < nc; c++) a.F[c * a.nfaces + flin] = Fo[c];
#undef SQ
}

template <int ND, int H, int D, int TP, int TF, int MODE>
__global__ void __launch_bounds__(TP * TF, FaceTile<ND, H>::MINB) face_kernel(FaceArgs a)
{
    extern __shared__ double sm[];
    int64_t x0 = 0, y = 0, z = 0, f0;
    if (D == 0) { f0 = (int64_t)blockIdx.x * TF; y = (int64_t)blockIdx.y * TP; z = blockIdx.z; }
    else if (D == 1) { x0 = (int64_t)blockIdx.x * TP; f0 = (int64_t)blockIdx.y * TF; z = blockIdx.z; }
    else { f0 = (int64_t)blockIdx.x * TF; x0 = (int64_t)blockIdx.y * TP; y = blockIdx.z; }
    face_block<ND, H, D, TP, TF, MODE>(a, f0, x0, y, z, sm);
}

template <int ND, int H, int D, int MODE>
cudaError_t launch_face_mode(const FaceArgs &a, dim3 grid, cudaStream_t s)
{
    constexpr int TP = FaceTile<ND, H>::TP;
    constexpr int TF = FaceTile<ND, H>::TF;
    constexpr size_t smem = face_smem_bytes<ND, H, TP, TF>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(face_kernel<ND, H, D, TP, TF, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    face_kernel<ND, H, D, TP, TF, MODE><<<grid, TP * TF, smem, s>>>(a);
    return cudaGetLastError();
}

// Host-side launch of one direction's sweep, in the mode its arguments ask
// for (a decision record to write, recorded decisions to apply, or neither).
template <int ND, int H, int D>
cudaError_t launch_face(const FaceArgs &a, cudaStream_t s)
{
    constexpr int TP = FaceTile<ND, H>::TP;
    constexpr int TF = FaceTile<ND, H>::TF;
    if ((a.flags && a.frozen) || (a.flags && (!a.argmax || !a.limrec)) ||
        (a.frozen && !a.frozen_argmax))
        return cudaErrorInvalidValue;
    dim3 grid;
    const int64_t nf = a.n[D] + 1 - a.skip_last;    // faces computed along D
    if (D == 0) grid = dim3((unsigned)((nf + TF - 1) / TF), (unsigned)((a.n[1] + TP - 1) / TP), (unsigned)a.n[2]);
    else if (D == 1) grid = dim3((unsigned)((a.n[0] + TP - 1) / TP), (unsigned)((nf + TF - 1) / TF), (unsigned)a.n[2]);
    else   // z tiles fastest: consecutive blocks share their halo planes through L2
        grid = dim3((unsigned)((nf + TF - 1) / TF), (unsigned)((a.n[0] + TP - 1) / TP), (unsigned)a.n[1]);
    if (a.flags) return launch_face_mode<ND, H, D, kSweepRecord>(a, grid, s);
    if (a.frozen) return launch_face_mode<ND, H, D, kSweepFrozen>(a, grid, s);
    return launch_face_mode<ND, H, D, kSweepPlain>(a, grid, s);
}

}  // namespace teno
