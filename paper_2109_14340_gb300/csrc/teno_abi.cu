// C ABI of the TENO-AA library (declared in include/teno.h): parameter
// validation, workspace layout, and the per-stage launch sequence
//   [wave maxima] -> prepare -> face sweep x [-> y [-> z]] -> combine.
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <mutex>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "teno.h"
#include "teno_face.cuh"

namespace teno {

// NVTX range around the enqueueing of one phase (visible to Nsight tools;
// a no-op when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Explicit instantiations live in teno_face8.cu / teno_face10.cu.
cudaError_t launch_face8(int nd, int d, const FaceArgs &a, cudaStream_t s);
cudaError_t launch_face10(int nd, int d, const FaceArgs &a, cudaStream_t s);
cudaError_t launch_face12(int nd, int d, const FaceArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------

struct CombineArgs {
    const double *F[3];      // face fluxes per direction, [nc][nfaces_d]
    int64_t nfaces[3];
    int64_t fstride[3];      // face-grid stride of the sweep axis in grid d
    int wrap[3];             // periodic axis: the last cell's right face is face 0
                             // (the same flux as face n, which may be left out)
    double inv_dx[3];
    const double *Uk;        // stage input (whose RHS the fluxes are)
    const double *Un;        // state at t^n (RK modes)
    double *out;             // rhs (mode 0) or next stage state
    double *P;               // RK modes: primitives of the next stage state (the
                             // next evaluation's input, with its non-physical
                             // cells counted here), or nullptr
    Status *st;
    int64_t n[3];
    int64_t ncell;
    int mode;                // 0: rhs, 1..3: RK stage 0..2
    Consts K;
};

// L(U)_i = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d (Eq. approximateEq), then the
// SSP-RK3 stage combination (Eq. Runge-kutta).  With a.P the new stage
// state's primitives are stored for the next evaluation's sweeps and its
// non-physical cells counted (each cell once, as that evaluation's input).
template <int ND>
__global__ void __launch_bounds__(256) combine_kernel(CombineArgs a)
{
    constexpr int nc = ND + 2;
    // one thread per cell; x from the block's row, y and z from the grid
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t y = blockIdx.y, z = blockIdx.z;
    bool bad = false;
    if (x < a.n[0] && TENO_IN(a.st, x + a.n[0] * (y + a.n[1] * z), a.ncell)) {
        const int64_t id = x + a.n[0] * (y + a.n[1] * z);
        int64_t flo[3];
#pragma unroll
        for (int d = 0; d < ND; d++) {
            const int64_t fn0 = a.n[0] + (d == 0), fn1 = a.n[1] + (d == 1);
            flo[d] = x + fn0 * (y + fn1 * z);
        }
        double Uc[nc], Uo[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Uc[c] = a.Uk[c * a.ncell + id];
        const double dt = a.st->dt;
#pragma unroll
        for (int c = 0; c < nc; c++) {
            double acc = 0.0;
#pragma unroll
            for (int d = 0; d < ND; d++) {
                const double *Fd = a.F[d] + c * a.nfaces[d];
                const int64_t xd = (d == 0) ? x : (d == 1 ? y : z);
                const int64_t fr = (a.wrap[d] && xd == a.n[d] - 1) ? flo[d] - xd * a.fstride[d]
                                                                    : flo[d] + a.fstride[d];
                const double t = (TENO_LOAD(a.st, Fd, fr, a.nfaces[d]) -
                                  TENO_LOAD(a.st, Fd, flo[d], a.nfaces[d])) * a.inv_dx[d];
                acc = acc - t;
            }
            double o;
            if (a.mode == 0) {
                o = acc;
            } else {
                const double t = Uc[c] + dt * acc;
                if (a.mode == 1) o = t;
                else if (a.mode == 2) o = 0.75 * a.Un[c * a.ncell + id] + 0.25 * t;
                else o = (1.0 / 3.0) * a.Un[c * a.ncell + id] + (2.0 / 3.0) * t;
            }
            a.out[c * a.ncell + id] = o;
            Uo[c] = o;
        }
        if (a.P) {
            CellQ<ND> q;
            cell_quantities<ND, 0>(Uo, a.K, q);
            store_prims<ND>(q, a.P, a.ncell, id);
            bad = nonphysical_cell<ND>(Uo[0], q);
        }
    }
    if (a.P) {            // every lane of the warp is here (no early return)
        const unsigned nb = __popc(__ballot_sync(0xffffffffu, bad));
        if ((threadIdx.x & 31) == 0 && nb) atomicAdd(&a.st->nonphys, (unsigned long long)nb);
    }
}

// Primitives of a right-hand-side input (store_prims), read by every sweep of
// the evaluation instead of recomputing them per staged cell; counts the
// input's non-physical cells (each cell once).
template <int ND>
__global__ void __launch_bounds__(256) prims_kernel(const double *U, int64_t ncell, Consts K,
                                                    double *P, Status *st)
{
    constexpr int nc = ND + 2;
    unsigned long long bad = 0;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < ncell;
         id += (int64_t)gridDim.x * blockDim.x) {
        double Uc[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Uc[c] = U[c * ncell + id];
        CellQ<ND> q;
        cell_quantities<ND, 0>(Uc, K, q);
        store_prims<ND>(q, P, ncell, id);
        if (nonphysical_cell<ND>(Uc[0], q)) bad++;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&st->nonphys, bad);
}

// A_d = max over cells of |u_d| + c, accumulated as bit patterns (the
// ordering of non-negative doubles); NaN never enters.  Optionally counts
// non-physical cells.
template <int ND>
__global__ void wave_max_kernel(const double *U, int64_t ncell, Consts K, Status *st, int count)
{
    constexpr int nc = ND + 2;
    double m[ND];
#pragma unroll
    for (int d = 0; d < ND; d++) m[d] = 0.0;
    unsigned long long bad = 0;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < ncell;
         id += (int64_t)gridDim.x * blockDim.x) {
        double Uc[nc];
#pragma unroll
        for (int c = 0; c < nc; c++) Uc[c] = U[c * ncell + id];
        CellQ<ND> q;
        cell_quantities<ND, 0>(Uc, K, q);
        if (!(Uc[0] > 0.0) || !(q.p > 0.0) || !isfinite(q.c) || !isfinite(q.H)) bad++;
#pragma unroll
        for (int d = 0; d < ND; d++) {
            const double e = fabs(q.u[d]) + q.c;
            if (e > m[d]) m[d] = e;
        }
    }
#pragma unroll
    for (int d = 0; d < ND; d++) {
        double v = m[d];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            if (w > v) v = w;
        }
        if ((threadIdx.x & 31) == 0 && v > 0.0)
            atomicMax(&st->amax[d], (unsigned long long)__double_as_longlong(v));
    }
    if (count) {
        for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
        if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&st->nonphys, bad);
    }
}

// dt = cfl / sum_d A_d / dx_d (written to *dt_out and the status block).
__global__ void cfl_finalize_kernel(Status *st, int nd, double cfl, double3 inv_dx, double *dt_out,
                                    int accumulate)
{
    const double idx[3] = {inv_dx.x, inv_dx.y, inv_dx.z};
    double S = __longlong_as_double((long long)st->amax[0]) * idx[0];
    for (int d = 1; d < nd; d++) S = S + __longlong_as_double((long long)st->amax[d]) * idx[d];
    const double dt = cfl / S;
    st->dt = dt;
    if (dt_out) *dt_out = dt;
    if (accumulate) st->t_accum = st->t_accum + dt;
}

// dt = cfl / sum_d A_d / dx_d with A_d the largest of ncopies rows of maxima
// (sub-domains): the arithmetic of cfl_finalize_kernel on the combined maxima.
__global__ void dt_from_speeds_kernel(const double *amax, int ncopies, int nd, double cfl,
                                      double3 inv_dx, double *dt_out)
{
    const double idx[3] = {inv_dx.x, inv_dx.y, inv_dx.z};
    double A[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < ncopies; k++)
        for (int d = 0; d < nd; d++) {
            const double v = amax[k * 3 + d];
            if (v > A[d]) A[d] = v;
        }
    double S = A[0] * idx[0];
    for (int d = 1; d < nd; d++) S = S + A[d] * idx[d];
    *dt_out = cfl / S;
}

// Stage preparation: dt from the host value or a device scalar, and the
// limiter's effective dt/dx per direction: dt/dx in 1D; (dt S) / A_d with
// S = sum_d A_d/dx_d in several dimensions (each direction's one-sided
// updates get the share A_d/dx_d / S of the update).
__global__ void prepare_kernel(Status *st, int nd, double dt_host, const double *dt_dev,
                               double3 inv_dx, int limiter)
{
    const double dt = dt_dev ? *dt_dev : dt_host;
    st->dt = dt;
    if (!limiter) return;
    const double idx[3] = {inv_dx.x, inv_dx.y, inv_dx.z};
    if (nd == 1) {
        st->lam[0] = dt * idx[0];
        return;
    }
    double A[3];
    for (int d = 0; d < nd; d++) A[d] = __longlong_as_double((long long)st->amax[d]);
    double S = A[0] * idx[0];
    for (int d = 1; d < nd; d++) S = S + A[d] * idx[d];
    for (int d = 0; d < nd; d++) st->lam[d] = (dt * S) / A[d];
}

// Scalar reconstruction of caller-provided stencils (teno_reconstruct): the
// certified filter first when enabled, else / then the exact path.
template <int H>
__global__ void recon_kernel(const double *v, int64_t count, double *out, uint8_t *flags, Consts K,
                             FastK FK, int fast)
{
    constexpr int W = 2 * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double vv[W], sh[W];
#pragma unroll
        for (int m = 0; m < W; m++) vv[m] = v[i * W + m];
#pragma unroll
        for (int m = 0; m < W; m++) sh[m] = vv[m] - vv[H - 1];
        uint8_t fl = 0;
        double r;
        if (fast && fast_decide<H>(vv, sh, FK, fl, flags != nullptr)) r = decided_value<H>(vv, fl);
        else r = teno_recon<H>(vv, K, fl);
        out[i] = r;
        if (flags) flags[i] = fl;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static int ncons(const teno_params *p) { return p->ndim + 2; }

static int64_t ncells(const teno_params *p) { return p->n[0] * p->n[1] * p->n[2]; }

static int64_t face_grid(const teno_params *p, int d)
{
    int64_t s = 1;
    for (int a = 0; a < 3; a++) s *= (a == d) ? p->n[a] + 1 : p->n[a];
    return s;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t status, flux[3], stage, prims, total;
};

static Layout layout(const teno_params *p)
{
    Layout L;
    const int nc = ncons(p);
    size_t off = 0;
    L.status = off;
    off += align256(sizeof(Status));
    for (int d = 0; d < 3; d++) {
        L.flux[d] = off;
        if (d < p->ndim) off += align256(sizeof(double) * (size_t)nc * face_grid(p, d));
    }
    L.stage = off;
    off += align256(sizeof(double) * (size_t)nc * ncells(p));
    L.prims = off;
    off += align256(sizeof(double) * (size_t)(p->ndim + 4) * ncells(p));
    L.total = off;
    return L;
}

static int validate(const teno_params *p)
{
    if (!p) return TENO_EINVAL;
    if (p->ndim < 1 || p->ndim > 3) return TENO_EINVAL;
    if (p->scheme != 8 && p->scheme != 10 && p->scheme != 12) return TENO_EINVAL;
    if (p->flux_split != TENO_SPLIT_LLF && p->flux_split != TENO_SPLIT_RUSANOV) return TENO_EINVAL;
    if (p->limiter != 0 && p->limiter != 1) return TENO_EINVAL;
    if (p->q != 7 || p->reserved != 0) return TENO_EINVAL;
    if (!(p->gamma > 1.0) || !(p->ct_cr > 0.0) || !(p->eps_beta >= 0.0) || !(p->eps_eta > 0.0))
        return TENO_EINVAL;
    if (!(p->ct_alpha1 >= 0.0) || !(p->ct_alpha2 >= 0.0) || !(p->limiter_eps >= 0.0))
        return TENO_EINVAL;
    const int H = p->scheme / 2;
    for (int a = 0; a < 3; a++) {
        if (a < p->ndim) {
            if (p->n[a] < H || p->n[a] > (int64_t)1 << 31) return TENO_EINVAL;
            if (!(p->dx[a] > 0.0)) return TENO_EINVAL;
            for (int side = 0; side < 2; side++) {
                const int b = side ? p->bc_hi[a] : p->bc_lo[a];
                const double *st = side ? p->bc_state_hi[a] : p->bc_state_lo[a];
                if (b < TENO_BC_PERIODIC || b > TENO_BC_HALO) return TENO_EINVAL;
                // a state array exactly on the Dirichlet and halo sides (16-byte aligned)
                if ((b == TENO_BC_DIRICHLET || b == TENO_BC_HALO) != (st != nullptr))
                    return TENO_EINVAL;
                if (st && ((uintptr_t)st & 15)) return TENO_EINVAL;
                // the limiter's direction weights need the whole domain's wave
                // speeds, which a sub-domain does not see
                if (b == TENO_BC_HALO && p->limiter && p->ndim > 1) return TENO_EINVAL;
            }
            if ((p->bc_lo[a] == TENO_BC_PERIODIC) != (p->bc_hi[a] == TENO_BC_PERIODIC))
                return TENO_EINVAL;
        } else if (p->n[a] != 1 || p->bc_state_lo[a] || p->bc_state_hi[a]) {
            return TENO_EINVAL;
        }
    }
    if (p->n[1] > 65535 || p->n[2] > 65535) return TENO_EINVAL;   // grid y / z limits
    return TENO_OK;
}

static int check_ptr(const void *ptr, bool nullable = false)
{
    if (!ptr) return nullable ? TENO_OK : TENO_EINVAL;
    return ((uintptr_t)ptr & 15) ? TENO_EINVAL : TENO_OK;
}

static Consts consts_of(const teno_params *p)
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
    K.limiter = p->limiter;
    return K;
}

int g_fast_filter = 1;

static FastK fastk_of(const teno_params *p)
{
    return fastk_make(p->ct_cr, p->ct_alpha1, p->ct_alpha2, p->eps_beta, p->eps_eta);
}

// The filter runs when it is switched on and its bounds hold for p's epsilons.
static int filter_on(const teno_params *p)
{
    return g_fast_filter && fast_filter_valid(p->eps_beta, p->eps_eta) ? 1 : 0;
}

static double3 inv_dx_of(const teno_params *p)
{
    return make_double3(1.0 / p->dx[0], 1.0 / p->dx[1], 1.0 / p->dx[2]);
}

static int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

#define CUDA_TRY(x)                                   \
    do {                                              \
        if ((x) != cudaSuccess) return TENO_ECUDA;    \
    } while (0)

static cudaError_t launch_wave_max(const teno_params *p, const double *U, Status *st,
                                   int count, cudaStream_t s)
{
    const Consts K = consts_of(p);
    const int64_t N = ncells(p);
    const int blk = 256, grd = grid_for(N, blk);
    cudaError_t e = cudaMemsetAsync(st->amax, 0, sizeof(st->amax), s);
    if (e != cudaSuccess) return e;
    if (p->ndim == 1) wave_max_kernel<1><<<grd, blk, 0, s>>>(U, N, K, st, count);
    else if (p->ndim == 2) wave_max_kernel<2><<<grd, blk, 0, s>>>(U, N, K, st, count);
    else wave_max_kernel<3><<<grd, blk, 0, s>>>(U, N, K, st, count);
    return cudaGetLastError();
}

// Primitives of U into the workspace's primitive rows (non-physical cells
// counted); returns their address.
static cudaError_t launch_prims(const teno_params *p, const double *U, char *ws, cudaStream_t s,
                                double **P_out)
{
    NvtxRange range("teno primitives");
    const Layout L = layout(p);
    Status *st = (Status *)(ws + L.status);
    double *P = (double *)(ws + L.prims);
    const Consts K = consts_of(p);
    const int64_t N = ncells(p);
    const int blk = 256, grd = grid_for(N, blk);
    if (p->ndim == 1) prims_kernel<1><<<grd, blk, 0, s>>>(U, N, K, P, st);
    else if (p->ndim == 2) prims_kernel<2><<<grd, blk, 0, s>>>(U, N, K, P, st);
    else prims_kernel<3><<<grd, blk, 0, s>>>(U, N, K, P, st);
    *P_out = P;
    return cudaGetLastError();
}

// Event record of the face-sweep launches (teno_profile_*).
struct ProfileRecord {
    bool on = false;
    int used = 0;
    int64_t faces = 0;
    static constexpr int kMax = 8192;
    cudaEvent_t ev[2 * kMax];
    int64_t nf[kMax];
    int created = 0;
    unsigned long long *exact = nullptr;   // device counter of exact-path reconstructions
};
static ProfileRecord g_prof;

static cudaError_t profile_mark(int which, int slot, cudaStream_t s)
{
    const int k = 2 * slot + which;
    while (g_prof.created <= k) {
        cudaError_t e = cudaEventCreate(&g_prof.ev[g_prof.created]);
        if (e != cudaSuccess) return e;
        g_prof.created++;
    }
    return cudaEventRecord(g_prof.ev[k], s);
}

// One right-hand-side evaluation of Uk into the face buffers, then combine.
// P_in: primitives of Uk (prims_kernel or the previous combine), read by the
// sweeps, or nullptr (the sweeps compute them and the x sweep counts the
// non-physical cells); P_out: where the combine stores the primitives of
// its output for the next stage, or nullptr.
// full_ct = false: a recorded decision byte carries its C_T exponent only
// where the exponent was needed to decide (the selection-only record).
static int stage(const teno_params *p, const double *Uk, const double *Un, double *out, int mode,
                 double dt_host, const double *dt_dev, uint8_t *flags, char *ws, cudaStream_t s,
                 const uint8_t *frozen, const double *P_in, double *P_out, bool full_ct = true)
{
    static const char *kStageName[4] = {"teno rhs", "teno rk3 stage 1", "teno rk3 stage 2",
                                        "teno rk3 stage 3"};
    static const char *kSweepName[3] = {"teno face sweep x", "teno face sweep y",
                                        "teno face sweep z"};
    NvtxRange range(kStageName[mode]);
    const Layout L = layout(p);
    Status *st = (Status *)(ws + L.status);
    const Consts K = consts_of(p);
    const double3 idx = inv_dx_of(p);
    const int nd = p->ndim, nc = ncons(p);
    if (p->limiter && nd > 1) CUDA_TRY(launch_wave_max(p, Uk, st, 0, s));
    prepare_kernel<<<1, 1, 0, s>>>(st, nd, dt_host, dt_dev, idx, p->limiter);
    CUDA_TRY(cudaGetLastError());
    uint8_t *fl = flags;
    const uint8_t *fz = frozen;
    // the decision record: all directions' decision bytes, then all
    // directions' maximising-cell words
    size_t dec_bytes = 0;
    for (int d = 0; d < nd; d++) dec_bytes += (size_t)face_grid(p, d) * nc * 2;
    size_t nfaces_all = 0;
    for (int d = 0; d < nd; d++) nfaces_all += (size_t)face_grid(p, d);
    uint16_t *am = flags ? (uint16_t *)(flags + dec_bytes) : nullptr;
    const uint16_t *fam = frozen ? (const uint16_t *)(frozen + dec_bytes) : nullptr;
    uint8_t *lr = flags ? flags + dec_bytes + 2 * nfaces_all : nullptr;   // limiter bytes
    for (int d = 0; d < nd; d++) {
        FaceArgs a;
        a.U = Uk;
        a.P = P_in;
        a.F = (double *)(ws + L.flux[d]);
        a.flags = fl;
        a.frozen = fz;
        a.argmax = am;
        a.frozen_argmax = fam;
        a.limrec = lr;
        a.st = st;
        for (int k = 0; k < 3; k++) a.n[k] = p->n[k];
        a.ncell = ncells(p);
        a.nfaces = face_grid(p, d);
        a.bc_lo = p->bc_lo[d];
        a.bc_hi = p->bc_hi[d];
        a.bcs_lo = p->bc_state_lo[d];
        a.bcs_hi = p->bc_state_hi[d];
        a.lam = &st->lam[d];
        a.fast = filter_on(p);
        a.need_ct = (fl && full_ct) ? 1 : 0;
        a.skip_last = (p->bc_lo[d] == TENO_BC_PERIODIC && !fl && !fz) ? 1 : 0;
        a.count_cells = (d == 0 && !P_in);        // the x sweep counts the stage input's cells
                                                  // unless its primitives were stored
        a.exact_count = g_prof.on ? g_prof.exact : nullptr;
        a.FK = fastk_of(p);
        a.K = K;
        const int slot = (g_prof.on && g_prof.used < ProfileRecord::kMax) ? g_prof.used++ : -1;
        if (slot >= 0) {
            g_prof.nf[slot] = a.nfaces - (a.skip_last ? a.ncell / p->n[d] : 0);   // faces computed
            CUDA_TRY(profile_mark(0, slot, s));
        }
        nvtxRangePushA(kSweepName[d]);
        cudaError_t e = (p->scheme == 8) ? launch_face8(nd, d, a, s)
                      : (p->scheme == 10 ? launch_face10(nd, d, a, s) : launch_face12(nd, d, a, s));
        nvtxRangePop();
        if (e != cudaSuccess) return TENO_ECUDA;
        if (slot >= 0) CUDA_TRY(profile_mark(1, slot, s));
        if (fl) fl += (size_t)face_grid(p, d) * nc * 2;
        if (fz) fz += (size_t)face_grid(p, d) * nc * 2;
        if (am) am += face_grid(p, d);
        if (fam) fam += face_grid(p, d);
        if (lr) lr += face_grid(p, d);
    }
    CombineArgs c;
    for (int d = 0; d < 3; d++) {
        c.F[d] = (const double *)(ws + L.flux[d]);
        c.nfaces[d] = d < nd ? face_grid(p, d) : 0;
        const int64_t fn0 = p->n[0] + (d == 0), fn1 = p->n[1] + (d == 1);
        c.fstride[d] = d == 0 ? 1 : (d == 1 ? fn0 : fn0 * fn1);
        c.wrap[d] = d < nd && p->bc_lo[d] == TENO_BC_PERIODIC;
    }
    c.inv_dx[0] = idx.x; c.inv_dx[1] = idx.y; c.inv_dx[2] = idx.z;
    c.Uk = Uk;
    c.Un = Un;
    c.out = out;
    c.P = P_out;
    c.st = st;
    for (int k = 0; k < 3; k++) c.n[k] = p->n[k];
    c.ncell = ncells(p);
    c.mode = mode;
    c.K = K;
    const int blk = 256;
    const dim3 grd((unsigned)((p->n[0] + blk - 1) / blk), (unsigned)p->n[1], (unsigned)p->n[2]);
    NvtxRange crange("teno combine");
    if (nd == 1) combine_kernel<1><<<grd, blk, 0, s>>>(c);
    else if (nd == 2) combine_kernel<2><<<grd, blk, 0, s>>>(c);
    else combine_kernel<3><<<grd, blk, 0, s>>>(c);
    CUDA_TRY(cudaGetLastError());
    return TENO_OK;
}

}  // namespace teno

using namespace teno;

extern "C" {

void teno_params_init(teno_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->ndim = 1;
    p->scheme = 8;
    p->flux_split = TENO_SPLIT_LLF;
    p->limiter = 0;
    p->n[0] = p->n[1] = p->n[2] = 1;
    p->dx[0] = p->dx[1] = p->dx[2] = 1.0;
    p->gamma = 1.4;
    p->ct_alpha1 = 14.0;
    p->ct_alpha2 = 6.4;
    p->ct_cr = 0.265;
    p->eps_beta = 1e-40;
    p->eps_eta = 1e-40;
    p->limiter_eps = 1e-13;
    p->q = 7;
}

int teno_workspace_bytes(const teno_params *p, size_t *bytes)
{
    int r = validate(p);
    if (r) return r;
    if (!bytes) return TENO_EINVAL;
    *bytes = layout(p).total;
    return TENO_OK;
}

int teno_flags_bytes(const teno_params *p, size_t *bytes)
{
    int r = validate(p);
    if (r) return r;
    if (!bytes) return TENO_EINVAL;
    size_t t = 0;
    for (int d = 0; d < p->ndim; d++) t += (size_t)face_grid(p, d) * (ncons(p) * 2 + 2 + 1);
    *bytes = t;
    return TENO_OK;
}

int teno_rhs(const teno_params *p, const double *U, double *rhs, double dt_limiter,
             uint8_t *flags, void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(rhs) || check_ptr(ws)) return TENO_EINVAL;
    if (U == rhs) return TENO_EINVAL;
    if (ws_bytes < layout(p).total) return TENO_EINVAL;
    if (p->limiter && !(dt_limiter >= 0.0)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *P = nullptr;
    CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
    return stage(p, U, U, rhs, 0, dt_limiter, nullptr, flags, (char *)ws, s, nullptr, P, nullptr);
}

int teno_rk3_step(const teno_params *p, double *U, double dt, const double *dt_device,
                  void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(ws) || ((uintptr_t)dt_device & 7)) return TENO_EINVAL;
    if (ws_bytes < layout(p).total) return TENO_EINVAL;
    if (!dt_device && !(dt >= 0.0)) return TENO_EINVAL;
    const Layout L = layout(p);
    double *Us = (double *)((char *)ws + L.stage);
    cudaStream_t s = (cudaStream_t)stream;
    // U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U = 1/3 U + 2/3 (U2 + dt L(U2));
    // each stage's combine stores the primitives of the next stage's input
    double *P = nullptr;
    CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
    if ((r = stage(p, U, U, Us, 1, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, P))) return r;
    if ((r = stage(p, Us, U, Us, 2, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, P))) return r;
    return stage(p, Us, U, U, 3, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, nullptr);
}

static int rk3_step_record(const teno_params *p, double *U, double dt, double *U1, double *U2,
                           uint8_t *flags, void *ws, size_t ws_bytes, void *stream, bool full_ct)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(U1) || check_ptr(U2) || check_ptr(ws) || !flags) return TENO_EINVAL;
    if (ws_bytes < layout(p).total || !(dt >= 0.0)) return TENO_EINVAL;
    size_t flb = 0;
    teno_flags_bytes(p, &flb);
    cudaStream_t s = (cudaStream_t)stream;
    // the stages of teno_rk3_step, with the stage states and decision records kept
    double *P = nullptr;
    CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
    if ((r = stage(p, U, U, U1, 1, dt, nullptr, flags, (char *)ws, s, nullptr, P, P, full_ct)))
        return r;
    if ((r = stage(p, U1, U, U2, 2, dt, nullptr, flags + flb, (char *)ws, s, nullptr, P, P, full_ct)))
        return r;
    return stage(p, U2, U, U, 3, dt, nullptr, flags + 2 * flb, (char *)ws, s, nullptr, P, nullptr,
                 full_ct);
}

int teno_rk3_step_record(const teno_params *p, double *U, double dt, double *U1, double *U2,
                         uint8_t *flags, void *ws, size_t ws_bytes, void *stream)
{
    return rk3_step_record(p, U, dt, U1, U2, flags, ws, ws_bytes, stream, true);
}

int teno_rk3_step_record_sel(const teno_params *p, double *U, double dt, double *U1, double *U2,
                             uint8_t *flags, void *ws, size_t ws_bytes, void *stream)
{
    return rk3_step_record(p, U, dt, U1, U2, flags, ws, ws_bytes, stream, false);
}

int teno_rhs_frozen(const teno_params *p, const double *U, double *rhs, double dt_limiter,
                    const uint8_t *decisions, void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(rhs) || check_ptr(ws) || !decisions || U == rhs) return TENO_EINVAL;
    if (ws_bytes < layout(p).total) return TENO_EINVAL;
    if (p->limiter && !(dt_limiter >= 0.0)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *P = nullptr;
    CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
    return stage(p, U, U, rhs, 0, dt_limiter, nullptr, nullptr, (char *)ws, s, decisions, P,
                 nullptr);
}

int teno_rk3_step_frozen(const teno_params *p, double *U, double dt, const uint8_t *decisions,
                         void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(ws) || !decisions) return TENO_EINVAL;
    if (ws_bytes < layout(p).total || !(dt >= 0.0)) return TENO_EINVAL;
    size_t flb = 0;
    teno_flags_bytes(p, &flb);
    const Layout L = layout(p);
    double *Us = (double *)((char *)ws + L.stage);
    cudaStream_t s = (cudaStream_t)stream;
    double *P = nullptr;
    CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
    if ((r = stage(p, U, U, Us, 1, dt, nullptr, nullptr, (char *)ws, s, decisions, P, P))) return r;
    if ((r = stage(p, Us, U, Us, 2, dt, nullptr, nullptr, (char *)ws, s, decisions + flb, P, P)))
        return r;
    return stage(p, Us, U, U, 3, dt, nullptr, nullptr, (char *)ws, s, decisions + 2 * flb, P,
                 nullptr);
}

int teno_cfl_dt(const teno_params *p, const double *U, double cfl, double *dt_device,
                void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(ws) || ((uintptr_t)dt_device & 7)) return TENO_EINVAL;
    if (ws_bytes < layout(p).total || !(cfl > 0.0)) return TENO_EINVAL;
    Status *st = (Status *)((char *)ws + layout(p).status);
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange range("teno cfl dt");
    CUDA_TRY(launch_wave_max(p, U, st, 0, s));
    cfl_finalize_kernel<<<1, 1, 0, s>>>(st, p->ndim, cfl, inv_dx_of(p), dt_device, 0);
    CUDA_TRY(cudaGetLastError());
    return TENO_OK;
}

int teno_rk3_stage(const teno_params *p, int stage_k, double *U, double *Us, double dt,
                   const double *dt_device, void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(Us) || check_ptr(ws) || U == Us || ((uintptr_t)dt_device & 7))
        return TENO_EINVAL;
    if (stage_k < 1 || stage_k > 3 || ws_bytes < layout(p).total) return TENO_EINVAL;
    if (!dt_device && !(dt >= 0.0)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *P = (double *)((char *)ws + layout(p).prims);
    // the stages of teno_rk3_step, the primitives carried in the workspace
    if (stage_k == 1) {
        CUDA_TRY(launch_prims(p, U, (char *)ws, s, &P));
        return stage(p, U, U, Us, 1, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, P);
    }
    if (stage_k == 2)
        return stage(p, Us, U, Us, 2, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, P);
    return stage(p, Us, U, U, 3, dt, dt_device, nullptr, (char *)ws, s, nullptr, P, nullptr);
}

int teno_wave_speeds(const teno_params *p, const double *U, double *amax_device, void *ws,
                     size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(ws) || !amax_device || ((uintptr_t)amax_device & 7))
        return TENO_EINVAL;
    if (ws_bytes < layout(p).total) return TENO_EINVAL;
    Status *st = (Status *)((char *)ws + layout(p).status);
    cudaStream_t s = (cudaStream_t)stream;
    NvtxRange range("teno wave speeds");
    CUDA_TRY(launch_wave_max(p, U, st, 0, s));
    // the maxima are kept as the bit patterns of non-negative doubles
    CUDA_TRY(cudaMemcpyAsync(amax_device, st->amax, sizeof(double) * p->ndim,
                             cudaMemcpyDeviceToDevice, s));
    return TENO_OK;
}

int teno_dt_from_speeds(const teno_params *p, const double *amax_device, int32_t ncopies,
                        double cfl, double *dt_device, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (!amax_device || ((uintptr_t)amax_device & 7) || !dt_device || ((uintptr_t)dt_device & 7))
        return TENO_EINVAL;
    if (ncopies < 1 || !(cfl > 0.0)) return TENO_EINVAL;
    dt_from_speeds_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(amax_device, ncopies, p->ndim, cfl,
                                                             inv_dx_of(p), dt_device);
    CUDA_TRY(cudaGetLastError());
    return TENO_OK;
}

int teno_status(void *ws, void *stream, int64_t *nonphysical)
{
    if (check_ptr(ws)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Status *st = (Status *)ws;
    unsigned long long v = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, &st->nonphys, sizeof(v), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemsetAsync(&st->nonphys, 0, sizeof(v), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (nonphysical) *nonphysical = (int64_t)v;
    return v ? TENO_ENONPHYSICAL : TENO_OK;
}

int teno_advance_host(const teno_params *p, double *U_host, double *U_dev, int nsteps,
                      double cfl, double *t_host, void *ws, size_t ws_bytes, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (!U_host || check_ptr(U_dev) || check_ptr(ws) || nsteps < 0 || !(cfl > 0.0))
        return TENO_EINVAL;
    if (ws_bytes < layout(p).total) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Status *st = (Status *)((char *)ws + layout(p).status);
    const size_t bytes = sizeof(double) * (size_t)ncons(p) * ncells(p);
    CUDA_TRY(cudaMemcpyAsync(U_dev, U_host, bytes, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(&st->t_accum, 0, sizeof(double), s));
    for (int k = 0; k < nsteps; k++) {
        CUDA_TRY(launch_wave_max(p, U_dev, st, 0, s));
        cfl_finalize_kernel<<<1, 1, 0, s>>>(st, p->ndim, cfl, inv_dx_of(p), nullptr, 1);
        CUDA_TRY(cudaGetLastError());
        if ((r = teno_rk3_step(p, U_dev, 0.0, &st->dt, ws, ws_bytes, stream))) return r;
    }
    CUDA_TRY(cudaMemcpyAsync(U_host, U_dev, bytes, cudaMemcpyDeviceToHost, s));
    double t = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&t, &st->t_accum, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (t_host) *t_host = t;
    return TENO_OK;
}

int teno_reconstruct(const teno_params *p, const double *v, int64_t count, double *out,
                     uint8_t *flags, void *stream)
{
    if (!p || (p->scheme != 8 && p->scheme != 10 && p->scheme != 12) || count < 0 || !v || !out)
        return TENO_EINVAL;
    if (!(p->ct_cr > 0.0) || !(p->eps_beta >= 0.0) || !(p->eps_eta > 0.0)) return TENO_EINVAL;
    if (count == 0) return TENO_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Consts K = consts_of(p);
    const FastK FK = fastk_of(p);
    const int fast = filter_on(p);
    const int blk = 128, grd = grid_for(count, blk);
    if (p->scheme == 8) recon_kernel<4><<<grd, blk, 0, s>>>(v, count, out, flags, K, FK, fast);
    else if (p->scheme == 10) recon_kernel<5><<<grd, blk, 0, s>>>(v, count, out, flags, K, FK, fast);
    else recon_kernel<6><<<grd, blk, 0, s>>>(v, count, out, flags, K, FK, fast);
    CUDA_TRY(cudaGetLastError());
    return TENO_OK;
}

int teno_set_decision_filter(int on)
{
    if (on != 0 && on != 1) return TENO_EINVAL;
    g_fast_filter = on;
    return TENO_OK;
}

int teno_profile_enable(int on)
{
    if (on && !g_prof.exact) CUDA_TRY(cudaMalloc(&g_prof.exact, sizeof(unsigned long long)));
    if (on) {
        CUDA_TRY(cudaDeviceSynchronize());
        CUDA_TRY(cudaMemset(g_prof.exact, 0, sizeof(unsigned long long)));
    }
    g_prof.on = on != 0;
    g_prof.used = 0;
    return TENO_OK;
}

int teno_profile_read(double *ms, int64_t *launches, int64_t *faces, int64_t *exact_recons)
{
    double tot = 0.0;
    int64_t nf = 0;
    for (int i = 0; i < g_prof.used; i++) {
        CUDA_TRY(cudaEventSynchronize(g_prof.ev[2 * i + 1]));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]));
        tot += t;
        nf += g_prof.nf[i];
    }
    if (ms) *ms = tot;
    if (launches) *launches = g_prof.used;
    if (faces) *faces = nf;
    if (exact_recons) {
        unsigned long long v = 0;
        if (g_prof.exact) {
            CUDA_TRY(cudaDeviceSynchronize());
            CUDA_TRY(cudaMemcpy(&v, g_prof.exact, sizeof(v), cudaMemcpyDeviceToHost));
        }
        *exact_recons = (int64_t)v;
    }
    return TENO_OK;
}

int teno_debug_bounds(void *ws, void *stream, int64_t *count, int64_t *line, int64_t *index,
                      int64_t *extent)
{
    if (check_ptr(ws)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Status *st = (Status *)ws;
    long long rec[4] = {0, 0, 0, 0};   // count, line, index, extent (contiguous in Status)
    static_assert(offsetof(Status, oob_line) == offsetof(Status, oob_count) + 8 &&
                      offsetof(Status, oob_extent) == offsetof(Status, oob_count) + 24,
                  "bounds record layout");
    CUDA_TRY(cudaMemcpyAsync(rec, &st->oob_count, sizeof(rec), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemsetAsync(&st->oob_count, 0, sizeof(rec), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (count) *count = rec[0];
    if (line) *line = rec[1];
    if (index) *index = rec[2];
    if (extent) *extent = rec[3];
    return rec[0] ? TENO_EBOUNDS : TENO_OK;
}

int teno_build_flags(void)
{
#ifdef TENO_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

const char *teno_strerror(int code)
{
    switch (code) {
    case TENO_OK: return "ok";
    case TENO_EINVAL: return "invalid parameter, pointer, size or alignment";
    case TENO_ECUDA: return "CUDA runtime error";
    case TENO_ENONPHYSICAL: return "non-physical state (rho <= 0, p <= 0, non-finite value or "
                                   "non-positive Roe sound speed squared)";
    case TENO_ETIMEOUT: return "bounded device wait timed out";
    case TENO_EBOUNDS: return "out-of-range index found by the bounds-checked build";
    default: return "unknown error code";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// teno_rhs_static: teno_rhs without a caller-supplied workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// right-hand side -- plugin code inside a host application that owns the
// device memory pool, code with a memory budget fixed at start-up, or code
// that must not call cudaMalloc while a CUDA graph is being captured.  This
// entry point takes its scratch (status header + face-flux buffers) from one
// file-scope device array instead of a workspace; it calls no cudaMalloc,
// cudaFree or other allocating routine.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_rhs_scratch[TENO_RHS_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
// Per device: the array's address and the context it was resolved in.  A
// device reset (cudaDeviceReset) or any other context teardown unloads the
// module holding the array, so an address is only reused while the current
// context is the one it came from (compared by the driver's unique context id,
// which a re-created context never repeats).
struct ScratchEntry {
    unsigned long long ctx_id;
    void *ptr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
CUresult (*g_ctx_get_current)(CUcontext *) = nullptr;
CUresult (*g_ctx_get_id)(CUcontext, unsigned long long *) = nullptr;
}  // namespace

// Unique id of the calling thread's current context (0 if none is current),
// through the driver entry points the runtime hands out (no link to libcuda).
// Called with g_scratch_mutex held.
static int current_context_id(unsigned long long *id)
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return TENO_ECUDA;
        g_ctx_get_current = (CUresult(*)(CUcontext *))f1;
        g_ctx_get_id = (CUresult(*)(CUcontext, unsigned long long *))f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return TENO_ECUDA;
    *id = 0;
    if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return TENO_ECUDA;
    return TENO_OK;
}

// Device address of g_rhs_scratch in the current context, resolved once per
// device and context (the host-side symbol is only a stand-in, never a device
// address).
static int rhs_scratch_address(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return TENO_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    int r = current_context_id(&id);
    if (r) return r;
    ScratchEntry &e = g_scratch[dev];
    if (!e.ptr || id == 0 || e.ctx_id != id) {
        void *ptr = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&ptr, g_rhs_scratch));   // initialises the context if needed
        if ((r = current_context_id(&id))) return r;
        e.ptr = ptr;
        e.ctx_id = id;
    }
    *out = e.ptr;
    return TENO_OK;
}

extern "C" int teno_rhs_static(const teno_params *p, const double *U, double *rhs,
                               double dt_limiter, uint8_t *flags, void *stream)
{
    int r = validate(p);
    if (r) return r;
    if (check_ptr(U) || check_ptr(rhs) || U == rhs) return TENO_EINVAL;
    if (p->limiter && !(dt_limiter >= 0.0)) return TENO_EINVAL;
    // The right-hand side needs the status header and the face-flux buffers
    // (the part of the workspace layout before the RK stage buffer).
    if (layout(p).stage > (size_t)TENO_RHS_STATIC_SCRATCH_BYTES) return TENO_EINVAL;
    void *scratch = nullptr;
    if ((r = rhs_scratch_address(&scratch))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps the previous call's contents: zero the status header
    // (counters and reduction slots) before use.
    CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(Status), s));
    return stage(p, U, U, rhs, 0, dt_limiter, nullptr, flags, (char *)scratch, s, nullptr, nullptr,
                 nullptr);
}
