// Batched mode (include/teno.h, teno_batch_*): thousands of independent 1D
// Euler problems of uneven size advanced together with per-problem CFL steps.
//
// One step = per-problem wave-speed maxima (persistent, one block per
// (problem, 256-cell tile)) -> per-problem dt -> three stages, each a
// persistent face sweep that pulls (problem, face tile) items from an atomic
// counter, then a combine over (problem, cell tile) items.  The face and cell
// arithmetic is the single-problem code (face_block, cell_quantities), so the
// results are bitwise those of teno_cfl_dt + teno_rk3_step per problem.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "teno.h"
#include "teno_face.cuh"

namespace teno {

struct BatchProb {
    int64_t n, u_off, f_off, p_off;   // cells; state, face-flux, primitive-row offsets
    double inv_dx;
    int32_t scheme, limiter, bc_lo, bc_hi;
};

struct BatchSlot {
    unsigned long long amax;   // bit pattern of max(|u| + c) >= 0
    double dt, lam, t;
};

constexpr int kCellTile = 256;
constexpr int kTiles[3] = {64, 128, 256};

// Item -> problem by binary search in an exclusive prefix of per-problem item
// counts (prefix[nprob] = total).
__device__ __forceinline__ int find_problem(const int32_t *prefix, int nprob, int item)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-problem wave-speed maxima of the step's state; the same pass stores its
// primitives for the first stage's sweep and counts its non-physical cells.
__global__ void __launch_bounds__(kCellTile) batch_wave_max_kernel(
    const BatchProb *probs, int nprob, const int32_t *cprefix, const double *U, BatchSlot *slots,
    double *P, Status *st, Consts K)
{
    __shared__ double red[kCellTile / 32];
    const int nitems = cprefix[nprob];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int p = find_problem(cprefix, nprob, it);
        const BatchProb d = probs[p];
        const int64_t i = (int64_t)(it - cprefix[p]) * kCellTile + threadIdx.x;
        double m = 0.0;
        if (i < d.n) {
            const double *Up = U + d.u_off;
            double Uc[3] = {Up[i], Up[d.n + i], Up[2 * d.n + i]};
            CellQ<1> q;
            cell_quantities<1, 0>(Uc, K, q);
            store_prims<1>(q, P + d.p_off, d.n, i);
            if (nonphysical_cell<1>(Uc[0], q)) atomicAdd(&st->nonphys, 1ull);
            const double e = fabs(q.u[0]) + q.c;
            if (e > m) m = e;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, m, o);
            if (w > m) m = w;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = red[0];
            for (int k = 1; k < kCellTile / 32; k++)
                if (red[k] > v) v = red[k];
            if (v > 0.0) atomicMax(&slots[p].amax, (unsigned long long)__double_as_longlong(v));
        }
        __syncthreads();
    }
}

// dt = cfl / (A / dx) and the limiter's dt/dx per problem, exactly as
// cfl_finalize_kernel + prepare_kernel do for one 1D problem.
__global__ void batch_finalize_kernel(const BatchProb *probs, int nprob, BatchSlot *slots,
                                      double cfl)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const double idx = probs[p].inv_dx;
    const double S = __longlong_as_double((long long)slots[p].amax) * idx;
    const double dt = cfl / S;
    slots[p].dt = dt;
    slots[p].lam = dt * idx;
    slots[p].t = slots[p].t + dt;
    slots[p].amax = 0ull;
}

// Registers bounded as for the 2D/3D sweeps: 384 threads' worth of blocks per SM.
template <int TF>
__global__ void __launch_bounds__(TF, (384 / TF > 1 ? 384 / TF : 1)) batch_face_kernel(
    const BatchProb *probs, int nprob, const int32_t *fprefix, const double *U, const double *P,
    double *F, BatchSlot *slots, Status *st, Consts K, FastK FK, int fast, int *counter)
{
    extern __shared__ double sm[];
    __shared__ int s_item;
    const int nitems = fprefix[nprob];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int p = find_problem(fprefix, nprob, it);
        const BatchProb d = probs[p];
        FaceArgs a;
        a.U = U + d.u_off;
        a.P = P + d.p_off;                  // the stage input's stored primitives
        a.F = F + d.f_off;
        a.flags = nullptr;
        a.frozen = nullptr;
        a.argmax = nullptr;
        a.frozen_argmax = nullptr;
        a.limrec = nullptr;
        a.st = st;
        a.n[0] = d.n; a.n[1] = 1; a.n[2] = 1;
        a.ncell = d.n;
        a.nfaces = d.n + 1;
        a.bc_lo = d.bc_lo;
        a.bc_hi = d.bc_hi;
        a.bcs_lo = nullptr;
        a.bcs_hi = nullptr;
        a.lam = &slots[p].lam;
        a.fast = fast;
        a.need_ct = 0;
        a.skip_last = 0;
        a.count_cells = 0;
        a.exact_count = nullptr;
        a.FK = FK;
        a.K = K;
        a.K.limiter = d.limiter;
        const int64_t f0 = (int64_t)(it - fprefix[p]) * TF;
        if (d.scheme == 10) face_block<1, 5, 0, 1, TF, kSweepPlain>(a, f0, 0, 0, 0, sm);
        else face_block<1, 4, 0, 1, TF, kSweepPlain>(a, f0, 0, 0, 0, sm);
        __syncthreads();
    }
}

// Flux difference and SSP-RK3 stage per cell (the arithmetic of combine_kernel
// for one 1D problem), with each problem's own dt.  Stages 1 and 2 store the
// new stage state's primitives for the next sweep and count its
// non-physical cells (the next evaluation's input; the step's own state is
// counted by the wave-maximum pass).
__global__ void __launch_bounds__(kCellTile) batch_combine_kernel(
    const BatchProb *probs, int nprob, const int32_t *cprefix, const double *Uk, const double *Un,
    double *out, const double *F, const BatchSlot *slots, double *P, Status *st, Consts K, int mode)
{
    const int nitems = cprefix[nprob];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int p = find_problem(cprefix, nprob, it);
        const BatchProb d = probs[p];
        const int64_t i = (int64_t)(it - cprefix[p]) * kCellTile + threadIdx.x;
        if (i >= d.n) continue;
        const double *Ukp = Uk + d.u_off;
        const double *Fp = F + d.f_off;
        double Uc[3] = {Ukp[i], Ukp[d.n + i], Ukp[2 * d.n + i]};
        double Uo[3];
        const double dt = slots[p].dt;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double *Fd = Fp + c * (d.n + 1);
            double acc = 0.0;
            const double t = (Fd[i + 1] - Fd[i]) * d.inv_dx;
            acc = acc - t;
            const double s = Uc[c] + dt * acc;
            double o;
            if (mode == 1) o = s;
            else if (mode == 2) o = 0.75 * Un[d.u_off + c * d.n + i] + 0.25 * s;
            else o = (1.0 / 3.0) * Un[d.u_off + c * d.n + i] + (2.0 / 3.0) * s;
            out[d.u_off + c * d.n + i] = o;
            Uo[c] = o;
        }
        if (mode < 3) {
            CellQ<1> q;
            cell_quantities<1, 0>(Uo, K, q);
            store_prims<1>(q, P + d.p_off, d.n, i);
            if (nonphysical_cell<1>(Uo[0], q)) atomicAdd(&st->nonphys, 1ull);
        }
    }
}

}  // namespace teno

using namespace teno;

struct teno_batch {
    teno_params common;
    std::vector<teno_batch_problem> probs;
    std::vector<BatchProb> desc;
    std::vector<int32_t> fprefix[3];
    std::vector<int32_t> cprefix;
    size_t u_len = 0, f_len = 0, p_len = 0;
    size_t off_slots = 0, off_counters = 0, off_desc = 0, off_fprefix[3] = {0, 0, 0},
           off_cprefix = 0, off_F = 0, off_Us = 0, off_P = 0, off_single = 0, total = 0;
    size_t single_bytes = 0;
    int tile_idx = 1;           // index into kTiles
    int blocks_per_sm = 2;
    int num_sms = 0;
    const void *uploaded_ws = nullptr;
    int uploaded_dev = -1;
    // captured step
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    const void *g_U = nullptr, *g_ws = nullptr;
    double g_cfl = 0.0;
    int g_tile = -1, g_bps = -1;
    int g_fast = -1;            // filter switch the graph was captured with
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int problem_params(const teno_batch *b, int p, teno_params *pp)
{
    *pp = b->common;
    const teno_batch_problem &q = b->probs[p];
    pp->ndim = 1;
    pp->n[0] = q.n; pp->n[1] = 1; pp->n[2] = 1;
    pp->dx[0] = q.dx; pp->dx[1] = 1.0; pp->dx[2] = 1.0;
    pp->scheme = q.scheme;
    pp->limiter = q.limiter;
    pp->bc_lo[0] = q.bc_lo; pp->bc_hi[0] = q.bc_hi;
    pp->bc_lo[1] = pp->bc_lo[2] = pp->bc_hi[1] = pp->bc_hi[2] = 0;
    for (int a = 0; a < 3; a++) pp->bc_state_lo[a] = pp->bc_state_hi[a] = nullptr;   // no Dirichlet
    size_t bytes;
    return teno_workspace_bytes(pp, &bytes);
}

Consts consts_common(const teno_params *p)
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

template <int TF>
cudaError_t set_face_attr()
{
    constexpr size_t smem = std::max(face_smem_bytes<1, 5, 1, TF>(), face_smem_bytes<1, 4, 1, TF>());
    return cudaFuncSetAttribute(batch_face_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

int upload(teno_batch *b, char *ws, cudaStream_t s)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (b->uploaded_ws == ws && b->uploaded_dev == dev) return TENO_OK;
    const int np = (int)b->probs.size();
    CUDA_TRY(cudaMemsetAsync(ws, 0, b->off_desc, s));       // status, slots, counters
    CUDA_TRY(cudaMemcpyAsync(ws + b->off_desc, b->desc.data(), sizeof(BatchProb) * np,
                             cudaMemcpyHostToDevice, s));
    for (int k = 0; k < 3; k++)
        CUDA_TRY(cudaMemcpyAsync(ws + b->off_fprefix[k], b->fprefix[k].data(),
                                 sizeof(int32_t) * (np + 1), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ws + b->off_cprefix, b->cprefix.data(), sizeof(int32_t) * (np + 1),
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));     // the host vectors are pageable
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    b->num_sms = prop.multiProcessorCount;
    CUDA_TRY(set_face_attr<64>());
    CUDA_TRY(set_face_attr<128>());
    CUDA_TRY(set_face_attr<256>());
    b->uploaded_ws = ws;
    b->uploaded_dev = dev;
    return TENO_OK;
}

// Enqueue one persistent-mode step on stream s.
int enqueue_step(teno_batch *b, double *U, double cfl, char *ws, int tile_idx, int bps,
                 cudaStream_t s)
{
    const int np = (int)b->probs.size();
    const Consts K = consts_common(&b->common);
    Status *st = (Status *)ws;
    BatchSlot *slots = (BatchSlot *)(ws + b->off_slots);
    int *counters = (int *)(ws + b->off_counters);
    const BatchProb *desc = (const BatchProb *)(ws + b->off_desc);
    const int32_t *fpre = (const int32_t *)(ws + b->off_fprefix[tile_idx]);
    const int32_t *cpre = (const int32_t *)(ws + b->off_cprefix);
    double *F = (double *)(ws + b->off_F);
    double *Us = (double *)(ws + b->off_Us);
    double *P = (double *)(ws + b->off_P);
    const int ncitems = b->cprefix[np];
    const int grid_c = std::max(1, std::min(ncitems, b->num_sms * 8));
    CUDA_TRY(cudaMemsetAsync(counters, 0, 3 * sizeof(int), s));
    batch_wave_max_kernel<<<grid_c, kCellTile, 0, s>>>(desc, np, cpre, U, slots, P, st, K);
    CUDA_TRY(cudaGetLastError());
    batch_finalize_kernel<<<(np + 127) / 128, 128, 0, s>>>(desc, np, slots, cfl);
    CUDA_TRY(cudaGetLastError());
    const int TF = kTiles[tile_idx];
    const int grid_f = b->num_sms * bps;
    const FastK FK = fastk_make(b->common.ct_cr, b->common.ct_alpha1, b->common.ct_alpha2,
                                b->common.eps_beta, b->common.eps_eta);
    const int fast = g_fast_filter && fast_filter_valid(b->common.eps_beta, b->common.eps_eta);
    for (int stg = 0; stg < 3; stg++) {
        const double *Uin = stg == 0 ? U : Us;
        if (TF == 64) {
            constexpr size_t sm = std::max(face_smem_bytes<1, 5, 1, 64>(), face_smem_bytes<1, 4, 1, 64>());
            batch_face_kernel<64><<<grid_f, 64, sm, s>>>(desc, np, fpre, Uin, P, F, slots, st, K, FK, fast, counters + stg);
        } else if (TF == 128) {
            constexpr size_t sm = std::max(face_smem_bytes<1, 5, 1, 128>(), face_smem_bytes<1, 4, 1, 128>());
            batch_face_kernel<128><<<grid_f, 128, sm, s>>>(desc, np, fpre, Uin, P, F, slots, st, K, FK, fast, counters + stg);
        } else {
            constexpr size_t sm = std::max(face_smem_bytes<1, 5, 1, 256>(), face_smem_bytes<1, 4, 1, 256>());
            batch_face_kernel<256><<<grid_f, 256, sm, s>>>(desc, np, fpre, Uin, P, F, slots, st, K, FK, fast, counters + stg);
        }
        CUDA_TRY(cudaGetLastError());
        batch_combine_kernel<<<grid_c, kCellTile, 0, s>>>(desc, np, cpre, Uin, U, stg == 2 ? U : Us, F,
                                                         slots, P, st, K, stg + 1);
        CUDA_TRY(cudaGetLastError());
    }
    return TENO_OK;
}

int per_problem_steps(teno_batch *b, double *U, int nsteps, double cfl, char *ws, cudaStream_t s)
{
    BatchSlot *slots = (BatchSlot *)(ws + b->off_slots);
    void *ws1 = ws + b->off_single;
    for (int k = 0; k < nsteps; k++) {
        for (size_t p = 0; p < b->probs.size(); p++) {
            teno_params pp;
            int r = problem_params(b, (int)p, &pp);
            if (r) return r;
            double *Up = U + b->probs[p].offset;
            double *dt_dev = &slots[p].dt;
            if ((r = teno_cfl_dt(&pp, Up, cfl, dt_dev, ws1, b->single_bytes, s))) return r;
            if ((r = teno_rk3_step(&pp, Up, 0.0, dt_dev, ws1, b->single_bytes, s))) return r;
        }
    }
    return TENO_OK;
}

}  // namespace

extern "C" {

int teno_batch_create(const teno_params *common, const teno_batch_problem *probs, int32_t nprob,
                      teno_batch **out)
{
    if (!common || !probs || !out || nprob <= 0) return TENO_EINVAL;
    teno_batch *b = new (std::nothrow) teno_batch();
    if (!b) return TENO_EINVAL;
    b->common = *common;
    b->common.ndim = 1;
    b->probs.assign(probs, probs + nprob);
    size_t f_off = 0, p_off = 0, u_end = 0, single = 0;
    int64_t ftiles[3] = {0, 0, 0}, ctiles = 0;
    for (int k = 0; k < 3; k++) b->fprefix[k].push_back(0);
    b->cprefix.push_back(0);
    for (int p = 0; p < nprob; p++) {
        const teno_batch_problem &q = probs[p];
        teno_params pp;
        // batched problems use the eight- and ten-point schemes only (the
        // persistent kernel holds both instantiations; a third would raise
        // its registers and shared memory for every problem)
        if (problem_params(b, p, &pp) != TENO_OK || q.offset < 0 || (q.offset & 1) ||
            (q.scheme != 8 && q.scheme != 10)) {
            delete b;
            return TENO_EINVAL;
        }
        size_t bytes = 0;
        teno_workspace_bytes(&pp, &bytes);
        single = std::max(single, bytes);
        BatchProb d;
        d.n = q.n;
        d.u_off = q.offset;
        d.f_off = (int64_t)f_off;
        d.p_off = (int64_t)p_off;
        d.inv_dx = 1.0 / q.dx;
        d.scheme = q.scheme;
        d.limiter = q.limiter;
        d.bc_lo = q.bc_lo;
        d.bc_hi = q.bc_hi;
        b->desc.push_back(d);
        f_off += 3 * (size_t)(q.n + 1);
        f_off = (f_off + 1) & ~(size_t)1;                 // keep 16-byte alignment
        p_off += (size_t)PrimRows<1>::NP * (size_t)q.n;
        u_end = std::max(u_end, (size_t)(q.offset + 3 * q.n));
        for (int k = 0; k < 3; k++) {
            ftiles[k] += (q.n + 1 + kTiles[k] - 1) / kTiles[k];
            b->fprefix[k].push_back((int32_t)ftiles[k]);
        }
        ctiles += (q.n + kCellTile - 1) / kCellTile;
        b->cprefix.push_back((int32_t)ctiles);
        if (ftiles[0] > (int64_t)1 << 30 || ctiles > (int64_t)1 << 30) {
            delete b;
            return TENO_EINVAL;
        }
    }
    // state blocks must not overlap
    std::vector<std::pair<int64_t, int64_t>> iv;
    for (auto &q : b->probs) iv.push_back({q.offset, q.offset + 3 * q.n});
    std::sort(iv.begin(), iv.end());
    for (size_t i = 1; i < iv.size(); i++)
        if (iv[i].first < iv[i - 1].second) { delete b; return TENO_EINVAL; }
    b->u_len = u_end;
    b->f_len = f_off;
    b->p_len = p_off;
    b->single_bytes = single;
    size_t off = a256(sizeof(Status));
    b->off_slots = off;
    off += a256(sizeof(BatchSlot) * nprob);
    b->off_counters = off;
    off += 256;
    b->off_desc = off;
    off += a256(sizeof(BatchProb) * nprob);
    for (int k = 0; k < 3; k++) {
        b->off_fprefix[k] = off;
        off += a256(sizeof(int32_t) * (nprob + 1));
    }
    b->off_cprefix = off;
    off += a256(sizeof(int32_t) * (nprob + 1));
    b->off_F = off;
    off += a256(sizeof(double) * b->f_len);
    b->off_Us = off;
    off += a256(sizeof(double) * b->u_len);
    b->off_P = off;
    off += a256(sizeof(double) * b->p_len);
    b->off_single = off;
    off += a256(single);
    b->total = off;
    *out = b;
    return TENO_OK;
}

int teno_batch_workspace_bytes(const teno_batch *b, size_t *bytes)
{
    if (!b || !bytes) return TENO_EINVAL;
    *bytes = b->total;
    return TENO_OK;
}

int teno_batch_rk3_steps(teno_batch *b, double *U, int32_t nsteps, double cfl, int32_t mode,
                         void *ws, size_t ws_bytes, void *stream)
{
    if (!b || !U || !ws || ((uintptr_t)U & 15) || ((uintptr_t)ws & 255)) return TENO_EINVAL;
    if (ws_bytes < b->total || nsteps < 0 || !(cfl > 0.0)) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int r = upload(b, (char *)ws, s);
    if (r) return r;
    if (mode == TENO_BATCH_PER_PROBLEM) return per_problem_steps(b, U, nsteps, cfl, (char *)ws, s);
    if (mode == TENO_BATCH_STREAM) {
        for (int k = 0; k < nsteps; k++)
            if ((r = enqueue_step(b, U, cfl, (char *)ws, b->tile_idx, b->blocks_per_sm, s))) return r;
        return TENO_OK;
    }
    if (mode != TENO_BATCH_GRAPH) return TENO_EINVAL;
    if (!b->exec || b->g_U != U || b->g_ws != ws || b->g_cfl != cfl || b->g_tile != b->tile_idx ||
        b->g_bps != b->blocks_per_sm || b->g_fast != g_fast_filter) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (!b->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        // the capture stream must see everything already queued on s
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(ev, s));
        CUDA_TRY(cudaStreamWaitEvent(b->cap_stream, ev, 0));
        CUDA_TRY(cudaStreamSynchronize(b->cap_stream));
        cudaEventDestroy(ev);
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        int er = enqueue_step(b, U, cfl, (char *)ws, b->tile_idx, b->blocks_per_sm, b->cap_stream);
        cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &g);
        if (er) return er;
        if (ee != cudaSuccess) return TENO_ECUDA;
        ee = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return TENO_ECUDA;
        b->g_U = U;
        b->g_ws = ws;
        b->g_cfl = cfl;
        b->g_tile = b->tile_idx;
        b->g_bps = b->blocks_per_sm;
        b->g_fast = g_fast_filter;
    }
    for (int k = 0; k < nsteps; k++) CUDA_TRY(cudaGraphLaunch(b->exec, s));
    return TENO_OK;
}

int teno_batch_autotune(teno_batch *b, double *U_scratch, void *ws, size_t ws_bytes, void *stream,
                        int32_t *chosen_tile, int32_t *chosen_blocks_per_sm)
{
    if (!b || !U_scratch || !ws || ws_bytes < b->total) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int r = upload(b, (char *)ws, s);
    if (r) return r;
    const double cfl = 0.4;
    // warm-up (module load, first touch)
    if ((r = enqueue_step(b, U_scratch, cfl, (char *)ws, 1, 1, s))) return r;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_t = b->tile_idx, best_b = b->blocks_per_sm;
    const int bps_c[5] = {1, 2, 3, 4, 6};
    for (int ti = 0; ti < 3; ti++) {
        for (int bi = 0; bi < 5; bi++) {
            int maxb = 0;
            const int TF = kTiles[ti];
            cudaError_t oe;
            if (TF == 64)
                oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_face_kernel<64>, 64,
                         std::max(face_smem_bytes<1, 5, 1, 64>(), face_smem_bytes<1, 4, 1, 64>()));
            else if (TF == 128)
                oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_face_kernel<128>, 128,
                         std::max(face_smem_bytes<1, 5, 1, 128>(), face_smem_bytes<1, 4, 1, 128>()));
            else
                oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, batch_face_kernel<256>, 256,
                         std::max(face_smem_bytes<1, 5, 1, 256>(), face_smem_bytes<1, 4, 1, 256>()));
            if (oe != cudaSuccess) return TENO_ECUDA;
            if (bps_c[bi] > maxb) continue;
            CUDA_TRY(cudaEventRecord(e0, s));
            if ((r = enqueue_step(b, U_scratch, cfl, (char *)ws, ti, bps_c[bi], s))) return r;
            CUDA_TRY(cudaEventRecord(e1, s));
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_t = ti;
                best_b = bps_c[bi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_idx = best_t;
    b->blocks_per_sm = best_b;
    if (chosen_tile) *chosen_tile = kTiles[best_t];
    if (chosen_blocks_per_sm) *chosen_blocks_per_sm = best_b;
    return TENO_OK;
}

int teno_batch_times(const teno_batch *b, void *ws, void *stream, double *t_host)
{
    if (!b || !ws || !t_host) return TENO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = b->probs.size();
    std::vector<BatchSlot> tmp(np);
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), (char *)ws + b->off_slots, sizeof(BatchSlot) * np,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t p = 0; p < np; p++) t_host[p] = tmp[p].t;
    return TENO_OK;
}

void teno_batch_destroy(teno_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

}  // extern "C"
