/*
 * teno.h -- C ABI of the GB300 (sm_103a) TENO-AA compressible-Euler library.
 *
 * The library evaluates the semi-discrete right-hand side of the compressible
 * Euler equations (arXiv 2109.14340, Sec. 1 Eq. Euler; Sec. 2 Eq.
 * approximateEq) with the eight-, ten- or twelve-point TENO-AA reconstruction
 * (Sec. 3, Sec. 4; the twelve-point candidate S6 built by the recipe of Sec.
 * 4.1, see teno_params.scheme) of Roe-averaged characteristic, flux-split
 * fluxes (Sec. 5), and advances it with SSP-RK3 (Sec. 5, Eq. Runge-kutta)
 * under a CFL time step.
 *
 * Conventions shared by every call:
 *  - State arrays are FP64, structure of arrays, interior cells only:
 *    U[c * ncells + (x + n[0] * (y + n[1] * z))], c = 0 .. ncons-1 with
 *    ncons = ndim + 2 and order (rho, rho*u_x, [rho*u_y, [rho*u_z,]] E).
 *    They live in device memory owned by the caller, 16-byte aligned.
 *  - Every call is enqueued on the caller's stream (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream).  No call allocates memory or
 *    synchronises, except teno_status (which synchronises the stream) and
 *    teno_advance_host (which copies host buffers and synchronises).
 *  - The workspace ws (ws_bytes >= teno_workspace_bytes) is device memory
 *    owned by the caller; calls sharing one workspace must be ordered on one
 *    stream.  Its contents carry no state between calls except the
 *    non-physical counter read by teno_status.
 *  - Every call returns TENO_OK or an error code; parameters are validated
 *    on the host before anything is enqueued.  Physical validity of the state
 *    (rho > 0, p > 0, finite values, positive Roe sound speed squared) is
 *    checked on the device without trapping: offending cells and faces are
 *    counted and reported by teno_status.
 */
#ifndef TENO_H
#define TENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define TENO_OK 0
#define TENO_EINVAL 1          /* bad parameter, pointer, size or alignment   */
#define TENO_ECUDA 2           /* a CUDA runtime call failed                  */
#define TENO_ENONPHYSICAL 3    /* teno_status: non-physical states were seen  */
#define TENO_ETIMEOUT 4        /* reserved for a bounded device-side wait that
                                  gave up; no call returns it: no kernel of
                                  this library waits on a flag, a peer or a
                                  barrier outside its own block (the batched
                                  work list is an atomic counter)             */
#define TENO_EBOUNDS 5         /* teno_debug_bounds: the bounds-checked build
                                  found an index outside its array           */

/* Boundary conditions per axis side (App. A). */
#define TENO_BC_PERIODIC 0     /* App. A.4: ghost -r = cell n-r (both sides)  */
#define TENO_BC_TRANSMISSIVE 1 /* zero-order extrapolation: ghost = end cell  */
#define TENO_BC_SLIPWALL 2     /* App. A.1: ghost -r = cell r-1, normal
                                  momentum negated                            */
#define TENO_BC_NOSLIP 3       /* App. A.2: ghost -r = cell r-1, all momentum
                                  components negated                          */
#define TENO_BC_DIRICHLET 4    /* App. A.3: given boundary-face primitive
                                  state phi' (bc_state_lo / bc_state_hi),
                                  ghost -r primitives = 2 phi' - those of cell
                                  r-1 (second order); not differentiated by
                                  the adjoint calls, not in batched mode      */
#define TENO_BC_HALO 5         /* domain decomposition: the H ghost cells of
                                  the side are a neighbouring sub-domain's
                                  cells, given in a caller-owned halo array
                                  (bc_state_lo / bc_state_hi) of conserved
                                  variables [ncons][H][m]: plane q holds cell
                                  -H + q below the sub-domain (low side) or
                                  n + q above it (high side), m = cells of a
                                  plane in the order of the two other axes, x
                                  fastest; the caller fills it before each
                                  evaluation (teno_rk3_stage).  Not with the
                                  limiter in 2D / 3D (its direction weights
                                  need the whole domain's wave speeds), not in
                                  the adjoint calls or batched mode           */

/* Flux splitting of the characteristic fluxes (Sec. 5). */
#define TENO_SPLIT_LLF 0       /* per field k: alpha_k = max |lambda_k| over
                                  the stencil cells                           */
#define TENO_SPLIT_RUSANOV 1   /* all fields: alpha = max (|u_d| + c) over the
                                  stencil cells                               */

typedef struct teno_params {
    int32_t ndim;          /* 1, 2 or 3                                         */
    int32_t scheme;        /* 8 (TENO8-AA, Sec. 4.3), 10 (TENO10-AA, Sec. 4.2)
                              or 12 (TENO12-AA: the next member of the family
                              of Sec. 3.1, its twelve-point candidate S6 built
                              by the recipe of Sec. 4.1 with the parameters
                              that give back the printed S3-S5: nu = 7,
                              tenth-order constraint, 11th-difference part
                              1/200 on cell i; beta_{6,12} from Eq.
                              measureTENO)                                    */
    int32_t flux_split;    /* TENO_SPLIT_LLF or TENO_SPLIT_RUSANOV              */
    int32_t limiter;       /* 1: positivity-preserving flux limiter (Sec. 5.3)  */
    int64_t n[3];          /* interior cells per axis, x fastest; 1 if unused;
                              H <= n[d] <= 2^31 on used axes (H = scheme / 2)
                              and n[1], n[2] <= 65535 (CUDA grid limits)    */
    double dx[3];          /* uniform spacing per axis (> 0)                    */
    double gamma;          /* ratio of specific heats (> 1), ideal-gas EOS      */
    double ct_alpha1;      /* alpha_1 of Eq. CT_definition, default 14          */
    double ct_alpha2;      /* alpha_2 of Eq. CT_definition, default 6.4         */
    double ct_cr;          /* C_r of Eq. m_definition, default 0.265            */
    double eps_beta;       /* epsilon of Eq. scale_separation, default 1e-40    */
    double eps_eta;        /* epsilon of the eta measure (Sec. 3.4), 1e-40      */
    double limiter_eps;    /* density / pressure floor of the limiter, 1e-13    */
    int32_t q;             /* exponent of Eq. scale_separation; must be 7       */
    int32_t bc_lo[3];      /* TENO_BC_* at the low end of each axis             */
    int32_t bc_hi[3];      /* TENO_BC_* at the high end of each axis            */
    int32_t reserved;      /* must be 0                                          */
    /* TENO_BC_DIRICHLET boundary states, caller-owned device arrays (16-byte
     * aligned), read on every right-hand-side evaluation (the caller may
     * update them between calls, e.g. a time-dependent inflow); NULL for
     * other sides.  Layout for axis d: primitives (rho, u_0 .. u_{ndim-1}, p)
     * major, then the boundary faces in the order of the two other axes,
     * x fastest: state[q * m + s], m = product of n over the axes != d,
     * s = the face's index among them (d = 0: y + n[1] z; d = 1: x + n[0] z;
     * d = 2: x + n[0] y).  TENO_BC_HALO sides take their halo array here
     * (layout at TENO_BC_HALO). */
    const double *bc_state_lo[3];
    const double *bc_state_hi[3];
} teno_params;

/* Fill *p with the paper's built-in parameters (eps = 1e-40, q = 7 of Sec.
 * 3.2; C_r = 0.265, alpha_1 = 14, alpha_2 = 6.4 of Sec. 3.4), gamma = 1.4,
 * TENO8-AA, LLF, no limiter, periodic 1D grid of one cell (caller sets n, dx). */
void teno_params_init(teno_params *p);

/* Workspace bytes needed by every call below for these parameters.
 * Returns TENO_EINVAL for invalid parameters (then *bytes is untouched). */
int teno_workspace_bytes(const teno_params *p, size_t *bytes);

/* Bytes of the per-face decision record written by teno_rhs (flags != NULL).
 * Part 1, for each direction d < ndim in turn, for each face of the face grid
 * (n with n[d] + 1, x fastest), for each characteristic field k < ncons, for
 * the + then - split flux, one byte: bits 0-1 selected large stencil S_L as
 * L - 2 (1: S3, 2: S4, 3: S5) or 0 for the small-stencil fallback of Eq.
 * renormalize; bits 2-4 the cut-offs delta_0..delta_2 of Eq. cutoff in the
 * fallback (else 0); S6 of the twelve-point scheme as bits 0-4 all zero (a
 * fallback always keeps at least one small stencil, so it never writes that
 * pattern); bits 5-7 the C_T exponent [beta] of Eq. CT_definition minus 7
 * (mod 8).  Part 2, for each direction in turn, for each face, one
 * little-endian 16-bit word: the stencil cells (0 .. 2H-1, from cell i-H+1)
 * where the splitting speeds are maximal (first maximum), 4 bits each for
 * |u_d - c|, |u_d|, |u_d + c| and |u_d| + c.  Part 3, for each direction in
 * turn, for each face, one byte: 1 where the positivity-preserving limiter
 * (Sec. 5.3) bound, i.e. blended the face flux toward the Lax-Friedrichs
 * flux, else 0 (always 0 with p->limiter == 0). */
int teno_flags_bytes(const teno_params *p, size_t *bytes);

/* Semi-discrete right-hand side L(U) = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d
 * (Eq. approximateEq, dimension by dimension as in Sec. 5).
 *   U          device, ncons * ncells doubles (read)
 *   rhs        device, ncons * ncells doubles (written); must not alias U
 *   dt_limiter time step used by the limiter's one-sided updates (ignored
 *              when p->limiter == 0)
 *   flags      device, teno_flags_bytes bytes, or NULL
 *   ws         device workspace of ws_bytes bytes */
int teno_rhs(const teno_params *p, const double *U, double *rhs, double dt_limiter,
             uint8_t *flags, void *ws, size_t ws_bytes, void *stream);

/* One SSP-RK3 step (Eq. Runge-kutta) in place on U:
 *   U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 *   U  <- 1/3 U + 2/3 (U2 + dt L(U2)).
 * dt is read from dt_device (device scalar) when it is not NULL, else the
 * host value dt is used.  Each stage's limiter uses the same dt. */
int teno_rk3_step(const teno_params *p, double *U, double dt, const double *dt_device,
                  void *ws, size_t ws_bytes, void *stream);

/* CFL time step (Sec. 5, CFL number 0.4 by default):
 *   A_d = max over cells of (|u_d| + c), dt = cfl / sum_d (A_d / dx_d),
 * written to the device scalar *dt_device (and kept in the workspace). */
int teno_cfl_dt(const teno_params *p, const double *U, double cfl, double *dt_device,
                void *ws, size_t ws_bytes, void *stream);

/* Synchronise the stream, read and clear the workspace's non-physical
 * counter (cells with rho <= 0, p <= 0 or non-finite values in a state whose
 * RHS was evaluated, plus faces with a non-positive Roe sound speed squared).
 * Returns TENO_ENONPHYSICAL if the count was non-zero, else TENO_OK. */
int teno_status(void *ws, void *stream, int64_t *nonphysical);

/* End-to-end call on HOST memory: copy U_host (ncons * ncells doubles) to the
 * device buffer U_dev, advance nsteps SSP-RK3 steps, each with dt from
 * teno_cfl_dt(cfl) computed on the device, copy the state back to U_host and
 * the summed time to *t_host, then synchronise the stream. */
int teno_advance_host(const teno_params *p, double *U_host, double *U_dev, int nsteps,
                      double cfl, double *t_host, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Batched mode: many independent 1D problems of uneven size advanced together.
 * Each problem is a 1D Euler grid with its own size, spacing, scheme width,
 * limiter switch and boundary rules, and its own CFL time step per step (the
 * per-problem reduction of teno_cfl_dt).  The shared parameters (gamma, C_T
 * parameters, flux splitting) come from a teno_params template with ndim 1.
 * ------------------------------------------------------------------------ */
typedef struct teno_batch_problem {
    int64_t n;             /* cells (>= scheme/2)                               */
    int64_t offset;        /* first double of this problem's state inside the
                              packed array; its state there is [3][n] SoA
                              (rho, rho*u, E); offsets 16-byte aligned, state
                              blocks must not overlap                          */
    double dx;             /* spacing (> 0)                                     */
    int32_t scheme;        /* 8 or 10 (12 is rejected in batched mode)          */
    int32_t limiter;       /* 0 or 1 (positivity-preserving limiter, Sec. 5.3) */
    int32_t bc_lo, bc_hi;  /* TENO_BC_* at the two ends, not TENO_BC_DIRICHLET  */
} teno_batch_problem;

typedef struct teno_batch teno_batch;   /* opaque host-side plan */

/* How teno_batch_rk3_steps launches one step. */
#define TENO_BATCH_GRAPH 0        /* persistent kernels over the (problem, tile)
                                     work list, the step captured once in a CUDA
                                     graph and replayed                         */
#define TENO_BATCH_STREAM 1       /* the same persistent kernels, launched
                                     directly                                   */
#define TENO_BATCH_PER_PROBLEM 2  /* reference: teno_cfl_dt + teno_rk3_step for
                                     each problem in turn                       */

/* Build the plan (work lists, per-problem descriptors) on the host.  The plan
 * owns host memory only (and, once a graph step runs, a CUDA graph and a
 * capture stream); release it with teno_batch_destroy. */
int teno_batch_create(const teno_params *common, const teno_batch_problem *probs,
                      int32_t nprob, teno_batch **out);

/* Device workspace bytes for this plan (status, per-problem slots, work lists,
 * face-flux buffers, stage buffer, and the largest per-problem workspace of
 * TENO_BATCH_PER_PROBLEM). */
int teno_batch_workspace_bytes(const teno_batch *b, size_t *bytes);

/* Autotuner: times one step (TENO_BATCH_STREAM) of every candidate tile width
 * (64/128/256 faces, i.e. 2/4/8 warps per pencil tile) and persistent grid size
 * (1/2/3/4/6 blocks per SM) on U_scratch (advanced in place: pass a copy) and keeps
 * the fastest in the plan.  Results do not depend on the choice.
 * *chosen_tile and *chosen_blocks_per_sm (nullable) report it. */
int teno_batch_autotune(teno_batch *b, double *U_scratch, void *ws, size_t ws_bytes,
                        void *stream, int32_t *chosen_tile, int32_t *chosen_blocks_per_sm);

/* Advance every problem nsteps SSP-RK3 steps, each problem with its own
 * dt = cfl / (A / dx) from its own state (Sec. 5), on the packed device state
 * U.  mode: TENO_BATCH_GRAPH, TENO_BATCH_STREAM or TENO_BATCH_PER_PROBLEM; all
 * three give bitwise identical states. */
int teno_batch_rk3_steps(teno_batch *b, double *U, int32_t nsteps, double cfl, int32_t mode,
                         void *ws, size_t ws_bytes, void *stream);

/* Synchronise and copy each problem's accumulated time (sum of its dt since
 * the workspace was first used by a persistent-mode step) to t_host[nprob]. */
int teno_batch_times(const teno_batch *b, void *ws, void *stream, double *t_host);

void teno_batch_destroy(teno_batch *b);

/* ------------------------------------------------------------------------
 * Adjoint (pattern: differentiation).  With the forward's discrete decisions
 * frozen -- stencil selection and cut-offs per face, field and sign (the
 * decision record of teno_flags_bytes), the cell maximising each splitting
 * speed -- the TENO-AA reconstruction (Sec. 3.3) is a fixed linear scheme and
 * L(U) is differentiable.  These calls apply the transposed Jacobian.  The
 * positivity limiter is not differentiated: p->limiter must be 0.
 * ------------------------------------------------------------------------ */

/* Workspace bytes for teno_rhs_vjp / teno_rk3_step_vjp (device, 256-byte
 * aligned). */
int teno_adjoint_workspace_bytes(const teno_params *p, size_t *bytes);

/* mu = (dL/dU)^T lam at the state U (Eq. approximateEq differentiated).
 *   U, lam, mu  device, ncons * ncells doubles; mu must not alias U or lam
 *   flags       the decision record of L(U) (teno_rhs with flags), or NULL to
 *               have it recomputed into the workspace first
 * Deterministic: every cell gathers its contributions in a fixed order. */
int teno_rhs_vjp(const teno_params *p, const double *U, const double *lam, const uint8_t *flags,
                 double *mu, void *ws, size_t ws_bytes, void *stream);

/* teno_rk3_step with the stages kept for the adjoint: U (in: U^n, out:
 * U^{n+1}), U1 and U2 receive the first two stage states and flags (3 x
 * teno_flags_bytes) the decision records of the three RHS evaluations.
 * Bitwise the same U^{n+1} as teno_rk3_step with the host dt.  ws is a
 * forward workspace (teno_workspace_bytes). */
int teno_rk3_step_record(const teno_params *p, double *U, double dt, double *U1, double *U2,
                         uint8_t *flags, void *ws, size_t ws_bytes, void *stream);

/* teno_rk3_step_record with a selection-only record: the same U^{n+1}, U1,
 * U2, argmax words and limiter bytes, and decision bytes whose selection and
 * cut-off bits (0-4) are those of the full record, while the C_T exponent
 * bits (5-7) are set only where the exponent was needed to decide and are 0
 * where the certified filter accepted S_p for every exponent the parameters
 * allow (it then skips the eta measure of Sec. 3.4).  The adjoint calls read
 * bits 0-4 and the argmax words only, so this record serves them at the
 * cost of a plain step; rollout() records with it. */
int teno_rk3_step_record_sel(const teno_params *p, double *U, double dt, double *U1, double *U2,
                             uint8_t *flags, void *ws, size_t ws_bytes, void *stream);

/* The frozen-decision map whose derivative the adjoint applies: L(U) (and one
 * SSP-RK3 step) with every reconstruction taken from the recorded decision
 * bytes (one teno_flags_bytes block for teno_rhs_frozen; three, one per
 * stage, for teno_rk3_step_frozen) instead of the smoothness indicators.
 * With the decisions U itself produces, the result equals teno_rhs /
 * teno_rk3_step up to rounding.  ws is a forward workspace. */
int teno_rhs_frozen(const teno_params *p, const double *U, double *rhs, double dt_limiter,
                    const uint8_t *decisions, void *ws, size_t ws_bytes, void *stream);
int teno_rk3_step_frozen(const teno_params *p, double *U, double dt, const uint8_t *decisions,
                         void *ws, size_t ws_bytes, void *stream);

/* Reverse of one SSP-RK3 step (Eq. Runge-kutta) at fixed dt: abar holds the
 * adjoint of U^{n+1} on entry and that of U^n on return.  Un, U1, U2, flags as
 * written by teno_rk3_step_record for that step. */
int teno_rk3_step_vjp(const teno_params *p, const double *Un, const double *U1, const double *U2,
                      const uint8_t *flags, double dt, double *abar, void *ws, size_t ws_bytes,
                      void *stream);

/* ------------------------------------------------------------------------
 * Domain decomposition (sub-domains exchanging halo planes).  A grid split
 * into slabs along an axis is advanced slab by slab: each slab is a
 * teno_params with TENO_BC_HALO on its inner sides, and the caller fills the
 * halo arrays from the neighbouring slabs' states before every evaluation
 * (a device copy on one GPU; a send / receive between GPUs).  Each slab
 * computes its boundary faces from the same stencil cells as the undivided
 * grid, so the slabs' states equal the undivided grid's bit for bit.
 * ------------------------------------------------------------------------ */

/* One stage of the SSP-RK3 step (Eq. Runge-kutta) of teno_rk3_step, so that
 * halos can be exchanged between stages: stage 1 reads U and writes
 * Us = U + dt L(U); stage 2 overwrites Us with 3/4 U + 1/4 (Us + dt L(Us));
 * stage 3 writes U = 1/3 U + 2/3 (Us + dt L(Us)).  The stage input (U, then
 * Us) is the state whose halo the caller provides.  Us: device, ncons *
 * ncells doubles, caller-owned, not aliasing U.  dt from dt_device when not
 * NULL, else the host dt.  The workspace carries the primitives of each
 * stage's output into the next stage: call stages 1, 2, 3 in order on the
 * same U, Us and ws, changing neither U nor Us in between (the halo arrays
 * may change).  The three stages give bitwise teno_rk3_step. */
int teno_rk3_stage(const teno_params *p, int stage, double *U, double *Us, double dt,
                   const double *dt_device, void *ws, size_t ws_bytes, void *stream);

/* The wave-speed maxima A_d = max over the interior cells of (|u_d| + c),
 * d < ndim, written as doubles to amax_device[0 .. ndim-1] (device memory,
 * 8-byte aligned): the per-sub-domain part of teno_cfl_dt. */
int teno_wave_speeds(const teno_params *p, const double *U, double *amax_device, void *ws,
                     size_t ws_bytes, void *stream);

/* dt = cfl / sum_d (A_d / dx_d) with A_d the largest of ncopies rows of
 * maxima amax_device[k * 3 + d] (k < ncopies, d < ndim; e.g. one row per
 * sub-domain, or one row already reduced across GPUs), written to the device
 * scalar *dt_device; bitwise the dt teno_cfl_dt gives for the whole grid. */
int teno_dt_from_speeds(const teno_params *p, const double *amax_device, int32_t ncopies,
                        double cfl, double *dt_device, void *stream);

/* Size of the device array behind teno_rhs_static: 16 MiB. */
#define TENO_RHS_STATIC_SCRATCH_BYTES (16u << 20)

/* teno_rhs without a workspace, for callers that cannot allocate device
 * memory where they need a right-hand side (plugin code inside an
 * application that owns the device memory pool, code with a memory budget
 * fixed at start-up, code that must not call cudaMalloc while a CUDA graph
 * is captured).  The paper has no counterpart; this is an integration aid.
 *   Same arguments and result as teno_rhs, minus ws / ws_bytes.  Scratch is
 *   one file-scope device array of TENO_RHS_STATIC_SCRATCH_BYTES, present on
 *   every GPU where the library's kernels are loaded until the process exits.
 *   Problems whose status header plus face-flux buffers (256 bytes + 8 *
 *   ncons * sum over directions of the face-grid size, each part rounded up
 *   to 256 bytes) exceed it are rejected with TENO_EINVAL before anything is
 *   enqueued.  Allocates nothing (no cudaMalloc / cudaFree).
 *   The first call on a device resolves the array's device address (one
 *   cudaGetSymbolAddress with that device current); make that first call
 *   before any stream capture.  The address is kept per device together with
 *   the id of the context it came from and resolved again when another
 *   context is current (after cudaDeviceReset, which unloads the array with
 *   the context), so that first-call rule applies again after a reset.
 *   All calls share the one array and each zeroes its status header: calls
 *   whose work overlaps on the GPU (different streams, or different host
 *   threads without ordering) race on it and must be serialised by the
 *   caller.  The non-physical counter is not reported (teno_status needs a
 *   workspace). */
int teno_rhs_static(const teno_params *p, const double *U, double *rhs, double dt_limiter,
                    uint8_t *flags, void *stream);

/* The scalar TENO-AA reconstruction at face i+1/2 (Sec. 3.2-3.4, Sec. 4.2 and
 * 4.3) of caller-provided stencils, e.g. split characteristic fluxes:
 *   v      device, count * scheme doubles; stencil i holds v[i*scheme + m] at
 *          offset m - scheme/2 + 1 from the upwind cell (m = 0 .. scheme-1)
 *   out    device, count doubles: the reconstructed face values
 *   flags  device, count bytes (nullable): the decision byte of each stencil
 *          (layout of teno_flags_bytes part 1)
 * Uses p->scheme and the C_T / epsilon parameters only. */
int teno_reconstruct(const teno_params *p, const double *v, int64_t count, double *out,
                     uint8_t *flags, void *stream);

/* Process-wide switch of the certified decision filter (default on): 1 lets
 * the face kernels decide the common case "largest stencil accepted" in
 * single precision with rigorous error bounds, falling back to the full FP64
 * evaluation whenever the bounds leave the decision open; 0 always evaluates
 * the decisions in FP64.  Results are identical either way (the filter only
 * answers when its answer equals the FP64 one); the switch exists to test
 * and time that.  The filter's error bounds carry the epsilons of Sec. 3.2
 * and Sec. 3.4 explicitly and are valid for eps_beta and eps_eta in
 * [0, 1e-40] (the paper's value is 1e-40): with a larger epsilon every
 * decision is evaluated in FP64 whatever the switch says.  Not thread-safe
 * with concurrent launches. */
int teno_set_decision_filter(int on);

/* Live timing of the dominant kernel (the face-sweep kernel) for roofline
 * reporting.  teno_profile_enable(1) clears the record and from then on
 * brackets every face-sweep launch with a pair of CUDA events recorded on
 * the launch's stream (at most 8192 launches are recorded); (0) stops.
 * teno_profile_read synchronises the recorded events and returns the summed
 * device milliseconds, the number of launches, the number of faces they
 * computed and how many of their reconstructions took the exact FP64 path
 * (the rest were decided by the single-precision filter; each face has
 * 2 (ndim + 2) reconstructions).  Any output pointer may be NULL.
 * teno_profile_enable(1) allocates an 8-byte device counter once (kept
 * until the context ends) and synchronises the device.  Not safe to call concurrently from
 * several host threads.  The paper has no counterpart: this is measurement
 * support. */
int teno_profile_enable(int on);
int teno_profile_read(double *ms, int64_t *launches, int64_t *faces, int64_t *exact_recons);

/* Bounds-checked build (libteno_gb300_debug.so, compiled with
 * -DTENO_DEBUG_BOUNDS; the same entry points): every global-memory index of
 * the face sweeps, the combine and the primitives kernel, and the sweeps'
 * shared-memory queue indices, are range-checked on the device; an index
 * outside its array is counted in the workspace's status block and the
 * access is skipped or redirected to an element inside the array (a load
 * gives 0), never faulting.  teno_debug_bounds synchronises the stream,
 * reads and clears that record: the number of such accesses, and the first
 * one's source line, index and array extent (any pointer may be NULL).
 * Returns TENO_EBOUNDS if there were any, else TENO_OK (always TENO_OK in the
 * release build, which has no checks).  teno_build_flags: bit 0 set in the
 * bounds-checked build.  The paper has no counterpart: these are test
 * support. */
int teno_debug_bounds(void *ws, void *stream, int64_t *count, int64_t *line, int64_t *index,
                      int64_t *extent);
int teno_build_flags(void);

/* Human-readable text of a return code (static storage). */
const char *teno_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TENO_H */
