/*
 * trotter.h -- C ABI of libtrotter.so: the second-order Trotter-Suzuki time
 * step of one particle on a 2-D lattice, as hand-written CUDA for sm_103a.
 *
 * The method (Wittek & Cucchietti, "A Second-Order Distributed
 * Trotter-Suzuki Solver with a Hybrid Kernel", Sec. 2): the tight-binding
 * Hamiltonian H = H0 + H1 + H2 per dimension (diagonal potential, even and
 * odd 2x2 hopping blocks); exp(-i H dt) is approximated by the symmetric
 * product U2(dt) = U1^T(dt) U1(dt) (Eq. secondorder).  One step applies the
 * pair rotations  a' = cos(theta) a + i sin(theta) b,
 *                 b' = i sin(theta) a + cos(theta) b
 * (the block exponential M of Sec. 2 with hopping -J and theta = J dt / 2)
 * over X-even, X-odd, Y-even, Y-odd neighbour pairs, then the diagonal phase
 * exp(-i V dt), then the four sweeps in reverse order.  Open boundaries: a
 * site without a partner is left unchanged.  hbar = 1, lattice spacing 1.
 *
 * Conventions shared by every call:
 *  - Dense host or device arrays are row-major, nx*ny elements, site (x, y)
 *    at index y*nx + x; x is the contiguous axis.
 *  - On the device a grid keeps separate real and imaginary planes with a
 *    row pitch of ts_grid_layout()'s `pitch` elements (a multiple of 32).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls marked "async" only enqueue work; errors of enqueued
 *    kernels surface at the next call marked "syncs".
 *  - No call throws, exits or aborts.  Every call returns a ts_status; on an
 *    error ts_last_error() returns a message (thread-local, valid until the
 *    calling thread's next call).
 *  - A grid handle is not thread-safe: use one handle from one thread at a
 *    time.  Distinct handles are independent.
 *  - Ownership: the caller owns every buffer it passes in (host arrays and a
 *    caller-supplied device slab); the library never frees caller memory.
 */
#ifndef TROTTER_H
#define TROTTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TS_OK = 0,
    TS_ERR_ARG = -1,          /* invalid argument (null pointer, bad size, ...) */
    TS_ERR_OOM = -2,          /* device allocation failed or budget exceeded     */
    TS_ERR_CUDA = -3,         /* a CUDA runtime call failed                      */
    TS_ERR_BUSY = -4,         /* request can never fit the configured budget     */
    TS_ERR_TIMEOUT = -5,      /* a bounded device or host wait gave up           */
    TS_ERR_STATE = -6,        /* call not valid in the handle's current state    */
    TS_ERR_UNSUPPORTED = -7   /* combination not implemented (e.g. dtype/path)   */
} ts_status;

typedef enum { TS_F32 = 0, TS_F64 = 1 } ts_dtype;
typedef enum { TS_HOST = 0, TS_DEVICE = 1 } ts_mem;

typedef struct ts_grid ts_grid;

/* Device layout of a grid: all planes live in one slab.
 *   pitch        row pitch of every plane, in elements (multiple of 32)
 *   plane_bytes  bytes per plane (multiple of 256)
 *   slab_bytes   total bytes: 7 planes (re, im, ping-pong re, im, the two
 *                potential-phase tables, V) plus reduction scratch
 *   nz           slabs of a 3-D grid (1 for a 2-D grid); slab z holds rows
 *                z*ny .. z*ny + ny - 1 of every plane. */
typedef struct {
    int64_t nx, ny, pitch;
    size_t plane_bytes, slab_bytes;
    ts_dtype dtype;
    int64_t nz;
} ts_layout;

/* Compute the layout of an nx x ny grid of `dtype` without allocating.
 * Errors: TS_ERR_ARG if nx or ny < 1, nx or ny > 2^20, or out == NULL. */
ts_status ts_grid_layout(int64_t nx, int64_t ny, ts_dtype dtype, ts_layout *out);

/* Three-dimensional lattices (Sec. 2's splitting with two hopping terms per
 * dimension, extended to z as Sec. 6 proposes).  Site (x, y, z) of a dense
 * array is at (z*ny + y)*nx + x; every call that takes or returns dense
 * arrays (state, V) then uses nx*ny*nz elements.  One step applies X-even,
 * X-odd, Y-even, Y-odd, Z-even, Z-odd, exp(-i V dt), then the mirror order.
 * ts_evolve runs, for FP32 grids with |theta| <= pi/4, one fused launch and
 * one pass over HBM per step (the slabs' rows take the Z sweeps as they
 * enter and leave the 2-D step, traded between neighbouring slabs; K is
 * ignored); otherwise, and for ts_evolve_plain, one kernel per sweep.
 * ts_observe adds <z>, <z^2> and the z bonds.  3-D grids take order 2 only,
 * no drive, no adjoint, and ts_evolve_batched evolves them one by one.
 * Errors: as for 2-D, and TS_ERR_ARG if ny * nz > 2^30. */
ts_status ts_grid_layout3(int64_t nx, int64_t ny, int64_t nz, ts_dtype dtype, ts_layout *out);
ts_status ts_create_grid3(int64_t nx, int64_t ny, int64_t nz, ts_dtype dtype, void *slab,
                          size_t slab_bytes, ts_grid **out);

/* Create a grid handle.  `slab` is a device pointer of at least
 * ts_grid_layout().slab_bytes bytes, 256-byte aligned, owned by the caller
 * (e.g. a torch tensor); pass NULL to have the library cudaMalloc (and later
 * free) its own slab.  The grid lives on the slab's device, which becomes the
 * calling thread's current device.  The state starts at zero and the potential at V = 0
 * with dt = theta = 0 (identity step) until ts_set_potential is called.
 * Errors: TS_ERR_ARG (sizes, alignment, slab too small), TS_ERR_OOM,
 * TS_ERR_CUDA.  Syncs the device (allocation and zero-fill). */
ts_status ts_create_grid(int64_t nx, int64_t ny, ts_dtype dtype, void *slab,
                         size_t slab_bytes, ts_grid **out);

/* Destroy a handle; frees only what the library allocated.  NULL is OK. */
ts_status ts_destroy_grid(ts_grid *g);

/* Query: the layout and the device pointers of the CURRENT state planes
 * (they swap between the two ping-pong pairs as the fused path runs). */
ts_status ts_grid_info(const ts_grid *g, ts_layout *layout, void **re, void **im);

/* Set the state psi from dense arrays of `src_dtype` in host or device
 * memory (nx*ny elements each).  FP64 input to an FP32 grid is rounded once
 * to nearest on the device.  Host input is staged through the grid's own
 * ping-pong planes, so no extra device memory is used.  Async for device
 * input; for host input the copies are issued on `stream` and the call
 * returns once they have landed (the host buffer may then be reused), while
 * any conversion kernel stays queued on `stream`.  Work on the grid that
 * follows on another stream must be ordered after it by the caller. */
ts_status ts_set_state(ts_grid *g, const void *re, const void *im,
                       ts_dtype src_dtype, ts_mem where, void *stream);

/* Read the state into dense arrays of `dst_dtype` (host or device).  Syncs
 * `stream`; reports TS_ERR_TIMEOUT if a bounded wait inside an earlier fused
 * launch gave up, TS_ERR_CUDA for a failed earlier launch. */
ts_status ts_get_state(ts_grid *g, void *re, void *im, ts_dtype dst_dtype,
                       ts_mem where, void *stream);

/* Table preparation (Sec. 2: the external potential is one diagonal factor
 * exp(-i V dt) per step).  V: dense FP64 array of nx*ny potential values in
 * host or device memory, or NULL for V = 0.  dt: the time step; theta: the
 * kinetic half-step angle J*dt/2 (hopping J = 2 theta / dt).  On the device
 * the per-site table (gamma_V = 1 - cos(V dt), s_V = sin(V dt)) is computed
 * to FP64 accuracy (FP64 for FP64 grids; double-float arithmetic for FP32
 * grids, within one ulp of the FP64 value rounded) and rounded once to the
 * grid's dtype.  The kinetic coefficients (1 - cos theta, sin theta,
 * tan(theta/2), and those of 2 theta for merged sweeps) are computed in
 * FP64 on the host and rounded once.  Async; with host V the call returns
 * once V has been copied to the device (V may then be reused) and the table
 * kernels stay queued on `stream`. */
ts_status ts_set_potential(ts_grid *g, const double *V, ts_mem where, double dt,
                           double theta, void *stream);

/* The same, choosing the order of the step that ts_evolve and
 * ts_evolve_plain apply (Sec. 2).  order 2: U2(dt), exactly ts_set_potential.
 * order 4: the fourth-order Suzuki step (Eq. fourthorder)
 *     U4(dt) = U2(p dt) U2(p dt) U2((1-4p) dt) U2(p dt) U2(p dt),
 *     p = 1 / (4 - 4^(1/3)),
 * where each substep U2(w dt) uses the kinetic angle w theta and the phase
 * exp(-i V w dt) (w = 1 - 4p is negative: that substep runs backwards).  The
 * grid's phase planes then hold the table at p dt, and a second table at
 * (1-4p) dt (two planes of ts_layout.plane_bytes) is cudaMalloc'd by the
 * library on the first order-4 call and freed by ts_destroy_grid, also for
 * grids on a caller-provided slab.  Fourth-order grids are evolved one by one
 * by ts_evolve_batched and are refused by the adjoint calls
 * (TS_ERR_UNSUPPORTED).  Errors: TS_ERR_ARG (order not 2 or 4, non-finite dt
 * or theta), TS_ERR_OOM (the second table), TS_ERR_CUDA. */
ts_status ts_set_potential_order(ts_grid *g, const double *V, ts_mem where, double dt,
                                 double theta, int order, void *stream);

/* Time-dependent potential (Sec. 2 writes the Schroedinger equation with a
 * time-dependent H(t); the time-dependent form of the method is an
 * extension of the time-independent one the paper details):
 *     V(x, y, t) = V0(x, y) + a(t) V1(x, y).
 * V0, dt and theta are those of the last ts_set_potential, which must come
 * first (and a later ts_set_potential or ts_set_potential_order ends the
 * drive).  V1: dense FP64 array of nx*ny values in host or device memory,
 * or NULL (zero); stored in the grid's dtype.  a: host array of n_a
 * amplitudes, copied; the n-th step evolved after this call uses a[n] in
 * its phase exp(-i (V0 + a[n] V1) dt).  Sampling a(t) at the middle of
 * each step, a[n] = a((n + 1/2) dt) from the time the drive starts, keeps
 * the step second order in time.  ts_evolve and ts_evolve_plain then fail
 * with TS_ERR_ARG, before launching anything, if they are asked for more
 * steps than amplitudes are left.  The drive phase exp(-i a[n] dt V1) is
 * computed on the device per site and step (no table); the fused path runs
 * at depth <= 4 (K = 0: 4).  Needs three more planes of ts_layout.plane_bytes,
 * cudaMalloc'd by the library on first use and freed by ts_destroy_grid.
 * ts_observe's e_pot is sum V0 |psi|^2 (without the drive term).  Driven
 * grids are evolved one by one by ts_evolve_batched and refused by the
 * adjoint calls.  Errors: TS_ERR_ARG (NULL grid, bad or non-finite a),
 * TS_ERR_UNSUPPORTED (grid set to order 4), TS_ERR_OOM, TS_ERR_CUDA.
 * Async for device V1 (host V1: returns when it may be reused). */
ts_status ts_set_drive(ts_grid *g, const double *V1, ts_mem where, const double *a,
                       int64_t n_a, void *stream);

/* End the drive: later steps use V0 alone.  The drive planes stay
 * allocated until ts_destroy_grid. */
ts_status ts_clear_drive(ts_grid *g);

/* Evolve `steps` second-order steps (Eq. secondorder) on the grid's current
 * state.  FP32 grids run the fused kernel: K whole steps per HBM round trip
 * on TMA-staged shared-memory tiles (temporal blocking; K = 0 picks the
 * depth automatically, 1 <= K <= 8 forces it; a remainder of steps % K runs
 * at a smaller depth).  FP64 grids run one sweep per launch (K must be 0,
 * else TS_ERR_UNSUPPORTED), with the sweeps of one axis merged where two
 * steps or substeps meet (X, Y and Z factors commute; two factors of one
 * family add their angles: n second-order steps take 6n + 2 sweeps in 2-D,
 * 9n + 3 in 3-D) and the lifting form for angles up to pi/2; the results
 * agree with ts_evolve_plain to FP64 rounding.  On a grid set to order 4
 * (ts_set_potential_order) each step is U4(dt): on FP32 grids with K = 0
 * each step is one launch that applies all five
 * substeps; with K >= 1 the p dt substeps of neighbouring steps run as
 * fused launches of depth at most K and each (1-4p) dt substep as a
 * depth-1 launch.  Async. */
ts_status ts_evolve(ts_grid *g, int64_t steps, int K, void *stream);

/* The plain path: one kernel per sweep (8 sweeps + the phase = 9 launches
 * per step), in place, for FP32 or FP64 grids.  The reference point the
 * fused path is measured against.  Async. */
ts_status ts_evolve_plain(ts_grid *g, int64_t steps, void *stream);

/* Check of the failure path of the bounded device waits.  Every mbarrier
 * wait in the fused kernels gives up after a time limit (2 s), sets a bit in
 * the grid's error word and returns, so a TMA copy that never lands is
 * reported instead of hanging the GPU.  This call enqueues one warp that runs
 * the same bounded wait on an mbarrier nothing completes (no copy in
 * flight), for limit_ns nanoseconds, and sets the same bit in g's error
 * word.  The grid's state and tables are not touched.  The next syncing
 * call on g (ts_get_state, ts_observe, ts_norm, ...) then returns
 * TS_ERR_TIMEOUT and clears the word; later calls work as before.
 * Errors: TS_ERR_ARG (NULL grid, limit_ns outside [1e3, 2e9]), TS_ERR_CUDA.
 * Async. */
ts_status ts_check_wait_timeout(ts_grid *g, int64_t limit_ns, void *stream);

/* Observables of the current state, reduced on the device with FP64
 * compensated (Neumaier) partial sums, finished on the device, copied back.
 * Syncs `stream`. */
typedef struct {
    double norm;        /* sum |psi|^2 (Sec. 2: conserved by the unitary U) */
    double x, y;        /* <x>, <y> = sum x|psi|^2 / norm, ...               */
    double x2, y2;      /* <x^2>, <y^2>                                      */
    double e_kin;       /* -J sum over neighbour pairs 2 Re(conj(psi_j) psi_k) */
    double e_pot;       /* sum V |psi|^2                                     */
    double z, z2;       /* <z>, <z^2> (3-D grids; 0 for 2-D grids)           */
} ts_observables;

ts_status ts_observe(ts_grid *g, ts_observables *out, void *stream);
ts_status ts_norm(ts_grid *g, double *out, void *stream);
ts_status ts_expect_xy(ts_grid *g, double *x, double *y, void *stream);
ts_status ts_energy(ts_grid *g, double *out, void *stream);   /* e_kin + e_pot */

/* Evolve n independent grids (steps[i] steps each, fused depth K as in
 * ts_evolve) on one stream.  Second-order 2-D FP32 grids with |theta| <=
 * pi/4 and no drive advance together in multi-grid launches of the fused
 * kernel; every other grid runs ts_evolve on its own (FP64 grids with K = 0,
 * whatever K is given).  Errors: TS_ERR_ARG (n < 0, NULL arrays, a NULL grid
 * or negative steps), then those of ts_evolve.  Async. */
ts_status ts_evolve_batched(ts_grid *const *g, int n, const int64_t *steps, int K,
                            void *stream);

/* Adjoint: gradient of the fidelity F = |<phi|psi_T>|^2 with respect to the
 * potential V on every site, where psi_T = U2(dt)^steps psi_0 evolves the
 * grid's current state with its current potential, dt and theta.
 * Write a step as psi_s = B P A psi_{s-1} (A, B: the first and last four
 * sweeps, P = exp(-i V dt)); with c = <phi|psi_T>, lambda_T = phi,
 * lambda_{s-1} = U_s^dagger lambda_s and m_s = P A psi_{s-1}:
 *   dF/dV_j = 2 dt Im( conj(c) sum_s conj((B^dagger lambda_s)[j]) m_s[j] ).
 * U^dagger is the step at -theta with the conjugate phase; the backward pass
 * runs it as a hand-written kernel on lambda and on psi together (m_s is
 * B^dagger psi_s), restarting psi from a checkpoint at the end of each
 * segment of `ckpt_every` steps.  FP32 grids, |theta| <= pi/4.
 *
 * ts_adjoint_workspace: bytes of device workspace for (steps, ckpt_every):
 *   about (14 + 2 ceil(steps/ckpt)) planes of the grid.
 * ts_adjoint_forward: target phi as dense arrays (host or device, FP32 or
 *   FP64); evolves the grid's state by `steps` (the grid then holds psi_T),
 *   keeps checkpoints in `ws` (caller-owned, 256-byte aligned), returns F
 *   (and c = overlap[0] + i overlap[1] if overlap != NULL).  Syncs.
 * ts_adjoint_backward: after a forward with the same ws, writes dF/dV as a
 *   dense nx*ny FP32 device array `grad`.  Syncs.  One forward/backward pair
 *   per grid at a time; TS_ERR_STATE without a matching forward.
 *   psi and lambda step back together, K steps per fused launch (K = 3).
 * ts_adjoint_backward_depth: the same with the depth K of those launches
 *   given (1..4; 0 = the default); other K return TS_ERR_ARG.  K changes only
 *   the order in which G's terms are summed, not the gradient it defines.
 * ts_adjoint_grad: forward then backward. */
ts_status ts_adjoint_workspace(const ts_grid *g, int64_t steps, int64_t ckpt_every,
                               size_t *bytes);
ts_status ts_adjoint_forward(ts_grid *g, const void *target_re, const void *target_im,
                             ts_dtype target_dtype, ts_mem where, int64_t steps,
                             int64_t ckpt_every, void *ws, size_t ws_bytes, double *fidelity,
                             double *overlap, void *stream);
ts_status ts_adjoint_backward(ts_grid *g, void *ws, size_t ws_bytes, float *grad, void *stream);
ts_status ts_adjoint_backward_depth(ts_grid *g, void *ws, size_t ws_bytes, int K, float *grad,
                                    void *stream);
ts_status ts_adjoint_grad(ts_grid *g, const void *target_re, const void *target_im,
                          ts_dtype target_dtype, ts_mem where, int64_t steps, int64_t ckpt_every,
                          void *ws, size_t ws_bytes, float *grad, double *fidelity, void *stream);

/* Serving: a continuous-batching request loop inside the library.
 *
 * Each request is one evolution: an nx x ny FP32 grid, a potential V, an
 * initial state, dt, theta (|theta| <= pi/4) and a step count.  A scheduler
 * thread admits requests in arrival order while the device memory they hold
 * (ts_grid_layout's slab_bytes each, FP32) fits hbm_budget_bytes and fewer
 * than max_slots are admitted, uploads their inputs on a copy stream, and
 * advances all admitted grids together: each epoch runs up to
 * max_epoch_steps steps as launches of one persistent multi-grid kernel
 * (depth K), replayed from cached CUDA graphs, so requests that arrive while
 * others run join at the next epoch and their work overlaps on the GPU.  A
 * request's result does not depend on what it ran with.  Finished states
 * stay on the device until ts_server_release.
 *
 * Input buffers (V, psi) stay owned by the caller and must remain valid and
 * unchanged until the request is admitted and uploaded (simplest: until it
 * completes).  Pinned host memory keeps submission fully asynchronous;
 * pageable memory works but stalls the scheduler during its copies.
 * All calls are thread-safe. */
typedef struct {
    size_t hbm_budget_bytes;   /* device memory for admitted requests          */
    int max_slots;             /* admitted requests at a time (1..4096)        */
    int K;                     /* fused depth, 0 = default (4)                 */
    int max_epoch_steps;       /* steps per epoch before re-admission, 0 = 32  */
} ts_server_cfg;

typedef struct {
    int64_t nx, ny, steps;
    double dt, theta;
    const double *V;           /* nx*ny FP64, or NULL for V = 0                */
    const void *psi_re, *psi_im;   /* initial state, nx*ny of psi_dtype        */
    ts_dtype psi_dtype;
    ts_mem where;              /* memory kind of V and psi                     */
} ts_request;

typedef struct {
    int status;                /* TS_OK done, 1 pending or running, else ts_status */
    int64_t latency_ns;        /* submission to completion                     */
    int64_t queue_ns;          /* submission to admission                      */
    int64_t nx, ny, steps;
} ts_result;

typedef struct {
    int64_t submitted, completed, failed, active, pending;
    double p50_ms, p99_ms, mean_ms;   /* latency of completed requests          */
    double site_steps_per_s;   /* completed sites x steps / (last completion - first submission) */
    size_t bytes_in_use, peak_bytes;
    int64_t epochs, graph_launches;
} ts_server_metrics;

typedef struct ts_server ts_server;

ts_status ts_server_create(const ts_server_cfg *cfg, ts_server **out);
/* TS_ERR_BUSY if the request alone exceeds the budget (it could never run). */
ts_status ts_server_submit(ts_server *s, const ts_request *r, uint64_t *ticket);
ts_status ts_server_poll(ts_server *s, uint64_t ticket, ts_result *out);
/* Blocks up to timeout_ms (< 0: forever); TS_ERR_TIMEOUT if not done by then. */
ts_status ts_server_wait(ts_server *s, uint64_t ticket, int64_t timeout_ms, ts_result *out);
/* Copy a finished request's state out (dense, host or device).  Syncs. */
ts_status ts_server_fetch(ts_server *s, uint64_t ticket, void *re, void *im, ts_dtype dtype,
                          ts_mem where);
/* Free a finished, failed or cancelled request and its device memory. */
ts_status ts_server_release(ts_server *s, uint64_t ticket);
/* Pending requests leave at once; running ones at the next epoch boundary. */
ts_status ts_server_cancel(ts_server *s, uint64_t ticket);
ts_status ts_server_stats(ts_server *s, ts_server_metrics *out);
/* Cancels what is still queued or running, waits for the GPU, frees all. */
ts_status ts_server_destroy(ts_server *s);

/* Sum of |psi|^2 over a pitched device state, without allocating anything.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code that runs where the device memory is
 * already fully reserved by another allocator (a framework's caching pool,
 * a serving process with a fixed HBM budget), or a loop that must not take
 * the synchronising, latency-unbounded path of a fresh allocation.  It makes
 * no cudaMalloc/cudaFree call and calls no allocating library routine.
 *
 *   re, im  device planes of `dtype`, ny rows of `pitch` elements (pitch >= nx);
 *   out     device pointer to one double that receives the sum (caller-owned);
 *   stream  as elsewhere; the call is asynchronous.
 *
 * Scratch: the per-block partial sums live in one fixed array of
 * ts_norm_noalloc_scratch_bytes() bytes (57,344) inside the library's device
 * image; every GPU that loads the library holds it until the process exits.
 * The reduction uses at most 1024 blocks, so any grid with sides in [1, 2^20]
 * fits; other sides, pitch < nx, null pointers or an unknown dtype return
 * TS_ERR_ARG with a message in ts_last_error().
 * Alignment: FP32 planes are read 4 sites at a time with 16-byte loads, so
 * for TS_F32 re and im must be 16-byte aligned and pitch a multiple of 4;
 * for TS_F64 they must be 8-byte aligned.  Anything else returns TS_ERR_ARG
 * before any kernel runs.  Each plane must span ny * pitch elements (the
 * last row's padding included): the last 16-byte load of a row may read up
 * to 3 floats past column nx - 1, never past the row's pitch.
 * The first call on each device looks the array's device address up (with
 * that device current); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (on different
 * streams, or from different threads) race and must be serialised by the
 * caller.  Nothing in the array needs clearing between calls. */
ts_status ts_norm_noalloc(const void *re, const void *im, ts_dtype dtype, int64_t nx,
                          int64_t ny, int64_t pitch, double *out, void *stream);
size_t ts_norm_noalloc_scratch_bytes(void);

/* The fused depth ts_evolve uses when K = 0. */
int ts_fused_default_depth(void);

/* Number of kernels this thread's calls enqueued since the last reset. */
int64_t ts_launch_count(int reset);

const char *ts_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TROTTER_H */
