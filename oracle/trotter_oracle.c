/*
 * Plain FP64 CPU oracle for the second-order Trotter-Suzuki step of one
 * particle on a 2-D lattice (Wittek & Cucchietti, "A Second-Order Distributed
 * Trotter-Suzuki Solver with a Hybrid Kernel", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is
 * compared against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes: the ordered Trotter product itself (not exp(-iHt)),
 * factor by factor, in double precision, without blocking, fusion, sweep
 * merging or renormalisation.  Compile with -O2 -ffp-contract=off so that
 * its results do not depend on FMA contraction.
 *
 * Conventions (hbar = 1, lattice spacing a = 1):
 *   - the state is two dense planes re[], im[] of nx*ny doubles,
 *     site (x, y) at index y*nx + x; x is the contiguous ("horizontal") axis;
 *   - hopping element V_hop = -J (Sec. 2: tunnelling element -hbar^2/2ma^2),
 *     so the exponential of one 2x2 block over a half step dt/2 is the plane
 *     rotation  [[c, i s], [i s, c]]  with theta = J dt / 2, c = cos theta,
 *     s = sin theta  (Sec. 2, the matrix M; the sign of its off-diagonal
 *     follows from V_hop < 0);
 *   - "even" pairs are (x, x+1) with x = 0, 2, 4, ...  (the blocks of H1 in
 *     Sec. 2, counted from 0), "odd" pairs start at x = 1, 3, ... (blocks of
 *     H2).  Open boundaries: a site with no partner is left unchanged;
 *   - the onsite constant hbar^2/ma^2 of the diagonal H0 is a global phase
 *     and is dropped (Sec. 2, last paragraph, the flat-potential remark);
 *   - one second-order step (Eq. secondorder, U2 = U1^T U1, with the kinetic
 *     factors at half angle and the potential phase at the full step in the
 *     middle) applies, in this order:
 *       X-even, X-odd, Y-even, Y-odd, phase exp(-i V dt),
 *       Y-odd, Y-even, X-odd, X-even.
 *
 * Parity: pinned by the CPU tests in tests/test_oracle_*.py (dense matrix
 * exponentials of the H1/H2 blocks on tiny grids, exact propagator by dense
 * eigendecomposition with dt^2 error scaling, unitarity, reversibility,
 * separability, flat potential, free-packet closed forms, two-site chain,
 * finite differences of the fidelity).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_THREADS 256

/* ------------------------------------------------------------------------ */
/* A tiny fork/join helper: split [0, n) into contiguous chunks, one per     */
/* thread.  With nthreads <= 1 the body runs inline.                         */
/* ------------------------------------------------------------------------ */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);

typedef struct {
    range_fn fn;
    void *ctx;
    int64_t lo, hi;
} range_job;

static void *range_thread(void *arg)
{
    range_job *j = (range_job *)arg;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_range(int64_t n, int nthreads, range_fn fn, void *ctx)
{
    if (nthreads > ORACLE_MAX_THREADS) nthreads = ORACLE_MAX_THREADS;
    if (nthreads <= 1 || n < 2 * (int64_t)nthreads) {
        fn(ctx, 0, n);
        return;
    }
    pthread_t th[ORACLE_MAX_THREADS];
    range_job jobs[ORACLE_MAX_THREADS];
    int started[ORACLE_MAX_THREADS];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        started[t] = pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0;
        if (!started[t]) range_thread(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* The exponential of one 2x2 block of H1 or H2 (Sec. 2, matrix M):          */
/*   a' = c a + i s b,   b' = i s a + c b.                                   */
/* ------------------------------------------------------------------------ */
static void rotate_pair(double *re, double *im, int64_t j, int64_t k,
                        double c, double s)
{
    double ar = re[j], ai = im[j], br = re[k], bi = im[k];
    re[j] = c * ar - s * bi;
    im[j] = c * ai + s * br;
    re[k] = c * br - s * ai;
    im[k] = c * bi + s * ar;
}

typedef struct {
    int64_t nx, ny;
    double *re, *im;
    int parity;
    double c, s;
    const double *V;
    double dt;
} sweep_ctx;

/* Horizontal sweep: pairs (x, x+1) with x = parity, parity+2, ... in every
 * row y in [lo, hi). */
static void sweep_x_rows(void *vctx, int64_t lo, int64_t hi)
{
    sweep_ctx *q = (sweep_ctx *)vctx;
    for (int64_t y = lo; y < hi; ++y)
        for (int64_t x = q->parity; x + 1 < q->nx; x += 2)
            rotate_pair(q->re, q->im, y * q->nx + x, y * q->nx + x + 1,
                        q->c, q->s);
}

/* Vertical sweep: pairs (y, y+1) with y = parity + 2*p for p in [lo, hi),
 * every column. */
static void sweep_y_pairs(void *vctx, int64_t lo, int64_t hi)
{
    sweep_ctx *q = (sweep_ctx *)vctx;
    for (int64_t p = lo; p < hi; ++p) {
        int64_t y = q->parity + 2 * p;
        if (y + 1 >= q->ny) continue;
        for (int64_t x = 0; x < q->nx; ++x)
            rotate_pair(q->re, q->im, y * q->nx + x, (y + 1) * q->nx + x,
                        q->c, q->s);
    }
}

/* Diagonal factor exp(-i V dt) (Sec. 2: the external potential adds one
 * diagonal factor per step).  V == NULL means V = 0 (identity). */
static void phase_rows(void *vctx, int64_t lo, int64_t hi)
{
    sweep_ctx *q = (sweep_ctx *)vctx;
    if (!q->V) return;
    for (int64_t y = lo; y < hi; ++y)
        for (int64_t x = 0; x < q->nx; ++x) {
            int64_t i = y * q->nx + x;
            double ph = q->V[i] * q->dt;
            double c = cos(ph), s = sin(ph);
            double r = q->re[i], m = q->im[i];
            /* (r + i m)(c - i s) */
            q->re[i] = c * r + s * m;
            q->im[i] = c * m - s * r;
        }
}

/* Public single-factor entry points (used by the pins on tiny grids). */
void oracle_sweep_x(int64_t nx, int64_t ny, double *re, double *im,
                    int parity, double theta, int nthreads)
{
    sweep_ctx q = {nx, ny, re, im, parity & 1, cos(theta), sin(theta), NULL, 0};
    parallel_range(ny, nthreads, sweep_x_rows, &q);
}

void oracle_sweep_y(int64_t nx, int64_t ny, double *re, double *im,
                    int parity, double theta, int nthreads)
{
    sweep_ctx q = {nx, ny, re, im, parity & 1, cos(theta), sin(theta), NULL, 0};
    int64_t npairs = (ny - (parity & 1)) / 2;
    if (npairs < 0) npairs = 0;
    parallel_range(npairs, nthreads, sweep_y_pairs, &q);
}

void oracle_phase(int64_t nx, int64_t ny, double *re, double *im,
                  const double *V, double dt, int nthreads)
{
    sweep_ctx q = {nx, ny, re, im, 0, 0, 0, V, dt};
    parallel_range(ny, nthreads, phase_rows, &q);
}

/* One second-order step U2(dt) (Eq. secondorder), kinetic half angle theta. */
void oracle_step2(int64_t nx, int64_t ny, double *re, double *im,
                  const double *V, double dt, double theta, int nthreads)
{
    oracle_sweep_x(nx, ny, re, im, 0, theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 1, theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 0, theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 1, theta, nthreads);
    oracle_phase(nx, ny, re, im, V, dt, nthreads);
    oracle_sweep_y(nx, ny, re, im, 1, theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 0, theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 1, theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 0, theta, nthreads);
}

/* One first-order step U1(dt) (Sec. 2): every kinetic factor at the full
 * angle J dt = 2 theta, then the potential.  Used only to pin the order. */
void oracle_step1(int64_t nx, int64_t ny, double *re, double *im,
                  const double *V, double dt, double theta, int nthreads)
{
    oracle_sweep_x(nx, ny, re, im, 0, 2.0 * theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 1, 2.0 * theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 0, 2.0 * theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 1, 2.0 * theta, nthreads);
    oracle_phase(nx, ny, re, im, V, dt, nthreads);
}

/* One fourth-order step (Eq. fourthorder):
 *   U4(dt) = U2(p dt) U2(p dt) U2((1-4p) dt) U2(p dt) U2(p dt),
 *   p = 1 / (4 - 4^(1/3)).  theta scales with dt (theta = J dt / 2). */
void oracle_step4(int64_t nx, int64_t ny, double *re, double *im,
                  const double *V, double dt, double theta, int nthreads)
{
    double p = 1.0 / (4.0 - cbrt(4.0));
    double w[5] = {p, p, 1.0 - 4.0 * p, p, p};
    for (int i = 0; i < 5; ++i)
        oracle_step2(nx, ny, re, im, V, w[i] * dt, w[i] * theta, nthreads);
}

/* Evolve `steps` steps of the given order (1, 2 or 4). Returns 0 on success,
 * -1 on a bad argument. */
int oracle_evolve(int64_t nx, int64_t ny, double *re, double *im,
                  const double *V, double dt, double theta, int64_t steps,
                  int order, int nthreads)
{
    if (nx < 1 || ny < 1 || steps < 0 || !re || !im) return -1;
    for (int64_t n = 0; n < steps; ++n) {
        switch (order) {
        case 1: oracle_step1(nx, ny, re, im, V, dt, theta, nthreads); break;
        case 2: oracle_step2(nx, ny, re, im, V, dt, theta, nthreads); break;
        case 4: oracle_step4(nx, ny, re, im, V, dt, theta, nthreads); break;
        default: return -1;
        }
    }
    return 0;
}

/* Time-dependent potential.  Sec. 2 writes the Schroedinger equation with a
 * time-dependent H(t) and treats the time-independent case, noting that the
 * time-dependent form is a direct extension.  Here V(t) = V0 + a(t) V1: step
 * n is U2(dt) built with the potential V0 + a[n] V1, where the caller gives
 * a[n] (sampling a(t) at the middle of the step, t = (n + 1/2) dt, keeps the
 * step second order in time).  V0 or V1 may be NULL (zero).  Returns 0 on
 * success, -1 on a bad argument or allocation failure. */
int oracle_evolve_driven(int64_t nx, int64_t ny, double *re, double *im,
                         const double *V0, const double *V1, const double *a,
                         double dt, double theta, int64_t steps, int nthreads)
{
    if (nx < 1 || ny < 1 || steps < 0 || !re || !im || (steps > 0 && !a)) return -1;
    const int64_t n = nx * ny;
    double *Vn = (double *)malloc((size_t)n * sizeof(double));
    if (!Vn) return -1;
    for (int64_t s = 0; s < steps; ++s) {
        for (int64_t i = 0; i < n; ++i)
            Vn[i] = (V0 ? V0[i] : 0.0) + a[s] * (V1 ? V1[i] : 0.0);
        oracle_step2(nx, ny, re, im, Vn, dt, theta, nthreads);
    }
    free(Vn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Three dimensions (Sec. 2 splits H into the diagonal and two terms per     */
/* dimension; Sec. 6 names three-dimensional systems as the next step).      */
/* Site (x, y, z) is at index (z*ny + y)*nx + x.  One second-order step      */
/* applies X-even, X-odd, Y-even, Y-odd, Z-even, Z-odd, the phase, then the  */
/* mirror order, each kinetic factor at the half angle theta.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nx, ny, nz;
    double *re, *im;
    int parity;
    double c, s;
} sweep3_ctx;

/* axis x: rows r = z*ny + y in [lo, hi) */
static void sweep3_x(void *vctx, int64_t lo, int64_t hi)
{
    sweep3_ctx *q = (sweep3_ctx *)vctx;
    for (int64_t r = lo; r < hi; ++r)
        for (int64_t x = q->parity; x + 1 < q->nx; x += 2)
            rotate_pair(q->re, q->im, r * q->nx + x, r * q->nx + x + 1, q->c, q->s);
}

/* axis y: slabs z in [lo, hi), pairs (y, y+1) inside each slab */
static void sweep3_y(void *vctx, int64_t lo, int64_t hi)
{
    sweep3_ctx *q = (sweep3_ctx *)vctx;
    for (int64_t z = lo; z < hi; ++z)
        for (int64_t y = q->parity; y + 1 < q->ny; y += 2)
            for (int64_t x = 0; x < q->nx; ++x) {
                int64_t j = (z * q->ny + y) * q->nx + x;
                rotate_pair(q->re, q->im, j, j + q->nx, q->c, q->s);
            }
}

/* axis z: pairs (z, z+1) with z = parity + 2p for p in [lo, hi) */
static void sweep3_z(void *vctx, int64_t lo, int64_t hi)
{
    sweep3_ctx *q = (sweep3_ctx *)vctx;
    const int64_t plane = q->nx * q->ny;
    for (int64_t p = lo; p < hi; ++p) {
        int64_t z = q->parity + 2 * p;
        if (z + 1 >= q->nz) continue;
        for (int64_t i = 0; i < plane; ++i)
            rotate_pair(q->re, q->im, z * plane + i, (z + 1) * plane + i, q->c, q->s);
    }
}

/* One sweep along axis 0 (x), 1 (y) or 2 (z) of the given parity. */
void oracle_sweep3(int64_t nx, int64_t ny, int64_t nz, double *re, double *im, int axis,
                   int parity, double theta, int nthreads)
{
    sweep3_ctx q = {nx, ny, nz, re, im, parity & 1, cos(theta), sin(theta)};
    if (axis == 0) {
        parallel_range(ny * nz, nthreads, sweep3_x, &q);
    } else if (axis == 1) {
        parallel_range(nz, nthreads, sweep3_y, &q);
    } else {
        int64_t npairs = (nz - (parity & 1)) / 2;
        if (npairs > 0) parallel_range(npairs, nthreads, sweep3_z, &q);
    }
}

void oracle_step3(int64_t nx, int64_t ny, int64_t nz, double *re, double *im,
                  const double *V, double dt, double theta, int nthreads)
{
    for (int axis = 0; axis < 3; ++axis)
        for (int parity = 0; parity < 2; ++parity)
            oracle_sweep3(nx, ny, nz, re, im, axis, parity, theta, nthreads);
    oracle_phase(nx, ny * nz, re, im, V, dt, nthreads);
    for (int axis = 2; axis >= 0; --axis)
        for (int parity = 1; parity >= 0; --parity)
            oracle_sweep3(nx, ny, nz, re, im, axis, parity, theta, nthreads);
}

int oracle_evolve3(int64_t nx, int64_t ny, int64_t nz, double *re, double *im,
                   const double *V, double dt, double theta, int64_t steps, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1 || steps < 0 || !re || !im) return -1;
    for (int64_t n = 0; n < steps; ++n) oracle_step3(nx, ny, nz, re, im, V, dt, theta, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. 2: the norm <psi|psi> is conserved by the unitary U).    */
/* All sums use Neumaier's compensated summation.                            */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

static double nsum_val(const nsum *a) { return a->s + a->c; }

/* out[0] = sum |psi|^2, out[1] = sum x|psi|^2, out[2] = sum y|psi|^2,
 * out[3] = sum x^2|psi|^2, out[4] = sum y^2|psi|^2. */
void oracle_moments(int64_t nx, int64_t ny, const double *re,
                    const double *im, double *out)
{
    nsum a[5];
    memset(a, 0, sizeof(a));
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            double p = re[i] * re[i] + im[i] * im[i];
            nsum_add(&a[0], p);
            nsum_add(&a[1], (double)x * p);
            nsum_add(&a[2], (double)y * p);
            nsum_add(&a[3], (double)x * (double)x * p);
            nsum_add(&a[4], (double)y * (double)y * p);
        }
    for (int q = 0; q < 5; ++q) out[q] = nsum_val(&a[q]);
}

/* <psi|H|psi> for H = -J * sum over nearest-neighbour pairs (|j><k| + h.c.)
 * + diag(V)  (the tight-binding Hamiltonian of Sec. 2 without its onsite
 * constant).  V == NULL means V = 0.  out[0] = kinetic part, out[1] =
 * potential part. */
void oracle_energy(int64_t nx, int64_t ny, const double *re, const double *im,
                   const double *V, double J, double *out)
{
    nsum kin = {0, 0}, pot = {0, 0};
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t i = y * nx + x;
            if (x + 1 < nx) {
                int64_t k = i + 1;
                nsum_add(&kin, -2.0 * J * (re[i] * re[k] + im[i] * im[k]));
            }
            if (y + 1 < ny) {
                int64_t k = i + nx;
                nsum_add(&kin, -2.0 * J * (re[i] * re[k] + im[i] * im[k]));
            }
            if (V) nsum_add(&pot, V[i] * (re[i] * re[i] + im[i] * im[i]));
        }
    out[0] = nsum_val(&kin);
    out[1] = nsum_val(&pot);
}

/* Three-dimensional moments: (sum |psi|^2, sum x|psi|^2, sum y|psi|^2,
 * sum z|psi|^2, sum x^2|psi|^2, sum y^2|psi|^2, sum z^2|psi|^2). */
void oracle_moments3(int64_t nx, int64_t ny, int64_t nz, const double *re,
                     const double *im, double *out)
{
    nsum a[7];
    memset(a, 0, sizeof(a));
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = (z * ny + y) * nx + x;
                double p = re[i] * re[i] + im[i] * im[i];
                nsum_add(&a[0], p);
                nsum_add(&a[1], (double)x * p);
                nsum_add(&a[2], (double)y * p);
                nsum_add(&a[3], (double)z * p);
                nsum_add(&a[4], (double)x * (double)x * p);
                nsum_add(&a[5], (double)y * (double)y * p);
                nsum_add(&a[6], (double)z * (double)z * p);
            }
    for (int q = 0; q < 7; ++q) out[q] = nsum_val(&a[q]);
}

/* <psi|H|psi> on the 3-D lattice: bonds along x, y and z. */
void oracle_energy3(int64_t nx, int64_t ny, int64_t nz, const double *re, const double *im,
                    const double *V, double J, double *out)
{
    nsum kin = {0, 0}, pot = {0, 0};
    const int64_t plane = nx * ny;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = (z * ny + y) * nx + x;
                if (x + 1 < nx)
                    nsum_add(&kin, -2.0 * J * (re[i] * re[i + 1] + im[i] * im[i + 1]));
                if (y + 1 < ny)
                    nsum_add(&kin, -2.0 * J * (re[i] * re[i + nx] + im[i] * im[i + nx]));
                if (z + 1 < nz)
                    nsum_add(&kin, -2.0 * J * (re[i] * re[i + plane] + im[i] * im[i + plane]));
                if (V) nsum_add(&pot, V[i] * (re[i] * re[i] + im[i] * im[i]));
            }
    out[0] = nsum_val(&kin);
    out[1] = nsum_val(&pot);
}

/* <a|b> = sum conj(a) b, compensated. */
void oracle_inner(int64_t n, const double *are, const double *aim,
                  const double *bre, const double *bim, double *out)
{
    nsum r = {0, 0}, m = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        nsum_add(&r, are[i] * bre[i]);
        nsum_add(&r, aim[i] * bim[i]);
        nsum_add(&m, are[i] * bim[i]);
        nsum_add(&m, -aim[i] * bre[i]);
    }
    out[0] = nsum_val(&r);
    out[1] = nsum_val(&m);
}

/* ------------------------------------------------------------------------ */
/* Adjoint: gradient of the fidelity F = |<phi|psi_T>|^2 with respect to the */
/* potential V on every site, for psi_T = U2(dt)^n psi_0.                    */
/*                                                                           */
/* Write one step as psi_s = B P A psi_{s-1}: A = the first four sweeps,     */
/* P = diag(exp(-i V dt)), B = the last four sweeps.  With c = <phi|psi_T>,  */
/* the costate lambda_n = phi, lambda_{s-1} = U_s^dagger lambda_s, the       */
/* mid-step state m_s = P A psi_{s-1} and lt_s = B^dagger lambda_s:          */
/*   dc/dV_j = -i dt sum_s conj(lt_s[j]) m_s[j]                              */
/*   dF/dV_j = 2 dt sum_s Im( conj(c) conj(lt_s[j]) m_s[j] ).               */
/* Every factor is unitary and symmetric, so its inverse is the same sweep   */
/* at -theta (or the conjugate phase).  The oracle walks the steps backward, */
/* rebuilding psi_{s-1} from psi_s by the inverse factors (no storage of the */
/* trajectory); the test-suite pins the result against finite differences   */
/* of the forward evolution.                                                  */
/* ------------------------------------------------------------------------ */
/* B^dagger: the factors of B in reverse order, each at -theta. */
static void apply_B_dag(int64_t nx, int64_t ny, double *re, double *im,
                        double theta, int nthreads)
{
    oracle_sweep_x(nx, ny, re, im, 0, -theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 1, -theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 0, -theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 1, -theta, nthreads);
}

/* A^dagger: the factors of A in reverse order, each at -theta. */
static void apply_A_dag(int64_t nx, int64_t ny, double *re, double *im,
                        double theta, int nthreads)
{
    oracle_sweep_y(nx, ny, re, im, 1, -theta, nthreads);
    oracle_sweep_y(nx, ny, re, im, 0, -theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 1, -theta, nthreads);
    oracle_sweep_x(nx, ny, re, im, 0, -theta, nthreads);
}

int oracle_adjoint_grad(int64_t nx, int64_t ny, const double *psi0_re,
                        const double *psi0_im, const double *phi_re,
                        const double *phi_im, const double *V, double dt,
                        double theta, int64_t steps, double *grad,
                        double *fidelity, double *overlap, int nthreads)
{
    if (nx < 1 || ny < 1 || steps < 0) return -1;
    int64_t n = nx * ny;
    double *pr = (double *)malloc(sizeof(double) * n);
    double *pi = (double *)malloc(sizeof(double) * n);
    double *lr = (double *)malloc(sizeof(double) * n);
    double *li = (double *)malloc(sizeof(double) * n);
    double *Vneg = (double *)malloc(sizeof(double) * n);
    if (!pr || !pi || !lr || !li || !Vneg) {
        free(pr); free(pi); free(lr); free(li); free(Vneg);
        return -2;
    }
    memcpy(pr, psi0_re, sizeof(double) * n);
    memcpy(pi, psi0_im, sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) Vneg[i] = V ? -V[i] : 0.0;

    /* forward: psi_T */
    oracle_evolve(nx, ny, pr, pi, V, dt, theta, steps, 2, nthreads);

    /* c = <phi|psi_T> */
    double cc[2];
    oracle_inner(n, phi_re, phi_im, pr, pi, cc);
    if (overlap) { overlap[0] = cc[0]; overlap[1] = cc[1]; }
    if (fidelity) *fidelity = cc[0] * cc[0] + cc[1] * cc[1];

    memcpy(lr, phi_re, sizeof(double) * n);
    memcpy(li, phi_im, sizeof(double) * n);
    nsum *acc = (nsum *)calloc((size_t)n, sizeof(nsum));
    if (!acc) {
        free(pr); free(pi); free(lr); free(li); free(Vneg);
        return -2;
    }

    for (int64_t s = steps; s >= 1; --s) {
        /* lt_s = B^dagger lambda_s ; m_s = B^dagger psi_s */
        apply_B_dag(nx, ny, lr, li, theta, nthreads);
        apply_B_dag(nx, ny, pr, pi, theta, nthreads);
        for (int64_t j = 0; j < n; ++j) {
            /* z = conj(c) * conj(lt[j]) * m[j] */
            double ar = cc[0] * lr[j] - cc[1] * li[j];   /* conj(c) conj(lt) = conj(c lt) */
            double ai = -(cc[0] * li[j] + cc[1] * lr[j]);
            double zi = ar * pi[j] + ai * pr[j];
            nsum_add(&acc[j], 2.0 * dt * zi);
        }
        /* lambda_{s-1} = A^dagger P^dagger lt_s ; psi_{s-1} = A^dagger P^dagger m_s */
        oracle_phase(nx, ny, lr, li, Vneg, dt, nthreads);
        oracle_phase(nx, ny, pr, pi, Vneg, dt, nthreads);
        apply_A_dag(nx, ny, lr, li, theta, nthreads);
        apply_A_dag(nx, ny, pr, pi, theta, nthreads);
    }
    for (int64_t j = 0; j < n; ++j) grad[j] = nsum_val(&acc[j]);
    free(acc);
    free(pr); free(pi); free(lr); free(li); free(Vneg);
    return 0;
}

/* Neumaier-compensated sum of an array (exposed so that its own pin can
 * check it against an exactly rounded sum). */
double oracle_compensated_sum(int64_t n, const double *v)
{
    nsum a = {0, 0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&a, v[i]);
    return nsum_val(&a);
}
