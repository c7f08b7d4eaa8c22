// C ABI of libtrotter.so (declared in include/trotter.h).
//
// Host-side only: argument checks, the slab layout, staging of host input
// through the grid's own ping-pong planes, kernel dispatch and error
// reporting.  Every step of the method runs in the kernels of plain.cu,
// fused.cu and reduce.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/trotter.h"
#include "grid.h"
#include "internal.h"
#include "trace.h"

namespace {

thread_local char g_err[512] = "";
thread_local int64_t g_launches = 0;

ts_status fail(ts_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

ts_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(TS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int64_t kMaxSide = int64_t(1) << 20;

// Depth of the fused path when the caller passes K = 0.  On one GB300 at
// 8192^2 (site-steps/s): K=1 2.2e11, K=2 5.2e11, K=3 7.5e11, K=4 7.75e11,
// K=5 7.2e11.  K = 3 runs at 88 % of the HBM copy bandwidth; K = 4 is 4 %
// faster there but bound by instruction latency, so its speed follows the SM
// clock (which drops under a power cap) while K = 3's follows HBM.
int auto_depth() { return 3; }
constexpr int kPlanes = 7;   // re_a, im_a, re_b, im_b, gamma_V, s_V, V

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t scratch_bytes()
{
    // partials, result, error word, multi-grid descriptor
    return round_up(sizeof(double) * ts::OBS_MAX_BLOCKS * ts::OBS_Q3, 256) +
           round_up(sizeof(double) * ts::OBS_Q3, 256) + 256 +
           round_up(sizeof(ts::GridDesc), 256);
}

}  // namespace

namespace ts {
void count_launches(int64_t n) { g_launches += n; }

ts_status grid_setup(const ts_layout &L, void *slab, bool owns_slab, ts_grid **out)
{
    ts_grid *g = new (std::nothrow) ts_grid();
    if (!g) return fail(TS_ERR_OOM, "grid set-up: host allocation failed");
    g->L = L;
    g->esize = L.dtype == TS_F64 ? 8 : 4;
    g->owns_slab = owns_slab;
    g->slab = (unsigned char *)slab;
    unsigned char *scr = g->slab + kPlanes * L.plane_bytes;
    g->partials = (double *)scr;
    scr += round_up(sizeof(double) * OBS_MAX_BLOCKS * OBS_Q3, 256);
    g->result = (double *)scr;
    scr += round_up(sizeof(double) * OBS_Q3, 256);
    g->err = (int *)scr;
    g->host_copied = nullptr;
    scr += 256;
    g->desc_dev = (GridDesc *)scr;
    g->cur = 0;
    g->dt = g->theta = g->J = 0.0;
    g->g1 = g->s1 = g->t1 = g->s2 = g->t2 = 0.0;
    g->order = 2;
    g->sub[0] = g->sub[1] = RotCoef{0.0, 0.0, 0.0, 0.0, 0.0};
    g->tab_b = nullptr;
    g->drive_slab = nullptr;
    g->drive_pos = 0;
    g->driven = false;
    g->tmaps_ok = false;
    if (L.dtype == TS_F32) {
        const char *why = "";
        bool ok = true;
        for (int c = 0; c < 2 && ok; ++c)
            ok = make_pair_tensor_map(&g->tm_state[c], g->plane(2 * c), (int)L.nx, (int)g->rows(),
                                      L.pitch, L.plane_bytes, &why);
        ok = ok && make_pair_tensor_map(&g->tm_phase, g->pg(), (int)L.nx, (int)g->rows(), L.pitch,
                                        L.plane_bytes, &why);
        if (!ok) {
            delete g;
            return fail(TS_ERR_CUDA, "grid set-up: %s", why);
        }
        g->tmaps_ok = true;
    }
    *out = g;
    return TS_OK;
}

size_t grid_scratch_offset(const ts_layout &L) { return kPlanes * L.plane_bytes; }

RotCoef rot_coef(double theta)
{
    // versine form (g = 1 - cos theta = 2 sin^2(theta/2), s = sin theta) and
    // lifting form (t = tan(theta/2), s); the merged angle 2 theta in lifting form
    const double sh1 = std::sin(0.5 * theta);
    return RotCoef{2.0 * sh1 * sh1, std::sin(theta), std::tan(0.5 * theta),
                   std::sin(2.0 * theta), std::tan(theta)};
}

void grid_set_coefficients(ts_grid *g, double dt, double theta, cudaStream_t st)
{
    g->dt = dt;
    g->theta = theta;
    g->J = dt != 0.0 ? 2.0 * theta / dt : 0.0;
    const RotCoef c = rot_coef(theta);
    g->g1 = c.g1;
    g->s1 = c.s1;
    g->t1 = c.t1;
    g->s2 = c.s2;
    g->t2 = c.t2;
    if (!g->f64()) grid_write_desc(g, st);
}

void grid_write_desc(ts_grid *g, cudaStream_t st)
{
    GridDesc &d = g->desc_host;
    d.tm_state[0] = g->tm_state[0];
    d.tm_state[1] = g->tm_state[1];
    d.tm_phase = g->tm_phase;
    for (int c = 0; c < 2; ++c) {
        d.re[c] = (float *)g->plane(2 * c);
        d.im[c] = (float *)g->plane(2 * c + 1);
    }
    d.nx = (int)g->L.nx;
    d.ny = (int)g->L.ny;
    d.pitch = g->L.pitch;
    d.t1 = (float)g->t1;
    d.s1 = (float)g->s1;
    d.g1 = (float)g->g1;
    d.t2 = (float)g->t2;
    d.s2 = (float)g->s2;
    // pageable source: the call returns once the host struct is staged, and
    // the device copy lands in stream order before later kernels read it
    cudaMemcpyAsync(g->desc_dev, &d, sizeof(GridDesc), cudaMemcpyHostToDevice, st);
}

cudaError_t evolve_multi(ts_grid *const *gs, const int64_t *steps, int n, int K, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    // Each grid runs floor(steps/K) launches at depth K, then one at depth
    // steps % K -- the same sequence as evolving it alone.  All grids with a
    // launch left share each launch; a table is rebuilt when the set changes.
    std::vector<int64_t> full(n), rem(n);
    int64_t max_full = 0;
    for (int i = 0; i < n; ++i) {
        full[i] = steps[i] / K;
        rem[i] = steps[i] % K;
        if (full[i] > max_full) max_full = full[i];
    }
    EpochEntry *tab = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tab, sizeof(EpochEntry) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    std::vector<EpochEntry> h;
    std::vector<int> hx, hy;
    auto run = [&](int depth, const std::vector<int> &idx, int64_t launches) -> cudaError_t {
        h.clear();
        hx.clear();
        hy.clear();
        for (int i : idx) {
            h.push_back(EpochEntry{gs[i]->desc_dev, 0, gs[i]->cur, 0});
            hx.push_back((int)gs[i]->L.nx);
            hy.push_back((int)gs[i]->L.ny);
        }
        const MultiPlan plan = fused_multi_plan(depth, (int)h.size(), hx.data(), hy.data(), h.data());
        if (plan.warps < 1) return cudaErrorInvalidConfiguration;
        cudaError_t err = cudaMemcpyAsync(tab, h.data(), sizeof(EpochEntry) * h.size(),
                                          cudaMemcpyHostToDevice, st);
        for (int64_t t = 0; t < launches && err == cudaSuccess; ++t)
            err = launch_fused_multi(depth, tab, (int)h.size(), plan, (int)(t & 1),
                                     gs[idx[0]]->err, st);
        if (err == cudaSuccess && (launches & 1))
            for (int i : idx) gs[i]->cur ^= 1;
        return err;
    };
    int64_t done = 0;
    while (e == cudaSuccess && done < max_full) {
        std::vector<int> idx;
        int64_t until = max_full;
        for (int i = 0; i < n; ++i)
            if (full[i] > done) {
                idx.push_back(i);
                if (full[i] < until) until = full[i];
            }
        e = run(K, idx, until - done);
        done = until;
    }
    for (int r = 1; r < K && e == cudaSuccess; ++r) {
        std::vector<int> idx;
        for (int i = 0; i < n; ++i)
            if (rem[i] == r) idx.push_back(i);
        if (!idx.empty()) e = run(r, idx, 1);
    }
    cudaError_t f = cudaFreeAsync(tab, st);
    return e != cudaSuccess ? e : f;
}

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}
}  // namespace ts

extern "C" {

const char *ts_last_error(void) { return g_err; }

int ts_fused_default_depth(void) { return auto_depth(); }

int64_t ts_launch_count(int reset)
{
    int64_t v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

ts_status ts_grid_layout3(int64_t nx, int64_t ny, int64_t nz, ts_dtype dtype, ts_layout *out)
{
    if (!out) return fail(TS_ERR_ARG, "ts_grid_layout: out is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return fail(TS_ERR_ARG,
                    "ts_grid_layout: sides must be in [1, 2^20], got %lld x %lld x %lld",
                    (long long)nx, (long long)ny, (long long)nz);
    if (ny * nz > (int64_t(1) << 30))
        return fail(TS_ERR_ARG, "ts_grid_layout: ny * nz must be at most 2^30, got %lld",
                    (long long)(ny * nz));
    if (dtype != TS_F32 && dtype != TS_F64)
        return fail(TS_ERR_ARG, "ts_grid_layout: unknown dtype %d", (int)dtype);
    const size_t es = dtype == TS_F64 ? 8 : 4;
    out->nx = nx;
    out->ny = ny;
    out->pitch = (int64_t)round_up((size_t)nx, 32);
    out->plane_bytes = round_up((size_t)out->pitch * (size_t)ny * (size_t)nz * es, 256);
    out->slab_bytes = kPlanes * out->plane_bytes + scratch_bytes();
    out->dtype = dtype;
    out->nz = nz;
    return TS_OK;
}

ts_status ts_grid_layout(int64_t nx, int64_t ny, ts_dtype dtype, ts_layout *out)
{
    return ts_grid_layout3(nx, ny, 1, dtype, out);
}

ts_status ts_create_grid(int64_t nx, int64_t ny, ts_dtype dtype, void *slab, size_t slab_bytes,
                         ts_grid **out)
{
    return ts_create_grid3(nx, ny, 1, dtype, slab, slab_bytes, out);
}

ts_status ts_create_grid3(int64_t nx, int64_t ny, int64_t nz, ts_dtype dtype, void *slab,
                          size_t slab_bytes, ts_grid **out)
{
    if (!out) return fail(TS_ERR_ARG, "ts_create_grid: out is NULL");
    *out = nullptr;
    ts_layout L;
    ts_status st = ts_grid_layout3(nx, ny, nz, dtype, &L);
    if (st != TS_OK) return st;
    if (slab) {
        if (((uintptr_t)slab & 255u) != 0)
            return fail(TS_ERR_ARG, "ts_create_grid: slab must be 256-byte aligned");
        if (slab_bytes < L.slab_bytes)
            return fail(TS_ERR_ARG, "ts_create_grid: slab has %zu bytes, needs %zu", slab_bytes,
                        L.slab_bytes);
        // The grid lives on the slab's device.  Making it current also binds
        // its context to this thread, which the tensor-map encoding (a driver
        // call) needs: a thread that has only used another runtime's cached
        // streams and allocations may have none yet.
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, slab) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(TS_ERR_ARG, "ts_create_grid: slab is not device memory");
        }
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e == cudaSuccess && cur != pa.device) e = cudaSetDevice(pa.device);
        if (e == cudaSuccess) e = cudaFree(nullptr);   // context current in this thread
        if (e != cudaSuccess) return cuda_fail(e, "ts_create_grid: device of the slab");
    }
    bool owns = slab == nullptr;
    if (owns) {
        cudaError_t e = cudaMalloc(&slab, L.slab_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(TS_ERR_OOM, "ts_create_grid: cudaMalloc(%zu): %s", L.slab_bytes,
                        cudaGetErrorString(e));
        }
    }
    ts_grid *g = nullptr;
    st = ts::grid_setup(L, slab, owns, &g);
    if (st != TS_OK) {
        if (owns) cudaFree(slab);
        return st;
    }
    cudaError_t e = cudaMemset(g->slab, 0, L.slab_bytes);
    if (e == cudaSuccess && !g->f64()) {
        ts::grid_write_desc(g, nullptr);
        e = cudaStreamSynchronize(nullptr);
    }
    if (e != cudaSuccess) {
        ts_destroy_grid(g);
        return cuda_fail(e, "ts_create_grid: zero-fill");
    }
    *out = g;
    return TS_OK;
}

ts_status ts_destroy_grid(ts_grid *g)
{
    if (!g) return TS_OK;
    ts::forget_adjoint(g);
    cudaError_t e = cudaSuccess;
    if (g->owns_slab) e = cudaFree(g->slab);
    for (unsigned char *extra : {g->tab_b, g->drive_slab}) {
        if (!extra) continue;
        cudaError_t f = cudaFree(extra);
        if (e == cudaSuccess) e = f;
    }
    if (g->host_copied) cudaEventDestroy(g->host_copied);
    delete g;
    if (e != cudaSuccess) return cuda_fail(e, "ts_destroy_grid: cudaFree");
    return TS_OK;
}

ts_status ts_grid_info(const ts_grid *g, ts_layout *layout, void **re, void **im)
{
    if (!g) return fail(TS_ERR_ARG, "ts_grid_info: grid is NULL");
    if (layout) *layout = g->L;
    if (re) *re = g->re();
    if (im) *im = g->im();
    return TS_OK;
}

namespace {

// Copy a dense host array into the staging region (the two non-current
// planes, contiguous in the slab) and convert it into `dst` on the device.
// Wait until the host-to-device copies enqueued so far on `st` have landed,
// so the caller's host buffer may be reused, without waiting for the kernels
// that consume them: those stay queued in stream order.  (Waiting for the
// whole stream would also wait for a table or conversion kernel that, on a
// busy GPU, may sit behind another stream's higher-priority work.)
ts_status wait_host_copies(ts_grid *g, cudaStream_t st, const char *who)
{
    cudaError_t e = cudaSuccess;
    if (!g->host_copied) e = cudaEventCreateWithFlags(&g->host_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(g->host_copied, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(g->host_copied);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return TS_OK;
}

// The copy and the conversion are stream-ordered, so the region can be
// staged into again by a later call on the same stream without a host wait.
// With `copied`, the host waits for this copy to land (not for the
// conversion) before the conversion is enqueued behind it.
ts_status stage_in(ts_grid *g, const void *host, ts_dtype src_dtype, void *dst, cudaStream_t st,
                   bool copied = false)
{
    const size_t n = (size_t)g->L.nx * (size_t)g->rows();
    const size_t es = src_dtype == TS_F64 ? 8 : 4;
    if (n * es > 2 * g->L.plane_bytes)
        return fail(TS_ERR_ARG, "staging region too small");  // cannot happen by layout
    void *stage = g->re_other();
    cudaError_t e = cudaMemcpyAsync(stage, host, n * es, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    if (copied) {
        ts_status s = wait_host_copies(g, st, "host-to-device copy");
        if (s != TS_OK) return s;
    }
    e = ts::launch_convert_in(stage, src_dtype == TS_F64, dst, g->f64(), (int)g->L.nx,
                              (int)g->rows(), g->L.pitch, st);
    if (e != cudaSuccess) return cuda_fail(e, "convert kernel");
    return TS_OK;
}

ts_status check_errword(ts_grid *g, cudaStream_t st)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "kernel error (reported at sync)");
    if (h != 0) {
        cudaMemsetAsync(g->err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        if (h & ts::ERRBIT_WAIT_TIMEOUT)
            return fail(TS_ERR_TIMEOUT, "a bounded wait in a fused kernel gave up (error word %d)", h);
        return fail(TS_ERR_CUDA, "a kernel reported error word %d", h);
    }
    return TS_OK;
}

}  // namespace

ts_status ts_set_state(ts_grid *g, const void *re, const void *im, ts_dtype src_dtype,
                       ts_mem where, void *stream)
{
    ts::TraceRange trace_("ts_set_state");
    if (!g || !re || !im) return fail(TS_ERR_ARG, "ts_set_state: null argument");
    if (src_dtype != TS_F32 && src_dtype != TS_F64)
        return fail(TS_ERR_ARG, "ts_set_state: unknown dtype");
    cudaStream_t st = (cudaStream_t)stream;
    const bool sf = src_dtype == TS_F64;
    const int nx = (int)g->L.nx, ny = (int)g->rows();   // rows: all slabs
    if (where == TS_DEVICE) {
        cudaError_t e = ts::launch_convert_in(re, sf, g->re(), g->f64(), nx, ny, g->L.pitch, st);
        if (e == cudaSuccess)
            e = ts::launch_convert_in(im, sf, g->im(), g->f64(), nx, ny, g->L.pitch, st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_set_state: convert kernel");
        return TS_OK;
    }
    if (where != TS_HOST) return fail(TS_ERR_ARG, "ts_set_state: unknown memory kind");
    if (sf == g->f64()) {
        // same type: straight pitched copies
        const size_t es = g->esize;
        cudaError_t e = cudaMemcpy2DAsync(g->re(), g->L.pitch * es, re, nx * es, nx * es, ny,
                                          cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(g->im(), g->L.pitch * es, im, nx * es, nx * es, ny,
                                  cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_set_state: host-to-device copy");
        return wait_host_copies(g, st, "ts_set_state: host-to-device copy");
    }
    // both planes pass through the one staging region, in stream order
    ts_status s = stage_in(g, re, src_dtype, g->re(), st);
    if (s != TS_OK) return s;
    return stage_in(g, im, src_dtype, g->im(), st, true);
}

ts_status ts_get_state(ts_grid *g, void *re, void *im, ts_dtype dst_dtype, ts_mem where,
                       void *stream)
{
    ts::TraceRange trace_("ts_get_state");
    if (!g || !re || !im) return fail(TS_ERR_ARG, "ts_get_state: null argument");
    if (dst_dtype != TS_F32 && dst_dtype != TS_F64)
        return fail(TS_ERR_ARG, "ts_get_state: unknown dtype");
    cudaStream_t st = (cudaStream_t)stream;
    ts_status s = check_errword(g, st);
    if (s != TS_OK) return s;
    const bool df = dst_dtype == TS_F64;
    const int nx = (int)g->L.nx, ny = (int)g->rows();   // rows: all slabs
    const size_t n = (size_t)nx * ny;
    cudaError_t e;
    if (where == TS_DEVICE) {
        e = ts::launch_convert_out(g->re(), g->f64(), re, df, nx, ny, g->L.pitch, st);
        if (e == cudaSuccess)
            e = ts::launch_convert_out(g->im(), g->f64(), im, df, nx, ny, g->L.pitch, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_get_state");
        return TS_OK;
    }
    if (where != TS_HOST) return fail(TS_ERR_ARG, "ts_get_state: unknown memory kind");
    if (df == g->f64()) {
        const size_t es = g->esize;
        e = cudaMemcpy2DAsync(re, nx * es, g->re(), g->L.pitch * es, nx * es, ny,
                              cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(im, nx * es, g->im(), g->L.pitch * es, nx * es, ny,
                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_get_state: device-to-host copy");
        return TS_OK;
    }
    // convert on the device into the staging region, then copy out
    const size_t es = df ? 8 : 4;
    void *stage = g->re_other();
    void *dsts[2] = {re, im};
    void *srcs[2] = {g->re(), g->im()};
    for (int c = 0; c < 2; ++c) {
        e = ts::launch_convert_out(srcs[c], g->f64(), stage, df, nx, ny, g->L.pitch, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dsts[c], stage, n * es, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_get_state");
    }
    return TS_OK;
}

ts_status ts_set_potential(ts_grid *g, const double *V, ts_mem where, double dt, double theta,
                           void *stream)
{
    return ts_set_potential_order(g, V, where, dt, theta, 2, stream);
}

ts_status ts_set_potential_order(ts_grid *g, const double *V, ts_mem where, double dt,
                                 double theta, int order, void *stream)
{
    ts::TraceRange trace_("ts_set_potential_order");
    if (!g) return fail(TS_ERR_ARG, "ts_set_potential: grid is NULL");
    if (!std::isfinite(dt) || !std::isfinite(theta))
        return fail(TS_ERR_ARG, "ts_set_potential: dt and theta must be finite");
    if (where != TS_HOST && where != TS_DEVICE)
        return fail(TS_ERR_ARG, "ts_set_potential: unknown memory kind");
    if (order != 2 && order != 4)
        return fail(TS_ERR_ARG, "ts_set_potential_order: order must be 2 or 4, got %d", order);
    if (order == 4 && g->is3d())
        return fail(TS_ERR_UNSUPPORTED, "ts_set_potential_order: order 4 on 2-D grids only");
    cudaStream_t st = (cudaStream_t)stream;
    g->driven = false;   // a new potential ends any time-dependent drive
    g->drive_a.clear();
    const int nx = (int)g->L.nx, ny = (int)g->rows();   // rows: all slabs
    cudaError_t e;
    // fourth order (Eq. fourthorder): U4(dt) = U2(p dt)^2 U2((1-4p) dt) U2(p dt)^2
    // with p = 1 / (4 - 4^(1/3)); substep a = p dt uses planes 4/5, substep
    // b = (1 - 4p) dt a second table in two library-owned planes
    const double p4 = 1.0 / (4.0 - std::cbrt(4.0));
    const double w[2] = {p4, 1.0 - 4.0 * p4};
    const size_t PB = g->L.plane_bytes;
    if (order == 4 && !g->tab_b) {
        unsigned char *tb = nullptr;
        e = cudaMalloc((void **)&tb, 2 * PB);
        if (e != cudaSuccess) return fail(TS_ERR_OOM, "ts_set_potential_order: second table: %s",
                                          cudaGetErrorString(e));
        if (!g->f64()) {
            const char *why = "";
            if (!ts::make_pair_tensor_map(&g->tm_phase_b, tb, nx, ny, g->L.pitch, PB, &why)) {
                cudaFree(tb);
                return fail(TS_ERR_CUDA, "ts_set_potential_order: %s", why);
            }
        }
        g->tab_b = tb;
    }
    ts::grid_set_coefficients(g, dt, theta, st);
    g->order = order;
    if (order == 4)
        for (int i = 0; i < 2; ++i) g->sub[i] = ts::rot_coef(w[i] * theta);
    if (!V) {
        e = cudaMemsetAsync(g->pg(), 0, 3 * g->L.plane_bytes, st);   // planes 4, 5, 6
        if (e == cudaSuccess && order == 4) e = cudaMemsetAsync(g->tab_b, 0, 2 * PB, st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_set_potential: clear");
        return TS_OK;
    }
    const double *src = V;
    if (where == TS_HOST) {
        const size_t n = (size_t)nx * ny;
        e = cudaMemcpyAsync(g->re_other(), V, n * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "ts_set_potential: host-to-device copy");
        // V may be reused once it is on the device; the table kernels read the
        // staged copy in stream order
        ts_status s = wait_host_copies(g, st, "ts_set_potential: host-to-device copy");
        if (s != TS_OK) return s;
        src = (const double *)g->re_other();
    }
    e = ts::launch_phase_table(src, g->pg(), g->ps(), g->vp(), g->f64(), nx, ny, g->L.pitch,
                               order == 4 ? w[0] * dt : dt, st);
    if (e == cudaSuccess && order == 4)
        e = ts::launch_phase_table(src, g->pg_b(), g->ps_b(), g->vp(), g->f64(), nx, ny,
                                   g->L.pitch, w[1] * dt, st);
    if (e != cudaSuccess) return cuda_fail(e, "ts_set_potential: table kernel");
    return TS_OK;
}

ts_status ts_set_drive(ts_grid *g, const double *V1, ts_mem where, const double *a, int64_t n_a,
                       void *stream)
{
    ts::TraceRange trace_("ts_set_drive");
    if (!g) return fail(TS_ERR_ARG, "ts_set_drive: grid is NULL");
    if (n_a < 0 || (n_a > 0 && !a)) return fail(TS_ERR_ARG, "ts_set_drive: bad amplitude array");
    if (where != TS_HOST && where != TS_DEVICE)
        return fail(TS_ERR_ARG, "ts_set_drive: unknown memory kind");
    if (g->order != 2 || g->is3d())
        return fail(TS_ERR_UNSUPPORTED, "ts_set_drive: second-order 2-D grids only");
    for (int64_t i = 0; i < n_a; ++i)
        if (!std::isfinite(a[i])) return fail(TS_ERR_ARG, "ts_set_drive: a[%lld] is not finite", (long long)i);
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = (int)g->L.nx, ny = (int)g->rows();   // rows: all slabs
    const size_t PB = g->L.plane_bytes;
    cudaError_t e;
    if (!g->drive_slab) {
        unsigned char *ds = nullptr;
        e = cudaMalloc((void **)&ds, 3 * PB);
        if (e != cudaSuccess)
            return fail(TS_ERR_OOM, "ts_set_drive: drive planes: %s", cudaGetErrorString(e));
        if (!g->f64()) {
            const char *why = "";
            if (!ts::make_pair_tensor_map(&g->tm_drive, ds, nx, ny, g->L.pitch, PB, &why, 3)) {
                cudaFree(ds);
                return fail(TS_ERR_CUDA, "ts_set_drive: %s", why);
            }
        }
        g->drive_slab = ds;
    }
    // the static table (gamma_V, s_V) next to V1, so one box load fetches all three
    e = cudaMemcpyAsync(g->drive_slab, g->pg(), 2 * PB, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "ts_set_drive: table copy");
    if (!V1) {
        e = cudaMemsetAsync(g->drive_v1(), 0, PB, st);
    } else {
        const double *src = V1;
        if (where == TS_HOST) {
            e = cudaMemcpyAsync(g->re_other(), V1, (size_t)nx * ny * sizeof(double),
                                cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "ts_set_drive: host-to-device copy");
            ts_status s = wait_host_copies(g, st, "ts_set_drive: host-to-device copy");
            if (s != TS_OK) return s;
            src = (const double *)g->re_other();
        }
        e = ts::launch_convert_in(src, true, g->drive_v1(), g->f64(), nx, ny, g->L.pitch, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "ts_set_drive: V1");
    g->drive_a.assign(a, a + n_a);
    g->drive_pos = 0;
    g->driven = true;
    return TS_OK;
}

ts_status ts_clear_drive(ts_grid *g)
{
    if (!g) return fail(TS_ERR_ARG, "ts_clear_drive: grid is NULL");
    g->driven = false;
    g->drive_a.clear();
    g->drive_pos = 0;
    return TS_OK;
}

namespace {

// `steps` second-order steps, one kernel per sweep, with the rotation
// coefficients c and the phase table (pg, ps).
ts_status plain_run(ts_grid *g, int64_t steps, const ts::RotCoef &c, const void *pg,
                    const void *ps, cudaStream_t st, const double *drive_adt = nullptr)
{
    const int nx = (int)g->L.nx, ny = (int)g->rows();   // rows: all slabs
    const int64_t pitch = g->L.pitch;
    void *re = g->re(), *im = g->im();
    const bool f = g->f64();
    double gg = c.g1, ss = c.s1;
    if (!f) {   // FP32 path: coefficients rounded once to float
        gg = (double)(float)gg;
        ss = (double)(float)ss;
    }
    // one sweep: X over all rows; Y inside each slab and Z between slabs on
    // 3-D grids (X-even, X-odd, Y-even, Y-odd[, Z-even, Z-odd], phase, mirror)
    const int sy = (int)g->L.ny, sz = (int)g->L.nz;
    auto sweep = [&](int axis, int parity) {
        if (axis == 0 || !g->is3d())
            return ts::launch_plain_sweep(re, im, f, nx, ny, pitch, axis, parity, gg, ss, st);
        if (axis == 1)
            return ts::launch_plain_sweep_y3(re, im, f, nx, sy, sz, pitch, parity, gg, ss, st);
        return ts::launch_plain_sweep_z(re, im, f, nx, sy, sz, pitch, parity, gg, ss, st);
    };
    const int n_fam = g->is3d() ? 6 : 4;
    for (int64_t n = 0; n < steps; ++n) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < n_fam && e == cudaSuccess; ++i) e = sweep(i / 2, i & 1);
        if (e == cudaSuccess)
            e = ts::launch_plain_phase(re, im, pg, ps, f, nx, ny, pitch, st);
        if (e == cudaSuccess && drive_adt)
            e = ts::launch_plain_drive(re, im, g->drive_v1(), f, nx, ny, pitch, drive_adt[n], st);
        for (int i = n_fam - 1; i >= 0 && e == cudaSuccess; --i) e = sweep(i / 2, i & 1);
        if (e != cudaSuccess) return cuda_fail(e, "plain sweep launch");
    }
    return TS_OK;
}



// FP64 grids (ts_evolve): second-order substeps one sweep per launch, with
// the sweeps merged where two substeps meet.  X, Y (and Z) factors act on
// different coordinates and commute, and two factors of one family add
// their angles, so the mirror half of substep i and the first half of
// substep i + 1,
//   [Yo Ye Xo Xe](i) [Xe Xo Ye Yo](i+1)  (plus Zo Ze / Ze Zo in 3-D),
// equal Xo(i) Xe(i + i+1) Xo(i+1) . Yo(i) Ye(i + i+1) Yo(i+1) [. Z]: three
// sweeps per axis instead of four.  A sweep at angle phi uses the lifting
// form (tan(phi/2), sin phi; 3 FMA per site instead of 4) when |phi| <= pi/2,
// the versine form otherwise.  Substep i is sub(i) = {kinetic half angle,
// phase table, drive angle or 0 with has_drive false}.
struct Substep {
    double theta;
    const void *pg, *ps;
    bool has_drive;
    double adt;
};

extern "C++" {
template <typename SubAt>
ts_status merged_run(ts_grid *g, int64_t n, SubAt sub, cudaStream_t st)
{
    if (n <= 0) return TS_OK;
    const int nx = (int)g->L.nx, ny = (int)g->rows();
    const int sy = (int)g->L.ny, sz = (int)g->L.nz;
    const int64_t pitch = g->L.pitch;
    void *re = g->re(), *im = g->im();
    const int n_axes = g->is3d() ? 3 : 2;
    auto sweep = [&](int axis, int parity, double phi) {
        const bool lift = std::fabs(phi) <= 0.5 * M_PI;
        const double h = std::sin(0.5 * phi);
        const double c = lift ? std::tan(0.5 * phi) : 2.0 * h * h, s = std::sin(phi);
        if (axis == 0 || !g->is3d())
            return ts::launch_plain_sweep(re, im, true, nx, ny, pitch, axis, parity, c, s, st, lift);
        if (axis == 1)
            return ts::launch_plain_sweep_y3(re, im, true, nx, sy, sz, pitch, parity, c, s, st, lift);
        return ts::launch_plain_sweep_z(re, im, true, nx, sy, sz, pitch, parity, c, s, st, lift);
    };
    Substep cur = sub(0);
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < n_axes && e == cudaSuccess; ++a) {
        e = sweep(a, 0, cur.theta);
        if (e == cudaSuccess) e = sweep(a, 1, cur.theta);
    }
    for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
        e = ts::launch_plain_phase(re, im, cur.pg, cur.ps, true, nx, ny, pitch, st);
        if (e == cudaSuccess && cur.has_drive)
            e = ts::launch_plain_drive(re, im, g->drive_v1(), true, nx, ny, pitch, cur.adt, st);
        if (i + 1 < n) {
            const Substep next = sub(i + 1);
            for (int a = 0; a < n_axes && e == cudaSuccess; ++a) {
                e = sweep(a, 1, cur.theta);
                if (e == cudaSuccess) e = sweep(a, 0, cur.theta + next.theta);
                if (e == cudaSuccess) e = sweep(a, 1, next.theta);
            }
            cur = next;
        } else {
            for (int a = n_axes - 1; a >= 0 && e == cudaSuccess; --a) {
                e = sweep(a, 1, cur.theta);
                if (e == cudaSuccess) e = sweep(a, 0, cur.theta);
            }
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "FP64 sweep launch");
    return TS_OK;
}
}  // extern "C++"

// `steps` second-order steps on the fused path at depth K (a remainder runs
// at a smaller depth), with the coefficients c and the phase table map tm.
ts_status fused_run(ts_grid *g, int64_t steps, int K, const ts::RotCoef &c,
                    const CUtensorMap *tm, cudaStream_t st, const double *drive_adt = nullptr)
{
    if (!g->tmaps_ok) return fail(TS_ERR_STATE, "fused path: tensor maps missing");
    int64_t left = steps;
    while (left > 0) {
        const int k = (int)(left >= K ? K : left);
        ts::FusedLaunch a;
        a.tm_state = &g->tm_state[g->cur];
        a.tm_phase = tm;
        a.out_re = (float *)g->re_other();
        a.out_im = (float *)g->im_other();
        a.nx = (int)g->L.nx;
        a.ny = (int)g->rows();
        a.pitch = g->L.pitch;
        a.t1 = (float)c.t1;
        a.s1 = (float)c.s1;
        a.g1 = (float)c.g1;
        a.t2 = (float)c.t2;
        a.s2 = (float)c.s2;
        a.err = g->err;
        cudaError_t e;
        if (drive_adt) {
            for (int i = 0; i < k; ++i) a.adt[i] = (float)drive_adt[steps - left + i];
            e = ts::launch_fused_drive(k, a, st);
        } else {
            e = ts::launch_fused(k, a, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
        g->cur ^= 1;
        left -= k;
    }
    return TS_OK;
}

ts::RotCoef grid_coef(const ts_grid *g) { return ts::RotCoef{g->g1, g->s1, g->t1, g->s2, g->t2}; }

ts_status plain_steps(ts_grid *g, int64_t steps, cudaStream_t st)
{
    return plain_run(g, steps, grid_coef(g), g->pg(), g->ps(), st);
}

ts_status fused_steps(ts_grid *g, int64_t steps, int K, cudaStream_t st)
{
    return fused_run(g, steps, K, grid_coef(g), &g->tm_phase, st);
}

// Fourth-order steps (Eq. fourthorder): the substeps a = U2(p dt) and
// b = U2((1-4p) dt) in the order a a b a a per step.  The a substeps of
// neighbouring steps run back to back (a run of 2 at either end, of 4
// between two b substeps), so on the fused path each run of r substeps is
// ceil(r / K) launches of near-equal depth; each b substep is one launch.
// 3-D steps on the fast path (FP32, |theta| <= pi/4, (nz + 32) ny < 2^31):
// one launch and one HBM round trip per step (fused.cu, fused3d_kernel).  Z
// factors commute with X and Y factors, so the step
//   Xe Xo Ye Yo Ze Zo P Zo Ze Yo Ye Xo Xe
// equals Ze Zo [Xe Xo Ye Yo P Yo Ye Xo Xe] Zo Ze: each slab runs the depth-1
// 2-D step with Y pairs kept inside it, its rows taking Ze, Zo as they enter
// and Zo, Ze as they leave, in trade with the neighbouring slabs' rows.
ts_status evolve3_fused(ts_grid *g, int64_t steps, cudaStream_t st)
{
    if (!g->tmaps_ok) return fail(TS_ERR_STATE, "fused path: tensor maps missing");
    const ts::RotCoef c = grid_coef(g);
    for (int64_t n = 0; n < steps; ++n) {
        ts::FusedLaunch a;
        a.tm_state = &g->tm_state[g->cur];
        a.tm_phase = &g->tm_phase;
        a.out_re = (float *)g->re_other();
        a.out_im = (float *)g->im_other();
        a.nx = (int)g->L.nx;
        a.ny = (int)g->L.ny;
        a.pitch = g->L.pitch;
        a.t1 = (float)c.t1;
        a.s1 = (float)c.s1;
        a.g1 = (float)c.g1;
        a.t2 = (float)c.t2;
        a.s2 = (float)c.s2;
        a.err = g->err;
        cudaError_t e = ts::launch_fused3d(a, (int)g->L.nz, st);
        if (e != cudaSuccess) return cuda_fail(e, "3-D fused kernel launch");
        g->cur ^= 1;
    }
    return TS_OK;
}

// Steps with the time-dependent potential V0 + a_n V1: the next `steps`
// amplitudes, each multiplied by dt; the fused kernel at depth <= 4 or, for
// ts_evolve_plain and FP32 grids with |theta| > pi/4, the plain path.
ts_status evolve_driven(ts_grid *g, int64_t steps, int K, bool plain, cudaStream_t st)
{
    const int64_t left = (int64_t)g->drive_a.size() - g->drive_pos;
    if (steps > left)
        return fail(TS_ERR_ARG, "ts_evolve: %lld steps asked for but %lld drive amplitudes are left",
                    (long long)steps, (long long)left);
    std::vector<double> adt((size_t)steps);
    for (int64_t i = 0; i < steps; ++i) adt[(size_t)i] = g->drive_a[(size_t)(g->drive_pos + i)] * g->dt;
    ts_status s;
    if (plain) {
        s = plain_run(g, steps, grid_coef(g), g->pg(), g->ps(), st, adt.data());
    } else {
        // depth 4 by default: with the drive phase computed per site the
        // kernel is arithmetic-bound, and 4 measured fastest (8192^2: 4.1e11
        // site-steps/s against 3.8e11 at depth 3)
        int depth = K == 0 ? ts::FUSED_DRIVE_MAX_K : K;
        if (depth > ts::FUSED_DRIVE_MAX_K) depth = ts::FUSED_DRIVE_MAX_K;
        s = fused_run(g, steps, depth, grid_coef(g), &g->tm_drive, st, adt.data());
    }
    if (s == TS_OK) g->drive_pos += steps;
    return s;
}

// Fourth-order steps, each one launch of the fused kernel over all five
// substeps a a b a a (the merged boundaries inside the step use the angles
// 2a, a + b, a + b, 2a; the a table streams through the phase ring, the b
// table through a shorter ring of its own): 32 B per site and U4 step.
ts_status fused_u4_steps(ts_grid *g, int64_t steps, cudaStream_t st)
{
    if (!g->tmaps_ok) return fail(TS_ERR_STATE, "fused path: tensor maps missing");
    const ts::RotCoef &A = g->sub[0], &B = g->sub[1];
    const double p4 = 1.0 / (4.0 - std::cbrt(4.0));
    const ts::RotCoef AB = ts::rot_coef((1.0 - 3.0 * p4) * g->theta);   // angle a + b
    for (int64_t n = 0; n < steps; ++n) {
        ts::FusedLaunch a;
        a.tm_state = &g->tm_state[g->cur];
        a.tm_phase = &g->tm_phase;
        a.tm_b = &g->tm_phase_b;
        a.out_re = (float *)g->re_other();
        a.out_im = (float *)g->im_other();
        a.nx = (int)g->L.nx;
        a.ny = (int)g->rows();
        a.pitch = g->L.pitch;
        a.t1 = (float)A.t1;
        a.s1 = (float)A.s1;
        a.g1 = (float)A.g1;
        a.t2 = (float)A.t2;
        a.s2 = (float)A.s2;
        a.tb = (float)B.t1;
        a.sb = (float)B.s1;
        a.gb = (float)B.g1;
        a.tab = (float)AB.t1;
        a.sab = (float)AB.s1;
        a.err = g->err;
        cudaError_t e = ts::launch_fused_u4(a, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused fourth-order launch");
        g->cur ^= 1;
    }
    return TS_OK;
}

ts_status evolve4(ts_grid *g, int64_t steps, int K, bool plain, cudaStream_t st)
{
    if (!plain && K == 0) return fused_u4_steps(g, steps, st);
    const int depth = K;
    auto run_a = [&](int64_t r) -> ts_status {
        if (plain) return plain_run(g, r, g->sub[0], g->pg(), g->ps(), st);
        const int64_t n = (r + depth - 1) / depth;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t k = r / n + (i < r % n ? 1 : 0);
            ts_status s = fused_run(g, k, (int)k, g->sub[0], &g->tm_phase, st);
            if (s != TS_OK) return s;
        }
        return TS_OK;
    };
    auto run_b = [&]() -> ts_status {
        if (plain) return plain_run(g, 1, g->sub[1], g->pg_b(), g->ps_b(), st);
        return fused_run(g, 1, 1, g->sub[1], &g->tm_phase_b, st);
    };
    ts_status s = run_a(2);
    for (int64_t n = 0; n < steps && s == TS_OK; ++n) {
        s = run_b();
        if (s == TS_OK) s = run_a(n + 1 < steps ? 4 : 2);
    }
    return s;
}

// ts_evolve on FP64 grids: the merged sweep sequence for every kind of step
// (second order, 3-D, fourth order, time-dependent potential).
ts_status evolve_f64(ts_grid *g, int64_t steps, cudaStream_t st)
{
    if (g->driven) {
        const int64_t left = (int64_t)g->drive_a.size() - g->drive_pos;
        if (steps > left)
            return fail(TS_ERR_ARG,
                        "ts_evolve: %lld steps asked for but %lld drive amplitudes are left",
                        (long long)steps, (long long)left);
        const int64_t pos = g->drive_pos;
        ts_status s = merged_run(g, steps, [&](int64_t i) {
            return Substep{g->theta, g->pg(), g->ps(), true,
                           g->drive_a[(size_t)(pos + i)] * g->dt};
        }, st);
        if (s == TS_OK) g->drive_pos += steps;
        return s;
    }
    if (g->order == 4) {   // substeps a a b a a per step
        const double p4 = 1.0 / (4.0 - std::cbrt(4.0));
        const Substep a = {p4 * g->theta, g->pg(), g->ps(), false, 0.0};
        const Substep b = {(1.0 - 4.0 * p4) * g->theta, g->pg_b(), g->ps_b(), false, 0.0};
        return merged_run(g, 5 * steps, [&](int64_t i) { return i % 5 == 2 ? b : a; }, st);
    }
    const Substep u = {g->theta, g->pg(), g->ps(), false, 0.0};
    return merged_run(g, steps, [&](int64_t) { return u; }, st);
}

}  // namespace

ts_status ts_evolve(ts_grid *g, int64_t steps, int K, void *stream)
{
    ts::TraceRange trace_("ts_evolve");
    if (!g) return fail(TS_ERR_ARG, "ts_evolve: grid is NULL");
    if (steps < 0) return fail(TS_ERR_ARG, "ts_evolve: negative step count");
    if (K < 0 || K > ts::FUSED_MAX_K) return fail(TS_ERR_ARG, "ts_evolve: K must be in [0, 8]");
    if (steps == 0) return TS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (g->f64()) {
        if (K != 0)
            return fail(TS_ERR_UNSUPPORTED,
                        "ts_evolve: FP64 grids run one sweep per launch (K must be 0)");
        return evolve_f64(g, steps, st);
    }
    if (g->is3d()) {
        // (TMA row coordinates reach about (nz + 2 W - 3) ny for a block of W
        // warps, W <= 16: the last z-block's halo slabs)
        if (std::fabs(g->theta) > 0.25 * M_PI || (g->L.nz + 32) * g->L.ny >= (int64_t(1) << 31))
            return plain_steps(g, steps, st);
        return evolve3_fused(g, steps, st);
    }
    if (g->driven) return evolve_driven(g, steps, K, std::fabs(g->theta) > 0.25 * M_PI, st);
    if (g->order == 4) {
        // the substep angles p theta and (1-4p) theta must both suit the fused kernel
        const double p4 = 1.0 / (4.0 - std::cbrt(4.0));
        const bool plain = std::fabs(g->theta) * std::fabs(1.0 - 4.0 * p4) > 0.25 * M_PI;
        return evolve4(g, steps, K, plain, st);
    }
    // The fused kernel applies the rotations at theta and 2 theta as three
    // shears with tan(theta/2) and tan(theta); it requires |theta| <= pi/4
    // (|2 theta| <= pi/2).  Larger angles -- far beyond any useful Trotter
    // step -- run the one-sweep-per-kernel path.
    if (std::fabs(g->theta) > 0.25 * M_PI) return plain_steps(g, steps, st);
    return fused_steps(g, steps, K == 0 ? auto_depth() : K, st);
}

ts_status ts_check_wait_timeout(ts_grid *g, int64_t limit_ns, void *stream)
{
    if (!g) return fail(TS_ERR_ARG, "ts_check_wait_timeout: grid is NULL");
    if (limit_ns < 1000 || limit_ns > 2000000000)
        return fail(TS_ERR_ARG, "ts_check_wait_timeout: limit_ns must be in [1e3, 2e9], got %lld",
                    (long long)limit_ns);
    cudaError_t e = ts::launch_wait_timeout_check(g->err, (uint64_t)limit_ns, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "wait-timeout check launch");
    return TS_OK;
}

ts_status ts_evolve_plain(ts_grid *g, int64_t steps, void *stream)
{
    ts::TraceRange trace_("ts_evolve_plain");
    if (!g) return fail(TS_ERR_ARG, "ts_evolve_plain: grid is NULL");
    if (steps < 0) return fail(TS_ERR_ARG, "ts_evolve_plain: negative step count");
    if (steps == 0) return TS_OK;
    if (g->driven) return evolve_driven(g, steps, 0, true, (cudaStream_t)stream);
    if (g->order == 4) return evolve4(g, steps, 0, true, (cudaStream_t)stream);
    return plain_steps(g, steps, (cudaStream_t)stream);
}

ts_status ts_evolve_batched(ts_grid *const *gs, int n, const int64_t *steps, int K, void *stream)
{
    ts::TraceRange trace_("ts_evolve_batched");
    if (n < 0 || (n > 0 && (!gs || !steps))) return fail(TS_ERR_ARG, "ts_evolve_batched: bad arguments");
    if (K < 0 || K > ts::FUSED_MAX_K) return fail(TS_ERR_ARG, "ts_evolve_batched: K must be in [0, 8]");
    cudaStream_t st = (cudaStream_t)stream;
    const int depth = K == 0 ? auto_depth() : K;
    // grids the multi-grid kernel can take: 2-D, FP32, second order, no
    // drive, |theta| <= pi/4; the rest evolve one by one
    std::vector<ts_grid *> multi;
    std::vector<int64_t> msteps;
    for (int i = 0; i < n; ++i) {
        if (!gs[i] || steps[i] < 0) return fail(TS_ERR_ARG, "ts_evolve_batched: grid %d", i);
        if (steps[i] == 0) continue;
        if (gs[i]->f64() || gs[i]->order != 2 || gs[i]->driven || gs[i]->is3d() ||
            std::fabs(gs[i]->theta) > 0.25 * M_PI) {
            // K is the fused FP32 depth; FP64 grids take their own sequence
            ts_status s = ts_evolve(gs[i], steps[i], gs[i]->f64() ? 0 : K, stream);
            if (s != TS_OK) return s;
        } else {
            multi.push_back(gs[i]);
            msteps.push_back(steps[i]);
        }
    }
    cudaError_t e = ts::evolve_multi(multi.data(), msteps.data(), (int)multi.size(), depth, st);
    if (e != cudaSuccess) return cuda_fail(e, "ts_evolve_batched: multi-grid launch");
    return TS_OK;
}

namespace {

// res: OBS_Q3 doubles; 2-D grids fill the first OBS_Q and zero the rest.
ts_status observe(ts_grid *g, bool norm_only, double *res, cudaStream_t st)
{
    cudaError_t e;
    int nq = ts::OBS_Q;
    for (int q = 0; q < ts::OBS_Q3; ++q) res[q] = 0.0;
    if (g->is3d() && !norm_only) {
        e = ts::launch_observe3(g->re(), g->im(), g->vp(), g->f64(), (int)g->L.nx, (int)g->L.ny,
                                (int)g->L.nz, g->L.pitch, g->J, g->partials, g->result, st);
        nq = ts::OBS_Q3;
    } else {
        // the norm needs no geometry: a 3-D grid is ny*nz rows of sites
        e = ts::launch_observe(g->re(), g->im(), g->vp(), g->f64(), (int)g->L.nx,
                               (int)g->rows(), g->L.pitch, g->J, norm_only, g->partials,
                               g->result, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "observables kernel");
    e = cudaMemcpyAsync(res, g->result, sizeof(double) * nq, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "observables copy");
    return check_errword(g, st);
}

}  // namespace

ts_status ts_observe(ts_grid *g, ts_observables *out, void *stream)
{
    ts::TraceRange trace_("ts_observe");
    if (!g || !out) return fail(TS_ERR_ARG, "ts_observe: null argument");
    double r[ts::OBS_Q3];
    ts_status s = observe(g, false, r, (cudaStream_t)stream);
    if (s != TS_OK) return s;
    out->norm = r[0];
    const double inv = r[0] != 0.0 ? 1.0 / r[0] : 0.0;
    out->x = r[1] * inv;
    out->y = r[2] * inv;
    out->x2 = r[3] * inv;
    out->y2 = r[4] * inv;
    out->e_kin = r[5];
    out->e_pot = r[6];
    out->z = r[7] * inv;
    out->z2 = r[8] * inv;
    return TS_OK;
}

ts_status ts_norm(ts_grid *g, double *out, void *stream)
{
    ts::TraceRange trace_("ts_norm");
    if (!g || !out) return fail(TS_ERR_ARG, "ts_norm: null argument");
    double r[ts::OBS_Q3];
    ts_status s = observe(g, true, r, (cudaStream_t)stream);
    if (s != TS_OK) return s;
    *out = r[0];
    return TS_OK;
}

ts_status ts_expect_xy(ts_grid *g, double *x, double *y, void *stream)
{
    if (!g || !x || !y) return fail(TS_ERR_ARG, "ts_expect_xy: null argument");
    ts_observables o;
    ts_status s = ts_observe(g, &o, stream);
    if (s != TS_OK) return s;
    *x = o.x;
    *y = o.y;
    return TS_OK;
}

ts_status ts_energy(ts_grid *g, double *out, void *stream)
{
    if (!g || !out) return fail(TS_ERR_ARG, "ts_energy: null argument");
    ts_observables o;
    ts_status s = ts_observe(g, &o, stream);
    if (s != TS_OK) return s;
    *out = o.e_kin + o.e_pot;
    return TS_OK;
}

}  // extern "C"
