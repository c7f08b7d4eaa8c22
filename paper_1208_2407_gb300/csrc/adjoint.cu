// Gradient of the fidelity F = |<phi|psi_T>|^2 with respect to the potential
// V on every site, psi_T = U2(dt)^n psi_0 (Sec. 2, Eq. secondorder).
//
// Write one step as psi_s = B P A psi_{s-1} (A: the first four sweeps, P the
// phase exp(-i V dt), B: the last four).  With c = <phi|psi_T>, the costate
// lambda_n = phi, lambda_{s-1} = U_s^dagger lambda_s, the mid-step state
// m_s = P A psi_{s-1} and lt_s = B^dagger lambda_s,
//   dF/dV_j = 2 dt Im( conj(c) G_j ),   G_j = sum_s conj(lt_s[j]) m_s[j].
// U^dagger is the same sweep sequence at -theta with the conjugate phase, and
// lt_s is its state at the phase point, so a backward step is the fused K = 1
// step at -theta with a hook there (fused.cu, mode 2).
//
// Checkpointing: the forward keeps psi every `ckpt` steps; the backward walks
// the segments from the last, recomputes each segment's mid-step states from
// its checkpoint (fused.cu, mode 1) and then steps the costate back through it.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "../../include/trotter.h"
#include "ffloat.cuh"
#include "grid.h"
#include "internal.h"
#include "trace.h"

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace planes, each of the grid's plane size.
enum : int {
    WS_T = 0,      // target phi: re, im
    WS_LA = 2,     // costate ping-pong pair A: re, im
    WS_LB = 4,     // ... pair B
    WS_RA = 6,     // recomputation ping-pong pair A
    WS_RB = 8,     // ... pair B
    WS_G = 10,     // G as double-float: re hi, re lo, im hi, im lo
    WS_CK = 14     // checkpoints (2 planes each), then the mid-step states
};

struct WsLayout {
    int64_t n_ck;          // checkpoints: psi at steps 0, ckpt, 2 ckpt, ...
    int64_t n_planes;
    size_t scratch_off;    // partials and result of the overlap reduction
    size_t bytes;
};

WsLayout ws_layout(const ts_grid *g, int64_t steps, int64_t ckpt)
{
    WsLayout w;
    w.n_ck = (steps + ckpt - 1) / ckpt;
    if (w.n_ck < 1) w.n_ck = 1;
    w.n_planes = WS_CK + 2 * w.n_ck + 2 * ckpt;
    w.scratch_off = (size_t)w.n_planes * g->L.plane_bytes;
    w.bytes = w.scratch_off + round_up(sizeof(double) * ts::OBS_MAX_BLOCKS * ts::OBS_Q, 256) +
              round_up(sizeof(double) * ts::OBS_Q, 256);
    return w;
}

ts_status err(ts_status s, const char *fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return (ts_status)ts::set_error(s, "%s", buf);
}

ts_status cuda_err(cudaError_t e, const char *what)
{
    return err(TS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// grad[y*nx + x] = 2 dt Im(conj(c) G) = 2 dt (c_re G_im - c_im G_re)
__global__ void grad_finalize_kernel(const float *__restrict__ g_rh, const float *__restrict__ g_rl,
                                     const float *__restrict__ g_ih, const float *__restrict__ g_il,
                                     int nx, int ny, int64_t pitch, double c_re, double c_im,
                                     double two_dt, float *__restrict__ grad)
{
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / nx, x = i - y * nx, o = y * pitch + x;
        const double gr = (double)g_rh[o] + (double)g_rl[o];
        const double gi = (double)g_ih[o] + (double)g_il[o];
        grad[i] = (float)(two_dt * (c_re * gi - c_im * gr));
    }
}

struct AdjointState {
    const void *ws = nullptr;
    int64_t steps = 0, ckpt = 0;
    double c_re = 0.0, c_im = 0.0;
};

// Per-grid record of the last forward pass (one adjoint in flight per grid).
std::mutex g_adj_mu;
std::unordered_map<const ts_grid *, AdjointState> g_adj;
}  // namespace

extern "C" {

ts_status ts_adjoint_workspace(const ts_grid *g, int64_t steps, int64_t ckpt_every, size_t *bytes)
{
    if (!g || !bytes) return err(TS_ERR_ARG, "ts_adjoint_workspace: null argument");
    if (steps < 1 || ckpt_every < 1)
        return err(TS_ERR_ARG, "ts_adjoint_workspace: steps and ckpt_every must be >= 1");
    *bytes = ws_layout(g, steps, ckpt_every).bytes;
    return TS_OK;
}

ts_status ts_adjoint_forward(ts_grid *g, const void *target_re, const void *target_im,
                             ts_dtype target_dtype, ts_mem where, int64_t steps,
                             int64_t ckpt_every, void *ws, size_t ws_bytes, double *fidelity,
                             double *overlap, void *stream)
{
    ts::TraceRange trace_("ts_adjoint_forward");
    if (!g || !target_re || !target_im || !ws || !fidelity)
        return err(TS_ERR_ARG, "ts_adjoint_forward: null argument");
    if (g->f64()) return err(TS_ERR_UNSUPPORTED, "ts_adjoint_forward: FP32 grids only");
    if (g->order != 2 || g->driven || g->is3d())
        return err(TS_ERR_UNSUPPORTED,
                   "ts_adjoint_forward: second-order 2-D grids with a static potential only");
    if (std::fabs(g->theta) > 0.25 * M_PI)
        return err(TS_ERR_UNSUPPORTED, "ts_adjoint_forward: |theta| must be <= pi/4");
    if (steps < 1 || ckpt_every < 1)
        return err(TS_ERR_ARG, "ts_adjoint_forward: steps and ckpt_every must be >= 1");
    if (target_dtype != TS_F32 && target_dtype != TS_F64)
        return err(TS_ERR_ARG, "ts_adjoint_forward: unknown dtype");
    if (where != TS_HOST && where != TS_DEVICE)
        return err(TS_ERR_ARG, "ts_adjoint_forward: unknown memory kind");
    const WsLayout w = ws_layout(g, steps, ckpt_every);
    if (ws_bytes < w.bytes || ((uintptr_t)ws & 255u))
        return err(TS_ERR_ARG, "ts_adjoint_forward: workspace needs %zu bytes, 256-aligned", w.bytes);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = (unsigned char *)ws;
    const size_t PB = g->L.plane_bytes;
    auto plane = [&](int64_t i) { return (void *)(base + (size_t)i * PB); };
    const int nx = (int)g->L.nx, ny = (int)g->L.ny;
    const int64_t pitch = g->L.pitch;
    const bool f64 = target_dtype == TS_F64;
    cudaError_t e = cudaSuccess;

    // target -> planes T (host input staged through the costate planes)
    const void *src[2] = {target_re, target_im};
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        const void *s = src[c];
        if (where == TS_HOST) {
            const size_t nbytes = (size_t)nx * ny * (f64 ? 8 : 4);
            e = cudaMemcpyAsync(plane(WS_LA), s, nbytes, cudaMemcpyHostToDevice, st);
            s = plane(WS_LA);
        }
        if (e == cudaSuccess)
            e = ts::launch_convert_in(s, f64, plane(WS_T + c), false, nx, ny, pitch, st);
        if (e == cudaSuccess && where == TS_HOST) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: target");

    // forward with checkpoints (psi at steps 0, ckpt, 2 ckpt, ...)
    for (int64_t k = 0; k < w.n_ck; ++k) {
        e = cudaMemcpyAsync(plane(WS_CK + 2 * k), g->re(), 2 * PB, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: checkpoint");
        const int64_t n = std::min(ckpt_every, steps - k * ckpt_every);
        ts_status s = ts_evolve(g, n, 0, stream);
        if (s != TS_OK) return s;
    }

    // c = <phi|psi_T>
    double *partials = (double *)(base + w.scratch_off);
    double *result = (double *)(base + w.scratch_off +
                                round_up(sizeof(double) * ts::OBS_MAX_BLOCKS * ts::OBS_Q, 256));
    e = ts::launch_inner((const float *)plane(WS_T), (const float *)plane(WS_T + 1),
                         (const float *)g->re(), (const float *)g->im(), nx, ny, pitch, partials,
                         result, st);
    double c[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(c, result, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: overlap");
    int h = 0;
    e = cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: error word");
    if (h) {
        cudaMemset(g->err, 0, sizeof(int));
        return err(TS_ERR_TIMEOUT, "ts_adjoint_forward: a bounded wait gave up (error word %d)", h);
    }
    *fidelity = c[0] * c[0] + c[1] * c[1];
    if (overlap) {
        overlap[0] = c[0];
        overlap[1] = c[1];
    }
    std::lock_guard<std::mutex> lk(g_adj_mu);
    AdjointState &a = g_adj[g];
    a.ws = ws;
    a.steps = steps;
    a.ckpt = ckpt_every;
    a.c_re = c[0];
    a.c_im = c[1];
    return TS_OK;
}

ts_status ts_adjoint_backward(ts_grid *g, void *ws, size_t ws_bytes, float *grad, void *stream)
{
    ts::TraceRange trace_("ts_adjoint_backward");
    if (!g || !ws || !grad) return err(TS_ERR_ARG, "ts_adjoint_backward: null argument");
    AdjointState a;
    {
        std::lock_guard<std::mutex> lk(g_adj_mu);
        auto it = g_adj.find(g);
        if (it == g_adj.end() || it->second.ws != ws)
            return err(TS_ERR_STATE, "ts_adjoint_backward: no forward pass with this workspace");
        a = it->second;
    }
    const WsLayout w = ws_layout(g, a.steps, a.ckpt);
    if (ws_bytes < w.bytes) return err(TS_ERR_ARG, "ts_adjoint_backward: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = (unsigned char *)ws;
    const size_t PB = g->L.plane_bytes;
    auto plane = [&](int64_t i) { return (void *)(base + (size_t)i * PB); };
    const int nx = (int)g->L.nx, ny = (int)g->L.ny;
    const int64_t pitch = g->L.pitch;

    CUtensorMap tmL[2], tmR[2];
    const char *why = "";
    if (!ts::make_pair_tensor_map(&tmL[0], plane(WS_LA), nx, ny, pitch, PB, &why) ||
        !ts::make_pair_tensor_map(&tmL[1], plane(WS_LB), nx, ny, pitch, PB, &why) ||
        !ts::make_pair_tensor_map(&tmR[0], plane(WS_RA), nx, ny, pitch, PB, &why) ||
        !ts::make_pair_tensor_map(&tmR[1], plane(WS_RB), nx, ny, pitch, PB, &why))
        return err(TS_ERR_CUDA, "ts_adjoint_backward: %s", why);

    cudaError_t e = cudaMemcpyAsync(plane(WS_LA), plane(WS_T), 2 * PB, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(plane(WS_G), 0, 4 * PB, st);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: set-up");

    ts::FusedLaunch fw;
    fw.tm_phase = &g->tm_phase;
    fw.nx = nx;
    fw.ny = ny;
    fw.pitch = pitch;
    fw.err = g->err;
    ts::FusedLaunch bw = fw;
    fw.t1 = (float)g->t1;   // forward recomputation at +theta
    fw.s1 = (float)g->s1;
    fw.g1 = (float)g->g1;
    fw.t2 = (float)g->t2;
    fw.s2 = (float)g->s2;
    bw.t1 = -(float)g->t1;  // backward steps U^dagger at -theta
    bw.s1 = -(float)g->s1;
    bw.g1 = (float)g->g1;
    bw.t2 = -(float)g->t2;
    bw.s2 = -(float)g->s2;
    bw.g_rh = (float *)plane(WS_G);
    bw.g_rl = (float *)plane(WS_G + 1);
    bw.g_ih = (float *)plane(WS_G + 2);
    bw.g_il = (float *)plane(WS_G + 3);

    int lc = 0;   // costate in pair lc (0: LA, 1: LB)
    const int64_t mid0 = WS_CK + 2 * w.n_ck;
    for (int64_t k = w.n_ck - 1; k >= 0; --k) {
        const int64_t n = std::min(a.ckpt, a.steps - k * a.ckpt);
        e = cudaMemcpyAsync(plane(WS_RA), plane(WS_CK + 2 * k), 2 * PB, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: restore checkpoint");
        int rc = 0;
        for (int64_t i = 0; i < n; ++i) {        // recompute m_s for the segment
            fw.tm_state = &tmR[rc];
            fw.out_re = (float *)plane(rc ? WS_RA : WS_RB);
            fw.out_im = (float *)plane((rc ? WS_RA : WS_RB) + 1);
            fw.m_re = (float *)plane(mid0 + 2 * i);
            fw.m_im = (float *)plane(mid0 + 2 * i + 1);
            e = ts::launch_fused_mid(1, fw, st);
            if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: recompute launch");
            rc ^= 1;
        }
        for (int64_t i = n - 1; i >= 0; --i) {   // costate back through the segment
            bw.tm_state = &tmL[lc];
            bw.out_re = (float *)plane(lc ? WS_LA : WS_LB);
            bw.out_im = (float *)plane((lc ? WS_LA : WS_LB) + 1);
            bw.m_re = (float *)plane(mid0 + 2 * i);
            bw.m_im = (float *)plane(mid0 + 2 * i + 1);
            e = ts::launch_fused_mid(2, bw, st);
            if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: backward launch");
            lc ^= 1;
        }
    }
    const int64_t sites = (int64_t)nx * ny;
    int blocks = (int)std::min<int64_t>((sites + 255) / 256, 152 * 32);
    grad_finalize_kernel<<<blocks, 256, 0, st>>>(
        (const float *)plane(WS_G), (const float *)plane(WS_G + 1), (const float *)plane(WS_G + 2),
        (const float *)plane(WS_G + 3), nx, ny, pitch, a.c_re, a.c_im, 2.0 * g->dt, grad);
    ts::count_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward");
    int h = 0;
    e = cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: error word");
    if (h) {
        cudaMemset(g->err, 0, sizeof(int));
        return err(TS_ERR_TIMEOUT, "ts_adjoint_backward: a bounded wait gave up (error word %d)", h);
    }
    return TS_OK;
}

ts_status ts_adjoint_grad(ts_grid *g, const void *target_re, const void *target_im,
                          ts_dtype target_dtype, ts_mem where, int64_t steps, int64_t ckpt_every,
                          void *ws, size_t ws_bytes, float *grad, double *fidelity, void *stream)
{
    ts_status s = ts_adjoint_forward(g, target_re, target_im, target_dtype, where, steps,
                                     ckpt_every, ws, ws_bytes, fidelity, nullptr, stream);
    if (s != TS_OK) return s;
    return ts_adjoint_backward(g, ws, ws_bytes, grad, stream);
}

}  // extern "C"

// A destroyed grid must not leave a stale record behind.
namespace ts {
void forget_adjoint(const ts_grid *g)
{
    std::lock_guard<std::mutex> lk(g_adj_mu);
    g_adj.erase(g);
}
}  // namespace ts
