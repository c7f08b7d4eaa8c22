// Gradient of the fidelity F = |<phi|psi_T>|^2 with respect to the potential
// V on every site, psi_T = U2(dt)^n psi_0 (Sec. 2, Eq. secondorder).
//
// Write one step as psi_s = B P A psi_{s-1} (A: the first four sweeps, P the
// phase exp(-i V dt), B: the last four).  With c = <phi|psi_T>, the costate
// lambda_n = phi, lambda_{s-1} = U_s^dagger lambda_s, the mid-step state
// m_s = P A psi_{s-1} and lt_s = B^dagger lambda_s,
//   dF/dV_j = 2 dt Im( conj(c) G_j ),   G_j = sum_s conj(lt_s[j]) m_s[j].
// U^dagger is the same sweep sequence at -theta with the conjugate phase, and
// lt_s is its state at the phase point.  The mid-step state is the forward
// state's value at the same point, m_s = P A psi_{s-1} = B^dagger psi_s, so
// the backward pass carries psi back with the costate: K backward steps are
// one fused launch at -theta over both states (fused.cu, mode 5), which adds
// conj(lt_s) m_s at every phase point; G's double-float planes are read and
// written once per launch, and nothing is recomputed or stored per step.
//
// Checkpointing: the forward keeps psi at the end of every segment of `ckpt`
// steps; the backward walks the segments from the last, restarting psi from
// the segment's checkpoint, so that the FP32 rounding of psi stepped
// backward accumulates over at most one segment.
//
// Bytes per site and step (FP32, K steps per launch): 72/K for the backward
// launches (psi and lambda read and written, 32; the table, 8; G read and
// written, 32), plus 16 per segment for the checkpoint.  The forward pass is
// ts_evolve plus one checkpoint copy (16 B) per segment.
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

#ifndef TS_ADJ_DEFAULT_K      // fused depth of the backward launches
#define TS_ADJ_DEFAULT_K 3
#endif

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace planes, each of the grid's plane size.
enum : int {
    WS_T = 0,      // target phi: re, im
    WS_QA = 2,     // backward ping-pong quad A: psi re, im, lambda re, im
    WS_QB = 6,     // ... quad B
    WS_G = 10,     // G as double-float: re hi, re lo, im hi, im lo
    WS_CK = 14     // checkpoints, 2 planes each
};

struct WsLayout {
    int64_t n_ck;          // checkpoints: psi at steps ckpt, 2 ckpt, ..., steps
    int64_t n_planes;
    size_t scratch_off;    // partials and result of the overlap reduction
    size_t bytes;
};

WsLayout ws_layout(const ts_grid *g, int64_t steps, int64_t ckpt)
{
    WsLayout w;
    w.n_ck = (steps + ckpt - 1) / ckpt;
    if (w.n_ck < 1) w.n_ck = 1;
    w.n_planes = WS_CK + 2 * w.n_ck;
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
            e = cudaMemcpyAsync(plane(WS_QA), s, nbytes, cudaMemcpyHostToDevice, st);
            s = plane(WS_QA);
        }
        if (e == cudaSuccess)
            e = ts::launch_convert_in(s, f64, plane(WS_T + c), false, nx, ny, pitch, st);
        if (e == cudaSuccess && where == TS_HOST) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: target");

    // forward with checkpoints (psi at the end of each segment: steps ckpt,
    // 2 ckpt, ..., steps)
    for (int64_t k = 0; k < w.n_ck; ++k) {
        const int64_t n = std::min(ckpt_every, steps - k * ckpt_every);
        ts_status s = ts_evolve(g, n, 0, stream);
        if (s != TS_OK) return s;
        e = cudaMemcpyAsync(plane(WS_CK + 2 * k), g->re(), 2 * PB, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_forward: checkpoint");
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

ts_status ts_adjoint_backward_depth(ts_grid *g, void *ws, size_t ws_bytes, int K, float *grad,
                                    void *stream)
{
    ts::TraceRange trace_("ts_adjoint_backward");
    if (!g || !ws || !grad) return err(TS_ERR_ARG, "ts_adjoint_backward: null argument");
    if (K < 0 || K > ts::FUSED_ADJ_MAX_K)
        return err(TS_ERR_ARG, "ts_adjoint_backward: depth K must be in [0, %d]",
                   ts::FUSED_ADJ_MAX_K);
    const int KA = K > 0 ? K : TS_ADJ_DEFAULT_K;
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

    // the two quads (psi, lambda)
    CUtensorMap tmQ[2];
    const char *why = "";
    if (!ts::make_pair_tensor_map(&tmQ[0], plane(WS_QA), nx, ny, pitch, PB, &why, 4) ||
        !ts::make_pair_tensor_map(&tmQ[1], plane(WS_QB), nx, ny, pitch, PB, &why, 4))
        return err(TS_ERR_CUDA, "ts_adjoint_backward: %s", why);

    // lambda_T = phi (in quad A), G = 0
    cudaError_t e =
        cudaMemcpyAsync(plane(WS_QA + 2), plane(WS_T), 2 * PB, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(plane(WS_G), 0, 4 * PB, st);
    if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: set-up");

    ts::FusedLaunch bw;
    bw.tm_phase = &g->tm_phase;
    bw.nx = nx;
    bw.ny = ny;
    bw.pitch = pitch;
    bw.err = g->err;
    bw.t1 = -(float)g->t1;  // backward steps U^dagger at -theta
    bw.s1 = -(float)g->s1;
    bw.g1 = (float)g->g1;
    bw.t2 = -(float)g->t2;
    bw.s2 = -(float)g->s2;
    bw.g_rh = (float *)plane(WS_G);
    bw.g_rl = (float *)plane(WS_G + 1);
    bw.g_ih = (float *)plane(WS_G + 2);
    bw.g_il = (float *)plane(WS_G + 3);

    int q = 0;   // psi and lambda in quad q (0: QA, 1: QB)
    auto quad = [&](int i) { return i ? WS_QB : WS_QA; };
    for (int64_t k = w.n_ck - 1; k >= 0; --k) {
        const int64_t n = std::min(a.ckpt, a.steps - k * a.ckpt);
        // psi at the end of segment k, beside the costate
        e = cudaMemcpyAsync(plane(quad(q)), plane(WS_CK + 2 * k), 2 * PB, cudaMemcpyDeviceToDevice,
                            st);
        if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: restore checkpoint");
        for (int64_t i = n; i > 0;) {            // steps i, i - 1, ..., i - kk + 1 of the segment
            const int kk = (int)std::min<int64_t>(KA, i);
            bw.tm_state = &tmQ[q];
            bw.out_re = (float *)plane(quad(q ^ 1));
            bw.out_im = (float *)plane(quad(q ^ 1) + 1);
            bw.out2_re = (float *)plane(quad(q ^ 1) + 2);
            bw.out2_im = (float *)plane(quad(q ^ 1) + 3);
            e = ts::launch_fused_adjoint(kk, bw, st);
            if (e != cudaSuccess) return cuda_err(e, "ts_adjoint_backward: backward launch");
            q ^= 1;
            i -= kk;
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

ts_status ts_adjoint_backward(ts_grid *g, void *ws, size_t ws_bytes, float *grad, void *stream)
{
    return ts_adjoint_backward_depth(g, ws, ws_bytes, 0, grad, stream);
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
