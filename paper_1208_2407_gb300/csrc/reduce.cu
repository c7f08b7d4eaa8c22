// Observables of the state: norm (Sec. 2: conserved by the unitary
// evolution), position moments and the energy <psi|H|psi> of the
// tight-binding Hamiltonian H = -J * (nearest-neighbour hops) + diag(V).
//
// FP32 grids: every product is formed exactly (two_prod) and each thread
// accumulates in double-float (hi + lo floats, ~48 significant bits) on the
// FP32 pipe; the per-thread sums are converted to FP64 once and combined
// across threads and blocks with Neumaier's compensated update.  (This
// GB300 runs FP64 at ~1/67 of the FP32 rate, so per-site FP64 work would
// make the reduction several times slower than one pass over HBM.)
// FP64 grids: every term in FP64; each thread sums a run of 4 sites in
// plain FP64 and adds the run into Neumaier-compensated per-thread sums.
// Either way the block writes FP64 partials and a final block sums them.
#include "common.cuh"
#include "ffloat.cuh"
#include "internal.h"
#include "walk.cuh"

namespace ts {

namespace {

constexpr int kThreads = 256;

struct Neu {
    double s, c;
    __device__ __forceinline__ void add(double v)
    {
        double t = s + v;
        c += (fabs(s) >= fabs(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ __forceinline__ double val() const { return s + c; }
};

// Merge two compensated sums (a += b).
__device__ __forceinline__ void neu_merge(Neu &a, const Neu &b)
{
    a.add(b.s);
    a.c += b.c;
}

// Block-level Neumaier reduction of NQ per-thread sums into partials.
template <int NQ>
__device__ __forceinline__ void block_reduce_write(Neu (&acc)[NQ], double *__restrict__ partials)
{
    __shared__ double sh_s[kThreads / 32][NQ], sh_c[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        Neu a = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Neu b;
            b.s = __shfl_down_sync(0xffffffffu, a.s, off);
            b.c = __shfl_down_sync(0xffffffffu, a.c, off);
            neu_merge(a, b);
        }
        if (lane == 0) {
            sh_s[warp][q] = a.s;
            sh_c[warp][q] = a.c;
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Neu a = {0.0, 0.0};
            if (lane < kThreads / 32) a = {sh_s[lane][q], sh_c[lane][q]};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                Neu b;
                b.s = __shfl_down_sync(0xffffffffu, a.s, off);
                b.c = __shfl_down_sync(0xffffffffu, a.c, off);
                neu_merge(a, b);
            }
            if (lane == 0) partials[(int64_t)blockIdx.x * OBS_Q + q] = a.val();
        }
    }
}

// FP32 state: exact products, double-float per-thread sums.  A thread takes
// chunks of 4 consecutive sites of one row (x0 a multiple of 4; the row
// pitch is a multiple of 32 floats, so the float4 loads stay inside the
// row's padding and columns >= nx are masked).
template <bool NORM_ONLY>
__global__ void __launch_bounds__(kThreads)
observe_f32_kernel(const float *__restrict__ re, const float *__restrict__ im,
                   const float *__restrict__ vp, int nx, int ny, int64_t pitch, float J_hi,
                   float J_lo, double *__restrict__ partials)
{
    constexpr int NQ = NORM_ONLY ? 1 : OBS_Q;
    FF acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = ff_make(0.f);

    const int chunks_per_row = (nx + 3) / 4;
    const int64_t nchunks = (int64_t)chunks_per_row * ny;
    for (Walk w(chunks_per_row, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < nchunks; w.next()) {
        const int y = (int)w.y;
        const int x0 = (int)w.x * 4;
        const int64_t o = (int64_t)y * pitch + x0;
        const float4 r4 = *reinterpret_cast<const float4 *>(re + o);
        const float4 m4 = *reinterpret_cast<const float4 *>(im + o);
        const float r[4] = {r4.x, r4.y, r4.z, r4.w}, m[4] = {m4.x, m4.y, m4.z, m4.w};
        FF P = ff_make(0.f), XP = ff_make(0.f), X2P = ff_make(0.f), KIN = ff_make(0.f),
           VP = ff_make(0.f);
        if constexpr (NORM_ONLY) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (x0 + u < nx)
                    P = ff_add(P, ff_add(two_prod(r[u], r[u]), two_prod(m[u], m[u])));
            }
            acc[0] = ff_add(acc[0], P);
        } else {
            const float4 v4 = *reinterpret_cast<const float4 *>(vp + o);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
            float rd[4] = {0.f, 0.f, 0.f, 0.f}, md[4] = {0.f, 0.f, 0.f, 0.f};
            if (y + 1 < ny) {
                const float4 a = *reinterpret_cast<const float4 *>(re + o + pitch);
                const float4 b = *reinterpret_cast<const float4 *>(im + o + pitch);
                rd[0] = a.x; rd[1] = a.y; rd[2] = a.z; rd[3] = a.w;
                md[0] = b.x; md[1] = b.y; md[2] = b.z; md[3] = b.w;
            }
            const float r_next = (x0 + 4 < nx) ? re[o + 4] : 0.f;
            const float m_next = (x0 + 4 < nx) ? im[o + 4] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (x0 + u >= nx) break;
                const FF p = ff_add(two_prod(r[u], r[u]), two_prod(m[u], m[u]));
                P = ff_add(P, p);
                XP = ff_add(XP, ff_mul_f(p, (float)u));
                X2P = ff_add(X2P, ff_mul_f(p, (float)(u * u)));
                VP = ff_add(VP, ff_mul_f(p, v[u]));
                // bonds to the right and downward neighbours
                const float rr = (u < 3) ? r[u + 1] : r_next, mr = (u < 3) ? m[u + 1] : m_next;
                if (x0 + u + 1 < nx) {
                    KIN = ff_add(KIN, two_prod(r[u], rr));
                    KIN = ff_add(KIN, two_prod(m[u], mr));
                }
                if (y + 1 < ny) {
                    KIN = ff_add(KIN, two_prod(r[u], rd[u]));
                    KIN = ff_add(KIN, two_prod(m[u], md[u]));
                }
            }
            const float fx0 = (float)x0, fy = (float)y;   // exact: sides <= 2^20
            acc[0] = ff_add(acc[0], P);
            // sum x p = x0 P + sum u p ; sum x^2 p = x0^2 P + 2 x0 (sum u p) + sum u^2 p
            const FF Px0 = ff_mul_f(P, fx0);
            acc[1] = ff_add(acc[1], ff_add(Px0, XP));
            acc[2] = ff_add(acc[2], ff_mul_f(P, fy));
            acc[3] = ff_add(acc[3], ff_add(ff_add(ff_mul_f(Px0, fx0), ff_mul_f(XP, 2.f * fx0)), X2P));
            acc[4] = ff_add(acc[4], ff_mul_f(ff_mul_f(P, fy), fy));
            acc[5] = ff_add(acc[5], KIN);
            acc[6] = ff_add(acc[6], VP);
        }
    }
    Neu nacc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        nacc[q] = {0.0, 0.0};
        nacc[q].add((double)acc[q].hi);
        nacc[q].add((double)acc[q].lo);
    }
    if constexpr (!NORM_ONLY) {
        // kinetic: -2 J * sum Re(conj(psi_j) psi_k), J = J_hi + J_lo
        const double k = nacc[5].val();
        nacc[5] = {0.0, 0.0};
        nacc[5].add(-2.0 * ((double)J_hi + (double)J_lo) * k);
    }
    block_reduce_write<NQ>(nacc, partials);
}

// <phi|psi>: exact products, double-float per-thread sums, FP64 combine.
__global__ void __launch_bounds__(kThreads)
inner_f32_kernel(const float *__restrict__ ar, const float *__restrict__ ai,
                 const float *__restrict__ br, const float *__restrict__ bi, int nx, int ny,
                 int64_t pitch, double *__restrict__ partials)
{
    FF sr = ff_make(0.f), si = ff_make(0.f);
    const int chunks_per_row = (nx + 3) / 4;
    const int64_t nchunks = (int64_t)chunks_per_row * ny;
    for (Walk w(chunks_per_row, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < nchunks; w.next()) {
        const int y = (int)w.y;
        const int x0 = (int)w.x * 4;
        const int64_t o = (int64_t)y * pitch + x0;
        const float4 a4 = *reinterpret_cast<const float4 *>(ar + o);
        const float4 b4 = *reinterpret_cast<const float4 *>(ai + o);
        const float4 c4 = *reinterpret_cast<const float4 *>(br + o);
        const float4 d4 = *reinterpret_cast<const float4 *>(bi + o);
        const float pr[4] = {a4.x, a4.y, a4.z, a4.w}, pi[4] = {b4.x, b4.y, b4.z, b4.w};
        const float qr[4] = {c4.x, c4.y, c4.z, c4.w}, qi[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (x0 + u >= nx) break;
            // conj(p) q = (pr qr + pi qi) + i (pr qi - pi qr)
            sr = ff_add(sr, ff_add(two_prod(pr[u], qr[u]), two_prod(pi[u], qi[u])));
            si = ff_add(si, ff_add(two_prod(pr[u], qi[u]), two_prod(-pi[u], qr[u])));
        }
    }
    Neu acc[2];
    acc[0] = {0.0, 0.0};
    acc[1] = {0.0, 0.0};
    acc[0].add((double)sr.hi);
    acc[0].add((double)sr.lo);
    acc[1].add((double)si.hi);
    acc[1].add((double)si.lo);
    block_reduce_write<2>(acc, partials);
}

template <typename T, bool NORM_ONLY>
__global__ void __launch_bounds__(kThreads)
observe_kernel(const T *__restrict__ re, const T *__restrict__ im, const T *__restrict__ vp,
               int nx, int ny, int64_t pitch, double J, double *__restrict__ partials)
{
    constexpr int NQ = NORM_ONLY ? 1 : OBS_Q;
    Neu acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = {0.0, 0.0};

    const int chunks_per_row = (nx + 3) / 4;
    const int64_t nchunks = (int64_t)chunks_per_row * ny;
    for (Walk w(chunks_per_row, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < nchunks; w.next()) {
        const int y = (int)w.y;
        const int x0 = (int)w.x * 4;
        const int64_t o = (int64_t)y * pitch;
        double run[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) run[q] = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = x0 + u;
            if (x >= nx) break;
            const double r = (double)re[o + x], m = (double)im[o + x];
            const double p = r * r + m * m;
            run[0] += p;
            if constexpr (!NORM_ONLY) {
                run[1] += (double)x * p;
                run[2] += (double)y * p;
                run[3] += (double)x * (double)x * p;
                run[4] += (double)y * (double)y * p;
                double kin = 0.0;
                if (x + 1 < nx)
                    kin += r * (double)re[o + x + 1] + m * (double)im[o + x + 1];
                if (y + 1 < ny)
                    kin += r * (double)re[o + pitch + x] + m * (double)im[o + pitch + x];
                run[5] += -2.0 * J * kin;
                run[6] += (double)vp[o + x] * p;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q].add(run[q]);
    }

    // block reduction: warp shuffles, then one warp over the warp results
    __shared__ double sh_s[kThreads / 32][NQ], sh_c[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        Neu a = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Neu b;
            b.s = __shfl_down_sync(0xffffffffu, a.s, off);
            b.c = __shfl_down_sync(0xffffffffu, a.c, off);
            neu_merge(a, b);
        }
        if (lane == 0) {
            sh_s[warp][q] = a.s;
            sh_c[warp][q] = a.c;
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Neu a = {0.0, 0.0};
            if (lane < kThreads / 32) a = {sh_s[lane][q], sh_c[lane][q]};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                Neu b;
                b.s = __shfl_down_sync(0xffffffffu, a.s, off);
                b.c = __shfl_down_sync(0xffffffffu, a.c, off);
                neu_merge(a, b);
            }
            if (lane == 0) partials[(int64_t)blockIdx.x * OBS_Q + q] = a.val();
        }
    }
}

// Observables of a 3-D grid (slab z = rows z*ny .. z*ny + ny - 1): every
// term in FP64 (it is called at report points only), runs of 4 sites summed
// plainly and added into Neumaier-compensated per-thread sums.
template <typename T>
__global__ void __launch_bounds__(kThreads)
observe3_kernel(const T *__restrict__ re, const T *__restrict__ im, const T *__restrict__ vp,
                int nx, int ny, int nz, int64_t pitch, double J, double *__restrict__ partials)
{
    constexpr int NQ = OBS_Q3;
    Neu acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = {0.0, 0.0};
    const int64_t rows = (int64_t)ny * nz;
    const int64_t slab = (int64_t)ny * pitch;
    const int chunks_per_row = (nx + 3) / 4;
    const int64_t nchunks = (int64_t)chunks_per_row * rows;
    for (Walk w(chunks_per_row, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < nchunks; w.next()) {
        const int64_t r = w.y;
        const int x0 = (int)w.x * 4;
        const int z = (int)(r / ny), y = (int)(r - (int64_t)z * ny);
        const int64_t o = r * pitch;
        double run[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) run[q] = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = x0 + u;
            if (x >= nx) break;
            const double a = (double)re[o + x], b = (double)im[o + x];
            const double p = a * a + b * b;
            run[0] += p;
            run[1] += (double)x * p;
            run[2] += (double)y * p;
            run[3] += (double)x * (double)x * p;
            run[4] += (double)y * (double)y * p;
            double kin = 0.0;
            if (x + 1 < nx) kin += a * (double)re[o + x + 1] + b * (double)im[o + x + 1];
            if (y + 1 < ny) kin += a * (double)re[o + pitch + x] + b * (double)im[o + pitch + x];
            if (z + 1 < nz) kin += a * (double)re[o + slab + x] + b * (double)im[o + slab + x];
            run[5] += -2.0 * J * kin;
            run[6] += (double)vp[o + x] * p;
            run[7] += (double)z * p;
            run[8] += (double)z * (double)z * p;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q].add(run[q]);
    }
    __shared__ double sh_s[kThreads / 32][NQ], sh_c[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        Neu a = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Neu b;
            b.s = __shfl_down_sync(0xffffffffu, a.s, off);
            b.c = __shfl_down_sync(0xffffffffu, a.c, off);
            neu_merge(a, b);
        }
        if (lane == 0) {
            sh_s[warp][q] = a.s;
            sh_c[warp][q] = a.c;
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Neu a = {0.0, 0.0};
            if (lane < kThreads / 32) a = {sh_s[lane][q], sh_c[lane][q]};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                Neu b;
                b.s = __shfl_down_sync(0xffffffffu, a.s, off);
                b.c = __shfl_down_sync(0xffffffffu, a.c, off);
                neu_merge(a, b);
            }
            if (lane == 0) partials[(int64_t)blockIdx.x * OBS_Q3 + q] = a.val();
        }
    }
}

__global__ void __launch_bounds__(kThreads)
observe_finalize_kernel(const double *__restrict__ partials, int nblocks, int nq, int stride,
                        double *__restrict__ result)
{
    __shared__ double sh_s[kThreads / 32], sh_c[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        Neu a = {0.0, 0.0};
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
            a.add(partials[(int64_t)b * stride + q]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            Neu o;
            o.s = __shfl_down_sync(0xffffffffu, a.s, off);
            o.c = __shfl_down_sync(0xffffffffu, a.c, off);
            neu_merge(a, o);
        }
        if (lane == 0) {
            sh_s[warp] = a.s;
            sh_c[warp] = a.c;
        }
        __syncthreads();
        if (warp == 0) {
            Neu t = {0.0, 0.0};
            if (lane < kThreads / 32) t = {sh_s[lane], sh_c[lane]};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                Neu o;
                o.s = __shfl_down_sync(0xffffffffu, t.s, off);
                o.c = __shfl_down_sync(0xffffffffu, t.c, off);
                neu_merge(t, o);
            }
            if (lane == 0) result[q] = t.val();
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_observe(const void *re, const void *im, const void *vplane, bool f64, int nx,
                           int ny, int64_t pitch, double J, bool norm_only, double *partials,
                           double *result, cudaStream_t st)
{
    const int64_t nchunks = (int64_t)((nx + 3) / 4) * ny;
    int64_t b = (nchunks + kThreads * 8 - 1) / (kThreads * 8);
    int nblocks = (int)(b < 1 ? 1 : (b > OBS_MAX_BLOCKS ? OBS_MAX_BLOCKS : b));
    if (f64) {
        if (norm_only)
            observe_kernel<double, true><<<nblocks, kThreads, 0, st>>>((const double *)re, (const double *)im, (const double *)vplane, nx, ny, pitch, J, partials);
        else
            observe_kernel<double, false><<<nblocks, kThreads, 0, st>>>((const double *)re, (const double *)im, (const double *)vplane, nx, ny, pitch, J, partials);
    } else {
        const float J_hi = (float)J, J_lo = (float)(J - (double)J_hi);
        if (norm_only)
            observe_f32_kernel<true><<<nblocks, kThreads, 0, st>>>((const float *)re, (const float *)im, (const float *)vplane, nx, ny, pitch, J_hi, J_lo, partials);
        else
            observe_f32_kernel<false><<<nblocks, kThreads, 0, st>>>((const float *)re, (const float *)im, (const float *)vplane, nx, ny, pitch, J_hi, J_lo, partials);
    }
    observe_finalize_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, norm_only ? 1 : OBS_Q, OBS_Q,
                                                    result);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_observe3(const void *re, const void *im, const void *vplane, bool f64, int nx,
                            int ny, int nz, int64_t pitch, double J, double *partials,
                            double *result, cudaStream_t st)
{
    const int64_t nchunks = (int64_t)((nx + 3) / 4) * ny * nz;
    int64_t b = (nchunks + kThreads * 8 - 1) / (kThreads * 8);
    int nblocks = (int)(b < 1 ? 1 : (b > OBS_MAX_BLOCKS ? OBS_MAX_BLOCKS : b));
    if (f64)
        observe3_kernel<double><<<nblocks, kThreads, 0, st>>>((const double *)re, (const double *)im, (const double *)vplane, nx, ny, nz, pitch, J, partials);
    else
        observe3_kernel<float><<<nblocks, kThreads, 0, st>>>((const float *)re, (const float *)im, (const float *)vplane, nx, ny, nz, pitch, J, partials);
    observe_finalize_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, OBS_Q3, OBS_Q3, result);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_inner(const float *phi_re, const float *phi_im, const float *psi_re,
                         const float *psi_im, int nx, int ny, int64_t pitch, double *partials,
                         double *result, cudaStream_t st)
{
    const int64_t nchunks = (int64_t)((nx + 3) / 4) * ny;
    int64_t b = (nchunks + kThreads * 8 - 1) / (kThreads * 8);
    int nblocks = (int)(b < 1 ? 1 : (b > OBS_MAX_BLOCKS ? OBS_MAX_BLOCKS : b));
    inner_f32_kernel<<<nblocks, kThreads, 0, st>>>(phi_re, phi_im, psi_re, psi_im, nx, ny, pitch,
                                                   partials);
    observe_finalize_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, 2, OBS_Q, result);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace ts
