// Observables of the state: norm (Sec. 2: conserved by the unitary
// evolution), position moments and the energy <psi|H|psi> of the
// tight-binding Hamiltonian H = -J * (nearest-neighbour hops) + diag(V).
//
// Accumulation is FP64 throughout: every |psi|^2 term of an FP32 state is
// formed exactly in FP64 (a product of two 24-bit significands fits in 53
// bits); each thread sums a short run of sites (one row segment of 4) in
// plain FP64 and adds the run into Neumaier-compensated per-thread sums; the
// block combines threads with Neumaier's two-term update and writes FP64
// partials; one final block sums the partials with the same update.
#include "common.cuh"
#include "internal.h"

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
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / chunks_per_row);
        const int x0 = (int)(c - (int64_t)y * chunks_per_row) * 4;
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

__global__ void __launch_bounds__(kThreads)
observe_finalize_kernel(const double *__restrict__ partials, int nblocks, int nq,
                        double *__restrict__ result)
{
    for (int q = 0; q < nq; ++q) {
        Neu a = {0.0, 0.0};
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a.add(partials[(int64_t)b * OBS_Q + q]);
        __shared__ double sh_s[kThreads], sh_c[kThreads];
        sh_s[threadIdx.x] = a.s;
        sh_c[threadIdx.x] = a.c;
        __syncthreads();
        if (threadIdx.x == 0) {
            Neu t = {0.0, 0.0};
            for (int i = 0; i < (int)blockDim.x; ++i) {
                t.add(sh_s[i]);
                t.c += sh_c[i];
            }
            result[q] = t.val();
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
        if (norm_only)
            observe_kernel<float, true><<<nblocks, kThreads, 0, st>>>((const float *)re, (const float *)im, (const float *)vplane, nx, ny, pitch, J, partials);
        else
            observe_kernel<float, false><<<nblocks, kThreads, 0, st>>>((const float *)re, (const float *)im, (const float *)vplane, nx, ny, pitch, J, partials);
    }
    observe_finalize_kernel<<<1, kThreads, 0, st>>>(partials, nblocks, norm_only ? 1 : OBS_Q, result);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace ts
