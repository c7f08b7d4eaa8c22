// Three-dimensional lattices (the extension of Sec. 2's splitting to a third
// dimension, named in Sec. 6 as the method's next step).  A 3-D grid keeps
// its slabs one after another in every plane, so the 2-D kernels handle the
// X sweeps, the phase and the tables; this file adds the Y sweep that stays
// inside each slab, the Z sweeps, and a streaming kernel that applies a short
// sequence of Z sweeps in one pass over HBM.
#include "common.cuh"
#include "internal.h"

namespace ts {

namespace {

constexpr int kThreads = 256;

inline dim3 grid2d(int64_t per_row, int64_t rows)
{
    int gx = (int)((per_row + kThreads - 1) / kThreads);
    if (gx < 1) gx = 1;
    int gy = rows < 1 ? 1 : (rows > 65535 ? 65535 : (int)rows);
    return dim3(gx, gy);
}

// Y pairs (y, y+1) inside every slab: index q over nz * pairs-per-slab.
// (g, s) are the versine coefficients, or with LIFT (t, s) of the lifting form.
template <typename T, bool LIFT = false>
__global__ void sweep_y3_kernel(T *__restrict__ re, T *__restrict__ im, int nx, int ny, int nz,
                                int64_t pitch, int parity, T g, T s)
{
    const int per_slab = (ny - parity) / 2;
    const int64_t npairs = (int64_t)per_slab * nz;
    for (int64_t q = blockIdx.y; q < npairs; q += gridDim.y) {
        const int64_t z = q / per_slab;
        const int64_t y = z * ny + parity + 2 * (q - z * per_slab);
        T *r0 = re + y * pitch, *m0 = im + y * pitch;
        T *r1 = r0 + pitch, *m1 = m0 + pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
            T ar = r0[x], ai = m0[x], br = r1[x], bi = m1[x];
            rot_pair<LIFT>(ar, ai, br, bi, g, s);
            r0[x] = ar;
            m0[x] = ai;
            r1[x] = br;
            m1[x] = bi;
        }
    }
}

// Z pairs (z, z+1): index q over pairs-of-slabs * ny rows.
template <typename T, bool LIFT = false>
__global__ void sweep_z_kernel(T *__restrict__ re, T *__restrict__ im, int nx, int ny, int nz,
                               int64_t pitch, int parity, T g, T s)
{
    const int npz = (nz - parity) / 2;
    const int64_t nrows = (int64_t)npz * ny;
    const int64_t slab = (int64_t)ny * pitch;
    for (int64_t q = blockIdx.y; q < nrows; q += gridDim.y) {
        const int64_t p = q / ny, y = q - p * ny;
        const int64_t z = parity + 2 * p;
        T *r0 = re + z * slab + y * pitch, *m0 = im + z * slab + y * pitch;
        T *r1 = r0 + slab, *m1 = m0 + slab;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
            T ar = r0[x], ai = m0[x], br = r1[x], bi = m1[x];
            rot_pair<LIFT>(ar, ai, br, bi, g, s);
            r0[x] = ar;
            m0[x] = ai;
            r1[x] = br;
            m1[x] = bi;
        }
    }
}

struct Col4 {
    float4 re, im;
};

__device__ __forceinline__ void pair_lift4(Col4 &a, Col4 &b, float t, float s)
{
    rot_lift(a.re.x, a.im.x, b.re.x, b.im.x, t, s);
    rot_lift(a.re.y, a.im.y, b.re.y, b.im.y, t, s);
    rot_lift(a.re.z, a.im.z, b.re.z, b.im.z, t, s);
    rot_lift(a.re.w, a.im.w, b.re.w, b.im.w, t, s);
}

constexpr int kZSeg = 64;   // slabs a thread stores; it loads M more on each side

// M Z sweeps in one pass.  A thread owns 4 columns of one row y and a
// segment [z0, z1) of slabs; it streams the slabs [z0 - M, z1 + M) through a
// window of M + 1 slabs: when slab t arrives, sweep i applies its pair
// (t - i, t - i + 1) (slab t - i + 1 is final for sweep i - 1 by then), and
// slab t - M is final for all M sweeps and is stored if it is in [z0, z1).
// A stored slab depends only on slabs within M of it, all loaded, so the
// halo slabs' wrong values (their outer partners are not loaded) never reach
// it.  Pairs need both slabs on the grid and in the loaded range.
template <int M>
__global__ void __launch_bounds__(128)
zstream_kernel(const float *__restrict__ in_re, const float *__restrict__ in_im,
               float *__restrict__ out_re, float *__restrict__ out_im, int nx, int ny, int nz,
               int64_t pitch, ZSeq q)
{
    const int chunks = (nx + 3) / 4;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= chunks) return;
    const int y = blockIdx.y;
    const int z0 = blockIdx.z * kZSeg;
    const int z1 = min(z0 + kZSeg, nz);
    const int lo = max(z0 - M, 0), hi = min(z1 + M, nz);
    const int64_t slab = (int64_t)ny * pitch;
    const int64_t col = (int64_t)y * pitch + 4 * c;
    Col4 win[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) {
        win[k].re = make_float4(0.f, 0.f, 0.f, 0.f);
        win[k].im = win[k].re;
    }
    // two slabs of loads in flight ahead of the one being swept
    auto load = [&](int t, Col4 &c) {
        c.re = *reinterpret_cast<const float4 *>(in_re + t * slab + col);
        c.im = *reinterpret_cast<const float4 *>(in_im + t * slab + col);
    };
    Col4 nx0 = win[0], nx1 = win[0];
    if (lo < hi) load(lo, nx0);
    if (lo + 1 < hi) load(lo + 1, nx1);
    for (int t = lo; t < hi + M; ++t) {
#pragma unroll
        for (int k = 0; k < M; ++k) win[k] = win[k + 1];
        if (t < hi) {
            win[M] = nx0;
            nx0 = nx1;
            if (t + 2 < hi) load(t + 2, nx1);
        }
#pragma unroll
        for (int i = 1; i <= M; ++i) {
            const int za = t - i;   // pair (za, za + 1) = window slots (M - i, M - i + 1)
            if (za >= lo && za + 1 < hi && (za & 1) == q.parity[i - 1])
                pair_lift4(win[M - i], win[M - i + 1], q.t[i - 1], q.s[i - 1]);
        }
        const int zs = t - M;
        if (zs >= z0 && zs < z1) {
            *reinterpret_cast<float4 *>(out_re + zs * slab + col) = win[0].re;
            *reinterpret_cast<float4 *>(out_im + zs * slab + col) = win[0].im;
        }
    }
}

}  // namespace

cudaError_t launch_plain_sweep_y3(void *re, void *im, bool f64, int nx, int ny, int nz,
                                  int64_t pitch, int parity, double g, double s, cudaStream_t st,
                                  bool lift)
{
    const int64_t npairs = (int64_t)((ny - parity) / 2) * nz;
    if (npairs <= 0) return cudaSuccess;
    dim3 grid = grid2d(nx, npairs);
    if (f64 && lift)
        sweep_y3_kernel<double, true><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, nz, pitch, parity, g, s);
    else if (f64)
        sweep_y3_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, nz, pitch, parity, g, s);
    else
        sweep_y3_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, nz, pitch, parity, (float)g, (float)s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_sweep_z(void *re, void *im, bool f64, int nx, int ny, int nz,
                                 int64_t pitch, int parity, double g, double s, cudaStream_t st,
                                 bool lift)
{
    const int64_t nrows = (int64_t)((nz - parity) / 2) * ny;
    if (nrows <= 0) return cudaSuccess;
    dim3 grid = grid2d(nx, nrows);
    if (f64 && lift)
        sweep_z_kernel<double, true><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, nz, pitch, parity, g, s);
    else if (f64)
        sweep_z_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, nz, pitch, parity, g, s);
    else
        sweep_z_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, nz, pitch, parity, (float)g, (float)s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_zstream(const float *in_re, const float *in_im, float *out_re, float *out_im,
                           int nx, int ny, int nz, int64_t pitch, const ZSeq &q, cudaStream_t st)
{
    if (ny > 65535) return cudaErrorInvalidValue;
    const int chunks = (nx + 3) / 4;
    // a block covers up to 128 column chunks of one row; narrower rows get
    // narrower blocks rather than idle threads
    const int threads = chunks >= 128 ? 128 : ((chunks + 31) / 32) * 32;
    dim3 grid((chunks + threads - 1) / threads, ny, (nz + kZSeg - 1) / kZSeg);
    if (grid.z > 65535) return cudaErrorInvalidValue;
    if (q.m == 2)
        zstream_kernel<2><<<grid, threads, 0, st>>>(in_re, in_im, out_re, out_im, nx, ny, nz, pitch, q);
    else if (q.m == 3)
        zstream_kernel<3><<<grid, threads, 0, st>>>(in_re, in_im, out_re, out_im, nx, ny, nz, pitch, q);
    else
        return cudaErrorInvalidValue;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ts
