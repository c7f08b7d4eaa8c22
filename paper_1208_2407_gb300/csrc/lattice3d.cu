// Three-dimensional lattices (the extension of Sec. 2's splitting to a third
// dimension, named in Sec. 6 as the method's next step).  A 3-D grid keeps
// its slabs one after another in every plane, so the 2-D kernels handle the
// X sweeps, the phase and the tables; this file adds the Y sweep that stays
// inside each slab and the Z sweeps of the one-sweep-per-kernel path (the
// fused 3-D step is in fused.cu).
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

}  // namespace ts
