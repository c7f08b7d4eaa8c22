// Conversions, the potential-phase table and the plain one-sweep-per-kernel
// path of the second-order Trotter-Suzuki step (Sec. 2, Eq. secondorder).
//
// The plain path is the reference point for the fused kernel: each of the
// eight sweeps and the phase is one launch over the whole grid, in place
// (the pairs of one sweep are disjoint, so in-place update is exact).
// Per site-step it moves 8 sweeps x (read + write of re, im) + the phase
// (read state + table, write state): 152 B in FP32, 304 B in FP64.
#include "common.cuh"
#include "internal.h"

namespace ts {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int per_block)
{
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

template <typename Ts, typename Td>
__global__ void convert_in_kernel(const Ts *__restrict__ src, Td *__restrict__ dst, int nx,
                                  int ny, int64_t pitch)
{
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t y = i / nx, x = i - y * nx;
        dst[y * pitch + x] = (Td)src[i];
    }
}

template <typename Ts, typename Td>
__global__ void convert_out_kernel(const Ts *__restrict__ src, Td *__restrict__ dst, int nx,
                                   int ny, int64_t pitch)
{
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t y = i / nx, x = i - y * nx;
        dst[i] = (Td)src[y * pitch + x];
    }
}

// Table preparation (Sec. 2: one diagonal factor exp(-i V dt) per step):
// gamma_V = 1 - cos(V dt) = 2 sin^2(V dt / 2) and s_V = sin(V dt) in FP64,
// each rounded once to T; V itself is kept (rounded to T) for the energy.
template <typename T>
__global__ void phase_table_kernel(const double *__restrict__ V, T *__restrict__ pg,
                                   T *__restrict__ ps, T *__restrict__ vp, int nx, int ny,
                                   int64_t pitch, double dt)
{
    const int64_t n = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t y = i / nx, x = i - y * nx;
        double v = V[i];
        double ph = v * dt;
        double sh = sin(0.5 * ph);
        int64_t j = y * pitch + x;
        pg[j] = (T)(2.0 * sh * sh);
        ps[j] = (T)sin(ph);
        vp[j] = (T)v;
    }
}

// X sweep: pairs (x, x+1), x = parity + 2p, every row; one thread per pair.
template <typename T>
__global__ void plain_sweep_x_kernel(T *__restrict__ re, T *__restrict__ im, int nx, int ny,
                                     int64_t pitch, int parity, T g, T s)
{
    const int npr = (nx - parity) / 2;   // pairs per row
    if (npr <= 0) return;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        T *r = re + (int64_t)y * pitch;
        T *m = im + (int64_t)y * pitch;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npr;
             p += gridDim.x * blockDim.x) {
            int x = parity + 2 * p;
            T ar = r[x], ai = m[x], br = r[x + 1], bi = m[x + 1];
            rot2(ar, ai, br, bi, g, s);
            r[x] = ar;
            m[x] = ai;
            r[x + 1] = br;
            m[x + 1] = bi;
        }
    }
}

// Y sweep: pairs (y, y+1), y = parity + 2q, every column; one thread per
// (column, pair) with the column fastest so that accesses coalesce.
template <typename T>
__global__ void plain_sweep_y_kernel(T *__restrict__ re, T *__restrict__ im, int nx, int ny,
                                     int64_t pitch, int parity, T g, T s)
{
    const int npc = (ny - parity) / 2;   // pairs per column
    for (int q = blockIdx.y; q < npc; q += gridDim.y) {
        int64_t y = parity + 2 * q;
        T *r0 = re + y * pitch, *m0 = im + y * pitch;
        T *r1 = r0 + pitch, *m1 = m0 + pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx;
             x += gridDim.x * blockDim.x) {
            T ar = r0[x], ai = m0[x], br = r1[x], bi = m1[x];
            rot2(ar, ai, br, bi, g, s);
            r0[x] = ar;
            m0[x] = ai;
            r1[x] = br;
            m1[x] = bi;
        }
    }
}

template <typename T>
__global__ void plain_phase_kernel(T *__restrict__ re, T *__restrict__ im,
                                   const T *__restrict__ pg, const T *__restrict__ ps, int nx,
                                   int ny, int64_t pitch)
{
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        int64_t o = (int64_t)y * pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx;
             x += gridDim.x * blockDim.x) {
            T r = re[o + x], m = im[o + x];
            phase1(r, m, pg[o + x], ps[o + x]);
            re[o + x] = r;
            im[o + x] = m;
        }
    }
}

inline dim3 grid2d(int64_t per_row, int rows)
{
    int gx = (int)((per_row + kThreads - 1) / kThreads);
    if (gx < 1) gx = 1;
    int gy = rows < 1 ? 1 : (rows > 65535 ? 65535 : rows);
    return dim3(gx, gy);
}

}  // namespace

cudaError_t launch_convert_in(const void *src, bool src_f64, void *dst, bool dst_f64, int nx,
                              int ny, int64_t pitch, cudaStream_t st)
{
    int grid = grid_for((int64_t)nx * ny, kThreads);
    if (src_f64 && dst_f64)
        convert_in_kernel<double, double><<<grid, kThreads, 0, st>>>((const double *)src, (double *)dst, nx, ny, pitch);
    else if (src_f64)
        convert_in_kernel<double, float><<<grid, kThreads, 0, st>>>((const double *)src, (float *)dst, nx, ny, pitch);
    else if (dst_f64)
        convert_in_kernel<float, double><<<grid, kThreads, 0, st>>>((const float *)src, (double *)dst, nx, ny, pitch);
    else
        convert_in_kernel<float, float><<<grid, kThreads, 0, st>>>((const float *)src, (float *)dst, nx, ny, pitch);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_convert_out(const void *src, bool src_f64, void *dst, bool dst_f64, int nx,
                               int ny, int64_t pitch, cudaStream_t st)
{
    int grid = grid_for((int64_t)nx * ny, kThreads);
    if (src_f64 && dst_f64)
        convert_out_kernel<double, double><<<grid, kThreads, 0, st>>>((const double *)src, (double *)dst, nx, ny, pitch);
    else if (src_f64)
        convert_out_kernel<double, float><<<grid, kThreads, 0, st>>>((const double *)src, (float *)dst, nx, ny, pitch);
    else if (dst_f64)
        convert_out_kernel<float, double><<<grid, kThreads, 0, st>>>((const float *)src, (double *)dst, nx, ny, pitch);
    else
        convert_out_kernel<float, float><<<grid, kThreads, 0, st>>>((const float *)src, (float *)dst, nx, ny, pitch);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_phase_table(const double *V, void *pg, void *ps, void *vplane, bool f64, int nx,
                               int ny, int64_t pitch, double dt, cudaStream_t st)
{
    int grid = grid_for((int64_t)nx * ny, kThreads);
    if (f64)
        phase_table_kernel<double><<<grid, kThreads, 0, st>>>(V, (double *)pg, (double *)ps, (double *)vplane, nx, ny, pitch, dt);
    else
        phase_table_kernel<float><<<grid, kThreads, 0, st>>>(V, (float *)pg, (float *)ps, (float *)vplane, nx, ny, pitch, dt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_sweep(void *re, void *im, bool f64, int nx, int ny, int64_t pitch,
                               int axis, int parity, double g, double s, cudaStream_t st)
{
    if (axis == 0) {
        dim3 grid = grid2d((nx - parity) / 2, ny);
        if (f64)
            plain_sweep_x_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else
            plain_sweep_x_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, pitch, parity, (float)g, (float)s);
    } else {
        dim3 grid = grid2d(nx, (ny - parity) / 2);
        if (f64)
            plain_sweep_y_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else
            plain_sweep_y_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, pitch, parity, (float)g, (float)s);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_phase(void *re, void *im, const void *pg, const void *ps, bool f64, int nx,
                               int ny, int64_t pitch, cudaStream_t st)
{
    dim3 grid = grid2d(nx, ny);
    if (f64)
        plain_phase_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, (const double *)pg, (const double *)ps, nx, ny, pitch);
    else
        plain_phase_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, (const float *)pg, (const float *)ps, nx, ny, pitch);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ts
