// Conversions, the potential-phase table and the plain one-sweep-per-kernel
// path of the second-order Trotter-Suzuki step (Sec. 2, Eq. secondorder).
//
// The plain path is the reference point for the fused kernel: each of the
// eight sweeps and the phase is one launch over the whole grid, in place
// (the pairs of one sweep are disjoint, so in-place update is exact).
// Per site-step it moves 8 sweeps x (read + write of re, im) + the phase
// (read state + table, write state): 152 B in FP32, 304 B in FP64.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ffloat.cuh"
#include "internal.h"
#include "walk.cuh"

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

// Dense (nx per row) <-> pitched conversions, one row per blockIdx.y step.
// When nx is a multiple of 4 every row starts 16-byte aligned in both
// layouts, and each thread moves 4 elements with vector accesses.
template <typename T>
struct Quad {
    T v[4];
};

template <typename T>
__device__ __forceinline__ Quad<T> load4(const T *p)
{
    Quad<T> q;
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
    }
    return q;
}

template <typename T>
__device__ __forceinline__ void store4(T *p, const T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
}

// IN: dense src -> pitched dst; otherwise pitched src -> dense dst
template <bool IN, typename Ts, typename Td>
__global__ void convert_kernel(const Ts *__restrict__ src, Td *__restrict__ dst, int nx, int ny,
                               int64_t pitch, bool vec4)
{
    for (int64_t y = blockIdx.y; y < ny; y += gridDim.y) {
        const Ts *s = src + y * (IN ? (int64_t)nx : pitch);
        Td *d = dst + y * (IN ? pitch : (int64_t)nx);
        if (vec4) {
            for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx / 4;
                 q += gridDim.x * blockDim.x) {
                const Quad<Ts> a = load4(s + 4 * q);
                Td b[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) b[k] = (Td)a.v[k];
                store4(d + 4 * q, b);
            }
        } else {
            for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx;
                 x += gridDim.x * blockDim.x)
                d[x] = (Td)s[x];
        }
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
    for (Walk w(nx, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < n; w.next()) {
        const int64_t i = w.i, y = w.y, x = w.x;
        double v = V[i];
        double ph = v * dt;
        double sh = sin(0.5 * ph);
        int64_t j = y * pitch + x;
        pg[j] = (T)(2.0 * sh * sh);
        ps[j] = (T)sin(ph);
        vp[j] = (T)v;
    }
}

// FP32 grids: the same table, evaluated in double-float on the FP32 pipe and
// rounded once (FP64 runs at ~1/67 of the FP32 rate on this GPU).
//  1. V (FP64) is split into v_hi + v_lo floats with integer bit operations
//     (v_hi = the top 24 significand bits, v_lo = the next 24), so no FP64
//     instruction is needed; phi/2 = V * dt/2 as a double-float product.
//  2. h = phi/2 is reduced by k = rint(h * 256/pi): t = h - k pi/256 with a
//     three-part Cody-Waite split of pi/256 (k * C1 and k * C2 exact for
//     |k| <= 4096), so |t| <= pi/512.
//  3. sin t = t + t^3 P(t^2), cos t = 1 + t^2 Q(t^2) (Taylor series; the
//     corrections are < 2e-5 relative, so FP32 suffices for them), and
//     sin h, cos h by the angle-addition formulas with sin/cos(k pi/256)
//     from a 256-entry double-float table built on the host in FP64.
//  4. s_V = 2 sin h cos h and gamma_V = 2 sin^2 h in double-float, each
//     rounded once to FP32 (the hi part of the normalised pair).
// The result carries ~40 correct bits, so the rounding agrees with
// FP64-then-round except when the exact value lies within ~2^-16 ulp of a
// rounding midpoint (then it is one ulp away).  |V dt| > 100 or |V| > 2^100
// take the FP64 path; V must be finite.
struct TrigTable {
    float4 sc[256];         // (sin hi, sin lo, cos hi, cos lo) of k pi/256
    float c1, c2, c3;       // pi/256 = c1 + c2 + c3
    float inv;              // 256/pi
    float hdt_hi, hdt_lo;   // dt/2 as double-float
    double hdt;             // dt/2
};

// Split a finite double v into hi + lo floats (hi = the top 24 significand
// bits, truncated; lo = the next 24) using integer operations only.  Below
// 2^-74 the split is of v * 2^S with S = -20 - exponent(v) (returned), so that
// both halves stay normal floats; zero and FP64 subnormals give 0.  Returns
// false above 2^100 or for non-finite v.
__device__ __forceinline__ bool split_double(double v, float &hi, float &lo, int &S)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long man = b & 0xfffffffffffffull;
    const unsigned sign = (unsigned)(b >> 63) << 31;
    int ue = e - 1023;                      // unbiased exponent
    S = 0;
    if (e == 0x7ff || ue > 100) return false;   // non-finite or huge: FP64 path
    if (e == 0) {                           // zero or FP64 subnormal: the table is 0
        hi = lo = 0.f;
        return true;
    }
    if (ue < -74) {
        S = -20 - ue;
        ue = -20;
    }
    hi = __uint_as_float(sign | ((unsigned)(ue + 127) << 23) | (unsigned)(man >> 29));
    // the remaining 29 fraction bits times 2^(ue - 52) (a normal float scale
    // since ue >= -74); I2F keeps 24 of the 29 bits
    const unsigned rest = (unsigned)(man & 0x1fffffffull);
    const float r = (float)rest * __uint_as_float((unsigned)(ue - 52 + 127) << 23);
    lo = sign ? -r : r;
    return true;
}

// x * 2^-S for S >= 0, in at most two exact power-of-two steps (the last
// one rounds into the subnormal range or to zero if it must).
__device__ __forceinline__ float scale_down(float x, int S)
{
    if (S > 252) return x * 0.f;
    if (S > 126) {
        x *= 1.17549435e-38f;               // 2^-126
        S -= 126;
    }
    return x * __uint_as_float((unsigned)(127 - S) << 23);
}

__global__ void phase_table_f32_kernel(const double *__restrict__ V, float *__restrict__ pg,
                                       float *__restrict__ ps, float *__restrict__ vp, int nx,
                                       int ny, int64_t pitch, const TrigTable tab)
{
    __shared__ float4 sc[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sc[i] = tab.sc[i];
    __syncthreads();
    const int64_t n = (int64_t)nx * ny;
    for (Walk w(nx, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
         w.i < n; w.next()) {
        const int64_t i = w.i, j = w.y * pitch + w.x;
        const double v = V[i];
        float vh, vl;
        int S;
        bool ok = split_double(v, vh, vl, S);
        if (ok && S > 0) {
            // |V| < 2^-74: sin h = h and 1 - cos(2h) = 2 h^2 to far below an
            // ulp; work at V * 2^S and scale the results back (exact for
            // normal results, one rounding into the subnormal range)
            const FF hS = ff_mul(fast_two_sum(vh, vl), FF{tab.hdt_hi, tab.hdt_lo});
            const float hh = scale_down(hS.hi, S);
            ps[j] = scale_down(2.f * hS.hi, S);
            pg[j] = 2.f * hh * hh;
            vp[j] = scale_down(fast_two_sum(vh, vl).hi, S);
            continue;
        }
        float kf = 0.f;
        FF h;
        if (ok) {
            h = ff_mul(fast_two_sum(vh, vl), FF{tab.hdt_hi, tab.hdt_lo});
            kf = rintf(h.hi * tab.inv);
            ok = fabsf(kf) <= 4096.f && isfinite(h.hi);
        }
        if (!ok) {   // rare: FP64 path
            const double ph = v * (2.0 * tab.hdt);
            const double sh = sin(0.5 * ph);
            pg[j] = (float)(2.0 * sh * sh);
            ps[j] = (float)sin(ph);
            vp[j] = (float)v;
            continue;
        }
        // t = h - k pi/256 (Cody-Waite; k*c1, k*c2 exact)
        FF t = two_sum(h.hi - kf * tab.c1, -kf * tab.c2);
        t = ff_add(t, FF{h.lo, 0.f});
        t = ff_add(t, two_prod(-kf, tab.c3));
        const float t2 = t.hi * t.hi;
        const float st = t.hi * t2 * fmaf(t2, fmaf(t2, -1.f / 5040.f, 1.f / 120.f), -1.f / 6.f);
        const float ct = fmaf(t2, fmaf(t2, fmaf(t2, -1.f / 720.f, 1.f / 24.f), -0.5f), -t.hi * t.lo);
        int k = ((int)kf) & 255;
        const float4 e = sc[k];
        const FF Sk = {e.x, e.y}, Ck = {e.z, e.w};
        // sin h = Sk + Sk ct + Ck (t + st) ; cos h = Ck + Ck ct - Sk (t + st)
        const FF tt = ff_add_f(t, st);
        const FF sh = ff_add(ff_add_f(Sk, Sk.hi * ct), ff_mul(Ck, tt));
        const FF ch = ff_add(ff_add_f(Ck, Ck.hi * ct), ff_mul(FF{-Sk.hi, -Sk.lo}, tt));
        const FF s2 = ff_mul(sh, ch);
        const FF g2 = ff_mul(sh, sh);
        ps[j] = 2.f * s2.hi;
        pg[j] = 2.f * g2.hi;
        vp[j] = fast_two_sum(vh, vl).hi;
    }
}

// X sweep: pairs (x, x+1), x = parity + 2p, every row; one thread per pair.
// (g, s) are the versine coefficients, or with LIFT (t, s) of the lifting form.
template <typename T, bool LIFT = false>
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
            rot_pair<LIFT>(ar, ai, br, bi, g, s);
            r[x] = ar;
            m[x] = ai;
            r[x + 1] = br;
            m[x + 1] = bi;
        }
    }
}

// Y sweep: pairs (y, y+1), y = parity + 2q, every column; one thread per
// (column, pair) with the column fastest so that accesses coalesce.
template <typename T, bool LIFT = false>
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
            rot_pair<LIFT>(ar, ai, br, bi, g, s);
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

template <typename T>
__global__ void plain_drive_kernel(T *__restrict__ re, T *__restrict__ im,
                                   const T *__restrict__ v1, int nx, int ny, int64_t pitch, T adt)
{
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        int64_t o = (int64_t)y * pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx;
             x += gridDim.x * blockDim.x) {
            T r = re[o + x], m = im[o + x], g, s;
            angle_versine(adt * v1[o + x], g, s);
            phase1(r, m, g, s);
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

template <bool IN>
cudaError_t launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int nx, int ny,
                           int64_t pitch, cudaStream_t st)
{
    const bool vec4 = (nx % 4) == 0 && ((uintptr_t)src % 16) == 0 && ((uintptr_t)dst % 16) == 0;
    dim3 grid = grid2d(vec4 ? nx / 4 : nx, ny);
    if (src_f64 && dst_f64)
        convert_kernel<IN, double, double><<<grid, kThreads, 0, st>>>((const double *)src, (double *)dst, nx, ny, pitch, vec4);
    else if (src_f64)
        convert_kernel<IN, double, float><<<grid, kThreads, 0, st>>>((const double *)src, (float *)dst, nx, ny, pitch, vec4);
    else if (dst_f64)
        convert_kernel<IN, float, double><<<grid, kThreads, 0, st>>>((const float *)src, (double *)dst, nx, ny, pitch, vec4);
    else
        convert_kernel<IN, float, float><<<grid, kThreads, 0, st>>>((const float *)src, (float *)dst, nx, ny, pitch, vec4);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_convert_in(const void *src, bool src_f64, void *dst, bool dst_f64, int nx,
                              int ny, int64_t pitch, cudaStream_t st)
{
    return launch_convert<true>(src, src_f64, dst, dst_f64, nx, ny, pitch, st);
}

cudaError_t launch_convert_out(const void *src, bool src_f64, void *dst, bool dst_f64, int nx,
                               int ny, int64_t pitch, cudaStream_t st)
{
    return launch_convert<false>(src, src_f64, dst, dst_f64, nx, ny, pitch, st);
}

cudaError_t launch_phase_table(const double *V, void *pg, void *ps, void *vplane, bool f64, int nx,
                               int ny, int64_t pitch, double dt, cudaStream_t st)
{
    int grid = grid_for((int64_t)nx * ny, kThreads);
    if (f64) {
        phase_table_kernel<double><<<grid, kThreads, 0, st>>>(V, (double *)pg, (double *)ps, (double *)vplane, nx, ny, pitch, dt);
    } else {
        thread_local TrigTable tab;   // per thread: grids may be prepared concurrently
        thread_local double tab_dt = std::nan("");
        if (!(tab_dt == dt)) {   // host FP64 constants, split into double-floats
            const double pi_k = M_PI / 256.0;
            for (int k = 0; k < 256; ++k) {
                const double sv = std::sin(k * pi_k), cv = std::cos(k * pi_k);
                const float sh = (float)sv, chf = (float)cv;
                tab.sc[k] = make_float4(sh, (float)(sv - sh), chf, (float)(cv - chf));
            }
            auto top12 = [](double v) {   // v rounded to 12 significant bits
                float f = (float)v;
                unsigned u;
                std::memcpy(&u, &f, 4);
                u &= 0xfffff000u;   // 12 significant bits
                std::memcpy(&f, &u, 4);
                return f;
            };
            tab.c1 = top12(pi_k);
            tab.c2 = top12(pi_k - tab.c1);
            tab.c3 = (float)(pi_k - tab.c1 - tab.c2);
            tab.inv = (float)(256.0 / M_PI);
            tab.hdt = 0.5 * dt;
            tab.hdt_hi = (float)tab.hdt;
            tab.hdt_lo = (float)(tab.hdt - tab.hdt_hi);
            tab_dt = dt;
        }
        phase_table_f32_kernel<<<grid, kThreads, 0, st>>>(V, (float *)pg, (float *)ps, (float *)vplane, nx, ny, pitch, tab);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_sweep(void *re, void *im, bool f64, int nx, int ny, int64_t pitch,
                               int axis, int parity, double g, double s, cudaStream_t st,
                               bool lift)
{
    if (axis == 0) {
        dim3 grid = grid2d((nx - parity) / 2, ny);
        if (f64 && lift)
            plain_sweep_x_kernel<double, true><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else if (f64)
            plain_sweep_x_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else
            plain_sweep_x_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, pitch, parity, (float)g, (float)s);
    } else {
        dim3 grid = grid2d(nx, (ny - parity) / 2);
        if (f64 && lift)
            plain_sweep_y_kernel<double, true><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else if (f64)
            plain_sweep_y_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, nx, ny, pitch, parity, g, s);
        else
            plain_sweep_y_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, nx, ny, pitch, parity, (float)g, (float)s);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_plain_drive(void *re, void *im, const void *v1, bool f64, int nx, int ny,
                               int64_t pitch, double adt, cudaStream_t st)
{
    dim3 grid = grid2d(nx, ny);
    if (f64)
        plain_drive_kernel<double><<<grid, kThreads, 0, st>>>((double *)re, (double *)im, (const double *)v1, nx, ny, pitch, adt);
    else
        plain_drive_kernel<float><<<grid, kThreads, 0, st>>>((float *)re, (float *)im, (const float *)v1, nx, ny, pitch, (float)adt);
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
