// Fused, temporally blocked second-order Trotter-Suzuki steps (FP32).
//
// One launch applies K whole steps U2(dt) (Sec. 2, Eq. secondorder) per HBM
// round trip: it reads the state (re, im) and the potential-phase table
// (gamma_V, s_V) once and writes the state once, 24 B per site, for K steps.
//
// Operator order.  One step applies X-even, X-odd, Y-even, Y-odd (half angle
// theta), the phase exp(-i V dt), then Y-odd, Y-even, X-odd, X-even.  X
// sweeps act on rows and Y sweeps on columns, so every X factor commutes with
// every Y factor.  Between two consecutive phases the factors
//   Yo Ye Xo Xe | Xe Xo Ye Yo   therefore equal   [Xo Xe(2t) Xo] [Yo Ye(2t) Yo]
// (Xe(t) Xe(t) = Xe(2t) exactly: the same disjoint pair rotations), so K steps
// take 6K + 2 sweeps instead of 8K.  The results equal the literal product up
// to FP32 rounding.
//
// Geometry ("warp streams").  A warp owns a strip of 128 columns (lane l
// holds columns 4l..4l+3 of a row in registers as float4 re/im) and walks
// down a range of rows.  Row pairs arrive through rings of shared-memory
// slots that TMA fills ahead of use (cp.async.bulk.tensor.3d: one 128 x 2 x 2
// box per slot covers the same two rows of two adjacent planes, (re, im) or
// (gamma_V, s_V)); an mbarrier per slot tracks each fill.
//  - X sweeps are row-local: pairs inside a lane's float4 rotate in
//    registers, the pair that straddles two lanes uses warp shuffles.  The
//    strip reads h = roundup(2K, 4) halo columns per side (the valid region
//    shrinks by 2 columns per side per step) and stores the inner 128 - 2h.
//  - Y sweeps couple consecutive rows held by the same lane.  The K steps form
//    a software pipeline down the rows: an even-family sweep on a row pair
//    that starts at an even row, or an odd-family one on a pair that starts
//    at an odd row, is "aligned" and completes at once; the other kind waits
//    for the next row and carries one row in registers.  The output trails
//    the input by 2K rows; a row range reads 2K halo rows above and below.
//  - The phase of step k is read from the phase ring, which keeps the slots of
//    the K most recent row pairs; its slots are loaded one row earlier than
//    the state's, so each step's phase point reads one slot (the fourth-order
//    kernel and depth 1 keep the state's rows and one slot more).
// Grid-edge sites: TMA fills rows/columns outside the grid with zeros, and a
// pair whose partner lies outside the grid gets coefficients (0, 0), i.e. the
// identity (open boundaries: the unpaired site is unchanged).
//
// Work split: a persistent launch gives each strip the same number of warps,
// each on one row range, the same ranges in every strip, so that warps of
// neighbouring strips walk the same rows together and share their halo
// columns through L2 (min_pairs_per_warp sets how short a range may be).  The
// multi-grid kernel picks between that split and an even split of all its
// grids' (strip, row-pair) units (fused_multi_plan).
//
// Every wait on an mbarrier is bounded (globaltimer): on a timeout the warp
// sets an error bit, waits (bounded) for its own outstanding copies and
// returns; the host reports TS_ERR_TIMEOUT at its next synchronising call.
#include <algorithm>
#include <cstdio>
#include <queue>
#include <type_traits>
#include <utility>
#include <vector>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "ffloat.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace ts {

namespace {

#ifndef TS_FUSED_WPC_SHALLOW     // warps per CTA for K <= 2
#define TS_FUSED_WPC_SHALLOW 2
#endif
#ifndef TS_FUSED_WPC_DEEP        // ... and for K >= 3
#define TS_FUSED_WPC_DEEP 1
#endif
#ifndef TS_FUSED_PF_K1           // row pairs prefetched ahead of use for K = 1
#define TS_FUSED_PF_K1 4
#endif
#ifndef TS_FUSED_PF_K2           // ... for K = 2
#define TS_FUSED_PF_K2 4
#endif
#ifndef TS_FUSED_PF_DEEP         // ... and for K >= 3
#define TS_FUSED_PF_DEEP 1
#endif
#ifndef TS_FUSED_MIN_BLOCKS      // __launch_bounds__ minimum resident blocks per SM
#define TS_FUSED_MIN_BLOCKS 1
#endif
#ifndef TS_FUSED_MIN_BLOCKS_K3   // ... for K = 3: 168 registers, 12 one-warp blocks per SM
#define TS_FUSED_MIN_BLOCKS_K3 9
#endif
#ifndef TS_FUSED_MIN_BLOCKS_K4   // ... for K = 4
#define TS_FUSED_MIN_BLOCKS_K4 1
#endif
#ifndef TS_FUSED_MULTI_MIN_BLOCKS_K3   // multi-grid kernel, K = 3
#define TS_FUSED_MULTI_MIN_BLOCKS_K3 1
#endif
#ifndef TS_FUSED_MULTI_MIN_BLOCKS_K4   // multi-grid kernel, K = 4
#define TS_FUSED_MULTI_MIN_BLOCKS_K4 1
#endif
#ifndef TS_FUSED_MIN_PAIRS       // row pairs per warp: at least this many ...
#define TS_FUSED_MIN_PAIRS 4
#endif
#ifndef TS_FUSED_MAX_MIN_PAIRS   // ... and at most this many as the floor
#define TS_FUSED_MAX_MIN_PAIRS 16
#endif
#ifndef TS_FUSED_FILL_WARPS_PER_SM   // warps per SM that keep HBM busy
#define TS_FUSED_FILL_WARPS_PER_SM 8
#endif
#ifndef TS_FUSED_PINGPONG_MIN_K  // interior row pairs alternate two carry sets for K in
#define TS_FUSED_PINGPONG_MIN_K 3    // [MIN_K, MAX_K] (beyond MAX_K the second set spills)
#endif
#ifndef TS_FUSED_PINGPONG_MAX_K
#define TS_FUSED_PINGPONG_MAX_K 6
#endif
#ifndef TS_FUSED_ALIGNED         // 1: strip-aligned work split when strips <= warps
#define TS_FUSED_ALIGNED 1
#endif
#ifndef TS_FUSED_FFMA2           // packed FP32 FMAs (__ffma2_rn): see Cfg<K>::PACKED
#define TS_FUSED_FFMA2 1
#endif
#ifndef TS_FUSED_DRIVE_WARP_BRANCH   // drive phase: pick the short or the reduced series
#define TS_FUSED_DRIVE_WARP_BRANCH 1     // per warp (1) or per lane (0)
#endif
#ifndef TS_FUSED3D_WARPS         // 3-D steps: warps per CTA (two slabs each); the CTA's
#define TS_FUSED3D_WARPS 12      // first and last warp hold halo slabs
#endif
#ifndef TS_FUSED_PF_DUAL         // row pairs prefetched ahead of use by the backward
#define TS_FUSED_PF_DUAL 1       // adjoint steps (two states per slot); one row pair
#endif                           // ahead leaves room for 8 warps per SM at depth 3
constexpr int PLANE_SLOT_BYTES = FUSED_BOX_ROWS * FUSED_BOX_COLS * 4;   // 1 KiB
constexpr int SLOT_BYTES = 2 * PLANE_SLOT_BYTES;     // one ring slot: two planes of 2 rows
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;    // 2 s per wait
constexpr uint32_t FULL = 0xffffffffu;

// Two rings per warp, both indexed by the row pair j (rows Ys + 2j, +1):
//  - the state ring (re, im) is read once, when row pair j enters the
//    pipeline, so it needs PF + 1 slots;
//  - the phase ring (gamma_V, s_V) is read by the phase of every step, the
//    last one K row pairs later, so it needs PF + K + 1 slots.
// Shallow pipelines (K <= 2) are memory bound and prefetch deeper; deep ones
// are arithmetic bound and keep shared memory small for occupancy.
// Planes of a phase-ring slot: (gamma_V, s_V); with a drive (MODE 3) also
// V1.  The fused fourth-order step (MODE 4) keeps the a substep's table in
// the phase ring and the b substep's in a third, shorter ring (the b ring):
// only substep 2 reads it, at iterations j + 2 and j + 3 of row pair j.
// MODE 6 (3-D steps) holds the rows of two slabs per slot: (gamma_V, s_V) of
// each in the phase ring, (re, im) of each in the state ring.
__host__ __device__ constexpr int phase_planes(int mode)
{
    return mode == 3 ? 3 : mode == 6 ? 4 : 2;
}
// Planes of a state-ring slot: (re, im); the backward adjoint steps (MODE 5)
// carry two states, the forward state psi and the costate lambda.
__host__ __device__ constexpr int state_planes(int mode) { return mode == 5 || mode == 6 ? 4 : 2; }

// __launch_bounds__ minimum resident blocks of the single-grid kernel; the
// backward adjoint steps (MODE 5) carry two states and are not held to the
// forward depth's occupancy
__host__ __device__ constexpr int min_blocks(int K, int MODE = 0)
{
    return MODE == 5   ? TS_FUSED_MIN_BLOCKS
           : K == 3    ? TS_FUSED_MIN_BLOCKS_K3
           : K == 4    ? TS_FUSED_MIN_BLOCKS_K4
                       : TS_FUSED_MIN_BLOCKS;
}

// ... and of the multi-grid kernel
__host__ __device__ constexpr int multi_min_blocks(int K)
{
    return K == 3   ? TS_FUSED_MULTI_MIN_BLOCKS_K3
           : K == 4 ? TS_FUSED_MULTI_MIN_BLOCKS_K4
                    : TS_FUSED_MIN_BLOCKS;
}

template <int K, int PP = 2, bool BRING = false, int SP = 2, int M = 0>
struct Cfg {
    // MODE 6 (3-D steps): one CTA of TS_FUSED3D_WARPS warps, two slabs each
    static constexpr int WPC = M == 6 ? TS_FUSED3D_WARPS
                               : K <= 2 ? TS_FUSED_WPC_SHALLOW
                                        : TS_FUSED_WPC_DEEP;
    static constexpr int PF = M == 6   ? 1
                              : SP == 4 ? TS_FUSED_PF_DUAL
                              : K == 1 ? TS_FUSED_PF_K1
                              : K == 2 ? TS_FUSED_PF_K2
                                       : TS_FUSED_PF_DEEP;
    static constexpr bool PINGPONG = M != 5 && K >= TS_FUSED_PINGPONG_MIN_K && K <= TS_FUSED_PINGPONG_MAX_K;
    // The backward adjoint steps carry two states: one carry set, which
    // leaves registers for the deeper pipelines, and interior row pairs one
    // per loop trip instead of two, a smaller loop body (2-3 % faster for
    // them; about 1 % slower for one state and for the 3-D steps).
    static constexpr bool ONE_PAIR = M == 5;
    // packed FP32 FMAs in the Y sweeps and the phase: 0 never, 1 for every
    // depth but 2 (where the scalar form measured faster), 2 always
    static constexpr bool PACKED = TS_FUSED_FFMA2 == 2 || (TS_FUSED_FFMA2 == 1 && K != 2);
    static constexpr int NSS = PF + 1;
    // phase ring: the phase of step k at iteration j falls on rows 2(j - k)
    // - 1 and 2(j - k) of the range, so each slot is loaded one row earlier
    // than the state's (PSHIFT): a step then reads one slot, and the ring
    // holds K pairs and the PF ahead.  MODE 4 keeps slots on the state's
    // rows (a step reads pairs j - k - 1 and j - k: K + 1 pairs), as its b
    // ring does, and so does depth 1 outside MODE 6 (with the slot saved,
    // more depth-1 warps fit in shared memory, and they measured 11 % slower:
    // their halo columns are shared through L2 by warps that keep pace).
    static constexpr bool PSHIFT = M == 6 || (M != 4 && K >= 2);
    static constexpr int NSP = PF + K + (PSHIFT ? 0 : 1);
    static constexpr int HALO = ((2 * K + 3) / 4) * 4;
    static constexpr int VALID = FUSED_BOX_COLS - 2 * HALO;
    // a phase slot holds (gamma_V, s_V) and, with a drive, the V1 rows too
    static constexpr int PSLOT = PP * PLANE_SLOT_BYTES;
    // b ring (MODE 4): row pair r is read at iterations r + 2 and r + 3 and
    // waited for at r + 2, so the ring holds r in [j - 3, j - 2 + PF]
    static constexpr int NSB = BRING ? PF + 2 : 0;
    static constexpr int NBAR = NSS + NSP + NSB;   // mbarriers per warp
    static constexpr int SSLOT = SP * PLANE_SLOT_BYTES;   // a state slot
    // MODE 5: the running sums of G's terms of the row pairs in flight, two
    // rows for each of the steps 0 .. K - 2, [slot][re, im][lane] as float4
    static constexpr int SUMS_BYTES = M == 5 ? 2 * (K - 1) * 1024 : 0;
    // MODE 5: G's rows for the next commit, staged by cp.async (two rows of
    // four planes, [row][plane][lane] as float4)
    static constexpr int GST_BYTES = M == 5 ? 4096 : 0;
    static constexpr int WARP_SMEM = NSS * SSLOT + NSP * PSLOT + NSB * SLOT_BYTES + SUMS_BYTES + GST_BYTES;
    static constexpr int SMEM = 1024 + WPC * (WARP_SMEM + NBAR * 8);
};

// The configuration of a mode's kernel at depth K.
template <int K, int MODE>
using CfgM = Cfg<K, phase_planes(MODE), MODE == 4, state_planes(MODE), MODE>;

// Four columns of one row of one state, held by one lane.
struct Frag {
    float4 re, im;
};

// The same columns of two states that take the same factors: the forward
// state psi (a) and the costate lambda (b) of a backward adjoint step, or
// (MODE 6) the same row of two neighbouring slabs, z (a) and z + 1 (b).
struct Frag2 {
    Frag a, b;
};

// The per-lane state of a mode: one state, or two for the backward adjoint
// steps and the 3-D steps.
template <int MODE>
using StateT = std::conditional_t<MODE == 5 || MODE == 6, Frag2, Frag>;

struct KParams {
    float *out_re, *out_im;
    int nx, ny;
    int64_t pitch;
    int n_strips, n_pairs;
    int64_t units;
    int total_warps;
    int strip_warps;         // > 0: warps per strip of the strip-aligned split
    float t1, s1, g1, t2, s2;
    int *err;
    // MODE 5 (backward adjoint steps): the costate's output planes (out_re,
    // out_im take psi), and G as double-float planes (g_rh + g_rl,
    // g_ih + g_il).  At each step's phase point the lane's rows add
    // conj(lambda~) m, lambda~ = B^dagger lambda_s and m = B^dagger psi_s the
    // mid-step state; a row's K terms are summed in FP32 inside the launch
    // and added into G once.
    float *out2_re, *out2_im;
    float *g_rh, *g_rl, *g_ih, *g_il;
    // MODE 6 (3-D steps): slabs, z-blocks, row ranges per slab; ny is a
    // slab's rows and out_re, out_im point at slab z of the output planes,
    // out2_re, out2_im at slab z + 1 (the warp's two slabs)
    int nz, n_zblocks, n_ranges;
    // MODE 3 (time-dependent potential V0 + a(t) V1): a_n dt of step k of
    // the launch; the phase ring carries V1 as a third plane
    float adt[FUSED_MAX_K];
    // MODE 4 (one fourth-order step U4 = a a b a a, K = 5): t1, s1, g1, t2,
    // s2 are the a substep's; the b substep's angle (lifting tb, sb; versine
    // gb) and the merged angle of an a-b boundary (lifting tab, sab)
    float tb, sb, gb, tab, sab;
};

// ---- PTX wrappers (the mbarrier helpers are in mbar.cuh) ------------------
// Make a tensor map that was written to global memory before this launch
// visible to the TMA unit (its descriptor cache is not coherent with writes).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *tm)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(tm))
                 : "memory");
}

// One box of two planes: x in [x, x+128), rows y, y+1, planes 0 and 1.
__device__ __forceinline__ void tma_load_pair(void *dst, const CUtensorMap *tm, int x, int y,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(0), "r"(smem_addr(bar))
        : "memory");
}

// ---- register-level sweeps ------------------------------------------------
// A pair rotation a' = c a + i s b, b' = i s a + c b splits into two real
// plane rotations, of (a_re, b_im) and of (b_re, a_im), each by theta:
//   x' = c x - s y, y' = s x + c y.
// When a lane holds both members it applies each as three shears
//   x -= t y;  y += s x;  x -= t y      (t = tan(theta/2), s = sin theta),
// 6 FMA per pair instead of 8; every shear has determinant 1.  A lane that
// holds one member of a pair (the pair straddling two lanes) updates only
// that member, in the versine form a' = a - g a + i s b (4 FMA).
struct XEven {
    float t0, s0, t1, s1;   // pairs (c0,c1) and (c2,c3) of the lane's float4, lifting form
};
struct XOdd {
    float t0, s0;           // pair (c1,c2), inside the lane, lifting form
    float gR, sR;           // pair (c3, next lane's c0), versine form
    float gL, sL;           // pair (previous lane's c3, c0), versine form
};

__device__ __forceinline__ void x_even(Frag &f, const XEven &c)
{
    rot_lift(f.re.x, f.im.x, f.re.y, f.im.y, c.t0, c.s0);
    rot_lift(f.re.z, f.im.z, f.re.w, f.im.w, c.t1, c.s1);
}

__device__ __forceinline__ void x_odd(Frag &f, const XOdd &c)
{
    const float nr = __shfl_down_sync(FULL, f.re.x, 1);
    const float ni = __shfl_down_sync(FULL, f.im.x, 1);
    const float pr = __shfl_up_sync(FULL, f.re.w, 1);
    const float pi = __shfl_up_sync(FULL, f.im.w, 1);
    rot_lift(f.re.y, f.im.y, f.re.z, f.im.z, c.t0, c.s0);
    rot1(f.re.w, f.im.w, nr, ni, c.gR, c.sR);
    rot1(f.re.x, f.im.x, pr, pi, c.gL, c.sL);
}

// Packed forms (Cfg<K>::PACKED): the column halves (x, y) and (z, w) of a
// lane's float4 are register pairs, and __ffma2_rn applies one FMA to both
// elements with the rounding of fmaf, so the results are bit for bit those of
// the scalar forms with half the FMA instructions.  Used where the members
// of every pair sit in the same column (Y sweeps, the phase).

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 join2(float2 lo, float2 hi)
{
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// rot_lift on two columns at once; nt = (-t, -t), s2 = (s, s)
__device__ __forceinline__ void rot_lift2(float2 &ar, float2 &ai, float2 &br, float2 &bi,
                                          float2 nt, float2 s2)
{
    ar = __ffma2_rn(nt, bi, ar);
    br = __ffma2_rn(nt, ai, br);
    bi = __ffma2_rn(s2, ar, bi);
    ai = __ffma2_rn(s2, br, ai);
    ar = __ffma2_rn(nt, bi, ar);
    br = __ffma2_rn(nt, ai, br);
}

// phase1 on two columns at once: r - g r + s m, m - g m - s r
__device__ __forceinline__ void phase2(float2 &r, float2 &m, float2 g, float2 s)
{
    const float2 ng = make_float2(-g.x, -g.y), ns = make_float2(-s.x, -s.y);
    const float2 nr = __ffma2_rn(s, m, __ffma2_rn(ng, r, r));
    m = __ffma2_rn(ns, r, __ffma2_rn(ng, m, m));
    r = nr;
}

// Y pair rotation of two rows (all four columns of the lane), lifting form.
template <bool PACKED>
__device__ __forceinline__ void y_pair(Frag &a, Frag &b, float t, float s)
{
    if constexpr (PACKED) {
    const float2 nt = make_float2(-t, -t), s2 = make_float2(s, s);
    float2 ar = lo2(a.re), ai = lo2(a.im), br = lo2(b.re), bi = lo2(b.im);
    float2 cr = hi2(a.re), ci = hi2(a.im), dr = hi2(b.re), di = hi2(b.im);
    rot_lift2(ar, ai, br, bi, nt, s2);
    rot_lift2(cr, ci, dr, di, nt, s2);
    a.re = join2(ar, cr);
    a.im = join2(ai, ci);
    b.re = join2(br, dr);
    b.im = join2(bi, di);
    } else {
    rot_lift(a.re.x, a.im.x, b.re.x, b.im.x, t, s);
    rot_lift(a.re.y, a.im.y, b.re.y, b.im.y, t, s);
    rot_lift(a.re.z, a.im.z, b.re.z, b.im.z, t, s);
    rot_lift(a.re.w, a.im.w, b.re.w, b.im.w, t, s);
    }
}

template <bool PACKED>
__device__ __forceinline__ void phase4(Frag &f, float4 g, float4 s)
{
    if constexpr (PACKED) {
    float2 r0 = lo2(f.re), m0 = lo2(f.im), r1 = hi2(f.re), m1 = hi2(f.im);
    phase2(r0, m0, lo2(g), lo2(s));
    phase2(r1, m1, hi2(g), hi2(s));
    f.re = join2(r0, r1);
    f.im = join2(m0, m1);
    } else {
    phase1(f.re.x, f.im.x, g.x, s.x);
    phase1(f.re.y, f.im.y, g.y, s.y);
    phase1(f.re.z, f.im.z, g.z, s.z);
    phase1(f.re.w, f.im.w, g.w, s.w);
    }
}

// Both states of a backward adjoint step take the same factor.
__device__ __forceinline__ void x_even(Frag2 &f, const XEven &c)
{
    x_even(f.a, c);
    x_even(f.b, c);
}

__device__ __forceinline__ void x_odd(Frag2 &f, const XOdd &c)
{
    x_odd(f.a, c);
    x_odd(f.b, c);
}

template <bool PACKED>
__device__ __forceinline__ void y_pair(Frag2 &a, Frag2 &b, float t, float s)
{
    y_pair<PACKED>(a.a, b.a, t, s);
    y_pair<PACKED>(a.b, b.b, t, s);
}

template <bool PACKED>
__device__ __forceinline__ void phase4(Frag2 &f, float4 g, float4 s)
{
    phase4<PACKED>(f.a, g, s);
    phase4<PACKED>(f.b, g, s);
}

// Drive phase exp(-i a dt V1) of one row of the lane (time-dependent
// potential): adt = a_n dt of the step, v1 = the row's V1 values, so the
// angle of a site is phi = adt V1.  With u = phi^2, sin(phi) = phi P(u) and
// 1 - cos(phi) = u Q(u), P and Q cubics in u fitted to sin(x)/x and
// (1 - cos x)/x^2 on u in [0, 0.64] (|phi| <= 0.8) by the Remez exchange
// (equal-ripple absolute error) and rounded to FP32: they are within 6.8e-9
// and 6.7e-10 of the functions there, and an FP32 emulation of this
// evaluation gives relative errors under 1.5e-7 in both results, as the
// Taylor polynomials through u^4 did with one more FMA each (3 % slower: the
// kernel is bound by instruction issue).  (A second, shorter series for
// smaller angles measured slower too.)
constexpr float DRIVE_P1 = -0x1.55553ep-3f, DRIVE_P2 = 0x1.11055ep-7f, DRIVE_P3 = -0x1.98c40ap-13f;
constexpr float DRIVE_Q1 = -0x1.55554cp-5f, DRIVE_Q2 = 0x1.6c0d6p-10f, DRIVE_Q3 = -0x1.9a398ap-16f;

__device__ __forceinline__ void versine_phi2(float2 phi, float2 &g, float2 &s)
{
    auto c2 = [](float v) { return make_float2(v, v); };
    const float2 u = __fmul2_rn(phi, phi);
    float2 P = __ffma2_rn(u, c2(DRIVE_P3), c2(DRIVE_P2));
    float2 Q = __ffma2_rn(u, c2(DRIVE_Q3), c2(DRIVE_Q2));
    P = __ffma2_rn(u, P, c2(DRIVE_P1));
    Q = __ffma2_rn(u, Q, c2(DRIVE_Q1));
    P = __ffma2_rn(u, P, c2(1.0f));
    Q = __ffma2_rn(u, Q, c2(0.5f));
    s = __fmul2_rn(phi, P);
    g = __fmul2_rn(u, Q);
}

// The same on one column (same operations, same rounding).
__device__ __forceinline__ void versine_phi(float phi, float &g, float &s)
{
    const float u = phi * phi;
    float P = fmaf(u, DRIVE_P3, DRIVE_P2);
    float Q = fmaf(u, DRIVE_Q3, DRIVE_Q2);
    P = fmaf(u, P, DRIVE_P1);
    Q = fmaf(u, Q, DRIVE_Q1);
    P = fmaf(u, P, 1.0f);
    Q = fmaf(u, Q, 0.5f);
    s = phi * P;
    g = u * Q;
}

template <bool PACKED>
__device__ __forceinline__ void versine_phi4(float4 phi, float4 &g, float4 &s)
{
    if constexpr (PACKED) {
        float2 g0, s0, g1, s1;
        versine_phi2(lo2(phi), g0, s0);
        versine_phi2(hi2(phi), g1, s1);
        g = join2(g0, g1);
        s = join2(s0, s1);
    } else {
        versine_phi(phi.x, g.x, s.x);
        versine_phi(phi.y, g.y, s.y);
        versine_phi(phi.z, g.z, s.z);
        versine_phi(phi.w, g.w, s.w);
    }
}

template <bool PACKED>
__device__ __forceinline__ void drive4(Frag &f, float4 v1, float adt)
{
    // the angles of the lane's four columns; the series serves when every
    // angle in the warp is at most 0.8 -- decided for the whole warp, so that
    // the branch does not diverge (all lanes are converged here); larger
    // angles take the reduced path, on the half angle
    float4 phi;
    if constexpr (PACKED) {
        const float2 a2 = make_float2(adt, adt);
        phi = join2(__fmul2_rn(a2, lo2(v1)), __fmul2_rn(a2, hi2(v1)));
    } else {
        phi = make_float4(adt * v1.x, adt * v1.y, adt * v1.z, adt * v1.w);
    }
    float4 g, s;
    const float m = fmaxf(fmaxf(fabsf(phi.x), fabsf(phi.y)), fmaxf(fabsf(phi.z), fabsf(phi.w)));
    auto all = [](bool b) { return TS_FUSED_DRIVE_WARP_BRANCH ? __all_sync(FULL, b) : b; };
    if (all(m <= 0.8f)) {
        versine_phi4<PACKED>(phi, g, s);
    } else {
        const float4 h = make_float4(0.5f * phi.x, 0.5f * phi.y, 0.5f * phi.z, 0.5f * phi.w);
        versine_reduced(h.x, g.x, s.x);
        versine_reduced(h.y, g.y, s.y);
        versine_reduced(h.z, g.z, s.z);
        versine_reduced(h.w, g.w, s.w);
    }
    phase4<PACKED>(f, g, s);
}

__device__ __forceinline__ Frag zero_frag()
{
    Frag f;
    f.re = make_float4(0.f, 0.f, 0.f, 0.f);
    f.im = f.re;
    return f;
}

template <typename S>
__device__ __forceinline__ S zero_state()
{
    if constexpr (std::is_same_v<S, Frag2>)
        return Frag2{zero_frag(), zero_frag()};
    else
        return zero_frag();
}

// Slot layout: [plane][row][128 floats]; state slots hold (re, im), phase
// slots hold (gamma_V, s_V).
__device__ __forceinline__ float4 lds4(const unsigned char *slot, int plane, int row, int lane)
{
    return *reinterpret_cast<const float4 *>(slot + plane * PLANE_SLOT_BYTES +
                                             row * (FUSED_BOX_COLS * 4) + lane * 16);
}

// Per-lane coefficients of one strip (x masks applied) and the scalars.
struct StripCoef {
    XEven E1, E2;   // even pairs at theta and 2 theta
    XOdd O;         // odd pairs at theta
    XOdd Ob;        // MODE 4: odd pairs at the b substep's angle
    XEven Eab;      // MODE 4: even pairs at the a + b angle
};

// Rows and columns this warp owns in its current row range.
struct Owned {
    int Y0, Y1;        // output rows [Y0, Y1)
    int xg;            // the lane's first column
    bool lane_ok;      // the lane's 4 columns are inside the valid strip and < nx
    float4 *sums;      // MODE 5: the lane's running sums (shared memory)
    float4 *gst;       // MODE 5: the lane's staged G rows (shared memory)
};

__device__ __forceinline__ bool owns_row(const Owned &w, const KParams &p, int row)
{
    return w.lane_ok && row >= w.Y0 && row < w.Y1 && row < p.ny;
}

// Adjoint hooks.  At the phase point of a backward step the lane's rows of
// the costate, lt = B^dagger lambda_s, meet the mid-step state of the same
// step, m = B^dagger psi_s: the term conj(lt) m = (lr mr + li mi) + i (lr mi - li mr).
__device__ __forceinline__ Frag adj_term(const Frag &lt, const Frag &m)
{
    Frag t;
    t.re = make_float4(fmaf(lt.re.x, m.re.x, lt.im.x * m.im.x),
                       fmaf(lt.re.y, m.re.y, lt.im.y * m.im.y),
                       fmaf(lt.re.z, m.re.z, lt.im.z * m.im.z),
                       fmaf(lt.re.w, m.re.w, lt.im.w * m.im.w));
    t.im = make_float4(fmaf(lt.re.x, m.im.x, -lt.im.x * m.re.x),
                       fmaf(lt.re.y, m.im.y, -lt.im.y * m.re.y),
                       fmaf(lt.re.z, m.im.z, -lt.im.z * m.re.z),
                       fmaf(lt.re.w, m.im.w, -lt.im.w * m.re.w));
    return t;
}

__device__ __forceinline__ Frag frag_add(const Frag &a, const Frag &b)
{
    Frag r;
    r.re = make_float4(a.re.x + b.re.x, a.re.y + b.re.y, a.re.z + b.re.z, a.re.w + b.re.w);
    r.im = make_float4(a.im.x + b.im.x, a.im.y + b.im.y, a.im.z + b.im.z, a.im.w + b.im.w);
    return r;
}

// G's rows are staged in shared memory by cp.async one iteration before the
// terms are added to them, so their loads overlap the iteration's sweeps
// (plain loads at the commit left the kernel waiting on them).  Each lane
// copies its own 16 bytes of each plane and reads back only those, so the
// lane's own wait orders the accesses.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// stage slot `slot` (0 or 1) of the lane: [plane rh, rl, ih, il][lane]
__device__ __forceinline__ void adj_stage(int row, int slot, const Owned &w, const KParams &p)
{
    const int64_t o = (int64_t)row * p.pitch + w.xg;
    float4 *st = w.gst + slot * 128;
    cp_async16(st, p.g_rh + o);
    cp_async16(st + 32, p.g_rl + o);
    cp_async16(st + 64, p.g_ih + o);
    cp_async16(st + 96, p.g_il + o);
}

// G += t for one owned row, in double-float (hi + lo planes, Knuth's
// two-sum), from its staged values
__device__ __forceinline__ void adj_commit(const Frag &t, int row, int slot, const Owned &w,
                                           const KParams &p)
{
    const int64_t o = (int64_t)row * p.pitch + w.xg;
    const float4 *st = w.gst + slot * 128;
    float4 rh = st[0], rl = st[32], ih = st[64], il = st[96];
    auto acc = [](float &hi, float &lo, float v) {
        FF s = two_sum(hi, v);
        s.lo += lo;
        s = fast_two_sum(s.hi, s.lo);
        hi = s.hi;
        lo = s.lo;
    };
    acc(rh.x, rl.x, t.re.x);
    acc(rh.y, rl.y, t.re.y);
    acc(rh.z, rl.z, t.re.z);
    acc(rh.w, rl.w, t.re.w);
    acc(ih.x, il.x, t.im.x);
    acc(ih.y, il.y, t.im.y);
    acc(ih.z, il.z, t.im.z);
    acc(ih.w, il.w, t.im.w);
    *reinterpret_cast<float4 *>(p.g_rh + o) = rh;
    *reinterpret_cast<float4 *>(p.g_rl + o) = rl;
    *reinterpret_cast<float4 *>(p.g_ih + o) = ih;
    *reinterpret_cast<float4 *>(p.g_il + o) = il;
}

// MODE 5 at the phase point of step k of the launch, rows (y1, y1 + 1) held
// in (P, Q) (psi in .a, lambda in .b).  The pair reached step k here one
// iteration after it reached step k - 1, so its running sum waits in shared
// memory between iterations: sum slots 2k and 2k + 1 hold the sum of the pair
// that is at step k now; car passes the sum of step k - 1 from the previous
// iteration to this step.  Step K - 1 adds the finished sum into G (owned
// rows only; other rows' sums are never stored).  Each lane touches only its
// own entries, so no synchronisation is needed.
template <int K>
__device__ __forceinline__ void adj_step(int k, const Frag2 &P, const Frag2 &Q, int y1,
                                         Frag &carP, Frag &carQ, const Owned &w,
                                         const KParams &p)
{
    Frag tP = adj_term(P.b, P.a), tQ = adj_term(Q.b, Q.a);
    if (k > 0) {
        tP = frag_add(carP, tP);
        tQ = frag_add(carQ, tQ);
    }
    if (k == K - 1) {
        // rows (y1, y1 + 1) were staged by the previous iteration, which
        // committed (y1 - 2, y1 - 1); stage the next iteration's rows
        cp_async_wait_all();
        if (owns_row(w, p, y1)) adj_commit(tP, y1, 0, w, p);
        if (owns_row(w, p, y1 + 1)) adj_commit(tQ, y1 + 1, 1, w, p);
        if (owns_row(w, p, y1 + 2)) adj_stage(y1 + 2, 0, w, p);
        if (owns_row(w, p, y1 + 3)) adj_stage(y1 + 3, 1, w, p);
        cp_async_commit();
    } else {
        float4 *a0 = w.sums + 2 * k * 64, *a1 = a0 + 64;
        carP.re = a0[0];
        carP.im = a0[32];
        carQ.re = a1[0];
        carQ.im = a1[32];
        a0[0] = tP.re;
        a0[32] = tP.im;
        a1[0] = tQ.re;
        a1[32] = tQ.im;
    }
}

__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// One row pair through the K-step pipeline.  The carried rows come in through
// `cin` and leave through `cout` (each slot is read before it is written, so
// the two may be the same array).  INTERIOR: every Y pair and
// every phase row the iteration touches lies on the grid and in the ring,
// so no masks or range checks are needed.  MODE 0: plain steps; MODE 3: a
// time-dependent potential; MODE 4: one fourth-order step; MODE 5: backward
// adjoint steps U^dagger on two states (the caller passes the coefficients at
// -theta; the phase is conjugated here) that accumulate G at each step's
// phase point, with the running sums of the rows in flight in shared memory
// (updated in place).
template <int K, bool INTERIOR, int MODE, typename S = StateT<MODE>>
__device__ __forceinline__ void pipeline_step(const S (&cin)[2 * K], S (&cout)[2 * K],
                                              S a, S b, int yin, int j,
                                              const unsigned char *ring_p, int pos_p,
                                              const unsigned char *ring_b, int cnt_b,
                                              const StripCoef &c, const KParams &p, int lane,
                                              const Owned &w, S &O0, S &O1)
{
    static_assert(MODE != 4 || K == 5, "the fused fourth-order step has five substeps");
    using C = CfgM<K, MODE>;
    constexpr bool CONJ = MODE == 5;   // backward steps: exp(+i V dt), sine -s_V
    // MODE 4: substep k of U4 = a a b a a is b for k == 2 (angle and table)
    auto is_b = [](int k) { return MODE == 4 && k == 2; };
    constexpr int NSP = C::NSP;
    auto yok = [&](int y) {
        return INTERIOR || (y >= 0 && y + 1 < p.ny);
    };
    auto slot_p = [&](int back) -> const unsigned char * {   // phase slot j - back
        int q = pos_p - back;
        if (q < 0) q += NSP;
        return ring_p + q * C::PSLOT;
    };
    auto slot_b = [&](int back) -> const unsigned char * {   // b-ring slot of row pair j - back
        return ring_b + ((cnt_b + j - back) % (C::NSB > 0 ? C::NSB : 1)) * SLOT_BYTES;
    };
    // step 0, first half: Xe, Xo (row-local), Ye aligned, Yo shifted
    x_even(a, c.E1);
    x_even(b, c.E1);
    x_odd(a, c.O);
    x_odd(b, c.O);
    {
        const bool v = yok(yin);
        y_pair<C::PACKED>(a, b, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
    }
    S P = cin[0], Q = a;          // rows (yin-1, yin)
    {
        const bool v = yok(yin - 1);
        y_pair<C::PACKED>(P, Q, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
    }
    cout[0] = b;
    int y1 = yin - 1;
    Frag carP, carQ;   // MODE 5: running sums handed from step k - 1 to step k
    if constexpr (MODE == 5) adj_step<K>(0, P, Q, y1, carP, carQ, w, p);
    // the phase of step k on one row from phase slot sp (row 0 or 1 of the
    // slot): conjugated in a backward step (exp(+i V dt) has sine -s_V); with
    // the drive term for MODE 3; MODE 6 holds two slabs, each with its table
    auto phase_row = [&](S &X, const unsigned char *sp, int row, int k) {
        if constexpr (MODE == 6) {
            phase4<C::PACKED>(X.a, lds4(sp, 0, row, lane), lds4(sp, 1, row, lane));
            phase4<C::PACKED>(X.b, lds4(sp, 2, row, lane), lds4(sp, 3, row, lane));
        } else {
            const float4 sv = lds4(sp, 1, row, lane);
            phase4<C::PACKED>(X, lds4(sp, 0, row, lane), CONJ ? neg4(sv) : sv);
            if constexpr (MODE == 3) drive4<C::PACKED>(X, lds4(sp, 2, row, lane), p.adt[k]);
        }
    };
    // phase of step 0 on rows (y1, y1+1): rows 0 and 1 of slot j (without
    // PSHIFT: slot j-1 row 1, slot j row 0)
    if constexpr (C::PSHIFT) {
        phase_row(P, slot_p(0), 0, 0);
        phase_row(Q, slot_p(0), 1, 0);
    } else {
        if (INTERIOR || j >= 1) phase_row(P, slot_p(1), 1, 0);
        phase_row(Q, slot_p(0), 0, 0);
    }
#pragma unroll
    for (int k = 1; k < K; ++k) {
        // angles of the two steps that meet here (MODE 4: a or b) and of
        // their merged factors (2a, or a + b)
        const bool bp = is_b(k - 1), bk = is_b(k), mixed = bp != bk;
        const float tp = bp ? p.tb : p.t1, sp_ = bp ? p.sb : p.s1;
        const float tk = bk ? p.tb : p.t1, sk = bk ? p.sb : p.s1;
        const float tm = mixed ? p.tab : p.t2, sm = mixed ? p.sab : p.s2;
        const XOdd &Op = bp ? c.Ob : c.O, &Ok = bk ? c.Ob : c.O;
        const XEven &Em = mixed ? c.Eab : c.E2;
        {   // Yo (theta of step k-1), aligned on (y1, y1+1), y1 odd
            const bool v = yok(y1);
            y_pair<C::PACKED>(P, Q, v ? tp : 0.f, v ? sp_ : 0.f);
        }
        // X group between two phases: Xo, Xe(merged), Xo
        x_odd(P, Op);
        x_odd(Q, Op);
        x_even(P, Em);
        x_even(Q, Em);
        x_odd(P, Ok);
        x_odd(Q, Ok);
        S P2 = cin[2 * k - 1], Q2 = P;        // rows (y1-1, y1)
        {   // Ye (merged), shifted: pair (y1-1, y1)
            const bool v = yok(y1 - 1);
            y_pair<C::PACKED>(P2, Q2, v ? tm : 0.f, v ? sm : 0.f);
        }
        cout[2 * k - 1] = Q;
        P = cin[2 * k];                       // rows (y1-2, y1-1)
        {   // Yo (theta of step k), shifted: pair (y1-2, y1-1)
            const bool v = yok(y1 - 2);
            y_pair<C::PACKED>(P, P2, v ? tk : 0.f, v ? sk : 0.f);
        }
        cout[2 * k] = Q2;
        Q = P2;
        y1 -= 2;
        if constexpr (MODE == 5) adj_step<K>(k, P, Q, y1, carP, carQ, w, p);
        // phase of step k on rows (y1, y1+1): rows 0 and 1 of slot j-k
        // (without PSHIFT, MODE 4: slot j-k-1 row 1, slot j-k row 0, and the
        // b substep's table from the b ring; MODE 5: the conjugate phase,
        // sine -s_V)
        auto slot_k = [&](int back) { return bk ? slot_b(back) : slot_p(back); };
        if constexpr (C::PSHIFT) {
            if (INTERIOR || j - k >= 0) {   // rows 0 and 1 of slot j-k
                phase_row(P, slot_p(k), 0, k);
                phase_row(Q, slot_p(k), 1, k);
            }
        } else {
            if (INTERIOR || j - k - 1 >= 0) phase_row(P, slot_k(k + 1), 1, k);
            if (INTERIOR || j - k >= 0) phase_row(Q, slot_k(k), 0, k);
        }
    }
    // last step, second half: Yo aligned, Ye shifted, Xo, Xe
    {
        const bool v = yok(y1);
        y_pair<C::PACKED>(P, Q, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
    }
    O0 = cin[2 * K - 1];      // rows (y1-1, y1) = (yin-2K, yin-2K+1)
    O1 = P;
    {
        const bool v = yok(y1 - 1);
        y_pair<C::PACKED>(O0, O1, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
    }
    cout[2 * K - 1] = Q;
    x_odd(O0, c.O);
    x_odd(O1, c.O);
    x_even(O0, c.E1);
    x_even(O1, c.E1);
}

// A warp's two slot rings: barriers, buffers, and the ring positions and
// mbarrier phase parities of the next row pair to be consumed (they carry
// over from one row range to the next).
struct WarpRings {
    uint64_t *bar_s, *bar_p, *bar_b;
    unsigned char *ring_s, *ring_p, *ring_b;
    float4 *sums, *gst;   // MODE 5: running sums, staged G rows (this lane's)
    int pos_s, pos_p;
    uint32_t par_s, par_p;
    // b ring: b copies are numbered across the warp's segments; copy L sits
    // in slot L % NSB with mbarrier phase parity (L / NSB) & 1, and cnt_b
    // copies came before the current segment (row pair r is copy cnt_b + r)
    int cnt_b;
};

template <int K, int PP = 2, bool BRING = false, int SP = 2, int M = 0>
__device__ __forceinline__ WarpRings carve_rings(unsigned char *smem_raw, int warp, int lane)
{
    using C = Cfg<K, PP, BRING, SP, M>;
    constexpr int NSS = C::NSS, NSP = C::NSP, NBAR = C::NBAR;
    WarpRings r;
    // barriers first, then 1 KiB-aligned slots (state ring, phase ring, b ring)
    r.bar_s = reinterpret_cast<uint64_t *>(smem_raw) + warp * NBAR;
    r.bar_p = r.bar_s + NSS;
    r.bar_b = r.bar_p + NSP;
    const uint32_t base_addr = smem_addr(smem_raw);
    const uint32_t slots_off =
        ((base_addr + C::WPC * NBAR * 8 + 1023u) & ~1023u) - base_addr;
    r.ring_s = smem_raw + slots_off + (size_t)warp * C::WARP_SMEM;
    r.ring_p = r.ring_s + NSS * C::SSLOT;
    r.ring_b = r.ring_p + NSP * C::PSLOT;
    r.sums = reinterpret_cast<float4 *>(r.ring_b + C::NSB * SLOT_BYTES) + lane;
    r.gst = reinterpret_cast<float4 *>(r.ring_b + C::NSB * SLOT_BYTES + C::SUMS_BYTES) + lane;
    r.pos_s = r.pos_p = 0;
    r.par_s = r.par_p = 0;
    r.cnt_b = 0;
    if (lane == 0) {
        for (int i = 0; i < NBAR; ++i) mbar_init(&r.bar_s[i], 1);
        fence_mbar_init();
    }
    __syncwarp();
    return r;
}

// Stream the row pairs [q0, q1) of strip sx of one grid through the K-step
// pipeline: rows [2 q0, 2 q1) are written to (p.out_re, p.out_im).  Returns
// false if a bounded wait gave up (the error bit is set and this warp's
// outstanding copies are drained).
// Per-segment constants of one warp.
struct Seg {
    const CUtensorMap *tm_state, *tm_phase, *tm_b;
    int XL, xg, Y0, Y1, Ys, n_iter, lane;
    int ytma;                // added to row coordinates of TMA copies (MODE 6: z ny)
    int yslab;               // MODE 6: rows from slab z to slab z + 1
    bool store_lane;
    StripCoef c;
    Owned own;
    // MODE 6: the warp's lower slab z (even), its index in the CTA, and
    // which of its two slabs (z, z + 1) it writes
    int z, w;
    bool store_a, store_b;
};

// MODE 6: where a warp sits in its CTA's block of slabs.
struct Slab3 {
    int z = 0, w = 0, ytma = 0;
    bool store_a = true, store_b = true;
};

// MODE 6 (TWO): one slot takes the rows of slab z and then those of slab
// z + 1 (yslab rows further on), two copies on one mbarrier.
template <int SSLOT, bool TWO = false>
__device__ __forceinline__ void issue_state(WarpRings &r, const Seg &s, int pos, int j)
{
    mbar_expect_tx(&r.bar_s[pos], SSLOT);
    unsigned char *dst = r.ring_s + pos * SSLOT;
    const int y = s.ytma + s.Ys + 2 * j;
    tma_load_pair(dst, s.tm_state, s.XL, y, &r.bar_s[pos]);
    if constexpr (TWO) tma_load_pair(dst + SSLOT / 2, s.tm_state, s.XL, y + s.yslab, &r.bar_s[pos]);
}

// b ring (MODE 4): the b substep's (gamma, s) rows of row pair j, copy
// number r.cnt_b + j
template <int NSB>
__device__ __forceinline__ void issue_b(WarpRings &r, const Seg &s, int j)
{
    const int pos = (r.cnt_b + j) % NSB;
    mbar_expect_tx(&r.bar_b[pos], SLOT_BYTES);
    tma_load_pair(r.ring_b + pos * SLOT_BYTES, s.tm_b, s.XL, s.Ys + 2 * j, &r.bar_b[pos]);
}

template <int NSB>
__device__ __forceinline__ bool wait_b(const WarpRings &r, int j, uint64_t limit)
{
    const int L = r.cnt_b + j;
    return mbar_wait(&r.bar_b[L % NSB], (uint32_t)(L / NSB) & 1u, limit);
}

// SHIFT: rows 2j - 1 and 2j of the range instead of 2j and 2j + 1 (a row
// outside the grid is off-grid in the pipeline, whatever it reads: zeros,
// or for MODE 6 a row of the neighbouring slab).
template <int K, int PP, bool TWO, bool SHIFT>
__device__ __forceinline__ void issue_phase(WarpRings &r, const Seg &s, int pos, int j)
{
    constexpr int PSLOT = Cfg<K, PP>::PSLOT;
    mbar_expect_tx(&r.bar_p[pos], PSLOT);
    unsigned char *dst = r.ring_p + pos * PSLOT;
    const int y = s.ytma + s.Ys + 2 * j - (SHIFT ? 1 : 0);
    tma_load_pair(dst, s.tm_phase, s.XL, y, &r.bar_p[pos]);
    if constexpr (TWO) tma_load_pair(dst + PSLOT / 2, s.tm_phase, s.XL, y + s.yslab, &r.bar_p[pos]);
}

// MODE 6: the Z sweeps of the two rows (r0, r1) that every warp of the CTA
// holds at the same y; warp w holds slabs z = z_w (even, in .a) and z + 1
// (in .b).  Even Z pairs (z, z + 1) lie inside a warp: a register rotation
// (lifting form).  Odd pairs (z + 1, z + 2) and (z - 1, z) join neighbouring
// warps: each warp puts its rows in an exchange buffer, the CTA meets at a
// barrier, and each warp updates its own members from their partners' old
// values in the versine form (a' = a - g a + i s b).  A pair needs both slabs
// on the grid and both in the CTA.
//
// The buffers are ring slots the warp has just consumed, at the same place in
// every warp's rings (the warps walk the same row pairs): the first exchange
// of row pair j goes through its state slot, whose refill is issued after
// the second barrier; the second through its phase slot, whose refill waits
// for the first barrier of row pair j + 1 (or the barrier that ends the
// segment).  So no warp overwrites rows another warp still reads.
__device__ __forceinline__ bool on_grid(int z, const KParams &p) { return z >= 0 && z < p.nz; }

template <bool PACKED>
__device__ __forceinline__ void z_even(Frag2 &r0, Frag2 &r1, const Seg &s, const KParams &p)
{
    const bool v = on_grid(s.z, p) && on_grid(s.z + 1, p);
    y_pair<PACKED>(r0.a, r0.b, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
    y_pair<PACKED>(r1.a, r1.b, v ? p.t1 : 0.f, v ? p.s1 : 0.f);
}

// `mine` is this warp's buffer (256 float4 = 4 KiB); the neighbours' lie
// WSTRIDE float4 away.  The barrier of the exchange also combines the warps'
// `fail` flags: it returns true, in every warp, if any warp of the CTA passed
// true.  The buffer's later refill is a TMA write (the async proxy), so each
// lane fences its generic writes before the barrier.  `after` runs right
// after the barrier unless a warp failed: the slots that the barrier frees
// are refilled there, before this exchange's reads and updates.
template <int NW, int WSTRIDE, typename F>
__device__ __forceinline__ bool z_odd(Frag2 &r0, Frag2 &r1, const Seg &s, const KParams &p,
                                      float4 *mine, bool fail, F &&after)
{
    const int lane = s.lane;
    mine[lane] = r0.a.re;
    mine[32 + lane] = r0.a.im;
    mine[64 + lane] = r1.a.re;
    mine[96 + lane] = r1.a.im;
    mine[128 + lane] = r0.b.re;
    mine[160 + lane] = r0.b.im;
    mine[192 + lane] = r1.b.re;
    mine[224 + lane] = r1.b.im;
    fence_proxy_async();
    const bool any_fail = __syncthreads_or(fail);
    if (any_fail) return true;
    after();
    const float g = p.g1, sn = p.s1;
    const float2 ng = make_float2(-g, -g), ns = make_float2(-sn, -sn), ps = make_float2(sn, sn);
    auto one = [&](Frag &f, const float4 *q, int row) {   // f <- f - g f + i s q, four columns
        const float4 qr = q[64 * row + lane], qi = q[64 * row + 32 + lane];
        const float2 r0n = __ffma2_rn(ns, lo2(qi), __ffma2_rn(ng, lo2(f.re), lo2(f.re)));
        const float2 m0n = __ffma2_rn(ps, lo2(qr), __ffma2_rn(ng, lo2(f.im), lo2(f.im)));
        const float2 r1n = __ffma2_rn(ns, hi2(qi), __ffma2_rn(ng, hi2(f.re), hi2(f.re)));
        const float2 m1n = __ffma2_rn(ps, hi2(qr), __ffma2_rn(ng, hi2(f.im), hi2(f.im)));
        f.re = join2(r0n, r1n);
        f.im = join2(m0n, m1n);
    };
    // slab z + 1 with the next warp's slab z + 2 (its .a rows)
    if (s.w + 1 < NW && on_grid(s.z + 1, p) && on_grid(s.z + 2, p)) {
        const float4 *q = mine + WSTRIDE;
        one(r0.b, q, 0);
        one(r1.b, q, 1);
    }
    // slab z with the previous warp's slab z - 1 (its .b rows)
    if (s.w > 0 && on_grid(s.z - 1, p) && on_grid(s.z, p)) {
        const float4 *q = mine - WSTRIDE + 128;
        one(r0.a, q, 0);
        one(r1.a, q, 1);
    }
    return false;
}

// Row pair j of a segment: wait for its slots, run the pipeline, store the
// finished rows, refill the freed slots.  Returns false if a bounded wait
// gave up (after setting the error bit and draining this warp's copies).
// Copies issued so far into each ring of a segment (row pairs [0, n)).
struct Issued {
    int s, p, b;
};

template <int K, int MODE, bool INTERIOR, typename S = StateT<MODE>>
__device__ __forceinline__ bool row_pair(WarpRings &r, const Seg &s, const KParams &p, int j,
                                         const S (&cin)[2 * K], S (&cout)[2 * K],
                                         Issued &iss)
{
    using C = CfgM<K, MODE>;
    constexpr int NSS = C::NSS, NSP = C::NSP, NSB = C::NSB;
    const int lane = s.lane;
    // MODE 6 waits for its phase slot just before the phase point: the slot
    // was refilled only after the previous row pair's first barrier (it
    // carried that row pair's second exchange), and a wait at the start of
    // the row pair cost 4 %.  A wait that gives up is combined over the CTA
    // at the second exchange's barrier.
    constexpr bool LATE_P = MODE == 6;
    bool ok = mbar_wait(&r.bar_s[r.pos_s], r.par_s, WAIT_LIMIT_NS) &&
              (LATE_P || mbar_wait(&r.bar_p[r.pos_p], r.par_p, WAIT_LIMIT_NS));
    if constexpr (MODE == 4)   // row pair j - 2's b rows, first read now
        ok = ok && (j < 2 || wait_b<NSB>(r, j - 2, WAIT_LIMIT_NS));
    ok = __all_sync(FULL, ok);
    // a bounded wait gave up: set the error bit, drain this warp's copies
    auto give_up = [&]() {
        if (lane == 0) atomicOr(p.err, ERRBIT_WAIT_TIMEOUT);
        if constexpr (C::GST_BYTES > 0) cp_async_wait_all();
        // drain this warp's outstanding copies (bounded) before leaving
        for (int jj = j, ps = r.pos_s, ph = r.par_s; jj < iss.s; ++jj) {
            mbar_wait(&r.bar_s[ps], ph, WAIT_LIMIT_NS / 4);
            if (++ps == NSS) { ps = 0; ph ^= 1u; }
        }
        for (int jj = j, ps = r.pos_p, ph = r.par_p; jj < iss.p; ++jj) {
            mbar_wait(&r.bar_p[ps], ph, WAIT_LIMIT_NS / 4);
            if (++ps == NSP) { ps = 0; ph ^= 1u; }
        }
        if constexpr (MODE == 4) {
            for (int jj = j < 2 ? 0 : j - 2; jj < iss.b; ++jj) wait_b<NSB>(r, jj, WAIT_LIMIT_NS / 4);
        }
        return false;
    };
    // MODE 6: the CTA's warps meet at barriers, so they give up together, at
    // the barrier of the row pair's first Z exchange (state wait) or second
    // (phase wait); until then a warp whose wait gave up computes on stale
    // slot contents, which is harmless since nothing of it is stored
    if (MODE != 6 && !ok) return give_up();
    const unsigned char *sj = r.ring_s + r.pos_s * C::SSLOT;
    // rows 0 and 1 of a state slot's planes (re, im) -- and (re, im) of the
    // costate in planes 2 and 3 for the backward adjoint steps
    auto load_rows = [&](Frag &a, Frag &b, int plane0) {
        a.re = lds4(sj, plane0, 0, lane);
        a.im = lds4(sj, plane0 + 1, 0, lane);
        b.re = lds4(sj, plane0, 1, lane);
        b.im = lds4(sj, plane0 + 1, 1, lane);
    };
    auto store_rows = [&](const Frag &o0, const Frag &o1, float *out_re, float *out_im, int yo) {
        float *rr = out_re + (int64_t)yo * p.pitch + s.xg;
        float *mm = out_im + (int64_t)yo * p.pitch + s.xg;
        if (INTERIOR || yo < p.ny) {
            *reinterpret_cast<float4 *>(rr) = o0.re;
            *reinterpret_cast<float4 *>(mm) = o0.im;
        }
        if (INTERIOR || yo + 1 < p.ny) {
            *reinterpret_cast<float4 *>(rr + p.pitch) = o1.re;
            *reinterpret_cast<float4 *>(mm + p.pitch) = o1.im;
        }
    };
    S a, b;
    if constexpr (MODE == 5 || MODE == 6) {
        load_rows(a.a, b.a, 0);
        load_rows(a.b, b.b, 2);
    } else {
        load_rows(a, b, 0);
    }
    // MODE 6: a 3-D step is Ze Zo [the 2-D step] Zo Ze (Z factors commute
    // with X and Y factors): the rows entering the pipeline take Ze, Zo, the
    // rows leaving it take Zo, Ze.  The exchanges go through this row pair's
    // state slot and then its phase slot (see z_odd).
    constexpr int WSTRIDE = C::WARP_SMEM / 16;
    if constexpr (MODE == 6) {
        z_even<C::PACKED>(a, b, s, p);
        float4 *xs = reinterpret_cast<float4 *>(r.ring_s + r.pos_s * C::SSLOT);
        // past this barrier every warp has read the previous row pair's
        // second exchange, in its phase slot: refill that slot with row pair
        // j - 1 + NSP.  (Both 3-D refills are issued right after the barrier
        // that frees their slot; issued after the exchange's updates and at
        // the end of the row pair, they measured 5 % slower.)
        if (z_odd<C::WPC, WSTRIDE>(a, b, s, p, xs, !ok, [&]() {
                const int jq = j - 1 + NSP;
                if (j >= 1 && jq < s.n_iter) {
                    if (lane == 0) {
                        fence_proxy_async();
                        issue_phase<K, phase_planes(MODE), true, true>(
                            r, s, r.pos_p == 0 ? NSP - 1 : r.pos_p - 1, jq);
                    }
                    iss.p += 1;
                }
            }))
            return give_up();
    }
    const int yin = s.Ys + 2 * j;
    bool okp = true;
    if constexpr (LATE_P)
        okp = __all_sync(FULL, mbar_wait(&r.bar_p[r.pos_p], r.par_p, WAIT_LIMIT_NS));
    S O0, O1;
    pipeline_step<K, INTERIOR, MODE>(cin, cout, a, b, yin, j, r.ring_p, r.pos_p, r.ring_b,
                                     r.cnt_b, s.c, p, lane, s.own, O0, O1);
    if constexpr (MODE == 6) {
        float4 *xp = reinterpret_cast<float4 *>(r.ring_p + r.pos_p * C::PSLOT);
        // past this barrier every warp has read this row pair's first
        // exchange, in its state slot: refill that slot with row pair j + NSS
        if (z_odd<C::WPC, WSTRIDE>(O0, O1, s, p, xp, !okp, [&]() {
                const int js = j + NSS;
                if (js < s.n_iter) {
                    if (lane == 0) {
                        fence_proxy_async();
                        issue_state<C::SSLOT, true>(r, s, r.pos_s, js);
                    }
                    iss.s += 1;
                }
            }))
            return give_up();
        z_even<C::PACKED>(O0, O1, s, p);
    }
    const int yo = yin - 2 * K;
    if (s.store_lane && yo >= s.Y0 && yo < s.Y1) {
        if constexpr (MODE == 6) {
            if (s.store_a) store_rows(O0.a, O1.a, p.out_re, p.out_im, yo);
            if (s.store_b) store_rows(O0.b, O1.b, p.out2_re, p.out2_im, yo);
        } else if constexpr (MODE == 5) {
            store_rows(O0.a, O1.a, p.out_re, p.out_im, yo);
            store_rows(O0.b, O1.b, p.out2_re, p.out2_im, yo);
        } else {
            store_rows(O0, O1, p.out_re, p.out_im, yo);
        }
    }
    // state slot j and the oldest phase slot read here (j - K + 1, or j - K
    // without PSHIFT) are no longer read: refill them with row pairs j + NSS
    // and that slot's pair + NSP (the same ring positions; MODE 6 refilled
    // its state slot at the second exchange and refills its phase slot at
    // the next row pair's first); MODE 4 also refills b slot j-3 with row
    // pair j - 3 + NSB
    __syncwarp();
    constexpr int PBACK = C::PSHIFT ? K - 1 : K;
    const int js = j + NSS, jp = j - PBACK + NSP, jb = j - 3 + NSB;
    const bool more_s = MODE != 6 && js < s.n_iter;
    const bool more_p = MODE != 6 && j >= PBACK && jp < s.n_iter;
    const bool more_b = MODE == 4 && j >= 3 && jb < s.n_iter;
    if (lane == 0 && (more_s || more_p || more_b)) {
        fence_proxy_async();
        if (more_s) issue_state<C::SSLOT, MODE == 6>(r, s, r.pos_s, js);
        if (more_p)
            issue_phase<K, phase_planes(MODE), MODE == 6, C::PSHIFT>(
                r, s, r.pos_p - PBACK < 0 ? r.pos_p - PBACK + NSP : r.pos_p - PBACK, jp);
        if constexpr (MODE == 4) {
            if (more_b) issue_b<NSB>(r, s, jb);   // the slot row pair j - 3 leaves
        }
    }
    iss.s += more_s;
    iss.p += more_p;
    iss.b += more_b;
    if (++r.pos_s == NSS) { r.pos_s = 0; r.par_s ^= 1u; }
    if (++r.pos_p == NSP) { r.pos_p = 0; r.par_p ^= 1u; }
    return true;
}

// Stream the row pairs [q0, q1) of strip sx of one grid through the K-step
// pipeline: rows [2 q0, 2 q1) are written to (p.out_re, p.out_im).  Returns
// false if a bounded wait gave up.
template <int K, int MODE>
__device__ __forceinline__ bool run_segment(WarpRings &r, const CUtensorMap *tm_state,
                                            const CUtensorMap *tm_phase, const CUtensorMap *tm_b,
                                            const KParams &p, int sx,
                                            int q0, int q1, int lane, const Slab3 &sl = Slab3())
{
    using C = CfgM<K, MODE>;
    using S = StateT<MODE>;
    constexpr int NSS = C::NSS, NSP = C::NSP, NSB = C::NSB, HALO = C::HALO, VALID = C::VALID;
    static_assert(NSB <= NSP, "the prologue issues the b ring inside the phase ring's loop");
    Seg s;
    s.tm_state = tm_state;
    s.tm_phase = tm_phase;
    s.tm_b = tm_b;
    s.ytma = sl.ytma;
    s.yslab = p.ny;
    s.z = sl.z;
    s.w = sl.w;
    s.store_a = sl.store_a;
    s.store_b = sl.store_b;
    s.lane = lane;
    s.XL = sx * VALID - HALO;            // first loaded column (multiple of 4)
    s.xg = s.XL + 4 * lane;              // this lane's first column
    s.Y0 = 2 * q0;                       // output rows [Y0, Y1)
    s.Y1 = 2 * q1;
    s.Ys = s.Y0 - 2 * K;                 // first loaded row
    s.n_iter = (s.Y1 - s.Y0) / 2 + 2 * K;   // row pairs loaded

    // pair (x, x+1) is rotated iff both sites are on the grid
    const int xg = s.xg;
    auto xok = [&](int x) { return x >= 0 && x + 1 < p.nx; };
    const bool e0 = xok(xg), e1 = xok(xg + 2), o0 = xok(xg + 1), oR = xok(xg + 3),
               oL = xok(xg - 1);
    s.c.E1 = {e0 ? p.t1 : 0.f, e0 ? p.s1 : 0.f, e1 ? p.t1 : 0.f, e1 ? p.s1 : 0.f};
    s.c.E2 = {e0 ? p.t2 : 0.f, e0 ? p.s2 : 0.f, e1 ? p.t2 : 0.f, e1 ? p.s2 : 0.f};
    s.c.O = {o0 ? p.t1 : 0.f, o0 ? p.s1 : 0.f, oR ? p.g1 : 0.f,
             oR ? p.s1 : 0.f, oL ? p.g1 : 0.f, oL ? p.s1 : 0.f};
    if constexpr (MODE == 4) {
        s.c.Ob = {o0 ? p.tb : 0.f, o0 ? p.sb : 0.f, oR ? p.gb : 0.f,
                  oR ? p.sb : 0.f, oL ? p.gb : 0.f, oL ? p.sb : 0.f};
        s.c.Eab = {e0 ? p.tab : 0.f, e0 ? p.sab : 0.f, e1 ? p.tab : 0.f, e1 ? p.sab : 0.f};
    }
    s.store_lane = lane >= HALO / 4 && lane < 32 - HALO / 4 && xg < p.nx;
    s.own = {s.Y0, s.Y1, xg, s.store_lane, r.sums, r.gst};

    const int n_pro_s = s.n_iter < NSS ? s.n_iter : NSS;
    const int n_pro_p = s.n_iter < NSP ? s.n_iter : NSP;
    const int n_pro_b = s.n_iter < NSB ? s.n_iter : NSB;
    if (lane == 0) {
        fence_proxy_async();
        for (int j = 0; j < n_pro_p; ++j) {
            if (j < n_pro_s) issue_state<C::SSLOT, MODE == 6>(r, s, (r.pos_s + j) % NSS, j);
            issue_phase<K, phase_planes(MODE), MODE == 6, C::PSHIFT>(r, s, (r.pos_p + j) % NSP, j);
            if constexpr (MODE == 4) {
                if (j < n_pro_b) issue_b<NSB>(r, s, j);
            }
        }
    }
    Issued iss = {n_pro_s, n_pro_p, n_pro_b};

    // Carried rows: interior row pairs go in twos; for deep pipelines the
    // first reads set A and writes set B and the second goes back into A, so
    // no row is copied between iterations (at the price of registers, which
    // shallow pipelines keep for occupancy); edge row pairs update A in place.
    // MODE 5 keeps one set and takes one row pair per trip.  Its running sums
    // of G's terms start at zero (the sums of rows this warp owns start
    // inside the segment; the rows of its first iterations are not this
    // warp's and are never stored)
    S cA[2 * K], cB[2 * K];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) cA[i] = zero_state<S>();
    if constexpr (C::SUMS_BYTES > 0) {
#pragma unroll
        for (int i = 0; i < 2 * (K - 1); ++i) {
            r.sums[i * 64] = make_float4(0.f, 0.f, 0.f, 0.f);
            r.sums[i * 64 + 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    auto interior = [&](int j) {
        const int yin = s.Ys + 2 * j;
        return j >= K && yin - 2 * K >= 0 && yin + 1 < p.ny;
    };
    for (int j = 0; j < s.n_iter;) {
        if (C::ONE_PAIR) {
            if (interior(j)) {
                if (!row_pair<K, MODE, true>(r, s, p, j, cA, cA, iss)) return false;
            } else if (!row_pair<K, MODE, false>(r, s, p, j, cA, cA, iss)) {
                return false;
            }
            j += 1;
            continue;
        }
        if (j + 1 < s.n_iter && interior(j) && interior(j + 1)) {
            if (C::PINGPONG) {
                if (!row_pair<K, MODE, true>(r, s, p, j, cA, cB, iss)) return false;
                if (!row_pair<K, MODE, true>(r, s, p, j + 1, cB, cA, iss))
                    return false;
            } else {
                if (!row_pair<K, MODE, true>(r, s, p, j, cA, cA, iss)) return false;
                if (!row_pair<K, MODE, true>(r, s, p, j + 1, cA, cA, iss))
                    return false;
            }
            j += 2;
        } else {
            if (!row_pair<K, MODE, false>(r, s, p, j, cA, cA, iss)) return false;
            j += 1;
        }
    }
    if constexpr (MODE == 4) {
        // the last two row pairs' b rows were never needed: let their copies
        // land before the slots are reused, then number the next segment's on
        bool ok = true;
        for (int jj = s.n_iter - 2 < 0 ? 0 : s.n_iter - 2; jj < s.n_iter; ++jj)
            ok = wait_b<NSB>(r, jj, WAIT_LIMIT_NS) && ok;
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) atomicOr(p.err, ERRBIT_WAIT_TIMEOUT);
            return false;
        }
        r.cnt_b += s.n_iter;
    }
    if constexpr (C::GST_BYTES > 0) cp_async_wait_all();
    // MODE 6: the other warps may still read this segment's last exchange in
    // this warp's phase slot, which the next segment's first copies refill
    if constexpr (MODE == 6) __syncthreads();
    __syncwarp();
    return true;
}

// One grid; the (strip, row-pair) units are split into equal contiguous
// ranges, one per warp of a persistent launch.
template <int K, int MODE>
__global__ void __launch_bounds__(Cfg<K>::WPC * 32, min_blocks(K, MODE))
fused_kernel(const __grid_constant__ CUtensorMap tm_state,
             const __grid_constant__ CUtensorMap tm_phase,
             const __grid_constant__ CUtensorMap tm_b,
             const KParams p)
{
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * Cfg<K>::WPC + warp;
    if (gw >= p.total_warps) return;
    WarpRings r = carve_rings<K, phase_planes(MODE), MODE == 4, state_planes(MODE), MODE>(smem_raw, warp, lane);
    if (p.strip_warps > 0) {
        // strip-aligned split: warp (sx, i) takes row range i of strip sx, so
        // warps of neighbouring strips walk the same rows at the same time and
        // the columns their halos share are read from L2
        const int sx = gw / p.strip_warps, i = gw - sx * p.strip_warps;
        const int q0 = (int)((int64_t)i * p.n_pairs / p.strip_warps);
        const int q1 = (int)((int64_t)(i + 1) * p.n_pairs / p.strip_warps);
        if (q1 > q0) run_segment<K, MODE>(r, &tm_state, &tm_phase, &tm_b, p, sx, q0, q1, lane);
        return;
    }
    const int64_t u_begin = (int64_t)gw * p.units / p.total_warps;
    const int64_t u_end = (int64_t)(gw + 1) * p.units / p.total_warps;
    for (int64_t u = u_begin; u < u_end;) {
        const int sx = (int)(u / p.n_pairs);
        const int q0 = (int)(u - (int64_t)sx * p.n_pairs);
        const int64_t q1_want = (int64_t)q0 + (u_end - u);
        const int q1 = (int)(q1_want < p.n_pairs ? q1_want : (int64_t)p.n_pairs);
        u += q1 - q0;
        if (!run_segment<K, MODE>(r, &tm_state, &tm_phase, &tm_b, p, sx, q0, q1, lane)) return;
    }
}

// Three-dimensional steps, one step per launch, one HBM round trip.  A CTA
// owns a block of 2 TS_FUSED3D_WARPS consecutive slabs of one strip and one
// range of rows; warp w runs the depth-1 pipeline on slabs z and z + 1,
// z = zb * VZ - 2 + 2 w (even), and all warps walk the same rows together.
// The rows entering the pipeline take Ze (inside the warp) and Zo (traded
// with the neighbouring warps), the rows leaving it Zo and Ze.  The two
// slabs at either end of the block lack partners outside it: they are a
// halo, computed but not stored (with the block's first slab even, two per
// side are enough for the four Z sweeps of a step), so a CTA stores
// VZ = 2 NW - 4 slabs.  Slabs outside the grid are zero rows from TMA and
// pair with nothing.  Units (z-block fastest, then strip, then row range) go
// round robin over the resident CTAs, so the CTAs of neighbouring z-blocks
// run together and read their shared halo slabs through L2.
template <int K>
__global__ void __launch_bounds__(TS_FUSED3D_WARPS * 32, 1)
fused3d_kernel(const __grid_constant__ CUtensorMap tm_state,
               const __grid_constant__ CUtensorMap tm_phase, const KParams p)
{
    static_assert(K == 1, "3-D steps run one step per launch");
    using C = CfgM<K, 6>;
    constexpr int NW = C::WPC, VZ = 2 * NW - 4;
    static_assert(VZ > 0 && VZ % 2 == 0, "the block's first slab must stay even");
    static_assert(NW <= 16, "the host's row-coordinate guard assumes at most 16 warps");
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRings r = carve_rings<K, phase_planes(6), false, state_planes(6), 6>(smem_raw, warp, lane);
    const int64_t slab = (int64_t)p.ny * p.pitch;
    for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) {
        const int zb = (int)(u % p.n_zblocks);
        const int64_t t = u / p.n_zblocks;
        const int sx = (int)(t % p.n_strips), rr = (int)(t / p.n_strips);
        const int q0 = (int)((int64_t)rr * p.n_pairs / p.n_ranges);
        const int q1 = (int)((int64_t)(rr + 1) * p.n_pairs / p.n_ranges);
        if (q1 <= q0) continue;                  // the same for every warp of the CTA
        Slab3 sl;
        sl.z = zb * VZ - 2 + 2 * warp;
        sl.w = warp;
        sl.ytma = sl.z * p.ny;
        const bool inner = warp >= 1 && warp < NW - 1;
        sl.store_a = inner && sl.z >= 0 && sl.z < p.nz;
        sl.store_b = inner && sl.z + 1 >= 0 && sl.z + 1 < p.nz;
        KParams pw = p;
        if (sl.store_a) {
            pw.out_re = p.out_re + sl.z * slab;
            pw.out_im = p.out_im + sl.z * slab;
        }
        if (sl.store_b) {
            pw.out2_re = p.out_re + (sl.z + 1) * slab;
            pw.out2_im = p.out_im + (sl.z + 1) * slab;
        }
        if (!run_segment<K, 6>(r, &tm_state, &tm_phase, nullptr, pw, sx, q0, q1, lane, sl))
            return;
    }
}

// Many grids in one persistent launch (the serving path), under one of two
// plans (fused_multi_plan picks one per launch):
//  - aligned: grid i owns warps [begin, begin + strips * strip_warps),
//    strip_warps per strip on the same row ranges in every strip (as in the
//    single-grid kernel's aligned split), so warps of neighbouring strips
//    walk the same rows together and read their shared halo columns from L2;
//  - even: the row pairs of all grids, concatenated in table order (grid i's
//    from unit `begin` on), are split into equal contiguous ranges, one per
//    warp -- balanced for any mix, but without that alignment.
// A grid's tensor maps live in its descriptor in global memory, written once
// when the grid was set up.
__device__ __forceinline__ void multi_params(KParams &p, const GridDesc *d, int cur, int *err)
{
    p.nx = d->nx;
    p.ny = d->ny;
    p.pitch = d->pitch;
    p.out_re = d->re[cur ^ 1];
    p.out_im = d->im[cur ^ 1];
    p.t1 = d->t1;
    p.s1 = d->s1;
    p.g1 = d->g1;
    p.t2 = d->t2;
    p.s2 = d->s2;
    p.err = err;
    p.n_pairs = (p.ny + 1) / 2;
    p.strip_warps = 0;
}

template <int K>
__global__ void __launch_bounds__(Cfg<K>::WPC * 32, multi_min_blocks(K))
fused_multi_kernel(const EpochEntry *__restrict__ tab, int n_grids, int64_t total_units,
                   int total_warps, int aligned, int flip, int *err)
{
    using C = Cfg<K>;
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * C::WPC + warp;
    if (gw >= total_warps) return;
    WarpRings r = carve_rings<K>(smem_raw, warp, lane);
    if (aligned) {
        // the grid of warp gw: the last entry whose first warp is <= gw
        int lo = 0, hi = n_grids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab[mid].begin <= gw)
                lo = mid;
            else
                hi = mid - 1;
        }
        const EpochEntry e = tab[lo];
        const GridDesc *d = e.desc;
        const int cur = e.cur0 ^ flip;
        if (lane == 0) {
            tensormap_acquire(&d->tm_state[cur]);
            tensormap_acquire(&d->tm_phase);
        }
        __syncwarp();
        KParams p;
        multi_params(p, d, cur, err);
        const int w = e.strip_warps, l = gw - (int)e.begin;
        const int sx = l / w, i = l - sx * w;
        const int q0 = (int)((int64_t)i * p.n_pairs / w);
        const int q1 = (int)((int64_t)(i + 1) * p.n_pairs / w);
        if (q1 > q0)
            run_segment<K, 0>(r, &d->tm_state[cur], &d->tm_phase, nullptr, p, sx, q0, q1, lane);
        return;
    }
    const int64_t u_begin = (int64_t)gw * total_units / total_warps;
    const int64_t u_end = (int64_t)(gw + 1) * total_units / total_warps;
    int gi = 0, fenced = -1;
    for (int64_t u = u_begin; u < u_end;) {
        while (gi + 1 < n_grids && tab[gi + 1].begin <= u) ++gi;
        const EpochEntry e = tab[gi];
        const GridDesc *d = e.desc;
        const int cur = e.cur0 ^ flip;
        if (fenced != gi) {
            if (lane == 0) {
                tensormap_acquire(&d->tm_state[cur]);
                tensormap_acquire(&d->tm_phase);
            }
            __syncwarp();
            fenced = gi;
        }
        KParams p;
        multi_params(p, d, cur, err);
        const int64_t local = u - e.begin;
        const int64_t g_units = (gi + 1 < n_grids ? tab[gi + 1].begin : total_units) - e.begin;
        const int sx = (int)(local / p.n_pairs);
        const int q0 = (int)(local - (int64_t)sx * p.n_pairs);
        int64_t q1_want = (int64_t)q0 + (u_end - u);
        const int64_t left_in_grid = g_units - local;
        if (q1_want > q0 + left_in_grid) q1_want = q0 + left_in_grid;
        const int q1 = (int)(q1_want < p.n_pairs ? q1_want : (int64_t)p.n_pairs);
        u += q1 - q0;
        if (!run_segment<K, 0>(r, &d->tm_state[cur], &d->tm_phase, nullptr, p, sx, q0, q1, lane)) return;
    }
}

// Resident blocks per SM and SM count of a kernel at its dynamic shared
// memory size, set up once per kernel (the first caller's function-local
// static initialisation, which C++ runs exactly once even when threads race).
struct Occupancy {
    cudaError_t err;
    int blocks_per_sm, num_sms;
};

// Fewest row pairs a warp takes.  Each warp runs a chain of dependent
// iterations, and each of its segments first fills a pipeline of 2K row
// pairs.  On small grids the chains set the launch time, so many warps with
// short ranges win (down to TS_FUSED_MIN_PAIRS).  Once a grid has enough
// work for TS_FUSED_FILL_WARPS_PER_SM warps per SM at that length, more
// warps only add fills, so the floor grows with the work (up to
// TS_FUSED_MAX_MIN_PAIRS).
inline int64_t min_pairs_per_warp(int64_t units, int num_sms)
{
    const int64_t by_work = units / ((int64_t)TS_FUSED_FILL_WARPS_PER_SM * num_sms);
    return std::min<int64_t>(TS_FUSED_MAX_MIN_PAIRS, std::max<int64_t>(TS_FUSED_MIN_PAIRS, by_work));
}

template <typename F>
Occupancy occupancy_of(F kernel, int threads, int smem);

// One 3-D step over an nx x ny x nz FP32 grid (a.ny = ny rows per slab).
cudaError_t launch3_k(const FusedLaunch &a, int nz, cudaStream_t st)
{
    using C = CfgM<1, 6>;
    constexpr int NW = C::WPC, VZ = 2 * NW - 4;
    static const Occupancy occ = occupancy_of(fused3d_kernel<1>, NW * 32, C::SMEM);
    if (occ.err != cudaSuccess) return occ.err;
    KParams p = {};
    p.out_re = a.out_re;
    p.out_im = a.out_im;
    p.nx = a.nx;
    p.ny = a.ny;
    p.nz = nz;
    p.pitch = a.pitch;
    p.n_strips = (a.nx + C::VALID - 1) / C::VALID;
    p.n_pairs = (a.ny + 1) / 2;
    p.n_zblocks = (nz + VZ - 1) / VZ;
    // Row ranges per slab: the resident CTAs take the units round robin, so
    // the launch lasts ceil(units / ctas) units while the work is units; a
    // range of q row pairs also loads 2 more for its pipeline fill.  Take the
    // count that keeps the most of the time useful, units / (ceil(units /
    // ctas) ctas) * q / (q + 2), over ranges of at least 8 row pairs.
    const int64_t ctas = (int64_t)occ.num_sms * occ.blocks_per_sm;
    const int64_t blocks = (int64_t)p.n_strips * p.n_zblocks;
    int64_t ranges = 1;
    double best = -1.0;
    for (int64_t r = 1; r <= std::max<int64_t>(1, p.n_pairs / 8); ++r) {
        const int64_t units = blocks * r, waves = (units + ctas - 1) / ctas;
        const double q = (double)p.n_pairs / (double)r;
        const double eff = (double)units / (double)(waves * ctas) * q / (q + 2.0);
        if (eff > best) {
            best = eff;
            ranges = r;
        }
    }
    p.n_ranges = (int)ranges;
    p.units = blocks * ranges;
    p.strip_warps = 0;
    p.t1 = a.t1;
    p.s1 = a.s1;
    p.g1 = a.g1;
    p.t2 = a.t2;
    p.s2 = a.s2;
    p.err = a.err;
    const int grid = (int)std::min<int64_t>(p.units, ctas);
    fused3d_kernel<1><<<grid, NW * 32, C::SMEM, st>>>(*a.tm_state, *a.tm_phase, p);
    count_launches(1);
    return cudaGetLastError();
}

template <typename F>
Occupancy occupancy_of(F kernel, int threads, int smem)
{
    Occupancy o = {cudaSuccess, 0, 0};
    o.err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (o.err != cudaSuccess) return o;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&o.num_sms, cudaDevAttrMultiProcessorCount, dev);
    o.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.blocks_per_sm, kernel, threads, smem);
    if (o.err == cudaSuccess && o.blocks_per_sm < 1) o.err = cudaErrorInvalidConfiguration;
    return o;
}

template <int K, int MODE>
cudaError_t launch_k(const FusedLaunch &a, cudaStream_t st)
{
    using C = CfgM<K, MODE>;
    static const Occupancy occ = occupancy_of(fused_kernel<K, MODE>, C::WPC * 32, C::SMEM);
    if (occ.err != cudaSuccess) return occ.err;
    const int blocks_per_sm = occ.blocks_per_sm, num_sms = occ.num_sms;
    KParams p;
    p.out_re = a.out_re;
    p.out_im = a.out_im;
    p.nx = a.nx;
    p.ny = a.ny;
    p.pitch = a.pitch;
    p.n_strips = (a.nx + C::VALID - 1) / C::VALID;
    p.n_pairs = (a.ny + 1) / 2;
    p.units = (int64_t)p.n_strips * p.n_pairs;
    // at most the resident warps, each with at least min_pairs_per_warp row pairs
    const int64_t mp = min_pairs_per_warp(p.units, num_sms);
    int64_t want = (p.units + mp - 1) / mp;
    int64_t cap = (int64_t)num_sms * blocks_per_sm * C::WPC;
    p.total_warps = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    p.strip_warps = 0;
    if (TS_FUSED_ALIGNED && p.n_strips <= cap) {
        int64_t w = cap / p.n_strips;
        const int64_t rows_cap = (p.n_pairs + mp - 1) / mp;
        if (w > rows_cap) w = rows_cap;
        if (w < 1) w = 1;
        p.strip_warps = (int)w;
        p.total_warps = (int)(w * p.n_strips);
    }
    p.t1 = a.t1;
    p.s1 = a.s1;
    p.g1 = a.g1;
    p.t2 = a.t2;
    p.s2 = a.s2;
    p.err = a.err;
    p.out2_re = a.out2_re;
    p.out2_im = a.out2_im;
    p.g_rh = a.g_rh;
    p.g_rl = a.g_rl;
    p.g_ih = a.g_ih;
    p.g_il = a.g_il;
    for (int k = 0; k < FUSED_MAX_K; ++k) p.adt[k] = a.adt[k];
    p.tb = a.tb;
    p.sb = a.sb;
    p.gb = a.gb;
    p.tab = a.tab;
    p.sab = a.sab;
    const int blocks = (p.total_warps + C::WPC - 1) / C::WPC;
    fused_kernel<K, MODE><<<blocks, C::WPC * 32, C::SMEM, st>>>(
        *a.tm_state, *a.tm_phase, a.tm_b ? *a.tm_b : *a.tm_phase, p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused(int K, const FusedLaunch &a, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_k<1, 0>(a, st);
    case 2: return launch_k<2, 0>(a, st);
    case 3: return launch_k<3, 0>(a, st);
    case 4: return launch_k<4, 0>(a, st);
    case 5: return launch_k<5, 0>(a, st);
    case 6: return launch_k<6, 0>(a, st);
    case 7: return launch_k<7, 0>(a, st);
    case 8: return launch_k<8, 0>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int K>
const Occupancy &multi_occupancy()
{
    using C = Cfg<K>;
    static const Occupancy occ = occupancy_of(fused_multi_kernel<K>, C::WPC * 32, C::SMEM);
    return occ;
}

template <int K>
cudaError_t prepare_multi_k()
{
    return multi_occupancy<K>().err;
}

template <int K>
cudaError_t launch_multi_k(const EpochEntry *tab, int n_grids, const MultiPlan &plan, int flip,
                           int *err, cudaStream_t st)
{
    using C = Cfg<K>;
    const Occupancy &occ = multi_occupancy<K>();
    if (occ.err != cudaSuccess) return occ.err;
    const int blocks = (plan.warps + C::WPC - 1) / C::WPC;
    fused_multi_kernel<K><<<blocks, C::WPC * 32, C::SMEM, st>>>(
        tab, n_grids, plan.units, plan.warps, plan.aligned ? 1 : 0, flip, err);
    count_launches(1);
    return cudaGetLastError();
}

// Resident warps of the multi-grid kernel at depth K (-1 on an error) and the SM count.
template <int K>
int64_t multi_capacity(int &num_sms)
{
    const Occupancy &occ = multi_occupancy<K>();
    if (occ.err != cudaSuccess) return -1;
    num_sms = occ.num_sms;
    return (int64_t)occ.num_sms * occ.blocks_per_sm * Cfg<K>::WPC;
}

cudaError_t fused_multi_prepare(int K)
{
    switch (K) {
    case 1: return prepare_multi_k<1>();
    case 2: return prepare_multi_k<2>();
    case 3: return prepare_multi_k<3>();
    case 4: return prepare_multi_k<4>();
    case 5: return prepare_multi_k<5>();
    case 6: return prepare_multi_k<6>();
    case 7: return prepare_multi_k<7>();
    case 8: return prepare_multi_k<8>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_multi(int K, const EpochEntry *tab, int n_grids, const MultiPlan &plan,
                               int flip, int *err, cudaStream_t st)
{
    if (n_grids < 1 || plan.warps < 1 || plan.units < 1) return cudaSuccess;
    switch (K) {
    case 1: return launch_multi_k<1>(tab, n_grids, plan, flip, err, st);
    case 2: return launch_multi_k<2>(tab, n_grids, plan, flip, err, st);
    case 3: return launch_multi_k<3>(tab, n_grids, plan, flip, err, st);
    case 4: return launch_multi_k<4>(tab, n_grids, plan, flip, err, st);
    case 5: return launch_multi_k<5>(tab, n_grids, plan, flip, err, st);
    case 6: return launch_multi_k<6>(tab, n_grids, plan, flip, err, st);
    case 7: return launch_multi_k<7>(tab, n_grids, plan, flip, err, st);
    case 8: return launch_multi_k<8>(tab, n_grids, plan, flip, err, st);
    default: return cudaErrorInvalidValue;
    }
}

MultiPlan fused_multi_plan(int K, int n, const int *nx, const int *ny, EpochEntry *tab)
{
    MultiPlan plan = {0, 0, false};
    int64_t cap;
    int num_sms = 1;
    switch (K) {
    case 1: cap = multi_capacity<1>(num_sms); break;
    case 2: cap = multi_capacity<2>(num_sms); break;
    case 3: cap = multi_capacity<3>(num_sms); break;
    case 4: cap = multi_capacity<4>(num_sms); break;
    case 5: cap = multi_capacity<5>(num_sms); break;
    case 6: cap = multi_capacity<6>(num_sms); break;
    case 7: cap = multi_capacity<7>(num_sms); break;
    case 8: cap = multi_capacity<8>(num_sms); break;
    default: return plan;
    }
    if (cap < 1 || n < 1) return plan;
    const int halo = ((2 * K + 3) / 4) * 4, valid = FUSED_BOX_COLS - 2 * halo;
    std::vector<int64_t> strips((size_t)n), pairs((size_t)n), w((size_t)n, 1);
    int64_t units = 0, all_strips = 0;
    for (int i = 0; i < n; ++i) {
        strips[(size_t)i] = (nx[i] + valid - 1) / valid;
        pairs[(size_t)i] = (ny[i] + 1) / 2;
        units += strips[(size_t)i] * pairs[(size_t)i];
        all_strips += strips[(size_t)i];
    }
    // even split: at most the resident warps, each with at least
    // min_pairs_per_warp row pairs
    const int64_t mp = min_pairs_per_warp(units, num_sms);
    const int64_t lin_warps = std::min(cap, std::max<int64_t>(1, (units + mp - 1) / mp));
    const int64_t lin_span = (units + lin_warps - 1) / lin_warps;
    // aligned split: one warp per strip to start with, then more warps (on
    // every strip of a grid at once) to the grid with the most row pairs per
    // warp while they fit; it is taken when its longest warp is within 10 %
    // of the even split's
    int64_t al_warps = all_strips, al_span = 0;
    if (all_strips <= cap) {
        auto work = [&](int i) { return (pairs[(size_t)i] + w[(size_t)i] - 1) / w[(size_t)i]; };
        std::priority_queue<std::pair<int64_t, int>> heap;
        for (int i = 0; i < n; ++i) heap.push({work(i), i});
        while (!heap.empty()) {
            const int i = heap.top().second;
            if (al_warps + strips[(size_t)i] > cap || pairs[(size_t)i] / (w[(size_t)i] + 1) < mp)
                break;
            heap.pop();
            ++w[(size_t)i];
            al_warps += strips[(size_t)i];
            heap.push({work(i), i});
        }
        for (int i = 0; i < n; ++i) al_span = std::max(al_span, work(i));
    }
    plan.aligned = all_strips <= cap && al_span * 10 <= lin_span * 11;
    plan.units = units;
    int64_t begin = 0;
    for (int i = 0; i < n; ++i) {
        tab[i].begin = begin;
        tab[i].strip_warps = plan.aligned ? (int)w[(size_t)i] : 0;
        begin += plan.aligned ? strips[(size_t)i] * w[(size_t)i] : strips[(size_t)i] * pairs[(size_t)i];
    }
    plan.warps = (int)(plan.aligned ? al_warps : lin_warps);
    return plan;
}

cudaError_t launch_fused_drive(int K, const FusedLaunch &a, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_k<1, 3>(a, st);
    case 2: return launch_k<2, 3>(a, st);
    case 3: return launch_k<3, 3>(a, st);
    case 4: return launch_k<4, 3>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_u4(const FusedLaunch &a, cudaStream_t st) { return launch_k<5, 4>(a, st); }

cudaError_t launch_fused3d(const FusedLaunch &a, int nz, cudaStream_t st)
{
    return launch3_k(a, nz, st);
}

cudaError_t launch_fused_adjoint(int K, const FusedLaunch &a, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_k<1, 5>(a, st);
    case 2: return launch_k<2, 5>(a, st);
    case 3: return launch_k<3, 5>(a, st);
    case 4: return launch_k<4, 5>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

bool make_pair_tensor_map(CUtensorMap *tm, const void *base, int nx, int ny, int64_t pitch,
                          size_t plane_bytes, const char **why, int planes, int box_planes)
{
    // looked up once (thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
        cudaDriverEntryPointQueryResult qr;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &qr) != cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    if (box_planes == 0) box_planes = planes;
    if (box_planes < 1 || box_planes > 4 || planes < box_planes) {
        *why = "tensor map: boxes of 1 to 4 planes, no more than the map has";
        return false;
    }
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * 4), (cuuint64_t)plane_bytes};
    cuuint32_t box[3] = {FUSED_BOX_COLS, FUSED_BOX_ROWS, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    // (a driver call: the calling thread needs a current context)
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base),
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        thread_local char msg[96];
        snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled rejected the plane layout (CUresult %d)",
                 (int)r);
        *why = msg;
        return false;
    }
    return true;
}

}  // namespace ts
