// Internal interface between the C-ABI layer (api.cu) and the kernel files.
// Not installed; the public boundary is include/trotter.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

struct ts_grid;

namespace ts {

// Error bits written by kernels into the grid's device error word.
enum : int { ERRBIT_WAIT_TIMEOUT = 1, ERRBIT_BAD_CONFIG = 2 };

// Number of FP64 quantities the observables reduction produces per block.
constexpr int OBS_Q = 7;
constexpr int OBS_Q3 = 9;   // 3-D grids: the 7 quantities plus sum z p and sum z^2 p
constexpr int OBS_MAX_BLOCKS = 1024;

// --- conversions, tables, plain path (plain.cu) ---------------------------
// dense (nx*ny, src type) -> pitched plane of dst type
cudaError_t launch_convert_in(const void *src, bool src_f64, void *dst, bool dst_f64,
                              int nx, int ny, int64_t pitch, cudaStream_t st);
// pitched plane -> dense
cudaError_t launch_convert_out(const void *src, bool src_f64, void *dst, bool dst_f64,
                               int nx, int ny, int64_t pitch, cudaStream_t st);
// V (dense FP64) -> (gamma_V, s_V, V) pitched planes of the grid's type
cudaError_t launch_phase_table(const double *V, void *pg, void *ps, void *vplane, bool f64,
                               int nx, int ny, int64_t pitch, double dt, cudaStream_t st);
// one sweep along x (axis 0) or y (axis 1) of the given parity, in place;
// (g, s) versine coefficients, or with lift (FP64 only) (tan(theta/2), s)
cudaError_t launch_plain_sweep(void *re, void *im, bool f64, int nx, int ny, int64_t pitch,
                               int axis, int parity, double g, double s, cudaStream_t st,
                               bool lift = false);
// the diagonal phase exp(-i V dt) from the stored table, in place
cudaError_t launch_plain_phase(void *re, void *im, const void *pg, const void *ps, bool f64,
                               int nx, int ny, int64_t pitch, cudaStream_t st);
// psi <- psi exp(-i adt V1) (the drive term of a time-dependent potential),
// in place; V1 is a pitched plane of the grid's dtype.
cudaError_t launch_plain_drive(void *re, void *im, const void *v1, bool f64, int nx, int ny,
                               int64_t pitch, double adt, cudaStream_t st);

// --- failure path of the bounded waits (selftest.cu) ----------------------
// One warp waits on an mbarrier that nothing completes; after limit_ns the
// wait gives up and ERRBIT_WAIT_TIMEOUT is or-ed into *err, as in the fused
// kernels.
cudaError_t launch_wait_timeout_check(int *err, uint64_t limit_ns, cudaStream_t st);

// --- three-dimensional lattices (lattice3d.cu) ----------------------------
// A 3-D grid of nx x ny x nz sites keeps slab z (rows z*ny .. z*ny + ny - 1
// of every plane) right after slab z - 1, so the 2-D kernels see a grid of
// ny*nz rows.  X sweeps, the phase and the tables need nothing else.
// One Y sweep inside every slab (pairs (y, y+1), y of the given parity
// counted from the slab's first row), in place.
cudaError_t launch_plain_sweep_y3(void *re, void *im, bool f64, int nx, int ny, int nz,
                                  int64_t pitch, int parity, double g, double s,
                                  cudaStream_t st, bool lift = false);
// One Z sweep: pairs of slabs (z, z+1), z of the given parity, in place.
cudaError_t launch_plain_sweep_z(void *re, void *im, bool f64, int nx, int ny, int nz,
                                 int64_t pitch, int parity, double g, double s, cudaStream_t st,
                                 bool lift = false);

// --- observables (reduce.cu) ----------------------------------------------
// partials: OBS_MAX_BLOCKS * OBS_Q doubles; result: OBS_Q doubles.
// norm_only computes only sum |psi|^2 (result[0]).
cudaError_t launch_observe(const void *re, const void *im, const void *vplane, bool f64,
                           int nx, int ny, int64_t pitch, double J, bool norm_only,
                           double *partials, double *result, cudaStream_t st);

// The same for a 3-D grid: OBS_Q3 quantities (sum p, sum x p, sum y p,
// sum x^2 p, sum y^2 p, kinetic, potential, sum z p, sum z^2 p), bonds along
// x, y (inside slabs) and z; partials hold OBS_MAX_BLOCKS * OBS_Q3 doubles.
cudaError_t launch_observe3(const void *re, const void *im, const void *vplane, bool f64,
                            int nx, int ny, int nz, int64_t pitch, double J, double *partials,
                            double *result, cudaStream_t st);

// <phi|psi> = sum conj(phi) psi over two FP32 pitched states: result[0] real,
// result[1] imaginary part (exact products, double-float then FP64 sums).
cudaError_t launch_inner(const float *phi_re, const float *phi_im, const float *psi_re,
                         const float *psi_im, int nx, int ny, int64_t pitch, double *partials,
                         double *result, cudaStream_t st);

// --- fused temporally blocked path (fused.cu) -----------------------------
struct FusedLaunch {
    const CUtensorMap *tm_state;   // (re, im) planes of the input pair, 3-D map
    const CUtensorMap *tm_phase;   // (gamma_V, s_V) planes, 3-D map
    const CUtensorMap *tm_b = nullptr;   // launch_fused_u4: the b substep's table
    float *out_re, *out_im;
    int nx, ny;
    int64_t pitch;
    // rotation at theta: lifting form (t1 = tan(theta/2), s1 = sin theta) and
    // versine form (g1 = 1 - cos theta, s1); at 2 theta: lifting (t2, s2)
    float t1, s1, g1, t2, s2;
    int *err;
    // launch_fused_adjoint: the costate's output planes (out_re, out_im take
    // psi) and G as double-float planes
    float *out2_re = nullptr, *out2_im = nullptr;
    float *g_rh = nullptr, *g_rl = nullptr, *g_ih = nullptr, *g_il = nullptr;
    // time-dependent potential (launch_fused_drive only): a_n dt of step k
    float adt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // the fused fourth-order step (launch_fused_u4): t1..s2 above are the
    // a substep's; the b substep's lifting (tb, sb) and versine (gb) forms,
    // and the merged angle a + b in lifting form (tab, sab)
    float tb = 0, sb = 0, gb = 0, tab = 0, sab = 0;
};
constexpr int FUSED_MAX_K = 8;
static_assert(sizeof(FusedLaunch::adt) / sizeof(float) == FUSED_MAX_K, "one a_n dt per step");
constexpr int FUSED_BOX_COLS = 128;   // columns a warp strip loads (box width)
constexpr int FUSED_BOX_ROWS = 2;     // rows per pipeline slot (box height)
cudaError_t launch_fused(int K, const FusedLaunch &a, cudaStream_t st);
// K (1..FUSED_ADJ_MAX_K) backward adjoint steps U^dagger (pass the
// coefficients at -theta) on two states at once: tm_state maps four planes
// (psi re, im, lambda re, im), psi goes to (out_re, out_im) and lambda to
// (out2_re, out2_im).  At each step's phase point G += conj(lambda~) m, with
// lambda~ = B^dagger lambda_s and m = B^dagger psi_s.
constexpr int FUSED_ADJ_MAX_K = 4;
cudaError_t launch_fused_adjoint(int K, const FusedLaunch &a, cudaStream_t st);
// K (1..4) steps with the time-dependent potential V0 + a_n V1: tm_phase
// maps three planes (gamma_V, s_V, V1) and adt[k] = a_n dt of step k.
constexpr int FUSED_DRIVE_MAX_K = 4;
cudaError_t launch_fused_drive(int K, const FusedLaunch &a, cudaStream_t st);
// One fourth-order step U4 = a a b a a in one launch (five substeps, depth
// 5): tm_phase maps the a substep's table, tm_b the b substep's.
cudaError_t launch_fused_u4(const FusedLaunch &a, cudaStream_t st);
// One 3-D step Xe Xo Ye Yo Ze Zo P Zo Ze Yo Ye Xo Xe over an nx x ny x nz
// FP32 grid in one HBM round trip: a.ny is the rows of one slab, tm_state
// and tm_phase map all ny * nz rows (slab after slab), out_re, out_im take
// the result.  Needs (nz + 32) * ny < 2^31.
cudaError_t launch_fused3d(const FusedLaunch &a, int nz, cudaStream_t st);

// Device-resident description of one FP32 grid for the multi-grid launch
// (written once per grid set-up; read by the kernel with generic loads, its
// tensor maps by TMA).
struct GridDesc {
    CUtensorMap tm_state[2];   // (re, im) of pair 0 / pair 1
    CUtensorMap tm_phase;      // (gamma_V, s_V)
    float *re[2], *im[2];      // planes of pair 0 / pair 1
    int nx, ny;
    int64_t pitch;
    float t1, s1, g1, t2, s2;  // rotation coefficients (see FusedLaunch)
};

// One grid of an epoch: its descriptor, where its work starts in the
// launch's plan (its first warp in an aligned plan, its first row-pair unit
// in an even one), its warps per strip (aligned plans), and which pair holds
// its state at flip = 0.
struct EpochEntry {
    const GridDesc *desc;
    int64_t begin;
    int cur0;
    int strip_warps;
};

// How one multi-grid launch splits its work over warps.
struct MultiPlan {
    int warps;       // warps launched
    int64_t units;   // row-pair units of all grids (strips x row pairs)
    bool aligned;    // strip-aligned (per-grid warps per strip) or even split
};

// Set the multi-grid kernel's attributes for depth K (call outside stream capture).
cudaError_t fused_multi_prepare(int K);
// Plan one multi-grid launch at depth K over n grids (sides nx[i] x ny[i])
// and fill tab[i].begin and tab[i].strip_warps (the caller sets desc and
// cur0).  The strip-aligned split (every strip of a grid on the same row
// ranges, so neighbouring strips share halo columns through L2) is taken
// when its longest warp is within 10 % of the even split's; mixes of many
// small grids get the even split.  warps == 0 on an error.
MultiPlan fused_multi_plan(int K, int n, const int *nx, const int *ny, EpochEntry *tab);
// K steps for every grid of a device epoch table planned by
// fused_multi_plan; the input pair of grid i is tab[i].cur0 ^ flip.
cudaError_t launch_fused_multi(int K, const EpochEntry *tab, int n_grids, const MultiPlan &plan,
                               int flip, int *err, cudaStream_t st);

// Build a 3-D FP32 tensor map over `planes` consecutive pitched planes
// (nx x ny each, `plane_bytes` apart) for the fused path.  Its boxes span
// 128 columns, 2 rows and `box_planes` planes (1 to 4; 0: all `planes`), so
// one box load fetches the same rows of those planes.  Returns false (and a
// message) if the driver entry point is unavailable or the encode call fails.
bool make_pair_tensor_map(CUtensorMap *tm, const void *base, int nx, int ny, int64_t pitch,
                          size_t plane_bytes, const char **why, int planes = 2,
                          int box_planes = 0);

// Thread-local count of kernel launches issued by this library.
void count_launches(int64_t n);

// Record a message for ts_last_error() and return `status` (api.cu).
int set_error(int status, const char *fmt, ...);

// Drop the adjoint record of a grid that is being destroyed (adjoint.cu).
void forget_adjoint(const ::ts_grid *g);

}  // namespace ts
