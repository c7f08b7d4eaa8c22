// The grid handle behind the opaque ts_grid of include/trotter.h (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <vector>

#include "../../include/trotter.h"
#include "internal.h"

namespace ts {
// Kinetic rotation coefficients of one angle theta (FP64, rounded once where
// used): versine form (g1 = 1 - cos theta, s1 = sin theta), lifting form
// (t1 = tan(theta/2), s1) and the merged angle 2 theta (t2 = tan theta,
// s2 = sin 2 theta).
struct RotCoef {
    double g1, s1, t1, s2, t2;
};
RotCoef rot_coef(double theta);
}  // namespace ts

// One grid: a slab of seven planes (re, im of ping-pong pairs 0 and 1,
// gamma_V, s_V, V) plus reduction scratch; see ts_grid_layout.
struct ts_grid {
    ts_layout L;
    size_t esize;
    unsigned char *slab;
    bool owns_slab;
    int cur;                 // 0: planes 0/1 hold the state, 1: planes 2/3
    double dt, theta, J;
    double g1, s1, t1, s2, t2;   // rotation coefficients (FP64): theta and 2 theta
    int order;                   // 2: U2(dt) per step; 4: U4(dt) (ts_set_potential_order)
    ts::RotCoef sub[2];          // order 4: substeps p dt and (1 - 4p) dt
    unsigned char *tab_b;        // order 4: (gamma_V, s_V) at (1 - 4p) dt, library-owned;
                                 // planes 4/5 then hold the table at p dt
    CUtensorMap tm_phase_b;
    // time-dependent potential V0 + a_n V1 (ts_set_drive): a library-owned
    // slab of three planes (copies of gamma_V, s_V, then V1), its tensor map,
    // the amplitudes a_n and the index of the next one
    unsigned char *drive_slab;
    CUtensorMap tm_drive;
    std::vector<double> drive_a;
    int64_t drive_pos;
    bool driven;
    double *partials, *result;
    int *err;
    cudaEvent_t host_copied;   // host-input copies done (created on first use)
    bool tmaps_ok;
    CUtensorMap tm_state[2], tm_phase;   // (re, im) of pair 0 / 1; (gamma_V, s_V)
    ts::GridDesc *desc_dev;              // the same, for multi-grid launches (in the slab)
    ts::GridDesc desc_host;

    void *plane(int i) const { return slab + (size_t)i * L.plane_bytes; }
    void *re() const { return plane(2 * cur); }
    void *im() const { return plane(2 * cur + 1); }
    void *re_other() const { return plane(2 * (cur ^ 1)); }
    void *im_other() const { return plane(2 * (cur ^ 1) + 1); }
    void *pg() const { return plane(4); }
    void *ps() const { return plane(5); }
    void *vp() const { return plane(6); }
    void *drive_v1() const { return drive_slab + 2 * L.plane_bytes; }
    void *pg_b() const { return tab_b; }
    void *ps_b() const { return tab_b + L.plane_bytes; }
    bool f64() const { return L.dtype == TS_F64; }
    // rows of every plane: ny per slab, nz slabs (3-D grids; nz = 1 in 2-D)
    int64_t rows() const { return L.ny * L.nz; }
    bool is3d() const { return L.nz > 1; }
};


namespace ts {
// Fill a grid handle for a caller-provided slab (tensor maps included) with
// no device work; ts_create_grid adds the zero-fill (api.cu).
ts_status grid_setup(const ts_layout &L, void *slab, bool owns_slab, ts_grid **out);
// Byte offset of the scratch area (partials, result, error word, descriptor).
size_t grid_scratch_offset(const ts_layout &L);
// Rotation coefficients for (dt, theta), and the descriptor (api.cu).
void grid_set_coefficients(ts_grid *g, double dt, double theta, cudaStream_t st);
// Write the grid's multi-grid descriptor (tensor maps, planes, coefficients)
// into its slab on stream st (api.cu).
void grid_write_desc(ts_grid *g, cudaStream_t st);
// Evolve n FP32 grids (|theta| <= pi/4) together with the multi-grid kernel
// at depth K (api.cu).
cudaError_t evolve_multi(ts_grid *const *gs, const int64_t *steps, int n, int K, cudaStream_t st);
}  // namespace ts
