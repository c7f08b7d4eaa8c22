// The grid handle behind the opaque ts_grid of include/trotter.h (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>

#include "../../include/trotter.h"

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
    double *partials, *result;
    int *err;
    bool tmaps_ok;
    CUtensorMap tm_state[2], tm_phase;   // (re, im) of pair 0 / 1; (gamma_V, s_V)

    void *plane(int i) const { return slab + (size_t)i * L.plane_bytes; }
    void *re() const { return plane(2 * cur); }
    void *im() const { return plane(2 * cur + 1); }
    void *re_other() const { return plane(2 * (cur ^ 1)); }
    void *im_other() const { return plane(2 * (cur ^ 1) + 1); }
    void *pg() const { return plane(4); }
    void *ps() const { return plane(5); }
    void *vp() const { return plane(6); }
    bool f64() const { return L.dtype == TS_F64; }
};

