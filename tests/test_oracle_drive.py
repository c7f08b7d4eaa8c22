"""Pins of the oracle's time-dependent potential V(t) = V0 + a(t) V1 (the
time-dependent extension of Sec. 2), each against something other than the
oracle itself: dense products of exact exponentials, a closed-form global
phase, a fine time-ordered exact propagator (second order in dt with a(t)
sampled at step midpoints), and the exact lattice drift of a packet under a
uniform time-dependent force.
"""
import math

import numpy as np
import pytest
import scipy.integrate

import oracle
from paper_1208_2407_gb300 import workloads as wl

from test_oracle_pins import J, cplx, dense_step2, full_hamiltonian, rand_state


def test_driven_steps_equal_dense_products():
    """Each step n is the dense U2(dt) built with V0 + a[n] V1."""
    nx, ny, dt = 4, 3, 0.2
    rng = np.random.default_rng(1)
    re, im = rand_state(rng, nx, ny)
    V0 = rng.uniform(-1, 1, (ny, nx))
    V1 = rng.uniform(-1, 1, (ny, nx))
    a = [0.7, -1.3, 0.2]
    psi = cplx(re, im)
    for an in a:
        psi = dense_step2(nx, ny, V0 + an * V1, dt) @ psi
    gre, gim = oracle.evolve_driven(re, im, V0, V1, a, dt, J * dt / 2)
    assert np.max(np.abs(cplx(gre, gim) - psi)) < 1e-14


def test_uniform_drive_is_a_global_phase():
    """V1 = 1 adds the global phase exp(-i dt sum_n a[n]) to the V0 result."""
    nx, ny, dt = 9, 7, 0.05
    rng = np.random.default_rng(2)
    re, im = rand_state(rng, nx, ny)
    V0 = rng.uniform(-0.5, 0.5, (ny, nx))
    a = rng.uniform(-2, 2, 23)
    dre, dim = oracle.evolve_driven(re, im, V0, np.ones((ny, nx)), a, dt, J * dt / 2)
    sre, sim = oracle.evolve(re, im, V0, dt, J * dt / 2, len(a))
    expect = np.exp(-1j * dt * np.sum(a)) * cplx(sre, sim)
    assert np.max(np.abs(cplx(dre, dim) - expect)) < 1e-13


def test_constant_drive_equals_static_potential():
    nx, ny, dt = 11, 6, 0.05
    rng = np.random.default_rng(3)
    re, im = rand_state(rng, nx, ny)
    V0 = rng.uniform(-0.5, 0.5, (ny, nx))
    V1 = rng.uniform(-0.5, 0.5, (ny, nx))
    dre, dim = oracle.evolve_driven(re, im, V0, V1, np.full(17, 0.4), dt, J * dt / 2)
    sre, sim = oracle.evolve(re, im, V0 + 0.4 * V1, dt, J * dt / 2, 17)
    assert np.max(np.abs(cplx(dre, dim) - cplx(sre, sim))) < 1e-14


def _drive(t):
    return 0.8 * np.sin(2.0 * t) + 0.3


def _fine_reference(nx, ny, V0, V1, T, psi, n_fine=4096):
    """Time-ordered exp(-i int H(t) dt) by a product of exact exponentials of
    H at the middle of n_fine sub-intervals (error O((T/n_fine)^2))."""
    H0 = full_hamiltonian(nx, ny, V0)
    D = np.ravel(V1)
    d = T / n_fine
    for k in range(n_fine):
        w, Q = np.linalg.eigh(H0 + _drive((k + 0.5) * d) * np.diag(D))
        psi = Q @ (np.exp(-1j * w * d) * (Q.conj().T @ psi))
    return psi


def test_midpoint_sampled_drive_is_second_order():
    """Against the time-ordered exact propagator the error falls ~4x when dt
    is halved with a(t) sampled at step midpoints; sampling at the start of
    each step would leave a first-order error (ratio ~2)."""
    nx, ny, T = 8, 6, 1.2
    rng = np.random.default_rng(4)
    re, im = wl.gaussian_packet(nx, ny, 3.4, 2.6, 1.5, 0.5, -0.3)
    V0 = 0.2 * rng.standard_normal((ny, nx))
    V1 = (np.arange(nx) - nx / 2)[None, :] * np.ones((ny, 1)) * 0.5
    ref = _fine_reference(nx, ny, V0, V1, T, cplx(re, im))
    errs, errs_left = [], []
    for dt in (0.1, 0.05, 0.025):
        n = int(round(T / dt))
        mid = _drive((np.arange(n) + 0.5) * dt)
        left = _drive(np.arange(n) * dt)
        g = oracle.evolve_driven(re, im, V0, V1, mid, dt, J * dt / 2)
        errs.append(np.linalg.norm(cplx(*g) - ref))
        g = oracle.evolve_driven(re, im, V0, V1, left, dt, J * dt / 2)
        errs_left.append(np.linalg.norm(cplx(*g) - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert abs(r1 - 4.0) < 0.4 and abs(r2 - 4.0) < 0.4, (errs, r1, r2)
    assert errs_left[1] / errs_left[2] < 2.5 and errs_left[2] > 5 * errs[2], errs_left


@pytest.mark.parametrize("k0", [0.0, 0.6])
def test_uniform_force_drift_closed_form(k0):
    """Under a uniform force a(t) along x (V1 = x - cx) every Bloch wave keeps
    its shape with quasi-momentum k - A(t), A(t) = int_0^t a; a Gaussian packet
    (momentum spread 1/(2 sigma)) then drifts as
        <x>(T) = x0 + int_0^T 2J sin(k0 - A(t)) exp(-1/(8 sigma^2)) dt,
    exactly on the infinite lattice.  The Trotter result agrees to O(dt^2)."""
    nx, ny, sigma, T = 200, 24, 6.0, 8.0
    x0 = nx / 2.0
    re, im = wl.gaussian_packet(nx, ny, x0, ny / 2.0, sigma, k0, 0.0)
    V1 = (np.arange(nx) - x0)[None, :] * np.ones((ny, 1))
    F0, w = 0.15, 0.7

    def A(t):
        return F0 * math.sin(w * t) / w            # a(t) = F0 cos(w t)

    damp = math.exp(-1.0 / (8.0 * sigma * sigma))
    drift, _ = scipy.integrate.quad(lambda t: 2 * J * math.sin(k0 - A(t)) * damp, 0.0, T,
                                    epsabs=1e-13, epsrel=1e-13)
    resid = []
    for dt in (0.05, 0.025):
        n = int(round(T / dt))
        a = F0 * np.cos(w * (np.arange(n) + 0.5) * dt)
        gre, gim = oracle.evolve_driven(re, im, None, V1, a, dt, J * dt / 2, nthreads=4)
        m = oracle.moments(gre, gim)
        resid.append(m[1] / m[0] - (x0 + drift))
    assert abs(resid[1]) < 2e-3, resid
    if abs(resid[0]) > 1e-4:
        assert 3.0 < resid[0] / resid[1] < 5.0, resid
