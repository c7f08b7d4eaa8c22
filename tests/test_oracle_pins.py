"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: dense matrix
exponentials of the Hamiltonian pieces of Sec. 2, the exact propagator
exp(-iHt) by eigendecomposition, conservation laws, closed forms and finite
differences.  A plausible mistake in the oracle (a wrong sign of the hopping
term, a wrong parity, a transposed axis, a missing factor, a full instead of a
half angle) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1208_2407_gb300 import workloads as wl

J = 1.0


# ---------------------------------------------------------------------------
# Dense tight-binding pieces (Sec. 2: H = H0 + H1 + H2 per dimension).
# Built from the matrix definitions, independently of the oracle's code.
# Site (x, y) has index y * nx + x.
# ---------------------------------------------------------------------------
def hop_matrix(nx, ny, axis, parity):
    """-J (|j><k| + |k><j|) summed over the pairs of one family.

    axis 'x': pairs ((x,y), (x+1,y)) with x % 2 == parity (x counted from 0);
    axis 'y': pairs ((x,y), (x,y+1)) with y % 2 == parity.
    """
    n = nx * ny
    H = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            if axis == "x" and x % 2 == parity and x + 1 < nx:
                j, k = y * nx + x, y * nx + x + 1
            elif axis == "y" and y % 2 == parity and y + 1 < ny:
                j, k = y * nx + x, (y + 1) * nx + x
            else:
                continue
            H[j, k] = H[k, j] = -J
    return H


def full_hamiltonian(nx, ny, V):
    H = sum(hop_matrix(nx, ny, a, p) for a in "xy" for p in (0, 1))
    if V is not None:
        H = H + np.diag(np.ravel(V))
    return H


def dense_step2(nx, ny, V, dt):
    """U2(dt) as the ordered product of exact exponentials of each piece."""
    E = {(a, p): scipy.linalg.expm(-1j * (dt / 2) * hop_matrix(nx, ny, a, p))
         for a in "xy" for p in (0, 1)}
    P = np.diag(np.exp(-1j * dt * (np.zeros(nx * ny) if V is None else np.ravel(V))))
    order = [("x", 0), ("x", 1), ("y", 0), ("y", 1)]
    U = np.eye(nx * ny, dtype=complex)
    for f in order:                 # applied first -> rightmost
        U = E[f] @ U
    U = P @ U
    for f in reversed(order):
        U = E[f] @ U
    return U


def rand_state(rng, nx, ny):
    re = rng.standard_normal((ny, nx))
    im = rng.standard_normal((ny, nx))
    s = math.sqrt(np.sum(re * re + im * im))
    return re / s, im / s


def cplx(re, im):
    return np.ravel(re) + 1j * np.ravel(im)


def exact_evolve(nx, ny, V, T, psi):
    w, Q = np.linalg.eigh(full_hamiltonian(nx, ny, V))
    return Q @ (np.exp(-1j * w * T) * (Q.conj().T @ psi))


# ---------------------------------------------------------------------------
# P1: one step equals the dense product of block exponentials (odd sizes too).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (4, 6), (5, 7), (1, 7), (7, 1), (6, 4), (2, 1)])
def test_step_equals_dense_product(nx, ny):
    rng = np.random.default_rng(nx * 100 + ny)
    re, im = rand_state(rng, nx, ny)
    V = rng.uniform(-1.0, 1.0, (ny, nx))
    dt = 0.37
    U = dense_step2(nx, ny, V, dt)
    want = U @ cplx(re, im)
    gre, gim = oracle.evolve(re, im, V, dt, J * dt / 2, 1)
    assert np.max(np.abs(cplx(gre, gim) - want)) < 1e-14


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("parity", [0, 1])
def test_single_sweep_equals_block_exponential(axis, parity):
    nx, ny = 5, 6
    rng = np.random.default_rng(7)
    re, im = rand_state(rng, nx, ny)
    theta = 0.3
    E = scipy.linalg.expm(-1j * (theta / J) * hop_matrix(nx, ny, axis, parity))
    gre, gim = oracle.sweep(re, im, axis, parity, theta)
    assert np.max(np.abs(cplx(gre, gim) - E @ cplx(re, im))) < 1e-14


def test_phase_equals_diagonal_exponential():
    nx, ny = 4, 3
    rng = np.random.default_rng(3)
    re, im = rand_state(rng, nx, ny)
    V = rng.uniform(-2, 2, (ny, nx))
    gre, gim = oracle.phase(re, im, V, 0.21)
    want = np.exp(-1j * 0.21 * np.ravel(V)) * cplx(re, im)
    assert np.max(np.abs(cplx(gre, gim) - want)) < 1e-15


# ---------------------------------------------------------------------------
# P2: converges to exp(-iHT) with error ~ dt^2 (second order), dt (first),
# dt^4 (fourth order, Eq. fourthorder).
# ---------------------------------------------------------------------------
def _trotter_errors(order, dts, nx=12, ny=10, T=1.6):
    rng = np.random.default_rng(11)
    re, im = wl.gaussian_packet(nx, ny, 5.3, 4.6, 1.7, 0.6, -0.4)
    V = 0.3 * np.sin(0.7 * np.arange(nx))[None, :] * np.cos(0.5 * np.arange(ny))[:, None]
    V = V + 0.05 * rng.standard_normal((ny, nx))
    exact = exact_evolve(nx, ny, V, T, cplx(re, im))
    errs = []
    for dt in dts:
        steps = int(round(T / dt))
        gre, gim = oracle.evolve(re, im, V, dt, J * dt / 2, steps, order=order)
        errs.append(np.linalg.norm(cplx(gre, gim) - exact))
    return errs


def test_second_order_error_scaling():
    e = _trotter_errors(2, [0.1, 0.05, 0.025])
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert abs(r1 - 4.0) < 0.3 and abs(r2 - 4.0) < 0.3, (e, r1, r2)
    assert e[2] < 1e-3


def test_first_order_error_scaling():
    e = _trotter_errors(1, [0.05, 0.025, 0.0125])
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert abs(r1 - 2.0) < 0.3 and abs(r2 - 2.0) < 0.3, (e, r1, r2)


def test_fourth_order_error_scaling():
    e = _trotter_errors(4, [0.2, 0.1, 0.05])
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 13.0 < r2 < 19.0 and r1 > 10.0, (e, r1, r2)


def test_flipped_sign_fails_exact_propagator():
    """A rotation with -i sin (the literal sign printed for M) would follow a
    Hamiltonian with +J hopping; the oracle must not match that one."""
    nx, ny, T, dt = 8, 6, 1.0, 0.01
    re, im = wl.gaussian_packet(nx, ny, 3.2, 2.5, 1.3, 0.8, 0.0)
    psi = cplx(re, im)
    good = exact_evolve(nx, ny, None, T, psi)
    Hflip = -full_hamiltonian(nx, ny, None)
    w, Q = np.linalg.eigh(Hflip)
    bad = Q @ (np.exp(-1j * w * T) * (Q.conj().T @ psi))
    gre, gim = oracle.evolve(re, im, None, dt, J * dt / 2, int(T / dt))
    got = cplx(gre, gim)
    assert np.linalg.norm(got - good) < 1e-4
    assert np.linalg.norm(got - bad) > 1e-2


# ---------------------------------------------------------------------------
# P3: unitarity (Sec. 2: U is unitary, the norm is conserved).
# ---------------------------------------------------------------------------
def test_norm_conserved_plain_workload():
    c = wl.plain_fp64_256()
    n0 = oracle.norm(c["re"], c["im"])
    re, im = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    assert abs(n0 - 1.0) < 1e-13
    assert abs(oracle.norm(re, im) - n0) < 1e-12


def test_norm_conserved_harmonic():
    c = wl.harmonic_2048(seed=1, n=384, steps=60)
    re, im = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"], nthreads=4)
    assert abs(oracle.norm(re, im) - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# P4: reversibility: U2(-dt) U2(dt) = 1 step by step.
# ---------------------------------------------------------------------------
def test_time_reversal():
    rng = np.random.default_rng(5)
    nx, ny = 37, 24
    re0, im0 = rand_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    dt = 0.05
    re, im = oracle.evolve(re0, im0, V, dt, dt / 2, 50)
    assert np.max(np.abs(re - re0)) > 1e-3       # it did move
    re, im = oracle.evolve(re, im, V, -dt, -dt / 2, 50)
    assert np.max(np.abs(re - re0)) < 1e-12 and np.max(np.abs(im - im0)) < 1e-12


# ---------------------------------------------------------------------------
# P5: separability: V = 0 and a product state stay a product of 1-D chains.
# ---------------------------------------------------------------------------
def test_separable_outer_product():
    nx, ny, dt, steps = 24, 17, 0.05, 40
    x, y = np.arange(nx), np.arange(ny)
    f = np.exp(-((x - 9.0) ** 2) / 12.0 + 0.7j * x)
    g = np.exp(-((y - 7.0) ** 2) / 8.0 - 0.3j * y)
    f /= np.linalg.norm(f)
    g /= np.linalg.norm(g)

    def chain_step(n):
        Ee = scipy.linalg.expm(-1j * (dt / 2) * hop_matrix(n, 1, "x", 0))
        Eo = scipy.linalg.expm(-1j * (dt / 2) * hop_matrix(n, 1, "x", 1))
        return Ee @ Eo @ Eo @ Ee

    fT = np.linalg.matrix_power(chain_step(nx), steps) @ f
    gT = np.linalg.matrix_power(chain_step(ny), steps) @ g
    psi = np.outer(g, f)
    gre, gim = oracle.evolve(psi.real, psi.imag, None, dt, dt / 2, steps)
    assert np.max(np.abs((gre + 1j * gim) - np.outer(gT, fT))) < 1e-13


# ---------------------------------------------------------------------------
# P6: a flat potential only adds the global phase exp(-i v0 T).
# ---------------------------------------------------------------------------
def test_flat_potential_global_phase():
    rng = np.random.default_rng(9)
    nx, ny, dt, steps, v0 = 19, 22, 0.05, 30, 0.73
    re, im = rand_state(rng, nx, ny)
    a_re, a_im = oracle.evolve(re, im, None, dt, dt / 2, steps)
    b_re, b_im = oracle.evolve(re, im, np.full((ny, nx), v0), dt, dt / 2, steps)
    want = np.exp(-1j * v0 * dt * steps) * (a_re + 1j * a_im)
    assert np.max(np.abs((b_re + 1j * b_im) - want)) < 1e-13


# ---------------------------------------------------------------------------
# P7: free packet against the closed forms of exact lattice dynamics.
# x(t) = x(0) + v t with v = 2 J sin p; sigma_k = 1 / (2 sigma):
#   <x>(t) = x0 + 2 J t sin(k) exp(-sigma_k^2 / 2)
#   Var x(t) = sigma^2 + 4 J^2 t^2 [1/2 (1 - cos 2k exp(-2 sigma_k^2))
#                                   - sin^2 k exp(-sigma_k^2)]
# ---------------------------------------------------------------------------
def _closed_form(x0, sigma, k, t):
    sk = 1.0 / (2.0 * sigma)
    mean = x0 + 2 * J * t * math.sin(k) * math.exp(-sk * sk / 2)
    var = sigma ** 2 + 4 * J * J * t * t * (
        0.5 * (1 - math.cos(2 * k) * math.exp(-2 * sk * sk))
        - math.sin(k) ** 2 * math.exp(-sk * sk))
    return mean, var


def test_free_packet_plain_workload():
    """The 256^2 FP64 workload: the packet drifts ~4.79 sites in t = 5; the
    residual against the exact-dynamics closed form is the Trotter error and
    shrinks as dt^2."""
    c = wl.plain_fp64_256()
    t = c["dt"] * c["steps"]
    mean, var = _closed_form(128.0, 16.0, 0.5, t)
    assert abs(mean - 128.0 - 4.79) < 0.01
    resid = []
    for dt in (c["dt"], c["dt"] / 2):
        re, im = oracle.evolve(c["re"], c["im"], None, dt, J * dt / 2, int(round(t / dt)))
        m = oracle.moments(re, im)
        resid.append(m[1] / m[0] - mean)
        assert abs(m[3] / m[0] - (m[1] / m[0]) ** 2 - var) < 1e-4 * var
        assert abs(m[2] / m[0] - 128.0) < 1e-9          # no drift along y (ky = 0)
    assert abs(resid[0]) < 3e-3
    assert abs(resid[0] / resid[1] - 4.0) < 0.1


@pytest.mark.parametrize("k", [0.0, 0.5, -1.1])
def test_free_packet_spreading(k):
    nx, ny, dt, steps, sigma, x0 = 192, 4, 0.05, 400, 4.0, 96.0
    re, im = wl.gaussian_packet(nx, ny, x0, 1.5, sigma, k, 0.0)
    # make the y-direction trivial: one row only carries the packet
    re, im = re[:1].copy(), im[:1].copy()
    s = math.sqrt(np.sum(re * re + im * im))
    re, im = re / s, im / s
    re, im = oracle.evolve(re, im, None, dt, dt / 2, steps)
    m = oracle.moments(re, im)
    mean, var = _closed_form(x0, sigma, k, dt * steps)
    assert abs(m[1] / m[0] - mean) < 2e-2
    assert abs((m[3] / m[0] - (m[1] / m[0]) ** 2) - var) < 5e-3 * var


# ---------------------------------------------------------------------------
# P8: two-site chain: each step rotates by the accumulated angle 2 theta.
# ---------------------------------------------------------------------------
def test_two_site_chain_rotation():
    theta, n = 0.113, 37
    a, b = 0.6 + 0.2j, -0.3 + 0.7j
    re = np.array([[a.real, b.real]])
    im = np.array([[a.imag, b.imag]])
    gre, gim = oracle.evolve(re, im, None, 2 * theta / J, theta, n)
    ang = 2 * n * theta
    wa = math.cos(ang) * a + 1j * math.sin(ang) * b
    wb = 1j * math.sin(ang) * a + math.cos(ang) * b
    assert abs(complex(gre[0, 0], gim[0, 0]) - wa) < 1e-14
    assert abs(complex(gre[0, 1], gim[0, 1]) - wb) < 1e-14


def test_single_site_is_pure_phase():
    re, im = np.array([[0.8]]), np.array([[0.6]])
    gre, gim = oracle.evolve(re, im, np.array([[1.7]]), 0.05, 0.025, 10)
    want = np.exp(-1j * 1.7 * 0.5) * (0.8 + 0.6j)
    assert abs(complex(gre[0, 0], gim[0, 0]) - want) < 1e-15


# ---------------------------------------------------------------------------
# Observables against direct dense definitions.
# ---------------------------------------------------------------------------
def test_energy_equals_dense_expectation():
    nx, ny = 6, 5
    rng = np.random.default_rng(13)
    re, im = rand_state(rng, nx, ny)
    V = rng.uniform(-1, 1, (ny, nx))
    psi = cplx(re, im)
    kin, pot = oracle.energy(re, im, V, J)
    Hk = full_hamiltonian(nx, ny, None)
    assert abs(kin - np.real(psi.conj() @ Hk @ psi)) < 1e-14
    assert abs(pot - np.real(psi.conj() @ (np.ravel(V) * psi))) < 1e-14


def test_moments_and_inner_against_numpy():
    rng = np.random.default_rng(17)
    nx, ny = 9, 7
    re, im = rand_state(rng, nx, ny)
    p = re * re + im * im
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    m = oracle.moments(re, im)
    want = [p.sum(), (X * p).sum(), (Y * p).sum(), (X * X * p).sum(), (Y * Y * p).sum()]
    assert np.allclose(m, want, rtol=1e-14, atol=1e-14)
    b_re, b_im = rand_state(rng, nx, ny)
    z = oracle.inner(re, im, b_re, b_im)
    assert abs(z - np.vdot(cplx(re, im), cplx(b_re, b_im))) < 1e-14


def test_compensated_sum_is_exactly_rounded_on_cancellation():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.standard_normal(1000) * 1e16, rng.standard_normal(1000)])
    v = np.concatenate([v, -v[:1000]])
    rng.shuffle(v)
    assert oracle.compensated_sum(v) == pytest.approx(math.fsum(v), abs=1e-12)


# ---------------------------------------------------------------------------
# P9: adjoint gradient of the fidelity.
# ---------------------------------------------------------------------------
def _fidelity(re, im, tre, tim, V, dt, steps):
    gre, gim = oracle.evolve(re, im, V, dt, dt / 2, steps)
    return abs(np.vdot(cplx(tre, tim), cplx(gre, gim))) ** 2


@pytest.mark.parametrize("nx,ny,steps", [(6, 5, 12), (8, 8, 20), (4, 7, 9)])
def test_adjoint_matches_finite_differences(nx, ny, steps):
    rng = np.random.default_rng(nx * 31 + ny)
    re, im = rand_state(rng, nx, ny)
    tre, tim = rand_state(rng, nx, ny)
    V = rng.uniform(-0.5, 0.5, (ny, nx))
    dt = 0.13
    g, F, _ = oracle.adjoint_grad(re, im, tre, tim, V, dt, dt / 2, steps)
    assert F == pytest.approx(_fidelity(re, im, tre, tim, V, dt, steps), abs=1e-14)
    h = 1e-5
    fd = np.zeros_like(V)
    for j in range(V.size):
        Vp, Vm = V.copy(), V.copy()
        Vp.flat[j] += h
        Vm.flat[j] -= h
        fd.flat[j] = (_fidelity(re, im, tre, tim, Vp, dt, steps)
                      - _fidelity(re, im, tre, tim, Vm, dt, steps)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    # a constant shift of V is a global phase: the gradient sums to zero
    assert abs(np.sum(g)) < 1e-12 * max(1.0, np.sum(np.abs(g)))


def test_adjoint_gradient_sums_to_zero_on_a_packet_pair():
    c = wl.adjoint_pair(n=48, steps=40, seed=3)
    g, F, _ = oracle.adjoint_grad(c["re"], c["im"], c["target_re"], c["target_im"], c["V"],
                                  c["dt"], c["theta"], c["steps"])
    assert 0.01 < F < 0.99
    assert abs(np.sum(g)) < 1e-12 * np.sum(np.abs(g))
