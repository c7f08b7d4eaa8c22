"""Pins of the oracle's three-dimensional step (Sec. 2's splitting with two
terms per dimension, extended to z as Sec. 6 proposes), each against
something other than the oracle: dense products of exact block exponentials
on tiny lattices, the exact propagator's dt^2 convergence, separability into
three 1-D chains, the 2-D oracle at nz = 1, and dense expectation values.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle

J = 1.0


def hop3(nx, ny, nz, axis, parity):
    """-J (|j><k| + |k><j|) over the pairs of one family along axis 0/1/2."""
    n = nx * ny * nz
    H = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (x, y, z)
                if c[axis] % 2 != parity:
                    continue
                d = list(c)
                d[axis] += 1
                if d[axis] >= (nx, ny, nz)[axis]:
                    continue
                j = (z * ny + y) * nx + x
                k = (d[2] * ny + d[1]) * nx + d[0]
                H[j, k] = H[k, j] = -J
    return H


def dense_step3(nx, ny, nz, V, dt):
    order = [(a, p) for a in range(3) for p in (0, 1)]
    E = {f: scipy.linalg.expm(-1j * (dt / 2) * hop3(nx, ny, nz, *f)) for f in order}
    P = np.diag(np.exp(-1j * dt * np.ravel(V)))
    U = np.eye(nx * ny * nz, dtype=complex)
    for f in order:
        U = E[f] @ U
    U = P @ U
    for f in reversed(order):
        U = E[f] @ U
    return U


def rand3(rng, nx, ny, nz):
    re = rng.standard_normal((nz, ny, nx))
    im = rng.standard_normal((nz, ny, nx))
    s = math.sqrt(np.sum(re * re + im * im))
    return re / s, im / s


def c(re, im):
    return np.ravel(re) + 1j * np.ravel(im)


@pytest.mark.parametrize("nx,ny,nz", [(2, 2, 2), (3, 2, 3), (2, 3, 4), (1, 3, 5), (4, 1, 3),
                                      (3, 3, 1)])
def test_step_equals_dense_product(nx, ny, nz):
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    re, im = rand3(rng, nx, ny, nz)
    V = rng.uniform(-1, 1, (nz, ny, nx))
    dt = 0.3
    gre, gim = oracle.evolve3(re, im, V, dt, J * dt / 2, 2)
    U = dense_step3(nx, ny, nz, V, dt)
    assert np.max(np.abs(c(gre, gim) - U @ (U @ c(re, im)))) < 1e-14


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("parity", [0, 1])
def test_single_sweep_equals_block_exponential(axis, parity):
    nx, ny, nz, th = 3, 4, 5, 0.37
    rng = np.random.default_rng(7 + axis * 2 + parity)
    re, im = rand3(rng, nx, ny, nz)
    gre, gim = oracle.sweep3(re, im, axis, parity, th)
    E = scipy.linalg.expm(-1j * (th / J) * hop3(nx, ny, nz, axis, parity))
    assert np.max(np.abs(c(gre, gim) - E @ c(re, im))) < 1e-14


def test_nz1_equals_2d_oracle_bitwise():
    rng = np.random.default_rng(3)
    re, im = rng.standard_normal((2, 13, 17))
    V = rng.uniform(-0.5, 0.5, (13, 17))
    a = oracle.evolve(re, im, V, 0.05, 0.025, 7)
    b = oracle.evolve3(re[None], im[None], V[None], 0.05, 0.025, 7)
    assert np.array_equal(a[0], b[0][0]) and np.array_equal(a[1], b[1][0])


def test_second_order_against_exact_propagator():
    nx, ny, nz, T = 5, 4, 4, 1.2
    rng = np.random.default_rng(5)
    re, im = rand3(rng, nx, ny, nz)
    V = 0.3 * rng.standard_normal((nz, ny, nx))
    H = sum(hop3(nx, ny, nz, a, p) for a in range(3) for p in (0, 1)) + np.diag(np.ravel(V))
    w, Q = np.linalg.eigh(H)
    exact = Q @ (np.exp(-1j * w * T) * (Q.conj().T @ c(re, im)))
    errs = []
    for dt in (0.1, 0.05, 0.025):
        n = int(round(T / dt))
        errs.append(np.linalg.norm(c(*oracle.evolve3(re, im, V, dt, J * dt / 2, n)) - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert abs(r1 - 4.0) < 0.3 and abs(r2 - 4.0) < 0.3, (errs, r1, r2)


def _chain(n, f, steps, dt):
    """A 1-D chain under the same split: even, odd, odd, even half sweeps."""
    Ee = scipy.linalg.expm(-1j * (dt / 2) * hop3(n, 1, 1, 0, 0))
    Eo = scipy.linalg.expm(-1j * (dt / 2) * hop3(n, 1, 1, 0, 1))
    U = Ee @ Eo @ Eo @ Ee
    for _ in range(steps):
        f = U @ f
    return f


def test_separable_product_state():
    """V = 0: the step of a product state f(x) g(y) h(z) is the product of
    three 1-D chain steps (X, Y and Z factors act on different coordinates)."""
    nx, ny, nz, dt, steps = 9, 7, 6, 0.1, 11
    rng = np.random.default_rng(9)
    f = rng.standard_normal(nx) + 1j * rng.standard_normal(nx)
    g = rng.standard_normal(ny) + 1j * rng.standard_normal(ny)
    h = rng.standard_normal(nz) + 1j * rng.standard_normal(nz)
    psi = np.einsum("z,y,x->zyx", h, g, f)
    gre, gim = oracle.evolve3(psi.real, psi.imag, None, dt, J * dt / 2, steps)
    expect = np.einsum("z,y,x->zyx", _chain(nz, h, steps, dt), _chain(ny, g, steps, dt),
                       _chain(nx, f, steps, dt))
    assert np.max(np.abs((gre + 1j * gim) - expect)) < 1e-13


def test_norm_and_reversal():
    rng = np.random.default_rng(10)
    re, im = rand3(rng, 11, 9, 7)
    V = rng.uniform(-0.5, 0.5, (7, 9, 11))
    fre, fim = oracle.evolve3(re, im, V, 0.05, 0.025, 40)
    assert abs(np.sum(fre ** 2 + fim ** 2) - 1.0) < 1e-12
    bre, bim = oracle.evolve3(fre, fim, V, -0.05, -0.025, 40)
    assert np.max(np.abs(c(bre, bim) - c(re, im))) < 1e-12


def test_moments_and_energy_against_dense():
    nx, ny, nz = 4, 3, 5
    rng = np.random.default_rng(11)
    re, im = rand3(rng, nx, ny, nz)
    V = rng.uniform(-1, 1, (nz, ny, nx))
    p = re ** 2 + im ** 2
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = oracle.moments3(re, im)
    ref = [p.sum(), (x * p).sum(), (y * p).sum(), (z * p).sum(), (x * x * p).sum(),
           (y * y * p).sum(), (z * z * p).sum()]
    assert np.allclose(m, ref, rtol=0, atol=1e-13)
    H0 = sum(hop3(nx, ny, nz, a, q) for a in range(3) for q in (0, 1))
    psi = c(re, im)
    kin, pot = oracle.energy3(re, im, V)
    assert abs(kin - np.vdot(psi, H0 @ psi).real) < 1e-13
    assert abs(pot - np.sum(np.ravel(V) * np.abs(psi) ** 2)) < 1e-13
