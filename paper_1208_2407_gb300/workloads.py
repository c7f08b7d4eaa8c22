"""Seeded synthetic inputs: wave packets, potentials and request mixes.

This module holds no step of the Trotter-Suzuki method itself: it only draws
and shapes the inputs (initial states, potentials, serving requests) that both
the CUDA library and the CPU oracle consume.  All randomness comes from
``numpy.random.default_rng(seed)``, drawn in the order documented per function,
so that every workload is reproducible from its seed.

Arrays are dense, row-major, shape (ny, nx), FP64: site (x, y) is ``a[y, x]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def gaussian_packet(nx: int, ny: int, x0: float, y0: float, sigma: float,
                    kx: float = 0.0, ky: float = 0.0):
    """psi(x, y) ~ exp(-((x-x0)^2 + (y-y0)^2) / (4 sigma^2)) exp(i (kx x + ky y)).

    sigma is the standard deviation of |psi|^2 along each axis; x and y are the
    absolute site coordinates.  Normalised so that sum |psi|^2 = 1 on the grid.
    The packet is separable, so it is built as an outer product.
    """
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    gx = np.exp(-((x - x0) ** 2) / (4.0 * sigma * sigma)) * np.exp(1j * kx * x)
    gy = np.exp(-((y - y0) ** 2) / (4.0 * sigma * sigma)) * np.exp(1j * ky * y)
    nrm = np.sqrt(np.sum(np.abs(gx) ** 2) * np.sum(np.abs(gy) ** 2))
    psi = np.outer(gy, gx) / nrm
    return np.ascontiguousarray(psi.real), np.ascontiguousarray(psi.imag)


def gaussian_packet3(nx: int, ny: int, nz: int, x0: float, y0: float, z0: float,
                     sigma: float, kx: float = 0.0, ky: float = 0.0, kz: float = 0.0):
    """The 3-D packet, arrays of shape (nz, ny, nx): the product of three 1-D
    Gaussians with the same sigma, normalised on the grid."""
    axes = []
    for n, c, k in ((nx, x0, kx), (ny, y0, ky), (nz, z0, kz)):
        t = np.arange(n, dtype=np.float64)
        g = np.exp(-((t - c) ** 2) / (4.0 * sigma * sigma)) * np.exp(1j * k * t)
        axes.append(g / np.sqrt(np.sum(np.abs(g) ** 2)))
    psi = np.einsum("z,y,x->zyx", axes[2], axes[1], axes[0])
    return np.ascontiguousarray(psi.real), np.ascontiguousarray(psi.imag)


def harmonic_potential3(nx: int, ny: int, nz: int, w: float):
    """V = 0.5 w^2 r^2 about the grid centre (nx/2, ny/2, nz/2), shape (nz, ny, nx)."""
    x = np.arange(nx, dtype=np.float64) - nx / 2.0
    y = np.arange(ny, dtype=np.float64) - ny / 2.0
    z = np.arange(nz, dtype=np.float64) - nz / 2.0
    return 0.5 * w * w * (x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)


def harmonic_3d(n: int = 128, steps: int = 200, seed: int = 0):
    """n^3 lattice, harmonic V (w = 1e-2), a packet drawn as in the 2-D case
    (centre in the middle half of each axis, sigma in [n/16, n/8], momentum
    components in [-1, 1]); draw order x0, y0, z0, sigma, kx, ky, kz."""
    rng = np.random.default_rng(seed)
    x0, y0, z0 = (rng.uniform(n / 4.0, 3.0 * n / 4.0) for _ in range(3))
    sigma = rng.uniform(n / 16.0, n / 8.0)
    kx, ky, kz = (rng.uniform(-1.0, 1.0) for _ in range(3))
    re, im = gaussian_packet3(n, n, n, x0, y0, z0, sigma, kx, ky, kz)
    V = harmonic_potential3(n, n, n, 1e-2)
    return dict(nx=n, ny=n, nz=n, re=re, im=im, V=V, dt=DT, theta=THETA, steps=steps, seed=seed)


def random_packet_params(rng: np.random.Generator, nx: int, ny: int,
                         sigma_range=(16.0, 64.0)):
    """Draw (x0, y0, sigma, kx, ky), in that order.

    Centre uniform in the middle half of each axis, sigma uniform in
    ``sigma_range``, each momentum component uniform in [-1, 1] rad/site.
    """
    x0 = rng.uniform(nx / 4.0, 3.0 * nx / 4.0)
    y0 = rng.uniform(ny / 4.0, 3.0 * ny / 4.0)
    sigma = rng.uniform(*sigma_range)
    kx = rng.uniform(-1.0, 1.0)
    ky = rng.uniform(-1.0, 1.0)
    return dict(x0=x0, y0=y0, sigma=sigma, kx=kx, ky=ky)


def harmonic_potential(nx: int, ny: int, w: float, cx: float | None = None,
                       cy: float | None = None):
    """V = 0.5 w^2 ((x-cx)^2 + (y-cy)^2), centred at (nx/2, ny/2) by default."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    return 0.5 * w * w * ((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2)


def random_gaussians_potential(rng: np.random.Generator, nx: int, ny: int,
                               count: int = 32, amp=(-0.5, 0.5), width=(20.0, 200.0)):
    """V = sum_g A_g exp(-((x-cx_g)^2 + (y-cy_g)^2) / (2 w_g^2)).

    Draw order: all centres x, all centres y (uniform on the grid), all
    amplitudes A_g (uniform in ``amp``), all widths w_g (uniform in ``width``,
    the Gaussian standard deviation in sites).  Each term is separable, so V
    is a (ny x count) @ (count x nx) product.
    """
    cx = rng.uniform(0.0, nx, count)
    cy = rng.uniform(0.0, ny, count)
    A = rng.uniform(amp[0], amp[1], count)
    w = rng.uniform(width[0], width[1], count)
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    gx = np.exp(-((x[None, :] - cx[:, None]) ** 2) / (2.0 * w[:, None] ** 2))
    gy = np.exp(-((y[None, :] - cy[:, None]) ** 2) / (2.0 * w[:, None] ** 2))
    return np.ascontiguousarray((gy.T * A[None, :]) @ gx)


# --------------------------------------------------------------------------
# The five workloads of the method's evaluation (sizes, distributions).
# --------------------------------------------------------------------------
DT = 0.05
THETA = 0.025   # J dt / 2 with hopping J = 1


def plain_fp64_256():
    """256 x 256, V = 0, packet at (128, 128), sigma 16, kx 0.5; 100 steps."""
    re, im = gaussian_packet(256, 256, 128.0, 128.0, 16.0, 0.5, 0.0)
    return dict(nx=256, ny=256, re=re, im=im, V=None, dt=DT, theta=THETA, steps=100)


def harmonic_2048(seed: int = 0, n: int = 2048, steps: int = 1000):
    """n x n, harmonic V (w = 1e-3) centred on the grid, seed-random packet."""
    rng = np.random.default_rng(seed)
    p = random_packet_params(rng, n, n)
    re, im = gaussian_packet(n, n, **p)
    V = harmonic_potential(n, n, 1e-3)
    return dict(nx=n, ny=n, re=re, im=im, V=V, dt=DT, theta=THETA, steps=steps,
                seed=seed, packet=p)


def roofline_grid(n: int = 8192, seed: int = 0, steps: int = 200):
    """n x n, 32 random Gaussians in V, one seed-random packet; 200 steps."""
    rng = np.random.default_rng(seed)
    p = random_packet_params(rng, n, n)
    V = random_gaussians_potential(rng, n, n)
    re, im = gaussian_packet(n, n, **p)
    return dict(nx=n, ny=n, re=re, im=im, V=V, dt=DT, theta=THETA, steps=steps,
                seed=seed, packet=p)


def adjoint_pair(n: int = 1024, steps: int = 500, seed: int = 0, dt: float = DT,
                 J: float = 1.0):
    """Seed-random initial packet and a target packet it actually reaches.

    Draw order: initial packet (as ``random_packet_params``), then a target
    offset (two uniforms in [-1, 1] scaled by the initial sigma / 2) and the
    target sigma factor (uniform in [0.8, 1.25]).  The target centre is the
    initial centre moved by the lattice group velocity 2 J sin(k) over the
    evolution time, plus that offset, so that the fidelity is well inside
    (0, 1).  The potential is the harmonic trap of the precision workload.
    """
    rng = np.random.default_rng(seed)
    p = random_packet_params(rng, n, n)
    T = steps * dt
    off = rng.uniform(-1.0, 1.0, 2) * p["sigma"] / 2.0
    sfac = rng.uniform(0.8, 1.25)
    tx = p["x0"] + 2.0 * J * np.sin(p["kx"]) * T + off[0]
    ty = p["y0"] + 2.0 * J * np.sin(p["ky"]) * T + off[1]
    re, im = gaussian_packet(n, n, **p)
    tre, tim = gaussian_packet(n, n, tx, ty, p["sigma"] * sfac, p["kx"], p["ky"])
    V = harmonic_potential(n, n, 1e-3)
    return dict(nx=n, ny=n, re=re, im=im, target_re=tre, target_im=tim, V=V, dt=dt,
                theta=J * dt / 2.0, steps=steps, seed=seed)


@dataclass
class Request:
    """One serving request: a grid, a step count, a potential and a packet."""
    rid: int
    arrival_s: float
    nx: int
    ny: int
    steps: int
    seed: int
    dt: float = DT
    theta: float = THETA
    extra: dict = field(default_factory=dict)

    def inputs(self):
        rng = np.random.default_rng(self.seed)
        p = random_packet_params(rng, self.nx, self.ny,
                                 sigma_range=(min(16.0, self.nx / 16, self.ny / 16),
                                              min(64.0, self.nx / 8, self.ny / 8)))
        V = random_gaussians_potential(rng, self.nx, self.ny)
        re, im = gaussian_packet(self.nx, self.ny, **p)
        return re, im, V


SERVE_SIDES = (128, 256, 512, 1024, 2048, 4096)


def serving_requests(count: int = 512, mean_gap_s: float = 2e-3, seed: int = 0,
                     sides=SERVE_SIDES, steps_range=(10, 2000)):
    """Poisson arrivals (exponential gaps, mean ``mean_gap_s``); each side drawn
    independently from ``sides``; steps uniform in ``steps_range`` inclusive.

    Draw order per request: gap, nx, ny, steps.  Each request's potential and
    packet come from its own seed (``seed * 100003 + rid``).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(mean_gap_s)
        nx = int(rng.choice(sides))
        ny = int(rng.choice(sides))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append(Request(rid=rid, arrival_s=t, nx=nx, ny=ny, steps=steps,
                           seed=seed * 100003 + rid))
    return out
