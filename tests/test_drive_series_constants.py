"""The fused kernel's drive phase evaluates sin(phi) = phi P(u) and
1 - cos(phi) = u Q(u), u = phi^2, with cubics P and Q whose FP32 constants
sit in fused.cu (DRIVE_P1..3, DRIVE_Q1..3).  This checks those constants on
the CPU, with no GPU: against sin x / x and (1 - cos x) / x^2 in FP64 over
the range the kernel uses them on (|phi| <= 0.8, u <= 0.64), and through an
FP32 emulation of the kernel's evaluation order against the exact angles."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FUSED = os.path.join(ROOT, "paper_1208_2407_gb300", "csrc", "fused.cu")
U_MAX = 0.64


def drive_constants():
    with open(FUSED) as f:
        src = f.read()
    out = {}
    for name in ("P1", "P2", "P3", "Q1", "Q2", "Q3"):
        m = re.search(r"DRIVE_%s = ([-+]?0x[0-9a-fA-F.]+p[-+]?\d+)f" % name, src)
        assert m, "DRIVE_%s not found in fused.cu" % name
        out[name] = float(np.float32(float.fromhex(m.group(1))))
    return out


def p_exact(u):
    # sin(x)/x and (1 - cos x)/x^2 as series in u = x^2 (alternating, converging fast
    # for u <= 0.64: the terms through u^12 leave less than 1e-40)
    return sum((-1) ** k * u ** k / math.factorial(2 * k + 1) for k in range(13))


def q_exact(u):
    return sum((-1) ** k * u ** k / math.factorial(2 * k + 2) for k in range(13))


def test_series_form_matches_sin_and_cos():
    # the series above against the library functions, so that they can serve as the
    # reference below (where sin(x)/x loses digits to cancellation near 0, the
    # comparison starts at x = 0.05)
    x = np.linspace(0.05, 0.8, 2001)
    u = x * x
    assert np.max(np.abs(p_exact(u) - np.sin(x) / x)) < 1e-15
    assert np.max(np.abs(q_exact(u) - (1 - np.cos(x)) / u)) < 1e-13


def test_cubics_are_within_their_stated_error():
    c = drive_constants()
    u = np.linspace(0.0, U_MAX, 200001)
    P = 1.0 + u * (c["P1"] + u * (c["P2"] + u * c["P3"]))
    Q = 0.5 + u * (c["Q1"] + u * (c["Q2"] + u * c["Q3"]))
    assert np.max(np.abs(P - p_exact(u))) < 7e-9
    assert np.max(np.abs(Q - q_exact(u))) < 7e-10
    # the Taylor cubics (the series cut after u^3) are 60-70 times further off, which
    # is what fitting the coefficients to the range buys
    Pt = 1.0 - u / 6 + u ** 2 / 120 - u ** 3 / 5040
    Qt = 0.5 - u / 24 + u ** 2 / 720 - u ** 3 / 40320
    assert np.max(np.abs(Pt - p_exact(u))) > 50 * np.max(np.abs(P - p_exact(u)))
    assert np.max(np.abs(Qt - q_exact(u))) > 50 * np.max(np.abs(Q - q_exact(u)))


def test_fp32_evaluation_relative_error():
    # the kernel's order of operations in FP32: u = phi phi, Horner with FMAs, then
    # s = phi P and g = u Q; an FMA rounds once, emulated here as the FP64 sum of an
    # exact FP32 product, rounded to FP32
    c = drive_constants()
    f32 = np.float32

    def fma(a, b, d):
        return (a.astype(np.float64) * b.astype(np.float64) + d.astype(np.float64)).astype(f32)

    def k(v):
        return f32(v)

    rng = np.random.default_rng(7)
    phi = np.concatenate([rng.uniform(-0.8, 0.8, 200000), np.linspace(-0.8, 0.8, 20001),
                          np.array([1e-30, -1e-12, 1e-6, 0.8, -0.8])]).astype(f32)
    u = (phi.astype(np.float64) * phi.astype(np.float64)).astype(f32)
    P = fma(u, np.full_like(u, k(c["P3"])), np.full_like(u, k(c["P2"])))
    Q = fma(u, np.full_like(u, k(c["Q3"])), np.full_like(u, k(c["Q2"])))
    P = fma(u, P, np.full_like(u, k(c["P1"])))
    Q = fma(u, Q, np.full_like(u, k(c["Q1"])))
    P = fma(u, P, np.full_like(u, f32(1.0)))
    Q = fma(u, Q, np.full_like(u, f32(0.5)))
    s = (phi.astype(np.float64) * P.astype(np.float64)).astype(f32)
    g = (u.astype(np.float64) * Q.astype(np.float64)).astype(f32)
    x = phi.astype(np.float64)
    s_true = np.sin(x)
    g_true = 2.0 * np.sin(x / 2) ** 2
    # relative errors where the exact results are FP32 normal numbers; below that
    # (phi^2 / 2 under 2^-126) the FP32 result may flush to zero
    tiny = np.finfo(np.float32).tiny
    ns = np.abs(s_true) >= tiny
    ng = g_true >= tiny
    assert np.all(s[phi == 0] == 0) and np.all(g[phi == 0] == 0)
    assert np.all(np.abs(g[~ng]) <= tiny)
    assert np.max(np.abs(s[ns] - s_true[ns]) / np.abs(s_true[ns])) < 1.5e-7
    assert np.max(np.abs(g[ng] - g_true[ng]) / g_true[ng]) < 1.5e-7
