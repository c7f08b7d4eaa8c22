"""The stored values of the 256^2 FP64 workload (tests/golden/, written by
tests/golden/make_golden.py from the oracle) against the oracle as it is now
and against what the mathematics fixes for them: the exact lattice drift of
a free packet, the symmetry in y, the norm and the packet's energy."""
import math

import numpy as np
import pytest

import oracle
from paper_1208_2407_gb300 import workloads as wl

from golden_values import load, sites

C1 = "c1_plain_fp64_256.txt"


def test_oracle_reproduces_the_stored_values():
    g = load(C1)
    c = wl.plain_fp64_256()
    re, im = oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    m = oracle.moments(re, im)
    kin, pot = oracle.energy(re, im, np.zeros_like(re))
    for key, val in (("norm", m[0]), ("x", m[1] / m[0]), ("y", m[2] / m[0]),
                     ("x2", m[3] / m[0]), ("y2", m[4] / m[0]), ("e_kin", kin), ("e_pot", pot)):
        assert val == pytest.approx(g[key], rel=1e-13, abs=1e-15), key
    for x, y in sites(g):
        assert abs(re[y, x] - g["re[%d,%d]" % (x, y)]) < 1e-15
        assert abs(im[y, x] - g["im[%d,%d]" % (x, y)]) < 1e-15


def test_stored_values_agree_with_closed_forms():
    g = load(C1)
    J, t, sigma, k = 1.0, 100 * 0.05, 16.0, 0.5
    damp = math.exp(-1.0 / (8.0 * sigma * sigma))          # exp(-sigma_k^2 / 2)
    # exact lattice drift of the packet centre (the Trotter error is O(dt^2))
    assert abs(g["x"] - (128.0 + 2.0 * J * t * math.sin(k) * damp)) < 5e-3
    assert abs(g["y"] - 128.0) < 1e-10                     # ky = 0: no drift in y
    assert abs(g["norm"] - 1.0) < 1e-12
    assert g["e_pot"] == 0.0
    # energy of the packet: -2J (cos kx + cos ky) exp(-sigma_k^2 / 2)
    assert abs(g["e_kin"] - (-2.0 * J * (math.cos(k) + 1.0) * damp)) < 1e-3
