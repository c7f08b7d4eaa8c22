"""The 256^2 workload on the GPU against the stored values in tests/golden/
(written from the FP64 oracle): FP64 grids on both of their sequences to
FP64 rounding, FP32 grids on the fused path to FP32 rounding."""
import pytest

from paper_1208_2407_gb300 import workloads as wl

from golden_values import load, sites
from gpu_helpers import ensure_library, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


@pytest.mark.parametrize("dtype,path,K,rtol,atol", [
    ("f64", "plain", 0, 1e-12, 1e-15),
    ("f64", "fused", 0, 1e-12, 1e-15),      # ts_evolve: merged sweeps
    ("f32", "fused", 0, 2e-6, 2e-8),
    ("f32", "fused", 4, 2e-6, 2e-8),
    ("f32", "plain", 0, 2e-6, 2e-8),
])
def test_workload_matches_stored_values(dtype, path, K, rtol, atol):
    g = load("c1_plain_fp64_256.txt")
    c = wl.plain_fp64_256()
    (re, im), obs = run_gpu(c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"],
                            dtype=dtype, path=path, K=K, observe=True)
    for key in ("norm", "x", "y", "x2", "y2", "e_kin"):
        assert obs[key] == pytest.approx(g[key], rel=rtol, abs=atol), key
    assert obs["e_pot"] == 0.0
    for x, y in sites(g):
        assert abs(re[y, x] - g["re[%d,%d]" % (x, y)]) < atol + rtol * 0.03
        assert abs(im[y, x] - g["im[%d,%d]" % (x, y)]) < atol + rtol * 0.03
