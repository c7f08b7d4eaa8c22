"""The C-ABI library builds, loads and exports every symbol include/trotter.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trotter.h")


def declared_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1208_2407_gb300 import build
    build.build()
    from paper_1208_2407_gb300 import trotter
    return trotter.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ts_create_grid", "ts_set_potential", "ts_evolve", "ts_norm",
                     "ts_evolve_batched", "ts_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1208_2407_gb300 import trotter
    assert set(declared_functions()) <= set(trotter.exported_symbols())


def test_layout_and_argument_errors_without_gpu(lib):
    from paper_1208_2407_gb300 import trotter
    L = trotter.ts_grid_layout(130, 66, trotter.TS_F32)
    assert L.pitch == 160 and L.pitch % 32 == 0
    assert L.plane_bytes % 256 == 0 and L.plane_bytes >= 160 * 66 * 4
    assert L.slab_bytes >= 7 * L.plane_bytes
    L64 = trotter.ts_grid_layout(130, 66, trotter.TS_F64)
    assert L64.plane_bytes >= 160 * 66 * 8
    for bad in ((0, 5), (5, 0), (-1, 3), (1 << 21, 2)):
        with pytest.raises(trotter.TrotterError) as e:
            trotter.ts_grid_layout(*bad, trotter.TS_F32)
        assert e.value.status == trotter.TS_ERR_ARG
    with pytest.raises(trotter.TrotterError) as e:
        trotter.ts_grid_layout(4, 4, 7)
    assert e.value.status == trotter.TS_ERR_ARG
    # null handles are rejected on the host, before any CUDA call
    for fn, args in ((lib.ts_evolve, (None, 1, 0, None)),
                     (lib.ts_evolve_plain, (None, 1, None)),
                     (lib.ts_set_potential, (None, None, 0, 0.05, 0.025, None))):
        assert fn(*args) == trotter.TS_ERR_ARG
    assert lib.ts_destroy_grid(None) == trotter.TS_OK
    out = ctypes.c_double()
    assert lib.ts_norm(None, ctypes.byref(out), None) == trotter.TS_ERR_ARG
    assert "null" in trotter.ts_last_error()


def declared_arity(path=HEADER):
    """Parameter count of every ts_* function the header declares."""
    text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(ts_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_argument_counts_match_the_header():
    """ctypes passes arguments blindly: a count that drifts from the C
    declaration would pass garbage, so the binding's signature table must
    agree with the header for every function it binds."""
    from paper_1208_2407_gb300 import trotter
    arity = declared_arity()
    wrong = {name: (len(args), arity[name]) for name, args in trotter._SIGNATURES.items()
             if name in arity and len(args) != arity[name]}
    assert not wrong, wrong


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: with the library missing, every entry into the
    product path raises instead of computing anything."""
    from paper_1208_2407_gb300 import trotter
    monkeypatch.setattr(trotter, "_lib", None)
    monkeypatch.setattr(trotter, "LIB_PATH", str(tmp_path / "libtrotter.so"))
    with pytest.raises(RuntimeError, match="not built"):
        trotter.load()
    with pytest.raises(RuntimeError, match="not built"):
        trotter.ts_grid_layout(64, 64, trotter.TS_F32)
