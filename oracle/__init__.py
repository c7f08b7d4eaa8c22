"""FP64 CPU oracle for the second-order Trotter-Suzuki step (paper Sec. 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_1208_2407_gb300``) never imports it, and it never imports
the product path: the two share no code.

The arithmetic lives in ``trotter_oracle.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``); this module compiles it on first use and wraps it
with ctypes.  Every function takes and returns dense row-major numpy arrays of
shape (ny, nx): site (x, y) is ``a[y, x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trotter_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_trotter_oracle.so")
_lock = threading.Lock()
_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(lib):
    """Declare the C signatures on a loaded oracle library (the built one or,
    in the planted-mistake tests, a mutant compiled from edited source)."""
    sig = {
        "oracle_sweep_x": [_I64, _I64, _DP, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int],
        "oracle_sweep_y": [_I64, _I64, _DP, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int],
        "oracle_phase": [_I64, _I64, _DP, _DP, _DP, ctypes.c_double, ctypes.c_int],
        "oracle_step2": [_I64, _I64, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double, ctypes.c_int],
        "oracle_evolve": [_I64, _I64, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double, _I64,
                          ctypes.c_int, ctypes.c_int],
        "oracle_evolve_driven": [_I64, _I64, _DP, _DP, _DP, _DP, _DP, ctypes.c_double,
                                 ctypes.c_double, _I64, ctypes.c_int],
        "oracle_moments": [_I64, _I64, _DP, _DP, _DP],
        "oracle_sweep3": [_I64, _I64, _I64, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                          ctypes.c_int],
        "oracle_evolve3": [_I64, _I64, _I64, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double,
                           _I64, ctypes.c_int],
        "oracle_moments3": [_I64, _I64, _I64, _DP, _DP, _DP],
        "oracle_energy3": [_I64, _I64, _I64, _DP, _DP, _DP, ctypes.c_double, _DP],
        "oracle_energy": [_I64, _I64, _DP, _DP, _DP, ctypes.c_double, _DP],
        "oracle_inner": [_I64, _DP, _DP, _DP, _DP, _DP],
        "oracle_adjoint_grad": [_I64, _I64, _DP, _DP, _DP, _DP, _DP, ctypes.c_double,
                                ctypes.c_double, _I64, _DP, _DP, _DP, ctypes.c_int],
        "oracle_compensated_sum": [_I64, _DP],
    }
    for name, args in sig.items():
        getattr(lib, name).argtypes = args
    for name in ("oracle_evolve", "oracle_evolve_driven", "oracle_evolve3", "oracle_adjoint_grad"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("oracle_sweep_x", "oracle_sweep_y", "oracle_phase", "oracle_step2",
                 "oracle_moments", "oracle_energy", "oracle_inner",
                 "oracle_sweep3", "oracle_moments3", "oracle_energy3"):
        getattr(lib, name).restype = None
    lib.oracle_compensated_sum.restype = ctypes.c_double
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
        return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _state(re, im):
    re = np.array(re, dtype=np.float64, order="C", copy=True)
    im = np.array(im, dtype=np.float64, order="C", copy=True)
    if re.shape != im.shape or re.ndim != 2:
        raise ValueError("re and im must be 2-D arrays of equal shape (ny, nx)")
    return re, im


def sweep(re, im, axis: str, parity: int, theta: float, nthreads: int = 1):
    """One sweep of pair rotations along ``axis`` ('x' or 'y') (Sec. 2, matrix M)."""
    lib = _load()
    re, im = _state(re, im)
    ny, nx = re.shape
    fn = lib.oracle_sweep_x if axis == "x" else lib.oracle_sweep_y
    fn(nx, ny, _ptr(re), _ptr(im), int(parity), float(theta), int(nthreads))
    return re, im


def phase(re, im, V, dt: float, nthreads: int = 1):
    """Diagonal factor exp(-i V dt) (Sec. 2, the external potential)."""
    lib = _load()
    re, im = _state(re, im)
    ny, nx = re.shape
    Vc = None if V is None else _f64(V)
    lib.oracle_phase(nx, ny, _ptr(re), _ptr(im), _ptr(Vc), float(dt), int(nthreads))
    return re, im


def evolve(re, im, V, dt: float, theta: float, steps: int, order: int = 2,
           nthreads: int = 1):
    """``steps`` Trotter steps of order 1, 2 (Eq. secondorder) or 4 (Eq. fourthorder)."""
    lib = _load()
    re, im = _state(re, im)
    ny, nx = re.shape
    Vc = None if V is None else _f64(V)
    if Vc is not None and Vc.shape != re.shape:
        raise ValueError("V must have the state's shape")
    rc = lib.oracle_evolve(nx, ny, _ptr(re), _ptr(im), _ptr(Vc), float(dt), float(theta),
                           int(steps), int(order), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_evolve rejected its arguments (rc=%d)" % rc)
    return re, im


def evolve_driven(re, im, V0, V1, a, dt: float, theta: float, nthreads: int = 1):
    """len(a) second-order steps with the potential V0 + a[n] V1 in step n
    (the time-dependent extension of Sec. 2; a sampled at step midpoints)."""
    lib = _load()
    re, im = _state(re, im)
    ny, nx = re.shape
    V0c = None if V0 is None else _f64(V0)
    V1c = None if V1 is None else _f64(V1)
    for v in (V0c, V1c):
        if v is not None and v.shape != re.shape:
            raise ValueError("V0 and V1 must have the state's shape")
    ac = _f64(np.ravel(a))
    rc = lib.oracle_evolve_driven(nx, ny, _ptr(re), _ptr(im), _ptr(V0c), _ptr(V1c), _ptr(ac),
                                  float(dt), float(theta), int(ac.size), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_evolve_driven rejected its arguments (rc=%d)" % rc)
    return re, im


def _state3(re, im):
    re = np.array(re, dtype=np.float64, order="C", copy=True)
    im = np.array(im, dtype=np.float64, order="C", copy=True)
    if re.shape != im.shape or re.ndim != 3:
        raise ValueError("re and im must be 3-D arrays of equal shape (nz, ny, nx)")
    return re, im


def sweep3(re, im, axis: int, parity: int, theta: float, nthreads: int = 1):
    """One 3-D sweep along axis 0 (x), 1 (y) or 2 (z); arrays (nz, ny, nx)."""
    lib = _load()
    re, im = _state3(re, im)
    nz, ny, nx = re.shape
    lib.oracle_sweep3(nx, ny, nz, _ptr(re), _ptr(im), int(axis), int(parity), float(theta),
                      int(nthreads))
    return re, im


def evolve3(re, im, V, dt: float, theta: float, steps: int, nthreads: int = 1):
    """``steps`` second-order steps on the 3-D lattice; arrays (nz, ny, nx)."""
    lib = _load()
    re, im = _state3(re, im)
    nz, ny, nx = re.shape
    Vc = None if V is None else _f64(V)
    if Vc is not None and Vc.shape != re.shape:
        raise ValueError("V must have the state's shape")
    rc = lib.oracle_evolve3(nx, ny, nz, _ptr(re), _ptr(im), _ptr(Vc), float(dt), float(theta),
                            int(steps), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_evolve3 rejected its arguments (rc=%d)" % rc)
    return re, im


def moments3(re, im):
    """(sum|psi|^2, sum x.., sum y.., sum z.., sum x^2.., sum y^2.., sum z^2..)."""
    lib = _load()
    re, im = _f64(re), _f64(im)
    nz, ny, nx = re.shape
    out = np.zeros(7)
    lib.oracle_moments3(nx, ny, nz, _ptr(re), _ptr(im), _ptr(out))
    return out


def energy3(re, im, V, J: float = 1.0):
    lib = _load()
    re, im = _f64(re), _f64(im)
    nz, ny, nx = re.shape
    Vc = None if V is None else _f64(V)
    out = np.zeros(2)
    lib.oracle_energy3(nx, ny, nz, _ptr(re), _ptr(im), _ptr(Vc), float(J), _ptr(out))
    return float(out[0]), float(out[1])


def moments(re, im):
    """(sum|psi|^2, sum x|psi|^2, sum y|psi|^2, sum x^2|psi|^2, sum y^2|psi|^2)."""
    lib = _load()
    re, im = _f64(re), _f64(im)
    ny, nx = re.shape
    out = np.zeros(5)
    lib.oracle_moments(nx, ny, _ptr(re), _ptr(im), _ptr(out))
    return out


def norm(re, im) -> float:
    return float(moments(re, im)[0])


def expect_xy(re, im):
    m = moments(re, im)
    return float(m[1] / m[0]), float(m[2] / m[0])


def energy(re, im, V, J: float = 1.0):
    """<psi|H|psi> split as (kinetic, potential); H = -J * hops + diag(V)."""
    lib = _load()
    re, im = _f64(re), _f64(im)
    ny, nx = re.shape
    Vc = None if V is None else _f64(V)
    out = np.zeros(2)
    lib.oracle_energy(nx, ny, _ptr(re), _ptr(im), _ptr(Vc), float(J), _ptr(out))
    return float(out[0]), float(out[1])


def inner(are, aim, bre, bim) -> complex:
    """<a|b> = sum conj(a) b."""
    lib = _load()
    are, aim, bre, bim = (_f64(a) for a in (are, aim, bre, bim))
    out = np.zeros(2)
    lib.oracle_inner(are.size, _ptr(are), _ptr(aim), _ptr(bre), _ptr(bim), _ptr(out))
    return complex(out[0], out[1])


def adjoint_grad(psi0_re, psi0_im, phi_re, phi_im, V, dt: float, theta: float,
                 steps: int, nthreads: int = 1):
    """dF/dV for F = |<phi|U2(dt)^steps psi0>|^2.  Returns (grad, F, overlap)."""
    lib = _load()
    p_re, p_im, f_re, f_im = (_f64(a) for a in (psi0_re, psi0_im, phi_re, phi_im))
    ny, nx = p_re.shape
    Vc = None if V is None else _f64(V)
    grad = np.zeros((ny, nx))
    fid = np.zeros(1)
    ov = np.zeros(2)
    rc = lib.oracle_adjoint_grad(nx, ny, _ptr(p_re), _ptr(p_im), _ptr(f_re), _ptr(f_im),
                                 _ptr(Vc), float(dt), float(theta), int(steps), _ptr(grad),
                                 _ptr(fid), _ptr(ov), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_adjoint_grad failed (rc=%d)" % rc)
    return grad, float(fid[0]), complex(ov[0], ov[1])


def compensated_sum(v) -> float:
    lib = _load()
    v = _f64(np.ravel(v))
    return float(lib.oracle_compensated_sum(v.size, _ptr(v)))
