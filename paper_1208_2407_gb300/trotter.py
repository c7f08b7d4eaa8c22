"""Python binding of libtrotter.so (include/trotter.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch supplies device
memory (the grid slab) and the current CUDA stream.  The module-level
functions carry the C names (``ts_create_grid``, ``ts_evolve``, ...) and take
raw pointers; :class:`Grid` wraps them for numpy/torch arrays.

If the library has not been built, the first call raises ``RuntimeError``:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtrotter.so")

TS_OK, TS_ERR_ARG, TS_ERR_OOM, TS_ERR_CUDA, TS_ERR_BUSY, TS_ERR_TIMEOUT, TS_ERR_STATE, \
    TS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
TS_F32, TS_F64 = 0, 1
TS_HOST, TS_DEVICE = 0, 1

STATUS_NAMES = {0: "TS_OK", -1: "TS_ERR_ARG", -2: "TS_ERR_OOM", -3: "TS_ERR_CUDA",
                -4: "TS_ERR_BUSY", -5: "TS_ERR_TIMEOUT", -6: "TS_ERR_STATE",
                -7: "TS_ERR_UNSUPPORTED"}


class TrotterError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class ts_layout(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("pitch", ctypes.c_int64),
                ("plane_bytes", ctypes.c_size_t), ("slab_bytes", ctypes.c_size_t),
                ("dtype", ctypes.c_int), ("nz", ctypes.c_int64)]


class ts_observables(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double)
                for n in ("norm", "x", "y", "x2", "y2", "e_kin", "e_pot", "z", "z2")]


class ts_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("K", ctypes.c_int), ("max_epoch_steps", ctypes.c_int)]


class ts_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double),
                ("V", ctypes.c_void_p), ("psi_re", ctypes.c_void_p), ("psi_im", ctypes.c_void_p),
                ("psi_dtype", ctypes.c_int), ("where", ctypes.c_int)]


class ts_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ns", ctypes.c_int64),
                ("queue_ns", ctypes.c_int64), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("steps", ctypes.c_int64)]


class ts_server_metrics(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("site_steps_per_s", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("epochs", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64)]


_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_DBL = ctypes.c_double

_SIGNATURES = {
    "ts_grid_layout": [_I64, _I64, _INT, ctypes.POINTER(ts_layout)],
    "ts_create_grid": [_I64, _I64, _INT, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)],
    "ts_grid_layout3": [_I64, _I64, _I64, _INT, ctypes.POINTER(ts_layout)],
    "ts_create_grid3": [_I64, _I64, _I64, _INT, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)],
    "ts_destroy_grid": [_VP],
    "ts_grid_info": [_VP, ctypes.POINTER(ts_layout), ctypes.POINTER(_VP), ctypes.POINTER(_VP)],
    "ts_set_state": [_VP, _VP, _VP, _INT, _INT, _VP],
    "ts_get_state": [_VP, _VP, _VP, _INT, _INT, _VP],
    "ts_set_potential": [_VP, _VP, _INT, _DBL, _DBL, _VP],
    "ts_set_potential_order": [_VP, _VP, _INT, _DBL, _DBL, _INT, _VP],
    "ts_set_drive": [_VP, _VP, _INT, _VP, _I64, _VP],
    "ts_clear_drive": [_VP],
    "ts_evolve": [_VP, _I64, _INT, _VP],
    "ts_evolve_plain": [_VP, _I64, _VP],
    "ts_check_wait_timeout": [_VP, _I64, _VP],
    "ts_observe": [_VP, ctypes.POINTER(ts_observables), _VP],
    "ts_norm": [_VP, ctypes.POINTER(_DBL), _VP],
    "ts_expect_xy": [_VP, ctypes.POINTER(_DBL), ctypes.POINTER(_DBL), _VP],
    "ts_energy": [_VP, ctypes.POINTER(_DBL), _VP],
    "ts_evolve_batched": [ctypes.POINTER(_VP), _INT, ctypes.POINTER(_I64), _INT, _VP],
    "ts_norm_noalloc": [_VP, _VP, _INT, _I64, _I64, _I64, _VP, _VP],
    "ts_adjoint_workspace": [_VP, _I64, _I64, ctypes.POINTER(ctypes.c_size_t)],
    "ts_adjoint_forward": [_VP, _VP, _VP, _INT, _INT, _I64, _I64, _VP, ctypes.c_size_t,
                           ctypes.POINTER(_DBL), ctypes.POINTER(_DBL), _VP],
    "ts_adjoint_backward": [_VP, _VP, ctypes.c_size_t, _VP, _VP],
    "ts_adjoint_backward_depth": [_VP, _VP, ctypes.c_size_t, _INT, _VP, _VP],
    "ts_adjoint_grad": [_VP, _VP, _VP, _INT, _INT, _I64, _I64, _VP, ctypes.c_size_t, _VP,
                        ctypes.POINTER(_DBL), _VP],
    "ts_server_create": [ctypes.POINTER(ts_server_cfg), ctypes.POINTER(_VP)],
    "ts_server_submit": [_VP, ctypes.POINTER(ts_request), ctypes.POINTER(ctypes.c_uint64)],
    "ts_server_poll": [_VP, ctypes.c_uint64, ctypes.POINTER(ts_result)],
    "ts_server_wait": [_VP, ctypes.c_uint64, _I64, ctypes.POINTER(ts_result)],
    "ts_server_fetch": [_VP, ctypes.c_uint64, _VP, _VP, _INT, _INT],
    "ts_server_release": [_VP, ctypes.c_uint64],
    "ts_server_cancel": [_VP, ctypes.c_uint64],
    "ts_server_stats": [_VP, ctypes.POINTER(ts_server_metrics)],
    "ts_server_destroy": [_VP],
}

_lock = threading.Lock()
_lib = None


def load():
    """Load libtrotter.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtrotter.so is not built (%s); run "
                               "`python -m paper_1208_2407_gb300.build`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _INT
        lib.ts_last_error.argtypes = []
        lib.ts_last_error.restype = ctypes.c_char_p
        lib.ts_launch_count.argtypes = [_INT]
        lib.ts_launch_count.restype = _I64
        lib.ts_fused_default_depth.argtypes = []
        lib.ts_fused_default_depth.restype = _INT
        lib.ts_norm_noalloc_scratch_bytes.argtypes = []
        lib.ts_norm_noalloc_scratch_bytes.restype = ctypes.c_size_t
        _lib = lib
        return lib


def exported_symbols():
    """Names the header declares, for the ABI test."""
    return sorted(list(_SIGNATURES) + ["ts_last_error", "ts_launch_count",
                                        "ts_norm_noalloc_scratch_bytes",
                                        "ts_fused_default_depth"])


def _check(status: int):
    if status != TS_OK:
        raise TrotterError(status, load().ts_last_error().decode(errors="replace"))


def _call(name, *args):
    _check(getattr(load(), name)(*args))


# --- C-named wrappers (raw pointers / handles) ------------------------------
def ts_grid_layout(nx: int, ny: int, dtype: int = TS_F32) -> ts_layout:
    L = ts_layout()
    _call("ts_grid_layout", nx, ny, dtype, ctypes.byref(L))
    return L


def ts_create_grid(nx, ny, dtype, slab_ptr, slab_bytes):
    h = _VP()
    _call("ts_create_grid", nx, ny, dtype, slab_ptr, slab_bytes, ctypes.byref(h))
    return h


def ts_grid_layout3(nx: int, ny: int, nz: int, dtype: int = TS_F32) -> ts_layout:
    L = ts_layout()
    _call("ts_grid_layout3", nx, ny, nz, dtype, ctypes.byref(L))
    return L


def ts_create_grid3(nx, ny, nz, dtype, slab_ptr, slab_bytes):
    h = _VP()
    _call("ts_create_grid3", nx, ny, nz, dtype, slab_ptr, slab_bytes, ctypes.byref(h))
    return h


def ts_destroy_grid(h):
    _call("ts_destroy_grid", h)


def ts_set_state(h, re_ptr, im_ptr, dtype, where, stream):
    _call("ts_set_state", h, re_ptr, im_ptr, dtype, where, stream)


def ts_get_state(h, re_ptr, im_ptr, dtype, where, stream):
    _call("ts_get_state", h, re_ptr, im_ptr, dtype, where, stream)


def ts_set_potential(h, v_ptr, where, dt, theta, stream):
    _call("ts_set_potential", h, v_ptr, where, dt, theta, stream)


def ts_evolve(h, steps, K, stream):
    _call("ts_evolve", h, steps, K, stream)


def ts_set_potential_order(h, v_ptr, where, dt, theta, order, stream):
    _call("ts_set_potential_order", h, v_ptr, where, dt, theta, order, stream)


def ts_set_drive(h, v1_ptr, where, a_ptr, n_a, stream):
    _call("ts_set_drive", h, v1_ptr, where, a_ptr, n_a, stream)


def ts_clear_drive(h):
    _call("ts_clear_drive", h)


def ts_evolve_plain(h, steps, stream):
    _call("ts_evolve_plain", h, steps, stream)


def ts_check_wait_timeout(h, limit_ns, stream):
    _call("ts_check_wait_timeout", h, limit_ns, stream)


def ts_observe(h, stream) -> ts_observables:
    o = ts_observables()
    _call("ts_observe", h, ctypes.byref(o), stream)
    return o


def ts_norm(h, stream) -> float:
    v = _DBL()
    _call("ts_norm", h, ctypes.byref(v), stream)
    return v.value


def ts_expect_xy(h, stream):
    x, y = _DBL(), _DBL()
    _call("ts_expect_xy", h, ctypes.byref(x), ctypes.byref(y), stream)
    return x.value, y.value


def ts_energy(h, stream) -> float:
    v = _DBL()
    _call("ts_energy", h, ctypes.byref(v), stream)
    return v.value


def ts_evolve_batched(handles, steps, K, stream):
    n = len(handles)
    arr = (_VP * n)(*[h.value if isinstance(h, _VP) else h for h in handles])
    st = (_I64 * n)(*[int(s) for s in steps])
    _call("ts_evolve_batched", arr, n, st, K, stream)


def ts_adjoint_workspace(h, steps, ckpt_every) -> int:
    n = ctypes.c_size_t()
    _call("ts_adjoint_workspace", h, steps, ckpt_every, ctypes.byref(n))
    return int(n.value)


def ts_adjoint_forward(h, tre_ptr, tim_ptr, dtype, where, steps, ckpt_every, ws_ptr, ws_bytes,
                       stream):
    F = _DBL()
    ov = (_DBL * 2)()
    _call("ts_adjoint_forward", h, tre_ptr, tim_ptr, dtype, where, steps, ckpt_every, ws_ptr,
          ws_bytes, ctypes.byref(F), ov, stream)
    return F.value, complex(ov[0], ov[1])


def ts_adjoint_backward(h, ws_ptr, ws_bytes, grad_ptr, stream):
    _call("ts_adjoint_backward", h, ws_ptr, ws_bytes, grad_ptr, stream)


def ts_adjoint_backward_depth(h, ws_ptr, ws_bytes, K, grad_ptr, stream):
    _call("ts_adjoint_backward_depth", h, ws_ptr, ws_bytes, K, grad_ptr, stream)


def ts_adjoint_grad(h, tre_ptr, tim_ptr, dtype, where, steps, ckpt_every, ws_ptr, ws_bytes,
                    grad_ptr, stream) -> float:
    F = _DBL()
    _call("ts_adjoint_grad", h, tre_ptr, tim_ptr, dtype, where, steps, ckpt_every, ws_ptr,
          ws_bytes, grad_ptr, ctypes.byref(F), stream)
    return F.value


def ts_norm_noalloc(re_ptr, im_ptr, dtype, nx, ny, pitch, out_ptr, stream):
    """Norm of a pitched device state into a caller-owned device double,
    using the library's fixed scratch instead of any allocation."""
    _call("ts_norm_noalloc", re_ptr, im_ptr, dtype, nx, ny, pitch, out_ptr, stream)


def ts_norm_noalloc_scratch_bytes() -> int:
    return int(load().ts_norm_noalloc_scratch_bytes())


def ts_fused_default_depth() -> int:
    return int(load().ts_fused_default_depth())


def ts_launch_count(reset: bool = False) -> int:
    return int(load().ts_launch_count(1 if reset else 0))


def ts_last_error() -> str:
    return load().ts_last_error().decode(errors="replace")


# --- torch-facing convenience ----------------------------------------------
def _torch():
    import torch
    return torch


def current_stream_ptr():
    torch = _torch()
    return _VP(torch.cuda.current_stream().cuda_stream)


def _dtype_code(dt) -> int:
    name = str(dt)
    if name.endswith("float64") or name in ("f64", "double"):
        return TS_F64
    if name.endswith("float32") or name in ("f32", "float"):
        return TS_F32
    raise ValueError("unsupported dtype %r" % (dt,))


def _array_ptr(a, shape):
    """(pointer, dtype code, where) for a numpy array or a torch tensor."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if tuple(a.shape) != shape or not a.is_contiguous():
            raise ValueError("expected a contiguous tensor of shape %s" % (shape,))
        where = TS_DEVICE if a.is_cuda else TS_HOST
        return _VP(a.data_ptr()), _dtype_code(a.dtype), where, a
    arr = np.ascontiguousarray(a)
    if arr.dtype not in (np.float32, np.float64):
        arr = arr.astype(np.float64)
    if arr.shape != shape:
        raise ValueError("expected an array of shape %s, got %s" % (shape, arr.shape))
    return _VP(arr.ctypes.data), _dtype_code(arr.dtype), TS_HOST, arr


class Grid:
    """One lattice on the current CUDA device, with its slab owned by torch.
    nz > 1 makes a 3-D lattice; its arrays have shape (nz, ny, nx)."""

    def __init__(self, nx: int, ny: int, dtype: str = "f32", nz: int = 1):
        torch = _torch()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dtype = TS_F64 if dtype in ("f64", "float64", np.float64) else TS_F32
        self.layout = ts_grid_layout3(self.nx, self.ny, self.nz, self.dtype)
        self.slab = torch.empty(int(self.layout.slab_bytes), dtype=torch.uint8, device="cuda")
        self.handle = ts_create_grid3(self.nx, self.ny, self.nz, self.dtype,
                                      _VP(self.slab.data_ptr()), int(self.layout.slab_bytes))

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.nz > 1 else (self.ny, self.nx)

    def close(self):
        if self.handle is not None:
            ts_destroy_grid(self.handle)
            self.handle = None
            self.slab = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, re, im, stream=None):
        rp, rd, rw, keep_r = _array_ptr(re, self.shape)
        ip, idt, iw, keep_i = _array_ptr(im, self.shape)
        if (rd, rw) != (idt, iw):
            raise ValueError("re and im must share dtype and memory kind")
        ts_set_state(self.handle, rp, ip, rd, rw, stream or current_stream_ptr())
        del keep_r, keep_i

    def get_state(self, dtype=np.float64, device: bool = False, stream=None):
        torch = _torch()
        code = _dtype_code(np.dtype(dtype))
        if device:
            tdt = torch.float64 if code == TS_F64 else torch.float32
            re = torch.empty(self.shape, dtype=tdt, device="cuda")
            im = torch.empty(self.shape, dtype=tdt, device="cuda")
            ts_get_state(self.handle, _VP(re.data_ptr()), _VP(im.data_ptr()), code, TS_DEVICE,
                         stream or current_stream_ptr())
            return re, im
        re = np.empty(self.shape, dtype=np.float64 if code == TS_F64 else np.float32)
        im = np.empty_like(re)
        ts_get_state(self.handle, _VP(re.ctypes.data), _VP(im.ctypes.data), code, TS_HOST,
                     stream or current_stream_ptr())
        return re, im

    def set_potential(self, V, dt: float, theta: float, stream=None, order: int = 2):
        """Phase table and kinetic coefficients for steps of length dt
        (order 2: U2(dt); order 4: the fourth-order Suzuki step U4(dt))."""
        st = stream or current_stream_ptr()
        args = (float(dt), float(theta), int(order), st)
        if V is None:
            ts_set_potential_order(self.handle, None, TS_HOST, *args)
            return
        torch = _torch()
        if isinstance(V, torch.Tensor):
            if V.dtype != torch.float64 or tuple(V.shape) != self.shape or not V.is_contiguous():
                raise ValueError("V must be a contiguous float64 tensor of the grid's shape")
            where = TS_DEVICE if V.is_cuda else TS_HOST
            ts_set_potential_order(self.handle, _VP(V.data_ptr()), where, *args)
            return
        Va = np.ascontiguousarray(V, dtype=np.float64)
        if Va.shape != self.shape:
            raise ValueError("V must have the grid's shape")
        ts_set_potential_order(self.handle, _VP(Va.ctypes.data), TS_HOST, *args)

    def set_drive(self, V1, a, stream=None):
        """Time-dependent potential V0 + a[n] V1 for the next len(a) steps
        (V0, dt, theta from set_potential, which must come first)."""
        st = stream or current_stream_ptr()
        av = np.ascontiguousarray(np.ravel(a), dtype=np.float64)
        ap = _VP(av.ctypes.data)
        if V1 is None:
            ts_set_drive(self.handle, None, TS_HOST, ap, av.size, st)
            return
        torch = _torch()
        if isinstance(V1, torch.Tensor):
            if V1.dtype != torch.float64 or tuple(V1.shape) != self.shape or not V1.is_contiguous():
                raise ValueError("V1 must be a contiguous float64 tensor of the grid's shape")
            where = TS_DEVICE if V1.is_cuda else TS_HOST
            ts_set_drive(self.handle, _VP(V1.data_ptr()), where, ap, av.size, st)
            return
        V1a = np.ascontiguousarray(V1, dtype=np.float64)
        if V1a.shape != self.shape:
            raise ValueError("V1 must have the grid's shape")
        ts_set_drive(self.handle, _VP(V1a.ctypes.data), TS_HOST, ap, av.size, st)

    def clear_drive(self):
        ts_clear_drive(self.handle)

    def evolve(self, steps: int, K: int = 0, stream=None):
        """`steps` steps (ts_evolve).  FP32 grids: the fused kernel at depth K
        (0: the library's default).  FP64 grids: one sweep per launch with
        the sweeps merged where steps meet (K must be 0).  Async."""
        ts_evolve(self.handle, int(steps), int(K), stream or current_stream_ptr())

    def evolve_plain(self, steps: int, stream=None):
        """`steps` steps one sweep per launch, the literal sequence
        (ts_evolve_plain): the reference point the other paths are measured
        against.  Async."""
        ts_evolve_plain(self.handle, int(steps), stream or current_stream_ptr())

    def observe(self, stream=None) -> dict:
        o = ts_observe(self.handle, stream or current_stream_ptr())
        return {n: getattr(o, n) for n, _ in ts_observables._fields_}

    def norm(self, stream=None) -> float:
        return ts_norm(self.handle, stream or current_stream_ptr())

    def expect_xy(self, stream=None):
        return ts_expect_xy(self.handle, stream or current_stream_ptr())

    def energy(self, stream=None) -> float:
        return ts_energy(self.handle, stream or current_stream_ptr())

    def state_planes(self):
        """Device pointers of the current re/im planes and the row pitch."""
        L = ts_layout()
        re, im = _VP(), _VP()
        _call("ts_grid_info", self.handle, ctypes.byref(L), ctypes.byref(re), ctypes.byref(im))
        return re.value, im.value, int(L.pitch)


def adjoint_fidelity_grad(grid, target_re, target_im, steps: int, ckpt_every: int = 50,
                          stream=None, K: int = 0):
    """(F, dF/dV) for the grid's current state and potential; the grid ends at
    psi_T.  dF/dV is returned as an (ny, nx) float32 CUDA tensor.  K is the
    fused depth of the backward pass's launches (0: the library default)."""
    torch = _torch()
    st = stream or current_stream_ptr()
    tp, tdt, tw, keep_t = _array_ptr(target_re, grid.shape)
    ip, idt, iw, keep_i = _array_ptr(target_im, grid.shape)
    nbytes = ts_adjoint_workspace(grid.handle, int(steps), int(ckpt_every))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    grad = torch.empty(grid.shape, dtype=torch.float32, device="cuda")
    if K == 0:
        F = ts_adjoint_grad(grid.handle, tp, ip, tdt, tw, int(steps), int(ckpt_every),
                            _VP(ws.data_ptr()), nbytes, _VP(grad.data_ptr()), st)
    else:
        F, _ = ts_adjoint_forward(grid.handle, tp, ip, tdt, tw, int(steps), int(ckpt_every),
                                  _VP(ws.data_ptr()), nbytes, st)
        ts_adjoint_backward_depth(grid.handle, _VP(ws.data_ptr()), nbytes, int(K),
                                  _VP(grad.data_ptr()), st)
    del keep_t, keep_i
    return F, grad


class Server:
    """The library's continuous-batching request loop (ts_server_*).

    ``submit`` keeps references to the request's input arrays until the
    request is released, as the C ABI requires them to stay valid."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, K: int = 0,
                 max_epoch_steps: int = 0):
        cfg = ts_server_cfg(int(hbm_budget_bytes), int(max_slots), int(K), int(max_epoch_steps))
        self.handle = _VP()
        _call("ts_server_create", ctypes.byref(cfg), ctypes.byref(self.handle))
        self._keep = {}

    def submit(self, nx, ny, steps, dt, theta, V, psi_re, psi_im) -> int:
        """Host numpy / torch arrays or CUDA tensors; V may be None."""
        shape = (int(ny), int(nx))
        rp, rdt, rw, k1 = _array_ptr(psi_re, shape)
        ip, idt, iw, k2 = _array_ptr(psi_im, shape)
        if (rdt, rw) != (idt, iw):
            raise ValueError("psi_re and psi_im must share dtype and memory kind")
        vp, k3 = None, None
        if V is not None:
            vp, vdt, vw, k3 = _array_ptr(V, shape)
            if vdt != TS_F64 or vw != rw:
                raise ValueError("V must be float64 in the same memory kind as psi")
        req = ts_request(int(nx), int(ny), int(steps), float(dt), float(theta), vp, rp, ip, rdt, rw)
        t = ctypes.c_uint64()
        _call("ts_server_submit", self.handle, ctypes.byref(req), ctypes.byref(t))
        self._keep[t.value] = (k1, k2, k3)
        return t.value

    def poll(self, ticket) -> ts_result:
        r = ts_result()
        _call("ts_server_poll", self.handle, ticket, ctypes.byref(r))
        return r

    def wait(self, ticket, timeout_ms: int = -1) -> ts_result:
        r = ts_result()
        _call("ts_server_wait", self.handle, ticket, int(timeout_ms), ctypes.byref(r))
        return r

    def fetch(self, ticket, ny, nx, dtype=np.float64):
        code = _dtype_code(np.dtype(dtype))
        re = np.empty((ny, nx), dtype=np.float64 if code == TS_F64 else np.float32)
        im = np.empty_like(re)
        _call("ts_server_fetch", self.handle, ticket, _VP(re.ctypes.data), _VP(im.ctypes.data),
              code, TS_HOST)
        return re, im

    def release(self, ticket):
        _call("ts_server_release", self.handle, ticket)
        self._keep.pop(ticket, None)

    def cancel(self, ticket):
        _call("ts_server_cancel", self.handle, ticket)

    def stats(self) -> dict:
        m = ts_server_metrics()
        _call("ts_server_stats", self.handle, ctypes.byref(m))
        return {n: getattr(m, n) for n, _ in ts_server_metrics._fields_}

    def close(self):
        if self.handle is not None and self.handle.value:
            _call("ts_server_destroy", self.handle)
        self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def evolve_batched(grids, steps, K: int = 0, stream=None):
    ts_evolve_batched([g.handle for g in grids], steps, K, stream or current_stream_ptr())
