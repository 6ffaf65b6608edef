"""Thin ctypes binding of ``liblbmhd.so`` (C ABI: include/lbmhd.h).

Every function here only marshals arguments: the lattice step, the
moments, the diagnostics and the state transfers all run in the CUDA
library.  The names follow the C ABI.  If the library has not been built
the first call raises; there is no fallback.

Fields are float64 numpy arrays of shape (ny, nx) (x fastest); device
fields are contiguous float64 CUDA torch tensors of the same shape.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbmhd.so")

ABI_VERSION = 1
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_dev": 2, "fp16_dev": 3, "ff": 4}
ERRORS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "EVERSION", -7: "ESTATE"}


class Params(ctypes.Structure):
    _fields_ = [("abi_version", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("tau_nu", ctypes.c_double), ("tau_eta", ctypes.c_double),
                ("C_S", ctypes.c_double), ("delta", ctypes.c_double),
                ("s5", ctypes.c_double), ("s6", ctypes.c_double),
                ("s7", ctypes.c_double), ("s8", ctypes.c_double),
                ("les", ctypes.c_int32), ("check_finite_every", ctypes.c_int32),
                ("fp16_scale", ctypes.c_double), ("stream", ctypes.c_void_p)]


DIAG_KEYS = ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y", "E_kin", "E_mag", "enstrophy",
             "cross_helicity", "divB_max", "divB_rms", "current_sq")


class Diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in DIAG_KEYS] + [("step", ctypes.c_int64)]


class LBMHDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was never built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            h, i, d, vp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            pp = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "lbmhd_params_default": (None, [ctypes.POINTER(Params)]),
                "lbmhd_create": (i, [i, i, ctypes.POINTER(Params), pp]),
                "lbmhd_init": (i, [h, vp, vp, vp, vp, vp]),
                "lbmhd_init_device": (i, [h, vp, vp, vp, vp, vp]),
                "lbmhd_step": (i, [h, i]),
                "lbmhd_moments": (i, [h, vp, vp, vp, vp, vp]),
                "lbmhd_moments_device": (i, [h, vp, vp, vp, vp, vp]),
                "lbmhd_diagnostics": (i, [h, ctypes.POINTER(Diag)]),
                "lbmhd_get_state": (i, [h, vp]),
                "lbmhd_set_state": (i, [h, vp]),
                "lbmhd_get_state_raw": (i, [h, vp, ctypes.c_size_t]),
                "lbmhd_set_state_raw": (i, [h, vp, ctypes.c_size_t]),
                "lbmhd_sync": (i, [h]),
                "lbmhd_copy_rows": (i, [h, i, h, i, i]),
                "lbmhd_step_rows": (i, [h, i, i]),
                "lbmhd3_create": (i, [i, i, i, ctypes.POINTER(Params), pp]),
                "lbmhd3_init": (i, [h, vp, vp, vp, vp, vp, vp, vp]),
                "lbmhd3_step": (i, [h, i]),
                "lbmhd3_moments": (i, [h, vp]),
                "lbmhd3_get_state": (i, [h, vp]),
                "lbmhd3_diagnostics": (i, [h, vp]),
                "lbmhd3_set_launch": (i, [h, i, i]),
                "lbmhd3_get_launch": (i, [h, ctypes.POINTER(i), ctypes.POINTER(i)]),
                "lbmhd3_sync": (i, [h]),
                "lbmhd3_debug": (i, [h, i]),
                "lbmhd3_step_count": (ctypes.c_int64, [h]),
                "lbmhd3_launch_count": (ctypes.c_int64, [h]),
                "lbmhd3_bytes_per_cell": (i, [i]),
                "lbmhd3_step_planes": (i, [h, i, i]),
                "lbmhd3_init_device": (i, [h, vp, vp, vp, vp, vp, vp, vp]),
                "lbmhd3_moments_device": (i, [h, vp, vp, vp, vp, vp, vp, vp]),
                "lbmhd3_set_state": (i, [h, vp]),
                "lbmhd3_get_state_raw": (i, [h, vp, ctypes.c_size_t]),
                "lbmhd3_set_state_raw": (i, [h, vp, ctypes.c_size_t]),
                "lbmhd3_step_commit": (i, [h]),
                "lbmhd3_pack_plane": (i, [h, i, ctypes.c_uint64, vp, vp]),
                "lbmhd3_unpack_plane": (i, [h, i, ctypes.c_uint64, vp, vp]),
                "lbmhd3_destroy": (None, [h]),
                "lbmhd_step_commit": (i, [h]),
                "lbmhd_pack_row": (i, [h, i, ctypes.c_uint, vp, vp]),
                "lbmhd_unpack_row": (i, [h, i, ctypes.c_uint, vp, vp]),
                "lbmhd_step_count": (ctypes.c_int64, [h]),
                "lbmhd_launch_count": (ctypes.c_int64, [h]),
                "lbmhd_bytes_per_cell": (i, [i]),
                "lbmhd_set_launch": (i, [h, i, i]),
                "lbmhd_get_launch": (i, [h, ctypes.POINTER(i), ctypes.POINTER(i)]),
                "lbmhd_diagnostics_noalloc": (i, [vp, i, i, i, ctypes.c_longlong, d, vp, vp]),
                "lbmhd_destroy": (None, [h]),
                "lbmhd_ff_eval": (i, [i, vp, vp, vp, ctypes.c_longlong]),
                "lbmhd_last_error": (ctypes.c_char_p, []),
                "lbmhd_adjoint_record": (i, [h, vp, vp, vp, vp, vp, i, i]),
                "lbmhd_adjoint_backward": (i, [h, vp, vp, vp, vp, vp,
                                                ctypes.POINTER(ctypes.c_double),
                                                vp, vp, vp, vp, vp]),
                "lbmhd_adjoint_release": (i, [h]),
                "lbmhd_batch_create": (i, [i, vp, vp, vp, vp, vp, ctypes.POINTER(Params), pp]),
                "lbmhd_batch_init": (i, [h, i, vp, vp, vp, vp, vp]),
                "lbmhd_batch_step": (i, [h, i]),
                "lbmhd_batch_moments": (i, [h, i, vp, vp, vp, vp, vp]),
                "lbmhd_batch_get_state": (i, [h, i, vp]),
                "lbmhd_batch_sync": (i, [h]),
                "lbmhd_batch_set_launch": (i, [h, i, i, i]),
                "lbmhd_batch_get_launch": (i, [h, ctypes.POINTER(i), ctypes.POINTER(i),
                                                ctypes.POINTER(i)]),
                "lbmhd_batch_autotune": (i, [h, ctypes.c_char_p, i,
                                              ctypes.POINTER(ctypes.c_double)]),
                "lbmhd_batch_step_count": (ctypes.c_int64, [h]),
                "lbmhd_batch_launch_count": (ctypes.c_int64, [h]),
                "lbmhd_batch_debug": (i, [h, i]),
                "lbmhd_batch_destroy": (None, [h]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(rc: int):
    if rc != 0:
        raise LBMHDError(rc, lib().lbmhd_last_error().decode())


def _host(a: np.ndarray, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _dev(t, shape):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and tuple(t.shape) == shape):
        raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")
    return ctypes.c_void_p(t.data_ptr())


def lbmhd_params_default(**overrides) -> Params:
    """Default parameters (lbmhd_params_default) with keyword overrides;
    ``precision`` may be a name from PRECISIONS, ``stream`` an int handle
    or a torch.cuda.Stream."""
    p = Params()
    lib().lbmhd_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream
        setattr(p, k, v)
    return p


class Handle:
    """An lbmhd_t* together with its lattice shape."""

    def __init__(self, ptr: int, nx: int, ny: int, params: Params):
        self.ptr = ctypes.c_void_p(ptr)
        self.nx, self.ny = nx, ny
        self.params = params

    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def precision(self) -> int:
        return int(self.params.precision)


def lbmhd_create(nx: int, ny: int, params: Params | None = None) -> Handle:
    params = params if params is not None else lbmhd_params_default()
    out = ctypes.c_void_p()
    _check(lib().lbmhd_create(int(nx), int(ny), ctypes.byref(params), ctypes.byref(out)))
    return Handle(out.value, nx, ny, params)


def lbmhd_init(h: Handle, rho, ux, uy, bx, by):
    arrs = [_host(a, h.shape) for a in (rho, ux, uy, bx, by)]
    _check(lib().lbmhd_init(h.ptr, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs]))


def lbmhd_init_device(h: Handle, rho, ux, uy, bx, by):
    _check(lib().lbmhd_init_device(h.ptr, *[_dev(t, h.shape) for t in (rho, ux, uy, bx, by)]))


def lbmhd_step(h: Handle, n: int = 1):
    _check(lib().lbmhd_step(h.ptr, int(n)))


def lbmhd_moments(h: Handle):
    out = [np.empty(h.shape) for _ in range(5)]
    _check(lib().lbmhd_moments(h.ptr, *[a.ctypes.data_as(ctypes.c_void_p) for a in out]))
    return tuple(out)


def lbmhd_moments_into(h: Handle, rho, ux, uy, bx, by):
    """lbmhd_moments into caller-provided float64 arrays (e.g. pinned)."""
    arrs = [rho, ux, uy, bx, by]
    for a in arrs:
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.shape != h.shape:
            raise ValueError(f"expected C-contiguous float64 arrays of shape {h.shape}")
    _check(lib().lbmhd_moments(h.ptr, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs]))


def lbmhd_moments_device(h: Handle, rho, ux, uy, bx, by):
    _check(lib().lbmhd_moments_device(h.ptr, *[_dev(t, h.shape) for t in (rho, ux, uy, bx, by)]))


def lbmhd_diagnostics(h: Handle) -> dict:
    d = Diag()
    _check(lib().lbmhd_diagnostics(h.ptr, ctypes.byref(d)))
    out = {k: getattr(d, k) for k in DIAG_KEYS}
    out["step"] = d.step
    return out


def lbmhd_get_state(h: Handle) -> np.ndarray:
    st = np.empty((19,) + h.shape)
    _check(lib().lbmhd_get_state(h.ptr, st.ctypes.data_as(ctypes.c_void_p)))
    return st


# numpy view of one stored value per format (FF: an FP32 (hi, lo) pair)
RAW_DTYPES = {0: (np.float64, ()), 1: (np.float32, ()), 2: (np.float32, ()),
              3: (np.float16, ()), 4: (np.float32, (2,))}


def lbmhd_get_state_raw(h: Handle) -> np.ndarray:
    """The stored state in its own format, shape (19, ny, nx) (FF: (19, ny,
    nx, 2)); see include/lbmhd.h."""
    dt, tail = RAW_DTYPES[h.precision]
    st = np.empty((19,) + h.shape + tail, dtype=dt)
    _check(lib().lbmhd_get_state_raw(h.ptr, st.ctypes.data_as(ctypes.c_void_p), st.nbytes))
    return st


def lbmhd_set_state_raw(h: Handle, state):
    dt, tail = RAW_DTYPES[h.precision]
    st = np.ascontiguousarray(state, dtype=dt)
    if st.shape != (19,) + h.shape + tail:
        raise ValueError(f"expected shape {(19,) + h.shape + tail}")
    _check(lib().lbmhd_set_state_raw(h.ptr, st.ctypes.data_as(ctypes.c_void_p), st.nbytes))


def lbmhd_set_state(h: Handle, state):
    st = _host(state, (19,) + h.shape)
    _check(lib().lbmhd_set_state(h.ptr, st.ctypes.data_as(ctypes.c_void_p)))


def lbmhd_copy_rows(dst: Handle, dst_row: int, src: Handle, src_row: int, nrows: int):
    _check(lib().lbmhd_copy_rows(dst.ptr, int(dst_row), src.ptr, int(src_row), int(nrows)))


def lbmhd_step_rows(h: Handle, y0: int, y1: int):
    _check(lib().lbmhd_step_rows(h.ptr, int(y0), int(y1)))


def lbmhd_step_commit(h: Handle):
    _check(lib().lbmhd_step_commit(h.ptr))


def _ptr(x):
    return x if isinstance(x, int) else x.data_ptr()


def _stream(stream):
    if stream is None or isinstance(stream, int):
        return ctypes.c_void_p(stream or 0)
    return ctypes.c_void_p(stream.cuda_stream)


def lbmhd_pack_row(h: Handle, row: int, plane_mask: int, buf, stream=None):
    """Gather the masked planes of one row into ``buf`` (a CUDA tensor or a
    device address; popcount(plane_mask) * nx stored values)."""
    _check(lib().lbmhd_pack_row(h.ptr, int(row), ctypes.c_uint(plane_mask),
                                ctypes.c_void_p(_ptr(buf)), _stream(stream)))


def lbmhd_unpack_row(h: Handle, row: int, plane_mask: int, buf, stream=None):
    """Scatter ``buf`` (as lbmhd_pack_row wrote it) into the masked planes of
    one row."""
    _check(lib().lbmhd_unpack_row(h.ptr, int(row), ctypes.c_uint(plane_mask),
                                  ctypes.c_void_p(_ptr(buf)), _stream(stream)))


def lbmhd_sync(h: Handle):
    _check(lib().lbmhd_sync(h.ptr))


def lbmhd_step_count(h: Handle) -> int:
    return int(lib().lbmhd_step_count(h.ptr))


def lbmhd_launch_count(h: Handle) -> int:
    return int(lib().lbmhd_launch_count(h.ptr))


def lbmhd_bytes_per_cell(precision) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return int(lib().lbmhd_bytes_per_cell(int(precision)))


def lbmhd_set_launch(h: Handle, vec: int, block: int):
    _check(lib().lbmhd_set_launch(h.ptr, int(vec), int(block)))


def lbmhd_get_launch(h: Handle):
    v, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbmhd_get_launch(h.ptr, ctypes.byref(v), ctypes.byref(b)))
    return v.value, b.value


FF_OPS = {"add": 0, "sub": 1, "mul": 2, "rcp": 3, "sqrt": 4, "kmul": 5, "norm": 6}


def lbmhd_ff_eval(op, x, y=None) -> np.ndarray:
    """One double-word operation elementwise on the device (see
    include/lbmhd.h); ``op`` a name from FF_OPS or its code."""
    if isinstance(op, str):
        op = FF_OPS[op]
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x) if y is None else np.ascontiguousarray(y, dtype=np.float64)
    assert x.shape == y.shape
    out = np.empty_like(x)
    _check(lib().lbmhd_ff_eval(int(op), x.ctypes.data_as(ctypes.c_void_p),
                               y.ctypes.data_as(ctypes.c_void_p),
                               out.ctypes.data_as(ctypes.c_void_p), x.size))
    return out


def lbmhd_diagnostics_noalloc(state, precision, nx: int, ny: int, plane_stride: int, out,
                              fp16_scale: float = 1024.0, stream=None):
    """Diagnostics of a caller-owned device state without any device
    allocation (see include/lbmhd.h).  ``state`` and ``out`` are CUDA torch
    tensors (or raw device addresses); ``out`` receives 12 doubles in the
    order of DIAG_KEYS.  Enqueued on ``stream`` (int handle or
    torch.cuda.Stream; None: the legacy default stream)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    sp = state if isinstance(state, int) else state.data_ptr()
    op = out if isinstance(out, int) else out.data_ptr()
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(lib().lbmhd_diagnostics_noalloc(ctypes.c_void_p(sp), int(precision), int(nx), int(ny),
                                           int(plane_stride), float(fp16_scale),
                                           ctypes.c_void_p(op), ctypes.c_void_p(stream or 0)))


def lbmhd_destroy(h: Handle):
    if h is not None and h.ptr:
        lib().lbmhd_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


# ---- 3D lattices ---------------------------------------------------------

DIAG3_KEYS = ("mass", "mom_x", "mom_y", "mom_z", "bsum_x", "bsum_y", "bsum_z", "E_kin",
              "E_mag", "cross_helicity", "divB_max", "divB_rms")


class Handle3:
    """An lbmhd3_t* together with its lattice shape (nz, ny, nx)."""

    def __init__(self, ptr: int, nx: int, ny: int, nz: int, params: Params):
        self.ptr = ctypes.c_void_p(ptr)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.params = params

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def precision(self) -> int:
        return int(self.params.precision)


def lbmhd3_create(nx: int, ny: int, nz: int, params: Params | None = None) -> Handle3:
    params = params if params is not None else lbmhd_params_default()
    out = ctypes.c_void_p()
    _check(lib().lbmhd3_create(int(nx), int(ny), int(nz), ctypes.byref(params),
                               ctypes.byref(out)))
    return Handle3(out.value, nx, ny, nz, params)


def lbmhd3_init(h: Handle3, rho, ux, uy, uz, bx, by, bz):
    arrs = [_host(a, h.shape) for a in (rho, ux, uy, uz, bx, by, bz)]
    _check(lib().lbmhd3_init(h.ptr, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs]))


def lbmhd3_step(h: Handle3, n: int = 1):
    _check(lib().lbmhd3_step(h.ptr, int(n)))


def lbmhd3_moments(h: Handle3):
    """(rho, ux, uy, uz, bx, by, bz), each (nz, ny, nx)."""
    out = np.empty((7,) + h.shape)
    _check(lib().lbmhd3_moments(h.ptr, out.ctypes.data_as(ctypes.c_void_p)))
    return tuple(out)


def lbmhd3_get_state(h: Handle3) -> np.ndarray:
    st = np.empty((45,) + h.shape)
    _check(lib().lbmhd3_get_state(h.ptr, st.ctypes.data_as(ctypes.c_void_p)))
    return st


def lbmhd3_diagnostics(h: Handle3) -> dict:
    out = np.empty(12)
    _check(lib().lbmhd3_diagnostics(h.ptr, out.ctypes.data_as(ctypes.c_void_p)))
    return dict(zip(DIAG3_KEYS, out.tolist()))


def lbmhd3_set_launch(h: Handle3, vec: int, block: int):
    _check(lib().lbmhd3_set_launch(h.ptr, int(vec), int(block)))


def lbmhd3_get_launch(h: Handle3):
    v, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbmhd3_get_launch(h.ptr, ctypes.byref(v), ctypes.byref(b)))
    return v.value, b.value


def lbmhd3_sync(h: Handle3):
    _check(lib().lbmhd3_sync(h.ptr))


def lbmhd3_debug(h: Handle3, flags: int):
    _check(lib().lbmhd3_debug(h.ptr, int(flags)))


def lbmhd3_step_count(h: Handle3) -> int:
    return int(lib().lbmhd3_step_count(h.ptr))


def lbmhd3_launch_count(h: Handle3) -> int:
    return int(lib().lbmhd3_launch_count(h.ptr))


def lbmhd3_init_device(h: Handle3, rho, ux, uy, uz, bx, by, bz):
    """Initialise from seven contiguous float64 CUDA tensors of shape
    (nz, ny, nx)."""
    _check(lib().lbmhd3_init_device(h.ptr, *[_dev(t, h.shape) for t in (rho, ux, uy, uz, bx, by, bz)]))


def lbmhd3_moments_device(h: Handle3, rho, ux, uy, uz, bx, by, bz):
    _check(lib().lbmhd3_moments_device(h.ptr, *[_dev(t, h.shape) for t in (rho, ux, uy, uz, bx, by, bz)]))


def lbmhd3_set_state(h: Handle3, state):
    st = _host(state, (45,) + h.shape)
    _check(lib().lbmhd3_set_state(h.ptr, st.ctypes.data_as(ctypes.c_void_p)))


def lbmhd3_get_state_raw(h: Handle3) -> np.ndarray:
    """The stored state in its own format, shape (45, nz, ny, nx) (FF: with a
    trailing 2 for the (hi, lo) pair)."""
    dt, tail = RAW_DTYPES[h.precision]
    st = np.empty((45,) + h.shape + tail, dtype=dt)
    _check(lib().lbmhd3_get_state_raw(h.ptr, st.ctypes.data_as(ctypes.c_void_p), st.nbytes))
    return st


def lbmhd3_set_state_raw(h: Handle3, state):
    dt, tail = RAW_DTYPES[h.precision]
    st = np.ascontiguousarray(state, dtype=dt)
    if st.shape != (45,) + h.shape + tail:
        raise ValueError(f"expected shape {(45,) + h.shape + tail}")
    _check(lib().lbmhd3_set_state_raw(h.ptr, st.ctypes.data_as(ctypes.c_void_p), st.nbytes))


def lbmhd3_step_planes(h: Handle3, z0: int, z1: int):
    _check(lib().lbmhd3_step_planes(h.ptr, int(z0), int(z1)))


def lbmhd3_step_commit(h: Handle3):
    _check(lib().lbmhd3_step_commit(h.ptr))


def lbmhd3_pack_plane(h: Handle3, z: int, plane_mask: int, buf, stream=None):
    """Gather the masked planes of z-plane z into device memory buf (an
    address or a tensor)."""
    _check(lib().lbmhd3_pack_plane(h.ptr, int(z), int(plane_mask), _ptr(buf), _stream(stream)))


def lbmhd3_unpack_plane(h: Handle3, z: int, plane_mask: int, buf, stream=None):
    _check(lib().lbmhd3_unpack_plane(h.ptr, int(z), int(plane_mask), _ptr(buf), _stream(stream)))


def lbmhd3_bytes_per_cell(precision) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return int(lib().lbmhd3_bytes_per_cell(int(precision)))


def lbmhd3_destroy(h: Handle3):
    if h is not None and h.ptr:
        lib().lbmhd3_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()


class Lattice:
    """Convenience owner of one handle (context manager)."""

    def __init__(self, nx: int, ny: int, **params):
        self.h = lbmhd_create(nx, ny, lbmhd_params_default(**params))

    def init(self, rho, ux, uy, bx, by):
        lbmhd_init(self.h, rho, ux, uy, bx, by)
        return self

    def step(self, n: int = 1):
        lbmhd_step(self.h, n)
        return self

    def moments(self):
        return lbmhd_moments(self.h)

    def diagnostics(self):
        return lbmhd_diagnostics(self.h)

    def state(self):
        return lbmhd_get_state(self.h)

    def set_state(self, st):
        lbmhd_set_state(self.h, st)

    def close(self):
        lbmhd_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- adjoint -------------------------------------------------------------


def _dev_or_null(t, shape):
    return ctypes.c_void_p(0) if t is None else _dev(t, shape)


def lbmhd_adjoint_record(h: Handle, rho0, ux0, uy0, bx0, by0, nsteps: int, every: int):
    """Initialise from five device fields and run nsteps steps, keeping FP64
    checkpoints every `every` steps."""
    _check(lib().lbmhd_adjoint_record(h.ptr, *[_dev(t, h.shape) for t in (rho0, ux0, uy0, bx0, by0)],
                                      int(nsteps), int(every)))


def lbmhd_adjoint_backward(h: Handle, grads, want_fields: bool = True):
    """grads: dL/d(final rho, ux, uy, bx, by) as CUDA float64 tensors (None =
    zero).  Returns (dtheta = [dC_S, dtau_nu, dtau_eta], field gradients as a
    tuple of 5 tensors, or None)."""
    import torch

    dth = (ctypes.c_double * 3)()
    outs = None
    if want_fields:
        outs = tuple(torch.empty(h.shape, dtype=torch.float64, device="cuda") for _ in range(5))
    out_ptrs = [ctypes.c_void_p(0)] * 5 if outs is None else [_dev(t, h.shape) for t in outs]
    _check(lib().lbmhd_adjoint_backward(h.ptr, *[_dev_or_null(g, h.shape) for g in grads], dth,
                                        *out_ptrs))
    return [dth[0], dth[1], dth[2]], outs


def lbmhd_adjoint_release(h: Handle):
    _check(lib().lbmhd_adjoint_release(h.ptr))


# ---- ensembles -------------------------------------------------------------

DEBUG_DROP_BARRIER_ARRIVAL = 1


class BatchHandle:
    """An lbmhd_batch_t* with its runs' shapes."""

    def __init__(self, ptr: int, shapes, params: Params):
        self.ptr = ctypes.c_void_p(ptr)
        self.shapes = [tuple(s) for s in shapes]  # (ny, nx) per run
        self.params = params

    @property
    def nruns(self):
        return len(self.shapes)


def lbmhd_batch_create(nx, ny, tau_nu, tau_eta, C_S, params: Params | None = None) -> BatchHandle:
    """nx, ny, tau_nu, tau_eta, C_S: sequences with one entry per run."""
    params = params if params is not None else lbmhd_params_default()
    n = len(nx)
    ai = lambda v: np.ascontiguousarray(v, dtype=np.int32)
    ad = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    arrs = [ai(nx), ai(ny), ad(tau_nu), ad(tau_eta), ad(C_S)]
    if any(len(a) != n for a in arrs):
        raise ValueError("per-run sequences must have equal length")
    out = ctypes.c_void_p()
    _check(lib().lbmhd_batch_create(n, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                    ctypes.byref(params), ctypes.byref(out)))
    return BatchHandle(out.value, list(zip(arrs[1].tolist(), arrs[0].tolist())), params)


def _run_shape(b: BatchHandle, run: int):
    if not 0 <= run < b.nruns:
        raise LBMHDError(-1, f"run index {run} out of range [0, {b.nruns})")
    return b.shapes[run]


def lbmhd_batch_init(b: BatchHandle, run: int, rho, ux, uy, bx, by):
    arrs = [_host(a, _run_shape(b, run)) for a in (rho, ux, uy, bx, by)]
    _check(lib().lbmhd_batch_init(b.ptr, int(run),
                                  *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs]))


def lbmhd_batch_step(b: BatchHandle, n: int = 1):
    _check(lib().lbmhd_batch_step(b.ptr, int(n)))


def lbmhd_batch_moments(b: BatchHandle, run: int):
    out = [np.empty(_run_shape(b, run)) for _ in range(5)]
    _check(lib().lbmhd_batch_moments(b.ptr, int(run),
                                     *[a.ctypes.data_as(ctypes.c_void_p) for a in out]))
    return tuple(out)


def lbmhd_batch_get_state(b: BatchHandle, run: int) -> np.ndarray:
    st = np.empty((19,) + _run_shape(b, run))
    _check(lib().lbmhd_batch_get_state(b.ptr, int(run), st.ctypes.data_as(ctypes.c_void_p)))
    return st


def lbmhd_batch_sync(b: BatchHandle):
    _check(lib().lbmhd_batch_sync(b.ptr))


def lbmhd_batch_set_launch(b: BatchHandle, vec: int, block: int, steps_per_launch: int):
    _check(lib().lbmhd_batch_set_launch(b.ptr, int(vec), int(block), int(steps_per_launch)))


def lbmhd_batch_get_launch(b: BatchHandle):
    v, bl, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().lbmhd_batch_get_launch(b.ptr, ctypes.byref(v), ctypes.byref(bl), ctypes.byref(s)))
    return v.value, bl.value, s.value


def lbmhd_batch_autotune(b: BatchHandle, cache_path: str | None = None,
                         trial_steps: int = 16) -> float:
    best = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(lib().lbmhd_batch_autotune(b.ptr, path, int(trial_steps), ctypes.byref(best)))
    return best.value


def lbmhd_batch_step_count(b: BatchHandle) -> int:
    return int(lib().lbmhd_batch_step_count(b.ptr))


def lbmhd_batch_launch_count(b: BatchHandle) -> int:
    return int(lib().lbmhd_batch_launch_count(b.ptr))


def lbmhd_batch_debug(b: BatchHandle, flags: int):
    _check(lib().lbmhd_batch_debug(b.ptr, int(flags)))


def lbmhd_batch_destroy(b: BatchHandle):
    if b is not None and b.ptr:
        lib().lbmhd_batch_destroy(b.ptr)
        b.ptr = ctypes.c_void_p()
