"""FP64 CPU oracle for the 3D extension of the LB-MHD step (arXiv:1607.08675).

TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
never does.  It loads ``lbmhd3_oracle.c`` (plain C, FP64,
``-ffp-contract=off``) through ctypes, building it with gcc on first use.
It shares no code with the CUDA path.

State layout: a float64 array of shape (45, nz, ny, nx); planes 0..26 are
the D3Q27 populations f_i (i = 9 kz + 3 ky + kx, c = (v[kx], v[ky], v[kz]),
v = (0, 1, -1)), plane 27 + 3q + a is component a of the magnetic
population g_q on the axis C_q = +x, -x, +y, -y, +z, -z.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmhd3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbmhd3_oracle.so")
_lock = threading.Lock()
_lib = None

NQ, NM = 27, 6
NPLANE = NQ + 3 * NM


def build(force: bool = False) -> str:
    """Compile the 3D oracle with gcc (OpenMP if the compiler has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base + extra + [_SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
    raise RuntimeError("3D oracle build failed:\n" + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
        sig = {
            "orc3_lattice": (None, [ip, dp, ip, dp]),
            "orc3_feq": (None, [d, dp, dp, dp]),
            "orc3_geq": (None, [dp, dp, dp]),
            "orc3_collide_cell": (None, [dp, dp, dp, dp]),
            "orc3_stream": (None, [i, i, i, dp, dp]),
            "orc3_init": (None, [i, i, i, dp, dp, dp, dp, dp, dp, dp, dp]),
            "orc3_step": (i, [i, i, i, dp, dp, dp, i, i]),
            "orc3_step_cells": (None, [i, i, i, dp, dp, l, lp, dp]),
            "orc3_moments": (None, [i, i, i, dp, dp]),
            "orc3_diagnostics": (None, [i, i, i, dp, dp]),
            "orc3_kinetic_shift": (None, [dp, dp, d, dp, dp]),
            "orc3_carati_taus": (None, [dp, dp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(tau_nu=0.6, tau_eta=0.6, C_S=0.1, delta=1.0, les=1) -> np.ndarray:
    """les: 0 none, 1 local Smagorinsky rates, 2 the paper's filtered
    equilibria (kinetic LES), 3 the cross-helicity closure."""
    return np.array([tau_nu, tau_eta, C_S, delta, float(les)], dtype=np.float64)


def lattice():
    """(c (27, 3), w (27,), C (6, 3), w' (6,))."""
    c = np.zeros(81, dtype=np.int32)
    w = np.zeros(NQ)
    cm = np.zeros(18, dtype=np.int32)
    wm = np.zeros(NM)
    _load().orc3_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                         cm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(wm))
    return c.reshape(NQ, 3), w, cm.reshape(NM, 3), wm


def feq(rho, u, B) -> np.ndarray:
    out = np.zeros(NQ)
    _load().orc3_feq(float(rho), _dp(np.asarray(u, np.float64)), _dp(np.asarray(B, np.float64)),
                     _dp(out))
    return out


def geq(u, B) -> np.ndarray:
    out = np.zeros(3 * NM)
    _load().orc3_geq(_dp(np.asarray(u, np.float64)), _dp(np.asarray(B, np.float64)), _dp(out))
    return out


def collide_cell(z: np.ndarray, p: np.ndarray):
    """(post-collision 45 values, (tau_e, tau_m, Q, J))."""
    z = np.ascontiguousarray(z, np.float64)
    out, aux = np.zeros(NPLANE), np.zeros(4)
    _load().orc3_collide_cell(_dp(z), _dp(p), _dp(out), _dp(aux))
    return out, aux


def kinetic_shift(fld, grad, delta):
    """Delta^2 corrections of the equilibria (les = 2) at one node.
    fld: rho, jx, jy, jz, Bx, By, Bz; grad (7, 3): d field / d (x, y, z).
    Returns (f shift (27,), g shift (18,))."""
    fld = np.ascontiguousarray(fld, np.float64)
    grad = np.ascontiguousarray(grad, np.float64).reshape(-1)
    fs, gs = np.zeros(NQ), np.zeros(3 * NM)
    _load().orc3_kinetic_shift(_dp(fld), _dp(grad), float(delta), _dp(fs), _dp(gs))
    return fs, gs


def carati_taus(p, f6):
    """(tau_e, tau_m) of the cross-helicity closure from the fields
    (rho, jx, jy, jz, Bx, By, Bz) at the neighbours x+, x-, y+, y-, z+, z-."""
    f6 = np.ascontiguousarray(f6, np.float64).reshape(-1)
    out = np.zeros(2)
    _load().orc3_carati_taus(_dp(np.ascontiguousarray(p, np.float64)), _dp(f6), _dp(out))
    return out


def init(rho, ux, uy, uz, bx, by, bz) -> np.ndarray:
    nz, ny, nx = rho.shape
    st = np.zeros((NPLANE, nz, ny, nx))
    arrs = [np.ascontiguousarray(a, np.float64) for a in (rho, ux, uy, uz, bx, by, bz)]
    _load().orc3_init(nx, ny, nz, *[_dp(a) for a in arrs], _dp(st))
    return st


def stream(state: np.ndarray) -> np.ndarray:
    _, nz, ny, nx = state.shape
    st = np.ascontiguousarray(state, np.float64)
    out = np.empty_like(st)
    _load().orc3_stream(nx, ny, nz, _dp(st), _dp(out))
    return out


def step(state: np.ndarray, p: np.ndarray, nsteps: int = 1, nthreads: int = 1) -> np.ndarray:
    _, nz, ny, nx = state.shape
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    work = np.empty_like(st)
    _load().orc3_step(nx, ny, nz, _dp(p), _dp(st), _dp(work), int(nsteps), int(nthreads))
    return st


def step_cells(state: np.ndarray, p: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """One step at the flat node indices idx: array (len(idx), 45)."""
    _, nz, ny, nx = state.shape
    st = np.ascontiguousarray(state, np.float64)
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.zeros((len(idx), NPLANE))
    _load().orc3_step_cells(nx, ny, nz, _dp(p), _dp(st), len(idx),
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
    return out


def moments(state: np.ndarray):
    """rho, ux, uy, uz, bx, by, bz, each (nz, ny, nx)."""
    _, nz, ny, nx = state.shape
    st = np.ascontiguousarray(state, np.float64)
    out = np.zeros((7, nz, ny, nx))
    _load().orc3_moments(nx, ny, nz, _dp(st), _dp(out))
    return tuple(out)


DIAG_KEYS = ("mass", "mom_x", "mom_y", "mom_z", "bsum_x", "bsum_y", "bsum_z", "E_kin", "E_mag",
             "cross_helicity", "divB_max", "divB_rms")


def diagnostics(state: np.ndarray) -> dict:
    _, nz, ny, nx = state.shape
    st = np.ascontiguousarray(state, np.float64)
    out = np.zeros(12)
    _load().orc3_diagnostics(nx, ny, nz, _dp(st), _dp(out))
    return dict(zip(DIAG_KEYS, out))
