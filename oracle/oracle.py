"""FP64 CPU oracle for the filtered LB-MHD step (arXiv:1607.08675).

TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
(the CUDA library and its Python binding) never does.  It loads
``lbmhd_oracle.c`` (plain C, FP64, ``-ffp-contract=off``) through ctypes,
building it with gcc on first use.  It shares no code with the CUDA path.

State layout: a float64 array of shape (19, ny, nx); planes 0..8 are the
D2Q9 populations f_i, plane 9 + 2k + a is component a of the D2Q5 vector
population g_k.  Parameters are a dict with keys tau_nu, tau_eta, C_S,
delta, s5, s6, s7, s8, les (see ``params``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbmhd_oracle.so")
_lock = threading.Lock()
_lib = None

NPLANE = 19


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if the compiler has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]
    for extra in (["-fopenmp"], []):
        cmd = base + extra + [_SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        i32, i64, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        sig = {
            "orc_lattice": (None, [ip, ip, ip, ip, dp, dp]),
            "orc_tmatrix": (None, [dp, dp, dp]),
            "orc_feq": (None, [d, d, d, d, d, dp]),
            "orc_geq": (None, [d, d, d, d, dp]),
            "orc_collide_cell": (None, [dp, dp, dp, dp]),
            "orc_stream": (None, [i32, i32, dp, dp]),
            "orc_init": (None, [i32, i32, dp, dp, dp, dp, dp, dp]),
            "orc_step": (i32, [i32, i32, dp, dp, dp, i32, i32]),
            "orc_step_cells": (None, [i32, i32, dp, dp, i64, lp, dp]),
            "orc_les_fields": (None, [i32, i32, dp, dp, dp]),
            "orc_moments": (None, [i32, i32, dp, dp, dp, dp, dp, dp]),
            "orc_diagnostics": (None, [i32, i32, dp, dp]),
            "orc_step_bgk": (i32, [i32, i32, d, d, dp, dp, i32]),
            "orc_kinetic_shift": (None, [dp, dp, d, dp]),
            "orc_collide_cell_shift": (None, [dp, dp, dp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(tau_nu=0.6, tau_eta=0.6, C_S=0.1, delta=1.0, s5=0.0, s6=0.0, s7=0.0, s8=0.0, les=1):
    """Parameter dict; s5..s8 <= 0 means tied (s5, s6 to 1/tau_nu; s7, s8 to
    the local s_nu).  les: 0 none, 1 local Smagorinsky rates, 2 the paper's
    filtered equilibria (kinetic LES)."""
    return dict(tau_nu=tau_nu, tau_eta=tau_eta, C_S=C_S, delta=delta, s5=s5, s6=s6, s7=s7,
                s8=s8, les=les)


def _pvec(p: dict) -> np.ndarray:
    keys = ["tau_nu", "tau_eta", "C_S", "delta", "s5", "s6", "s7", "s8", "les"]
    return np.array([float(p[k]) for k in keys], dtype=np.float64)


def lattice():
    """Return (cx, cy, Cx, Cy, w, w') as numpy arrays."""
    lib = _load()
    cx, cy = (ctypes.c_int * 9)(), (ctypes.c_int * 9)()
    mx, my = (ctypes.c_int * 5)(), (ctypes.c_int * 5)()
    w, wm = np.zeros(9), np.zeros(5)
    lib.orc_lattice(cx, cy, mx, my, _dp(w), _dp(wm))
    return (np.array(cx[:]), np.array(cy[:]), np.array(mx[:]), np.array(my[:]), w, wm)


def tmatrix():
    """Return (T, T^-1, T_m) as built by the oracle."""
    lib = _load()
    T, Ti, Tm = np.zeros((9, 9)), np.zeros((9, 9)), np.zeros((5, 5))
    lib.orc_tmatrix(_dp(T), _dp(Ti), _dp(Tm))
    return T, Ti, Tm


def feq(rho, ux, uy, bx, by) -> np.ndarray:
    f = np.zeros(9)
    _load().orc_feq(rho, ux, uy, bx, by, _dp(f))
    return f


def geq(ux, uy, bx, by) -> np.ndarray:
    """D2Q5 vector equilibrium, shape (5, 2)."""
    g = np.zeros(10)
    _load().orc_geq(ux, uy, bx, by, _dp(g))
    return g.reshape(5, 2)


def collide_cell(z: np.ndarray, p: dict):
    """Collide one node's 19 streamed populations; returns (out, aux) with
    aux = (tau_nu_eff, tau_m_eff, Q, J)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    out, aux = np.zeros(19), np.zeros(4)
    _load().orc_collide_cell(_dp(z), _dp(_pvec(p)), _dp(out), _dp(aux))
    return out, aux


def kinetic_shift(fields, grads, delta=1.0) -> np.ndarray:
    """Delta^2 times the filtered-equilibrium corrections (M3, M4, M7 = M8,
    N_y1) at one node; fields = (rho, jx, jy, Bx, By), grads[q] = (d/dx,
    d/dy) of field q."""
    f = np.ascontiguousarray(fields, dtype=np.float64)
    g = np.ascontiguousarray(np.asarray(grads, dtype=np.float64).reshape(10))
    out = np.zeros(4)
    _load().orc_kinetic_shift(_dp(f), _dp(g), float(delta), _dp(out))
    return out


def collide_cell_shift(z: np.ndarray, p: dict, shift) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float64)
    sh = np.ascontiguousarray(shift, dtype=np.float64)
    out = np.zeros(19)
    _load().orc_collide_cell_shift(_dp(z), _dp(_pvec(p)), _dp(sh), _dp(out))
    return out


def init(rho, ux, uy, bx, by) -> np.ndarray:
    ny, nx = np.shape(rho)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, bx, by)]
    st = np.zeros((NPLANE, ny, nx))
    _load().orc_init(nx, ny, *[_dp(a) for a in arrs], _dp(st))
    return st


def stream(state: np.ndarray) -> np.ndarray:
    _, ny, nx = state.shape
    state = np.ascontiguousarray(state)
    out = np.zeros_like(state)
    _load().orc_stream(nx, ny, _dp(state), _dp(out))
    return out


def step(state: np.ndarray, p: dict, nsteps: int = 1, nthreads: int = 1) -> np.ndarray:
    """Return the state after ``nsteps`` steps (input left untouched)."""
    _, ny, nx = state.shape
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    work = np.zeros_like(st)
    _load().orc_step(nx, ny, _dp(_pvec(p)), _dp(st), _dp(work), int(nsteps), int(nthreads))
    return st


def step_cells(state: np.ndarray, p: dict, idx: np.ndarray) -> np.ndarray:
    """Post-step populations at flat node indices ``idx``; shape (len, 19)."""
    _, ny, nx = state.shape
    state = np.ascontiguousarray(state, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), NPLANE))
    _load().orc_step_cells(nx, ny, _dp(_pvec(p)), _dp(state), len(idx),
                           idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
    return out


def les_fields(state: np.ndarray, p: dict) -> np.ndarray:
    """(tau_nu_eff, tau_m_eff, Q, J) at every node of the next step; shape
    (4, ny, nx)."""
    _, ny, nx = state.shape
    state = np.ascontiguousarray(state, dtype=np.float64)
    aux = np.zeros((4, ny, nx))
    _load().orc_les_fields(nx, ny, _dp(_pvec(p)), _dp(state), _dp(aux))
    return aux


def moments(state: np.ndarray):
    """(rho, ux, uy, bx, by), each (ny, nx)."""
    _, ny, nx = state.shape
    state = np.ascontiguousarray(state, dtype=np.float64)
    out = [np.zeros((ny, nx)) for _ in range(5)]
    _load().orc_moments(nx, ny, _dp(state), *[_dp(a) for a in out])
    return tuple(out)


DIAG_KEYS = ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y", "E_kin", "E_mag", "enstrophy",
             "cross_helicity", "divB_max", "divB_rms", "current_sq")


def diagnostics(state: np.ndarray) -> dict:
    _, ny, nx = state.shape
    state = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros(12)
    _load().orc_diagnostics(nx, ny, _dp(state), _dp(out))
    return dict(zip(DIAG_KEYS, out.tolist()))


def step_bgk(state: np.ndarray, tau_nu: float, tau_eta: float, nsteps: int = 1) -> np.ndarray:
    _, ny, nx = state.shape
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    work = np.zeros_like(st)
    _load().orc_step_bgk(nx, ny, tau_nu, tau_eta, _dp(st), _dp(work), int(nsteps))
    return st
