"""Host-side checks of the C ABI: the library loads, exports every entry
point include/lbmhd.h declares, and validates parameters before touching
the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_1607_08675_gb300 import build, lbmhd

    build.build()
    return lbmhd


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbmhd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmhd_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_function(L):
    for n in declared_functions():
        if n in ("lbmhd_last_error",):
            continue
        assert hasattr(L, n), n


def test_params_default(L):
    p = L.lbmhd_params_default()
    assert p.abi_version == 1 and p.precision == 0
    assert (p.tau_nu, p.tau_eta, p.C_S, p.delta, p.les) == (0.6, 0.6, 0.1, 1.0, 1)
    assert (p.s5, p.s6, p.s7, p.s8) == (0.0, 0.0, 0.0, 0.0)
    assert p.fp16_scale == 1024.0 and not p.stream


def test_bytes_per_cell(L):
    assert [L.lbmhd_bytes_per_cell(p) for p in ("fp64", "fp32", "fp32_dev", "fp16_dev", "ff")] == [
        304, 152, 152, 76, 304]
    assert L.lbmhd_bytes_per_cell(7) == 0


@pytest.mark.parametrize("bad,code", [
    (dict(tau_nu=0.5), -1), (dict(tau_eta=0.4), -1), (dict(C_S=-0.1), -1),
    (dict(delta=0.0), -1), (dict(s5=2.5), -1), (dict(precision=9), -1),
    (dict(tau_nu=float("nan")), -1), (dict(les=4), -1), (dict(fp16_scale=0.0), -1),
    (dict(check_finite_every=-1), -1),
    # xi <= 0 (Sec. 4.3) at tau_nu = 0.6 with s8 large and s7 small
    (dict(s7=0.2, s8=1.9), -1),
    (dict(abi_version=2), -6),
])
def test_invalid_params_rejected_before_any_device_call(L, bad, code):
    p = L.lbmhd_params_default(**bad)
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_create(16, 16, p)
    assert e.value.code == code
    assert L.lib().lbmhd_last_error().decode()


def test_invalid_sizes_rejected(L):
    for nx, ny in ((0, 4), (4, 0), (-1, 3), (1 << 16, 1 << 15)):
        with pytest.raises(L.LBMHDError) as e:
            L.lbmhd_create(nx, ny)
        assert e.value.code == -1


def test_null_handle_calls_fail_cleanly(L):
    lib = L.lib()
    assert lib.lbmhd_step(None, 1) == -1
    assert lib.lbmhd_sync(None) == -1
    assert lib.lbmhd_step_count(None) == 0
    lib.lbmhd_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1607_08675_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f == "inputs.py", f


def test_noalloc_diagnostics_refuses_misaligned_pointers_on_the_host(L):
    """lbmhd_diagnostics_noalloc checks pointer alignment before any CUDA
    call, so the refusal needs no GPU: a state off the stored value size or
    an out pointer off 8 bytes is EINVAL (the addresses are never touched)."""
    lib = L.lib()
    base = 1 << 20  # an aligned fake address; nothing dereferences it
    for prec, size in ((0, 8), (4, 8), (1, 4), (2, 4), (3, 2)):
        for off in sorted({1, size // 2} - {0}):
            rc = lib.lbmhd_diagnostics_noalloc(ctypes.c_void_p(base + off), prec, 8, 4, 32,
                                               1024.0, ctypes.c_void_p(base), None)
            assert rc == -1, (prec, off)
            assert "aligned" in lib.lbmhd_last_error().decode()
    for off in (1, 2, 4):
        rc = lib.lbmhd_diagnostics_noalloc(ctypes.c_void_p(base), 0, 8, 4, 32, 1024.0,
                                           ctypes.c_void_p(base + off), None)
        assert rc == -1 and "aligned" in lib.lbmhd_last_error().decode()
