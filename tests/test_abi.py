"""The C-ABI library builds, loads and exports every entry point of
include/fsp.h; host-side validation rejects bad arguments before any device
work (no GPU needed for these calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2405_02603_gb300 as fsp
    return fsp.lib()


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(L, s), s


def test_header_compiles_as_c_and_cpp(tmp_path):
    """include/fsp.h is a plain C interface: it compiles as C11 (pedantic)
    and as C++17 without CUDA headers."""
    import shutil
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "fsp.h"\nint main(void) { fsp_plan *p = 0; (void)p; return (int)FSP_OK; }\n')
    inc = os.path.join(ROOT, "include")
    if shutil.which("gcc"):
        subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc,
                        str(src)], check=True)
    if shutil.which("g++"):
        subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, "-x", "c++", str(src)],
                       check=True)


def test_status_strings(L):
    for code in range(7):
        assert L.fsp_status_str(code).startswith(b"FSP_")
    assert L.fsp_status_str(99).startswith(b"FSP_?")


def test_plan_create_validation_needs_no_device(L):
    p = ctypes.c_void_p()
    bad = [(1, 1.0, 1.0, 0, 0), (0, 1.0, 0.1, 0, 0), (8, -1.0, -0.125, 0, 0), (8, 1.0, 0.2, 0, 0),
           (8, 1.0, 0.125, 7, 0), (8, 1.0, 0.125, 0, 5), (8, float("inf"), 0.1, 0, 0)]
    for N, Lb, h, algo, dt in bad:
        assert L.fsp_plan_create(ctypes.byref(p), N, Lb, h, algo, dt, None) == 1, (N, Lb, h, algo, dt)
        assert not p.value
    # 2N not 2/3/5-smooth, and N above the supported maximum
    assert L.fsp_plan_create(ctypes.byref(p), 7, 1.0, 1.0 / 7, 0, 0, None) == 2
    assert L.fsp_plan_create(ctypes.byref(p), 2048, 1.0, 1.0 / 2048, 0, 0, None) == 2
    assert L.fsp_plan_create(None, 8, 1.0, 0.125, 0, 0, None) == 1


def test_aniso_plan_validation_needs_no_device(L):
    p = ctypes.c_void_p()
    c = L.fsp_plan_create_aniso
    assert c(None, 8, 8, 16, 0.1, 0.1, 0.1, 0, 0, None) == 1
    # sizes, spacings, method, dtype
    for args in [(1, 8, 8, 0.1, 0.1, 0.1, 0, 0), (8, 8, 8, 0.1, -0.1, 0.1, 0, 0), (8, 8, 8, 0.1, 0.1, float("nan"), 0, 0),
                 (8, 8, 8, 0.1, 0.1, 0.1, 7, 0), (8, 8, 8, 0.1, 0.1, 0.1, 0, 9)]:
        assert c(ctypes.byref(p), *args, None) == 1, args
        assert not p.value
    # 2 n_a not smooth, n_a too large, 4 n_a not smooth for VG
    assert c(ctypes.byref(p), 8, 7, 8, 0.1, 0.1, 0.1, 0, 0, None) == 2
    assert c(ctypes.byref(p), 8, 8, 2048, 0.1, 0.1, 0.1, 0, 0, None) == 2
    # the Vico-Greengard window beyond 3 min L_a (1 x 1 x 2.5 box); double-float on a non-cube
    # without the specialised kernels (n_a = 16)
    assert c(ctypes.byref(p), 16, 16, 40, 1.0 / 16, 1.0 / 16, 1.0 / 16, 1, 0, None) == 2
    assert c(ctypes.byref(p), 16, 16, 40, 1.0 / 16, 1.0 / 16, 1.0 / 16, 2, 0, None) == 2
    assert c(ctypes.byref(p), 16, 16, 32, 1.0 / 16, 1.0 / 16, 1.0 / 16, 0, 2, None) == 2


def test_unknown_plan_is_rejected(L):
    fake = ctypes.c_void_p(0x1000)
    assert L.fsp_solve(fake, fake, fake, None) == 1
    assert L.fsp_solve(None, fake, fake, None) == 1
    assert L.fsp_plan_destroy(fake) == 1
    assert L.fsp_plan_destroy(None) == 1
    assert L.fsp_plan_bytes(fake) == 0
    assert L.fsp_plan_precompute_ms(fake) < 0
    assert L.fsp_plan_spectrum(fake, fake) == 1
    assert L.fsp_plan_sync(fake, None) == 1
    assert L.fsp_plan_field_init(fake, None) == 1
    assert L.fsp_plan_field_init(None, None) == 1
    assert L.fsp_solve_field(fake, fake, None, fake, fake, fake, None) == 1
    assert L.fsp_solve_field(None, fake, None, fake, fake, fake, None) == 1


def test_fft_and_kernel_validation(L):
    assert L.fsp_fft_c2c(7, 1, 0, -1, None, None, None) == 2
    assert L.fsp_fft_c2c(8, 1, 0, 0, None, None, None) == 1
    assert L.fsp_fft_c2c(8, 0, 0, -1, None, None, None) == 0  # nothing to do
    assert L.fsp_fft_c2c(8, 1, 3, -1, None, None, None) == 1
    assert L.fsp_kernel_T(1, 1.0, 0, None, None) == 1
    assert L.fsp_kernel_T(8, 1.0, 0, None, None) == 1
    assert L.fsp_kernel_T(11, 1.0, 0, None, None) == 2


def test_spectrum_restore_validation_needs_no_device(L, tmp_path):
    """fsp_plan_create_from_spectrum refuses bad arguments before any CUDA
    call; the binding checks the array shape and the file format first."""
    import numpy as np
    import paper_2405_02603_gb300 as fsp
    out = ctypes.c_void_p()
    S = np.ones((9, 9, 9))
    ptr = ctypes.c_void_p(S.ctypes.data)
    assert L.fsp_plan_create_from_spectrum(None, 8, 1.0, 0, 0, ptr, None) == 1
    assert L.fsp_plan_create_from_spectrum(ctypes.byref(out), 8, 1.0, 0, 0, None, None) == 1
    bad = S.copy()
    bad[4, 4, 4] = np.inf
    assert L.fsp_plan_create_from_spectrum(ctypes.byref(out), 8, 1.0, 0, 0,
                                           ctypes.c_void_p(bad.ctypes.data), None) == 1
    assert out.value is None
    S7 = np.ones((8, 8, 8))  # 2N = 14 is not 2/3/5-smooth
    assert L.fsp_plan_create_from_spectrum(ctypes.byref(out), 7, 1.0, 0, 0,
                                           ctypes.c_void_p(S7.ctypes.data), None) == 2
    with pytest.raises(fsp.FspError) as ei:
        fsp.Plan.from_spectrum(8, 1.0, "he", "f64", np.ones((8, 8, 8)))
    assert ei.value.status == fsp.FSP_EINVAL
    np.savez(tmp_path / "other.npz", format=np.array("not-a-spectrum"), S=S)
    with pytest.raises(fsp.FspError) as ei:
        fsp.Plan.load(tmp_path / "other.npz")
    assert ei.value.status == fsp.FSP_EINVAL


def test_product_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2405_02603_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "fsp_oracle" not in text, f
