import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle._load()
    return oracle


@pytest.fixture(scope="session")
def fsp():
    """The CUDA library's Python binding (builds libfsp.so if needed)."""
    import paper_2405_02603_gb300 as m
    m.lib()
    return m


def to_dev(a, dtype="f64"):
    import numpy as np
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if dtype == "f32" else np.float64))
    return t.cuda()


def e_max(got, ref):
    """max |got - ref| / max |ref| for real or complex arrays."""
    import numpy as np
    got = np.asarray(got)
    ref = np.asarray(ref)
    got = got.astype(np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = ref.astype(np.complex128 if np.iscomplexobj(ref) else np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


_T_CACHE = {}


def oracle_T(orc, algo, N, L=1.0):
    """Oracle kernel T, cached per (algo, N, L) across tests."""
    key = (algo, N, float(L))
    if key not in _T_CACHE:
        _T_CACHE[key] = orc.kernel_T(algo, N, L)
    return _T_CACHE[key]


# Whole-field E_max = max|phi - phi_oracle| / max|phi_oracle| allowed per
# (N, dtype) for the bench's source (seeded 8-Gaussian mixture, float32-
# rounded) with the Vico-Greengard kernel: twice the value measured on the
# GB300 (tests/test_gpu_precision.py), which is
#            N = 128     N = 256     N = 512
#   f32      2.22e-7     2.72e-7     2.74e-7
#   f64df    9.31e-15    1.08e-14    1.22e-14
#   f64      6.12e-16    7.95e-16    9.18e-16
E_MAX_MEASURED = {
    (128, "f32"): 2.22e-7, (256, "f32"): 2.72e-7, (512, "f32"): 2.74e-7,
    (128, "f64df"): 9.31e-15, (256, "f64df"): 1.08e-14, (512, "f64df"): 1.22e-14,
    (128, "f64"): 6.12e-16, (256, "f64"): 7.95e-16, (512, "f64"): 9.18e-16,
}
E_MAX_GATE = {k: 2.0 * v for k, v in E_MAX_MEASURED.items()}


# FP32-mixed gate per size for the other parity tests (mixtures, random
# fields, boxes by their largest axis, field components): twice the envelope
# (running maximum over sizes up to N) of the largest E_max measured on the
# GB300 among those tests at each size.
F32_MEASURED = {
    2: 6.31e-8, 3: 1.43e-7, 4: 1.48e-7, 5: 1.32e-7, 6: 1.32e-7, 8: 2.04e-7, 9: 1.38e-7, 10: 1.47e-7,
    12: 2.24e-7, 15: 2.04e-7, 16: 2.03e-7, 18: 2.43e-7, 20: 1.86e-7, 24: 2.39e-7, 25: 2.33e-7, 27: 2.55e-7,
    30: 2.04e-7, 32: 2.16e-7, 40: 2.25e-7, 45: 2.70e-7, 48: 2.23e-7, 50: 2.00e-7, 60: 1.78e-7, 64: 2.48e-7,
    80: 2.09e-7, 96: 2.52e-7, 128: 3.25e-7, 256: 2.79e-7, 512: 2.79e-7, 1024: 2.76e-7,
}


def f32_gate(N):
    """FP32-mixed E_max gate at grid size N (largest axis for a box)."""
    sizes = sorted(F32_MEASURED)
    upto = [k for k in sizes if k <= N] or sizes[:1]
    nxt = [k for k in sizes if k >= N]
    env = max(F32_MEASURED[k] for k in upto + nxt[:1])
    return 2.0 * env


def check_emax(err, N, dtype, label=""):
    """Print and gate one E_max: FP64 and double-float at the 1e-12 target,
    FP32-mixed at f32_gate(N)."""
    print("EMAX %s N=%d %s %.3e" % (label, N, dtype, err))
    gate = f32_gate(N) if dtype == "f32" else 1e-12
    assert err <= gate, (label, N, dtype, err, gate)
