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
