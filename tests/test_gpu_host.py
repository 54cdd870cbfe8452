"""Pinned host buffers on the GPU's nearest NUMA node (fsp_host_alloc) feed
the host-buffer solves: the pipelined and the single host solve through such
buffers give bitwise the device solve's field, and the buffers' pages sit on
the requested node when the system reports NUMA placement."""
import numpy as np
import pytest

import fsp_inputs as I

pytestmark = pytest.mark.gpu


def _pages(addr, nbytes):
    import bench
    return bench.numa_pages(addr, nbytes)


def test_host_buffers_feed_host_solves(fsp):
    import torch
    N = 64
    node = fsp.device_host_numa()
    p = fsp.Plan(N, 1.0, "vg_dct", "f32")
    srcs = [I.gaussian_mixture(N, seed=s).astype(np.float32) for s in (1, 2, 3)]
    ref = [p.solve(torch.from_numpy(x).cuda()).cpu().numpy() for x in srcs]
    hin = [fsp.HostBuffer((N, N, N), np.float32, node) for _ in srcs]
    hout = [fsp.HostBuffer((N, N, N), np.float32, node) for _ in srcs]
    for b, x in zip(hin, srcs):
        b.array[...] = x
    p.solve_host_many([b.array for b in hin], [b.array for b in hout])
    for b, r in zip(hout, ref):
        assert np.array_equal(b.array, r)
    hout[0].array[...] = 0
    p.solve_host(hin[0].array, hout[0].array)
    assert np.array_equal(hout[0].array, ref[0])
    if node >= 0:
        pages = _pages(hin[0].array.ctypes.data, hin[0].nbytes)
        if pages:
            assert set(pages) == {node}, pages
    for b in hin + hout:
        b.close()
    p.close()


def test_host_alloc_rejects_bad_arguments(fsp):
    import ctypes
    lib = fsp.lib()
    q = ctypes.c_void_p()
    assert lib.fsp_host_alloc(None, 4096, -1) == fsp.FSP_EINVAL
    assert lib.fsp_host_alloc(ctypes.byref(q), 0, -1) == fsp.FSP_EINVAL
    assert lib.fsp_host_free(None, 4096) == fsp.FSP_EINVAL
    assert lib.fsp_host_alloc(ctypes.byref(q), 4096, -1) == fsp.FSP_OK
    assert lib.fsp_host_free(q, 4096) == fsp.FSP_OK
