"""Python binding of libfsp.so, the GB300 free-space spectral Poisson solver.

Thin ctypes marshalling over the C ABI declared in include/fsp.h: every step of
every solve runs in the library's CUDA kernels.  PyTorch is used only to own
device memory (``tensor.data_ptr()``) and to name streams
(``torch.cuda.current_stream().cuda_stream``).  There is no CPU fallback: if
the library is missing or a call fails, an exception is raised.

    import torch, paper_2405_02603_gb300 as fsp
    plan = fsp.Plan(N=256, L=1.0, algo="vg_dct", dtype="f32")
    phi = plan.solve(rho)          # rho: CUDA tensor (N, N, N) float32
"""
import ctypes
import os

from . import build as _build

FSP_OK, FSP_EINVAL, FSP_EUNSUPPORTED, FSP_ENOMEM, FSP_ECUDA, FSP_EBUSY, FSP_ETIMEOUT = range(7)
STATUS_NAMES = ["FSP_OK", "FSP_EINVAL", "FSP_EUNSUPPORTED", "FSP_ENOMEM", "FSP_ECUDA", "FSP_EBUSY",
                "FSP_ETIMEOUT"]
ALGOS = {"he": 0, "vg": 1, "vg_dct": 2}
DTYPES = {"f64": 0, "f32": 1, "f64df": 2}

_lib = None


class ServerStats(ctypes.Structure):
    """fsp_server_stats"""
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "spec_hits", "spec_misses",
                                               "evictions", "queued", "running", "cached_spectra")] + \
               [("bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("builds_in_flight", ctypes.c_uint64), ("peak_bytes_in_use", ctypes.c_size_t)]


class FspError(RuntimeError):
    """A non-FSP_OK status returned by the library."""

    def __init__(self, status, where=""):
        self.status = int(status)
        name = STATUS_NAMES[self.status] if 0 <= self.status < len(STATUS_NAMES) else str(status)
        super().__init__("%s%s" % (where + ": " if where else "", name))


def library_path():
    return _build.library_path()


def lib(build_if_missing=True):
    """Load libfsp.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.library_path()
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise FspError(FSP_ECUDA, "libfsp.so not built (" + path + ")")
    L = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.fsp_status_str.restype = ctypes.c_char_p
    L.fsp_status_str.argtypes = [i]
    L.fsp_plan_create.argtypes = [ctypes.POINTER(vp), i, d, d, i, i, vp]
    L.fsp_plan_create_aniso.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, d, i, i, vp]
    L.fsp_solve.argtypes = [vp, vp, vp, vp]
    L.fsp_solve_host.argtypes = [vp, vp, vp, vp]
    L.fsp_solve_host_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]
    L.fsp_solve_host_many.restype = i
    L.fsp_plan_sync.argtypes = [vp, vp]
    L.fsp_plan_destroy.argtypes = [vp]
    L.fsp_plan_bytes.argtypes = [vp]
    L.fsp_plan_bytes.restype = sz
    L.fsp_plan_precompute_ms.argtypes = [vp]
    L.fsp_plan_precompute_ms.restype = d
    L.fsp_plan_spectrum.argtypes = [vp, vp]
    L.fsp_plan_create_from_spectrum.argtypes = [ctypes.POINTER(vp), i, d, i, i, vp, vp]
    L.fsp_kernel_T.argtypes = [i, d, i, vp, vp]
    L.fsp_fft_c2c.argtypes = [i, i, i, i, vp, vp, vp]
    L.fsp_plan_set_timing.argtypes = [vp, ctypes.POINTER(vp), i]
    L.fsp_solve_noalloc.argtypes = [i, vp, vp, vp, vp]
    L.fsp_plan_field_init.argtypes = [vp, vp]
    L.fsp_solve_field.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fsp_plan_uses_fast_path.argtypes = [vp]
    L.fsp_plan_uses_fast_path.restype = i
    L.fsp_dist_partition.argtypes = [i, i, i] + [ctypes.POINTER(i)] * 4
    L.fsp_dist_partition.restype = i
    L.fsp_dist_block_elems.argtypes = [i, i, i, i, i, i]
    L.fsp_dist_block_elems.restype = ctypes.c_longlong
    L.fsp_dist_create.argtypes = [ctypes.POINTER(vp), i, d, i, i, i, i, vp]
    L.fsp_dist_create.restype = i
    L.fsp_dist_forward.argtypes = [vp, vp, ctypes.POINTER(vp), vp]
    L.fsp_dist_forward.restype = i
    L.fsp_dist_middle.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.fsp_dist_middle.restype = i
    L.fsp_dist_backward.argtypes = [vp, ctypes.POINTER(vp), vp, vp]
    L.fsp_dist_backward.restype = i
    L.fsp_dist_destroy.argtypes = [vp]
    L.fsp_dist_destroy.restype = i
    L.fsp_device_host_numa.argtypes = [i]
    L.fsp_device_host_numa.restype = i
    L.fsp_host_alloc.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, i]
    L.fsp_host_alloc.restype = i
    L.fsp_host_free.argtypes = [vp, ctypes.c_size_t]
    L.fsp_host_free.restype = i
    L.fsp_plan_check_bounds.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
    L.fsp_plan_check_bounds.restype = i
    L.fsp_bounds_freed_bad.argtypes = []
    L.fsp_bounds_freed_bad.restype = ctypes.c_ulonglong
    L.fsp_plan_launches.argtypes = [vp]
    L.fsp_plan_launches.restype = i
    L.fsp_plan_set_wait_timeout.argtypes = [vp, d]
    L.fsp_plan_inject_stall.argtypes = [vp]
    vpp = ctypes.POINTER(vp)
    L.fsp_batch_create.argtypes = [vpp, vpp, vpp, vpp, i, vp]
    L.fsp_batch_launch.argtypes = [vp, vp]
    L.fsp_batch_wait.argtypes = [vp, vp]
    L.fsp_batch_set_timeout.argtypes = [vp, d]
    L.fsp_batch_inject_stall.argtypes = [vp]
    L.fsp_batch_set_form.argtypes = [vp, i]
    L.fsp_batch_set_form.restype = i
    L.fsp_batch_destroy.argtypes = [vp]
    L.fsp_solve_batched.argtypes = [vpp, vpp, vpp, i, vp]
    L.fsp_batch_autotune.argtypes = [vp, vp]
    L.fsp_batch_autotune.restype = i
    u64 = ctypes.c_uint64
    L.fsp_server_create.argtypes = [vpp, ctypes.c_size_t, i]
    L.fsp_server_submit.argtypes = [vp, i, d, i, i, vp, vp, ctypes.POINTER(u64)]
    L.fsp_server_poll.argtypes = [vp, u64, ctypes.POINTER(i), ctypes.POINTER(d)]
    L.fsp_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.fsp_server_destroy.argtypes = [vp]
    L.fsp_autotune.argtypes = [i, i, vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.fsp_tuning_get.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.fsp_tuning_set.argtypes = [ctypes.c_char_p]
    for name in ("fsp_autotune", "fsp_tuning_get", "fsp_tuning_set"):
        getattr(L, name).restype = i
    for name in ("fsp_server_create", "fsp_server_submit", "fsp_server_poll", "fsp_server_get_stats",
                 "fsp_server_destroy"):
        getattr(L, name).restype = i
    for name in ("fsp_batch_create", "fsp_batch_launch", "fsp_batch_wait", "fsp_batch_set_timeout",
                 "fsp_batch_inject_stall", "fsp_batch_destroy", "fsp_solve_batched"):
        getattr(L, name).restype = i
    for name in ("fsp_plan_set_timing", "fsp_plan_create", "fsp_plan_create_aniso", "fsp_solve", "fsp_solve_host", "fsp_plan_sync", "fsp_plan_destroy",
                 "fsp_plan_spectrum", "fsp_kernel_T", "fsp_fft_c2c", "fsp_solve_noalloc", "fsp_plan_field_init",
                 "fsp_solve_field", "fsp_plan_set_wait_timeout", "fsp_plan_inject_stall"):
        getattr(L, name).restype = i
    _lib = L
    table = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.txt")
    if os.path.exists(table):  # pinned tile shapes measured on a GB300
        check(L.fsp_tuning_set(open(table, "rb").read()), "fsp_tuning_set")
    return L


def check(status, where=""):
    if status != FSP_OK:
        raise FspError(status, where)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(dtype):
    return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)


def _algo_code(algo):
    return ALGOS[algo] if isinstance(algo, str) else int(algo)


def torch_dtype(dtype):
    import torch
    return torch.float32 if _dtype_code(dtype) == 1 else torch.float64


SPECTRUM_FORMAT = "fsp-spectrum-1"  # the .npz layout of Plan.save


class Plan:
    """One solver instance for (N, L, algo, dtype): fsp_plan_create / fsp_solve / fsp_plan_destroy.

    N and L may also be 3-sequences (n_x, n_y, n_z) and (L_x, L_y, L_z): a
    non-cubic box (fsp_plan_create_aniso), arrays of shape (n_z, n_y, n_x)."""

    def __init__(self, N, L=1.0, algo="vg_dct", dtype="f64", h=None, stream=None):
        self.algo, self.dtype = algo, dtype
        self._p = ctypes.c_void_p()
        if isinstance(N, (tuple, list)):
            n = tuple(int(v) for v in N)
            Ls = tuple(float(v) for v in L) if isinstance(L, (tuple, list)) else (float(L),) * 3
            hs = tuple(Ls[a] / n[a] for a in range(3)) if h is None else tuple(float(v) for v in h)
            self.n3, self.h3, self.L3 = n, hs, Ls
            self.N, self.L, self.h = n[0], Ls[0], hs[0]
            self.shape = (n[2], n[1], n[0])
            check(lib().fsp_plan_create_aniso(ctypes.byref(self._p), n[0], n[1], n[2], hs[0], hs[1], hs[2],
                                              _algo_code(algo), _dtype_code(dtype), _stream_handle(stream)),
                  "fsp_plan_create_aniso")
        else:
            self.N, self.L = int(N), float(L)
            self.h = self.L / self.N if h is None else float(h)
            self.n3, self.h3, self.L3 = (self.N,) * 3, (self.h,) * 3, (self.L,) * 3
            self.shape = (self.N,) * 3
            check(lib().fsp_plan_create(ctypes.byref(self._p), self.N, self.L, self.h, _algo_code(algo),
                                        _dtype_code(dtype), _stream_handle(stream)), "fsp_plan_create")
        self.npoints = self.shape[0] * self.shape[1] * self.shape[2]

    @property
    def handle(self):
        return self._p

    @property
    def bytes(self):
        return int(lib().fsp_plan_bytes(self._p))

    @property
    def fast_path(self):
        """True when the specialised power-of-two kernels serve this plan."""
        return lib().fsp_plan_uses_fast_path(self._p) == 1

    def check_bounds(self):
        """Guard bytes changed around the plan's buffers (plans created with
        FSP_CHECK_BOUNDS=1 in the environment)."""
        bad = ctypes.c_ulonglong()
        check(lib().fsp_plan_check_bounds(self._p, ctypes.byref(bad)), "fsp_plan_check_bounds")
        return int(bad.value)

    @property
    def launches(self):
        """Kernel launches per solve (3 with the fused plane passes, else 5)."""
        return int(lib().fsp_plan_launches(self._p))

    @property
    def precompute_ms(self):
        return float(lib().fsp_plan_precompute_ms(self._p))

    def solve_into(self, rho, phi, stream=None):
        """Enqueue phi = G * rho on the stream (both CUDA tensors, contiguous)."""
        self._check_tensor(rho)
        self._check_tensor(phi)
        check(lib().fsp_solve(self._p, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                              _stream_handle(stream)), "fsp_solve")
        return phi

    def solve(self, rho, stream=None):
        import torch
        phi = torch.empty_like(rho)
        return self.solve_into(rho, phi, stream)

    def field_init(self, stream=None):
        """Plan-time set-up of field solves (fsp_plan_field_init)."""
        check(lib().fsp_plan_field_init(self._p, _stream_handle(stream)), "fsp_plan_field_init")

    def solve_field_into(self, rho, ex, ey, ez, phi=None, stream=None):
        """Enqueue E = -grad phi (and phi if given) of rho: fsp_solve_field."""
        for t in (rho, ex, ey, ez) + ((phi,) if phi is not None else ()):
            self._check_tensor(t)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        check(lib().fsp_solve_field(self._p, ptr(rho), ptr(phi), ptr(ex), ptr(ey), ptr(ez), _stream_handle(stream)),
              "fsp_solve_field")
        return (ex, ey, ez) if phi is None else (ex, ey, ez, phi)

    def solve_field(self, rho, with_phi=False, stream=None):
        """(E_x, E_y, E_z), or (E_x, E_y, E_z, phi) with with_phi, as new tensors."""
        import torch
        outs = [torch.empty_like(rho) for _ in range(4 if with_phi else 3)]
        return self.solve_field_into(rho, *outs[:3], phi=outs[3] if with_phi else None, stream=stream)

    def solve_host(self, rho_host, phi_host, stream=None):
        """Host arrays (numpy or CPU tensors, ideally pinned): copy in, solve, copy out."""
        rp = rho_host.data_ptr() if hasattr(rho_host, "data_ptr") else rho_host.ctypes.data
        pp = phi_host.data_ptr() if hasattr(phi_host, "data_ptr") else phi_host.ctypes.data
        check(lib().fsp_solve_host(self._p, ctypes.c_void_p(rp), ctypes.c_void_p(pp), _stream_handle(stream)),
              "fsp_solve_host")
        return phi_host

    def solve_host_many(self, rhos_host, phis_host, stream=None):
        """Pipelined solves of host arrays (copies overlap the solves)."""
        def ptr(t):
            return t.data_ptr() if hasattr(t, "data_ptr") else t.ctypes.data
        check(lib().fsp_solve_host_many(self._p, _ptr_array([ptr(r) for r in rhos_host]),
                                        _ptr_array([ptr(f) for f in phis_host]), len(rhos_host),
                                        _stream_handle(stream)), "fsp_solve_host_many")
        return phis_host

    def spectrum(self):
        import numpy as np
        out = np.empty(tuple(d + 1 for d in self.shape), dtype=np.float64)
        check(lib().fsp_plan_spectrum(self._p, ctypes.c_void_p(out.ctypes.data)), "fsp_plan_spectrum")
        return out

    @classmethod
    def from_spectrum(cls, N, L, algo, dtype, S, stream=None):
        """A cubic plan whose multiplier is the stored spectrum S ((N+1)^3
        doubles, as spectrum() returns them): fsp_plan_create_from_spectrum,
        one copy instead of the plan-time precompute."""
        import numpy as np
        N, L = int(N), float(L)
        S = np.ascontiguousarray(S, dtype=np.float64)
        if S.shape != (N + 1,) * 3:
            raise FspError(FSP_EINVAL, "spectrum must have shape %s, got %s" % ((N + 1,) * 3, S.shape))
        self = cls.__new__(cls)
        self.algo, self.dtype = algo, dtype
        self._p = ctypes.c_void_p()
        self.N, self.L, self.h = N, L, L / N
        self.n3, self.h3, self.L3 = (N,) * 3, (self.h,) * 3, (L,) * 3
        self.shape = (N,) * 3
        self.npoints = N ** 3
        check(lib().fsp_plan_create_from_spectrum(ctypes.byref(self._p), N, L, _algo_code(algo), _dtype_code(dtype),
                                                  ctypes.c_void_p(S.ctypes.data), _stream_handle(stream)),
              "fsp_plan_create_from_spectrum")
        return self

    def save(self, path):
        """Write the plan's (N, L, algo, dtype) and spectrum to a .npz file
        (cubic plans), for Plan.load to restore without the precompute."""
        import numpy as np
        if self.n3 != (self.N,) * 3 or self.L3 != (self.L,) * 3:
            raise FspError(FSP_EUNSUPPORTED, "save: cubic plans only")
        name = lambda table, v: next(k for k, c in table.items() if c == table.get(v, v))  # noqa: E731
        np.savez(path, format=np.array(SPECTRUM_FORMAT), N=np.int64(self.N), L=np.float64(self.L),
                 algo=np.array(name(ALGOS, self.algo)), dtype=np.array(name(DTYPES, self.dtype)), S=self.spectrum())

    @classmethod
    def load(cls, path, dtype=None, stream=None):
        """The plan a file of Plan.save describes, in its dtype or in `dtype`
        (an FP64 spectrum restores any dtype exactly as a fresh plan)."""
        import numpy as np
        with np.load(path, allow_pickle=False) as z:
            if str(z["format"]) != SPECTRUM_FORMAT:
                raise FspError(FSP_EINVAL, "not a spectrum file of this format: %r" % str(z["format"]))
            return cls.from_spectrum(int(z["N"]), float(z["L"]), str(z["algo"]),
                                     str(z["dtype"]) if dtype is None else dtype, z["S"], stream)

    def set_timing(self, events):
        """Record the 6 torch.cuda.Event objects around the 5 passes of each
        later solve (None turns the hook off)."""
        if events is None:
            check(lib().fsp_plan_set_timing(self._p, None, 0), "fsp_plan_set_timing")
            self._events = None
            return
        self._events = list(events)  # keep them alive while the hook is set
        arr = (ctypes.c_void_p * 6)(*[ctypes.c_void_p(e.cuda_event) for e in self._events])
        check(lib().fsp_plan_set_timing(self._p, arr, 6), "fsp_plan_set_timing")

    def sync(self, stream=None):
        check(lib().fsp_plan_sync(self._p, _stream_handle(stream)), "fsp_plan_sync")

    def close(self):
        if self._p is not None and self._p.value:
            check(lib().fsp_plan_destroy(self._p), "fsp_plan_destroy")
        self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t):
        import torch
        if not (t.is_cuda and t.is_contiguous() and t.dtype == torch_dtype(self.dtype) and t.numel() == self.npoints):
            raise FspError(FSP_EINVAL, "tensor must be a contiguous CUDA %s tensor of %d elements"
                           % (torch_dtype(self.dtype), self.npoints))


def kernel_T(N, L=1.0, algo="vg_dct", stream=None):
    """The FP64 real-space kernel T[m], m in [0,N]^3, computed on the device."""
    import torch
    t = torch.empty((N + 1,) * 3, dtype=torch.float64, device="cuda")
    check(lib().fsp_kernel_T(int(N), float(L), _algo_code(algo), ctypes.c_void_p(t.data_ptr()),
                             _stream_handle(stream)), "fsp_kernel_T")
    return t


def autotune(N, dtype="f32", stream=None):
    """Time the generic engine's tile shapes for (N, dtype); returns (lgL_row,
    lgL_col) and records them for plans created afterwards."""
    a, b = ctypes.c_int(), ctypes.c_int()
    check(lib().fsp_autotune(int(N), _dtype_code(dtype), _stream_handle(stream), ctypes.byref(a), ctypes.byref(b)),
          "fsp_autotune")
    return a.value, b.value


def tuning_get():
    """The tuning table as text ("N dtype lgL_row lgL_col" per line)."""
    n = ctypes.c_size_t()
    check(lib().fsp_tuning_get(None, 0, ctypes.byref(n)), "fsp_tuning_get")
    buf = ctypes.create_string_buffer(n.value)
    check(lib().fsp_tuning_get(buf, n.value, ctypes.byref(n)), "fsp_tuning_get")
    return buf.value.decode()


def tuning_set(text):
    """Merge table text into the tuning table (pins tile shapes)."""
    check(lib().fsp_tuning_set(text.encode() if isinstance(text, str) else text), "fsp_tuning_set")


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[ctypes.c_void_p(x) for x in xs])


class Batch:
    """Many solves of mixed N in one persistent launch, replayed as a CUDA graph
    (fsp_batch_create / fsp_batch_launch / fsp_batch_wait)."""

    def __init__(self, plans, rhos, phis, stream=None):
        if not (len(plans) == len(rhos) == len(phis)) or not plans:
            raise FspError(FSP_EINVAL, "Batch wants equal, non-empty lists")
        for p, r, f in zip(plans, rhos, phis):
            p._check_tensor(r)
            p._check_tensor(f)
        self.plans, self.rhos, self.phis = list(plans), list(rhos), list(phis)  # keep them alive
        self._b = ctypes.c_void_p()
        check(lib().fsp_batch_create(ctypes.byref(self._b), _ptr_array([p.handle.value for p in plans]),
                                     _ptr_array([r.data_ptr() for r in rhos]), _ptr_array([f.data_ptr() for f in phis]),
                                     len(plans), _stream_handle(stream)), "fsp_batch_create")

    def launch(self, stream=None):
        check(lib().fsp_batch_launch(self._b, _stream_handle(stream)), "fsp_batch_launch")

    def wait(self, stream=None):
        """Synchronise and return the device status (FSP_OK or FSP_ETIMEOUT)."""
        return int(lib().fsp_batch_wait(self._b, _stream_handle(stream)))

    def set_timeout(self, ms):
        check(lib().fsp_batch_set_timeout(self._b, float(ms)), "fsp_batch_set_timeout")

    def autotune(self, stream=None):
        """Tune the batch's tile shapes by timing its own launches."""
        check(lib().fsp_batch_autotune(self._b, _stream_handle(stream)), "fsp_batch_autotune")

    def inject_stall(self):
        check(lib().fsp_batch_inject_stall(self._b), "fsp_batch_inject_stall")

    def set_form(self, form):
        """0: one persistent kernel; 1: the solves' own launches on 8 streams."""
        check(lib().fsp_batch_set_form(self._b, int(form)), "fsp_batch_set_form")

    def close(self):
        if self._b is not None and self._b.value:
            check(lib().fsp_batch_destroy(self._b), "fsp_batch_destroy")
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans, rhos, phis, stream=None):
    """fsp_solve_batched: create, launch, wait and destroy a batch."""
    check(lib().fsp_solve_batched(_ptr_array([p.handle.value for p in plans]), _ptr_array([r.data_ptr() for r in rhos]),
                                  _ptr_array([f.data_ptr() for f in phis]), len(plans), _stream_handle(stream)),
          "fsp_solve_batched")
    return phis


class Server:
    """Continuous-batching solve server (fsp_server_*): submit requests of any
    size; a worker thread in the library admits them into free slots as slots
    and the device-memory budget allow, with spectra cached per
    (N, L, algo, dtype)."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, budget_bytes=100 << 30, max_slots=8):
        self._v = ctypes.c_void_p()
        check(lib().fsp_server_create(ctypes.byref(self._v), int(budget_bytes), int(max_slots)), "fsp_server_create")
        self._keep = {}

    def submit(self, rho, phi, L=1.0, algo="he", dtype="f32"):
        """Queue phi = G * rho (CUDA tensors of N^3 values); returns a ticket."""
        import torch
        N = round(rho.numel() ** (1.0 / 3.0))
        want = torch_dtype(dtype)
        for t in (rho, phi):
            if not (t.is_cuda and t.is_contiguous() and t.dtype == want and t.numel() == N ** 3):
                raise FspError(FSP_EINVAL, "Server.submit wants contiguous CUDA %s tensors of N^3 values" % want)
        tk = ctypes.c_uint64()
        check(lib().fsp_server_submit(self._v, int(N), float(L), _algo_code(algo), _dtype_code(dtype),
                                      ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                      ctypes.byref(tk)), "fsp_server_submit")
        self._keep[tk.value] = (rho, phi)
        return tk.value

    def poll(self, ticket):
        """(state, latency_ms, status); a finished ticket is reported once."""
        st, lat = ctypes.c_int(), ctypes.c_double()
        rc = lib().fsp_server_poll(self._v, ctypes.c_uint64(ticket), ctypes.byref(st), ctypes.byref(lat))
        if rc == FSP_EINVAL and ticket not in self._keep:
            raise FspError(rc, "fsp_server_poll: unknown ticket")
        if st.value >= self.DONE:
            self._keep.pop(ticket, None)
        return st.value, lat.value, rc

    def wait(self, ticket, timeout_s=120.0):
        """Busy-poll until the ticket finishes; returns its latency in ms."""
        import time
        t0 = time.perf_counter()
        while True:
            state, lat, rc = self.poll(ticket)
            if state >= self.DONE:
                check(rc, "server request")
                return lat
            if time.perf_counter() - t0 > timeout_s:
                raise FspError(FSP_ETIMEOUT, "Server.wait")
            time.sleep(0)

    def stats(self):
        s = ServerStats()
        check(lib().fsp_server_get_stats(self._v, ctypes.byref(s)), "fsp_server_get_stats")
        return {name: int(getattr(s, name)) for name, _ in ServerStats._fields_}

    def close(self):
        if self._v is not None and self._v.value:
            check(lib().fsp_server_destroy(self._v), "fsp_server_destroy")
        self._v = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_noalloc(S, rho, phi, stream=None):
    """FP64 solve for N <= 32 with no device allocation (fsp_solve_noalloc).

    S: CUDA float64 tensor of (N+1)^3 spectrum values (e.g. Plan.spectrum()
    copied to the device); rho, phi: CUDA float64 tensors of N^3 values.
    For callers that cannot allocate device memory; calls share one static
    scratch array, so calls that overlap on the GPU must not be issued."""
    import torch
    N = round(rho.numel() ** (1.0 / 3.0))
    for t in (S, rho, phi):
        if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.float64):
            raise FspError(FSP_EINVAL, "solve_noalloc wants contiguous CUDA float64 tensors")
    if rho.numel() != N ** 3 or phi.numel() != N ** 3 or S.numel() != (N + 1) ** 3:
        raise FspError(FSP_EINVAL, "solve_noalloc: sizes must be N^3, N^3 and (N+1)^3")
    check(lib().fsp_solve_noalloc(int(N), ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                  ctypes.c_void_p(phi.data_ptr()), _stream_handle(stream)), "fsp_solve_noalloc")
    return phi


def fft_c2c(x, sign=-1, stream=None):
    """Batched 1D FFTs along the last axis of a complex CUDA tensor (library kernels)."""
    import torch
    x = x.contiguous()
    dtype = 0 if x.dtype == torch.complex128 else 1
    if x.dtype not in (torch.complex128, torch.complex64):
        raise FspError(FSP_EINVAL, "fft_c2c wants complex64 or complex128")
    out = torch.empty_like(x)
    n = x.shape[-1]
    count = x.numel() // n if n else 0
    check(lib().fsp_fft_c2c(n, count, dtype, int(sign), ctypes.c_void_p(x.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "fsp_fft_c2c")
    return out


__all__ = ["autotune", "tuning_get", "tuning_set", "Plan", "Batch", "Server", "solve_batched", "FspError", "kernel_T", "fft_c2c", "solve_noalloc", "lib", "check", "library_path", "ALGOS", "DTYPES"]


def device_host_numa(device=None):
    """Host NUMA node closest to the GPU (-1 when unknown)."""
    import torch
    return int(lib().fsp_device_host_numa(torch.cuda.current_device() if device is None else int(device)))


class HostBuffer:
    """Pinned host memory bound to one NUMA node (fsp_host_alloc); `array`
    is a numpy view of it (shape, dtype).  numa_node=None: the node nearest
    the current GPU; -1: no binding."""

    def __init__(self, shape, dtype, numa_node=None):
        import numpy as np
        self.dtype = np.dtype(dtype)
        self.shape = tuple(shape)
        self.nbytes = int(np.prod(self.shape)) * self.dtype.itemsize
        self.numa_node = device_host_numa() if numa_node is None else int(numa_node)
        self._p = ctypes.c_void_p()
        check(lib().fsp_host_alloc(ctypes.byref(self._p), self.nbytes, self.numa_node), "fsp_host_alloc")
        buf = (ctypes.c_char * self.nbytes).from_address(self._p.value)
        self.array = np.frombuffer(buf, dtype=self.dtype).reshape(self.shape)

    def close(self):
        if self._p is not None and self._p.value:
            self.array = None
            check(lib().fsp_host_free(self._p, self.nbytes), "fsp_host_free")
        self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------- slab-decomposed solve --
def dist_partition(N, nranks, rank):
    """(z0, z1, kx0, kx1): the z-planes and half-spectrum columns of a rank."""
    v = [ctypes.c_int() for _ in range(4)]
    check(lib().fsp_dist_partition(int(N), int(nranks), int(rank), *[ctypes.byref(x) for x in v]),
          "fsp_dist_partition")
    return tuple(x.value for x in v)


def dist_block_elems(N, nranks, rank, phase, peer, sending):
    """Complex values of the block `rank` sends to (or receives from) `peer`."""
    n = int(lib().fsp_dist_block_elems(int(N), int(nranks), int(rank), int(phase), int(peer), int(bool(sending))))
    if n < 0:
        raise FspError(FSP_EINVAL, "fsp_dist_block_elems")
    return n


class DistPlan:
    """One rank's share of a slab-decomposed solve (fsp_dist_*).  The caller
    moves the blocks between ranks: `exchange_local` for ranks of one process,
    torch.distributed all-to-all for ranks on several GPUs."""

    def __init__(self, N, L=1.0, algo="vg_dct", dtype="f64", nranks=1, rank=0, stream=None):
        self.N, self.L, self.dtype, self.R, self.rank = int(N), float(L), dtype, int(nranks), int(rank)
        self._d = ctypes.c_void_p()
        check(lib().fsp_dist_create(ctypes.byref(self._d), self.N, self.L, _algo_code(algo), _dtype_code(dtype),
                                    self.R, self.rank, _stream_handle(stream)), "fsp_dist_create")
        self.z0, self.z1, self.kx0, self.kx1 = dist_partition(self.N, self.R, self.rank)

    def blocks(self, phase, sending):
        """Fresh device blocks of this rank for one phase, indexed by peer."""
        import torch
        ct = torch.complex128 if self.dtype == "f64" else torch.complex64
        return [torch.empty(max(1, dist_block_elems(self.N, self.R, self.rank, phase, q, sending)), dtype=ct,
                            device="cuda") for q in range(self.R)]

    def forward(self, rho_slab, send, stream=None):
        check(lib().fsp_dist_forward(self._d, ctypes.c_void_p(rho_slab.data_ptr()),
                                     _ptr_array([t.data_ptr() for t in send]), _stream_handle(stream)),
              "fsp_dist_forward")

    def middle(self, recv, send, stream=None):
        check(lib().fsp_dist_middle(self._d, _ptr_array([t.data_ptr() for t in recv]),
                                    _ptr_array([t.data_ptr() for t in send]), _stream_handle(stream)),
              "fsp_dist_middle")

    def backward(self, recv, phi_slab, stream=None):
        check(lib().fsp_dist_backward(self._d, _ptr_array([t.data_ptr() for t in recv]),
                                      ctypes.c_void_p(phi_slab.data_ptr()), _stream_handle(stream)),
              "fsp_dist_backward")

    def close(self):
        if self._d is not None and self._d.value:
            check(lib().fsp_dist_destroy(self._d), "fsp_dist_destroy")
        self._d = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exchange_local(sends, recvs):
    """The all-to-all of ranks that share one process: recvs[q][r] = sends[r][q]."""
    for r, row in enumerate(sends):
        for q, blk in enumerate(row):
            recvs[q][r].copy_(blk)


def solve_distributed_local(N, rho, L=1.0, algo="vg_dct", dtype="f64", nranks=2):
    """Emulate `nranks` ranks in this process on the current GPU: split rho
    (device, N^3) into z-slabs, run the three phases with device-to-device
    exchanges, gather phi."""
    import torch
    ranks = [DistPlan(N, L, algo, dtype, nranks, r) for r in range(nranks)]
    phi = torch.empty_like(rho)
    send0 = [p.blocks(0, True) for p in ranks]
    recv0 = [p.blocks(0, False) for p in ranks]
    for p, snd in zip(ranks, send0):
        p.forward(rho[p.z0:p.z1].clone(), snd)  # a fresh, aligned slab
    exchange_local(send0, recv0)
    send1 = [p.blocks(1, True) for p in ranks]
    recv1 = [p.blocks(1, False) for p in ranks]
    for p, rcv, snd in zip(ranks, recv0, send1):
        p.middle(rcv, snd)
    exchange_local(send1, recv1)
    for p, rcv in zip(ranks, recv1):
        out = torch.empty((p.z1 - p.z0,) + tuple(rho.shape[1:]), dtype=rho.dtype, device=rho.device)
        p.backward(rcv, out)
        phi[p.z0:p.z1] = out
    torch.cuda.synchronize()
    for p in ranks:
        p.close()
    return phi


def exchange_dist(sends, recvs, group=None):
    """The all-to-all of one rank among processes: recvs[q] receives rank q's
    block for this rank, sends[q] goes to rank q (torch.distributed point-to-
    point: NCCL for device blocks, gloo for host blocks)."""
    import torch
    import torch.distributed as dist
    me, R = dist.get_rank(group), dist.get_world_size(group)
    real = lambda t: torch.view_as_real(t) if t.is_complex() else t  # noqa: E731
    ops = []
    for q in range(R):
        if q == me:
            recvs[q].copy_(sends[q])
            continue
        ops.append(dist.P2POp(dist.isend, real(sends[q]).contiguous(), q, group=group))
        ops.append(dist.P2POp(dist.irecv, real(recvs[q]), q, group=group))
    # posted as one group: separate NCCL sends and receives would each wait
    # for a peer whose matching call is queued behind its own send
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
