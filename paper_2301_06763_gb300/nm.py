"""Python binding of libnestconv (the C ABI in include/nm.h).

Argument marshalling only: every step of a solve runs in the CUDA library.  The
library must have been built (``paper_2301_06763_gb300.build.build()``); when it
is missing this module raises instead of computing anything another way.

Tensors are PyTorch tensors (PyTorch provides device memory and streams):
``rho`` is (levels, N, N, N) float64 (FP64 plans) or float32 (FP32 plans),
contiguous, on the plan's device; ``phi`` is (levels, N, N, N) float64.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnestconv.so")

NM_OK, NM_EINVAL, NM_ENOMEM, NM_ECUDA, NM_ETIMEOUT, NM_EUNSUPPORTED = range(6)
FP64, FP32, FP64X = 0, 1, 2
ORIGINAL, DIPOLE_PAIR, DIPOLE_TRIPLE, DIPOLE_TRIPLE_DIRECT = 0, 1, 2, 3
TRILINEAR, DIAGONAL = 0, 1
_PREC = {"fp64": FP64, "fp32": FP32, "fp64x": FP64X}
_METHOD = {"original": ORIGINAL, "dipole": DIPOLE_PAIR, "dipole3": DIPOLE_TRIPLE,
           "dipole3_ds": DIPOLE_TRIPLE_DIRECT}
_INTERP = {"trilinear": TRILINEAR, "diagonal": DIAGONAL}


class Options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("N", ctypes.c_int), ("dx0", ctypes.c_double),
                ("G", ctypes.c_double), ("precision", ctypes.c_int), ("method", ctypes.c_int),
                ("interp", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int), ("radix", ctypes.c_int), ("tile", ctypes.c_int),
                ("pipeline", ctypes.c_int), ("fuse", ctypes.c_int)]

    def as_dict(self):
        return {"group": self.group, "radix": self.radix, "tile": self.tile, "pipeline": self.pipeline,
                "fuse": self.fuse}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64),
                ("units", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


class NMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status_string(status), message))
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnestconv.so is not built (%s); run "
                               "paper_2301_06763_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        st = ctypes.c_int
        sig = {
            "nm_default_options": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(Options)]),
            "nm_plan": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(P)]),
            "nm_plan_ex": (st, [ctypes.POINTER(Options), ctypes.POINTER(P)]),
            "nm_green": (st, [P, P]),
            "nm_potential": (st, [P, P, P, P]),
            "nm_potential_host": (st, [P, P, P, P]),
            "nm_acceleration": (st, [P, P, P, P]),
            "nm_debug_fail_alloc": (st, [ctypes.c_int]),
            "nm_debug_fft": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]),
            "nm_potential_host_many": (st, [P, ctypes.c_int, P, P, P]),
            "nm_acceleration_ex": (st, [P, P, P, ctypes.c_int, ctypes.c_int, P]),
            "nm_workspace_bytes": (st, [P, ctypes.POINTER(ctypes.c_size_t)]),
            "nm_spectrum_bytes": (st, [P, ctypes.POINTER(ctypes.c_size_t)]),
            "nm_batch_potential": (st, [ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(P),
                                        ctypes.POINTER(P), P]),
            "nm_get_green_octant": (st, [P, P]),
            "nm_get_options": (st, [P, ctypes.POINTER(Options)]),
            "nm_destroy": (st, [P]),
            "nm_footprint_bytes": (st, [ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_size_t)]),
            "nm_get_schedule": (st, [P, ctypes.POINTER(Schedule)]),
            "nm_set_schedule": (st, [P, ctypes.POINTER(Schedule)]),
            "nm_autotune": (st, [P, P, P, ctypes.c_int, P]),
            "nm_potential_noalloc": (st, [ctypes.POINTER(Options), P, P, P]),
            "nm_kernel_launches": (ctypes.c_uint64, []),
            "nm_device_status": (st, [ctypes.c_int]),
            "nm_debug_fault_timeout": (st, [ctypes.c_int]),
            "nm_profile_enable": (st, [ctypes.c_int]),
            "nm_profile_read": (st, [ctypes.POINTER(KernelStat), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]),
            "nm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "nm_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(s):
    return lib().nm_status_string(int(s)).decode()


def last_error():
    return lib().nm_last_error().decode()


def _check(status):
    if status != NM_OK:
        raise NMError(status, last_error())


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(lib().nm_kernel_launches())


def make_options(levels, N, dx0, G=1.0, precision="fp64", method="original", interp="diagonal"):
    o = Options()
    _check(lib().nm_default_options(int(levels), int(N), float(dx0), ctypes.byref(o)))
    o.G = float(G)
    o.precision = _PREC[precision]
    o.method = _METHOD[method]
    o.interp = _INTERP[interp]
    return o


def footprint_bytes(levels, N, dx0=1.0, G=1.0, precision="fp64", method="original", interp="diagonal"):
    """Device bytes a plan of this shape would allocate (default schedule)."""
    v = ctypes.c_size_t()
    _check(lib().nm_footprint_bytes(ctypes.byref(make_options(levels, N, dx0, G, precision, method, interp)),
                                    ctypes.byref(v)))
    return int(v.value)


def device_status(clear=True):
    """NM_OK, or NM_ETIMEOUT if a bounded device wait ran out (synchronises)."""
    return int(lib().nm_device_status(1 if clear else 0))


def debug_fault_timeout(on):
    """Test hook: make the TMA-fed kernels' waits run out (see nm.h)."""
    _check(lib().nm_debug_fault_timeout(1 if on else 0))


def debug_fail_alloc(n):
    """Test hook: the n-th next plan workspace allocation fails (see nm.h)."""
    _check(lib().nm_debug_fail_alloc(int(n)))


def debug_fft(data, inverse=False, stream=None):
    """Test hook: transform the rows of ``data`` (a contiguous CUDA complex64 or
    complex128 tensor of shape (lines, P)) in place with the passes' line
    transform."""
    import torch
    if not data.is_cuda or not data.is_contiguous() or data.dim() != 2 or \
            data.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("data must be a contiguous CUDA complex tensor of shape (lines, P)")
    prec = FP32 if data.dtype == torch.complex64 else FP64
    _check(lib().nm_debug_fft(int(data.shape[1]), prec, 1 if inverse else 0, int(data.shape[0]),
                              ctypes.c_void_p(data.data_ptr()), _stream_handle(stream)))
    return data


def profile_enable(on=True):
    """Bracket every library kernel with CUDA events (see nm_profile_enable)."""
    _check(lib().nm_profile_enable(1 if on else 0))


def profile_read():
    """{kernel name: (launches, units, total_ms)} since profile_enable(True)."""
    cap = 256
    arr = (KernelStat * cap)()
    n = ctypes.c_int()
    _check(lib().nm_profile_read(arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), int(arr[i].units), float(arr[i].total_ms))
            for i in range(min(n.value, cap))}


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """One nested mesh: ``levels`` levels of N^3 cells, coarsest cell ``dx0``."""

    def __init__(self, levels, N, dx0, G=1.0, precision="fp64", method="original", interp="diagonal"):
        o = make_options(levels, N, dx0, G, precision, method, interp)
        h = ctypes.c_void_p()
        _check(lib().nm_plan_ex(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.levels, self.N, self.dx0, self.G = int(levels), int(N), float(dx0), float(G)
        self.precision, self.method, self.interp = precision, method, interp

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    @property
    def shape(self):
        return (self.levels, self.N, self.N, self.N)

    @property
    def rho_dtype(self):
        import torch
        return torch.float32 if self.precision == "fp32" else torch.float64

    def green(self, stream=None):
        _check(lib().nm_green(self.handle, _stream_handle(stream)))

    def _check_tensor(self, t, dtype, name):
        if t.dtype != dtype or tuple(t.shape) != self.shape or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("%s must be a contiguous CUDA %s tensor of shape %s" % (name, dtype, self.shape))

    def potential(self, rho, phi=None, stream=None):
        """Solve on the device; returns ``phi`` (allocated when not given)."""
        import torch
        self._check_tensor(rho, self.rho_dtype, "rho")
        if phi is None:
            phi = torch.empty(self.shape, dtype=torch.float64, device=rho.device)
        self._check_tensor(phi, torch.float64, "phi")
        _check(lib().nm_potential(self.handle, ctypes.c_void_p(rho.data_ptr()),
                                  ctypes.c_void_p(phi.data_ptr()), _stream_handle(stream)))
        return phi

    def acceleration(self, phi, g=None, stream=None, coarse_side="mean", iters=32):
        """g = -grad Phi ((levels, 3, N, N, N) float64) of a potential from
        ``potential``; coarse_side "mean" (method B) or "flux" (method C,
        ``iters`` sweeps)."""
        import torch
        self._check_tensor(phi, torch.float64, "phi")
        if g is None:
            g = torch.empty((self.levels, 3, self.N, self.N, self.N), dtype=torch.float64, device=phi.device)
        if g.dtype != torch.float64 or tuple(g.shape) != (self.levels, 3, self.N, self.N, self.N) \
                or not g.is_contiguous() or not g.is_cuda:
            raise ValueError("g must be a contiguous CUDA float64 tensor of shape (levels, 3, N, N, N)")
        side = {"mean": 0, "flux": 1}[coarse_side]
        _check(lib().nm_acceleration_ex(self.handle, ctypes.c_void_p(phi.data_ptr()),
                                        ctypes.c_void_p(g.data_ptr()), side, int(iters), _stream_handle(stream)))
        return g

    def potential_host(self, rho, phi=None, stream=None):
        """Solve from host memory (numpy arrays or CPU tensors); synchronous."""
        rho_np = rho.numpy() if hasattr(rho, "numpy") and not isinstance(rho, np.ndarray) else rho
        want = np.float32 if self.precision == "fp32" else np.float64
        if rho_np.dtype != want or rho_np.shape != self.shape or not rho_np.flags.c_contiguous:
            raise ValueError("rho must be a C-contiguous %s array of shape %s" % (want, self.shape))
        if phi is None:
            phi = np.empty(self.shape, dtype=np.float64)
        phi_np = phi.numpy() if hasattr(phi, "numpy") and not isinstance(phi, np.ndarray) else phi
        if phi_np.dtype != np.float64 or phi_np.shape != self.shape or not phi_np.flags.c_contiguous:
            raise ValueError("phi must be a C-contiguous float64 array of shape %s" % (self.shape,))
        _check(lib().nm_potential_host(self.handle, ctypes.c_void_p(rho_np.ctypes.data),
                                       ctypes.c_void_p(phi_np.ctypes.data), _stream_handle(stream)))
        return phi

    def potential_host_many(self, rhos, phis, stream=None):
        """len(rhos) solves from host memory, uploads and downloads overlapped
        with the solves (page-locked buffers: CPU tensors from pin_memory());
        synchronous."""
        want = np.float32 if self.precision == "fp32" else np.float64
        n = len(rhos)
        if len(phis) != n:
            raise ValueError("rhos and phis differ in length")
        rp, pp = (ctypes.c_void_p * max(n, 1))(), (ctypes.c_void_p * max(n, 1))()
        for i, (r, f) in enumerate(zip(rhos, phis)):
            rn = r.numpy() if hasattr(r, "numpy") and not isinstance(r, np.ndarray) else r
            fn = f.numpy() if hasattr(f, "numpy") and not isinstance(f, np.ndarray) else f
            if rn.dtype != want or rn.shape != self.shape or not rn.flags.c_contiguous:
                raise ValueError("rho must be a C-contiguous %s array of shape %s" % (want, self.shape))
            if fn.dtype != np.float64 or fn.shape != self.shape or not fn.flags.c_contiguous:
                raise ValueError("phi must be a C-contiguous float64 array of shape %s" % (self.shape,))
            rp[i], pp[i] = rn.ctypes.data, fn.ctypes.data
        _check(lib().nm_potential_host_many(self.handle, n, rp, pp, _stream_handle(stream)))
        return phis

    def schedule(self):
        sc = Schedule()
        _check(lib().nm_get_schedule(self.handle, ctypes.byref(sc)))
        return sc.as_dict()

    def set_schedule(self, group, radix, tile, pipeline=0, fuse=0):
        sc = Schedule(int(group), int(radix), int(tile), int(pipeline), int(fuse))
        _check(lib().nm_set_schedule(self.handle, ctypes.byref(sc)))

    def autotune(self, rho, phi=None, reps=3, stream=None):
        """Time the candidate schedules on these buffers, keep the fastest."""
        import torch
        self._check_tensor(rho, self.rho_dtype, "rho")
        if phi is None:
            phi = torch.empty(self.shape, dtype=torch.float64, device=rho.device)
        self._check_tensor(phi, torch.float64, "phi")
        _check(lib().nm_autotune(self.handle, ctypes.c_void_p(rho.data_ptr()),
                                 ctypes.c_void_p(phi.data_ptr()), int(reps), _stream_handle(stream)))
        return self.schedule()

    def workspace_bytes(self):
        v = ctypes.c_size_t()
        _check(lib().nm_workspace_bytes(self.handle, ctypes.byref(v)))
        return int(v.value)

    def spectrum_bytes(self):
        v = ctypes.c_size_t()
        _check(lib().nm_spectrum_bytes(self.handle, ctypes.byref(v)))
        return int(v.value)

    def green_octant(self):
        out = np.empty((self.N + 1,) * 3, dtype=np.float64)
        _check(lib().nm_get_green_octant(self.handle, ctypes.c_void_p(out.ctypes.data)))
        return out

    def close(self):
        if self._h is not None:
            _check(lib().nm_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_potential(plans, rhos, phis, stream=None):
    """Solve several meshes in one batched schedule (see nm_batch_potential)."""
    n = len(plans)
    if not (len(rhos) == len(phis) == n):
        raise ValueError("plans, rhos and phis must have the same length")
    for p, r, f in zip(plans, rhos, phis):
        p._check_tensor(r, p.rho_dtype, "rho")
        import torch
        p._check_tensor(f, torch.float64, "phi")
    H = (ctypes.c_void_p * max(n, 1))(*[p.handle for p in plans])
    R = (ctypes.c_void_p * max(n, 1))(*[r.data_ptr() for r in rhos])
    F = (ctypes.c_void_p * max(n, 1))(*[f.data_ptr() for f in phis])
    _check(lib().nm_batch_potential(n, H, R, F, _stream_handle(stream)))
    return phis
