"""Python face of the mass-spring library: argument marshalling over the C ABI.

Every step of the simulation runs in the library's CUDA kernels; this module
only converts numpy / torch arguments into pointers and sizes.  PyTorch
supplies the CUDA stream and, through the allocator hook, device memory from
its caching allocator.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MsAllocator, MsInfo, MsParams, check

__all__ = ["Sim", "make_params", "torch_allocator"]


ORDERS = {None: 0, False: 0, "auto": 0, True: 1, "morton": 1, "caller": 2}
KERNELS = {None: 0, "auto": 0, "gather": 1, "tiled": 2, "persistent": 3, "lattice": 4}


INTEGRATORS = {"symplectic_euler": 0, "forward_euler": 1, "verlet": 2, "rk4": 3}


def make_params(params: dict, reorder=None, strict_stability: bool = False, kernel=None,
                integrator="symplectic_euler") -> MsParams:
    """reorder: None/False = library default, True/"morton", or "caller";
    kernel: None/"auto", "gather", "tiled", "persistent" or "lattice"."""
    p = MsParams()
    p.dt = float(params["dt"])
    for a in range(3):
        p.g[a] = float(params["g"][a])
    p.k_c = float(params.get("k_c", 0.0))
    p.mu = float(params.get("mu", 0.0))
    p.vel_damping = float(params.get("vel_damping", 0.0))
    p.contact_on = 1 if params.get("contact", False) else 0
    p.integrator = INTEGRATORS[integrator] if isinstance(integrator, str) else int(integrator)
    p.strict_stability = 1 if strict_stability else 0
    p.reorder = ORDERS[reorder]
    p.kernel = KERNELS[kernel]
    return p


class _TorchAllocator:
    """ms_allocator backed by torch's CUDA caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self._alloc = _lib.ALLOC_FN(self._do_alloc)
        self._free = _lib.FREE_FN(self._do_free)
        self.struct = MsAllocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, stream, ctx):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:
            return None

    def _do_free(self, ptr, nbytes, stream, ctx):
        try:
            self._torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass


_ALLOCATOR = None


def torch_allocator() -> _TorchAllocator:
    global _ALLOCATOR
    if _ALLOCATOR is None:
        _ALLOCATOR = _TorchAllocator()
    return _ALLOCATOR


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a if shape is None else a.reshape(shape)


def _torch():
    import torch
    return torch


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Sim:
    """One mass-spring system resident on the GPU (ms_create ... ms_destroy).

    system: dict of arrays (x, v, m, fixed, [fext], ij, k, c, L0, [A, phi, freq]);
    c may be a scalar (uniform damping).  Materials form instead of k / c:
    mat (S,) ids with tables mat_k, [mat_c], [mat_L0scale] (ms_create_materials).  params: dt, g, k_c, mu, vel_damping, contact.
    """

    def __init__(self, system: dict, params: dict, reorder=None, stream=None,
                 use_torch_allocator: bool = True, strict_stability: bool = False, kernel=None,
                 integrator="symplectic_euler"):
        lib = _lib.load()
        self._lib = lib
        x = _f32(system["x"], (-1, 3)); N = x.shape[0]
        v = _f32(system["v"], (N, 3)); m = _f32(system["m"], (N,))
        fixed = np.ascontiguousarray(system.get("fixed", np.zeros(N)), np.uint8)
        fext = system.get("fext")
        fext = None if fext is None else _f32(fext, (N, 3))
        ij = np.ascontiguousarray(system["ij"], np.int32).reshape(-1, 2); S = ij.shape[0]
        if system.get("mat") is not None:       # materials form: ms_create_materials
            self._init_materials(system, params, reorder, stream, use_torch_allocator, strict_stability, kernel,
                                 integrator, x, v, m, fixed, fext, ij)
            return
        k = _f32(system["k"], (S,))
        c = system.get("c", 0.0)
        c_uniform = 0.0
        if np.isscalar(c) or np.ndim(c) == 0:
            c_uniform, c = float(c), None
        elif system.get("c_uniform") is not None:
            c_uniform, c = float(system["c_uniform"]), None
        else:
            c = _f32(c, (S,))
        L0 = system.get("L0")
        L0 = None if L0 is None else _f32(L0, (S,))
        self.N, self.S = N, S
        self._params = make_params(params, reorder, strict_stability, kernel, integrator)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.stream = _stream_handle(stream)
        handle = C.c_void_p()
        check(lib.ms_create(C.byref(self._params), N, _ptr(x), _ptr(v), _ptr(m), _ptr(fixed), _ptr(fext),
                            S, _ptr(ij), _ptr(k), _ptr(c), float(c_uniform), _ptr(L0),
                            C.byref(self._alloc.struct) if self._alloc else None,
                            C.c_void_p(self.stream), C.byref(handle)))
        self.h = handle
        if system.get("A") is not None:
            self.set_actuation(system.get("freq", 0.0), system["A"], system["phi"])

    def _init_materials(self, system, params, reorder, stream, use_torch_allocator, strict_stability, kernel,
                        integrator, x, v, m, fixed, fext, ij):
        """system["mat"] (S,) material ids with tables mat_k, [mat_c], [mat_L0scale]
        and optional per-spring base rest lengths L0."""
        lib = self._lib
        N, S = x.shape[0], ij.shape[0]
        mat = np.ascontiguousarray(system["mat"], np.uint16).reshape(S)
        mat_k = _f32(system["mat_k"]); n_mat = mat_k.shape[0]
        mat_c = None if system.get("mat_c") is None else _f32(system["mat_c"], (n_mat,))
        scale = None if system.get("mat_L0scale") is None else _f32(system["mat_L0scale"], (n_mat,))
        L0 = system.get("L0")
        L0 = None if L0 is None else _f32(L0, (S,))
        self.N, self.S = N, S
        self._params = make_params(params, reorder, strict_stability, kernel, integrator)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.stream = _stream_handle(stream)
        handle = C.c_void_p()
        check(lib.ms_create_materials(C.byref(self._params), N, _ptr(x), _ptr(v), _ptr(m), _ptr(fixed), _ptr(fext),
                                      S, _ptr(ij), _ptr(mat), int(n_mat), _ptr(mat_k), _ptr(mat_c), _ptr(scale),
                                      _ptr(L0), C.byref(self._alloc.struct) if self._alloc else None,
                                      C.c_void_p(self.stream), C.byref(handle)))
        self.h = handle
        if system.get("A") is not None:
            self.set_actuation(system.get("freq", 0.0), system["A"], system["phi"])

    # -- C ABI wrappers ---------------------------------------------------
    def set_actuation(self, freq: float, amp=None, phase=None):
        if amp is None:
            check(self._lib.ms_set_actuation(self.h, 0.0, None, None))
            return
        amp = _f32(amp, (self.S,)); phase = _f32(phase, (self.S,))
        check(self._lib.ms_set_actuation(self.h, float(freq), _ptr(amp), _ptr(phase)))

    def step(self, nsteps: int = 1):
        check(self._lib.ms_step(self.h, int(nsteps)))

    def get_state(self, x=None, v=None):
        """Host copy (numpy float32 (N,3)) of positions and velocities, or, if
        torch CUDA tensors are given, a stream-ordered device copy into them."""
        if x is not None and hasattr(x, "is_cuda") and x.is_cuda:
            check(self._lib.ms_get_state(self.h, C.c_void_p(x.data_ptr()),
                                         None if v is None else C.c_void_p(v.data_ptr()), 1))
            return x, v
        if x is not None and hasattr(x, "data_ptr"):          # pinned torch host tensors
            check(self._lib.ms_get_state(self.h, C.c_void_p(x.data_ptr()),
                                         None if v is None else C.c_void_p(v.data_ptr()), 0))
            return x, v
        xo = np.empty((self.N, 3), np.float32); vo = np.empty((self.N, 3), np.float32)
        check(self._lib.ms_get_state(self.h, _ptr(xo), _ptr(vo), 0))
        return xo, vo

    def set_state(self, x=None, v=None):
        if (x is not None and hasattr(x, "is_cuda") and x.is_cuda):
            check(self._lib.ms_set_state(self.h, C.c_void_p(x.data_ptr()),
                                         None if v is None else C.c_void_p(v.data_ptr()), 1))
            return
        if x is not None and hasattr(x, "data_ptr"):
            check(self._lib.ms_set_state(self.h, C.c_void_p(x.data_ptr()),
                                         None if v is None else C.c_void_p(v.data_ptr()), 0))
            return
        xa = None if x is None else _f32(x, (self.N, 3))
        va = None if v is None else _f32(v, (self.N, 3))
        check(self._lib.ms_set_state(self.h, _ptr(xa), _ptr(va), 0))

    def sync(self):
        check(self._lib.ms_sync(self.h))

    def set_wait_limit(self, max_polls: int = 0):
        """Polls of a bounded device-side wait (the persistent grid kernel's
        barrier) before it gives up; 0 = the default."""
        check(self._lib.ms_set_wait_limit(self.h, int(max_polls)))

    def test_barrier_deficit(self, missing: int):
        """Failure-detection test hook: the grid barrier waits for `missing`
        arrivals that never come, so its bounded waits run out."""
        check(self._lib.ms_test_barrier_deficit(self.h, int(missing)))

    def energy(self, out=None):
        """(kinetic, elastic, gravitational, ground) energy of the current
        state, reduced on the device.  With a CUDA float64 tensor `out` of 4
        elements (e.g. a row of a preallocated trace) the result is written
        there without a host copy or synchronisation; otherwise a tuple."""
        if out is not None:
            if not (hasattr(out, "is_cuda") and out.is_cuda and out.dtype == _torch().float64 and out.numel() >= 4
                    and out.is_contiguous()):
                raise ValueError("out must be a contiguous CUDA float64 tensor of at least 4 elements")
            check(self._lib.ms_energy(self.h, C.c_void_p(out.data_ptr()), 1))
            return out
        e = np.empty(4, np.float64)
        check(self._lib.ms_energy(self.h, _ptr(e), 0))
        return tuple(float(q) for q in e)

    def trace(self, masses, capacity: int):
        """Record the positions of `masses` (caller indices) after each of the
        next `capacity` steps; an empty list switches tracing off."""
        idx = np.ascontiguousarray(np.asarray(masses, np.int32).ravel())
        self._trace_n = int(idx.size)
        check(self._lib.ms_trace_set(self.h, _ptr(idx) if idx.size else None, int(idx.size), int(capacity)))

    def get_trace(self):
        """(steps, len(masses), 3) float32 positions recorded since trace()."""
        n = C.c_int32(0)
        check(self._lib.ms_trace_get(self.h, None, C.byref(n), 0))
        out = np.empty((n.value, getattr(self, "_trace_n", 0), 3), np.float32)
        if n.value:
            check(self._lib.ms_trace_get(self.h, _ptr(out), C.byref(n), 0))
        return out

    def info(self) -> dict:
        inf = MsInfo()
        check(self._lib.ms_get_info(self.h, C.byref(inf)))
        return {name: getattr(inf, name) for name, _ in MsInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._lib.ms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
