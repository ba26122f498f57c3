"""Batched voxel-robot populations over the C ABI (msb_*): argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MsbInfo, MsbVoxelSpec, check
from .sim import _stream_handle, make_params, torch_allocator

__all__ = ["Population"]


class Population:
    """A population of independent voxel robots advanced by one persistent launch.

    designs: list of (materials (nz,ny,nx) uint8, phase (nz,ny,nx) float) pairs;
    materials: (n_mat, 3) table of (k, c, amplitude), row 0 = empty;
    logk: optional list of (nz,ny,nx) per-voxel log-stiffness overrides.
    """

    def __init__(self, designs, materials, freq: float, voxel_edge: float, voxel_mass: float,
                 params: dict, logk=None, stream=None, use_torch_allocator: bool = True):
        lib = _lib.load()
        self._lib = lib
        dims = np.array([[m.shape[2], m.shape[1], m.shape[0]] for m, _ in designs], np.int32)
        mats = np.ascontiguousarray(np.concatenate([np.asarray(m, np.uint8).ravel() for m, _ in designs]))
        phase = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float32).ravel() for _, p in designs]))
        lk = None
        if logk is not None:
            lk = np.ascontiguousarray(np.concatenate([np.asarray(q, np.float32).ravel() for q in logk]))
            assert lk.size == mats.size
        tab = np.asarray(materials, np.float32)
        self._k = np.ascontiguousarray(tab[:, 0]); self._c = np.ascontiguousarray(tab[:, 1])
        self._a = np.ascontiguousarray(tab[:, 2])
        spec = MsbVoxelSpec(float(voxel_edge), float(voxel_mass), float(freq), tab.shape[0],
                            self._k.ctypes.data, self._c.ctypes.data, self._a.ctypes.data)
        self._params = make_params(params)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        check(lib.msb_create(C.byref(self._params), C.byref(spec), len(designs), dims.ctypes.data,
                             mats.ctypes.data, phase.ctypes.data, None if lk is None else lk.ctypes.data,
                             C.byref(self._alloc.struct) if self._alloc else None, C.c_void_p(self.stream),
                             C.byref(h)))
        self.h = h
        self.n_robots = len(designs)

    def autotune(self, sample_steps: int = 100, policy: int = 0):
        check(self._lib.msb_autotune(self.h, int(sample_steps), int(policy)))

    def set_threads(self, threads: int):
        """CTA size of the persistent kernel: 512 or 1024 threads."""
        check(self._lib.msb_set_threads(self.h, int(threads)))

    def run(self, nsteps: int):
        check(self._lib.msb_run(self.h, int(nsteps)))

    def run_loop(self, nsteps: int):
        check(self._lib.msb_run_loop(self.h, int(nsteps)))

    def com_travel(self, out=None):
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            check(self._lib.msb_com_travel(self.h, C.c_void_p(out.data_ptr()), 1))
            return out
        o = np.empty(self.n_robots, np.float32)
        check(self._lib.msb_com_travel(self.h, o.ctypes.data, 0))
        return o

    def robot_info(self, r: int):
        n = C.c_int32(); first = C.c_int64()
        check(self._lib.msb_robot_info(self.h, int(r), C.byref(n), C.byref(first)))
        return n.value, first.value

    def get_state(self):
        inf = self.info()
        x = np.empty((inf["n_masses"], 3), np.float32); v = np.empty_like(x)
        check(self._lib.msb_get_state(self.h, x.ctypes.data, v.ctypes.data))
        return x, v

    def robot_state(self, r: int, x=None, v=None):
        if x is None:
            x, v = self.get_state()
        n, first = self.robot_info(r)
        return x[first:first + n], v[first:first + n]

    def reset(self):
        check(self._lib.msb_reset(self.h))

    def info(self) -> dict:
        inf = MsbInfo()
        check(self._lib.msb_get_info(self.h, C.byref(inf)))
        return {name: getattr(inf, name) for name, _ in MsbInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._lib.msb_destroy(self.h)
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
