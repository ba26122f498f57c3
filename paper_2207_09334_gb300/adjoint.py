"""Gradients of voxel-robot rollouts over the C ABI (msa_*), and a
torch.autograd.Function around them.  Argument marshalling only: the forward
rollout, the checkpointing and the reverse pass run in the library's kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MsbVoxelSpec, check
from .sim import _stream_handle, make_params, torch_allocator

__all__ = ["Adjoint", "RolloutLoss"]


class Adjoint:
    """Reverse-mode gradients of per-robot rollout losses.

    materials: list of (nz,ny,nx) uint8 grids (the population's structure);
    the phases and log-stiffnesses are the differentiable parameters passed
    to gradients().
    """

    def __init__(self, materials, material_table, freq, voxel_edge, voxel_mass, params,
                 checkpoint_every: int = 100, max_steps: int = 2000, stream=None,
                 use_torch_allocator: bool = True, threads: int = 0):
        lib = _lib.load()
        self._lib = lib
        self.dims = np.array([[m.shape[2], m.shape[1], m.shape[0]] for m in materials], np.int32)
        mats = np.ascontiguousarray(np.concatenate([np.asarray(m, np.uint8).ravel() for m in materials]))
        tab = np.asarray(material_table, np.float32)
        self._k = np.ascontiguousarray(tab[:, 0]); self._c = np.ascontiguousarray(tab[:, 1])
        self._a = np.ascontiguousarray(tab[:, 2])
        spec = MsbVoxelSpec(float(voxel_edge), float(voxel_mass), float(freq), tab.shape[0],
                            self._k.ctypes.data, self._c.ctypes.data, self._a.ctypes.data)
        self._params = make_params(params)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        check(lib.msa_create(C.byref(self._params), C.byref(spec), len(materials), self.dims.ctypes.data,
                             mats.ctypes.data, int(checkpoint_every), int(max_steps),
                             C.byref(self._alloc.struct) if self._alloc else None, C.c_void_p(self.stream),
                             C.byref(h)))
        self.h = h
        self.n_robots = len(materials)
        nv = C.c_int64(); nm = C.c_int64()
        check(lib.msa_sizes(h, C.byref(nv), C.byref(nm)))
        self.n_voxels, self.n_masses = nv.value, nm.value
        counts = self.dims.prod(axis=1)
        self.voxel_robot = np.repeat(np.arange(self.n_robots), counts)
        if threads:
            check(lib.msa_set_threads(h, int(threads)))

    @property
    def threads(self) -> int:
        """Threads per robot of the adjoint kernel (256, 512, 768 or 1024;
        chosen from the population unless given to the constructor)."""
        return int(self._lib.msa_threads(self.h))

    def gradients(self, nsteps: int, phase, logk, seed_x=None):
        """Returns (loss[n_robots], d loss_r / d phase, d loss_r / d logk).
        numpy in -> numpy out (host); torch CUDA tensors in -> torch out (device)."""
        if hasattr(phase, "is_cuda") and phase.is_cuda:
            import torch
            phase = phase.detach().contiguous().float(); logk = logk.detach().contiguous().float()
            loss = torch.empty(self.n_robots, device=phase.device)
            gp = torch.empty_like(phase); gk = torch.empty_like(logk)
            sx = None if seed_x is None else seed_x.detach().contiguous().float()
            check(self._lib.msa_gradients(self.h, int(nsteps), C.c_void_p(phase.data_ptr()),
                                          C.c_void_p(logk.data_ptr()),
                                          None if sx is None else C.c_void_p(sx.data_ptr()),
                                          C.c_void_p(loss.data_ptr()), C.c_void_p(gp.data_ptr()),
                                          C.c_void_p(gk.data_ptr()), 1))
            return loss, gp, gk
        phase = np.ascontiguousarray(phase, np.float32).ravel()
        logk = np.ascontiguousarray(logk, np.float32).ravel()
        assert phase.size == self.n_voxels and logk.size == self.n_voxels
        sx = None if seed_x is None else np.ascontiguousarray(seed_x, np.float32).reshape(self.n_masses, 3)
        loss = np.empty(self.n_robots, np.float32)
        gp = np.empty(self.n_voxels, np.float32); gk = np.empty(self.n_voxels, np.float32)
        check(self._lib.msa_gradients(self.h, int(nsteps), phase.ctypes.data, logk.ctypes.data,
                                      None if sx is None else sx.ctypes.data, loss.ctypes.data,
                                      gp.ctypes.data, gk.ctypes.data, 0))
        return loss, gp, gk

    def close(self):
        if getattr(self, "h", None):
            self._lib.msa_destroy(self.h)
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


def _make_function():
    import torch

    class RolloutLoss(torch.autograd.Function):
        """loss[r] = centre-of-mass x-travel of robot r after nsteps (CUDA
        tensors phase, logk over all voxels); backward through the adjoint."""

        @staticmethod
        def forward(ctx, phase, logk, adj: Adjoint, nsteps: int):
            loss, gp, gk = adj.gradients(nsteps, phase, logk)
            ctx.save_for_backward(gp, gk)
            ctx.vr = torch.as_tensor(adj.voxel_robot, device=phase.device)
            return loss

        @staticmethod
        def backward(ctx, grad_loss):
            gp, gk = ctx.saved_tensors
            w = grad_loss[ctx.vr]
            return w * gp, w * gk, None, None

    return RolloutLoss


class _Lazy:
    _fn = None

    def apply(self, *args):
        if _Lazy._fn is None:
            _Lazy._fn = _make_function()
        return _Lazy._fn.apply(*args)


RolloutLoss = _Lazy()
