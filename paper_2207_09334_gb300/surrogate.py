"""Design surrogate MLP over the C ABI (mlp_*): argument marshalling only.
The forward, backward and Adam kernels (tensor-core GEMMs included) run in
the library."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import check
from .sim import _stream_handle, torch_allocator

__all__ = ["Surrogate", "gemm_bf16"]


def gemm_bf16(A, B, out=None):
    """C = A @ B.T on the tensor cores; A [M,K], B [N,K] bfloat16 CUDA tensors."""
    import torch
    M, K = A.shape; N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    check(_lib.load().mlp_gemm_bf16(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                    C.c_void_p(out.data_ptr()), M, N, K,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


class Surrogate:
    """MLP n_in -> hidden -> hidden -> 1 (GELU), bf16 activations, fp32 master weights."""

    def __init__(self, n_in: int = 2048, hidden: int = 512, max_batch: int = 1024, seed: int = 0,
                 stream=None, use_torch_allocator: bool = True):
        import torch
        lib = _lib.load()
        self._lib = lib
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        check(lib.mlp_create(int(n_in), int(hidden), int(max_batch), int(seed),
                             C.byref(self._alloc.struct) if self._alloc else None, C.c_void_p(self.stream),
                             C.byref(h)))
        self.h = h
        self.n_in, self.hidden, self.max_batch = n_in, hidden, max_batch
        self.n_params = int(lib.mlp_num_params(h))
        self._loss = torch.zeros(1, device="cuda")

    def params(self):
        p = np.empty(self.n_params, np.float32)
        check(self._lib.mlp_get_params(self.h, p.ctypes.data, None))
        return p

    def grads(self):
        g = np.empty(self.n_params, np.float32)
        check(self._lib.mlp_get_params(self.h, None, g.ctypes.data))
        return g

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        check(self._lib.mlp_set_params(self.h, p.ctypes.data))

    def load_materials(self, mats):
        """mats: uint8 CUDA tensor [B, n_in/4] of material ids."""
        check(self._lib.mlp_encode(self.h, C.c_void_p(mats.data_ptr()), int(mats.shape[0])))

    def load_input(self, x_bf16):
        check(self._lib.mlp_set_input(self.h, C.c_void_p(x_bf16.data_ptr()), int(x_bf16.shape[0])))

    def forward(self, B: int, out=None):
        import torch
        if out is None:
            out = torch.empty(B, device="cuda")
        check(self._lib.mlp_forward(self.h, int(B), C.c_void_p(out.data_ptr())))
        return out

    def backward(self, target, B: int):
        check(self._lib.mlp_backward(self.h, C.c_void_p(target.data_ptr()), int(B),
                                     C.c_void_p(self._loss.data_ptr())))
        return self._loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        check(self._lib.mlp_adam(self.h, float(lr), float(beta1), float(beta2), float(eps)))

    def train_step(self, mats, target, lr=1e-3):
        self.load_materials(mats)
        loss = self.backward(target, mats.shape[0])
        self.adam(lr)
        return loss

    def forward_materials(self, mats, out=None):
        """Predictions for one batch of device materials [B, n_in/4] (uint8,
        contiguous), read in place by the first GEMM (no copy into the model)."""
        import torch
        if out is None:
            out = torch.empty(mats.shape[0], device="cuda")
        check(self._lib.mlp_forward_materials(self.h, C.c_void_p(mats.data_ptr()), int(mats.shape[0]),
                                              C.c_void_p(out.data_ptr())))
        return out

    def predict(self, mats, chunk=None):
        """Predictions for materials [N, n_in/4] (N a multiple of 128), in chunks of max_batch."""
        import torch
        N = mats.shape[0]
        chunk = chunk or self.max_batch
        out = torch.empty(N, device="cuda")
        mats = mats.contiguous()
        for s in range(0, N, chunk):
            e = min(N, s + chunk)
            self.forward_materials(mats[s:e], out[s:e])
        return out

    def sync(self):
        check(self._lib.mlp_sync(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._lib.mlp_destroy(self.h)
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
