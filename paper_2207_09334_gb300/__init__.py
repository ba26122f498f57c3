"""GB300-native mass-spring simulation (Cronos, arXiv 2207.09334).

The explicit mass-spring step runs in hand-written sm_103a CUDA kernels
behind the C ABI declared in include/cronos_ms.h; this package is its thin
Python binding.  There is no CPU fallback: if the compiled library is
missing, loading fails.
"""
from ._lib import MsError, library_path, load  # noqa: F401
from .sim import Sim, make_params, torch_allocator  # noqa: F401
from .batch import Population  # noqa: F401
from .adjoint import Adjoint, RolloutLoss  # noqa: F401
from .surrogate import Surrogate, gemm_bf16  # noqa: F401

__version__ = "0.1.0"
