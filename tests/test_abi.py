"""The C-ABI library loads and exports every declared symbol; host-side input
validation returns status codes (no GPU needed: validation runs before any
CUDA call)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_09334_gb300 import build
    build.build()
    from paper_2207_09334_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", src):
            name = m.group(1)
            pre = src[:m.start()].rstrip()
            if name in ("if", "sizeof", "defined") or pre.endswith("(*") or pre.endswith("*)"):
                continue
            if re.match(r"(ms|msb|msa|mlp)_", name):
                names.append(name)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ms_create" in names and "ms_step" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_names_match_header():
    from paper_2207_09334_gb300 import _lib
    declared = set(declared_functions())
    for n in _lib.SIGNATURES:
        assert n in declared, f"binding declares {n}, header does not"


def _create(lib, N=2, x=None, mass=None, ij=None, k=None, dt=1e-3, strict=0, kc=0.0, kernel=0):
    from paper_2207_09334_gb300._lib import MsParams
    p = MsParams(); p.dt = dt; p.g[2] = -9.81; p.k_c = kc; p.contact_on = 1 if kc else 0
    p.strict_stability = strict
    p.kernel = kernel
    x = np.array(x if x is not None else [[0, 0, 0], [1, 0, 0]], np.float32)
    v = np.zeros_like(x)
    m = np.array(mass if mass is not None else [1.0] * len(x), np.float32)
    ij = np.array(ij if ij is not None else [[0, 1]], np.int32)
    k = np.array(k if k is not None else [1.0] * len(ij), np.float32)
    out = C.c_void_p()
    rc = lib.ms_create(C.byref(p), len(x), x.ctypes.data, v.ctypes.data, m.ctypes.data, None, None,
                       len(ij), ij.ctypes.data, k.ctypes.data, None, 0.0, None, None, None, C.byref(out))
    return rc, out


@pytest.mark.parametrize("kw,what", [
    (dict(x=[[0, 0, float("nan")], [1, 0, 0]]), "non-finite"),
    (dict(mass=[1.0, -1.0]), "mass"),
    (dict(ij=[[0, 2]]), "out of range"),
    (dict(ij=[[1, 1]]), "itself"),
    (dict(k=[-1.0]), "k must"),
    (dict(dt=0.0), "dt"),
])
def test_create_rejects_bad_input(lib, kw, what):
    rc, out = _create(lib, **kw)
    assert rc == 1 and not out.value
    assert what in lib.ms_last_error().decode()


def test_create_rejects_unstable_in_strict_mode(lib):
    rc, out = _create(lib, k=[1e9], dt=1e-2, strict=1)
    assert rc == 4 and not out.value
    assert "stability" in lib.ms_last_error().decode()


def test_gather_kernel_rejects_too_many_partners(lib):
    # mass 0 owns 40 distinct partners: beyond the gather layout's 31
    x = [[0, 0, 0]] + [[1 + i, 0, 0] for i in range(40)]
    rc, _ = _create(lib, x=x, ij=[[0, i + 1] for i in range(40)], kernel=1)
    assert rc == 1 and "31" in lib.ms_last_error().decode()


def test_tiled_kernel_rejects_tiles_that_overflow_shared_memory(lib):
    # a hub joined to 5000 far-away masses: the tile holding the hub needs
    # more halo entries than a CTA's shared memory holds
    n = 5001
    x = [[float(i), 0.0, 0.0] for i in range(n)]
    rc, _ = _create(lib, x=x, ij=[[0, i] for i in range(1, n)], kernel=2)
    assert rc == 1 and "shared-memory" in lib.ms_last_error().decode()


def test_persistent_kernel_takes_symplectic_euler_only(lib):
    from paper_2207_09334_gb300._lib import MsParams
    p = MsParams(); p.dt = 1e-3; p.kernel = 3; p.integrator = 2
    x = np.array([[0, 0, 0], [1, 0, 0]], np.float32); v = np.zeros_like(x)
    m = np.ones(2, np.float32); ij = np.array([[0, 1]], np.int32); k = np.ones(1, np.float32)
    out = C.c_void_p()
    rc = lib.ms_create(C.byref(p), 2, x.ctypes.data, v.ctypes.data, m.ctypes.data, None, None,
                       1, ij.ctypes.data, k.ctypes.data, None, 0.0, None, None, None, C.byref(out))
    assert rc == 1 and "symplectic Euler" in lib.ms_last_error().decode()


def test_bad_kernel_choice(lib):
    rc, _ = _create(lib, kernel=7)
    assert rc == 1 and "kernel" in lib.ms_last_error().decode()


def test_null_handles_are_errors(lib):
    assert lib.ms_step(None, 1) == 1
    assert lib.ms_sync(None) == 1
    assert lib.ms_destroy(None) == 0
    assert b"sm_103a" in lib.ms_version()
