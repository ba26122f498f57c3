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


def _create_materials(lib, mat, n_mat, mat_k, mat_c=None, scale=None):
    from paper_2207_09334_gb300._lib import MsParams
    p = MsParams(); p.dt = 1e-3; p.g[2] = -9.81
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32); v = np.zeros_like(x)
    m = np.ones(3, np.float32); ij = np.array([[0, 1], [1, 2]], np.int32)
    mat = np.array(mat, np.uint16); mk = np.array(mat_k, np.float32)
    mc = None if mat_c is None else np.array(mat_c, np.float32)
    sc = None if scale is None else np.array(scale, np.float32)
    ptr = lambda a: None if a is None else a.ctypes.data
    out = C.c_void_p()
    rc = lib.ms_create_materials(C.byref(p), 3, x.ctypes.data, v.ctypes.data, m.ctypes.data, None, None, 2,
                                 ij.ctypes.data, mat.ctypes.data, n_mat, mk.ctypes.data, ptr(mc), ptr(sc), None,
                                 None, None, C.byref(out))
    return rc, out


@pytest.mark.parametrize("args,what", [
    (([0, 2], 2, [1.0, 2.0]), "material id out of range"),
    (([0, 1], 2, [1.0, -2.0]), "mat_k"),
    (([0, 1], 2, [1.0, 2.0], [0.1, float("nan")]), "mat_c"),
    (([0, 1], 2, [1.0, 2.0], None, [1.0, -1.0]), "mat_L0scale"),
    (([0, 0], 0, [1.0]), "n_mat"),
])
def test_create_materials_rejects_bad_tables(lib, args, what):
    rc, out = _create_materials(lib, *args)
    assert rc == 1 and not out.value
    assert what in lib.ms_last_error().decode()


@pytest.mark.gpu
def test_two_material_system_equals_the_per_spring_form(lib, ora):
    """A lattice of two materials (soft and stiff, different damping, the stiff
    one pre-stretched by a rest-length factor) built through
    ms_create_materials steps bit for bit like the same system given as
    per-spring arrays to ms_create, and matches the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import synth
    import paper_2207_09334_gb300 as ms
    x, ij, L0 = synth.box_lattice(7, 6, 5, 0.01, origin=(0, 0, 0.002))
    N, S = x.shape[0], ij.shape[0]
    rng = np.random.default_rng(3)
    mat = rng.integers(0, 2, S).astype(np.uint16)
    mat_k = np.array([2e3, 3e4], np.float32); mat_c = np.array([0.02, 0.08], np.float32)
    scale = np.array([1.0, 0.97], np.float32)
    base = dict(x=x, v=np.zeros((N, 3), np.float32), m=np.full(N, 1e-3, np.float32),
                fixed=np.zeros(N, np.uint8), ij=ij)
    per_spring = dict(base, k=mat_k[mat], c=mat_c[mat], L0=(L0 * scale[mat]).astype(np.float32))
    by_mat = dict(base, mat=mat, mat_k=mat_k, mat_c=mat_c, mat_L0scale=scale, L0=L0)
    p = synth.params(dt=1e-4, g=(0, 0, -9.81), contact=True, k_c=1e5, mu=0.5)
    out = []
    for s in (by_mat, per_spring):
        with ms.Sim(s, p, kernel="tiled") as sim:
            sim.step(300)
            out.append(sim.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    q = dict(p); q["dt"] = float(np.float32(q["dt"])); q["k_c"] = float(np.float32(q["k_c"]))
    q["mu"] = float(np.float32(q["mu"])); q["g"] = tuple(float(np.float32(g)) for g in p["g"])
    xo, _ = ora.run(per_spring, q, 300)
    size = float(np.ptp(x, axis=0).max())
    assert np.abs(out[0][0] - xo).max() <= 1e-4 * size


@pytest.mark.parametrize("x,ij,what", [
    ([[0, 0, 0], [1, 0, 0], [0.5, 0.3, 0]], [[0, 1], [1, 2]], "grid"),        # off the grid
    ([[0, 0, 0], [1, 0, 0], [3, 0, 0]], [[0, 1], [1, 2]], "neighbours"),      # a spring two cells long
    ([[0, 0, 0], [1, 0, 0]], [[0, 1], [1, 0]], "same pair"),                   # two springs on one pair
])
def test_lattice_kernel_rejects_other_networks(lib, x, ij, what):
    """kernel = 4 checks on the host that the network is a box lattice and
    names the reason when it is not (no device memory is touched)."""
    rc, out = _create(lib, x=x, ij=ij, kernel=4)
    assert rc == 1 and not out.value
    msg = lib.ms_last_error().decode()
    assert "lattice" in msg and what in msg, msg
