"""The allocation-free step entry point (ms_step_csr_noalloc) against the FP64
oracle and against the regular entry points (ms_create + ms_step +
ms_get_state).

Some callers cannot allocate device memory when they advance a system: a
plugin inside a host application that owns every device allocation, or a
real-time loop that must not call an allocator.  They pass all inputs and
outputs themselves; the working memory is a fixed array inside the library.
This file is collected last so that a run stopping at its first failure has
already run every other test.

Gates are those of the other step tests: positions within 1e-4 of the body
size after a run with ground contact (1e-5 without), the centre-of-mass
displacement within 1 % of the oracle's.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09334_gb300 as ms
    ms.load()
    return ms


def f32p(p):
    q = dict(p)
    for key in ("dt", "k_c", "mu", "vel_damping"):
        if key in q:
            q[key] = float(np.float32(q[key]))
    q["g"] = tuple(float(np.float32(g)) for g in p["g"])
    return q


def body_size(s):
    return float(np.ptp(np.asarray(s["x"], np.float64), axis=0).max())


def csr(system):
    """Both-direction CSR incidence of the system's springs (host arrays)."""
    ij = system["ij"]; N = system["x"].shape[0]
    a = np.concatenate([ij[:, 0], ij[:, 1]]); b = np.concatenate([ij[:, 1], ij[:, 0]])
    e = np.concatenate([np.arange(len(ij))] * 2)
    order = np.lexsort((b, a))
    a, b, e = a[order], b[order], e[order]
    row = np.zeros(N + 1, np.int32)
    np.add.at(row, a + 1, 1)
    row = np.cumsum(row).astype(np.int32)
    c = np.broadcast_to(np.asarray(system["c"], np.float32), (len(ij),))
    return row, b.astype(np.int32), system["k"][e].astype(np.float32), c[e].astype(np.float32), \
        system["L0"][e].astype(np.float32)


def step_noalloc(ms, system, params, nsteps, x_in, v_in, with_fixed=True):
    import torch
    lib = ms.load()
    p = ms.make_params(params)
    N = system["x"].shape[0]
    row, partner, k, c, L0 = csr(system)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dm = d(system["m"].astype(np.float32))
    dfix = d(system["fixed"].astype(np.uint8)) if with_fixed else None
    drow, dp, dk, dc, dL = d(row), d(partner), d(k), d(c), d(L0)
    xo = torch.empty((N, 3), device="cuda"); vo = torch.empty((N, 3), device="cuda")
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    rc = lib.ms_step_csr_noalloc(C.byref(p), N, ptr(x_in), ptr(v_in), ptr(dm), ptr(dfix), ptr(drow), ptr(dp),
                                 ptr(dk), ptr(dc), ptr(dL), int(nsteps), ptr(xo), ptr(vo),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.ms_last_error().decode()
    torch.cuda.synchronize()
    return xo.cpu().numpy().astype(np.float64), vo.cpu().numpy().astype(np.float64)


def test_noalloc_matches_oracle_and_regular_step_on_two_calls_in_a_row(ms, ora):
    """Soft cube thrown onto the ground (contact and friction): two calls of
    100 steps, the second continuing from the first call's output, against
    the oracle after 100 and 200 steps and against ms_step on the same system."""
    import torch
    s = synth.soft_cube(n=8, z0=0.001)
    s["v"][:] = np.array([0.2, -0.1, -0.5], np.float32)
    p = synth.soft_cube_params(contact=True)
    size = float(np.ptp(s["x"], axis=0).max())
    x0 = torch.tensor(s["x"], device="cuda"); v0 = torch.tensor(s["v"], device="cuda")
    xa, va = step_noalloc(ms, s, p, 100, x0, v0)                  # first call
    xb, vb = step_noalloc(ms, s, p, 100, torch.tensor(xa, dtype=torch.float32, device="cuda"),
                          torch.tensor(va, dtype=torch.float32, device="cuda"))   # second call
    xo, vo, zmin, snaps = s["x"], s["v"], np.inf, []
    for c in range(20):                                           # oracle in chunks, watching contact
        xo, vo = ora.run(s, f32p(p), 10, n0=10 * c, x=xo, v=vo)
        zmin = min(zmin, xo[:, 2].min())
        if c in (9, 19):
            snaps.append((xo, vo))
    (xo1, vo1), (xo2, vo2) = snaps
    assert zmin < -1e-5                                           # contact really happened
    m = s["m"].astype(np.float64)
    for got, want in ((xa, xo1), (xb, xo2)):
        assert np.abs(got - want).max() <= 1e-4 * size, (np.abs(got - want).max(), size)
        d_o = ora.centre_of_mass(m, want) - ora.centre_of_mass(m, s["x"])
        d_g = ora.centre_of_mass(m, got) - ora.centre_of_mass(m, s["x"])
        assert np.linalg.norm(d_g - d_o) <= 0.01 * np.linalg.norm(d_o)
    assert np.abs(vb - vo2).max() <= 1e-2 * np.abs(vo2).max()
    # the regular entry point on the same system, same gates
    with ms.Sim(s, p, kernel="gather") as sim:
        sim.step(100)
        x1, _ = sim.get_state()
        sim.step(100)
        x2, _ = sim.get_state()
    for got, want in ((xa, x1), (xb, x2)):
        assert np.abs(got - want).max() <= 1e-4 * size


@pytest.mark.parametrize("nsteps", [1, 2, 60])
def test_noalloc_anchored_cantilever_matches_oracle(ms, ora, nsteps):
    """A 40x4x4 cantilever clamped at x = 0, sagging under gravity (no
    contact): anchored masses keep their place and zero velocity.  nsteps = 1
    reads the inputs and writes the outputs directly; 2 and 60 pass through
    the scratch buffers."""
    import torch
    s = synth.cantilever()
    s["fext"] = None
    p = synth.params(dt=1e-4, g=(0, 0, -9.81))
    v = np.zeros_like(s["v"]); v[:, 1] = 0.01       # anchored masses are given a velocity: it must be dropped
    s["v"] = v
    xg, vg = step_noalloc(ms, s, p, nsteps, torch.tensor(s["x"], device="cuda"), torch.tensor(v, device="cuda"))
    xo, vo = ora.run(s, f32p(p), nsteps)
    anchored = s["fixed"].astype(bool)
    assert np.array_equal(xg[anchored], s["x"][anchored].astype(np.float64))
    assert np.all(vg[anchored] == 0.0)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(s), np.abs(xg - xo).max()
    # velocities: the first step starts from identical FP32 positions, so only
    # the force arithmetic rounds; from the second step on, the FP32 rounding
    # of the 0.4 m coordinates (ulp 3e-8 m) is felt through up to 26 springs of
    # 1e4 N/m on 1e-3 kg masses (about 2e-4 m/s per step) and then through the
    # stiffest mode (w ~ 1.3e4 1/s)
    vgate = 1e-5 if nsteps == 1 else 2e-3
    assert np.abs(vg - vo).max() <= vgate, np.abs(vg - vo).max()


def test_noalloc_without_anchor_array(ms, ora):
    """fixed = NULL: every mass is free (a free-floating lattice with no
    gravity, spinning and vibrating), against the oracle after 40 steps."""
    import torch
    x, ij, L0 = synth.box_lattice(6, 5, 4, 0.01)
    rng = np.random.default_rng(7)
    N, S = x.shape[0], ij.shape[0]
    s = dict(x=x + np.float32(2e-4) * rng.standard_normal((N, 3)).astype(np.float32),
             v=(0.05 * rng.standard_normal((N, 3))).astype(np.float32),
             m=np.full(N, 1e-3, np.float32), fixed=np.zeros(N, np.uint8), ij=ij,
             k=rng.uniform(1e3, 5e3, S).astype(np.float32), c=np.float32(0.02), L0=L0)
    p = synth.params(dt=1e-4, g=(0, 0, 0))
    xg, vg = step_noalloc(ms, s, p, 40, torch.tensor(s["x"], device="cuda"), torch.tensor(s["v"], device="cuda"),
                          with_fixed=False)
    xo, vo = ora.run(s, f32p(p), 40)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(s)
    assert np.abs(vg - vo).max() <= 1e-3 * np.abs(vo).max()


def test_noalloc_rejects_systems_beyond_its_scratch(ms):
    import torch
    lib = ms.load()
    p = ms.make_params(synth.params())
    N = 262144 + 1
    t = torch.zeros(8, device="cuda")
    ptr = C.c_void_p(t.data_ptr())
    rc = lib.ms_step_csr_noalloc(C.byref(p), N, ptr, ptr, ptr, None, ptr, ptr, ptr, ptr, ptr, 1, ptr, ptr, None)
    assert rc == 1 and "262144" in lib.ms_last_error().decode()
