"""Parity at the benchmark's sizes.

* The 256^3 throughput lattice (16.8 M masses, 216 M springs), stepped by
  the default kernel for it (the lattice kernel) exactly as bench.py times
  it, against the FP64 oracle on sampled masses after 1 and after 5 steps;
  the same for the general tiled kernel.
* The 64^3 lattice with the same parameters, 200 steps, every mass, with the
  lattice and the tiled kernels.

The oracle cannot step the whole 256^3 lattice in a test, but after n steps a
mass depends only on the masses within n springs of it.  So the oracle steps
the sub-system of the masses within n hops of the samples, with every spring
among them: the samples' results are then exact (masses n hops out miss some
of their springs, and their error reaches the samples only after n + 1
steps).

Tolerances, from FP32 rounding at this scale:
  * one step, velocity change: the spring lengths (about 1 mm) carry ~2e-10 m
    of rounding in FP32 (l^2 and rsqrt), i.e. up to 1e-5 N per spring at
    k = 5e4 N/m; over 26 springs and m = 1e-3 kg that is ~2.5e-6 m/s.  Gate:
    1e-5 m/s, against a gravity term of 4.9e-4 m/s.
  * one step, positions: x1 = x0 + dt v1 is rounded to FP32 at |x| ~ 0.26 m
    (half an ulp is 1.5e-8 m).  Gate: 3e-8 m.
  * after the first step the FP32 position rounding itself feeds the
    springs: the stiffest mode has omega dt ~ 1.1, so a position error dx
    becomes a velocity error of up to ~omega dx ~ 1.1 / dt * dx (7e-4 m/s for
    dx = 3e-8 m).  Five steps: gates 1e-3 m/s and 3e-7 m (dt times the
    velocity gate per step, plus the per-step rounding).
"""
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


def hops(ij, N, seeds, n):
    """Masses within n springs of the seeds (boolean mask)."""
    mark = np.zeros(N, bool)
    mark[seeds] = True
    for _ in range(n):
        touch = mark[ij[:, 0]] | mark[ij[:, 1]]
        grow = np.zeros(N, bool)
        grow[ij[touch].ravel()] = True
        mark |= grow
    return mark


def subsystem(s, keep):
    """The masses in `keep` and every spring among them; returns (system, index map)."""
    ij = s["ij"]
    sel = keep[ij[:, 0]] & keep[ij[:, 1]]
    sub = np.flatnonzero(keep)
    remap = np.full(keep.size, -1, np.int64)
    remap[sub] = np.arange(sub.size)
    c = s["c"]
    sub_c = np.full(int(sel.sum()), c, np.float32) if np.ndim(c) == 0 else np.asarray(c)[sel]
    return dict(x=s["x"][sub], v=s["v"][sub], m=s["m"][sub], fixed=s["fixed"][sub],
                ij=remap[ij[sel]].astype(np.int32), k=s["k"][sel], c=sub_c, L0=s["L0"][sel]), remap


@pytest.fixture(scope="module")
def workload256():
    return synth.throughput_lattice(256), synth.throughput_params()


@pytest.fixture(scope="module", params=["auto", "tiled"])
def lattice256(ms, workload256, request):
    """The bench's workload, stepped once and then four more times by the
    bench's kernel (the default: the lattice kernel) or the tiled kernel."""
    s, p = workload256
    with ms.Sim(s, p, kernel=request.param) as sim:
        assert sim.info()["kernel"] == (4 if request.param == "auto" else 2)
        sim.step(1)
        x1, v1 = sim.get_state()
        sim.step(4)
        x5, v5 = sim.get_state()
    return s, p, (x1, v1), (x5, v5)


@pytest.mark.slow
def test_full_size_lattice_one_step_on_sampled_masses(ora, lattice256):
    s, p, (x1, v1), _ = lattice256
    n = 256
    N = s["x"].shape[0]
    rng = np.random.default_rng(7)
    samples = np.unique(np.concatenate([
        rng.integers(0, N, 4000),                   # anywhere
        np.arange(0, n * n, 997),                   # anchored bottom layer
        N - n * n + np.arange(0, n * n, 991),       # top face
        [0, n - 1, n * n - 1, N - n * n, N - n, N - 1],   # corners
    ]))
    sub, remap = subsystem(s, hops(s["ij"], N, samples, 1))
    xo, vo = ora.run(sub, f32p(p), 1)
    loc = remap[samples]

    v0 = s["v"][samples].astype(np.float64)
    dv_g = v1[samples].astype(np.float64) - v0
    dv_o = vo[loc] - v0
    assert np.abs(dv_g - dv_o).max() <= 1e-5, np.abs(dv_g - dv_o).max()
    assert np.abs(x1[samples].astype(np.float64) - xo[loc]).max() <= 3e-8
    anchored = s["fixed"][samples].astype(bool)
    assert anchored.any() and (~anchored).any()
    assert np.array_equal(x1[samples][anchored], s["x"][samples][anchored])
    assert np.all(v1[samples][anchored] == 0)
    # gravity dominates the free masses' velocity change
    gdt = np.float32(p["dt"]) * np.float32(p["g"][2])
    assert abs(dv_g[~anchored, 2].mean() - gdt) < 0.05 * abs(gdt)


@pytest.mark.slow
def test_full_size_lattice_five_steps_on_sampled_masses(ora, lattice256):
    """Five steps of the full-size lattice: the samples' 5-hop neighbourhoods
    (up to 11^3 masses each) stepped by the oracle."""
    s, p, _, (x5, v5) = lattice256
    n = 256
    N = s["x"].shape[0]
    rng = np.random.default_rng(11)
    samples = np.unique(np.concatenate([
        rng.integers(0, N, 150),
        [0, n - 1, n * n - 1, N - n * n, N - n, N - 1],
        n * n * 3 + np.arange(0, n * n, 4099),       # the layer just above the anchored one, and up
    ]))
    sub, remap = subsystem(s, hops(s["ij"], N, samples, 5))
    xo, vo = ora.run(sub, f32p(p), 5)
    loc = remap[samples]
    v0 = s["v"][samples].astype(np.float64)
    dv_g = v5[samples].astype(np.float64) - v0
    dv_o = vo[loc] - v0
    assert np.abs(dv_g - dv_o).max() <= 1e-3, np.abs(dv_g - dv_o).max()
    assert np.abs(x5[samples].astype(np.float64) - xo[loc]).max() <= 3e-7, \
        np.abs(x5[samples].astype(np.float64) - xo[loc]).max()
    free = ~s["fixed"][samples].astype(bool)
    gdt = 5 * np.float32(p["dt"]) * np.float32(p["g"][2])
    assert abs(dv_g[free, 2].mean() - gdt) < 0.1 * abs(gdt)


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["auto", "tiled"])
def test_lattice64_200_steps_every_mass(ms, ora, kernel):
    """The 64^3 lattice (262 144 masses, 3.3 M springs) with the benchmark's
    parameters, 200 steps, every mass against the oracle (1e-5 of the body
    size, the benchmark's contact-free position gate); the default kernel for
    it is the lattice kernel."""
    s = synth.throughput_lattice(64)
    p = synth.throughput_params()
    with ms.Sim(s, p, kernel=kernel) as sim:
        assert sim.info()["kernel"] == (4 if kernel == "auto" else 2)
        sim.step(120)
        sim.step(80)
        xg, vg = sim.get_state()
    xo, vo = ora.run(s, f32p(p), 200)
    body = float(np.ptp(np.asarray(s["x"], np.float64), axis=0).max())
    err = np.abs(xg.astype(np.float64) - xo).max()
    assert err <= 1e-5 * body, (err, 1e-5 * body)
    assert np.abs(vg.astype(np.float64) - vo).max() <= 1e-3
