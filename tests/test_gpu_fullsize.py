"""Parity at the full benchmark size: the 256^3 throughput lattice (16.8 M
masses, 216 M springs), stepped by the default (tiled) kernel exactly as
bench.py times it, checked against the FP64 oracle on sampled masses.

The oracle cannot step the whole lattice in a test, but one step of a mass
depends only on its springs and their partners' state at t_0.  So the oracle
steps the sub-system made of the sampled masses, their partners and every
spring that touches a sampled mass; the sampled masses' results are then
exact (their partners' are not, and are not compared).

Tolerances, from FP32 rounding at this scale:
  * velocity change over the step: the spring lengths (about 1 mm) carry
    ~2e-10 m of rounding in FP32 (l^2 and rsqrt), i.e. up to 1e-5 N per
    spring at k = 5e4 N/m; over 26 springs and m = 1e-3 kg that is ~2.5e-6
    m/s per step.  Gate: 1e-5 m/s, against a gravity term of 4.9e-4 m/s.
  * positions: x1 = x0 + dt v1 is rounded to FP32 at |x| ~ 0.26 m (half an
    ulp is 1.5e-8 m).  Gate: 3e-8 m.
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


@pytest.mark.slow
def test_full_size_lattice_one_step_on_sampled_masses(ms, ora):
    n = 256
    s = synth.throughput_lattice(n)
    p = synth.throughput_params()
    N = s["x"].shape[0]
    rng = np.random.default_rng(7)
    samples = np.unique(np.concatenate([
        rng.integers(0, N, 4000),                   # anywhere
        np.arange(0, n * n, 997),                   # anchored bottom layer
        N - n * n + np.arange(0, n * n, 991),       # top face
        [0, n - 1, n * n - 1, N - n * n, N - n, N - 1],   # corners
    ]))
    with ms.Sim(s, p) as sim:
        assert sim.info()["kernel"] == 2             # the bench's kernel
        sim.step(1)
        x1, v1 = sim.get_state()

    # the sub-system the sampled masses' first step depends on
    ij = s["ij"]
    mark = np.zeros(N, bool)
    mark[samples] = True
    sel = mark[ij[:, 0]] | mark[ij[:, 1]]
    sub_ij = ij[sel]
    sub = np.unique(np.concatenate([samples, sub_ij.ravel()]))
    remap = np.full(N, -1, np.int64)
    remap[sub] = np.arange(sub.size)
    c = s["c"]
    sub_c = np.full(sub_ij.shape[0], c, np.float32) if np.ndim(c) == 0 else np.asarray(c)[sel]
    subsys = dict(x=s["x"][sub], v=s["v"][sub], m=s["m"][sub], fixed=s["fixed"][sub],
                  ij=remap[sub_ij].astype(np.int32), k=s["k"][sel], c=sub_c, L0=s["L0"][sel])
    xo, vo = ora.run(subsys, f32p(p), 1)
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
