"""Instrumentation on the GPU: the device energy reduction and the per-step
trace, against the FP64 oracle.

* Energy at a given state: the oracle evaluates its energy on the GPU's own
  state (read back), so the only differences are the GPU's FP32 terms and
  sums: relative 1e-5 of the magnitude of each term.
* Energy along a run: GPU and oracle each follow their own trajectory; the
  trajectories agree to the step parity tolerance, the energies to 2e-3 of
  the total (FP32 positions limit how well small spring extensions are
  resolved; see the test).
* Trace: the recorded positions are the GPU state after each step (bit for
  bit), and agree with the oracle's trajectory to the parity tolerance.
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


def actuated_lattice(seed=11):
    """7x6x5 lattice, random masses, stiffness, damping and actuation, the
    bottom layer anchored, a few masses started below the ground."""
    x, ij, L0 = synth.box_lattice(7, 6, 5, 0.01, origin=(0, 0, 0.0))
    rng = np.random.default_rng(seed)
    S = ij.shape[0]; N = x.shape[0]
    x = x + (2e-4 * rng.standard_normal(x.shape)).astype(np.float32)
    fixed = (np.arange(N) < 7 * 6).astype(np.uint8)
    v = (0.05 * rng.standard_normal((N, 3))).astype(np.float32)
    v[fixed == 1] = 0.0                                     # anchored masses do not move
    return dict(x=x, v=v,
                m=rng.uniform(1e-3, 4e-3, N).astype(np.float32), fixed=fixed,
                ij=ij, k=rng.uniform(1e3, 1e4, S).astype(np.float32), c=rng.uniform(0, 0.1, S).astype(np.float32),
                L0=L0, A=rng.uniform(0, 0.2, S).astype(np.float32),
                phi=rng.uniform(0, 2 * np.pi, S).astype(np.float32), freq=5.0)


def check_terms(e_gpu, e_ora, rtol=1e-5):
    for q, (g, o) in enumerate(zip(e_gpu, e_ora)):
        assert abs(g - o) <= rtol * max(abs(o), 1e-12) + 1e-12, (q, g, o)


@pytest.mark.parametrize("kernel", ["gather", "tiled", "persistent"])
def test_energy_matches_oracle_on_the_same_state(ms, ora, kernel):
    s = actuated_lattice()
    p = synth.params(dt=1e-4, g=(0, 0, -9.81), contact=True, k_c=1e4, mu=0.5)
    with ms.Sim(s, p, kernel=kernel) as sim:
        check_terms(sim.energy(), ora.energy(s, f32p(p), s["x"], s["v"], t=0.0))
        sim.step(137)
        x, v = sim.get_state()
        e = sim.energy()
        assert e[3] > 0.0                                   # some masses are below the ground
        t = 137 * float(np.float32(p["dt"]))
        check_terms(e, ora.energy(s, f32p(p), x, v, t=t))
        assert sim.energy() == e                            # fixed reduction order


def test_energy_on_a_multi_tile_lattice(ms, ora):
    """Many tiles and a ragged last tile (23x24x25): every spring counted once."""
    x, ij, L0 = synth.box_lattice(23, 24, 25, 1e-3)
    N = x.shape[0]; S = ij.shape[0]
    rng = np.random.default_rng(3)
    s = dict(x=x + (1e-5 * rng.standard_normal(x.shape)).astype(np.float32),
             v=(1e-3 * rng.standard_normal((N, 3))).astype(np.float32), m=np.full(N, 1e-3, np.float32),
             fixed=np.zeros(N, np.uint8), ij=ij, k=rng.uniform(5e3, 5e4, S).astype(np.float32),
             c=np.float32(0.05), L0=L0)
    p = synth.throughput_params()
    for kernel in ("tiled", "gather"):
        with ms.Sim(s, p, kernel=kernel) as sim:
            check_terms(sim.energy(), ora.energy(s, f32p(p), s["x"], s["v"]))


def test_device_energy_trace_follows_the_oracle(ms, ora):
    """Energy every 25 steps into a device tensor (no host copies in the
    loop) on a damping-free 6^3 cube without gravity.
    * The device trace equals the host-mode values of an identical second run
      bit for bit, and each of those matches the oracle's energy of the same
      (read back) state to 1e-4 of the total.
    * Along the run the GPU's total energy follows the oracle's own FP64
      trajectory to 2e-3 of the total: the springs' extensions here are about
      1e-5 m while an FP32 position at 0.1 m carries 7e-9 m of rounding, so
      the FP32 trajectory's elastic energy differs by up to ~1e-3 relative."""
    import torch
    s = synth.soft_cube(n=6, c=0.0)
    rng = np.random.default_rng(5)
    s["v"] = (0.05 * rng.standard_normal(s["x"].shape)).astype(np.float32)
    p = synth.params(dt=1e-4, g=(0, 0, 0))
    K = 40
    trace = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    with ms.Sim(s, p) as sim:
        for q in range(K):
            sim.step(25)
            sim.energy(trace[q])
        sim.sync()
    dev = trace.cpu().numpy()
    host = []
    xo, vo = s["x"], s["v"]
    E0 = sum(ora.energy(s, f32p(p), xo, vo))
    with ms.Sim(s, p) as sim:
        for q in range(K):
            sim.step(25)
            host.append(sim.energy())
            xg, vg = sim.get_state()
            assert abs(sum(host[-1]) - sum(ora.energy(s, f32p(p), xg, vg))) <= 1e-4 * E0
    assert np.array_equal(dev, np.array(host))
    for q in range(K):
        xo, vo = ora.run(s, f32p(p), 25, n0=25 * q, x=xo, v=vo)
        eo = sum(ora.energy(s, f32p(p), xo, vo))
        assert abs(dev[q].sum() - eo) <= 2e-3 * E0, (q, dev[q].sum(), eo)


def test_trace_records_the_tip_every_step(ms, ora):
    s = synth.cantilever(40, 4, 4, c=0.1)
    p = synth.params(dt=1e-4, g=(0, 0, -9.81))
    N = s["x"].shape[0]
    tip = [N - 1, N - 4]
    with ms.Sim(s, p) as sim:
        sim.trace(tip, capacity=300)
        sim.step(120)
        x120, _ = sim.get_state()
        sim.step(280)                                       # 100 steps beyond the capacity
        tr = sim.get_trace()
        assert tr.shape == (300, 2, 3)
        assert np.array_equal(tr[119], x120[tip])
        sim.trace([], 0)
        assert sim.get_trace().shape[0] == 0
    xo, vo = s["x"], s["v"]
    for q in range(6):
        xo, vo = ora.run(s, f32p(p), 50, n0=50 * q, x=xo, v=vo)
        np.testing.assert_allclose(tr[50 * q + 49], xo[tip], rtol=0, atol=1e-5 * 0.4)
    assert abs(tr[-1, 0, 2] - s["x"][tip[0], 2]) > 1e-5      # the tip moved


def test_trace_is_refused_by_the_persistent_kernel(ms):
    s = synth.soft_cube(n=3)
    with ms.Sim(s, synth.soft_cube_params(contact=False), kernel="persistent") as sim:
        with pytest.raises(ms.MsError):
            sim.trace([0], 10)
