"""Failure detection on the GPU without a fault: a bounded device-side wait
is made to run out, and the library reports it as a status code.

The persistent grid kernel (one cooperative launch for all steps of a call)
meets its CTAs at a grid barrier every step.  Its test hook makes the barrier
wait for one arrival more than there are CTAs -- a flag that nothing ever
sets -- so every CTA's wait gives up after the poll limit, the CTA leaves its
step loop and the kernel returns.  No async copy is in flight in that kernel,
nothing traps, and the context stays usable.
"""
import time

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


def lattice24(seed=5):
    """24^3 masses: above the cluster kernel's size, 27 tiles of the grid kernel."""
    x, ij, L0 = synth.box_lattice(24, 24, 24, 1e-3, origin=(0, 0, 0.001))
    rng = np.random.default_rng(seed)
    S = ij.shape[0]; N = x.shape[0]
    return dict(x=x, v=(1e-3 * rng.standard_normal((N, 3))).astype(np.float32),
                m=np.full(N, 1e-3, np.float32), fixed=np.zeros(N, np.uint8), ij=ij,
                k=rng.uniform(5e3, 5e4, S).astype(np.float32), c=np.float32(0.05), L0=L0)


def test_grid_barrier_wait_runs_out_and_reports_timeout(ms):
    import torch
    s = lattice24()
    p = synth.params(dt=5e-5, g=(0, 0, -9.81))
    N = s["x"].shape[0]
    with ms.Sim(s, p, kernel="persistent") as sim:
        assert sim.info()["kernel"] == 3
        sim.step(20)
        sim.sync()                                    # a healthy run first
        sim.set_wait_limit(64)
        sim.test_barrier_deficit(1)
        t0 = time.perf_counter()
        sim.step(50)
        with pytest.raises(ms.MsError) as e:
            sim.sync()
        took = time.perf_counter() - t0
        assert e.value.code == 6 and "wait" in str(e.value)     # MS_ERR_TIMEOUT
        assert took < 5.0, took                      # every CTA gave up after 64 polls
        x = torch.empty((N, 3), device="cuda"); v = torch.empty((N, 3), device="cuda")
        sim.get_state(x, v)                          # device copy: no status check
        torch.cuda.synchronize()
        assert torch.isfinite(x).all() and torch.isfinite(v).all()
        # the flag is sticky for this object
        with pytest.raises(ms.MsError):
            sim.sync()
    # the context is still usable: a new object steps and syncs cleanly
    with ms.Sim(s, p, kernel="persistent") as sim:
        sim.step(20)
        sim.sync()
        xg, _ = sim.get_state()
        assert np.isfinite(xg).all()


def test_barrier_hook_needs_the_grid_kernel(ms):
    s = synth.soft_cube(n=4)
    with ms.Sim(s, synth.soft_cube_params(), kernel="tiled") as sim:
        with pytest.raises(ms.MsError) as e:
            sim.test_barrier_deficit(1)
        assert e.value.code == 1
        sim.test_barrier_deficit(0)                  # off is always accepted
        sim.set_wait_limit(0)
