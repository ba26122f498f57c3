"""Batched voxel-robot population (one persistent launch) vs the FP64 oracle.

The oracle expands every voxel into its own 28 springs (no merging) and runs
each robot separately; the library merges shared springs and advances all
robots together.  Gates: positions within 1e-4 x body size after 200 steps
with ground contact and friction; centre-of-mass x-travel within 1 % (or
2 micrometres for robots that barely move) after 2000 steps.
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
        q[key] = float(np.float32(q[key]))
    q["g"] = tuple(float(np.float32(g)) for g in p["g"])
    return q


def population(n, seed, side_range=(2, 5)):
    rng = np.random.default_rng(seed)
    designs = []
    for _ in range(n):
        dims = tuple(int(s) for s in rng.integers(side_range[0], side_range[1] + 1, size=3))
        designs.append(synth.random_voxel_design(rng, dims))
    return designs


def make_pop(ms, designs, **kw):
    return ms.Population(designs, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE,
                         synth.VOXEL_MASS, synth.voxel_params(), **kw)


def oracle_robot(ora, design, nsteps):
    mat, phase = design
    s = ora.voxel_system(mat, phase, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS)
    x, v = ora.run(s, f32p(synth.voxel_params()), nsteps)
    m = s["m"]
    travel = ora.centre_of_mass(m, x)[0] - ora.centre_of_mass(m, s["x"])[0]
    return s, x, v, travel


@pytest.mark.parametrize("policy,threads", [(1, 512), (2, 512), (1, 1024), (2, 1024)])
def test_population_matches_oracle_200_steps(ms, ora, policy, threads):
    """Both schedules (block- and warp-per-robot) with both CTA sizes.  With
    1024 threads a warp item holds 32 robots, so the larger robots no longer
    fit a warp's share of shared memory and run block-per-robot, and block
    robots of at most 512 masses run two to a CTA, one per half (pair items,
    each half on its own named barrier)."""
    designs = population(10, seed=21)
    with make_pop(ms, designs) as pop:
        pop.set_threads(threads)
        pop.autotune(policy=policy)
        inf = pop.info()
        assert inf["threads"] == threads
        if policy == 2:
            assert inf["n_warp_items"] == (10 if threads == 512 else 9)
        pop.run(200)
        xg, _ = pop.get_state()
        in_contact = 0
        for r, d in enumerate(designs):
            s, xo, _, _ = oracle_robot(ora, d, 200)
            n, first = pop.robot_info(r)
            assert n == s["x"].shape[0]
            size = float(np.ptp(s["x"], axis=0).max())
            err = np.abs(xg[first:first + n] - xo).max()
            assert err <= 1e-4 * size, (r, err, size)
            m = s["m"]
            to = ora.centre_of_mass(m, xo)[0] - ora.centre_of_mass(m, s["x"])[0]
            tg = ora.centre_of_mass(m, xg[first:first + n].astype(np.float64))[0] - ora.centre_of_mass(m, s["x"])[0]
            assert abs(tg - to) <= max(0.01 * abs(to), 1e-6), (r, tg, to)
            in_contact += int(xo[:, 2].min() < 0.0)
        assert in_contact >= 1                     # contact is exercised


@pytest.mark.parametrize("threads", [512, 1024, 0])
def test_population_with_config3_sized_robots_matches_oracle(ms, ora, threads):
    """Robots of the benchmark population's largest sizes (sides 10 to 12
    voxels): more than 512 masses each, so the block schedule's per-robot loop
    over masses takes several passes, and a solid 12 x 12 x 12 robot reaches
    the 2197-mass maximum.  Mixed with small robots so that both schedules
    run in the same launch, with robots of 343 to 448 masses that 1024-thread
    CTAs run two at a time (pair items) and small ones four at a time (quad
    items).  200 steps with contact and friction against the
    per-voxel oracle: positions within 1e-4 of the body size, centre-of-mass
    travel within 1 %.  CTAs of 512 or 1024 threads, or (0) the size and
    schedules msb_autotune chooses, after which the robots must start from
    their initial state again."""
    rng = np.random.default_rng(31)
    solid = (rng.integers(1, 4, size=(12, 12, 12)).astype(np.uint8), rng.uniform(0, 2 * np.pi, (12, 12, 12)))
    designs = [solid,
               synth.random_voxel_design(rng, (10, 11, 12)),
               synth.random_voxel_design(rng, (11, 11, 11)),
               synth.random_voxel_design(rng, (12, 10, 11)),
               # 257 to 512 masses: a pair item with 1024-thread CTAs
               (rng.integers(1, 4, size=(6, 6, 6)).astype(np.uint8), rng.uniform(0, 2 * np.pi, (6, 6, 6))),
               (rng.integers(1, 4, size=(6, 7, 6)).astype(np.uint8), rng.uniform(0, 2 * np.pi, (6, 7, 6))),
               (rng.integers(1, 4, size=(7, 6, 6)).astype(np.uint8), rng.uniform(0, 2 * np.pi, (7, 6, 6)))]
    designs += population(6, seed=32, side_range=(2, 4))
    with make_pop(ms, designs) as pop:
        if threads:
            pop.set_threads(threads)
        else:
            pop.autotune(sample_steps=20)
        inf = pop.info()
        assert inf["max_robot_masses"] == 13 ** 3
        assert inf["n_block_items"] >= 7
        assert inf["threads"] == (threads or inf["threads"]) and inf["threads"] in (512, 1024)
        pop.run(200)
        xg, _ = pop.get_state()
        big = 0
        for r, d in enumerate(designs):
            s, xo, _, _ = oracle_robot(ora, d, 200)
            n, first = pop.robot_info(r)
            assert n == s["x"].shape[0]
            big += int(n > 512)
            size = float(np.ptp(s["x"], axis=0).max())
            err = np.abs(xg[first:first + n] - xo).max()
            assert err <= 1e-4 * size, (r, n, err, size)
            m = s["m"]
            to = ora.centre_of_mass(m, xo)[0] - ora.centre_of_mass(m, s["x"])[0]
            tg = ora.centre_of_mass(m, xg[first:first + n].astype(np.float64))[0] - ora.centre_of_mass(m, s["x"])[0]
            assert abs(tg - to) <= max(0.01 * abs(to), 1e-6), (r, n, tg, to)
        assert big >= 4


@pytest.mark.slow
def test_population_com_travel_2000_steps(ms, ora):
    """Over 2000 steps the travel of a robot hopping on a frictional ground
    is chaotic: perturbing the FP64 start positions by 1e-9 m moves it by up
    to several percent.  The GPU's travel must lie within that intrinsic
    spread (three times the largest deviation of four perturbed oracle runs),
    or within 1 % / 2 micrometres."""
    designs = population(6, seed=22, side_range=(2, 4))
    with make_pop(ms, designs) as pop:
        pop.run(2000)
        tg = pop.com_travel()
    p = f32p(synth.voxel_params())
    for r, d in enumerate(designs):
        s, _, _, to = oracle_robot(ora, d, 2000)
        m = s["m"]
        spread = 0.0
        for q in range(4):
            xp = s["x"].astype(np.float64) + 1e-9 * np.random.default_rng(100 + q).standard_normal(s["x"].shape)
            x1, _ = ora.run(s, p, 2000, x=xp)
            tq = ora.centre_of_mass(m, x1)[0] - ora.centre_of_mass(m, xp)[0]
            spread = max(spread, abs(tq - to))
        assert abs(tg[r] - to) <= max(3 * spread, 0.01 * abs(to), 2e-6), (r, tg[r], to, spread)


def test_block_and_warp_schedules_are_bit_identical(ms):
    designs = population(12, seed=23)
    out = []
    for policy in (1, 2):
        with make_pop(ms, designs) as pop:
            pop.autotune(policy=policy)
            pop.run(150)
            out.append(pop.get_state()[0])
    assert np.array_equal(out[0], out[1])


def test_graph_replay_continues_time(ms):
    """Two replays of the captured 100-step launch equal one 200-step launch
    (the actuation clock advances on the device)."""
    designs = population(8, seed=24)
    with make_pop(ms, designs) as a:
        a.run(100); a.run(100)
        xa = a.get_state()[0]; ta = a.com_travel()
    with make_pop(ms, designs) as b:
        b.run(200)
        xb = b.get_state()[0]; tb = b.com_travel()
    assert np.array_equal(xa, xb) and np.array_equal(ta, tb)


def test_per_robot_loop_matches_batched_launch(ms):
    designs = population(6, seed=25)
    with make_pop(ms, designs) as a:
        a.run(120)
        xa = a.get_state()[0]; ta = a.com_travel()
    with make_pop(ms, designs) as b:
        b.run_loop(120)
        xb = b.get_state()[0]; tb = b.com_travel()
    np.testing.assert_allclose(xa, xb, rtol=0, atol=1e-7)
    np.testing.assert_allclose(ta, tb, rtol=0, atol=1e-7)


def test_autotune_keeps_state_and_results(ms):
    designs = population(16, seed=26, side_range=(1, 6))
    with make_pop(ms, designs) as a:
        a.autotune(sample_steps=20, policy=0)
        a.run(100)
        xa = a.get_state()[0]
    with make_pop(ms, designs) as b:
        b.autotune(policy=1)
        b.run(100)
        xb = b.get_state()[0]
    assert np.array_equal(xa, xb)


def test_reset_restores_start(ms):
    designs = population(4, seed=27)
    with make_pop(ms, designs) as a:
        x0 = a.get_state()[0]
        a.run(50)
        a.reset()
        assert np.array_equal(a.get_state()[0], x0)
        assert np.all(a.com_travel() == 0)
