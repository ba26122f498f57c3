"""GPU (FP32, sm_103a) explicit step vs the FP64 oracle on identical seeded inputs.

Tolerances (the position gates of the benchmark workloads):
  * contact-free runs: max |x_gpu - x_oracle| <= 1e-5 x body size after the run;
  * runs with ground contact: <= 1e-4 x body size after 200 steps, and the
    centre-of-mass displacement within 1 % of the oracle's.
Body size = largest axis-aligned extent of the start positions.
The oracle gets the FP32-rounded values of every parameter the GPU sees.
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


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


KERNELS = ["gather", "tiled", "persistent"]


def gpu_run(ms, s, p, n, reorder=None, chunks=1, kernel=None):
    with ms.Sim(s, p, reorder=reorder, kernel=kernel) as sim:
        done = 0
        for q in range(chunks):
            todo = n * (q + 1) // chunks - done
            sim.step(todo)
            done += todo
        assert done == n
        x, v = sim.get_state()
    return x.astype(np.float64), v.astype(np.float64)


def test_hand_worked_steps_on_gpu(ms):
    cases = json.load(open(os.path.join(HERE, "golden", "hand_steps.json")))["cases"]
    for case in cases:
        s = dict(x=np.array(case["x"], np.float32), v=np.array(case["v"], np.float32),
                 m=np.array(case["m"], np.float32), fixed=np.array(case["fixed"], np.uint8),
                 ij=np.array(case["ij"], np.int32), k=np.array(case["k"], np.float32),
                 c=np.array(case["c"], np.float32), L0=np.array(case["L0"], np.float32),
                 freq=case.get("freq", 0.0))
        if "A" in case:
            s["A"] = np.array(case["A"], np.float32); s["phi"] = np.array(case["phi"], np.float32)
        x, v = gpu_run(ms, s, synth.params(dt=case["dt"], g=(0, 0, 0)), case["nsteps"])
        np.testing.assert_allclose(x, case["x_out"], rtol=2e-6, atol=1e-6, err_msg=case["name"])
        np.testing.assert_allclose(v, case["v_out"], rtol=2e-6, atol=1e-6, err_msg=case["name"])


@pytest.mark.parametrize("kernel,reorder", [("gather", "caller"), ("gather", "morton"), ("tiled", "morton"),
                                            ("tiled", "caller"), ("persistent", None)])
def test_soft_cube_contact_free_1000_steps(ms, ora, kernel, reorder):
    s = synth.soft_cube()
    p = synth.soft_cube_params(contact=False)
    xg, vg = gpu_run(ms, s, p, 1000, reorder=reorder, chunks=4, kernel=kernel)
    xo, vo = ora.run(s, f32p(p), 1000)
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


@pytest.mark.parametrize("kernel", KERNELS)
def test_soft_cube_contact_200_steps(ms, ora, kernel):
    """Cube 1 mm above the ground, thrown down and sideways: contact and
    friction are active within the 200 steps."""
    s = synth.soft_cube(z0=0.001)
    s["v"][:] = np.array([0.3, -0.2, -0.6], np.float32)
    p = synth.soft_cube_params(contact=True)
    xg, _ = gpu_run(ms, s, p, 200, kernel=kernel)
    xo, vo = s["x"], s["v"]
    zmin = np.inf
    for c in range(20):
        xo, vo = ora.run(s, f32p(p), 10, n0=10 * c, x=xo, v=vo)
        zmin = min(zmin, xo[:, 2].min())
    assert zmin < -1e-5                       # contact really happened (the cube bounces)
    err = np.abs(xg - xo).max()
    assert err <= 1e-4 * body_size(s), (err, 1e-4 * body_size(s))
    m = s["m"].astype(np.float64)
    d_o = ora.centre_of_mass(m, xo) - ora.centre_of_mass(m, s["x"])
    d_g = ora.centre_of_mass(m, xg) - ora.centre_of_mass(m, s["x"])
    assert np.linalg.norm(d_g - d_o) <= 0.01 * np.linalg.norm(d_o)


@pytest.mark.slow
def test_soft_cube_full_drop_com_travel(ms, ora):
    """The dropped-cube workload: 0.05 m drop onto the ground, 10,000 steps.
    The vertical centre-of-mass travel agrees within 1 %.  The sideways drift
    of this symmetric drop comes from amplified rounding (perturbing the FP64
    start by 1e-9 m moves it by about 0.5 mm, and FP32 rounding perturbs every
    step), so it is only bounded: below 10 % of the vertical travel.  The
    cube must rest on the plane, not sink through it."""
    s = synth.soft_cube()
    p = synth.soft_cube_params(contact=True)
    xg, _ = gpu_run(ms, s, p, 10000, chunks=10)
    xo, _ = ora.run(s, f32p(p), 10000)
    m = s["m"].astype(np.float64)
    c0 = ora.centre_of_mass(m, s["x"])
    d_o = ora.centre_of_mass(m, xo) - c0
    d_g = ora.centre_of_mass(m, xg) - c0
    assert abs(d_g[2] - d_o[2]) <= 0.01 * abs(d_o[2])
    assert np.linalg.norm(d_g[:2]) <= 0.1 * abs(d_o[2]), (d_g, d_o)
    assert xg[:, 2].min() > -1e-3


@pytest.mark.parametrize("kernel", KERNELS)
def test_cantilever_with_anchors_and_external_force(ms, ora, kernel):
    s = synth.cantilever(40, 4, 4, c=0.1)
    p = synth.params(dt=1e-4, g=(0, 0, 0))
    xg, vg = gpu_run(ms, s, p, 2000, chunks=2, kernel=kernel)
    xo, vo = ora.run(s, f32p(p), 2000)
    fixed = s["fixed"].astype(bool)
    assert np.all(xg[fixed] == s["x"][fixed]) and np.all(vg[fixed] == 0)
    assert np.abs(xo[:, 2] - s["x"][:, 2]).max() > 1e-5
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


@pytest.mark.parametrize("kernel", KERNELS)
def test_actuated_heterogeneous_lattice(ms, ora, kernel):
    x, ij, L0 = synth.box_lattice(7, 6, 5, 0.01, origin=(0, 0, 0.02))
    rng = np.random.default_rng(11)
    S = ij.shape[0]; N = x.shape[0]
    s = dict(x=x, v=(0.01 * rng.standard_normal((N, 3))).astype(np.float32),
             m=rng.uniform(1e-3, 4e-3, N).astype(np.float32), fixed=np.zeros(N, np.uint8), ij=ij,
             k=rng.uniform(1e3, 1e4, S).astype(np.float32), c=rng.uniform(0, 0.1, S).astype(np.float32),
             L0=L0, A=rng.uniform(0, 0.2, S).astype(np.float32),
             phi=rng.uniform(0, 2 * np.pi, S).astype(np.float32), freq=5.0)
    p = synth.params(dt=1e-4, g=(0, 0, -9.81))
    xg, _ = gpu_run(ms, s, p, 1000, chunks=3, kernel=kernel)
    xo, _ = ora.run(s, f32p(p), 1000)
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


def test_parallel_springs_are_merged_exactly(ms, ora):
    """A voxel robot expanded by the oracle keeps the springs of neighbouring
    voxels as separate parallel springs; the library merges each pair into
    one record (summed k and c, weighted rest length, combined actuation)."""
    rng = np.random.default_rng(5)
    mat, phase = synth.random_voxel_design(rng, (4, 3, 3))
    s = ora.voxel_system(mat, phase, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS)
    s["m"] = s["m"].astype(np.float32)
    p = synth.voxel_params()
    with ms.Sim(s, p) as sim:
        inf = sim.info()
        assert inf["n_records"] < s["ij"].shape[0]
        sim.step(200)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 200)
    err = np.abs(xg - xo).max()
    assert err <= 1e-4 * body_size(s), (err, 1e-4 * body_size(s))


@pytest.mark.parametrize("kernel", KERNELS)
def test_throughput_lattice_ragged(ms, ora, kernel):
    """Throughput-lattice parameters (k ~ U[5e3,5e4], c = 0.05, anchored
    bottom, v ~ N(0,1e-3), dt = 5e-5) on a 23x24x25 box: many slices and
    blocks and a ragged last block; 200 steps."""
    x, ij, L0 = synth.box_lattice(23, 24, 25, 1e-3)
    N = x.shape[0]; S = ij.shape[0]
    rk = np.random.default_rng(0)
    rv = np.random.default_rng(1)
    fixed = (np.arange(N) < 23 * 24).astype(np.uint8)
    v = (rv.standard_normal((N, 3)) * 1e-3).astype(np.float32); v[fixed == 1] = 0
    s = dict(x=x, v=v, m=np.full(N, 1e-3, np.float32), fixed=fixed, ij=ij,
             k=rk.uniform(5e3, 5e4, S).astype(np.float32), c=np.float32(0.05), L0=L0)
    p = synth.throughput_params()
    xg, vg = gpu_run(ms, s, p, 200, kernel=kernel)
    xo, vo = ora.run(s, f32p(p), 200)
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


@pytest.mark.parametrize("kernel", KERNELS)
def test_runs_are_bit_identical(ms, kernel):
    s = synth.soft_cube(z0=0.001)
    s["v"][:] = np.array([0.3, -0.2, -0.6], np.float32)
    p = synth.soft_cube_params(contact=True)
    a, _ = gpu_run(ms, s, p, 300, kernel=kernel)
    b, _ = gpu_run(ms, s, p, 300, kernel=kernel)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kernel", KERNELS)
def test_state_round_trip_and_resume(ms, kernel):
    """get_state / set_state checkpoint: 100 + 100 steps with a save/restore
    in between equals 200 straight steps (bit for bit)."""
    import torch
    s = synth.soft_cube(n=5, z0=0.001)
    s["v"][:] = np.array([0.1, 0.0, -0.4], np.float32)
    p = synth.soft_cube_params(contact=True)
    with ms.Sim(s, p, reorder=True, kernel=kernel) as a:
        a.step(200)
        xa, va = a.get_state()
    with ms.Sim(s, p, reorder=True, kernel=kernel) as b:
        b.step(100)
        xd = torch.empty((s["x"].shape[0], 3), device="cuda")
        vd = torch.empty_like(xd)
        b.get_state(xd, vd)                      # device-side checkpoint
        b.step(37)                               # wander off ...
        b.set_state(xd, vd)                      # ... and restore
        b.step(100)
        xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_kernels_agree(ms):
    """Gather and tiled kernels sum each mass's springs in different orders;
    on a contact-free run they agree to rounding."""
    s = synth.soft_cube(n=6)
    p = synth.soft_cube_params(contact=False)
    xa, _ = gpu_run(ms, s, p, 300, kernel="gather")
    xb, _ = gpu_run(ms, s, p, 300, kernel="tiled")
    np.testing.assert_allclose(xb, xa, rtol=0, atol=1e-7)


def test_nonfinite_state_is_reported(ms):
    s = synth.soft_cube(n=3)
    s["k"][:] = 1e9                                # violently unstable at this dt
    p = synth.soft_cube_params(contact=False, dt=1e-2)
    s["x"][0, 0] += 1e-3
    with ms.Sim(s, p) as sim:
        sim.step(2000)
        with pytest.raises(ms.MsError) as e:
            sim.sync()
        assert e.value.code == 5


@pytest.mark.parametrize("kernel", KERNELS)
def test_empty_spring_set_is_free_fall(ms, kernel):
    s = dict(x=np.array([[0, 0, 1.0]], np.float32), v=np.array([[0.5, 0, 0]], np.float32),
             m=np.array([1e-3], np.float32), fixed=np.zeros(1, np.uint8),
             ij=np.zeros((0, 2), np.int32), k=np.zeros(0, np.float32), c=np.zeros(0, np.float32),
             L0=np.zeros(0, np.float32))
    p = synth.params(dt=1e-3)
    x, v = gpu_run(ms, s, p, 100, kernel=kernel)
    g = np.float32(-9.81); dt = np.float32(1e-3)
    assert abs(v[0, 2] - 100 * dt * g) < 1e-4
    assert abs(x[0, 0] - (0.0 + 100 * dt * 0.5)) < 1e-6


@pytest.mark.parametrize("kernel", ["gather", "tiled"])
@pytest.mark.parametrize("integ", ["forward_euler", "verlet", "rk4"])
def test_other_integrators_match_oracle(ms, ora, kernel, integ):
    """The paper's forward Euler (eq. 4) and position Verlet (eq. 5-6) on a
    small soft lattice without contact.  Forward Euler amplifies every mode by
    sqrt(1 + (omega dt)^2) per step, so the lattice is soft enough that the top
    mode has omega dt ~ 0.05 (growth below 1.5x over the run)."""
    s = synth.soft_cube(n=6, k=1e2, c=0.01)
    rng = np.random.default_rng(9)
    s["x"] += (2e-4 * rng.standard_normal(s["x"].shape)).astype(np.float32)
    p = synth.params(dt=2e-5, g=(0, 0, -9.81))
    with ms.Sim(s, p, kernel=kernel, integrator=integ) as sim:
        sim.step(150); sim.step(150)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 300, integrator=integ)
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


@pytest.mark.parametrize("kernel", ["gather", "tiled", "persistent"])
def test_quasi_uniform_irregular_lattice(ms, ora, kernel):
    """An irregular network (best-candidate points, degree 2..16, no lattice
    directions): the general-graph path, dropped onto the ground."""
    s = synth.quasi_uniform_lattice(1500, box=(0.1, 0.1, 0.1), seed=1)
    s["x"][:, 2] += np.float32(0.002)
    s["v"][:] = np.array([0.1, 0.0, -0.3], np.float32)
    p = synth.soft_cube_params(contact=True)
    xg, _ = gpu_run(ms, s, p, 200, kernel=kernel)
    xo, _ = ora.run(s, f32p(p), 200)
    err = np.abs(xg - xo).max()
    assert err <= 1e-4 * body_size(s), (err, 1e-4 * body_size(s))


@pytest.mark.parametrize("kernel", ["gather", "tiled"])
def test_rk4_with_actuation_anchors_and_ground_contact(ms, ora, kernel):
    """RK4 stages see the actuation at t_n + c dt and the penalty contact
    (friction off, as RK4 takes no impulse clamp): actuated lattice with an
    anchored layer, started partly below the ground."""
    x, ij, L0 = synth.box_lattice(6, 5, 4, 0.01, origin=(0, 0, -0.002))
    rng = np.random.default_rng(21)
    S = ij.shape[0]; N = x.shape[0]
    s = dict(x=x, v=(0.01 * rng.standard_normal((N, 3))).astype(np.float32),
             m=rng.uniform(1e-3, 4e-3, N).astype(np.float32), fixed=(np.arange(N) < 6).astype(np.uint8), ij=ij,
             k=rng.uniform(1e3, 1e4, S).astype(np.float32), c=rng.uniform(0, 0.1, S).astype(np.float32),
             L0=L0, A=rng.uniform(0, 0.2, S).astype(np.float32),
             phi=rng.uniform(0, 2 * np.pi, S).astype(np.float32), freq=5.0)
    p = synth.params(dt=1e-4, g=(0, 0, -9.81), contact=True, k_c=1e4, mu=0.0)
    with ms.Sim(s, p, kernel=kernel, integrator="rk4") as sim:
        sim.step(300); sim.step(200)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 500, integrator="rk4")
    err = np.abs(xg - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


def test_persistent_wide_tiles_soft_cube(ms, ora):
    """8000 masses: 16 CTAs of 512 masses with two lanes per mass, per-spring
    damping, dropped onto the ground with friction, over two calls."""
    s = synth.soft_cube(n=20, z0=0.001)
    rng = np.random.default_rng(23)
    S = s["ij"].shape[0]
    s["c"] = rng.uniform(0.0, 0.2, S).astype(np.float32)
    s["v"][:] = np.array([0.1, -0.05, -0.3], np.float32)
    p = synth.soft_cube_params(contact=True)
    with ms.Sim(s, p, kernel="persistent") as sim:
        assert sim.info()["kernel"] == 3
        sim.step(120); sim.step(80)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 200)
    err = np.abs(xg.astype(np.float64) - xo).max()
    assert err <= 1e-4 * body_size(s), (err, 1e-4 * body_size(s))


def test_persistent_wide_tiles_actuated_irregular_network(ms, ora):
    """5000 best-candidate points (10 tiles of 512, degree <= 16): actuation
    and an external force on the wide tiles, against the oracle."""
    s = synth.quasi_uniform_lattice(5000, box=(0.17, 0.17, 0.17), seed=3)
    rng = np.random.default_rng(29)
    S = s["ij"].shape[0]; N = s["x"].shape[0]
    s["A"] = rng.uniform(0, 0.1, S).astype(np.float32)
    s["phi"] = rng.uniform(0, 2 * np.pi, S).astype(np.float32)
    s["freq"] = 4.0
    s["fext"] = (1e-3 * rng.standard_normal((N, 3))).astype(np.float32)
    p = synth.soft_cube_params(contact=False)
    with ms.Sim(s, p, kernel="persistent") as sim:
        assert sim.info()["kernel"] == 3
        sim.step(150); sim.step(150)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 300)
    err = np.abs(xg.astype(np.float64) - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


def test_persistent_actuation_that_does_not_fit_shared_memory_is_refused(ms):
    """8000 masses of a 26-neighbour lattice: the records fit the wide tiles,
    their actuation coefficients do not; set_actuation says so and the
    system keeps stepping passively."""
    s = synth.soft_cube(n=20, z0=0.001)
    S = s["ij"].shape[0]
    with ms.Sim(s, synth.soft_cube_params(contact=True), kernel="persistent") as sim:
        with pytest.raises(ms.MsError) as e:
            sim.set_actuation(2.0, np.full(S, 0.1, np.float32), np.zeros(S, np.float32))
        assert e.value.code == 1 and "tiled kernel" in str(e.value)
        sim.step(10)
        x, _ = sim.get_state()
        assert np.isfinite(x).all()


def lattice24(seed, c_per_spring):
    """24^3 lattice (13 824 masses: above the cluster kernel, 27 tiles of the
    grid kernel) in the throughput lattice's style, resting on the ground."""
    x, ij, L0 = synth.box_lattice(24, 24, 24, 1e-3, origin=(0, 0, -2e-5))
    rng = np.random.default_rng(seed)
    S = ij.shape[0]; N = x.shape[0]
    return dict(x=x, v=(1e-3 * rng.standard_normal((N, 3))).astype(np.float32),
                m=np.full(N, 1e-3, np.float32), fixed=np.zeros(N, np.uint8), ij=ij,
                k=rng.uniform(5e3, 5e4, S).astype(np.float32),
                c=rng.uniform(0.0, 0.1, S).astype(np.float32) if c_per_spring else np.float32(0.05), L0=L0)


def test_persistent_grid_kernel_is_bit_identical_to_the_tiled_kernel(ms):
    """Above 8192 masses the persistent kernel runs the tiled layout in one
    cooperative launch: the same arithmetic in the same order as the per-step
    tiled launches, so the states agree bit for bit (contact, friction,
    per-spring damping, an odd and an even call length)."""
    s = lattice24(31, True)
    p = synth.params(dt=5e-5, g=(0, 0, -9.81), contact=True, k_c=1e5, mu=0.5)
    out = []
    for kernel in ("persistent", "tiled"):
        with ms.Sim(s, p, kernel=kernel) as sim:
            assert sim.info()["kernel"] == (3 if kernel == "persistent" else 2)
            sim.step(151); sim.step(100)
            out.append(sim.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_persistent_grid_kernel_actuated_lattice_matches_oracle(ms, ora):
    """22^3 masses (21 tiles) joined by edge and face-diagonal springs only
    (degree <= 19 with compact rows, so the actuation coefficients fit the
    grid kernel's shared memory), actuated, with an external force, against
    the oracle."""
    x, ij, L0 = synth.box_lattice(22, 22, 22, 1e-3, origin=(0, 0, 0.01))
    keep = L0 < 1.6e-3                                   # a and a sqrt 2, not a sqrt 3
    # plus one spring of length 2a beside an edge spring (mass 0 to mass 2): two
    # springs of one mass in one direction, so rows are compact (19 slots), not
    # one slot per lattice direction
    ij = np.concatenate([ij[keep], np.array([[0, 2]], np.int32)])
    L0 = np.concatenate([L0[keep], np.array([2e-3], np.float32)])
    rng = np.random.default_rng(37)
    S = ij.shape[0]; N = x.shape[0]
    s = dict(x=x, v=(1e-3 * rng.standard_normal((N, 3))).astype(np.float32), m=np.full(N, 1e-3, np.float32),
             fixed=(np.arange(N) < 22 * 22).astype(np.uint8), ij=ij, k=rng.uniform(5e3, 5e4, S).astype(np.float32),
             c=np.float32(0.05), L0=L0, A=rng.uniform(0, 0.1, S).astype(np.float32),
             phi=rng.uniform(0, 2 * np.pi, S).astype(np.float32), freq=40.0,
             fext=(1e-4 * rng.standard_normal((N, 3))).astype(np.float32))
    p = synth.params(dt=5e-5, g=(0, 0, -9.81), contact=False)
    with ms.Sim(s, p, kernel="persistent") as sim:
        assert sim.info()["kernel"] == 3
        sim.step(120); sim.step(80)
        xg, _ = sim.get_state()
    xo, _ = ora.run(s, f32p(p), 200)
    err = np.abs(xg.astype(np.float64) - xo).max()
    assert err <= 1e-5 * body_size(s), (err, 1e-5 * body_size(s))


def test_persistent_kernel_refuses_more_tiles_than_multiprocessors(ms):
    """The grid kernel needs every tile resident at once: a 64^3 lattice
    (512 tiles) is refused with a message, not launched."""
    s = synth.throughput_lattice(n=64)
    with pytest.raises(ms.MsError) as e:
        ms.Sim(s, synth.throughput_params(), kernel="persistent")
    assert e.value.code == 1 and "multiprocessor" in str(e.value)


def test_set_state_rejects_non_finite_host_input_and_keeps_the_state(ms):
    """ms_set_state checks host input on the device: a NaN at caller mass 5
    returns MS_ERR_ARG naming that mass, and the state is not modified."""
    s = synth.soft_cube(n=4)
    with ms.Sim(s, synth.soft_cube_params(contact=False)) as sim:
        sim.step(3)
        x0, v0 = sim.get_state()
        xb = x0.copy(); xb[5, 1] = np.nan
        xb[9, 0] = np.inf
        with pytest.raises(ms.MsError) as e:
            sim.set_state(xb, v0)
        assert e.value.code == 1 and "mass 5" in str(e.value)
        x1, v1 = sim.get_state()
        assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
        sim.set_state(x0 + np.float32(1e-4), v0)          # a finite state is accepted
        x2, _ = sim.get_state()
        assert np.allclose(x2, x0 + np.float32(1e-4))


def test_persistent_cluster_of_16_tiles(ms, ora):
    """4096 masses: the persistent kernel's largest cluster (16 CTAs of 256
    masses, non-portable cluster size), against the oracle; actuated, with
    contact and friction, over two calls."""
    s = synth.soft_cube(n=16, z0=0.001)
    rng = np.random.default_rng(17)
    S = s["ij"].shape[0]
    s["A"] = rng.uniform(0, 0.1, S).astype(np.float32)
    s["phi"] = rng.uniform(0, 2 * np.pi, S).astype(np.float32)
    s["freq"] = 5.0
    s["v"][:] = np.array([0.2, 0.0, -0.3], np.float32)
    p = synth.soft_cube_params(contact=True)
    xg, _ = gpu_run(ms, s, p, 200, chunks=2, kernel="persistent")
    xo, _ = ora.run(s, f32p(p), 200)
    err = np.abs(xg - xo).max()
    assert err <= 1e-4 * body_size(s), (err, 1e-4 * body_size(s))
