"""The lattice kernel (kernel 4: topology and rest lengths from the grid, only
k stored per spring) against the FP64 oracle on identical seeded inputs.

Gates are those of the other step tests: max |x_gpu - x_oracle| <= 1e-5 of the
body size after a contact-free run, <= 1e-4 after 200 steps with ground
contact (and the centre-of-mass displacement within 1 %).  The lattices are
sized so that bricks of 16 x 16 x 8 cells are cut by a ragged tail on every
axis, and some have holes (cells without a mass, inside a brick) with or
without missing springs between present masses.  A lattice where every pair
of neighbouring masses has its spring runs the kernel without a per-term
test (cells without a mass sit at a far sentinel position with k = 0); one
with a missing spring between two masses runs the variant that tests every
term.
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


def body_size(s):
    return float(np.ptp(np.asarray(s["x"], np.float64), axis=0).max())


def ragged_lattice(nx=37, ny=21, nz=11, seed=0, a=1e-3, origin=(0.0, 0.0, 0.0)):
    """The throughput lattice's recipe on a box whose sides are not multiples
    of the brick: k ~ U[5e3, 5e4], c = 0.05, bottom layer anchored,
    v ~ N(0, 1e-3)."""
    x, ij, L0 = synth.box_lattice(nx, ny, nz, a, origin=origin)
    rng = np.random.default_rng(seed)
    N, S = x.shape[0], ij.shape[0]
    return dict(x=x, v=(1e-3 * rng.standard_normal((N, 3))).astype(np.float32),
                m=np.full(N, 1e-3, np.float32), fixed=(np.arange(N) < nx * ny).astype(np.uint8), ij=ij,
                k=rng.uniform(5e3, 5e4, S).astype(np.float32), c=np.float32(0.05), L0=L0)


def drop(s, keep_mass, keep_spring=None):
    """Remove masses (and their springs), and optionally some springs."""
    ij = s["ij"]
    ks = keep_mass[ij[:, 0]] & keep_mass[ij[:, 1]]
    if keep_spring is not None:
        ks &= keep_spring
    remap = -np.ones(keep_mass.size, np.int64)
    remap[keep_mass] = np.arange(int(keep_mass.sum()))
    out = {key: (val[keep_mass] if key in ("x", "v", "m", "fixed", "fext") else val) for key, val in s.items()}
    out["ij"] = remap[ij[ks]].astype(np.int32)
    for key in ("k", "L0"):
        out[key] = s[key][ks]
    if np.ndim(s["c"]) == 1:
        out["c"] = s["c"][ks]
    return out


def run_gpu(ms, s, p, n, chunks=1, integrator="symplectic_euler", kernel="lattice", guard=None):
    with ms.Sim(s, p, kernel=kernel, integrator=integrator) as sim:
        info = sim.info()
        assert info["kernel"] == (4 if kernel == "lattice" else info["kernel"])
        if guard is not None:
            assert info["lattice_guard"] == guard
        done = 0
        for q in range(chunks):
            todo = n * (q + 1) // chunks - done
            sim.step(todo)
            done += todo
        x, v = sim.get_state()
    return x.astype(np.float64), v.astype(np.float64)


def test_ragged_throughput_lattice_200_steps(ms, ora):
    """37 x 21 x 11 masses: 3 x 2 x 2 bricks, each axis ending in a partial
    brick; gravity, anchored bottom layer, 200 steps in two calls."""
    s = ragged_lattice()
    p = synth.throughput_params()
    xg, vg = run_gpu(ms, s, p, 200, chunks=2, guard=0)
    xo, vo = ora.run(s, f32p(p), 200)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(s), np.abs(xg - xo).max()
    assert np.abs(vg - vo).max() <= 1e-3


def soft(s, seed):
    """The soft lattice of the integrator test (k ~ U[50, 150], v ~ N(0, 0.02))
    and its parameters (dt = 2e-5, gravity), on which every integrator is
    stable."""
    s["k"] = np.random.default_rng(seed).uniform(50.0, 150.0, s["ij"].shape[0]).astype(np.float32)
    s["v"] = (0.02 * np.random.default_rng(seed + 1).standard_normal(s["v"].shape)).astype(np.float32)
    return s, synth.params(dt=2e-5, g=(0, 0, -9.81))


@pytest.mark.parametrize("integ", ["symplectic_euler", "rk4"])
def test_lattice_with_holes_and_missing_springs(ms, ora, integ):
    """Cells without a mass inside the bricks (a random 10 % of the masses
    removed with their springs), and 15 % of the remaining springs removed
    between masses that stay: those pairs read k = NaN, the kernel tests every
    term, and they must exert nothing, the dashpot included.  External force
    on some masses.  RK4 on the soft lattice."""
    s = ragged_lattice(nx=29, ny=13, nz=9, seed=4)
    p = synth.throughput_params()
    if integ == "rk4":
        s, p = soft(s, 14)
    rng = np.random.default_rng(5)
    keep_m = rng.random(s["x"].shape[0]) > 0.10
    keep_m[: 29 * 13] = True                       # the anchored layer stays whole
    keep_s = rng.random(s["ij"].shape[0]) > 0.15
    t = drop(s, keep_m, keep_s)
    t["fext"] = (2e-4 * rng.standard_normal(t["x"].shape)).astype(np.float32)
    xg, _ = run_gpu(ms, t, p, 150, integrator=integ, guard=1)
    xo, _ = ora.run(t, f32p(p), 150, integrator=integ)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(t), np.abs(xg - xo).max()


@pytest.mark.parametrize("integ", ["symplectic_euler", "rk4"])
def test_lattice_with_holes_and_every_spring(ms, ora, integ):
    """Holes (a random 12 % of the masses removed with their springs) with
    every spring between the remaining neighbours kept: the kernel runs
    without the per-term test, and the cells without a mass (the sentinel
    position, k = 0 on their slots) must exert nothing, also when staged from
    the RK4 stage buffers.  External force on some masses.  RK4 on the soft
    lattice of the integrator test."""
    s = ragged_lattice(nx=29, ny=13, nz=9, seed=6)
    p = synth.throughput_params()
    if integ == "rk4":
        s, p = soft(s, 12)
    rng = np.random.default_rng(7)
    keep_m = rng.random(s["x"].shape[0]) > 0.12
    keep_m[: 29 * 13] = True
    t = drop(s, keep_m)
    t["fext"] = (2e-4 * rng.standard_normal(t["x"].shape)).astype(np.float32)
    xg, _ = run_gpu(ms, t, p, 150, chunks=2, integrator=integ, guard=0)
    xo, _ = ora.run(t, f32p(p), 150, integrator=integ)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(t), np.abs(xg - xo).max()


def test_lattice_ground_contact_200_steps(ms, ora):
    """A 19 x 17 x 6 slab thrown onto the ground (contact and friction, no
    anchors), the contact gates: 1e-4 of the body size and the centre-of-mass
    displacement within 1 %."""
    x, ij, L0 = synth.box_lattice(19, 17, 6, 0.01, origin=(0.0, 0.0, 0.001))
    N, S = x.shape[0], ij.shape[0]
    rng = np.random.default_rng(8)
    s = dict(x=x, v=np.tile(np.array([0.3, -0.2, -0.6], np.float32), (N, 1)), m=np.full(N, 1e-3, np.float32),
             fixed=np.zeros(N, np.uint8), ij=ij, k=rng.uniform(5e3, 1e4, S).astype(np.float32),
             c=np.float32(0.1), L0=L0)
    p = synth.soft_cube_params(contact=True)
    xg, _ = run_gpu(ms, s, p, 200)
    xo, vo, zmin = s["x"], s["v"], np.inf
    for c in range(20):
        xo, vo = ora.run(s, f32p(p), 10, n0=10 * c, x=xo, v=vo)
        zmin = min(zmin, xo[:, 2].min())
    assert zmin < -1e-5
    assert np.abs(xg - xo).max() <= 1e-4 * body_size(s), np.abs(xg - xo).max()
    m = s["m"].astype(np.float64)
    d_o = ora.centre_of_mass(m, xo) - ora.centre_of_mass(m, s["x"])
    d_g = ora.centre_of_mass(m, xg) - ora.centre_of_mass(m, s["x"])
    assert np.linalg.norm(d_g - d_o) <= 0.01 * np.linalg.norm(d_o)


@pytest.mark.parametrize("integ", ["forward_euler", "verlet", "rk4"])
def test_lattice_other_integrators(ms, ora, integ):
    """The paper's forward Euler (eq. 4), position Verlet (eq. 5-6) and RK4
    (eq. 7-8) on the lattice kernel.  Forward Euler amplifies every mode by
    sqrt(1 + (omega dt)^2) per step, so the lattice is soft (k ~ U[50, 150],
    dt = 2e-5: the top mode has omega dt ~ 0.05, growth below 1.5x over the
    run), as in the tiled kernel's test."""
    s = ragged_lattice(nx=18, ny=9, nz=5, seed=9)
    s["k"] = np.random.default_rng(10).uniform(50.0, 150.0, s["ij"].shape[0]).astype(np.float32)
    s["v"] = (0.02 * np.random.default_rng(11).standard_normal(s["v"].shape)).astype(np.float32)
    p = synth.params(dt=2e-5, g=(0, 0, -9.81))
    xg, _ = run_gpu(ms, s, p, 300, chunks=2, integrator=integ)
    xo, _ = ora.run(s, f32p(p), 300, integrator=integ)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(s), np.abs(xg - xo).max()


def test_lattice_runs_are_bit_identical_and_state_round_trips(ms):
    s = ragged_lattice(nx=20, ny=10, nz=6, seed=2)
    p = synth.throughput_params()
    out = []
    for _ in range(2):
        with ms.Sim(s, p, kernel="lattice") as sim:
            sim.step(50)
            out.append(sim.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    with ms.Sim(s, p, kernel="lattice") as sim:
        sim.step(25)
        x, v = sim.get_state()
        sim.step(25)
        a = sim.get_state()
        sim.set_state(x, v)                             # checkpoint restore
        sim.step(25)
        b = sim.get_state()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_lattice_energy_and_trace(ms, ora):
    """ms_energy on the lattice layout against the oracle's energies of the
    same state (positions moved 1e-5 m off the grid through set_state, so that
    the springs' extensions are well above FP32 rounding); the trace records
    the positions get_state reports."""
    s = ragged_lattice(nx=21, ny=11, nz=7, seed=3, origin=(0.0, 0.0, -2e-4))
    p = synth.throughput_params(contact=True, k_c=1e5)
    rng = np.random.default_rng(6)
    x0 = (s["x"] + 1e-5 * rng.standard_normal(s["x"].shape)).astype(np.float32)
    x0[s["fixed"].astype(bool)] = s["x"][s["fixed"].astype(bool)]
    with ms.Sim(s, p, kernel="lattice") as sim:
        sim.set_state(x0, s["v"])
        e0 = sim.energy()
        tip = [0, 21 * 11 * 7 - 1, 1000]
        sim.trace(tip, 10)
        sim.step(10)
        x, v = sim.get_state()
        e = sim.energy()
        tr = sim.get_trace()
        assert sim.energy() == e                        # fixed reduction order
    v0 = s["v"].copy(); v0[s["fixed"].astype(bool)] = 0
    for got_all, (xs, vs) in ((e0, (x0, v0)), (e, (x, v))):
        want_all = ora.energy(s, f32p(p), xs.astype(np.float64), vs.astype(np.float64))
        for got, want in zip(got_all, want_all):
            assert abs(got - want) <= 1e-5 * max(abs(want), 1e-12) + 1e-12, (got, want)
    assert e[3] > 0                                     # part of it is in the ground
    assert np.array_equal(tr[-1], x[tip])


@pytest.mark.parametrize("integ", ["symplectic_euler", "rk4"])
def test_actuated_lattice(ms, ora, integ):
    """Actuated rest lengths L0 (1 + A sin(2 pi f t + phi)) on the lattice
    kernel (reading R3; every spring its own A, phi): the kernel reads each
    spring's (alpha, beta) = A (cos phi, sin phi) beside its k.  Holes and
    missing springs as well (the variant that tests every term).  RK4 stages
    see the actuation at t_n + c dt.  Against the oracle after 300 steps, and
    ms_energy against the oracle's energy with the actuated rest lengths at
    the final time."""
    s = ragged_lattice(nx=19, ny=11, nz=9, seed=15)
    if integ == "rk4":
        s, p = soft(s, 16)
    else:
        p = synth.throughput_params()
    rng = np.random.default_rng(17)
    keep_m = rng.random(s["x"].shape[0]) > 0.08
    keep_m[: 19 * 11] = True
    keep_s = rng.random(s["ij"].shape[0]) > 0.05
    t = drop(s, keep_m, keep_s)
    S = t["ij"].shape[0]
    t["A"] = rng.uniform(0.0, 0.05, S).astype(np.float32)
    t["phi"] = rng.uniform(0.0, 2 * np.pi, S).astype(np.float32)
    t["freq"] = 40.0
    n = 300
    with ms.Sim(t, p, kernel="lattice", integrator=integ) as sim:
        assert sim.info()["kernel"] == 4 and sim.info()["lattice_guard"] == 1
        sim.step(n // 2)
        sim.step(n - n // 2)
        xg, vg = sim.get_state()
        eg = sim.energy()
    xo, vo = ora.run(t, f32p(p), n, integrator=integ)
    assert np.abs(xg - xo).max() <= 1e-5 * body_size(t), np.abs(xg - xo).max()
    eo = ora.energy(t, f32p(p), xg.astype(np.float64), vg.astype(np.float64), t=n * float(np.float32(p["dt"])))
    assert abs(eg[1] - eo[1]) <= 1e-4 * abs(eo[1]), (eg[1], eo[1])


def test_actuating_then_stopping_a_lattice(ms, ora):
    """ms_set_actuation on a lattice that took the lattice kernel by default
    (a box of 2^18 masses) is accepted, and clearing it (amp = NULL) returns
    the plain step: the state then follows the unactuated oracle."""
    s = ragged_lattice(nx=64, ny=64, nz=64, seed=18)
    p = synth.throughput_params()
    S = s["ij"].shape[0]
    with ms.Sim(s, p) as sim:
        assert sim.info()["kernel"] == 4
        sim.set_actuation(40.0, np.full(S, 0.01, np.float32), np.zeros(S, np.float32))
        sim.set_actuation(0.0, None, None)
        sim.step(3)
        idx = np.arange(0, s["x"].shape[0], 997)
        xg, _ = sim.get_state()
    sub = ora.run(s, f32p(p), 3)[0]
    assert np.abs(xg[idx] - sub[idx]).max() <= 1e-5 * body_size(s)


def test_default_kernel_by_size(ms):
    """With kernel 0 a box lattice takes the lattice layout from 2^18 masses
    (64^3) and the tiled layout below; an irregular network of that size stays
    tiled."""
    p = synth.throughput_params()
    for dims, want in (((64, 64, 64), 4), ((63, 64, 64), 2)):
        s = ragged_lattice(nx=dims[0], ny=dims[1], nz=dims[2], seed=3)
        with ms.Sim(s, p) as sim:
            assert sim.info()["kernel"] == want, (dims, sim.info()["kernel"])
    s = ragged_lattice(nx=64, ny=64, nz=64, seed=3)
    s["x"] = s["x"] + np.float32(1e-4) * np.random.default_rng(3).standard_normal(s["x"].shape).astype(np.float32)
    with ms.Sim(s, p) as sim:
        assert sim.info()["kernel"] == 2


def test_lattice_kernel_refusals(ms):
    s = ragged_lattice(nx=8, ny=8, nz=4)
    p = synth.throughput_params()
    with ms.Sim(s, p, kernel="lattice") as sim:
        with pytest.raises(ms.MsError) as e:
            sim.set_actuation(2.0, np.full(s["ij"].shape[0], np.nan), np.zeros(s["ij"].shape[0]))
        assert e.value.code == 1
    t = dict(s, c=np.linspace(0.01, 0.02, s["ij"].shape[0]).astype(np.float32))
    with pytest.raises(ms.MsError) as e:
        ms.Sim(t, p, kernel="lattice")
    assert "dashpot" in str(e.value)
