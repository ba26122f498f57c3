"""Pins of the FP64 oracle against results the paper and the mathematics fix.

None of these compares the oracle with a retyped copy of its own formula:
each checks a closed form, an invariant, a hand-worked example, a special
case solved by a library routine, or a count.  A plausible mistake in the
oracle (a dropped term, a wrong sign or index, a transposed operand, the
wrong integrator) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def point_mass(x0, v0, m=1e-3):
    return dict(x=np.array([x0], np.float64), v=np.array([v0], np.float64), m=np.array([m]),
                fixed=np.zeros(1, np.uint8), ij=np.zeros((0, 2), np.int32), k=np.zeros(0),
                c=np.zeros(0), L0=np.zeros(0), freq=0.0)


# ---------------------------------------------------------------- free fall
@pytest.mark.parametrize("damping", [0.0, 3e-3])
def test_free_fall_closed_form(ora, damping):
    """eq. 2-3 with gravity only.  Symplectic Euler: v_n = r^n v0 + dt g sum_{k=1..n} r^k,
    x_n = x0 + dt sum_{m=1..n} v_m, r = 1 - d (geometric sums in closed form)."""
    x0 = np.array([0.1, -0.2, 0.3]); v0 = np.array([0.3, -0.2, 1.0]); g = np.array([0.0, 0.0, -9.81])
    dt, n = 1e-3, 1500
    s = point_mass(x0, v0)
    x, v = ora.run(s, synth.params(dt=dt, g=tuple(g), vel_damping=damping), n)
    r = 1.0 - damping
    if damping == 0.0:
        v_ref = v0 + n * dt * g
        x_ref = x0 + n * dt * v0 + dt * dt * g * n * (n + 1) / 2
    else:
        geo = lambda q: r * (1 - r ** q) / (1 - r)            # sum_{k=1..q} r^k
        v_ref = r ** n * v0 + dt * g * geo(n)
        sum_geo = r / (1 - r) * (n - geo(n))                  # sum_{m=1..n} geo(m)
        x_ref = x0 + dt * (v0 * geo(n) + dt * g * sum_geo)
    np.testing.assert_allclose(v[0], v_ref, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(x[0], x_ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("integ,ref", [
    ("forward_euler", lambda x0, v0, g, h, n: x0 + n * h * v0 + h * h * g * n * (n - 1) / 2),
    ("verlet", lambda x0, v0, g, h, n: x0 + n * h * v0 + h * h * g * n * n / 2),
    ("rk4", lambda x0, v0, g, h, n: x0 + n * h * v0 + h * h * g * n * n / 2),
])
def test_free_fall_other_integrators(ora, integ, ref):
    """eq. 4 lags the position by one kick; eq. 5-6 and RK4 integrate a constant
    acceleration exactly (a parabola)."""
    x0 = np.array([0.0, 0.0, 1.0]); v0 = np.array([0.2, 0.0, 0.5]); g = np.array([0.0, 0.0, -9.81])
    h, n = 2e-3, 400
    x, _ = ora.run(point_mass(x0, v0), synth.params(dt=h, g=tuple(g)), n, integrator=integ)
    np.testing.assert_allclose(x[0], ref(x0, v0, g, h, n), rtol=1e-11, atol=1e-12)


# ------------------------------------------------------- hand-worked steps
def _golden_cases():
    with open(os.path.join(HERE, "golden", "hand_steps.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_worked_steps(ora, case):
    s = dict(x=np.array(case["x"], float), v=np.array(case["v"], float), m=np.array(case["m"], float),
             fixed=np.array(case["fixed"], np.uint8), ij=np.array(case["ij"], np.int32),
             k=np.array(case["k"], float), c=np.array(case["c"], float), L0=np.array(case["L0"], float),
             freq=case.get("freq", 0.0))
    if "A" in case:
        s["A"] = np.array(case["A"], float); s["phi"] = np.array(case["phi"], float)
    x, v = ora.run(s, synth.params(dt=case["dt"], g=(0, 0, 0)), case["nsteps"])
    np.testing.assert_allclose(x, case["x_out"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(v, case["v_out"], rtol=1e-12, atol=1e-13)


def test_zero_length_spring_exerts_nothing(ora):
    s = point_mass([0, 0, 0], [0, 0, 0])
    s.update(x=np.zeros((2, 3)), v=np.zeros((2, 3)), m=np.ones(2), fixed=np.zeros(2, np.uint8),
             ij=np.array([[0, 1]], np.int32), k=np.array([5.0]), c=np.array([1.0]), L0=np.array([1.0]))
    x, v = ora.run(s, synth.params(dt=0.1, g=(0, 0, 0)), 3)
    assert np.all(np.isfinite(x)) and np.all(x == 0) and np.all(v == 0)


# ------------------------------------------------------------ 1-D chains
def chain(n_free, k, m, L0, fixed_first, eps_mode=None):
    """Chain along x: node 0 (anchored if fixed_first) ... node n_free."""
    N = n_free + (1 if fixed_first else 0)
    x = np.zeros((N, 3)); x[:, 0] = np.arange(N) * L0
    ij = np.array([(i, i + 1) for i in range(N - 1)], np.int32)
    fixed = np.zeros(N, np.uint8)
    if fixed_first:
        fixed[0] = 1
    return dict(x=x, v=np.zeros((N, 3)), m=np.full(N, m), fixed=fixed, ij=ij,
                k=np.full(N - 1, k), c=np.zeros(N - 1), L0=np.full(N - 1, L0), freq=0.0)


@pytest.mark.parametrize("j", [1, 3])
def test_chain_eigenmode_closed_form(ora, j):
    """Fixed-free chain of n free masses: mode j has shape sin(i theta_j),
    theta_j = (2j-1) pi/(2n+1), omega_j = 2 sqrt(k/m) sin(theta_j/2).  The 1-D
    axial chain is exactly linear, and symplectic Euler maps the modal
    coordinate by q_{n+1} = (2 - h^2 w^2) q_n - q_{n-1}, so
    q_n = q0 [cos(n psi) - (h^2 w^2/2)/sin(psi) sin(n psi)], cos psi = 1 - h^2 w^2/2."""
    n, k, m, L0, h = 12, 4e3, 2e-3, 0.01, 1e-4
    s = chain(n, k, m, L0, fixed_first=True)
    theta = (2 * j - 1) * math.pi / (2 * n + 1)
    w = 2 * math.sqrt(k / m) * math.sin(theta / 2)
    shape = np.sin(np.arange(n + 1) * theta)          # node 0 is the wall
    eps = 1e-5
    s["x"][:, 0] += eps * shape
    psi = math.acos(1 - (h * w) ** 2 / 2)
    B = -((h * w) ** 2 / 2) / math.sin(psi)
    xs, vs = s["x"].copy(), s["v"].copy()
    for step in (1, 7, 150, 1000):
        xs, vs = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), step if step == 1 else step - prev, n0=0, x=xs, v=vs)
        prev = step
        q = eps * (math.cos(step * psi) + B * math.sin(step * psi))
        u = xs[:, 0] - np.arange(n + 1) * L0
        np.testing.assert_allclose(u, q * shape, rtol=0, atol=1e-9 * eps * n + 1e-17)
        assert np.all(xs[:, 1:] == 0)


def test_chain_frequency_by_zero_crossings(ora):
    """Natural frequency of the fixed-free chain, measured the way the
    Euler-Bernoulli tests measure it (count crossings of the start position
    by the traced tip mass), against omega_1 = 2 sqrt(k/m) sin(pi/(2(2n+1)))."""
    n, k, m, L0, h = 6, 1e3, 1e-3, 0.01, 1e-5
    s = chain(n, k, m, L0, fixed_first=True)
    theta = math.pi / (2 * n + 1)
    w1 = 2 * math.sqrt(k / m) * math.sin(theta / 2)
    s["x"][:, 0] += 1e-5 * np.sin(np.arange(n + 1) * theta)
    T = 0.2
    steps = int(round(T / h))
    chunk = 50
    xs, vs = s["x"], s["v"]
    tip0 = n * L0                    # equilibrium position of the tip
    trace = []
    for c0 in range(0, steps, chunk):
        xs, vs = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), chunk, n0=c0, x=xs, v=vs)
        trace.append(xs[-1, 0] - tip0)
    trace = np.array(trace)
    crossings = np.flatnonzero(np.sign(trace[1:]) != np.sign(trace[:-1]))
    # interpolate crossing times, frequency from first to last crossing
    tc = [(c + trace[c] / (trace[c] - trace[c + 1])) * chunk * h for c in crossings]
    f_meas = (len(tc) - 1) / (2 * (tc[-1] - tc[0]))
    f_ref = w1 / (2 * math.pi)
    assert abs(f_meas - f_ref) / f_ref < 2e-3, (f_meas, f_ref)


def test_modified_energy_is_exact_for_linear_chain(ora):
    """Symplectic Euler conserves E = 1/2 v'Mv + 1/2 u'Ku - (h/2) u'Kv exactly for a
    linear system; the free-free axial chain's K is the graph Laplacian * k."""
    n, k, m, L0, h = 9, 2e3, 1e-3, 0.01, 2e-4
    s = chain(n, k, m, L0, fixed_first=False)
    N = s["x"].shape[0]
    rng = np.random.default_rng(7)
    s["x"][:, 0] += 1e-5 * rng.standard_normal(N)
    s["v"][:, 0] = 1e-3 * rng.standard_normal(N)
    K = np.zeros((N, N))
    for i in range(N - 1):
        K[i, i] += k; K[i + 1, i + 1] += k; K[i, i + 1] -= k; K[i + 1, i] -= k
    def E(x, v):
        u = x[:, 0] - np.arange(N) * L0
        vv = v[:, 0]
        return 0.5 * m * vv @ vv + 0.5 * u @ K @ u - 0.5 * h * u @ K @ vv
    E0 = E(s["x"], s["v"])
    x, v = s["x"], s["v"]
    for c in range(20):
        x, v = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), 500, n0=500 * c, x=x, v=v)
        assert abs(E(x, v) - E0) <= 1e-9 * E0


# --------------------------------------------------- integrators on eq. 3
def test_forward_euler_and_verlet_on_harmonic_oscillator(ora):
    """Single mass on a spring to an anchor (1-D, linear): forward Euler (eq. 4)
    gives q_n = q0 r^n cos(n a), r = sqrt(1 + h^2 w^2), tan a = h w; Verlet
    (eq. 5-6) gives q_n = q0 cos(n psi), cos psi = 1 - h^2 w^2/2."""
    k, m, L0, h, q0 = 50.0, 0.5, 1.0, 2e-2, 1e-3
    s = chain(1, k, m, L0, fixed_first=True)
    s["x"][1, 0] += q0
    w = math.sqrt(k / m)
    n = 300
    x, _ = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), n, integrator="forward_euler")
    r = math.sqrt(1 + (h * w) ** 2); a = math.atan(h * w)
    assert abs((x[1, 0] - L0) - q0 * r ** n * math.cos(n * a)) < 1e-12
    x, _ = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), n, integrator="verlet")
    psi = math.acos(1 - (h * w) ** 2 / 2)
    assert abs((x[1, 0] - L0) - q0 * math.cos(n * psi)) < 1e-12


def test_rk4_matches_taylor_propagator(ora):
    """For z' = A z, one classical RK4 step is z <- (I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24) z."""
    k, m, L0, h, q0, p0 = 80.0, 0.2, 1.0, 1e-2, 1e-3, 2e-3
    s = chain(1, k, m, L0, fixed_first=True)
    s["x"][1, 0] += q0; s["v"][1, 0] = p0
    n = 250
    x, v = ora.run(s, synth.params(dt=h, g=(0, 0, 0)), n, integrator="rk4")
    Am = np.array([[0.0, 1.0], [-k / m, 0.0]]) * h
    R = np.eye(2) + Am + Am @ Am / 2 + Am @ Am @ Am / 6 + Am @ Am @ Am @ Am / 24
    z = np.linalg.matrix_power(R, n) @ np.array([q0, p0])
    assert abs((x[1, 0] - L0) - z[0]) < 1e-13 and abs(v[1, 0] - z[1]) < 1e-12


# ------------------------------------------------------------ invariants
def random_lattice(seed=3, with_actuation=True):
    x, ij, L0 = synth.box_lattice(4, 3, 3, 0.01)
    rng = np.random.default_rng(seed)
    N = x.shape[0]; S = ij.shape[0]
    s = dict(x=x.astype(np.float64) + 1e-3 * rng.standard_normal((N, 3)),
             v=0.05 * rng.standard_normal((N, 3)), m=rng.uniform(1e-3, 3e-3, N),
             fixed=np.zeros(N, np.uint8), ij=ij, k=rng.uniform(1e2, 1e3, S),
             c=rng.uniform(0, 0.05, S), L0=L0.astype(np.float64), freq=3.0)
    if with_actuation:
        s["A"] = rng.uniform(0, 0.2, S); s["phi"] = rng.uniform(0, 2 * np.pi, S)
    return s


def test_linear_and_angular_momentum_conserved(ora):
    """No gravity, contact or anchors: spring forces are pairwise opposite and
    central, so sum m v and sum x cross m v are constant under symplectic Euler
    (x_{n+1} x v' = x_n x v' because x_{n+1} - x_n is parallel to v')."""
    s = random_lattice()
    P = lambda v: (s["m"][:, None] * v).sum(0)
    Lm = lambda x, v: np.cross(x, s["m"][:, None] * v).sum(0)
    P0, L0_ = P(s["v"]), Lm(s["x"], s["v"])
    x, v = ora.run(s, synth.params(dt=1e-4, g=(0, 0, 0)), 2000)
    assert np.abs(x - s["x"]).max() > 1e-4          # it did move
    np.testing.assert_allclose(P(v), P0, rtol=0, atol=1e-12 * np.abs(P0).max())
    np.testing.assert_allclose(Lm(x, v), L0_, rtol=0, atol=1e-12 * np.abs(L0_).max())


def test_actuation_work_balances_the_energy_change(ora):
    """Actuated springs with damping, gravity and contact off.  The energy the
    actuation puts in is the time integral of dE/dt at a fixed state:
    dE/dt = -sum k (l - L) dL/dt, with dL/dt = L0 A 2 pi f cos(2 pi f t + phi)
    (the rest-length law of the actuation reading).  This must equal the
    change of kinetic + elastic energy along the oracle's trajectory, to the
    integrator's first-order accuracy (0.6 % at this step, 0.3 % at half of it).
    A wrong sign, phase, amplitude or frequency in the rest length of either
    the force or the energy breaks the balance by far more: the phase's sign
    flipped in the energy alone gives 240 %."""
    x0, ij, L0 = synth.box_lattice(4, 3, 3, 0.01)
    rng = np.random.default_rng(3)
    N = x0.shape[0]; S = ij.shape[0]
    s = dict(x=x0.astype(np.float64), v=np.zeros((N, 3)), m=rng.uniform(1e-3, 3e-3, N),
             fixed=np.zeros(N, np.uint8), ij=ij, k=rng.uniform(1e2, 1e3, S), c=np.zeros(S),
             L0=L0.astype(np.float64), freq=3.0, A=rng.uniform(0.05, 0.2, S), phi=rng.uniform(0, 2 * np.pi, S))
    dt, n_steps = 2e-5, 20000
    p = synth.params(dt=dt, g=(0, 0, 0))
    w = 2 * np.pi * s["freq"]

    def total(x, v, n):
        ke, pe, _, _ = ora.energy(s, p, x, v, t=n * dt)
        return ke + pe

    def power(x, n):                      # dE/dt at a fixed state
        d = x[ij[:, 1]] - x[ij[:, 0]]
        l = np.sqrt((d * d).sum(axis=1))
        L = s["L0"] * (1 + s["A"] * np.sin(w * n * dt + s["phi"]))
        dL = s["L0"] * s["A"] * w * np.cos(w * n * dt + s["phi"])
        return float(np.sum(-s["k"] * (l - L) * dL))

    arrays = ora._Arrays(s)
    x, v = s["x"].copy(), s["v"].copy()
    e0, work, p_prev = total(x, v, 0), 0.0, power(x, 0)
    for n in range(n_steps):
        x, v = ora.run(s, p, 1, n0=n, x=x, v=v, arrays=arrays)
        p_now = power(x, n + 1)
        work += 0.5 * (p_prev + p_now) * dt
        p_prev = p_now
    d_e = total(x, v, n_steps) - e0
    assert abs(work) > 1e-3                          # the actuation did pump energy in
    assert abs(d_e - work) <= 0.02 * abs(work), (d_e, work)


def test_nonlinear_lattice_energy_has_no_drift(ora):
    """Energy Conservation Tests: damping off, kinetic + elastic energy
    oscillates about a constant; a least-squares slope over the run stays far
    below the oscillation amplitude.  (Gravity is left out: under a constant
    force symplectic Euler's energy carries an exact O(dt) bias,
    -m g^2 dt^2 n/2, which the free-fall pin already fixes.)"""
    s = random_lattice(seed=5, with_actuation=False)
    s["c"][:] = 0.0
    p = synth.params(dt=5e-5, g=(0, 0, 0))
    x, v = s["x"], s["v"]
    E0 = sum(ora.energy(s, p, x, v))
    E = []
    for c in range(200):
        x, v = ora.run(s, p, 250, n0=250 * c, x=x, v=v)
        E.append(sum(ora.energy(s, p, x, v)))
    E = np.array(E)
    slope = np.polyfit(np.arange(E.size), E, 1)[0] * E.size
    assert abs(slope) < 2e-3 * E0, (slope, E0)
    assert (E.max() - E.min()) < 0.05 * E0
    assert abs(E.mean() - E0) < 0.01 * E0


# --------------------------------------------------------- ground contact
def test_resting_penetration(ora):
    """A mass on the ground plane settles at z = -m g / k_c."""
    m, kc, g = 1e-3, 1e5, 9.81
    s = point_mass([0, 0, 0.0005], [0, 0, 0], m=m)
    p = synth.params(dt=1e-4, k_c=kc, contact=True, mu=0.5, vel_damping=5e-3)
    x, v = ora.run(s, p, 20000)
    assert abs(x[0, 2] - (-m * g / kc)) < 1e-12 and abs(v[0, 2]) < 1e-9
    # started exactly there, it stays there
    s2 = point_mass([0, 0, -m * g / kc], [0, 0, 0], m=m)
    x, v = ora.run(s2, synth.params(dt=1e-4, k_c=kc, contact=True), 1000)
    assert abs(x[0, 2] + m * g / kc) < 1e-15


def test_coulomb_friction_stopping(ora):
    """A particle in equilibrium penetration (Fn = m g) sliding at v0 loses
    mu g dt of speed per step until it sticks: |v_n| = max(0, v0 - n mu g dt),
    x_n = x0 + dt sum_{j<=n} |v_j| v0/|v0|."""
    m, kc, g, mu, dt = 2e-3, 1e5, 9.81, 0.5, 1e-4
    v0 = np.array([0.3, 0.4, 0.0]); s0 = np.linalg.norm(v0)
    z0 = -m * g / kc
    s = point_mass([0.0, 0.0, z0], v0, m=m)
    p = synth.params(dt=dt, k_c=kc, contact=True, mu=mu)
    for n in (1, 50, 101, 200):
        x, v = ora.run(s, p, n)
        speeds = np.maximum(0.0, s0 - np.arange(1, n + 1) * mu * g * dt)
        np.testing.assert_allclose(np.linalg.norm(v[0, :2]), speeds[-1], rtol=0, atol=1e-12)
        np.testing.assert_allclose(x[0, :2], dt * speeds.sum() * v0[:2] / s0, rtol=0, atol=1e-12)


# ------------------------------------------------------ energy potentials
def test_gravitational_energy_is_the_potential_of_free_fall(ora):
    """Energy Conservation Tests (gravitational energy): along the exact
    free-fall trajectory x(t) = x0 + v0 t + g t^2/2, v(t) = v0 + g t, the sum
    kinetic + gravitational energy is constant.  A gravity vector with three
    non-zero components checks every axis; a flipped sign or a wrong factor
    in the gravitational term leaves a remainder that grows with t."""
    m = np.array([2e-3, 5e-3])
    g = np.array([0.7, -1.3, -9.81])
    x0 = np.array([[0.1, 0.2, 0.5], [-0.3, 0.0, 1.0]]); v0 = np.array([[0.2, -0.1, 1.5], [0.0, 0.4, -0.2]])
    s = dict(x=x0, v=v0, m=m, fixed=np.zeros(2, np.uint8), ij=np.zeros((0, 2), np.int32),
             k=np.zeros(0), c=np.zeros(0), L0=np.zeros(0))
    p = synth.params(g=tuple(g))
    E = []
    for t in np.linspace(0.0, 0.6, 13):
        ke, pe, gpe, cpe = ora.energy(s, p, x0 + v0 * t + 0.5 * g * t * t, v0 + g * t)
        assert pe == 0.0 and cpe == 0.0
        E.append(ke + gpe)
    ke0 = ora.energy(s, p, x0, v0)[0]
    assert ke0 > 0 and np.ptp(E) <= 1e-12 * ke0 * 10, np.ptp(E)
    # and the potential falls along g: a mass moved by +g/|g| loses m |g| per metre
    step = g / np.linalg.norm(g)
    d = ora.energy(s, p, x0 + step, v0)[2] - ora.energy(s, p, x0, v0)[2]
    assert abs(d + m.sum() * np.linalg.norm(g)) <= 1e-12


def test_ground_energy_is_the_potential_of_the_penalty_force(ora):
    """Reading R4's penalty k_c max(0, -z): a mass entering the ground at v0
    with gravity off moves as z(t) = -(v0/w) sin(w t), v = -v0 cos(w t),
    w = sqrt(k_c/m), while z < 0; kinetic + ground energy stays m v0^2/2.
    Above the plane, and with contact off, the ground term is zero."""
    m, kc, v0 = 3e-3, 2e4, 0.8
    w = math.sqrt(kc / m)
    s = dict(x=np.zeros((1, 3)), v=np.zeros((1, 3)), m=np.array([m]), fixed=np.zeros(1, np.uint8),
             ij=np.zeros((0, 2), np.int32), k=np.zeros(0), c=np.zeros(0), L0=np.zeros(0))
    p = synth.params(g=(0, 0, 0), k_c=kc, contact=True)
    for t in np.linspace(0.01, 0.99, 9) * math.pi / w:
        x = np.array([[0.3, -0.2, -(v0 / w) * math.sin(w * t)]])
        v = np.array([[0.0, 0.0, -v0 * math.cos(w * t)]])
        ke, pe, gpe, cpe = ora.energy(s, p, x, v)
        assert cpe > 0
        assert abs(ke + cpe - 0.5 * m * v0 * v0) <= 1e-14
    assert ora.energy(s, p, np.array([[0, 0, 1e-3]]), np.zeros((1, 3)))[3] == 0.0
    assert ora.energy(s, synth.params(g=(0, 0, 0), k_c=kc, contact=False),
                      np.array([[0, 0, -1e-3]]), np.zeros((1, 3)))[3] == 0.0


def test_resting_penetration_is_the_minimum_of_the_potential(ora):
    """Gravity plus the ground penalty: the total potential of a resting mass
    is stationary at the penetration the oracle's dynamics settle at,
    z* = -m g / k_c (test_resting_penetration), and curves up with k_c.
    A sign slip in either term, or a factor 2 in the ground term, moves the
    stationary point away from z*."""
    m, kc, g = 1e-3, 1e5, 9.81
    s = dict(x=np.zeros((1, 3)), v=np.zeros((1, 3)), m=np.array([m]), fixed=np.zeros(1, np.uint8),
             ij=np.zeros((0, 2), np.int32), k=np.zeros(0), c=np.zeros(0), L0=np.zeros(0))
    p = synth.params(g=(0, 0, -g), k_c=kc, contact=True)
    V = lambda z: sum(ora.energy(s, p, np.array([[0.0, 0.0, z]]), np.zeros((1, 3)))[2:])
    zs, h = -m * g / kc, 1e-9
    dV = (V(zs + h) - V(zs - h)) / (2 * h)
    d2V = (V(zs + h) - 2 * V(zs) + V(zs - h)) / (h * h)
    assert abs(dV) <= 1e-6 * m * g, dV
    assert abs(d2V - kc) <= 1e-3 * kc, d2V


# --------------------------------------------------------- threaded oracle
def test_threaded_oracle_equals_the_serial_oracle_bit_for_bit(ora):
    """The all-cores timing variant sums each mass's springs in the serial
    order, so its states equal ora_run's exactly: an actuated, damped, anchored
    lattice with ground contact and friction, on 1, 3 and 8 threads."""
    s = random_lattice(seed=11)
    s["fixed"] = (np.arange(s["x"].shape[0]) % 7 == 0).astype(np.uint8)
    s["x"][:, 2] -= 0.004                      # part of it starts inside the ground
    p = synth.params(dt=1e-4, k_c=1e4, mu=0.4, contact=True, vel_damping=1e-4)
    xs, vs = ora.run(s, p, 300)
    for T in (1, 3, 8):
        xt, vt, used = ora.run_threads(s, p, 300, T)
        assert 1 <= used <= T
        assert np.array_equal(xt, xs) and np.array_equal(vt, vs), T


# ------------------------------------------------------------- cantilever
def _stiffness_matrix(s):
    """Linear-elastic stiffness of a spring network about its start geometry."""
    import scipy.sparse as sp
    x = s["x"].astype(np.float64); ij = s["ij"]; k = s["k"].astype(np.float64)
    d = x[ij[:, 1]] - x[ij[:, 0]]
    u = d / np.linalg.norm(d, axis=1)[:, None]
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            kab = k * u[:, a] * u[:, b]
            for (p, q, sg) in ((0, 0, 1), (1, 1, 1), (0, 1, -1), (1, 0, -1)):
                rows.append(3 * ij[:, p] + a); cols.append(3 * ij[:, q] + b); vals.append(sg * kab)
    N = x.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(3 * N, 3 * N))


@pytest.mark.slow
def test_cantilever_relaxes_to_linear_static_solution(ora):
    """Euler-Bernoulli beam setup (tip load, damped relaxation): the relaxed
    tip deflection of the 40x4x4 lattice matches the linear static solve
    K_ff u = f (scipy sparse) within 1 %."""
    import scipy.sparse.linalg as spla
    s = synth.cantilever(40, 4, 4, a=0.01, m=1e-3, k=1e4, c=0.1, tip_load=0.01)
    K = _stiffness_matrix(s)
    free = np.repeat(s["fixed"] == 0, 3)
    f = s["fext"].astype(np.float64).ravel()
    u = np.zeros(f.size)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), f[free])
    tip = (np.arange(s["x"].shape[0]) % 40) == 39
    dz_lin = u.reshape(-1, 3)[tip, 2].mean()
    p = synth.params(dt=1e-4, g=(0, 0, 0), vel_damping=2e-3)
    x, v = ora.run(s, p, 20000)
    dz = (x[tip, 2] - s["x"][tip, 2]).mean()
    assert abs(dz - dz_lin) <= 0.01 * abs(dz_lin), (dz, dz_lin)
    assert 4e-4 < -dz_lin < 7e-4


@pytest.mark.slow
def test_cantilever_natural_frequency_matches_generalized_eigenproblem(ora):
    """Natural Frequency Analysis: the lowest root of K phi = w^2 M phi
    (scipy eigsh, shift-invert) against the frequency of the released
    beam's tip trace (zero crossings of the tip z about its mean)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nx = 20
    s = synth.cantilever(nx, 4, 4, a=0.01, m=1e-3, k=1e4, c=0.0, tip_load=0.01)
    K = _stiffness_matrix(s)
    free = np.repeat(s["fixed"] == 0, 3)
    Kf = K[free][:, free].tocsc()
    Mf = sp.diags(np.repeat(s["m"].astype(np.float64), 3)[free])
    w2 = spla.eigsh(Kf, k=1, M=Mf, sigma=0.0, which="LM", return_eigenvectors=False)
    f_ref = math.sqrt(w2[0]) / (2 * math.pi)
    # deflect statically, release with no damping and no load
    f = s["fext"].astype(np.float64).ravel()
    u = np.zeros(f.size); u[free] = spla.spsolve(Kf, f[free])
    s2 = dict(s); s2.pop("fext")
    x = s["x"].astype(np.float64) + u.reshape(-1, 3)
    h = 1e-4
    tip = (np.arange(s["x"].shape[0]) % nx) == nx - 1
    v = np.zeros_like(x); trace = []
    for c in range(400):
        x, v = ora.run(s2, synth.params(dt=h, g=(0, 0, 0)), 20, n0=20 * c, x=x, v=v)
        trace.append(x[tip, 2].mean())
    tr = np.array(trace) - np.mean(trace)
    cr = np.flatnonzero(np.sign(tr[1:]) != np.sign(tr[:-1]))
    tc = [(c + tr[c] / (tr[c] - tr[c + 1])) * 20 * h for c in cr]
    f_meas = (len(tc) - 1) / (2 * (tc[-1] - tc[0]))
    assert abs(f_meas - f_ref) / f_ref < 0.02, (f_meas, f_ref)


# ---------------------------------------------------------- lattice shapes
@pytest.mark.parametrize("dims", [(10, 10, 10), (4, 3, 2), (40, 4, 4), (1, 1, 5), (2, 2, 2)])
def test_lattice_spring_counts(dims):
    """26-neighbourhood, each pair once: 10^3 nodes give 2700 axis + 4860 face +
    2916 body = 10476 springs; the generator and the closed-form count agree
    and every pair is unique, within sqrt(3) spacing and listed once."""
    x, ij, L0 = synth.box_lattice(*dims, 0.01)
    assert ij.shape[0] == synth.lattice_spring_count(*dims)
    key = np.minimum(ij[:, 0], ij[:, 1]).astype(np.int64) * x.shape[0] + np.maximum(ij[:, 0], ij[:, 1])
    assert np.unique(key).size == ij.shape[0]
    d = np.linalg.norm(x[ij[:, 1]].astype(float) - x[ij[:, 0]], axis=1)
    assert d.max() < 0.01 * math.sqrt(3) * 1.0001
    np.testing.assert_allclose(d, L0, rtol=1e-5)   # float32 positions


def test_lattice_counts_at_workload_sizes():
    assert synth.lattice_spring_count(10, 10, 10) == 10476
    assert synth.lattice_spring_count(256, 256, 256) == 216338940


def test_voxel_expansion_single_and_pair(ora):
    """Voxel lattice: a single voxel has 8 corner masses of voxel_mass/8 and 28
    springs (12 edges, 12 face diagonals, 4 body diagonals); two face-sharing
    voxels share 4 corners and keep their own springs (56 = 2*28)."""
    mats = synth.VOXEL_MATERIALS
    one = np.ones((1, 1, 1), np.uint8)
    s = ora.voxel_system(one, np.zeros((1, 1, 1)), mats, 2.0, 0.01, 0.03)
    assert s["x"].shape[0] == 8 and s["ij"].shape[0] == 28
    np.testing.assert_allclose(s["m"], 0.03 / 8)
    L = np.sort(s["L0"])
    np.testing.assert_allclose(L[:12], 0.01, rtol=1e-6)
    np.testing.assert_allclose(L[12:24], 0.01 * math.sqrt(2), rtol=1e-6)
    np.testing.assert_allclose(L[24:], 0.01 * math.sqrt(3), rtol=1e-6)
    two = np.ones((1, 1, 2), np.uint8)
    s2 = ora.voxel_system(two, np.zeros((1, 1, 2)), mats, 2.0, 0.01, 0.03)
    assert s2["x"].shape[0] == 12 and s2["ij"].shape[0] == 56
    assert abs(s2["m"].sum() - 0.06) < 1e-15
    assert s2["x"][:, 2].min() == 0.0


def test_best_candidate_points_are_spread():
    """Best-candidate sampling keeps points apart: its smallest nearest-neighbour
    distance is several times that of uniform random points of the same count."""
    n = 400
    p = synth.best_candidate_points(n, seed=3)
    r = np.random.default_rng(3).random((n, 3))
    def min_nn(a):
        d = np.sqrt(((a[:, None] - a[None]) ** 2).sum(-1)); np.fill_diagonal(d, np.inf)
        return d.min()
    assert min_nn(p) > 3 * min_nn(r)


def test_quasi_uniform_lattice_shape():
    s = synth.quasi_uniform_lattice(600, seed=2)
    deg = np.bincount(s["ij"].ravel(), minlength=600)
    assert deg.max() <= 26 and deg.min() >= 1
    assert np.all(s["ij"][:, 0] < s["ij"][:, 1])


def test_batched_largest_components_equal_the_per_design_rule():
    """synth.largest_components (one labelling over a batch of designs) keeps
    exactly the component that the single-design rule keeps, ties and empty
    designs included."""
    rng = np.random.default_rng(12)
    mats = rng.integers(0, 4, size=(400, 5, 6, 7)).astype(np.uint8)
    mats[3] = 0
    mats[7] = 0; mats[7, 0, 0, 0] = 2; mats[7, 4, 5, 6] = 1      # a tie: two single voxels
    got = synth.largest_components(mats, chunk=64)
    for m, g in zip(mats, got):
        want = np.where(synth._largest_component(m > 0), m, 0)
        assert np.array_equal(g, want)
    assert got[7, 0, 0, 0] == 2 and got[7, 4, 5, 6] == 0
