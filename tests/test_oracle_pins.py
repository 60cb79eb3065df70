"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an invariant,
a textbook special case, a finite difference of a separately computed energy, or a
brute-force property.  Rotations used to *build* test frames come from scipy.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation as R

import oracle
from paper_2509_04277_gb300 import workloads as W


def _rod(n=12, length=0.3, **kw):
    base = dict(radius=1e-3, E_bend=100e9, E_stretch=100e9, G=40e9, density=6500.0, dt=1e-5,
                n_iters=10, inextensible=True, clamp=1, damping_alpha=0.0)
    base.update(kw)
    orientation = base.pop("orientation", None)
    return W.straight_rod(n, length, orientation=orientation, **base)


def _continuous(q):
    q = np.array(q, dtype=np.float64)
    for j in range(1, len(q)):
        if np.dot(q[j - 1], q[j]) < 0:
            q[j] = -q[j]
    return q


def _frames_constant_increment(m, theta, axis, q0=None):
    """Frames q_j = q0 * Rot(j theta axis) (body-frame increments), via scipy."""
    q0 = R.identity() if q0 is None else q0
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return _continuous([(q0 * R.from_rotvec(j * theta * axis)).as_quat() for j in range(m)])


def _centreline_from_frames(quat, l0, start=(0.0, 0.0, 0.0)):
    """Positions with every segment along its frame's third director (penalty-free)."""
    d3 = R.from_quat(quat).apply([0.0, 0.0, 1.0])
    pos = np.zeros((len(quat) + 1, 3))
    pos[0] = start
    pos[1:] = np.asarray(start)[None, :] + np.cumsum(l0 * d3, axis=0)
    return pos


def _elastic(rod, pos, quat):
    e = oracle.energy(rod, {"pos": pos, "quat": quat})
    return e["bend"] + e["penalty"] + e["stretch"]


# ------------------------------------------------------------------ Darboux vector (Eq. 5-6)


@pytest.mark.parametrize("theta", [1e-3, 0.05, 0.7])
def test_darboux_constant_increment_closed_form(theta):
    """Frames related by a constant body-frame rotation theta about a: the discrete
    Darboux vector is exactly (2/l) sin(theta/2) a, for any axis and base frame."""
    rod = _rod(10)
    l0 = rod.length / (rod.n_nodes - 1)
    g = np.random.default_rng(3)
    for _ in range(3):
        axis = g.standard_normal(3)
        axis /= np.linalg.norm(axis)
        q = _frames_constant_increment(rod.n_nodes - 1, theta, axis, R.random(random_state=g))
        u = oracle.darboux(rod, q)
        expect = (2.0 / l0) * math.sin(theta / 2) * axis
        np.testing.assert_allclose(u, np.tile(expect, (len(u), 1)), rtol=1e-12, atol=1e-12)


def test_darboux_circular_arc_curvature():
    """A circular arc of radius rho: the bending component tends to 1/rho with O(theta^2)
    relative error, theta = l/rho (Eq. 1 in the continuum limit)."""
    rho = 0.25
    for n in (33, 129):
        rod = _rod(n, length=0.5)
        l0 = rod.length / (n - 1)
        th = l0 / rho
        q = _frames_constant_increment(n - 1, th, [1.0, 0.0, 0.0])
        u = oracle.darboux(rod, q)
        rel = abs(u[:, 0].mean() * rho - 1.0)
        assert rel < th * th / 20, (n, rel)
        assert np.abs(u[:, 1:]).max() < 1e-12


# ------------------------------------------------------------------ energies and forces


def test_bending_and_twist_energy_textbook():
    """Uniform curvature kappa and twist tau: V_b -> 1/2 (E I kappa^2 + G J tau^2) L_joint,
    with I = pi r^4 / 4 and J = pi r^4 / 2 (the second-moment reading of Eq. 3)."""
    n = 257
    rod = _rod(n, length=1.0, radius=2e-3, E_bend=70e9, G=26e9)
    l0 = rod.length / (n - 1)
    kappa, tw = 0.5, 0.8
    w = np.array([kappa, 0.0, tw])
    theta = np.linalg.norm(w) * l0
    q = _frames_constant_increment(n - 1, theta, w)
    pos = _centreline_from_frames(q, l0)
    e = oracle.energy(rod, {"pos": pos, "quat": q})
    r = rod.radius
    I = math.pi * r**4 / 4
    Jp = math.pi * r**4 / 2
    expect = 0.5 * (rod.E_bend * I * kappa**2 + rod.G * Jp * tw**2) * (n - 2) * l0
    assert abs(e["bend"] / expect - 1) < 1e-4
    assert e["penalty"] < 1e-20


def test_rest_state_has_zero_force_and_torque():
    """The rest shape carries no force or torque, straight or curved (helical) rest."""
    n = 24
    for curved in (False, True):
        rod = _rod(n, length=0.4, orientation=R.random(random_state=np.random.default_rng(5)))
        l0 = rod.length / (n - 1)
        if curved:
            q0 = R.random(random_state=np.random.default_rng(6))
            rod.rest_quat = _frames_constant_increment(n - 1, 0.2, [0.3, -0.4, 0.8], q0)
        q = rod.rest_quat
        pos = _centreline_from_frames(q, l0, start=(0.1, -0.2, 0.3))
        F, tau, _ = oracle.forces(rod, pos, q)
        scaleF = rod.E_bend * math.pi * rod.radius**4 / 4 / l0**2
        assert np.abs(F).max() < 1e-9 * scaleF
        assert np.abs(tau).max() < 1e-9 * scaleF * l0


@pytest.mark.parametrize("extensible", [False, True])
def test_forces_are_minus_energy_gradient(extensible):
    """F_i = -dV/dr_i, checked against central differences of the energy."""
    rod = _rod(9, length=0.2, inextensible=not extensible, pos_sigma=2e-3, ang_sigma=0.1, seed=11)
    rod.rest_quat = _frames_constant_increment(8, 0.1, [1.0, 0.5, 0.2], R.from_rotvec([0, math.pi / 2, 0]))
    pos, quat = rod.pos.copy(), rod.quat.copy()
    F, _, g = oracle.forces(rod, pos, quat)
    h = 1e-7
    Ffd = np.zeros_like(F)
    for i in range(pos.shape[0]):
        for k in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, k] += h
            p2[i, k] -= h
            Ffd[i, k] = -(_elastic(rod, p1, quat) - _elastic(rod, p2, quat)) / (2 * h)
    np.testing.assert_allclose(F, Ffd, rtol=1e-6, atol=1e-6 * np.abs(F).max())
    # quaternion 4-gradient (components treated as independent coordinates)
    gfd = np.zeros_like(g)
    for j in range(quat.shape[0]):
        for k in range(4):
            q1, q2 = quat.copy(), quat.copy()
            q1[j, k] += h
            q2[j, k] -= h
            gfd[j, k] = (_elastic(rod, pos, q1) - _elastic(rod, pos, q2)) / (2 * h)
    np.testing.assert_allclose(g, gfd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_torque_is_minus_energy_derivative_under_body_rotation():
    """tau_k = -d/d eps V(q_j * Rot(eps e_k)) (body-frame rotation of one frame)."""
    rod = _rod(9, length=0.2, pos_sigma=2e-3, ang_sigma=0.1, seed=12)
    pos, quat = rod.pos.copy(), rod.quat.copy()
    _, tau, _ = oracle.forces(rod, pos, quat)
    h = 1e-6
    tfd = np.zeros_like(tau)
    for j in range(quat.shape[0]):
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            q1, q2 = quat.copy(), quat.copy()
            a = (R.from_quat(quat[j]) * R.from_rotvec(e)).as_quat()
            b = (R.from_quat(quat[j]) * R.from_rotvec(-e)).as_quat()
            q1[j] = a if np.dot(a, quat[j]) > 0 else -a
            q2[j] = b if np.dot(b, quat[j]) > 0 else -b
            tfd[j, k] = -(_elastic(rod, pos, q1) - _elastic(rod, pos, q2)) / (2 * h)
    np.testing.assert_allclose(tau, tfd, rtol=1e-5, atol=1e-6 * np.abs(tau).max())


def test_translation_and_rotation_invariance():
    """Internal forces: sum F = 0 and total world torque sum r x F + sum R tau = 0."""
    rod = _rod(15, length=0.3, pos_sigma=3e-3, ang_sigma=0.2, seed=13, inextensible=False)
    rod.rest_quat = _frames_constant_increment(14, 0.15, [0.2, 1.0, -0.3], R.from_rotvec([0.1, 0.2, 0.3]))
    F, tau, _ = oracle.forces(rod, rod.pos, rod.quat)
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * scale
    world_tau = R.from_quat(rod.quat).apply(tau)
    total = np.cross(rod.pos, F).sum(axis=0) + world_tau.sum(axis=0)
    assert np.abs(total).max() < 1e-10 * scale * rod.length


# ------------------------------------------------------------------ dynamics


def test_quaternions_stay_unit():
    rod = W.guidewire(64, seed=21)
    s = oracle.step(rod, oracle.state_of(rod), 200, drive=np.array([0.01, 0, 0, 0, 0, 0, 2.0, 0]))
    assert np.abs(np.linalg.norm(s["quat"], axis=1) - 1).max() < 1e-12


def test_driven_base_follows_input_exactly():
    """Node 0 and frame 0 are kinematic: r_0(t) = r_0 + t dt v, q_0 follows omega."""
    rod = W.guidewire(32, seed=22)
    v = np.array([0.02, -0.01, 0.005])
    w = np.array([0.0, 0.0, 3.0])
    drive = np.concatenate([v, [0], w, [0]])
    n = 50
    s = oracle.step(rod, oracle.state_of(rod), n, drive=drive)
    np.testing.assert_allclose(s["pos"][0], rod.pos[0] + n * rod.dt * v, rtol=0, atol=1e-14)
    # rotation about the body z axis by n * dt * |w| (to first order in dt per step)
    ang = 2 * math.atan2(*(R.from_quat(rod.quat[0]).inv() * R.from_quat(s["quat"][0])).as_quat()[[2, 3]])
    assert abs(ang - n * rod.dt * w[2]) < 1e-6


def test_gravity_accelerates_free_rod_at_g_over_mass_scale():
    """A free rod in its rest shape under gravity: every node accelerates at g / mass_scale
    (gravity uses the physical mass, the dynamics the scaled inertial mass)."""
    rod = _rod(10, length=0.2, clamp=0, gravity=(0.0, 0.0, -9.81), mass_scale=7.0, inertia_scale=3.0)
    n = 20
    s = oracle.step(rod, oracle.state_of(rod), n)
    a = -9.81 / 7.0
    np.testing.assert_allclose(s["vel"][:, 2], n * rod.dt * a, rtol=1e-9)
    np.testing.assert_allclose(s["pos"][:, 2] - rod.pos[:, 2], a * rod.dt**2 * n * (n + 1) / 2, rtol=1e-9)


def test_rayleigh_damping_decay():
    """Rigid translation of a free rod decays as (1 + alpha dt)^-n (implicit damping)."""
    rod = _rod(8, length=0.1, clamp=0, damping_alpha=50.0)
    st = oracle.state_of(rod)
    st["vel"][:] = [0.1, 0.2, -0.3]
    n = 40
    s = oracle.step(rod, st, n)
    expect = np.array([[0.1, 0.2, -0.3]]) * (1 + 50.0 * rod.dt) ** -n
    np.testing.assert_allclose(s["vel"], np.broadcast_to(expect, s["vel"].shape), rtol=1e-9)


# ------------------------------------------------------------------ frames as rigid bodies
#
# Force integration treats each frame as a rigid body (end of Section 2.1, Fig. 5): the
# body-frame angular velocity follows Euler's equations J dw/dt = tau - w x (J w), the
# orientation follows dq/dt = 1/2 q (x) (0, w).  A single free frame (2 nodes, no joint,
# a negligible penalty constant, a soft axial spring, no gravity) is torque-free, so its motion is the
# textbook symmetric top: with J = diag(J1, J1, J3), w3 is constant and (w1, w2) turns
# at Omega = (J3 - J1) / J1 * w3 in the positive sense about the body z axis, and the
# world-frame angular momentum R(q) J w is constant.


def _free_frame(dt, alpha=0.0):
    return W.straight_rod(2, 0.01, radius=1e-3, E_bend=1e9, E_stretch=1.0, G=0.4e9, density=6500.0, dt=dt,
                          n_iters=0, inextensible=False, clamp=0, damping_alpha=alpha, Kp=1e-300,
                          mass_scale=1.0, inertia_scale=1.0)


def _spin(rod, w0, n):
    st = oracle.state_of(rod)
    st["omega"][0] = w0
    return st, oracle.step(rod, st, n)


def test_free_frame_precesses_as_a_symmetric_top():
    """Torque-free symmetric top, t = 0.5 s: w3 is constant, the transverse part turns
    by +Omega t about body z (a sign error or a dropped w x Jw turns it by -Omega t or
    not at all), its length and the world angular momentum are kept to first order in dt
    (the error halves with dt), and the nodes do not move."""
    d = oracle.derive(_free_frame(1e-4))
    J = np.array([d["J1"], d["J2"], d["J3"]])
    assert J[0] == J[1] and J[2] == pytest.approx(2 * J[0], rel=1e-14)  # rho l0 diag(I, I, 2I)
    w0 = np.array([3.0, 0.0, 10.0])
    Om = (J[2] - J[0]) / J[0] * w0[2]
    T = 0.5
    errs = []
    for dt in (1e-4, 5e-5):
        rod = _free_frame(dt)
        n = int(round(T / dt))
        st, s = _spin(rod, w0, n)
        w = s["omega"][0]
        assert w[2] == pytest.approx(w0[2], rel=1e-13)
        phase = math.atan2(w[1], w[0])
        dphase = (phase - Om * T + math.pi) % (2 * math.pi) - math.pi
        assert abs(dphase) < 1e-5, (dt, phase, Om * T)
        mag_err = abs(math.hypot(w[0], w[1]) / 3.0 - 1.0)
        L0 = R.from_quat(st["quat"][0]).apply(J * w0)
        L1 = R.from_quat(s["quat"][0]).apply(J * w)
        L_err = np.linalg.norm(L1 - L0) / np.linalg.norm(L0)
        assert mag_err < 0.5 * Om**2 * dt * T * 1.01  # explicit Euler: (1 + Om^2 dt^2)^(n/2)
        assert L_err < 1e-3
        np.testing.assert_allclose(s["pos"], st["pos"], rtol=0, atol=1e-200)  # penalty constant 1e-300
        errs.append((mag_err, L_err))
    for k in range(2):
        assert 1.8 < errs[0][k] / errs[1][k] < 2.2, errs


def test_free_frame_spin_about_body_axis():
    """Spin about the body z axis (a principal axis, no gyroscopic term): w stays put
    and the frame turns about its own third director (body frame, q (x) w, not w (x) q)
    by w t, to second order in dt per step."""
    rod = _free_frame(1e-4)
    w0 = np.array([0.0, 0.0, 7.0])
    n = 300
    st, s = _spin(rod, w0, n)
    np.testing.assert_allclose(s["omega"][0], w0, rtol=1e-15, atol=1e-200)
    rel = R.from_quat(st["quat"][0]).inv() * R.from_quat(s["quat"][0])
    rv = rel.as_rotvec()
    np.testing.assert_allclose(rv[:2], 0.0, atol=1e-12)
    assert abs(rv[2] - n * rod.dt * w0[2]) < 1e-6
    # the third director turned about the world image of body z, i.e. it stays put,
    # while the first director turned by w t in the plane normal to it
    d3_0 = R.from_quat(st["quat"][0]).apply([0, 0, 1])
    d3_1 = R.from_quat(s["quat"][0]).apply([0, 0, 1])
    np.testing.assert_allclose(d3_1, d3_0, atol=1e-12)


def test_free_frame_angular_damping():
    """Implicit Rayleigh damping of the angular velocity: w3 decays exactly as
    (1 + alpha dt)^-n, and the transverse part, turned as in the undamped top, decays at
    the same rate up to the first-order growth of explicit Euler."""
    alpha, dt, n = 40.0, 1e-4, 2000
    rod = _free_frame(dt, alpha=alpha)
    w0 = np.array([2.0, -1.0, 10.0])
    st, s = _spin(rod, w0, n)
    w = s["omega"][0]
    decay = (1 + alpha * dt) ** -n
    assert w[2] == pytest.approx(w0[2] * decay, rel=1e-12)
    ratio = math.hypot(w[0], w[1]) / math.hypot(w0[0], w0[1]) / decay
    assert abs(ratio - 1.0) < 0.5 * 100.0 * dt * n * dt * 1.01  # Omega <= 10: (Omega dt)^2 n / 2
    # no damping of a pure spin's direction: w stays along body z
    st2, s2 = _spin(rod, np.array([0.0, 0.0, 5.0]), n)
    np.testing.assert_allclose(s2["omega"][0], [0.0, 0.0, 5.0 * decay], rtol=1e-12, atol=1e-200)


def test_two_node_constraint_projection_exact():
    """One distance constraint (N = 2): after the step |r_1 - r_0| = l0 exactly, the
    impulse is along the constraint direction and momentum is conserved."""
    rod = _rod(2, length=0.01, clamp=0, n_iters=1, mass_scale=2.0, inertia_scale=1.0)
    st = oracle.state_of(rod)
    st["vel"] = np.array([[0.3, -0.2, 0.1], [-0.5, 0.4, 0.2]])
    s = oracle.step(rod, st, 1)
    d = oracle.derive(rod)
    assert abs(np.linalg.norm(s["pos"][1] - s["pos"][0]) - d["l0"]) < 1e-16
    m = 1.0 / d["w_interior"] / 2  # end nodes carry half mass
    # momentum: elastic forces are internal (sum zero) and impulses are equal and opposite
    np.testing.assert_allclose((s["vel"] * m).sum(axis=0), (st["vel"] * m).sum(axis=0), atol=1e-14)


def test_constraint_error_decreases_with_iterations():
    """Gauss-Seidel sweeps on a state that violates the constraints by ~1 % (node
    jitter): the max relative length error after a step does not grow with the
    iteration count and falls by an order of magnitude."""
    rod = W.guidewire(128, seed=23)
    st = oracle.state_of(rod)
    st["vel"] = np.random.default_rng(1).standard_normal(st["vel"].shape) * 0.05
    st["vel"][0] = 0
    errs = []
    for it in (1, 2, 4, 10, 40):
        rod.n_iters = it
        s = oracle.step(rod, st, 1)
        seg = np.linalg.norm(np.diff(s["pos"], axis=0), axis=1)
        errs.append(np.abs(seg / (rod.length / 127) - 1).max())
    assert all(b <= a * 1.0000001 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] / 10


def test_guidewire_inextensibility_over_rollout():
    rod = W.guidewire(512, seed=2)
    drive = W.sinusoid_drive(2, 30, 10 * rod.dt)
    s = oracle.state_of(rod)
    worst = 0.0
    for k in range(30):
        s = oracle.step(rod, s, 10, drive=drive[k])
        seg = np.linalg.norm(np.diff(s["pos"], axis=0), axis=1)
        worst = max(worst, np.abs(seg / (rod.length / 511) - 1).max())
    assert worst < 1e-3


def test_literal_masses_blow_up_and_default_scaling_is_stable():
    """The extensible 64-element rod with physical masses is beyond explicit stability
    at dt = 1e-5 s (the default inertial scaling exists for this reason)."""
    lit = W.extensible_pendulum(literal_masses=True)
    with np.errstate(all="ignore"):
        s = oracle.step(lit, oracle.state_of(lit), 1000)
    assert not np.isfinite(s["pos"]).all() or np.abs(s["pos"]).max() > 10.0
    rod = W.extensible_pendulum()
    s = oracle.step(rod, oracle.state_of(rod), 1000)
    assert np.isfinite(s["pos"]).all()
    seg = np.linalg.norm(np.diff(s["pos"], axis=0), axis=1)
    assert np.abs(seg / (1.0 / 63) - 1).max() < 0.05


def test_energy_bounded_without_damping():
    """alpha = 0, extensible rod, omega dt ~ 0.01: the total energy oscillates by
    less than 1 % over 10^4 steps with no secular trend (symplectic Euler)."""
    rod = W.straight_rod(16, 0.5, pos_sigma=2e-4, ang_sigma=2e-3, seed=7, radius=1e-3, E_bend=50e9,
                         E_stretch=50e9, G=20e9, density=6500.0, dt=1e-5, n_iters=0, inextensible=False,
                         clamp=1, damping_alpha=0.0)
    d = oracle.derive(rod)
    rod.mass_scale, rod.inertia_scale, rod.dt = d["mass_scale"], d["inertia_scale"], 1e-5 / 50
    s = oracle.state_of(rod)
    E0 = oracle.energy(rod, s)["total"]
    Es = []
    for _ in range(100):
        s = oracle.step(rod, s, 100)
        Es.append(oracle.energy(rod, s)["total"])
    Es = np.array(Es) / E0
    assert Es.max() - Es.min() < 0.01
    slope = np.polyfit(np.arange(len(Es)), Es, 1)[0] * len(Es)
    assert abs(slope) < 2e-3


def _cantilever(n, steps=40000):
    rod = W.straight_rod(n, 0.2, radius=1e-3, E_bend=250e9, E_stretch=250e9, G=250e9 / 2.6, density=6500.0,
                         dt=1e-5, n_iters=10, inextensible=True, clamp=1, damping_alpha=150.0,
                         gravity=(0.0, 0.0, -9.81))
    s = oracle.step(rod, oracle.state_of(rod), steps)
    d = oracle.derive(rod)
    w = rod.density * d["A"] * 9.81
    theory = w * rod.length**4 / (8 * d["K1"]) + w * rod.length**2 / (2 * d["Kp"])
    return -s["pos"][-1, 2], theory, np.abs(s["vel"]).max()


def test_cantilever_tip_deflection_timoshenko():
    """Clamped rod under its own weight at damped equilibrium: tip deflection
    w L^4 / (8 E I) + w L^2 / (2 Kp) (Euler-Bernoulli plus the penalty as shear
    stiffness).  The discrete clamp (frame 0 fixed over the first segment) gives a
    first-order offset -2/(N-1); Richardson extrapolation over N = 33, 65 removes it."""
    d33, theory, v33 = _cantilever(33)
    d65, _, v65 = _cantilever(65)
    assert max(v33, v65) < 1e-8
    for n, dn in ((33, d33), (65, d65)):
        rel = dn / theory - 1
        assert abs(rel + 2.0 / (n - 1)) < 0.25 * 2.0 / (n - 1), (n, rel)
    extrap = 2 * d65 - d33
    assert abs(extrap / theory - 1) < 5e-3


def test_static_twist_profile_linear():
    """Frame 0 clamped, end torque T about the axis: every joint carries T, so
    (K3 / l) sin(dtheta) = T and the twist angle is linear, theta_j = j asin(T l / K3)."""
    n = 17
    rod = _rod(n, length=0.2, orientation=R.identity(), E_bend=200e9, G=80e9, damping_alpha=300.0)
    d = oracle.derive(rod)
    T = 0.3 * d["K3"] / d["l0"]
    tau = np.zeros((n - 1, 3))
    tau[-1, 2] = T
    s = oracle.step(rod, oracle.state_of(rod), 60000, tau_ext=tau)
    q = s["quat"]
    theta = 2 * np.arctan2(q[:, 2], q[:, 3])
    np.testing.assert_allclose(theta, np.arange(n - 1) * math.asin(0.3), atol=1e-9)
    assert abs(math.asin(0.3) - 0.3) > 1e-3  # the check separates asin from the linear law


# ------------------------------------------------------------------ forward-mode derivative


def test_jvp_matches_central_differences():
    rod = W.adjoint_rod(12, seed=31)
    st = oracle.state_of(rod)
    K, uhat = oracle.material(rod)
    steps = 30
    g = np.random.default_rng(2)
    d_pos = g.standard_normal(st["pos"].shape) * 1e-3
    d_pos[0] = 0
    d_vel = g.standard_normal(st["vel"].shape) * 1e-2
    d_K = g.standard_normal(K.shape) * K * 0.1
    d_uhat = g.standard_normal(uhat.shape) * 0.5
    d_quat = g.standard_normal(st["quat"].shape) * 1e-2  # raw components (also off the unit sphere)
    d_omega = g.standard_normal(st["omega"].shape) * 1.0
    st["omega"] = g.standard_normal(st["omega"].shape) * 2.0  # spinning frames: the gyroscopic term is active
    h = 1e-6

    def run(sg, which):
        s2 = {k: v.copy() for k, v in st.items()}
        on = lambda k: sg * h if k in which else 0.0  # noqa: E731
        s2["pos"] = st["pos"] + on("pos") * d_pos
        s2["vel"] = st["vel"] + on("vel") * d_vel
        s2["quat"] = st["quat"] + on("quat") * d_quat
        s2["omega"] = st["omega"] + on("omega") * d_omega
        traj, _ = oracle.rollout(rod, s2, steps, K=K + on("K") * d_K, uhat=uhat + on("uhat") * d_uhat)
        return traj

    zero = {k: None for k in ("d_pos", "d_vel", "d_K", "d_uhat", "d_quat", "d_omega")}
    full = dict(d_pos=d_pos, d_vel=d_vel, d_K=d_K, d_uhat=d_uhat, d_quat=d_quat, d_omega=d_omega)
    for which in (("pos", "vel", "K", "uhat"), ("quat",), ("omega",), ("pos", "vel", "K", "uhat", "quat", "omega")):
        kw = dict(zero)
        kw.update({"d_" + k: full["d_" + k] for k in which})
        _, dtraj = oracle.rollout_jvp(rod, st, steps, K=K, uhat=uhat, **kw)
        fd = (run(1, which) - run(-1, which)) / (2 * h)
        assert np.abs(fd).max() > 0, which
        np.testing.assert_allclose(dtraj, fd, rtol=1e-4, atol=5e-6 * np.abs(fd).max(), err_msg=str(which))


def test_flop_count_linear_in_elements():
    a = oracle.count_flops(W.guidewire(64), 2)
    b = oracle.count_flops(W.guidewire(128), 2)
    assert 1.9 < b / a < 2.05


# ------------------------------------------------------------------ binding (catheter/guidewire)


def test_binding_one_way_puts_inner_nodes_on_outer_centreline():
    """v1 with a static outer rod: after one step every bound inner node sits exactly on
    the outer rod's centreline point it is bound to (the last binding color leaves the
    other color's constraints satisfied because the outer rod does not move)."""
    cat, gw = W.catheter_guidewire(32, seed=82, beta0=-5.4)
    so, si = oracle.state_of(cat), oracle.state_of(gw)
    si["pos"][:, 1] += 1e-3  # lateral offset of the inner rod
    beta = -5.4
    so2, si2 = oracle.step_pair(cat, so, gw, si, 1, beta, 1)
    k0 = int(np.floor(beta))
    a = beta - k0
    worst = 0.0
    for i in range(32):
        k = i + k0
        if 0 <= k <= 30:
            p = (1 - a) * so2["pos"][k] + a * so2["pos"][k + 1]
            worst = max(worst, np.abs(si2["pos"][i] - p).max())
    assert worst < 1e-12


def test_binding_two_way_conserves_momentum():
    """v2 on free rods without gravity: binding impulses are equal and opposite, so the
    pair's total (inertial) momentum is unchanged by a step."""
    cat, gw = W.catheter_guidewire(24, seed=83, beta0=-3.3)
    for r in (cat, gw):
        r.clamp = 0
    so, si = oracle.state_of(cat), oracle.state_of(gw)
    g = np.random.default_rng(4)
    so["vel"] = g.standard_normal(so["vel"].shape) * 0.01
    si["vel"] = g.standard_normal(si["vel"].shape) * 0.01
    si["pos"][:, 2] += 5e-4

    def momentum(rod, s):
        d = oracle.derive(rod)
        m = np.full(rod.n_nodes, d["mass_scale"] * d["m_interior"])
        m[0] *= 0.5
        m[-1] *= 0.5
        return (m[:, None] * s["vel"]).sum(axis=0)

    p0 = momentum(cat, so) + momentum(gw, si)
    so2, si2 = oracle.step_pair(cat, so, gw, si, 2, -3.3, 1)
    p1 = momentum(cat, so2) + momentum(gw, si2)
    scale = np.abs(momentum(gw, si2) - momentum(gw, si)).max()
    assert scale > 1e-6  # binding did act
    np.testing.assert_allclose(p1, p0, atol=1e-12 * max(1.0, scale) + 1e-15)


def test_binding_mode_zero_is_two_independent_rods():
    cat, gw = W.catheter_guidewire(20, seed=84, beta0=-2.5)
    so, si = oracle.state_of(cat), oracle.state_of(gw)
    dc = np.array([0.01, 0, 0, 0, 0, 0, 1.0, 0])
    dg = np.array([0.02, 0, 0, -2.5, 0, 0, -1.0, 0])
    so2, si2 = oracle.step_pair(cat, so, gw, si, 0, -2.5, 5, drive_outer=dc, drive_inner=dg)
    np.testing.assert_array_equal(so2["pos"], oracle.step(cat, so, 5, drive=dc)["pos"])
    np.testing.assert_array_equal(si2["pos"], oracle.step(gw, si, 5, drive=dg)["pos"])


# ------------------------------------------------------------------ vessel contact


def _straight_tube_rod(mu, v, n=8):
    """A short straight rod along +x inside a nearly straight tube (centreline radius 1 km
    through the origin, tangent to +x), translating rigidly with velocity v."""
    rod = _rod(n, length=0.05, clamp=0, n_iters=1, mass_scale=1.0, inertia_scale=1.0)
    rod.quat = rod.rest_quat.copy()
    rod.pos = np.zeros((n, 3))
    rod.pos[:, 0] = np.linspace(0, 0.05, n)
    st = oracle.state_of(rod)
    st["vel"][:] = v
    tube = np.array([0.0, 1000.0, 0.0, 1000.0, 2e-3, mu])
    return rod, st, tube


def test_vessel_contact_inactive_inside():
    """Nodes well inside the vessel: the step is the step without a vessel."""
    rod, st, tube = _straight_tube_rod(0.3, [0.01, 0.0, 0.0])
    a = oracle.step_tube(rod, st, tube, 3)
    b = oracle.step(rod, st, 3)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_vessel_contact_puts_penetrating_nodes_on_the_wall():
    """A rigid rod moving into the wall (+z) fast enough to cross it in one step: after
    the step every node lies exactly at the allowed distance (inner radius minus rod
    radius) from the centreline; the normal velocity is what lands it there."""
    vz = 200.0  # crosses the 1 mm clearance in one 1e-5 s step
    rod, st, tube = _straight_tube_rod(0.0, [0.0, 0.0, vz])
    s = oracle.step_tube(rod, st, tube, 1)
    allow = tube[4] - rod.radius
    # distance to the (locally straight) centreline: |(y - y_c, z)| with y_c ~ x^2 / (2 Rc)
    yc = 1000.0 - np.sqrt(1000.0**2 - s["pos"][:, 0] ** 2)
    dist = np.sqrt((s["pos"][:, 1] - yc) ** 2 + s["pos"][:, 2] ** 2)
    np.testing.assert_allclose(dist, allow, rtol=1e-9)


def _wall_normal(pos, tube):
    """Outward wall normal at each node: from the nearest centreline point to the node."""
    dx, dy = pos[:, 0] - tube[0], pos[:, 1] - tube[1]
    rho = np.hypot(dx, dy)
    c = np.stack([tube[0] + tube[3] * dx / rho, tube[1] + tube[3] * dy / rho, np.full(len(pos), tube[2])], 1)
    d = pos - c
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_vessel_contact_coulomb_friction():
    """Coulomb's law at the wall, per node, with n the wall normal at the node's predicted
    position r + dt v (where the constraint is evaluated): the velocity change splits into a normal part dvn and a tangential part dvt
    with |dvt| = mu |dvn| opposing the tangential velocity while sliding; mu = 0 leaves
    the tangential velocity alone; a large mu stops it (sticking)."""
    v0 = np.array([0.2, 0.0, 200.0])
    for mu in (0.0, 1e-3, 10.0):
        rod, st, tube = _straight_tube_rod(mu, v0)
        s = oracle.step_tube(rod, st, tube, 1)
        n = _wall_normal(st["pos"] + rod.dt * v0, tube)
        dv = s["vel"] - v0
        dvn = np.sum(dv * n, axis=1)
        dvt = dv - dvn[:, None] * n
        vt0 = v0 - np.sum(v0 * n, axis=1)[:, None] * n
        assert np.all(dvn < -90.0)  # pushed back by ~ (200 dt - 1 mm) / dt = 100 m/s
        if mu == 0.0:
            assert np.all(np.linalg.norm(dvt, axis=1) < 1e-9 * np.abs(dvn))
        elif mu == 1e-3:
            np.testing.assert_allclose(np.linalg.norm(dvt, axis=1), mu * np.abs(dvn), rtol=1e-6)
            cos = np.sum(dvt * vt0, axis=1) / (np.linalg.norm(dvt, axis=1) * np.linalg.norm(vt0, axis=1))
            np.testing.assert_allclose(cos, -1.0, atol=1e-9)
        else:
            vt1 = s["vel"] - np.sum(s["vel"] * n, axis=1)[:, None] * n
            assert np.all(np.linalg.norm(vt1, axis=1) < 1e-6 * np.linalg.norm(vt0, axis=1))


# ------------------------------------------------------------------ self-collision

RS = 0.45e-3  # rod radius of the self-contact pins


def _free_rod(n, spacing=1.35):
    """Unclamped rod parameters with l0 = spacing r (min index gap 2 for spacing > 1)."""
    return _rod(n, length=(n - 1) * spacing * RS, radius=RS, clamp=0, n_iters=1)


def _far_line(n):
    pos = np.zeros((n, 3))
    pos[:, 0] = np.arange(n) * 10 * RS
    return pos


def test_self_candidates_match_kdtree():
    """Detection against an independent neighbour search (scipy's k-d tree): every pair
    at least min_sep apart in index and closer than 3 r, listed ascending per node."""
    from scipy.spatial import cKDTree

    for rod in (W.torus_knot(64), W.torus_knot(512), W.coil(130)):
        pos = rod.pos
        cand, pairs = oracle.self_candidates(rod, pos)
        l0 = rod.length / (rod.n_nodes - 1)
        m = max(2, int(np.floor(2 * rod.radius / l0)) + 1)
        ref = {(i, j) for i, j in cKDTree(pos).query_pairs(3 * rod.radius) if j - i >= m}
        got = {(i, int(j)) for i in range(len(cand)) for j in cand[i] if j > i}
        assert got == ref and pairs == len(ref) and len(ref) > 100
        assert all(np.all(np.diff(c) > 0) for c in cand)


def test_coil_overflows_a_skin_list_but_not_the_candidate_list():
    """The coil input of the GPU overflow test keeps its purpose: within the skin list's
    grown reach (3 r + 2 x 1.5 r) some mass point has more than the list's 24 places of
    partners above it, within the plain 3 r none has more than the 16 candidate places,
    and some neighbouring turns overlap (so the contact response runs)."""
    from scipy.spatial import cKDTree

    rod = W.coil(130)
    pos = rod.pos
    l0 = rod.length / (rod.n_nodes - 1)
    m = max(2, int(np.floor(2 * rod.radius / l0)) + 1)

    def most_above(reach):
        count = np.zeros(rod.n_nodes, int)
        for i, j in cKDTree(pos).query_pairs(reach):
            if abs(j - i) >= m:
                count[min(i, j)] += 1
        return count.max()

    assert most_above(6 * rod.radius) > 24
    assert most_above(3 * rod.radius) <= 16
    assert any(abs(j - i) >= m for i, j in cKDTree(pos).query_pairs(2 * rod.radius))


def test_self_contact_single_pair_lands_on_contact_distance():
    """One overlapping pair (nodes 1 and 5): only they change; their predicted distance
    becomes exactly 2 r and their momentum is conserved (equal masses)."""
    rod = _free_rod(8)
    pos = _far_line(8)
    pos[5] = pos[1] + [0.0, 1.8 * RS, 0.3 * RS]
    vel = np.random.default_rng(3).normal(size=(8, 3)) * 0.01
    v2 = oracle.self_contact_pass(rod, pos, vel, 0.0)
    assert set(np.flatnonzero(np.any(v2 != vel, axis=1))) == {1, 5}
    delta = (pos[5] - pos[1]) + rod.dt * (v2[5] - v2[1])
    assert np.linalg.norm(delta) == pytest.approx(2 * RS, rel=1e-12)
    np.testing.assert_allclose(v2[1] + v2[5], vel[1] + vel[5], rtol=0, atol=1e-15)


def test_self_contact_coulomb_friction():
    """Relative tangential velocity of one colliding pair, with n the pair's normal at the
    predicted positions: mu = 0 leaves it; a small mu cuts it by exactly mu du_n (sliding)
    against its direction; a large mu stops it (sticking)."""
    rod = _free_rod(8)
    pos = _far_line(8)
    pos[5] = pos[1] + [0.0, 2.2 * RS, 0.0]
    vel = np.zeros((8, 3))
    vel[5] = [0.05, -10.0, 0.0]  # closes the 0.2 r gap and 0.2 r more in one step
    u0 = vel[5] - vel[1]
    d0 = (pos[5] - pos[1]) + rod.dt * u0
    n = d0 / np.linalg.norm(d0)
    ut0 = u0 - (u0 @ n) * n
    for mu in (0.0, 1e-3, 10.0):
        v2 = oracle.self_contact_pass(rod, pos, vel, mu)
        du = (v2[5] - v2[1]) - u0
        dun = du @ n
        dut = du - dun * n
        assert dun > 0
        if mu == 0.0:
            assert np.linalg.norm(dut) < 1e-12 * dun
        elif mu == 1e-3:
            assert np.linalg.norm(dut) == pytest.approx(mu * dun, rel=1e-9)
            assert (dut @ ut0) / (np.linalg.norm(dut) * np.linalg.norm(ut0)) == pytest.approx(-1.0, abs=1e-12)
        else:
            u1 = v2[5] - v2[1]
            assert np.linalg.norm(u1 - (u1 @ n) * n) < 1e-12 * np.linalg.norm(ut0)


def test_self_contact_symmetric_sandwich():
    """Node 3 squeezed equally between nodes 1 and 5 from opposite sides: the
    penetration-weighted mean of its two pair responses is zero, while 1 and 5 are pushed
    apart symmetrically."""
    rod = _free_rod(8)
    pos = _far_line(8)
    c = np.array([100 * RS, 5 * RS, 0.0])
    pos[3] = c
    pos[1] = c - [1.8 * RS, 0.0, 0.0]
    pos[5] = c + [1.8 * RS, 0.0, 0.0]
    v2 = oracle.self_contact_pass(rod, pos, np.zeros((8, 3)), 0.2)
    np.testing.assert_allclose(v2[3], 0.0, atol=1e-15)
    assert v2[1][0] < 0 < v2[5][0]
    np.testing.assert_allclose(v2[1], -v2[5], rtol=1e-14)


def test_self_contact_is_continuous_at_the_contact_distance():
    """The response (normal part and, while sliding, the friction cut) vanishes linearly
    as the predicted gap closes to 2 r - no jump when a pair enters or leaves contact -
    and is exactly zero outside."""
    rod = _free_rod(8)
    ratios = []
    for eps in (1e-2, 1e-3, 1e-4, -1e-3):
        pos = _far_line(8)
        pos[5] = pos[1] + [0.0, 2 * RS * (1 - eps), 0.0]
        vel = np.zeros((8, 3))
        vel[5] = [1.0, 0.0, 0.0]  # mu du_n = 0.3 * 90 eps m/s < 1 m/s: sliding throughout
        v2 = oracle.self_contact_pass(rod, pos, vel, 0.3)
        dv = np.linalg.norm(v2 - vel)
        phi = 2 * RS - np.linalg.norm((pos[5] - pos[1]) + rod.dt * (vel[5] - vel[1]))
        if eps < 0:
            assert dv == 0.0
        else:
            ratios.append(dv / phi)
    assert max(ratios) / min(ratios) < 1.01


def test_self_contact_straight_rod_untouched():
    """Neighbours closer than 2 r along a straight rod never collide (index gap rule),
    and no other pair is in contact: the pass changes nothing."""
    rod = _free_rod(20, spacing=0.8)
    pos = np.zeros((20, 3))
    pos[:, 0] = np.arange(20) * 0.8 * RS
    vel = np.random.default_rng(4).normal(size=(20, 3)) * 1e-3
    cand, pairs = oracle.self_candidates(rod, pos)
    assert pairs > 0  # index gap 3 sits at 2.4 r < 3 r: candidates, not contacts
    np.testing.assert_array_equal(oracle.self_contact_pass(rod, pos, vel, 0.5), vel)


def test_self_collision_keeps_the_knot_from_passing_through_itself():
    """The trefoil (64 nodes, straight at rest) driven for 200 steps: with self-collision
    no two mass points come closer than 2 r (to 1 %), and the segments stay within 0.5 %
    of their rest length (the contact pass closes each iteration, after the distance
    sweeps); without it the strands pass through one another."""
    rod = W.torus_knot(64)
    drive = np.array([0.05, 0, 0, 0, 0, 0, 2.0, 0])
    m = max(2, int(np.floor(2 * rod.radius / (rod.length / 63))) + 1)
    idx = np.arange(64)
    far = np.abs(idx[:, None] - idx[None, :]) >= m

    def closest(p):
        return (np.linalg.norm(p[:, None] - p[None, :], axis=2)[far]).min() / (2 * rod.radius)

    with_sc = oracle.step_contact(rod, oracle.state_of(rod), self_mu=0.1, n_steps=200, drive=drive)
    without = oracle.step_contact(rod, oracle.state_of(rod), n_steps=200, drive=drive)
    assert closest(with_sc["pos"]) > 0.99
    assert closest(without["pos"]) < 0.6
    seg = np.linalg.norm(np.diff(with_sc["pos"], axis=0), axis=1)
    assert np.abs(seg / (rod.length / 63) - 1).max() < 5e-3


def test_self_contact_weighting_is_continuous_in_the_contact_set():
    """A mass point touching two others takes the penetration-weighted mean of the two
    responses: as the second overlap shrinks to zero its response tends to the response
    of the first pair alone (a plain mean over the touching pairs would jump to half)."""
    rod = _free_rod(8)
    c = np.array([100 * RS, 5 * RS, 0.0])

    def response(eps):
        pos = _far_line(8)
        pos[3] = c
        pos[1] = c - [1.7 * RS, 0.0, 0.0]
        pos[5] = c + [0.0, 2 * RS * (1 - eps), 0.0] if eps is not None else c + [0.0, 10 * RS, 0.0]
        vel = np.zeros((8, 3))
        vel[3] = [0.0, 0.0, 0.02]
        return oracle.self_contact_pass(rod, pos, vel, 0.1)[3]

    alone = response(None)
    assert np.linalg.norm(alone - [0.0, 0.0, 0.02]) > 1e-3
    errs = [np.linalg.norm(response(eps) - alone) for eps in (1e-2, 1e-3, 1e-4)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3 * np.linalg.norm(alone)
