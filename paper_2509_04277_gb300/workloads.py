"""Seeded synthetic inputs for the rod workloads (shared by the CUDA path and the oracle).

This module only *generates inputs*: rest shapes, jittered initial states, material
draws and drive signals.  It contains none of the method's arithmetic (no Darboux
vectors, energies, forces, constraint projections or integration).  Rotations are
built with ``scipy.spatial.transform.Rotation`` so that no quaternion algebra of the
method lives here.  All randomness comes from numpy's counter-based Philox generator,
one stream per seed.

Conventions used by every consumer of these arrays:
  * a rod of ``n`` nodes has ``n - 1`` material frames (Section 2.1, "Discretization");
  * quaternions are stored as ``(x, y, z, w)`` with ``w`` the real part;
  * node 0 and frame 0 form the clamped / driven base when ``clamp == 1``.

The workloads mirror the paper's experiments (Section 3): the free-space pendulum
(a rod locked at one end, Section 3.1), the 512-element guidewire driven at haptic
rate (Section 3.3), the 2x512 catheter/guidewire pair (Section 3.4), plus a batch of
uneven rods and an adjoint rollout.  The paper's vascular meshes and recorded haptic
trajectories are not available; seeded sinusoidal drives stand in for the haptic input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

# --------------------------------------------------------------------------- helpers


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox) for one seed."""
    return np.random.Generator(np.random.Philox(int(seed)))


def _hemisphere_continuous(q: np.ndarray) -> np.ndarray:
    """Flip signs so that consecutive quaternions have a non-negative dot product
    (the same rotation, chosen on one hemisphere)."""
    q = q.copy()
    if q.shape[0] and q[0, 3] < 0:
        q[0] = -q[0]
    for j in range(1, q.shape[0]):
        if float(np.dot(q[j - 1], q[j])) < 0.0:
            q[j] = -q[j]
    return q


# --------------------------------------------------------------------------- rod specs


@dataclass
class RodSpec:
    """Material, geometry and initial state of one rod (SI units)."""

    n_nodes: int
    length: float
    radius: float
    E_bend: float
    E_stretch: float
    G: float
    density: float
    dt: float
    n_iters: int = 10
    inextensible: bool = True
    clamp: int = 1
    Kp: float = 0.0  # 0 -> default rule
    damping_alpha: float = 0.0
    mass_scale: float = 0.0  # 0 -> default rule
    inertia_scale: float = 0.0  # 0 -> default rule
    gravity: tuple = (0.0, 0.0, 0.0)
    pos: np.ndarray = field(default=None, repr=False)  # (n, 3)
    quat: np.ndarray = field(default=None, repr=False)  # (n-1, 4) xyzw
    rest_quat: np.ndarray = field(default=None, repr=False)  # (n-1, 4) xyzw
    vel: np.ndarray = field(default=None, repr=False)  # (n, 3)
    omega: np.ndarray = field(default=None, repr=False)  # (n-1, 3), body frame
    stiff_mul: np.ndarray = field(default=None, repr=False)  # (n-2, 3) or None

    def copy(self) -> "RodSpec":
        out = RodSpec(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        for k in ("pos", "quat", "rest_quat", "vel", "omega", "stiff_mul"):
            v = getattr(self, k)
            setattr(out, k, None if v is None else np.array(v, dtype=np.float64, copy=True))
        return out


def straight_rod(
    n: int,
    length: float,
    *,
    orientation: Rotation | None = None,
    base=(0.0, 0.0, 0.0),
    pos_sigma: float = 0.0,
    ang_sigma: float = 0.0,
    seg_sigma: float = 0.0,
    seed: int = 0,
    jitter_base: bool = False,
    **material,
) -> RodSpec:
    """A straight rod at rest along the frame's third director, plus seeded jitter.

    ``orientation`` maps the body frame to the world (default: e_z -> e_x, i.e. the
    rod lies along +x).  Rest frames are all equal to ``orientation`` (zero intrinsic
    curvature); the initial frames are ``orientation * jitter_j`` with a small
    rotation vector drawn N(0, ang_sigma^2) per component; node positions get
    N(0, pos_sigma^2) jitter.  ``seg_sigma`` instead tilts every segment direction by
    a small random rotation (N(0, seg_sigma^2) per component) while keeping each
    segment at its rest length, which suits inextensible rods.  The clamped base
    (node 0, frame 0) is not jittered unless ``jitter_base``.
    """
    if orientation is None:
        orientation = Rotation.from_rotvec([0.0, math.pi / 2, 0.0])
    g = rng(seed)
    m = n - 1
    axis = orientation.apply([0.0, 0.0, 1.0])
    l0 = length / m
    s = np.arange(n, dtype=np.float64) * l0
    pos = np.asarray(base, dtype=np.float64)[None, :] + s[:, None] * axis[None, :]
    dpos = g.standard_normal((n, 3)) * pos_sigma
    rvec = g.standard_normal((m, 3)) * ang_sigma
    if not jitter_base:
        dpos[0] = 0.0
        rvec[0] = 0.0
    pos = pos + dpos
    if seg_sigma > 0.0:
        tilt = Rotation.from_rotvec(g.standard_normal((m, 3)) * seg_sigma)
        dirs = (orientation * tilt).apply([0.0, 0.0, 1.0])
        pos = np.empty((n, 3))
        pos[0] = base
        pos[1:] = np.asarray(base, dtype=np.float64)[None, :] + np.cumsum(l0 * dirs, axis=0)
    rest = np.tile(orientation.as_quat()[None, :], (m, 1))
    quat = (orientation * Rotation.from_rotvec(rvec)).as_quat()
    rest = _hemisphere_continuous(rest)
    quat = _hemisphere_continuous(quat)
    return RodSpec(
        n_nodes=n,
        length=length,
        pos=pos,
        quat=quat,
        rest_quat=rest,
        vel=np.zeros((n, 3)),
        omega=np.zeros((m, 3)),
        **material,
    )


# --------------------------------------------------------------------------- drives


def sinusoid_drive(seed: int, n_launches: int, launch_dt: float, axis=(1.0, 0.0, 0.0),
                   insert_amp=(1e-3, 5e-3), insert_freq=(0.5, 2.0),
                   twist_amp=(0.1, 0.5), twist_freq=(0.5, 2.0)) -> np.ndarray:
    """Seeded insertion/rotation input for a driven base, one sample per launch.

    Base insertion s(t) = A sin(2 pi f t + phi) along ``axis`` and rotation about the
    rod axis theta(t) = B sin(2 pi f' t + phi').  The kernel integrates velocities, so
    each row is the time derivative at the launch start t_k = k * launch_dt
    (zero-order hold over the launch):  [v_x, v_y, v_z, 0, w_x, w_y, w_z, 0] with
    the angular velocity given in the body frame of the base (twist about d3).
    """
    g = rng(seed)
    A = g.uniform(*insert_amp)
    f = g.uniform(*insert_freq)
    ph = g.uniform(0, 2 * math.pi)
    B = g.uniform(*twist_amp)
    f2 = g.uniform(*twist_freq)
    ph2 = g.uniform(0, 2 * math.pi)
    t = np.arange(n_launches, dtype=np.float64) * launch_dt
    sdot = 2 * math.pi * f * A * np.cos(2 * math.pi * f * t + ph)
    thdot = 2 * math.pi * f2 * B * np.cos(2 * math.pi * f2 * t + ph2)
    out = np.zeros((n_launches, 8))
    out[:, 0:3] = sdot[:, None] * np.asarray(axis, dtype=np.float64)[None, :]
    out[:, 6] = thdot
    return out


# --------------------------------------------------------------------------- workloads


def extensible_pendulum(n: int = 64, seed: int = 1, *, literal_masses: bool = False) -> RodSpec:
    """Plain extensible CoRdE rod, one end clamped, gravity on (free-space test,
    Section 3.1): L = 1 m, r = 1 mm, E = 50 GPa, G = 20 GPa, rho = 6500 kg/m^3,
    Rayleigh damping 0.1 1/s, dt = 1e-5 s.  Node jitter 1e-4 m, frame jitter 1e-3 rad.
    ``literal_masses`` keeps the physical masses and inertias (mass/inertia scale 1)."""
    sc = 1.0 if literal_masses else 0.0
    return straight_rod(
        n, 1.0, pos_sigma=1e-4, ang_sigma=1e-3, seed=seed,
        radius=1e-3, E_bend=50e9, E_stretch=50e9, G=20e9, density=6500.0,
        dt=1e-5, n_iters=0, inextensible=False, clamp=1, damping_alpha=0.1,
        gravity=(0.0, 0.0, -9.81), mass_scale=sc, inertia_scale=sc,
    )


def guidewire(n: int = 512, seed: int = 2) -> RodSpec:
    """Inextensible 512-element guidewire (Section 3.3): L = 1.5 m, r = 0.45 mm,
    E = 60 GPa, G = E / 2.6, rho = 6500, 10 constraint iterations, dt = 1e-4 s,
    driven base, no gravity.  Initial shape: straight along x with segment tilts and
    frame jitter of 1e-3 rad."""
    E = 60e9
    return straight_rod(
        n, 1.5, seg_sigma=1e-3, ang_sigma=1e-3, seed=seed,
        radius=0.45e-3, E_bend=E, E_stretch=E, G=E / 2.6, density=6500.0,
        dt=1e-4, n_iters=10, inextensible=True, clamp=1, damping_alpha=0.0,
    )


def catheter(n: int = 512, seed: int = 3) -> RodSpec:
    """Catheter of the 2x512 pair (Section 3.4): r = 1 mm, E = 2 GPa, L = 1.5 m."""
    E = 2e9
    return straight_rod(
        n, 1.5, seg_sigma=1e-3, ang_sigma=1e-3, seed=seed,
        radius=1e-3, E_bend=E, E_stretch=E, G=E / 2.6, density=6500.0,
        dt=1e-4, n_iters=10, inextensible=True, clamp=1, damping_alpha=0.0,
    )


def batched_rods(n_rods: int = 4096, seed: int = 4, n_min: int = 16, n_max: int = 2048,
                 dt: float = 1e-4, n_iters=None) -> list[RodSpec]:
    """Independent inextensible rods with log-uniform element counts in
    [n_min, n_max], E ~ U[1, 100] GPa, radius ~ U[0.2, 2] mm, L = 1 m, G = E / 2.6,
    rho = 6500, base orientation uniform on SO(3), gravity on (free-space pendulums
    locked at one end, Section 3.1).  ``n_iters``: constraint iterations per rod (a
    sequence of n_rods counts), else 10 for every rod."""
    g = rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(n_min), math.log(n_max), size=n_rods))).astype(int)
    ns = np.clip(ns, n_min, n_max)
    Es = g.uniform(1e9, 100e9, size=n_rods)
    rs = g.uniform(0.2e-3, 2e-3, size=n_rods)
    orients = Rotation.random(n_rods, random_state=g)
    seeds = g.integers(0, 2**31 - 1, size=n_rods)
    rods = []
    for k in range(n_rods):
        rods.append(straight_rod(
            int(ns[k]), 1.0, orientation=orients[k], seg_sigma=1e-3, ang_sigma=1e-3,
            seed=int(seeds[k]), radius=float(rs[k]), E_bend=float(Es[k]),
            E_stretch=float(Es[k]), G=float(Es[k]) / 2.6, density=6500.0, dt=dt,
            n_iters=10 if n_iters is None else int(n_iters[k]), inextensible=True, clamp=1, damping_alpha=0.0,
            gravity=(0.0, 0.0, -9.81),
        ))
    return rods


def batched_lengths(n_rods: int = 4096, seed: int = 4, n_min: int = 16, n_max: int = 2048) -> np.ndarray:
    """Only the element counts of ``batched_rods`` (same draw, cheap)."""
    g = rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(n_min), math.log(n_max), size=n_rods))).astype(int)
    return np.clip(ns, n_min, n_max)


def adjoint_rod(n: int = 256, seed: int = 5) -> RodSpec:
    """256-element inextensible rod for the adjoint rollout: per-joint bending and
    twist stiffness multipliers log-normal (sigma 0.3) about a 1 N m^2 scale.
    The rod has E chosen so that E I = 1 N m^2 at r = 1 mm."""
    g = rng(seed)
    r = 1e-3
    I = math.pi * r**4 / 4
    E = 1.0 / I
    rod = straight_rod(
        n, 1.0, seg_sigma=1e-3, ang_sigma=1e-3, seed=seed + 1000,
        radius=r, E_bend=E, E_stretch=E, G=E / 2.6, density=6500.0,
        dt=1e-4, n_iters=10, inextensible=True, clamp=1, damping_alpha=0.0,
        gravity=(0.0, 0.0, -9.81),
    )
    mul = np.exp(g.standard_normal((n - 2, 2)) * 0.3)
    rod.stiff_mul = np.stack([mul[:, 0], mul[:, 0], mul[:, 1]], axis=1)
    return rod


def tip_target(seed: int, n_steps: int, dt: float, start) -> np.ndarray:
    """Seeded smooth target curve for the tip: start + a few-mm sinusoidal excursion."""
    g = rng(seed)
    amp = g.uniform(1e-3, 5e-3, size=3)
    fr = g.uniform(1.0, 5.0, size=3)
    ph = g.uniform(0, 2 * math.pi, size=3)
    t = (np.arange(n_steps, dtype=np.float64) + 1) * dt
    return np.asarray(start, dtype=np.float64)[None, :] + amp[None, :] * np.sin(
        2 * math.pi * fr[None, :] * t[:, None] + ph[None, :]) * (t[:, None] / t[-1])


def random_directions(seed: int, n_dirs: int, size: int) -> np.ndarray:
    """Seeded unit directions for directional-derivative checks."""
    d = rng(seed).standard_normal((n_dirs, size))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def catheter_guidewire(n: int = 512, seed: int = 3, beta0: float = -100.25):
    """The 2 x n catheter/guidewire pair (Section 3.4): both rods 1.5 m long with n nodes
    (shared segment length), along +x; the guidewire runs inside the catheter, its node i
    at the catheter arclength (i + beta0) l0 (beta0 < 0: the guidewire base lies behind the
    catheter base and its proximal part is outside).  Returns (catheter, guidewire)."""
    cat = catheter(n, seed=seed)
    gw = guidewire(n, seed=seed + 1)
    l0 = gw.length / (n - 1)
    base = (beta0 * l0, 0.0, 0.0)
    gw2 = straight_rod(n, gw.length, base=base, seg_sigma=1e-3, ang_sigma=1e-3, seed=seed + 1,
                       radius=gw.radius, E_bend=gw.E_bend, E_stretch=gw.E_stretch, G=gw.G, density=gw.density,
                       dt=gw.dt, n_iters=gw.n_iters, inextensible=True, clamp=1, damping_alpha=0.0)
    return cat, gw2


def pair_drives(seed: int, n_launches: int, launch_dt: float, l0: float, beta0: float):
    """Seeded insertion/twist drives of the catheter and guidewire bases (1 kHz samples,
    zero-order hold per launch) and the binding offset beta of every launch: beta0 plus
    the guidewire's base displacement relative to the catheter's, in segments (prefix
    sums of the held velocities).  Returns (drive_catheter, drive_guidewire), each
    [n_launches, 8]; beta is in slot 3 of the guidewire rows."""
    dc = sinusoid_drive(seed, n_launches, launch_dt)
    dg = sinusoid_drive(seed + 7, n_launches, launch_dt)
    rel = (dg[:, 0] - dc[:, 0]) * launch_dt
    disp = np.concatenate([[0.0], np.cumsum(rel)[:-1]])
    dg[:, 3] = beta0 + disp / l0
    return dc, dg


def vessel_guidewire(n: int = 512, seed: int = 11, rc: float = 0.5, rt: float = 2e-3, mu: float = 0.1,
                     offset: float = 0.8):
    """The guidewire inside a curved vessel (the insertion test of Section 3.3 with an
    analytic tube in place of the phantom mesh): the vessel centreline is the circle of
    radius rc about (0, rc) in the plane z = 0, tangent to +x at the origin; inner radius
    rt, Coulomb friction mu.  The guidewire (straight at rest) starts as a polygon on the
    circle of radius rc + offset (rt - r) (towards the outer wall) with segments of rest
    length, frames along the segments, seeded segment tilts of 2e-5 rad; the wall holds it
    bent, so it presses against the outer wall within a few steps.
    Returns (rod, tube) with tube = [cx, cy, cz, Rc, Rt, mu]."""
    rod = guidewire(n, seed=seed)
    g = rng(seed + 17)
    m = n - 1
    l0 = rod.length / m
    big_r = rc + offset * (rt - rod.radius)
    dphi = 2.0 * math.asin(l0 / (2.0 * big_r))
    phi_seg = (np.arange(m) + 0.5) * dphi  # chord j points along the tangent at its middle
    align = Rotation.from_rotvec([0.0, math.pi / 2, 0.0])
    frames = Rotation.from_rotvec(np.stack([np.zeros(m), np.zeros(m), phi_seg], axis=1)) * align
    frames = frames * Rotation.from_rotvec(g.standard_normal((m, 3)) * 2e-5)
    pos = np.zeros((n, 3))
    pos[0] = (0.0, rc - big_r, 0.0)
    pos[1:] = pos[0] + np.cumsum(l0 * frames.apply([0.0, 0.0, 1.0]), axis=0)
    rod.pos = pos
    rod.quat = _hemisphere_continuous(frames.as_quat())
    rod.rest_quat = _hemisphere_continuous(np.tile(align.as_quat()[None, :], (m, 1)))
    tube = np.array([0.0, rc, 0.0, rc, rt, mu])
    return rod, tube


def _chord_march(curve: np.ndarray, l0: float, n: int) -> np.ndarray:
    """n points along a densely sampled polyline, consecutive points exactly l0 apart."""
    out = np.zeros((n, 3))
    out[0] = curve[0]
    k = 0
    for i in range(1, n):
        p = out[i - 1]
        while k + 1 < len(curve) and np.linalg.norm(curve[k + 1] - p) < l0:
            k += 1
        if k + 1 >= len(curve):
            raise ValueError("curve too short for n points at this spacing")
        # point on segment curve[k] -> curve[k+1] at distance l0 from p (the far root)
        a, b = curve[k], curve[k + 1]
        d = b - a
        f = a - p
        A, B, C = d @ d, 2 * (f @ d), f @ f - l0 * l0
        s = (-B + math.sqrt(max(B * B - 4 * A * C, 0.0))) / (2 * A)
        out[i] = a + s * d
    return out


def _transported_frames(pos: np.ndarray, l0: float) -> list:
    """Segment frames along a polyline of spacing l0: the first takes its director d3 = z to
    the first segment, each next one follows by the smallest rotation between consecutive
    segments (parallel transport)."""
    t = np.diff(pos, axis=0) / l0
    rots = []
    cur = Rotation.align_vectors(t[0][None, :], np.array([[0.0, 0.0, 1.0]]))[0]
    rots.append(cur)
    for j in range(1, len(t)):
        ax = np.cross(t[j - 1], t[j])
        s = np.linalg.norm(ax)
        ang = math.atan2(s, float(t[j - 1] @ t[j]))
        step = Rotation.from_rotvec(ax / s * ang) if s > 0 else Rotation.identity()
        cur = step * cur
        rots.append(cur)
    return rots


def torus_knot(n: int = 512, seed: int = 21, gap: float = 1.05, spacing: float = 1.35):
    """Knot-like self-collision configuration (stands in for the haptic knot tying of
    Section 3.5): a guidewire (r = 0.45 mm, E = 60 GPa, straight at rest, base driven) laid
    on a (2, q) torus knot - two strands twisted around each other along a ring, strand
    separation 2 gap r - cut open at a seeded angle so that its two ends lie side by side.
    Nodes sit on the curve exactly l0 = spacing r apart (spheres of neighbouring mass
    points overlap, as the paper's knot needs); frames follow the segments by parallel
    transport, with seeded tilts of 2e-5 rad.  The ring's core radius follows from n
    (R = (n - 1) l0 / 4 pi) and q is the odd number giving a twist pitch near 20 mm
    (q = 3, a trefoil, for small n)."""
    rod = guidewire(n, seed=seed)
    g = rng(seed + 31)
    r = rod.radius
    l0 = spacing * r
    a = gap * r
    R = (n - 1) * l0 / (4.0 * math.pi)
    q = max(3, int(round(4.0 * math.pi * R / 0.02)))
    if q % 2 == 0:
        q += 1
    phi0 = g.uniform(0.0, 2.0 * math.pi)
    phi = phi0 + np.linspace(0.0, 4.0 * math.pi, 400 * n)
    th = 0.5 * q * (phi - phi0)
    rho = R + a * np.cos(th)
    curve = np.stack([rho * np.cos(phi), rho * np.sin(phi), a * np.sin(th)], axis=1)
    pos = _chord_march(curve, l0, n)
    m = n - 1
    rots = _transported_frames(pos, l0)
    frames = Rotation.concatenate(rots) * Rotation.from_rotvec(g.standard_normal((m, 3)) * 2e-5)
    rod.length = l0 * m
    rod.pos = pos - pos[0]
    rod.quat = _hemisphere_continuous(frames.as_quat())
    rod.rest_quat = np.tile(rots[0].as_quat()[None, :], (m, 1))
    return rod


def coil(n: int = 130, seed: int = 720, radius: float = 3.0, pitch: float = 1.96, spacing: float = 1.35):
    """A guidewire (r = 0.45 mm) wound into a tight helix, coil radius `radius` r and
    pitch `pitch` r (neighbouring turns pressed slightly into each other), nodes exactly
    l0 = spacing r apart; the helix is also the rest shape, so the coil holds its form.
    Dense on purpose: within 6 r a mass point has up to ~26 partners above it, within the
    plain 3 r reach of the self-collision detection at most ~4."""
    rod = guidewire(n, seed=seed)
    g = rng(seed + 31)
    r = rod.radius
    l0 = spacing * r
    rh, p = radius * r, pitch * r
    turns = (n - 1) * l0 / (2.0 * math.pi * rh) + 2.0
    th = np.linspace(0.0, 2.0 * math.pi * turns, 400 * n)
    curve = np.stack([rh * np.cos(th), rh * np.sin(th), p * th / (2.0 * math.pi)], axis=1)
    pos = _chord_march(curve, l0, n)
    m = n - 1
    rots = _transported_frames(pos, l0)
    rest = Rotation.concatenate(rots)
    frames = rest * Rotation.from_rotvec(g.standard_normal((m, 3)) * 2e-5)
    rod.length = l0 * m
    rod.pos = pos - pos[0]
    rod.quat = _hemisphere_continuous(frames.as_quat())
    rod.rest_quat = _hemisphere_continuous(rest.as_quat())
    return rod
