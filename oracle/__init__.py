"""FP64 CPU oracle of the CoRdE rod time step (ctypes wrapper of ``corde_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline are the only users.  The oracle shares no code with the CUDA path and does not
import it; rods are passed in as any object carrying the attributes of a rod
description (n_nodes, length, radius, E_bend, E_stretch, G, density, Kp, damping_alpha,
mass_scale, inertia_scale, dt, gravity, n_iters, inextensible, clamp, rest_quat,
stiff_mul).  Which paper passage each C function follows is stated in the C source.

Parity status: every function is pinned by the tests in ``tests/test_oracle_*.py``
(closed forms, invariants, finite differences, the cantilever and twist statics).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corde_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (portable flags, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("length", ctypes.c_double), ("radius", ctypes.c_double), ("E_bend", ctypes.c_double),
        ("E_stretch", ctypes.c_double), ("G", ctypes.c_double), ("density", ctypes.c_double),
        ("Kp", ctypes.c_double), ("damping_alpha", ctypes.c_double), ("mass_scale", ctypes.c_double),
        ("inertia_scale", ctypes.c_double), ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
        ("n_nodes", ctypes.c_int), ("n_iters", ctypes.c_int), ("inextensible", ctypes.c_int),
        ("clamp", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(OracleParams)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_derive.argtypes = [_P, _D]
            L.oracle_darboux.argtypes = [_P, _D, _D]
            L.oracle_energy.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D]
            L.oracle_forces.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D]
            L.oracle_step.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int]
            L.oracle_rollout.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int, _D, ctypes.c_int]
            L.oracle_rollout_jvp.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int, _D, _D, _D, _D,
                                             _D, _D, _D, _D]
            L.oracle_count_flops.argtypes = [_P, _D, _D, _D, ctypes.c_int]
            L.oracle_count_flops.restype = ctypes.c_int64
            L.oracle_step_batch.argtypes = [ctypes.c_int, _P, _D, _D, _D, _D, _D, ctypes.c_int]
            L.oracle_step_tube.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int]
            L.oracle_step_contact.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int]
            L.oracle_self_candidates.argtypes = [_P, _D, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            L.oracle_self_contact_pass.argtypes = [_P, _D, _D, ctypes.c_double]
            L.oracle_step_pair.argtypes = [_P, _D, _D, _D, _D, _D, _D, _P, _D, _D, _D, _D, _D, _D, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int]
            for name in ("oracle_derive", "oracle_darboux", "oracle_energy", "oracle_forces", "oracle_step",
                         "oracle_rollout", "oracle_rollout_jvp", "oracle_step_batch", "oracle_step_pair",
                         "oracle_step_tube", "oracle_step_contact", "oracle_self_candidates",
                         "oracle_self_contact_pass"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def params(rod) -> OracleParams:
    p = OracleParams()
    for k in ("length", "radius", "E_bend", "E_stretch", "G", "density", "Kp", "damping_alpha",
              "mass_scale", "inertia_scale", "dt"):
        setattr(p, k, float(getattr(rod, k)))
    for i in range(3):
        p.gravity[i] = float(rod.gravity[i])
    p.n_nodes = int(rod.n_nodes)
    p.n_iters = int(rod.n_iters)
    p.inextensible = int(bool(rod.inextensible))
    p.clamp = int(rod.clamp)
    return p


def _arr(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name} rejected its arguments (rc={rc})")


def derive(rod) -> dict:
    out = np.zeros(16)
    _check(lib().oracle_derive(ctypes.byref(params(rod)), _ptr(out)), "oracle_derive")
    keys = ["l0", "A", "I", "K1", "K2", "K3", "Ks", "Kp", "mass_scale", "inertia_scale", "m_interior",
            "J1", "J2", "J3", "w_interior"]
    return {k: float(out[i]) for i, k in enumerate(keys)}


def darboux(rod, quat) -> np.ndarray:
    q = _arr(quat)
    u = np.zeros((max(q.shape[0] - 1, 0), 3))
    _check(lib().oracle_darboux(ctypes.byref(params(rod)), _ptr(q), _ptr(u)), "oracle_darboux")
    return u


def state_of(rod) -> dict:
    """Initial state arrays of a rod description (copies)."""
    n = rod.n_nodes
    return {
        "pos": _arr(rod.pos).copy(),
        "quat": _arr(rod.quat).copy(),
        "vel": _arr(rod.vel).copy() if rod.vel is not None else np.zeros((n, 3)),
        "omega": _arr(rod.omega).copy() if rod.omega is not None else np.zeros((n - 1, 3)),
    }


def energy(rod, state) -> dict:
    out = np.zeros(6)
    s = {k: _arr(v) for k, v in state.items()}
    _check(lib().oracle_energy(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.stiff_mul)),
                               _ptr(s["pos"]), _ptr(s["quat"]), _ptr(s.get("vel")), _ptr(s.get("omega")),
                               _ptr(out)), "oracle_energy")
    keys = ["bend", "penalty", "stretch", "gravity", "kin_lin", "kin_ang"]
    e = {k: float(out[i]) for i, k in enumerate(keys)}
    e["total"] = float(out.sum())
    return e


def forces(rod, pos, quat):
    """Elastic forces (N x 3), body torques (M x 3) and quaternion gradients (M x 4, xyzw)."""
    pos = _arr(pos)
    quat = _arr(quat)
    n, m = pos.shape[0], quat.shape[0]
    F = np.zeros((n, 3))
    tau = np.zeros((m, 3))
    g = np.zeros((m, 4))
    _check(lib().oracle_forces(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.stiff_mul)),
                               _ptr(pos), _ptr(quat), _ptr(F), _ptr(tau), _ptr(g)), "oracle_forces")
    return F, tau, g


def step(rod, state, n_steps=1, drive=None, f_ext=None, tau_ext=None) -> dict:
    """Advance a copy of ``state`` by ``n_steps`` time steps (constant drive)."""
    s = {k: _arr(v).copy() for k, v in state.items()}
    _check(lib().oracle_step(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.stiff_mul)),
                             _ptr(s["pos"]), _ptr(s["quat"]), _ptr(s["vel"]), _ptr(s["omega"]),
                             _ptr(_arr(drive)), _ptr(_arr(f_ext)), _ptr(_arr(tau_ext)), int(n_steps)),
           "oracle_step")
    return s


def rollout(rod, state, n_steps, drive_table=None, K=None, uhat=None):
    """Positions after every step (n_steps x N x 3) and the final state.  ``K`` and
    ``uhat`` ((N-2) x 3) override the per-joint stiffness and intrinsic Darboux vectors."""
    s = {k: _arr(v).copy() for k, v in state.items()}
    traj = np.zeros((n_steps, rod.n_nodes, 3))
    _check(lib().oracle_rollout(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.stiff_mul)),
                                _ptr(_arr(K)), _ptr(_arr(uhat)), _ptr(s["pos"]), _ptr(s["quat"]), _ptr(s["vel"]),
                                _ptr(s["omega"]), _ptr(_arr(drive_table)), int(n_steps), _ptr(traj), 1),
           "oracle_rollout")
    return traj, s


def rollout_jvp(rod, state, n_steps, drive_table=None, K=None, uhat=None, d_pos=None, d_vel=None, d_K=None,
                d_uhat=None, d_quat=None, d_omega=None):
    """Trajectory and its exact directional derivative (forward mode, dual numbers) along
    tangents of the initial positions, velocities, frames ((N-1) x 4, xyzw components) and
    body angular velocities, and of the per-joint stiffness and intrinsic Darboux vectors."""
    s = {k: _arr(v) for k, v in state.items()}
    traj = np.zeros((n_steps, rod.n_nodes, 3))
    dtraj = np.zeros_like(traj)
    _check(lib().oracle_rollout_jvp(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.stiff_mul)),
                                    _ptr(_arr(K)), _ptr(_arr(uhat)), _ptr(s["pos"]), _ptr(s["quat"]),
                                    _ptr(s["vel"]), _ptr(s["omega"]), _ptr(_arr(drive_table)), int(n_steps),
                                    _ptr(_arr(d_pos)), _ptr(_arr(d_vel)), _ptr(_arr(d_K)), _ptr(_arr(d_uhat)),
                                    _ptr(_arr(d_quat)), _ptr(_arr(d_omega)), _ptr(traj), _ptr(dtraj)),
           "oracle_rollout_jvp")
    return traj, dtraj


def material(rod):
    """Per-joint stiffness (K1, K2, K3) and intrinsic Darboux vectors as the oracle uses them."""
    d = derive(rod)
    J = max(rod.n_nodes - 2, 0)
    mul = np.ones((J, 3)) if rod.stiff_mul is None else _arr(rod.stiff_mul)
    K = mul * np.array([d["K1"], d["K2"], d["K3"]])[None, :]
    uhat = darboux(rod, rod.rest_quat) if rod.rest_quat is not None else np.zeros((J, 3))
    return K, uhat


def count_flops(rod, n_steps=1) -> int:
    n = lib().oracle_count_flops(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(_arr(rod.pos)),
                                 _ptr(_arr(rod.quat)), int(n_steps))
    if n < 0:
        raise ValueError("oracle_count_flops rejected its arguments")
    return int(n)


def step_batch(rods, states, n_steps) -> int:
    """Step many independent rods in place (OpenMP over rods); returns threads used."""
    P = (OracleParams * len(rods))(*[params(r) for r in rods])
    rest = np.ascontiguousarray(np.concatenate([_arr(r.rest_quat) for r in rods]))
    pos = np.ascontiguousarray(np.concatenate([s["pos"] for s in states]))
    quat = np.ascontiguousarray(np.concatenate([s["quat"] for s in states]))
    vel = np.ascontiguousarray(np.concatenate([s["vel"] for s in states]))
    om = np.ascontiguousarray(np.concatenate([s["omega"] for s in states]))
    threads = lib().oracle_step_batch(len(rods), P, _ptr(rest), _ptr(pos), _ptr(quat), _ptr(vel), _ptr(om),
                                      int(n_steps))
    if threads < 0:
        raise ValueError("oracle_step_batch rejected its arguments")
    no = fo = 0
    for r, s in zip(rods, states):
        n = r.n_nodes
        s["pos"][:] = pos[no:no + n]
        s["vel"][:] = vel[no:no + n]
        s["quat"][:] = quat[fo:fo + n - 1]
        s["omega"][:] = om[fo:fo + n - 1]
        no += n
        fo += n - 1
    return threads


def step_pair(outer, s_outer, inner, s_inner, mode, beta, n_steps=1, drive_outer=None, drive_inner=None):
    """Advance copies of an outer/inner rod pair (catheter, guidewire) with binding mode
    0/1/2 and offset beta (inner node i at outer arclength (i + beta) l0)."""
    so = {k: _arr(v).copy() for k, v in s_outer.items()}
    si = {k: _arr(v).copy() for k, v in s_inner.items()}
    _check(lib().oracle_step_pair(ctypes.byref(params(outer)), _ptr(_arr(outer.rest_quat)), _ptr(so["pos"]),
                                  _ptr(so["quat"]), _ptr(so["vel"]), _ptr(so["omega"]), _ptr(_arr(drive_outer)),
                                  ctypes.byref(params(inner)), _ptr(_arr(inner.rest_quat)), _ptr(si["pos"]),
                                  _ptr(si["quat"]), _ptr(si["vel"]), _ptr(si["omega"]), _ptr(_arr(drive_inner)),
                                  int(mode), float(beta), int(n_steps)), "oracle_step_pair")
    return so, si


def step_tube(rod, state, tube, n_steps=1, drive=None):
    """Advance a copy of ``state`` inside an analytic vessel tube = [cx, cy, cz, Rc, Rt, mu]."""
    s = {k: _arr(v).copy() for k, v in state.items()}
    _check(lib().oracle_step_tube(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(s["pos"]),
                                  _ptr(s["quat"]), _ptr(s["vel"]), _ptr(s["omega"]), _ptr(_arr(drive)),
                                  _ptr(_arr(tube)), int(n_steps)), "oracle_step_tube")
    return s


def step_contact(rod, state, tube=None, self_mu=None, n_steps=1, drive=None):
    """Advance a copy of ``state`` with contact: the vessel tube = [cx, cy, cz, Rc, Rt, mu]
    (None: no vessel) and self-collision with friction ``self_mu`` (None: none)."""
    s = {k: _arr(v).copy() for k, v in state.items()}
    sp = None if self_mu is None else np.array([float(self_mu)])
    _check(lib().oracle_step_contact(ctypes.byref(params(rod)), _ptr(_arr(rod.rest_quat)), _ptr(s["pos"]),
                                     _ptr(s["quat"]), _ptr(s["vel"]), _ptr(s["omega"]), _ptr(_arr(drive)),
                                     _ptr(_arr(tube)), _ptr(sp), int(n_steps)), "oracle_step_contact")
    return s


def self_candidates(rod, pos, cap=64):
    """Self-collision candidate partners of every node of ``pos`` (list of ascending
    index arrays) and the number of candidate pairs."""
    pos = _arr(pos)
    n = pos.shape[0]
    counts = np.zeros(n, dtype=np.int32)
    lst = np.zeros((n, cap), dtype=np.int32)
    pairs = lib().oracle_self_candidates(ctypes.byref(params(rod)), _ptr(pos), counts.ctypes.data,
                                         lst.ctypes.data, int(cap))
    if pairs < 0:
        raise RuntimeError("oracle_self_candidates failed")
    return [lst[i, :min(counts[i], cap)].copy() for i in range(n)], int(pairs)


def self_contact_pass(rod, pos, vel, mu):
    """One Jacobi pass of the self-contact constraints: the velocities after it."""
    pos = _arr(pos)
    v = _arr(vel).copy()
    _check(lib().oracle_self_contact_pass(ctypes.byref(params(rod)), _ptr(pos), _ptr(v),
                                          float(mu)), "oracle_self_contact_pass")
    return v
