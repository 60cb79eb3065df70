"""Thin ctypes binding of ``libcorde.so`` (declared in ``include/corde.h``).

The module-level functions carry the C names and only marshal arguments; every step of
the rod computation runs in the library's CUDA kernels.  ``RodBatch`` bundles a handle
with numpy/torch conveniences for tests and the benchmark.  There is no CPU fallback:
if the library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcorde.so")

CORDE_OK = 0
CORDE_ERR_ARG = -1
CORDE_ERR_CUDA = -2
CORDE_ERR_OOM = -3
CORDE_ERR_UNSUPPORTED = -4
CORDE_ERR_NONFINITE = -5


class CordeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class RodParams(ctypes.Structure):
    _fields_ = [
        ("length", ctypes.c_double), ("radius", ctypes.c_double), ("E_bend", ctypes.c_double),
        ("E_stretch", ctypes.c_double), ("G", ctypes.c_double), ("density", ctypes.c_double),
        ("Kp", ctypes.c_double), ("damping_alpha", ctypes.c_double), ("mass_scale", ctypes.c_double),
        ("inertia_scale", ctypes.c_double), ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
        ("n_nodes", ctypes.c_int), ("n_iters", ctypes.c_int), ("inextensible", ctypes.c_int),
        ("clamp", ctypes.c_int),
    ]


_VP = ctypes.c_void_p
_lib = None

# name -> (restype, argtypes); the exported C ABI
SIGNATURES = {
    "rod_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(RodParams), _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                  ctypes.POINTER(_VP)]),
    "rod_step": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "rod_step_io": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "rod_set_input": (ctypes.c_int, [_VP, _VP, _VP]),
    "rod_bind": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "rod_set_tube": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "rod_set_self_collision": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "rod_self_collision_stats": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "rod_get_state": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "rod_set_state": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "rod_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]),
    "rod_get_derived": (ctypes.c_int, [_VP, _VP, _VP]),
    "rod_set_material": (ctypes.c_int, [_VP, _VP, _VP]),
    "rod_diagnostics": (ctypes.c_int, [_VP, _VP]),
    "rod_set_plan": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "rod_set_launch_overlap": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rod_set_adjoint_record_budget": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "rod_set_adjoint_pipeline": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rod_adjoint_info": (ctypes.c_int, [_VP, _VP]),
    "rod_set_plan_cluster": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "rod_set_plan_grid": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "rod_autotune": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "rod_autotune_steps": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "rod_get_plan": (ctypes.c_int, [_VP, _VP]),
    "rod_last_launch_count": (ctypes.c_int, [_VP]),
    "rod_set_graph_mode": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rod_mailbox_enable": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "rod_mailbox_write": (ctypes.c_int, [_VP, _VP]),
    "rod_mailbox_read": (ctypes.c_int, [_VP, _VP]),
    "rod_mailbox_log": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "rod_mailbox_disable": (ctypes.c_int, [_VP]),
    "rod_mailbox_positions_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rod_mailbox_positions": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "rod_mailbox_exchange": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_longlong, _VP, ctypes.c_longlong, _VP]),
    "rod_mailbox_tick": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_longlong, _VP, _VP, ctypes.c_longlong, _VP]),
    "rod_mailbox_lockstep": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "rod_mailbox_status": (ctypes.c_int, [_VP, _VP]),
    "rod_steps_done": (ctypes.c_int64, [_VP]),
    "rod_rollout": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "rod_adjoint": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "rod_adjoint_noalloc": (ctypes.c_int, [ctypes.POINTER(RodParams), _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                           ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "rod_barrier_floor": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), _VP]),
    "rod_device_info": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "rod_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "rod_destroy": (None, [_VP]),
    "rod_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rod_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise CordeError(CORDE_ERR_UNSUPPORTED,
                             f"libcorde.so not found at {path}; build it with __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != CORDE_OK:
        msg = load().rod_last_error()
        raise CordeError(rc, f"{what}: {msg.decode() if msg else load().rod_strerror(rc).decode()}")


def _ptr(x):
    """Pointer of a numpy array / torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C names


def rod_create(params, pos, quat, rest_quat=None, vel=None, omega=None, stiff_mul=None, stream=None):
    P = (RodParams * len(params))(*params)
    h = _VP()
    _check(load().rod_create(len(params), P, _ptr(pos), _ptr(quat), _ptr(rest_quat), _ptr(vel), _ptr(omega),
                             _ptr(stiff_mul), _stream(stream), ctypes.byref(h)), "rod_create")
    return h


def rod_step(h, n_steps, drive=None, stream=None):
    _check(load().rod_step(h, int(n_steps), _ptr(drive), _stream(stream)), "rod_step")


def rod_step_io(h, n_steps, drive=None, pos_out=None, stream=None):
    """rod_step that also writes the positions after the last step to pos_out
    ([n_elements, 4] float32, device or pinned host memory)."""
    _check(load().rod_step_io(h, int(n_steps), _ptr(drive), _ptr(pos_out), _stream(stream)), "rod_step_io")


def rod_bind(h, outer, inner, mode):
    _check(load().rod_bind(h, int(outer), int(inner), int(mode)), "rod_bind")


def rod_set_tube(h, rod, tube, enable=True):
    """tube = (cx, cy, cz, Rc, Rt, mu): analytic vessel of rod `rod` (enable=False removes it)."""
    t = np.zeros(8, dtype=np.float64)
    t[:6] = np.asarray(tube, dtype=np.float64)[:6]
    t[6] = 1.0 if enable else 0.0
    _check(load().rod_set_tube(h, int(rod), t.ctypes.data), "rod_set_tube")


def rod_set_self_collision(h, rod, mu, enable=True):
    """Self-collision of rod `rod` with strand friction mu (enable=False turns it off)."""
    p = np.array([float(mu), 1.0 if enable else 0.0], dtype=np.float64)
    _check(load().rod_set_self_collision(h, int(rod), p.ctypes.data), "rod_set_self_collision")


def rod_self_collision_stats(h, rod) -> dict:
    out = np.zeros(5, dtype=np.int32)
    _check(load().rod_self_collision_stats(h, int(rod), out.ctypes.data), "rod_self_collision_stats")
    return {"candidate_pairs": int(out[0]), "max_partners_above": int(out[1]), "overlapping_pairs": int(out[2]),
            "overflow": int(out[3]), "skin_builds": int(out[4])}


def rod_set_input(h, drive, stream=None):
    _check(load().rod_set_input(h, _ptr(drive), _stream(stream)), "rod_set_input")


def rod_get_state(h, pos4=None, quat4=None, vel4=None, omega4=None, stream=None):
    _check(load().rod_get_state(h, _ptr(pos4), _ptr(quat4), _ptr(vel4), _ptr(omega4), _stream(stream)),
           "rod_get_state")


def rod_set_state(h, pos4=None, quat4=None, vel4=None, omega4=None, stream=None):
    _check(load().rod_set_state(h, _ptr(pos4), _ptr(quat4), _ptr(vel4), _ptr(omega4), _stream(stream)),
           "rod_set_state")


def rod_info(h):
    n = ctypes.c_int()
    e = ctypes.c_int64()
    _check(load().rod_info(h, ctypes.byref(n), ctypes.byref(e)), "rod_info")
    return n.value, e.value


def rod_get_derived(h, per_rod=None, per_joint=None):
    _check(load().rod_get_derived(h, _ptr(per_rod), _ptr(per_joint)), "rod_get_derived")


def rod_set_material(h, per_joint, stream=None):
    _check(load().rod_set_material(h, _ptr(per_joint), _stream(stream)), "rod_set_material")


def rod_diagnostics(h, out):
    return load().rod_diagnostics(h, _ptr(out))


def rod_set_plan(h, ept, nt):
    _check(load().rod_set_plan(h, int(ept), int(nt)), "rod_set_plan")


def rod_set_adjoint_record_budget(h, n_bytes):
    _check(load().rod_set_adjoint_record_budget(h, int(n_bytes)), "rod_set_adjoint_record_budget")


def rod_set_adjoint_pipeline(h, enable=True):
    """Pipelined reverse pass (a cluster of two blocks per rod) where it applies."""
    _check(load().rod_set_adjoint_pipeline(h, 1 if enable else 0), "rod_set_adjoint_pipeline")


def rod_set_launch_overlap(h, enable):
    _check(load().rod_set_launch_overlap(h, int(enable)), "rod_set_launch_overlap")


def rod_set_plan_cluster(h, ept, nt, cluster):
    _check(load().rod_set_plan_cluster(h, int(ept), int(nt), int(cluster)), "rod_set_plan_cluster")


def rod_set_plan_grid(h, ept, nt, blocks):
    _check(load().rod_set_plan_grid(h, int(ept), int(nt), int(blocks)), "rod_set_plan_grid")


def rod_autotune(h, n_steps, stream=None):
    _check(load().rod_autotune(h, int(n_steps), _stream(stream)), "rod_autotune")


def rod_autotune_steps(h, candidates, min_steps, stream=None) -> int:
    """Steps per launch, among candidates, with the shortest time per step."""
    c = np.ascontiguousarray(candidates, dtype=np.int32)
    best = np.zeros(1, dtype=np.int32)
    _check(load().rod_autotune_steps(h, c.ctypes.data, int(c.size), int(min_steps), best.ctypes.data,
                                     _stream(stream)), "rod_autotune_steps")
    return int(best[0])


def rod_get_plan(h, out):
    _check(load().rod_get_plan(h, _ptr(out)), "rod_get_plan")


def rod_set_graph_mode(h, mode):
    _check(load().rod_set_graph_mode(h, int(mode)), "rod_set_graph_mode")


def rod_mailbox_enable(h, period, log_capacity=65536):
    _check(load().rod_mailbox_enable(h, int(period), int(log_capacity)), "rod_mailbox_enable")


def rod_mailbox_write(h, drive):
    d = np.ascontiguousarray(drive, dtype=np.float32)
    _check(load().rod_mailbox_write(h, d.ctypes.data), "rod_mailbox_write")


def rod_mailbox_read(h, n_rods):
    """[n_rods, 2] records: dict arrays seq, step (int) and pos, vel ([n_rods, 2, 3] float32)."""
    raw = np.zeros((n_rods, 2, 8), dtype=np.uint32)
    _check(load().rod_mailbox_read(h, raw.ctypes.data), "rod_mailbox_read")
    return {"seq": raw[..., 0].astype(np.int64), "step": raw[..., 1].astype(np.int64),
            "pos": raw[..., 2:5].view(np.float32), "vel": raw[..., 5:8].view(np.float32)}


def rod_mailbox_log(h, capacity=65536):
    out = np.zeros((capacity, 2), dtype=np.int32)
    n = ctypes.c_int()
    _check(load().rod_mailbox_log(h, out.ctypes.data, int(capacity), ctypes.byref(n)), "rod_mailbox_log")
    return out[:min(n.value, capacity)].copy(), n.value


def rod_mailbox_disable(h):
    _check(load().rod_mailbox_disable(h), "rod_mailbox_disable")


def rod_mailbox_positions_enable(h, enable=True):
    _check(load().rod_mailbox_positions_enable(h, 1 if enable else 0), "rod_mailbox_positions_enable")


def rod_mailbox_positions(h, rod, out):
    """Latest consistent position snapshot of rod `rod` into out ([N, 4] float32 host
    array; None: nothing is copied); returns the global step it was taken after (-1:
    none yet)."""
    step = ctypes.c_longlong(0)
    _check(load().rod_mailbox_positions(h, int(rod), None if out is None else _ptr(out), ctypes.addressof(step)),
           "rod_mailbox_positions")
    return int(step.value)


def rod_mailbox_exchange(h, drive, rod, target_step, out, timeout_us=1_000_000):
    """One haptic tick: writes drive (None: no write), waits until rod `rod`'s snapshot of a
    step >= target_step is published, copies it into out ([N, 4] float32 host array) and
    returns its step."""
    d = None if drive is None else np.ascontiguousarray(drive, dtype=np.float32)
    step = ctypes.c_longlong(0)
    _check(load().rod_mailbox_exchange(h, None if d is None else d.ctypes.data, int(rod), int(target_step), _ptr(out),
                                       int(timeout_us), ctypes.addressof(step)), "rod_mailbox_exchange")
    return int(step.value)


def rod_mailbox_tick(h, rod, target_step, next_drive, out, timeout_us=1_000_000):
    """One closed lock-step tick: waits until rod `rod`'s snapshot of a step >= target_step
    is published, writes next_drive at once (None: no write), then copies the snapshot
    into out ([N, 4] float32 host array; None: no copy) and returns its step."""
    d = None if next_drive is None else np.ascontiguousarray(next_drive, dtype=np.float32)
    step = ctypes.c_longlong(0)
    _check(load().rod_mailbox_tick(h, int(rod), int(target_step), None if d is None else d.ctypes.data,
                                   None if out is None else _ptr(out), int(timeout_us), ctypes.addressof(step)),
           "rod_mailbox_tick")
    return int(step.value)


def rod_mailbox_lockstep(h, enable=True, timeout_us=1_000_000):
    _check(load().rod_mailbox_lockstep(h, 1 if enable else 0, int(timeout_us)), "rod_mailbox_lockstep")


def rod_mailbox_status(h) -> int:
    out = np.zeros(1, dtype=np.uint32)
    _check(load().rod_mailbox_status(h, out.ctypes.data), "rod_mailbox_status")
    return int(out[0])


def rod_steps_done(h) -> int:
    return int(load().rod_steps_done(h))


def rod_last_launch_count(h) -> int:
    return int(load().rod_last_launch_count(h))


def rod_destroy(h):
    load().rod_destroy(h)


def rod_rollout(h, n_steps, ckpt_every, pos_traj=None, stream=None):
    _check(load().rod_rollout(h, int(n_steps), int(ckpt_every), _ptr(pos_traj), _stream(stream)), "rod_rollout")


def rod_adjoint(h, dL_dpos_traj=None, dL_dK=None, dL_duhat=None, dL_dvel0=None, dL_dpos0=None, dL_dquat0=None,
                dL_domega0=None, stream=None):
    _check(load().rod_adjoint(h, _ptr(dL_dpos_traj), _ptr(dL_dK), _ptr(dL_duhat), _ptr(dL_dvel0), _ptr(dL_dpos0),
                              _ptr(dL_dquat0), _ptr(dL_domega0), _stream(stream)), "rod_adjoint")


def rod_adjoint_info(h) -> dict:
    """How the last rod_adjoint ran its largest launch (mode, record buffers and layout,
    threads, blocks per SM, blocks, SMs)."""
    out = np.zeros(7, dtype=np.int32)
    _check(load().rod_adjoint_info(h, out.ctypes.data), "rod_adjoint_info")
    per_sm, blocks, sms = int(out[2]), int(out[3]), int(out[4])
    return {"mode": "record" if out[0] else "recompute", "record_buffers": int(out[0]),
            "compact_records": bool(out[5]), "pipelined": bool(out[6]), "threads_per_block": int(out[1]),
            "blocks_per_sm": per_sm, "blocks": blocks, "sms": sms,
            "waves": -(-blocks // (per_sm * sms)) if per_sm * sms > 0 else None}


def rod_barrier_floor(scope, threads=128, cluster=1, n_iters=100000, stream=None) -> float:
    """ns per empty barrier: scope 0 block, 1 warp, 2 cluster, 3 cooperative grid."""
    ns = ctypes.c_double()
    _check(load().rod_barrier_floor(int(scope), int(threads), int(cluster), int(n_iters), ctypes.byref(ns),
                                    _stream(stream)), "rod_barrier_floor")
    return ns.value


def rod_device_info() -> dict:
    """Number of SMs and resident threads per SM of the current device."""
    n, t = ctypes.c_int(), ctypes.c_int()
    _check(load().rod_device_info(ctypes.byref(n), ctypes.byref(t)), "rod_device_info")
    return {"n_sms": n.value, "max_threads_per_sm": t.value}


def rod_fp32_peak(packed=False, blocks_per_sm=4, threads=256, n_iters=20000, stream=None) -> float:
    """Measured FP32 FMA throughput of the device in TFLOP/s (packed: float2 lanes)."""
    tf = ctypes.c_double()
    _check(load().rod_fp32_peak(int(bool(packed)), int(blocks_per_sm), int(threads), int(n_iters),
                                ctypes.byref(tf), _stream(stream)), "rod_fp32_peak")
    return tf.value


def rod_adjoint_noalloc(params, pos, quat, rest_quat=None, vel=None, omega=None, stiff_mul=None, drive=None,
                        n_steps=1, ckpt_every=1, dL_dpos_traj=None, pos_traj=None, dL_dK=None, dL_duhat=None,
                        dL_dvel0=None, dL_dpos0=None, stream=None):
    """Rollout and reverse pass of one rod with no device allocation (all pointers are
    caller-owned device buffers; intermediates live in the library's static array)."""
    _check(load().rod_adjoint_noalloc(ctypes.byref(params), _ptr(pos), _ptr(quat), _ptr(rest_quat), _ptr(vel),
                                      _ptr(omega), _ptr(stiff_mul), _ptr(drive), int(n_steps), int(ckpt_every),
                                      _ptr(dL_dpos_traj), _ptr(pos_traj), _ptr(dL_dK), _ptr(dL_duhat),
                                      _ptr(dL_dvel0), _ptr(dL_dpos0), _stream(stream)), "rod_adjoint_noalloc")


# ------------------------------------------------------------------ convenience


def params_of(rod) -> RodParams:
    p = RodParams()
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


def _cat(arrs, cols):
    return np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float32).reshape(-1, cols) for a in arrs]))


class RodBatch:
    """A handle over a list of rod descriptions (objects with the RodSpec attributes)."""

    def __init__(self, rods, stream=None):
        self.rods = list(rods)
        self.n_nodes = np.array([r.n_nodes for r in self.rods], dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.n_nodes)])
        self.n_rods = len(self.rods)
        self.n_elem = int(self.offsets[-1])
        pos = _cat([r.pos for r in self.rods], 3)
        quat = _cat([r.quat for r in self.rods], 4)
        rest = _cat([r.rest_quat for r in self.rods], 4) if all(r.rest_quat is not None for r in self.rods) else None
        vel = _cat([r.vel for r in self.rods], 3) if all(r.vel is not None for r in self.rods) else None
        om = _cat([r.omega for r in self.rods], 3) if all(r.omega is not None for r in self.rods) else None
        mul = None
        if any(r.stiff_mul is not None for r in self.rods):
            mul = _cat([r.stiff_mul if r.stiff_mul is not None else np.ones((r.n_nodes - 2, 3)) for r in self.rods],
                       3)
        self.handle = rod_create([params_of(r) for r in self.rods], pos, quat, rest, vel, om, mul, stream)

    def close(self):
        if self.handle is not None:
            rod_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_steps, drive=None, stream=None):
        rod_step(self.handle, n_steps, drive, stream)

    def set_input(self, drive, stream=None):
        d = drive
        if isinstance(drive, np.ndarray):
            d = np.ascontiguousarray(drive, dtype=np.float32).reshape(self.n_rods, 8)
        rod_set_input(self.handle, d, stream)

    def state_numpy(self) -> dict:
        """Synchronous copy of the whole state into host float32 arrays [E, 4]."""
        import torch

        out = {k: np.zeros((self.n_elem, 4), dtype=np.float32) for k in ("pos4", "quat4", "vel4", "omega4")}
        rod_get_state(self.handle, out["pos4"], out["quat4"], out["vel4"], out["omega4"])
        if torch.cuda.is_available():
            torch.cuda.current_stream().synchronize()
        return out

    def rod_state(self, st: dict, r: int) -> dict:
        """Per-rod views (pos N x 3, quat (N-1) x 4, vel N x 3, omega (N-1) x 3), float64 copies."""
        a, b = int(self.offsets[r]), int(self.offsets[r + 1])
        return {
            "pos": st["pos4"][a:b, :3].astype(np.float64),
            "quat": st["quat4"][a:b - 1].astype(np.float64),
            "vel": st["vel4"][a:b, :3].astype(np.float64),
            "omega": st["omega4"][a:b - 1, :3].astype(np.float64),
        }

    def set_rod_states(self, states: list):
        """Overwrite every rod's state from per-rod dicts in the rod_state layout (host, synchronous)."""
        import torch

        buf = {k: np.zeros((self.n_elem, 4), dtype=np.float32) for k in ("pos4", "quat4", "vel4", "omega4")}
        buf["quat4"][:, 3] = 1.0
        for r, s in enumerate(states):
            a, b = int(self.offsets[r]), int(self.offsets[r + 1])
            buf["pos4"][a:b, :3] = s["pos"]
            buf["vel4"][a:b, :3] = s["vel"]
            buf["quat4"][a:b - 1] = s["quat"]
            buf["omega4"][a:b - 1, :3] = s["omega"]
        rod_set_state(self.handle, buf["pos4"], buf["quat4"], buf["vel4"], buf["omega4"])
        if torch.cuda.is_available():
            torch.cuda.current_stream().synchronize()

    def derived(self) -> np.ndarray:
        out = np.zeros((self.n_rods, 16), dtype=np.float64)
        rod_get_derived(self.handle, out, None)
        return out

    def per_joint(self) -> np.ndarray:
        out = np.zeros((self.n_elem, 8), dtype=np.float32)
        rod_get_derived(self.handle, None, out)
        return out

    def diagnostics(self):
        out = np.zeros((self.n_rods, 4), dtype=np.float64)
        rc = rod_diagnostics(self.handle, out)
        return rc, out

    def plan(self) -> np.ndarray:
        """[n_rods, 3] (elements per thread, threads per block, blocks per rod: 0 = one block,
        C >= 2 a cluster of C blocks, -C a cooperative grid of C blocks)."""
        out = np.zeros((self.n_rods, 3), dtype=np.int32)
        rod_get_plan(self.handle, out)
        return out

    def set_plan_cluster(self, ept, nt, cluster):
        rod_set_plan_cluster(self.handle, ept, nt, cluster)

    def set_plan_grid(self, ept, nt, blocks):
        """Spread every rod it can hold over `blocks` blocks of a cooperative grid."""
        rod_set_plan_grid(self.handle, ept, nt, blocks)

    def bind(self, outer, inner, mode):
        rod_bind(self.handle, outer, inner, mode)

    def set_tube(self, rod, tube, enable=True):
        """Analytic vessel (cx, cy, cz, Rc, Rt, mu) for rod `rod`; enable=False removes it."""
        rod_set_tube(self.handle, rod, tube, enable)

    def set_self_collision(self, rod, mu, enable=True):
        rod_set_self_collision(self.handle, rod, mu, enable)

    def self_collision_stats(self, rod) -> dict:
        return rod_self_collision_stats(self.handle, rod)

    def set_adjoint_record_budget(self, n_bytes: int):
        rod_set_adjoint_record_budget(self.handle, n_bytes)

    def set_adjoint_pipeline(self, enable: bool):
        rod_set_adjoint_pipeline(self.handle, enable)

    def set_launch_overlap(self, enable: bool):
        rod_set_launch_overlap(self.handle, 1 if enable else 0)

    def set_plan(self, ept, nt):
        rod_set_plan(self.handle, ept, nt)

    def autotune(self, n_steps, stream=None):
        rod_autotune(self.handle, n_steps, stream)

    def autotune_steps(self, candidates, min_steps, stream=None) -> int:
        return rod_autotune_steps(self.handle, candidates, min_steps, stream)

    def set_graph_mode(self, mode):
        rod_set_graph_mode(self.handle, mode)

    def last_launch_count(self) -> int:
        return rod_last_launch_count(self.handle)

    def rollout(self, n_steps, ckpt_every, record=True, stream=None):
        """Recorded forward rollout; returns the position trajectory (torch, device,
        [n_steps, n_elem, 4]) or None."""
        import torch

        traj = torch.empty((n_steps, self.n_elem, 4), dtype=torch.float32, device="cuda") if record else None
        rod_rollout(self.handle, n_steps, ckpt_every, traj, stream)
        return traj

    def adjoint(self, dL_dpos_traj, stream=None) -> dict:
        """Gradients of the loss through the last rollout (torch device tensors [n_elem, 4])."""
        import torch

        out = {k: torch.zeros((self.n_elem, 4), dtype=torch.float32, device="cuda")
               for k in ("K", "uhat", "vel0", "pos0", "quat0", "omega0")}
        g = None if dL_dpos_traj is None else dL_dpos_traj.contiguous()
        rod_adjoint(self.handle, g, out["K"], out["uhat"], out["vel0"], out["pos0"], out["quat0"], out["omega0"],
                    stream)
        return out
