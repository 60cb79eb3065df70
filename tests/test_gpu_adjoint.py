"""The CUDA adjoint (reverse-mode gradient through the rollout, checkpoint-and-recompute)
against the FP64 oracle: exact forward-mode directional derivatives (dual numbers) and
FP64 central finite differences, on seeded directions over the per-joint stiffness,
intrinsic Darboux vectors, initial velocities and initial positions.

Loss: L = sum_t |r_tip(t) - target(t)|^2 over the rollout.  Bar (relative error of the
gradient <= 1e-3), checked two ways on the seeded directions d_k:
  * vector: RMS_k(gpu_k - ref_k) / RMS_k(ref_k) <= 1e-3 (for standard-normal directions
    this estimates |g_gpu - g_ref| / |g_ref| of the scaled gradient);
  * per direction: |gpu_k - ref_k| <= 1e-3 max(|ref_k|, 0.1 RMS_k(ref)), so a direction
    nearly orthogonal to the gradient is held to an absolute error of 1e-4 |g| instead of
    a relative error of a value near zero.
"""
import numpy as np
import pytest

import oracle
from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL_TOL = 1e-3


@pytest.fixture(scope="module")
def corde(cuda):
    from paper_2509_04277_gb300 import build, corde as C

    build.build()
    C.load()
    return C


def _gpu_grad(corde, torch, rods, n_steps, ckpt, targets, drive=None):
    b = corde.RodBatch(rods)
    if drive is not None:
        b.set_input(drive)
    traj = b.rollout(n_steps, ckpt)
    g = torch.zeros_like(traj)
    loss = []
    for r, rod in enumerate(rods):
        tip = int(b.offsets[r + 1]) - 1
        tgt = torch.as_tensor(targets[r], dtype=torch.float32, device="cuda")
        diff = traj[:, tip, :3] - tgt
        g[:, tip, :3] = 2.0 * diff
        loss.append(float((diff.double() ** 2).sum()))
    grads = b.adjoint(g)
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    pj = b.per_joint().astype(np.float64)
    b.close()
    return out, loss, pj, b.offsets


def _frame_tangent(quat, dtheta):
    """Tangents q (x) (0, dtheta / 2) of unit quaternions (xyzw rows): the first-order
    change of each frame under a small body-frame rotation dtheta (on the unit sphere)."""
    qv, qw = quat[:, :3], quat[:, 3:4]
    v = 0.5 * dtheta
    out = np.zeros_like(quat)
    out[:, :3] = qw * v + np.cross(qv, v)
    out[:, 3] = -(qv * v).sum(axis=1)
    return out


def _directions(rod, K, seed, n_dirs, frames=True):
    """Seeded directions over the per-joint stiffness and intrinsic Darboux vectors and the
    initial positions, velocities, frames (tangents of body-frame rotations) and body
    angular velocities."""
    g = np.random.default_rng(seed)
    J, N = K.shape[0], rod.n_nodes
    dirs = []
    for _ in range(n_dirs):
        d = {
            "K": K * g.standard_normal(K.shape),
            "uhat": g.standard_normal((J, 3)) * 0.5,
            "vel": g.standard_normal((N, 3)) * 1e-2,
            "pos": g.standard_normal((N, 3)) * 1e-4,
            "quat": np.zeros((N - 1, 4)),
            "omega": np.zeros((N - 1, 3)),
        }
        if frames:
            d["quat"] = _frame_tangent(np.asarray(rod.quat, np.float64), g.standard_normal((N - 1, 3)) * 1e-3)
            d["omega"] = g.standard_normal((N - 1, 3)) * 0.1
        dirs.append(d)
    return dirs


def _gpu_directional(grads, off, rod, d):
    n = rod.n_nodes
    J = n - 2
    sl = slice(off, off + n)
    fr = slice(off, off + n - 1)
    return float((grads["K"][off:off + J, :3] * d["K"]).sum() + (grads["uhat"][off:off + J, :3] * d["uhat"]).sum()
                 + (grads["vel0"][sl, :3] * d["vel"]).sum() + (grads["pos0"][sl, :3] * d["pos"]).sum()
                 + (grads["quat0"][fr, :4] * d["quat"]).sum() + (grads["omega0"][fr, :3] * d["omega"]).sum())


def _oracle_loss_and_jvp(rod, K, uhat, target, n_steps, d, drive_row=None):
    st = oracle.state_of(rod)
    table = None if drive_row is None else np.tile(np.asarray(drive_row, np.float64), (n_steps, 1))
    traj, dtraj = oracle.rollout_jvp(rod, st, n_steps, drive_table=table, K=K, uhat=uhat, d_pos=d["pos"],
                                     d_vel=d["vel"], d_K=d["K"], d_uhat=d["uhat"], d_quat=d["quat"],
                                     d_omega=d["omega"])
    diff = traj[:, -1, :] - target
    return float((diff ** 2).sum()), float((2 * diff * dtraj[:, -1, :]).sum())


def _oracle_fd(rod, K, uhat, target, n_steps, d, h=1e-6, drive_row=None):
    table = None if drive_row is None else np.tile(np.asarray(drive_row, np.float64), (n_steps, 1))

    def L(sg):
        st = oracle.state_of(rod)
        st["pos"] = st["pos"] + sg * h * d["pos"]
        st["vel"] = st["vel"] + sg * h * d["vel"]
        st["quat"] = st["quat"] + sg * h * d["quat"]
        st["omega"] = st["omega"] + sg * h * d["omega"]
        traj, _ = oracle.rollout(rod, st, n_steps, drive_table=table, K=K + sg * h * d["K"],
                                 uhat=uhat + sg * h * d["uhat"])
        return float(((traj[:, -1, :] - target) ** 2).sum())

    return (L(1) - L(-1)) / (2 * h)


def _check(gpu_vals, ref_vals, what):
    gpu_vals = np.asarray(gpu_vals)
    ref_vals = np.asarray(ref_vals)
    rms = np.sqrt(np.mean(ref_vals ** 2))
    vec = np.sqrt(np.mean((gpu_vals - ref_vals) ** 2)) / rms
    assert vec <= REL_TOL, f"{what}: vector relative error {vec:.3e}"
    rel = np.abs(gpu_vals - ref_vals) / np.maximum(np.abs(ref_vals), 0.1 * rms)
    assert rel.max() <= REL_TOL, f"{what}: max relative error {rel.max():.3e}\ngpu={gpu_vals}\nref={ref_vals}"
    return vec, rel.max()


def _material_from_gpu(pj, off, n):
    J = n - 2
    return pj[off:off + J, 0:3].copy(), pj[off:off + J, 4:7].copy()


def test_adjoint_small_rod_ragged_segments(corde):
    """20-node rod, 30 steps, checkpoints every 7 steps (ragged last segment), driven base."""
    import torch

    rod = W.adjoint_rod(20, seed=51)
    n_steps = 30
    target = W.tip_target(52, n_steps, rod.dt, rod.pos[-1] + np.array([0.0, 0.0, 1e-3]))
    drive = np.array([[0.01, 0.0, -0.005, 0, 0.0, 0.0, 2.0, 0]], np.float32)
    grads, loss, pj, offs = _gpu_grad(corde, torch, [rod], n_steps, 7, [target], drive=drive)
    K, uhat = _material_from_gpu(pj, 0, rod.n_nodes)
    gv, rv = [], []
    for d in _directions(rod, K, 53, 8):
        L, dL = _oracle_loss_and_jvp(rod, K, uhat, target, n_steps, d, drive_row=drive[0])
        gv.append(_gpu_directional(grads, 0, rod, d))
        rv.append(dL)
    assert abs(loss[0] / L - 1) < 1e-3
    _check(gv, rv, "small rod vs oracle JVP")


def test_adjoint_extensible_rod(corde):
    import torch

    rod = W.extensible_pendulum(24, seed=54)
    n_steps = 40
    target = W.tip_target(55, n_steps, rod.dt, rod.pos[-1])
    grads, _, pj, _ = _gpu_grad(corde, torch, [rod], n_steps, 10, [target])
    K, uhat = _material_from_gpu(pj, 0, rod.n_nodes)
    gv, rv = [], []
    for d in _directions(rod, K, 56, 6):
        _, dL = _oracle_loss_and_jvp(rod, K, uhat, target, n_steps, d)
        gv.append(_gpu_directional(grads, 0, rod, d))
        rv.append(dL)
    _check(gv, rv, "extensible rod vs oracle JVP")


def test_adjoint_256_element_rod_200_steps(corde):
    """The adjoint workload: 256-element inextensible rod, 200 steps at dt = 1e-4 s,
    checkpoints every 20 steps; 32 seeded directions against the oracle's exact JVP and
    against FP64 central differences (h = 1e-6 on the scaled direction)."""
    import torch

    rod = W.adjoint_rod(256, seed=5)
    n_steps = 200
    target = W.tip_target(5, n_steps, rod.dt, rod.pos[-1] + np.array([0.0, 2e-3, -1e-3]))
    grads, loss, pj, _ = _gpu_grad(corde, torch, [rod], n_steps, 20, [target])
    K, uhat = _material_from_gpu(pj, 0, rod.n_nodes)
    gv, jv, fv = [], [], []
    for d in _directions(rod, K, 57, 32):
        _, dL = _oracle_loss_and_jvp(rod, K, uhat, target, n_steps, d)
        gv.append(_gpu_directional(grads, 0, rod, d))
        jv.append(dL)
        fv.append(_oracle_fd(rod, K, uhat, target, n_steps, d))
    _check(jv, fv, "oracle JVP vs oracle central FD")
    _check(gv, jv, "GPU adjoint vs oracle JVP")
    _check(gv, fv, "GPU adjoint vs oracle central FD")


def _frame_only(d):
    out = {k: np.zeros_like(v) for k, v in d.items()}
    out["quat"], out["omega"] = d["quat"], d["omega"]
    return out


@pytest.mark.parametrize("spin", [False, True])
def test_adjoint_initial_frames_and_angular_velocities(corde, spin):
    """dL/dq0 and dL/domega0 alone: directions over the initial frames (tangents of
    body-frame rotations) and body angular velocities only, on a 64-node rod over 100
    steps with checkpoints every 20, at rest and with spinning frames (the gyroscopic
    term active), against the oracle's exact JVP and FP64 central differences."""
    import torch

    rod = W.adjoint_rod(64, seed=71)
    if spin:
        rod.omega = np.random.default_rng(72).standard_normal((63, 3)) * 0.5
    n_steps = 100
    target = W.tip_target(73, n_steps, rod.dt, rod.pos[-1] + np.array([0.0, 1e-3, 0.0]))
    grads, _, pj, _ = _gpu_grad(corde, torch, [rod], n_steps, 20, [target])
    assert np.abs(grads["omega0"][0, :3]).max() == 0.0  # frame 0 is kinematic: its omega comes from the drive
    K, uhat = _material_from_gpu(pj, 0, rod.n_nodes)
    gv, jv, fv = [], [], []
    for d in _directions(rod, K, 74 + spin, 12):
        d = _frame_only(d)
        _, dL = _oracle_loss_and_jvp(rod, K, uhat, target, n_steps, d)
        gv.append(_gpu_directional(grads, 0, rod, d))
        jv.append(dL)
        fv.append(_oracle_fd(rod, K, uhat, target, n_steps, d))
    _check(jv, fv, "oracle JVP vs oracle central FD (frames)")
    _check(gv, jv, "GPU adjoint vs oracle JVP (frames)")
    _check(gv, fv, "GPU adjoint vs oracle central FD (frames)")


def test_adjoint_batched_256_rods_sampled(corde):
    """The adjoint batched over 256 rods in one launch; 6 sampled rods checked."""
    import torch

    rods = [W.adjoint_rod(256, seed=1000 + k) for k in range(256)]
    n_steps = 60
    targets = [W.tip_target(2000 + k, n_steps, r.dt, r.pos[-1]) for k, r in enumerate(rods)]
    grads, _, pj, offs = _gpu_grad(corde, torch, rods, n_steps, 20, targets)
    for r in (0, 17, 101, 128, 200, 255):
        rod = rods[r]
        off = int(offs[r])
        K, uhat = _material_from_gpu(pj, off, rod.n_nodes)
        gv, rv = [], []
        for d in _directions(rod, K, 3000 + r, 4):
            _, dL = _oracle_loss_and_jvp(rod, K, uhat, targets[r], n_steps, d)
            gv.append(_gpu_directional(grads, off, rod, d))
            rv.append(dL)
        _check(gv, rv, f"batched rod {r}")


def test_autograd_function_matches_adjoint(corde):
    import torch

    from paper_2509_04277_gb300.autograd import RodRollout

    rod = W.adjoint_rod(64, seed=58)
    n_steps = 50
    b = corde.RodBatch([rod])
    pj = torch.as_tensor(b.per_joint(), device="cuda")
    st = b.state_numpy()
    K = pj[:, 0:4].clone().requires_grad_(True)
    uhat = pj[:, 4:8].clone().requires_grad_(True)
    vel0 = torch.as_tensor(st["vel4"], device="cuda").requires_grad_(True)
    pos0 = torch.as_tensor(st["pos4"], device="cuda").requires_grad_(True)
    quat0 = torch.as_tensor(st["quat4"], device="cuda").requires_grad_(True)
    omega0 = torch.as_tensor(st["omega4"], device="cuda").requires_grad_(True)
    traj = RodRollout.apply(b, n_steps, 10, K, uhat, vel0, pos0, quat0, omega0)
    target = torch.as_tensor(W.tip_target(59, n_steps, rod.dt, rod.pos[-1]), dtype=torch.float32, device="cuda")
    loss = ((traj[:, -1, :3] - target) ** 2).sum()
    loss.backward()
    assert K.grad is not None and torch.isfinite(K.grad).all()
    Kn = pj[:rod.n_nodes - 2, 0:3].double().cpu().numpy()
    un = pj[:rod.n_nodes - 2, 4:7].double().cpu().numpy()
    d = _directions(rod, Kn, 60, 1)[0]
    _, dL = _oracle_loss_and_jvp(rod, Kn, un, target.double().cpu().numpy(), n_steps, d)
    g = {"K": K.grad.double().cpu().numpy(), "uhat": uhat.grad.double().cpu().numpy(),
         "vel0": vel0.grad.double().cpu().numpy(), "pos0": pos0.grad.double().cpu().numpy(),
         "quat0": quat0.grad.double().cpu().numpy(), "omega0": omega0.grad.double().cpu().numpy()}
    assert np.abs(g["quat0"]).max() > 0
    _check([_gpu_directional(g, 0, rod, d)], [dL], "autograd.Function")
    b.close()


def test_adjoint_requires_rollout_and_rejects_long_rods(corde):
    rod = W.guidewire(600, seed=61)
    b = corde.RodBatch([rod])
    with pytest.raises(corde.CordeError):
        corde.rod_adjoint(b.handle)
    b.rollout(5, 5, record=False)
    with pytest.raises(corde.CordeError) as e:
        corde.rod_adjoint(b.handle)
    assert e.value.code == corde.CORDE_ERR_UNSUPPORTED
    b.close()


def test_record_and_recompute_modes_give_identical_gradients(corde):
    """The reverse pass either keeps each segment's sweep velocities from one forward pass
    (record mode, the default when the scratch fits) or runs every step forward again
    (recompute mode, budget 0).  Record mode keeps every half-sweep's input (full layout)
    or, for launches with more rods than SMs and where only that fits, the first even and
    every odd one (compact layout: the reverse pass rebuilds the others, bit for bit).  It
    streams a step's records into two shared buffers, or into one when two do not fit the
    block (a 300-node rod on 256 threads with 16 iterations) or when one lets more blocks
    share an SM and so saves a wave (8 more rods of 150 nodes with 20 iterations than the
    GPU has SMs: one block per SM with two buffers, two with one; with 10 iterations two
    blocks fit with two buffers).  Several rods of ragged lengths and different iteration
    counts, and a segment length that leaves a short last segment."""
    import dataclasses

    import torch

    rods = [dataclasses.replace(W.adjoint_rod(n, seed=970 + n), n_iters=it)
            for n, it in ((7, 3), (33, 10), (100, 6), (256, 10))]
    n_sms = corde.rod_device_info()["n_sms"]
    many = [dataclasses.replace(W.adjoint_rod(150, seed=1200 + k), n_iters=20) for k in range(n_sms + 8)]
    many10 = [W.adjoint_rod(150, seed=1400 + k) for k in range(n_sms + 8)]
    groups = (rods, [dataclasses.replace(W.adjoint_rod(300, seed=975), n_iters=16)], many, many10)
    n_steps, ckpt = 47, 10
    out, modes = {}, {}
    for budget in (1 << 30, 0):
        for gi, group in enumerate(groups):
            b = corde.RodBatch(group)
            b.set_adjoint_record_budget(budget)
            traj = b.rollout(n_steps, ckpt)
            g = torch.zeros_like(traj)
            g[:, :, :3] = 1e-2 * torch.sin(traj[:, :, :3] * 37.0)
            grads = b.adjoint(g)
            out[budget, gi] = {k: v.cpu().numpy() for k, v in grads.items()}
            modes[budget, gi] = corde.rod_adjoint_info(b.handle)
            b.close()
    # record mode: two buffers where they fit and cost no wave, else one; compact records
    # for more rods than SMs or where only they fit
    rec = [modes[1 << 30, gi] for gi in range(len(groups))]
    assert [m["record_buffers"] for m in rec] == [2, 1, 1, 2], modes
    assert [m["compact_records"] for m in rec] == [False, True, True, True], modes
    # few rods with the full layout and two buffers: pipelined over two SMs per rod
    assert [m["pipelined"] for m in rec] == [True, False, False, False], modes
    assert all(m["blocks_per_sm"] == 2 and m["waves"] == 1 for m in rec[2:]), modes
    assert all(modes[0, gi]["mode"] == "recompute" for gi in range(len(groups))), modes
    for gi in range(len(groups)):
        a, c = out[1 << 30, gi], out[0, gi]
        for key in a:
            assert np.isfinite(a[key]).all(), key
            np.testing.assert_array_equal(a[key], c[key], err_msg=f"group {gi}: {key}")
    h = corde.RodBatch(rods[:1])
    with pytest.raises(corde.CordeError):
        corde.rod_set_adjoint_record_budget(h.handle, -1)
    h.close()


def test_pipelined_reverse_matches_unpipelined(corde):
    """With few rods each rod's reverse pass runs on a cluster of two blocks: one records
    the checkpoint segments, the other reverses them a segment later (scratch in two sets
    by segment parity, one cluster barrier per segment).  Its gradients equal the one-block
    record mode's bit for bit: rods of three lengths and iteration counts, a short last
    segment, one and five segments."""
    import dataclasses

    import torch

    rods = [dataclasses.replace(W.adjoint_rod(n, seed=1500 + n), n_iters=it) for n, it in ((64, 4), (200, 10), (256, 7))]
    for n_steps, ckpt in ((47, 10), (12, 20)):
        out, info = [], []
        for pipe in (True, False):
            b = corde.RodBatch(rods)
            b.set_adjoint_pipeline(pipe)
            traj = b.rollout(n_steps, ckpt)
            g = torch.zeros_like(traj)
            g[:, :, :3] = 1e-2 * torch.cos(traj[:, :, :3] * 23.0)
            grads = b.adjoint(g)
            out.append({k: v.cpu().numpy() for k, v in grads.items()})
            info.append(corde.rod_adjoint_info(b.handle))
            b.close()
        assert info[0]["pipelined"] and not info[1]["pipelined"], info
        for key in out[0]:
            assert np.isfinite(out[0][key]).all(), key
            np.testing.assert_array_equal(out[0][key], out[1][key], err_msg=f"{n_steps} steps: {key}")
