"""Self-collision (bounding-sphere broad phase, sphere-sphere narrow phase, Jacobi contact
impulses with Coulomb friction inside the constraint iterations) on the GPU against the
oracle.

Tolerances as for the plain rod: one step from a shared state |dr| <= 1e-5 L, free
running |dr| <= 1e-4 L, quaternion components 1e-4.  The response is continuous in the
predicted gap and in the set of touching pairs (penetration-weighted mean), so FP32 and
FP64 disagreeing on a pair at the contact distance moves the result by rounding only.
"""
import numpy as np
import pytest

import oracle
from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
ROLL_TOL = 1e-4
QUAT_TOL = 1e-4
MU = 0.1
PULL = np.array([0.05, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0])  # base pulled at 5 cm/s, twisted at 2 rad/s


@pytest.fixture(scope="module")
def corde(cuda):
    from paper_2509_04277_gb300 import build, corde as C

    build.build()
    C.load()
    return C


def _cmp(rod, gpu, ref, tol):
    dr = np.abs(gpu["pos"] - ref["pos"]).max() / rod.length
    dq = np.abs(gpu["quat"] - ref["quat"]).max()
    assert np.isfinite(gpu["pos"]).all()
    assert dr <= tol, f"position error {dr:.3e} L"
    assert dq <= QUAT_TOL, f"quaternion error {dq:.3e}"


def _drive(torch, rows):
    return torch.as_tensor(np.asarray(rows, np.float32).reshape(-1, 8), device="cuda").contiguous()


def _drive64(row):
    return np.asarray(row, np.float32).astype(np.float64)


def _touching(rod, pos):
    n = len(pos)
    m = max(2, int(np.floor(2 * rod.radius / (rod.length / (n - 1)))) + 1)
    idx = np.arange(n)
    far = np.abs(idx[:, None] - idx[None, :]) >= m
    d = np.linalg.norm(pos[:, None] - pos[None, :], axis=2)
    return int(np.sum((d < 2 * rod.radius * (1 + 1e-3)) & far) // 2), float(d[far].min() / (2 * rod.radius))


@pytest.mark.parametrize("n", [64, 130, 512, 1000])
def test_self_one_step_parity(corde, n):
    """The knot after 40 steps of settling (strands pressed together), then 3 single steps
    each restarted from the GPU state; plans from <2, 32> (warp-synchronous) to <4, 256> (1000 nodes)."""
    import torch

    rod = W.torus_knot(n, seed=700 + n)
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    d = _drive(torch, PULL)
    b.step(40, drive=d)
    for _ in range(3):
        st0 = b.rod_state(b.state_numpy(), 0)
        b.step(1, drive=d)
        ref = oracle.step_contact(rod, st0, self_mu=MU, n_steps=1, drive=_drive64(PULL))
        _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    touching, _ = _touching(rod, ref["pos"])
    assert touching > 0
    b.close()


def test_self_detection_matches_oracle(corde):
    """The candidate pairs the GPU found at the last detection of a launch are the oracle's
    pairs of the same positions (the broad phase drops none), on every step of launches
    of 1 to 20 steps: later steps test only the skin list of an earlier build (until a
    mass point has moved 1.5 radii since), and the set stays exact."""
    import torch

    rod = W.torus_knot(512, seed=710)
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    d = _drive(torch, PULL)
    b.step(30, drive=d)
    s0 = b.rod_state(b.state_numpy(), 0)
    filtered = 0
    for k in range(1, 21):
        # the positions at the start of the last step of a k-step launch: the end of a
        # (k - 1)-step launch from the same state (the same arithmetic, bit for bit)
        b.set_rod_states([s0])
        if k > 1:
            b.step(k - 1, drive=d)
        pos = b.rod_state(b.state_numpy(), 0)["pos"]
        b.set_rod_states([s0])
        b.step(k, drive=d)
        stats = b.self_collision_stats(0)
        cand, pairs = oracle.self_candidates(rod, pos)
        assert stats["candidate_pairs"] == pairs, (k, stats, pairs)
        assert stats["max_partners_above"] == max(int(np.sum(c > i)) for i, c in enumerate(cand)), k
        assert not stats["overflow"], (k, stats)
        assert stats["overlapping_pairs"] >= 0
        assert 0 <= stats["skin_builds"] <= k  # the list may come from the previous launch
        filtered += k - stats["skin_builds"]
    assert filtered > 100  # most steps ran on the skin list
    b.close()


def test_self_skin_list_kept_between_launches(corde):
    """The skin list and the positions it was built at outlive a launch: launches of one
    step mostly reuse the previous launch's list (every candidate set still exact, as
    test_self_detection_matches_oracle checks on every step), and a change of the rod's
    self-collision settings discards it (the next launch builds)."""
    import torch

    rod = W.torus_knot(512, seed=710)
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    d = _drive(torch, PULL)
    b.step(10, drive=d)
    builds = []
    for _ in range(20):
        b.step(1, drive=d)
        builds.append(b.self_collision_stats(0)["skin_builds"])
    assert sum(builds) < 10, builds  # most one-step launches reused the kept list
    b.set_self_collision(0, MU)      # new settings: the kept list is discarded
    b.step(1, drive=d)
    assert b.self_collision_stats(0)["skin_builds"] == 1
    pos = b.rod_state(b.state_numpy(), 0)["pos"]
    assert np.isfinite(pos).all()
    b.close()


def test_self_skin_overflow_falls_back_to_full_detection(corde):
    """A tight coil: within the grown reach of the skin list (6 r) some mass points have
    more than the list's 24 places of partners above them, within the plain 3 r at most
    four.  Every build overflows, so every step detects from scratch (overflow bit 3 and
    no other); the candidate pairs are still the oracle's, and each step matches the
    oracle's."""
    import torch

    rod = W.coil(130, seed=720)
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    d = _drive(torch, PULL)
    for _ in range(3):
        st0 = b.rod_state(b.state_numpy(), 0)
        b.step(1, drive=d)
        stats = b.self_collision_stats(0)
        assert stats["overflow"] == 8, stats
        cand, pairs = oracle.self_candidates(rod, st0["pos"])
        assert stats["candidate_pairs"] == pairs, (stats, pairs)
        assert stats["max_partners_above"] == max(int(np.sum(c > i)) for i, c in enumerate(cand))
        ref = oracle.step_contact(rod, st0, self_mu=MU, n_steps=1, drive=_drive64(PULL))
        _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    touching, _ = _touching(rod, ref["pos"])
    assert touching > 0
    b.close()


def test_self_free_running_512(corde):
    """The knot workload: 10 launches of 10 steps against 100 oracle steps; no two mass
    points of the GPU result closer than 2 r (to 1 %)."""
    import torch

    rod = W.torus_knot(512, seed=21)
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    d = _drive(torch, PULL)
    for _ in range(10):
        b.step(10, drive=d)
    ref = oracle.step_contact(rod, oracle.state_of(rod), self_mu=MU, n_steps=100, drive=_drive64(PULL))
    got = b.rod_state(b.state_numpy(), 0)
    _cmp(rod, got, ref, ROLL_TOL)
    _, closest = _touching(rod, got["pos"])
    assert closest > 0.99
    b.close()


def test_self_with_vessel_and_mixed_batch(corde):
    """One handle: a knot with self-collision, a knot with self-collision inside a vessel,
    a plain guidewire and a vessel guidewire, stepped through the CUDA graph."""
    knot_a = W.torus_knot(200, seed=720)
    knot_b = W.torus_knot(100, seed=721)
    plain = W.guidewire(300, seed=722)
    vg, tube = W.vessel_guidewire(256, seed=723)
    # a vessel around knot_b: the torus of its own ring, wide enough to hold both strands
    n_b = knot_b.n_nodes
    R_b = (n_b - 1) * knot_b.length / (n_b - 1) / (4 * np.pi)
    c_b = knot_b.pos.mean(axis=0)
    tube_b = np.array([c_b[0], c_b[1], c_b[2], R_b, 4 * knot_b.radius, 0.05])
    b = corde.RodBatch([knot_a, knot_b, plain, vg])
    b.set_graph_mode(1)
    b.set_self_collision(0, MU)
    b.set_self_collision(1, 0.0)
    b.set_tube(1, tube_b)
    b.set_tube(3, tube)
    for _ in range(3):
        b.step(7)
    assert b.last_launch_count() >= 2
    st = b.state_numpy()
    refs = [oracle.step_contact(knot_a, oracle.state_of(knot_a), self_mu=MU, n_steps=21),
            oracle.step_contact(knot_b, oracle.state_of(knot_b), tube=tube_b, self_mu=0.0, n_steps=21),
            oracle.step(plain, oracle.state_of(plain), 21),
            oracle.step_tube(vg, oracle.state_of(vg), tube, 21)]
    for r, (rod, ref) in enumerate(zip([knot_a, knot_b, plain, vg], refs)):
        _cmp(rod, b.rod_state(st, r), ref, ROLL_TOL)
    b.close()


def test_self_disable_restores_plain_step(corde):
    rod = W.torus_knot(128, seed=730)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    b.set_self_collision(0, MU)
    b.set_self_collision(0, MU, enable=False)
    assert tuple(a.plan()[0]) == tuple(b.plan()[0])
    a.step(20)
    b.step(20)
    sa, sb = a.state_numpy(), b.state_numpy()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])
    a.close()
    b.close()


def test_self_argument_errors(corde):
    knot = W.torus_knot(64, seed=740)
    b = corde.RodBatch([knot, W.guidewire(64, seed=741), W.extensible_pendulum(), W.guidewire(1100, seed=742)])
    with pytest.raises(corde.CordeError):
        b.set_self_collision(0, -0.1)
    with pytest.raises(corde.CordeError):
        b.set_self_collision(2, MU)  # extensible: no constraint iterations
    with pytest.raises(corde.CordeError):
        b.set_self_collision(3, MU)  # more than 1024 nodes
    with pytest.raises(corde.CordeError):
        b.set_self_collision(4, MU)
    b.set_self_collision(0, MU)
    with pytest.raises(corde.CordeError):
        b.bind(0, 1, 0)
    with pytest.raises(corde.CordeError):
        b.rollout(10, 5)
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_enable(b.handle, 10)
    b.close()
