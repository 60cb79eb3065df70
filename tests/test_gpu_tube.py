"""Contact with an analytic vessel (collision constraints with Coulomb friction, iterated
with the distance constraints) on the GPU against the oracle.

Tolerances as for the plain rod: one step from a shared state |dr| <= 1e-5 L, 100
free-running steps |dr| <= 1e-4 L, quaternion components 1e-4.  The contact response is
continuous at the wall (the velocity change and the friction cut both vanish as the
predicted offset reaches the allowed distance), so FP32 and FP64 taking a node in or out
of contact in different iterations moves the result by rounding only.
"""
import numpy as np
import pytest

import oracle
from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
ROLL_TOL = 1e-4
QUAT_TOL = 1e-4
INSERT = np.array([0.05, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0])  # push 5 cm/s along +x, twist 2 rad/s


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


def _offset(pos, tube):
    """Distance of each node from the vessel centreline."""
    rho = np.hypot(pos[:, 0] - tube[0], pos[:, 1] - tube[1])
    return np.hypot(rho - tube[3], pos[:, 2] - tube[2])


def _in_contact(rod, st, tube):
    return int(np.sum(_offset(st["pos"], tube) > (tube[4] - rod.radius) * (1 - 1e-3)))


@pytest.mark.parametrize("n", [33, 130, 512])
def test_tube_one_step_parity(corde, n):
    import torch

    rod, tube = W.vessel_guidewire(n, seed=600 + n, offset=0.99)
    b = corde.RodBatch([rod])
    b.set_tube(0, tube)
    d = _drive(torch, INSERT)
    b.step(30, drive=d)  # let the wire settle onto the wall
    for _ in range(3):
        st0 = b.rod_state(b.state_numpy(), 0)
        b.step(1, drive=d)
        ref = oracle.step_tube(rod, st0, tube, 1, drive=INSERT.astype(np.float32).astype(np.float64))
        _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    assert _in_contact(rod, b.rod_state(b.state_numpy(), 0), tube) > 0
    b.close()


def test_tube_free_running_512(corde):
    """The insertion workload: 10 launches of 10 steps, the base pushed along the vessel."""
    import torch

    rod, tube = W.vessel_guidewire(512, seed=11)
    b = corde.RodBatch([rod])
    b.set_tube(0, tube)
    d = _drive(torch, INSERT)
    for _ in range(10):
        b.step(10, drive=d)
    ref = oracle.step_tube(rod, oracle.state_of(rod), tube, 100, drive=INSERT.astype(np.float32).astype(np.float64))
    got = b.rod_state(b.state_numpy(), 0)
    _cmp(rod, got, ref, ROLL_TOL)
    # every node inside the vessel, up to FP32 rounding of metre-scale coordinates
    assert _offset(got["pos"], tube).max() <= tube[4] - rod.radius + 2e-6
    assert _in_contact(rod, got, tube) > 10
    b.close()


def test_tube_disabled_is_the_plain_step(corde):
    rod, tube = W.vessel_guidewire(200, seed=7)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    b.set_tube(0, tube)
    b.set_tube(0, tube, enable=False)
    a.step(30)
    b.step(30)
    sa, sb = a.state_numpy(), b.state_numpy()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])
    a.close()
    b.close()


def test_tube_mixed_batch_with_graph(corde):
    """Rods with and without a vessel in one handle, stepped through the CUDA graph."""
    rods, tubes = [], []
    for k, n in enumerate([64, 300, 511, 100]):
        rod, tube = W.vessel_guidewire(n, seed=620 + k, rc=0.3 + 0.1 * k, mu=0.05 * k)
        rods.append(rod)
        tubes.append(tube if k % 2 == 0 else None)
    b = corde.RodBatch(rods)
    b.set_graph_mode(1)
    for r, t in enumerate(tubes):
        if t is not None:
            b.set_tube(r, t)
    for _ in range(4):
        b.step(5)
    st = b.state_numpy()
    for r, (rod, t) in enumerate(zip(rods, tubes)):
        s0 = oracle.state_of(rod)
        ref = oracle.step_tube(rod, s0, t, 20) if t is not None else oracle.step(rod, s0, 20)
        _cmp(rod, b.rod_state(st, r), ref, ROLL_TOL)
    b.close()


def test_tube_long_rod_over_cluster(corde):
    """Contact in the cluster kernel: a 4096-node wire over a cluster of blocks."""
    import torch

    rod, tube = W.vessel_guidewire(4096, seed=640, offset=0.99)
    b = corde.RodBatch([rod])
    assert b.plan()[0][2] >= 2
    b.set_tube(0, tube)
    d = _drive(torch, INSERT)
    b.step(80, drive=d)  # the long wire reaches the wall after about 80 steps
    st0 = b.rod_state(b.state_numpy(), 0)
    b.step(1, drive=d)
    ref = oracle.step_tube(rod, st0, tube, 1, drive=INSERT.astype(np.float32).astype(np.float64))
    _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    assert _in_contact(rod, ref, tube) > 0
    b.close()


def test_tube_argument_errors(corde):
    rod, tube = W.vessel_guidewire(64, seed=650)
    b = corde.RodBatch([rod, W.guidewire(64, seed=651), W.extensible_pendulum()])
    bad = tube.copy()
    bad[4] = rod.radius * 0.5  # inner radius below the rod radius
    with pytest.raises(corde.CordeError):
        b.set_tube(0, bad)
    bad = tube.copy()
    bad[3] = 0.0
    with pytest.raises(corde.CordeError):
        b.set_tube(0, bad)
    with pytest.raises(corde.CordeError):
        b.set_tube(3, tube)
    with pytest.raises(corde.CordeError):
        b.set_tube(2, tube)  # extensible rod: no constraint iterations
    b.set_tube(0, tube)
    with pytest.raises(corde.CordeError):
        b.bind(0, 1, 0)
    b.close()
