"""Long rods spread over a thread-block cluster (distributed-shared-memory halo, cluster
barriers) against the oracle, and against the one-block path on the same rod."""
import numpy as np
import pytest

import oracle
from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
ROLL_TOL = 1e-4


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
    assert dq <= 1e-4, f"quaternion error {dq:.3e}"


@pytest.mark.parametrize("n", [2049, 3072, 4096])
def test_long_rod_default_cluster_plan(corde, n):
    import torch

    rod = W.guidewire(n, seed=500 + n)
    b = corde.RodBatch([rod])
    ept, nt, C = b.plan()[0]
    assert C >= 2 and ept * nt * C >= n
    drive = torch.as_tensor(np.array([[0.01, 0, 0, 0, 0, 0, 1.0, 0]], np.float32), device="cuda")
    for _ in range(2):
        st0 = b.rod_state(b.state_numpy(), 0)
        b.step(1, drive=drive)
        ref = oracle.step(rod, st0, 1, drive=drive.cpu().numpy()[0].astype(np.float64))
        _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    b.close()


@pytest.mark.parametrize("ept,nt,C", [(2, 256, 2), (2, 256, 4), (4, 256, 2), (2, 256, 8)])
def test_forced_cluster_matches_oracle_and_block_path(corde, ept, nt, C):
    rod = W.guidewire(1000, seed=510 + C)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    b.set_plan_cluster(ept, nt, C)
    assert tuple(b.plan()[0]) == (ept, nt, C)
    for _ in range(5):
        a.step(10)
        b.step(10)
    ga, gb = a.rod_state(a.state_numpy(), 0), b.rod_state(b.state_numpy(), 0)
    ref = oracle.step(rod, oracle.state_of(rod), 50)
    _cmp(rod, gb, ref, ROLL_TOL)
    assert np.abs(ga["pos"] - gb["pos"]).max() < 1e-5 * rod.length
    a.close()
    b.close()


def test_cluster_of_16_blocks(corde):
    """8192 nodes over 16 blocks (non-portable cluster size); skipped if the GPU cannot
    schedule a 16-block cluster of this shape."""
    rod = W.guidewire(8192, seed=520)
    b = corde.RodBatch([rod])
    b.set_plan_cluster(2, 256, 16)
    try:
        b.step(5)
        st = b.state_numpy()
    except corde.CordeError as e:
        b.close()
        pytest.skip(f"16-block cluster not schedulable: {e}")
    ref = oracle.step(rod, oracle.state_of(rod), 5)
    _cmp(rod, b.rod_state(st, 0), ref, ROLL_TOL)
    b.close()


def test_batch_mixing_block_and_cluster_rods(corde):
    rods = [W.guidewire(300, seed=530), W.guidewire(5000, seed=531), W.guidewire(1500, seed=532)]
    b = corde.RodBatch(rods)
    plans = b.plan()
    assert plans[1][2] >= 2 and plans[0][2] == 0
    b.step(10)
    st = b.state_numpy()
    for r, rod in enumerate(rods):
        ref = oracle.step(rod, oracle.state_of(rod), 10)
        _cmp(rod, b.rod_state(st, r), ref, ROLL_TOL)
    b.close()


@pytest.mark.parametrize("ept,nt,C", [(2, 256, 8), (4, 256, 4), (4, 512, 3)])
def test_grid_equals_cluster_bit_for_bit(corde, ept, nt, C):
    """The cooperative-grid form (global-memory halo, grid syncs) runs the same step body
    as the cluster form with the same blocks: after 30 driven steps the states are equal
    bit for bit, and rod_get_plan reports -C blocks."""
    import torch

    rod = W.guidewire(min(ept * nt * C, 4096) - 5, seed=540 + C)
    drive = torch.as_tensor(np.array([[0.02, -0.01, 0, 0, 0.1, 0, 2.0, 0]], np.float32), device="cuda")
    out = []
    for grid in (False, True):
        b = corde.RodBatch([rod])
        if grid:
            b.set_plan_grid(ept, nt, C)
            assert tuple(b.plan()[0]) == (ept, nt, -C)
        else:
            b.set_plan_cluster(ept, nt, C)
        for _ in range(3):
            b.step(10, drive=drive)
        out.append(b.state_numpy())
        b.close()
    for k in out[0]:
        np.testing.assert_array_equal(out[0][k], out[1][k], err_msg=k)


def test_rod_longer_than_a_cluster_runs_on_a_grid(corde):
    """A 40000-node rod (beyond the 32768 a 16-block cluster holds) gets the default grid
    plan (2048 nodes per block) and matches the oracle step by step."""
    import torch

    n = 40000
    rod = W.guidewire(n, seed=550)
    rod.length = 1.5 * n / 512  # the guidewire's segment length
    rod.pos = rod.pos * (n / 512)
    b = corde.RodBatch([rod])
    ept, nt, C = b.plan()[0]
    assert C < 0 and ept * nt * -C >= n
    drive = torch.as_tensor(np.array([[0.01, 0, 0, 0, 0, 0, 1.0, 0]], np.float32), device="cuda")
    for _ in range(2):
        st0 = b.rod_state(b.state_numpy(), 0)
        b.step(1, drive=drive)
        ref = oracle.step(rod, st0, 1, drive=drive.cpu().numpy()[0].astype(np.float64))
        _cmp(rod, b.rod_state(b.state_numpy(), 0), ref, STEP_TOL)
    b.step(10, drive=drive)
    rc, diag = b.diagnostics()
    assert rc == 0 and diag[0, 1] < 1e-6
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_enable(b.handle, 10)
    b.close()
