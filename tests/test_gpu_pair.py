"""Catheter/guidewire pair (binding modes v0, v1, v2) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
ROLL_TOL = 1e-4
QUAT_TOL = 1e-4


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


def _drive_tensor(torch, dc, dg):
    return torch.as_tensor(np.stack([dc, dg]).astype(np.float32), device="cuda").contiguous()


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("n", [33, 130])
def test_pair_one_step_parity(corde, mode, n):
    import torch

    beta = -7.35 if n > 40 else -4.6
    cat, gw = W.catheter_guidewire(n, seed=90 + n, beta0=beta)
    b = corde.RodBatch([cat, gw])
    b.bind(0, 1, mode)
    dc = np.array([0.01, 0.0, 0.002, 0.0, 0.0, 0.0, 1.0, 0.0])
    dg = np.array([0.02, -0.001, 0.0, beta, 0.0, 0.0, -2.0, 0.0])
    d = _drive_tensor(torch, dc, dg)
    for _ in range(3):
        st = b.state_numpy()
        so, si = b.rod_state(st, 0), b.rod_state(st, 1)
        b.step(1, drive=d)
        st2 = b.state_numpy()
        ro, ri = oracle.step_pair(cat, so, gw, si, mode, beta, 1, drive_outer=dc, drive_inner=dg)
        _cmp(cat, b.rod_state(st2, 0), ro, STEP_TOL)
        _cmp(gw, b.rod_state(st2, 1), ri, STEP_TOL)
    b.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pair_2x512_free_running(corde, mode):
    """The 2 x 512 pair workload: 10 launches of 10 steps with 1 kHz base drives and the
    relative insertion updating the binding offset every launch."""
    import torch

    cat, gw = W.catheter_guidewire(512, seed=3, beta0=-100.25)
    l0 = gw.length / 511
    dcs, dgs = W.pair_drives(3, 10, 10 * gw.dt, l0, -100.25)
    b = corde.RodBatch([cat, gw])
    b.bind(0, 1, mode)
    so, si = oracle.state_of(cat), oracle.state_of(gw)
    for k in range(10):
        b.step(10, drive=_drive_tensor(torch, dcs[k], dgs[k]))
        beta = float(np.float32(dgs[k, 3]))
        so, si = oracle.step_pair(cat, so, gw, si, mode, beta, 10, drive_outer=dcs[k], drive_inner=dgs[k])
    st = b.state_numpy()
    _cmp(cat, b.rod_state(st, 0), so, ROLL_TOL)
    _cmp(gw, b.rod_state(st, 1), si, ROLL_TOL)
    assert b.last_launch_count() == 1
    b.close()


def test_pair_mixed_with_single_rods(corde):
    """A handle with a bound pair and independent rods steps both kinds in one call."""
    cat, gw = W.catheter_guidewire(64, seed=95, beta0=-6.5)
    lone = W.guidewire(100, seed=96)
    b = corde.RodBatch([lone, cat, gw])
    b.bind(1, 2, 2)
    b.step(5)
    assert b.last_launch_count() == 2
    st = b.state_numpy()
    ref = oracle.step(lone, oracle.state_of(lone), 5)
    _cmp(lone, b.rod_state(st, 0), ref, ROLL_TOL)
    so, si = oracle.step_pair(cat, oracle.state_of(cat), gw, oracle.state_of(gw), 2, 0.0, 5)
    _cmp(cat, b.rod_state(st, 1), so, ROLL_TOL)
    _cmp(gw, b.rod_state(st, 2), si, ROLL_TOL)
    with pytest.raises(corde.CordeError):
        b.bind(0, 1, 1)  # rod 1 already paired
    b.close()
