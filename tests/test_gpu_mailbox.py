"""Mailbox of a running launch: the host writes the base drive into a kernel while it
runs and reads the base/tip feedback back (the paper's haptic loop, Section 2.2)."""
import threading
import time

import numpy as np
import pytest

from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def corde(cuda):
    from paper_2509_04277_gb300 import build, corde as C

    build.build()
    C.load()
    return C


@pytest.mark.parametrize("n", [512, 3000])
def test_mailbox_input_equals_set_input(corde, n):
    rod = W.guidewire(n, seed=600 + n)
    drive = np.array([[0.02, -0.01, 0.0, 0.0, 0.0, 0.0, 1.5, 0.0]], np.float32)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    corde.rod_mailbox_enable(a.handle, 1, 64)
    corde.rod_mailbox_write(a.handle, drive)
    a.step(100)
    b.set_input(drive)
    b.step(100)
    sa, sb = a.state_numpy(), b.state_numpy()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])
    log, cnt = corde.rod_mailbox_log(a.handle)
    assert cnt == 1 and tuple(log[0]) == (0, 2)
    fb = corde.rod_mailbox_read(a.handle, 1)
    assert fb["step"][0, 0] == 100 and fb["step"][0, 1] == 100
    np.testing.assert_array_equal(fb["pos"][0, 0], sa["pos4"][0, :3])
    np.testing.assert_array_equal(fb["pos"][0, 1], sa["pos4"][n - 1, :3])
    np.testing.assert_array_equal(fb["vel"][0, 1], sa["vel4"][n - 1, :3])
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()


def test_mailbox_updates_a_running_kernel_and_replays_exactly(corde):
    """One launch of 20000 steps while the host writes a new drive every ~2 ms and reads
    the feedback; the kernel's log of picked-up inputs replayed through the normal path
    (rod_set_input + rod_step segments) reproduces the final state bit for bit."""
    import torch

    rod = W.guidewire(512, seed=610)
    a = corde.RodBatch([rod])
    period, n_steps = 10, 20000
    corde.rod_mailbox_enable(a.handle, period, 4096)
    drives = {}
    stamps = []
    stop = threading.Event()
    stream = torch.cuda.Stream()

    def haptic():
        k = 0
        while not stop.is_set() and k < 500:
            k += 1
            d = np.zeros((1, 8), np.float32)
            d[0, 0] = 0.01 * np.sin(0.3 * k)
            d[0, 6] = 2.0 * np.cos(0.2 * k)
            corde.rod_mailbox_write(a.handle, d)
            drives[2 * k] = d
            stamps.append(int(corde.rod_mailbox_read(a.handle, 1)["step"][0, 1]))
            time.sleep(0.002)

    with torch.cuda.stream(stream):
        a.step(n_steps, stream=stream)
        th = threading.Thread(target=haptic)
        th.start()
        stream.synchronize()
    stop.set()
    th.join()
    log, cnt = corde.rod_mailbox_log(a.handle)
    assert cnt == len(log) and cnt >= 5, "the kernel picked up too few inputs"
    assert len(set(stamps)) >= 3, "feedback did not advance while the kernel ran"
    assert all(log[i, 0] < log[i + 1, 0] for i in range(len(log) - 1))
    final = a.state_numpy()
    # replay
    b = corde.RodBatch([rod])
    pos = 0
    for (step, seq) in log:
        if step > pos:
            b.step(step - pos)
            pos = step
        b.set_input(drives[int(seq)])
    b.step(n_steps - pos)
    rep = b.state_numpy()
    for k in final:
        np.testing.assert_array_equal(final[k], rep[k])
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()


@pytest.mark.parametrize("n", [512, 3000])
def test_mailbox_position_snapshots_are_whole_steps(corde, n):
    """A free-falling straight rod (no clamp, gravity on: every node has the same height at
    any step) published every 5 steps during a 20000-step launch: each snapshot the host
    pulls while the kernel runs holds one step (all heights equal), steps increase, and
    the last snapshot is the final state.  3000 nodes run on a cluster of blocks."""
    import torch

    rod = W.straight_rod(n, 1.0, seed=620, radius=1e-3, E_bend=50e9, E_stretch=50e9, G=20e9, density=6500.0,
                         dt=1e-5, n_iters=4, inextensible=True, clamp=0, damping_alpha=0.0, gravity=(0.0, 0.0, -9.81))
    a = corde.RodBatch([rod])
    g_eff = 9.81 / a.derived()[0, 8]  # gravity acts on the inertial mass: g / mass_scale
    dt, period = 1e-5, 5
    corde.rod_mailbox_enable(a.handle, period, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    out = np.zeros((n, 4), np.float32)
    assert corde.rod_mailbox_positions(a.handle, 0, out) == -1
    assert corde.rod_mailbox_positions(a.handle, 0, None) == -1  # the step only
    a.step(20000)  # asynchronous: the host pulls snapshots while it runs
    steps, seen = [], 0
    t0 = time.time()
    while time.time() - t0 < 30.0:
        s = corde.rod_mailbox_positions(a.handle, 0, out)
        if s > 0 and (not steps or s != steps[-1]):
            steps.append(s)
            if s >= 50:
                # heights of one step agree to rounding; one period moves them g dt^2 period s
                spread = float(out[:, 2].max() - out[:, 2].min())
                assert spread < 0.2 * g_eff * dt * dt * period * s, f"torn snapshot at step {s}"
                seen += 1
        if s == 20000:
            break
    torch.cuda.synchronize()
    assert steps == sorted(steps) and all(k % 5 == 0 for k in steps)
    assert seen >= 3
    s = corde.rod_mailbox_positions(a.handle, 0, out)
    assert s == 20000
    assert corde.rod_mailbox_positions(a.handle, 0, None) == 20000
    np.testing.assert_array_equal(out, a.state_numpy()["pos4"])
    corde.rod_mailbox_disable(a.handle)
    a.close()


def _wait_snapshot(corde, h, out, step, limit_s=10.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        if corde.rod_mailbox_positions(h, 0, out) >= step:
            return True
    return False


def test_lockstep_each_input_drives_the_next_period_exactly(corde):
    """Lock-step: one 200-step launch; the host writes drive k, waits for the snapshot after
    steps 10 k .. 10 k + 9 and writes drive k + 1.  Every snapshot equals, bit for bit, the
    positions of the same drives replayed as ordinary 10-step launches."""
    import torch

    rod = W.guidewire(512, seed=630)
    a, b = corde.RodBatch([rod]), corde.RodBatch([rod])
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    corde.rod_mailbox_lockstep(a.handle, True, 2_000_000)
    drives = W.sinusoid_drive(631, 20, 10 * rod.dt).astype(np.float32)
    base = corde.rod_steps_done(a.handle)
    snaps = []
    out = np.zeros((512, 4), np.float32)
    a.step(200)  # asynchronous; waits for each input
    for k in range(20):
        corde.rod_mailbox_write(a.handle, drives[k].reshape(1, 8))
        assert _wait_snapshot(corde, a.handle, out, base + 10 * (k + 1)), f"no snapshot for tick {k}"
        snaps.append(out.copy())
    torch.cuda.synchronize()
    assert corde.rod_mailbox_status(a.handle) == 0
    for k in range(20):
        b.set_input(drives[k].reshape(1, 8))
        b.step(10)
        np.testing.assert_array_equal(snaps[k], b.state_numpy()["pos4"])
    sa, sb = a.state_numpy(), b.state_numpy()
    for key in sa:
        np.testing.assert_array_equal(sa[key], sb[key])
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()


def test_lockstep_wait_runs_out_cleanly(corde):
    """No input ever arrives: the launch's first wait runs out after 20 ms of GPU time, the
    launch ends without stepping, the status reports it once, and the device stays usable."""
    import torch

    rod = W.guidewire(256, seed=640)
    a = corde.RodBatch([rod])
    before = a.state_numpy()
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_lockstep(a.handle, True, 20_000)
    t0 = time.time()
    a.step(100)
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert corde.rod_mailbox_status(a.handle) & 1
    assert corde.rod_mailbox_status(a.handle) == 0
    after = a.state_numpy()
    for key in before:
        np.testing.assert_array_equal(before[key], after[key])
    corde.rod_mailbox_disable(a.handle)
    a.step(10)  # the context is fine
    torch.cuda.synchronize()
    a.close()


def test_lockstep_on_a_cluster_replays_exactly_and_runs_out_cleanly(corde):
    """A 3000-node rod on a thread-block cluster in lock-step: the base's thread waits, the
    other blocks wait at the cluster-wide OR.  Ten ticks equal ordinary 10-step launches
    bit for bit; then no input comes, the wait runs out after 20 ms, every block leaves,
    and the status reports it."""
    import torch

    rod = W.guidewire(3000, seed=641)
    a, b = corde.RodBatch([rod]), corde.RodBatch([rod])
    assert a.plan()[0][2] > 1  # on a cluster
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    corde.rod_mailbox_lockstep(a.handle, True, 20_000)
    drives = W.sinusoid_drive(642, 10, 10 * rod.dt).astype(np.float32)
    base = corde.rod_steps_done(a.handle)
    out = np.zeros((3000, 4), np.float32)
    snaps = []
    t0 = time.time()
    a.step(300)  # 30 ticks' worth; the host stops after 10
    for k in range(10):
        got = corde.rod_mailbox_exchange(a.handle, drives[k].reshape(1, 8), 0, base + 10 * (k + 1), out, 5_000_000)
        assert got == base + 10 * (k + 1)
        snaps.append(out.copy())
    torch.cuda.synchronize()
    assert time.time() - t0 < 10.0
    assert corde.rod_mailbox_status(a.handle) & 1
    for k in range(10):
        b.set_input(drives[k].reshape(1, 8))
        b.step(10)
        np.testing.assert_array_equal(snaps[k], b.state_numpy()["pos4"])
    corde.rod_mailbox_disable(a.handle)
    a.step(10)  # the context is fine
    torch.cuda.synchronize()
    a.close()
    b.close()


def test_lockstep_pair_with_moving_binding_offset(corde):
    """A bound catheter/guidewire pair (v2) in lock-step: each tick's two drive rows (the
    inner row's slot 3 is the binding offset, 0.15 segments further each tick) drive the next 10 steps;
    both rods' snapshots equal ordinary 10-step launches with the same rows, bit for bit."""
    import torch

    cat, gw = W.catheter_guidewire(64, seed=650, beta0=-6.5)
    a, b = corde.RodBatch([cat, gw]), corde.RodBatch([cat, gw])
    a.bind(0, 1, 2)
    b.bind(0, 1, 2)
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    corde.rod_mailbox_lockstep(a.handle, True, 2_000_000)
    dcs, dgs = W.pair_drives(651, 20, 10 * gw.dt, gw.length / 63, -6.5)
    rows = np.stack([dcs, dgs], axis=1).astype(np.float32)
    rows[:, 1, 3] = -6.5 + 0.15 * np.arange(20)  # the binding point crosses three outer segments
    base = corde.rod_steps_done(a.handle)
    out0, out1 = np.zeros((64, 4), np.float32), np.zeros((64, 4), np.float32)
    snaps = []
    a.step(200)
    for k in range(20):
        corde.rod_mailbox_write(a.handle, rows[k])
        target = base + 10 * (k + 1)
        assert _wait_snapshot(corde, a.handle, out0, target)
        t0 = time.time()
        while corde.rod_mailbox_positions(a.handle, 1, out1) < target and time.time() - t0 < 10.0:
            pass
        snaps.append((out0.copy(), out1.copy()))
    torch.cuda.synchronize()
    assert corde.rod_mailbox_status(a.handle) == 0
    for k in range(20):
        b.step(10, drive=torch.as_tensor(rows[k], device="cuda"))
        st = b.state_numpy()["pos4"]
        np.testing.assert_array_equal(snaps[k][0], st[:64])
        np.testing.assert_array_equal(snaps[k][1], st[64:])
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()


def test_exchange_ticks_replay_exactly_and_report_a_lost_wait(corde):
    """rod_mailbox_exchange (one call per tick: write the drive, wait for the snapshot of
    the tick's last step, copy it) drives a lock-step launch; every snapshot equals the
    positions of ordinary 10-step launches with the same drives.  Then the host stops
    sending: the kernel's 20 ms wait runs out, and the next exchange reports it."""
    import torch

    rod = W.guidewire(512, seed=660)
    a, b = corde.RodBatch([rod]), corde.RodBatch([rod])
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    corde.rod_mailbox_lockstep(a.handle, True, 20_000)
    drives = W.sinusoid_drive(661, 15, 10 * rod.dt).astype(np.float32)
    base = corde.rod_steps_done(a.handle)
    out = np.zeros((512, 4), np.float32)
    snaps = []
    a.step(400)  # 40 ticks' worth; the host stops after 15
    for k in range(15):
        got = corde.rod_mailbox_exchange(a.handle, drives[k].reshape(1, 8), 0, base + 10 * (k + 1), out, 5_000_000)
        assert got == base + 10 * (k + 1)
        snaps.append(out.copy())
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_exchange(a.handle, None, 0, base + 10 * 16, out, 5_000_000)
    torch.cuda.synchronize()
    assert corde.rod_mailbox_status(a.handle) & 1
    for k in range(15):
        b.set_input(drives[k].reshape(1, 8))
        b.step(10)
        np.testing.assert_array_equal(snaps[k], b.state_numpy()["pos4"])
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_exchange(a.handle, None, 0, 0, out, -1)
    # no launch running: the host-side wait gives up after its timeout
    corde.rod_mailbox_status(a.handle)  # clear the bit from the lost wait above
    t0 = time.time()
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_exchange(a.handle, drives[0].reshape(1, 8), 0, base + 10**9, out, 20_000)
    assert 0.015 < time.time() - t0 < 2.0
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()


def test_tick_closed_loop_replays_exactly(corde):
    """rod_mailbox_tick (wait for tick k's snapshot, write tick k + 1's drive at once, then
    copy): every snapshot of a 15-tick closed loop equals the positions of ordinary
    10-step launches with the same drives; after the last tick no drive follows, the
    kernel's 20 ms wait runs out and the next tick call reports it without writing."""
    import torch

    rod = W.guidewire(512, seed=670)
    a, b = corde.RodBatch([rod]), corde.RodBatch([rod])
    corde.rod_mailbox_enable(a.handle, 10, 64)
    corde.rod_mailbox_positions_enable(a.handle)
    corde.rod_mailbox_lockstep(a.handle, True, 20_000)
    drives = W.sinusoid_drive(671, 15, 10 * rod.dt).astype(np.float32)
    base = corde.rod_steps_done(a.handle)
    out = np.zeros((512, 4), np.float32)
    snaps = []
    a.step(400)  # 40 ticks' worth; the host stops after 15
    corde.rod_mailbox_write(a.handle, drives[0].reshape(1, 8))
    for k in range(15):
        nxt = drives[k + 1].reshape(1, 8) if k + 1 < 15 else None
        got = corde.rod_mailbox_tick(a.handle, 0, base + 10 * (k + 1), nxt, out, 5_000_000)
        assert got == base + 10 * (k + 1)
        snaps.append(out.copy())
    with pytest.raises(corde.CordeError):
        corde.rod_mailbox_tick(a.handle, 0, base + 10 * 16, drives[0].reshape(1, 8), None, 5_000_000)
    torch.cuda.synchronize()
    assert corde.rod_mailbox_status(a.handle) & 1
    for k in range(15):
        b.set_input(drives[k].reshape(1, 8))
        b.step(10)
        np.testing.assert_array_equal(snaps[k], b.state_numpy()["pos4"])
    corde.rod_mailbox_disable(a.handle)
    a.close()
    b.close()

