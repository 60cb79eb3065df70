"""Launch overlap (programmatic stream serialisation): a stepping kernel is scheduled while
the stream's previous one still runs and waits for its writes before touching memory.
Every kernel family gives, bit for bit, the state of ordinary launches."""
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


def _run(corde, rods, setup, n_calls, steps, overlap, drives=None):
    import torch

    b = corde.RodBatch(rods)
    setup(b)
    b.set_launch_overlap(overlap)
    for k in range(n_calls):
        d = None if drives is None else torch.as_tensor(drives[k], device="cuda")
        b.step(steps, drive=d)
    torch.cuda.synchronize()
    st = b.state_numpy()
    b.close()
    return st


def _same(a, b):
    for key in a:
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_single_rod_back_to_back_launches(corde):
    rod = W.guidewire(512, seed=901)
    drives = W.sinusoid_drive(902, 30, 10 * rod.dt)[:, None, :].astype(np.float32)
    on = _run(corde, [rod], lambda b: None, 30, 10, True, drives)
    off = _run(corde, [rod], lambda b: None, 30, 10, False, drives)
    _same(on, off)


def test_graph_with_blocks_cluster_pair_and_self_collision(corde):
    """Several length bins (a CUDA graph with one branch per bin), a rod on a cluster, a
    bound pair and a self-colliding knot, 12 calls of 5 steps."""
    rods = W.batched_rods(24, seed=903) + [W.guidewire(3000, seed=904)]
    cat, gw = W.catheter_guidewire(64, seed=905, beta0=-6.5)
    knot = W.torus_knot(128, seed=906)
    all_rods = rods + [cat, gw, knot]

    def setup(b):
        b.bind(len(rods), len(rods) + 1, 2)
        b.set_self_collision(len(rods) + 2, 0.1)

    on = _run(corde, all_rods, setup, 12, 5, True)
    off = _run(corde, all_rods, setup, 12, 5, False)
    _same(on, off)


def test_toggling_rebuilds_the_graph_and_bad_values_are_refused(corde):
    rods = W.batched_rods(16, seed=907)
    a = corde.RodBatch(rods)
    b = corde.RodBatch(rods)
    b.set_launch_overlap(False)
    for k in range(6):
        a.set_launch_overlap(k % 2 == 0)
        a.step(4)
        b.step(4)
    _same(a.state_numpy(), b.state_numpy())
    with pytest.raises(corde.CordeError):
        corde.rod_set_launch_overlap(a.handle, 2)
    a.close()
    b.close()
