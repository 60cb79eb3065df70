"""rod_step_io: the kernels write the positions after their last step to a device or
mapped pinned host buffer and may read the drive from pinned host memory; the result is
the state rod_step leaves, bit for bit."""
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


def _state_pos(torch, corde, b):
    out = torch.empty((b.n_elem, 4), dtype=torch.float32, device="cuda")
    corde.rod_get_state(b.handle, out, None, None, None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("where", ["device", "pinned"])
def test_io_single_rod_matches_rod_step(corde, where):
    import torch

    rod = W.guidewire(512, seed=801)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    drive_np = np.array([[0.01, 0.0, 0.002, 0.0, 0.0, 0.0, 1.5, 0.0]], np.float32)
    d_dev = torch.as_tensor(drive_np, device="cuda")
    d_pin = torch.as_tensor(drive_np).pin_memory()
    out = (torch.empty((b.n_elem, 4), dtype=torch.float32, device="cuda") if where == "device"
           else torch.empty((b.n_elem, 4), dtype=torch.float32).pin_memory())
    for k in range(3):
        a.step(10, drive=d_dev)
        corde.rod_step_io(b.handle, 10, d_pin if where == "pinned" else d_dev, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy() if where == "device" else out.numpy().copy()
        np.testing.assert_array_equal(got, _state_pos(torch, corde, a))
        np.testing.assert_array_equal(got, _state_pos(torch, corde, b))
    a.close()
    b.close()


def test_io_graph_batch_pair_and_self(corde):
    """A handle with several length bins (graph), a bound pair and a self-colliding knot:
    every rod's positions arrive in one buffer; a second buffer re-captures the graph."""
    import torch

    rods = W.batched_rods(40, seed=802)
    cat, gw = W.catheter_guidewire(64, seed=803, beta0=-6.5)
    knot = W.torus_knot(128, seed=804)
    b = corde.RodBatch(rods + [cat, gw, knot])
    ref = corde.RodBatch(rods + [cat, gw, knot])
    for h in (b, ref):
        h.bind(len(rods), len(rods) + 1, 2)
        h.set_self_collision(len(rods) + 2, 0.1)
    outs = [torch.empty((b.n_elem, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    for k in range(4):
        ref.step(5)
        corde.rod_step_io(b.handle, 5, None, outs[k % 2])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[k % 2].numpy(), _state_pos(torch, corde, ref))
    assert b.last_launch_count() >= 3
    b.close()
    ref.close()


def test_io_null_output_is_rod_step_and_misaligned_is_rejected(corde):
    import torch

    rod = W.guidewire(100, seed=805)
    a = corde.RodBatch([rod])
    b = corde.RodBatch([rod])
    a.step(7)
    corde.rod_step_io(b.handle, 7, None, None)
    np.testing.assert_array_equal(_state_pos(torch, corde, a), _state_pos(torch, corde, b))
    buf = torch.empty((b.n_elem + 1) * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(corde.CordeError):
        corde.rod_step_io(b.handle, 1, None, buf.data_ptr() + 4)  # not 16-byte aligned: refused on the host
    a.close()
    b.close()
