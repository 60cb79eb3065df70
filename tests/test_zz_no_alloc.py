"""rod_adjoint_noalloc: the gradient entry point for callers that cannot allocate device
memory where they need a gradient (real-time haptic or control loops, applications that
own their device memory through a pool).  Its outputs must equal those of the allocating
path (rod_rollout + rod_adjoint on a handle) on the same inputs, on two calls in a row
(the static scratch array keeps the previous call's contents).  This file is collected
last so that a failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_2509_04277_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_no_alloc_adjoint_matches_handle_path(cuda):
    import torch

    from paper_2509_04277_gb300 import build, corde

    build.build()
    corde.load()
    rod = W.adjoint_rod(96, seed=71)
    n, n_steps, ckpt = rod.n_nodes, 40, 9
    drive = np.array([0.01, -0.002, 0.0, 0.0, 0.0, 0.0, 1.5, 0.0], np.float32)
    target = torch.as_tensor(W.tip_target(72, n_steps, rod.dt, rod.pos[-1]), dtype=torch.float32, device="cuda")

    # allocating path through a handle
    b = corde.RodBatch([rod])
    b.set_input(drive[None, :])
    traj = b.rollout(n_steps, ckpt)
    g = torch.zeros_like(traj)
    g[:, n - 1, :3] = 2.0 * (traj[:, n - 1, :3] - target)
    ref = b.adjoint(g)
    torch.cuda.synchronize()
    b.close()

    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")  # noqa: E731
    inputs = dict(pos=dev(rod.pos), quat=dev(rod.quat), rest_quat=dev(rod.rest_quat), vel=dev(rod.vel),
                  omega=dev(rod.omega), stiff_mul=dev(rod.stiff_mul), drive=dev(drive))
    params = corde.params_of(rod)
    for call in range(2):
        out = {k: torch.full((n, 4), float("nan"), device="cuda") for k in ("dK", "duhat", "dvel0", "dpos0")}
        ptraj = torch.full((n_steps, n, 4), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        corde.rod_adjoint_noalloc(params, inputs["pos"], inputs["quat"], inputs["rest_quat"], inputs["vel"],
                                  inputs["omega"], inputs["stiff_mul"], inputs["drive"], n_steps, ckpt, g, ptraj,
                                  out["dK"], out["duhat"], out["dvel0"], out["dpos0"])
        torch.cuda.synchronize()
        if call == 1:
            # the call took no device memory (the first call on a device loads its kernels)
            assert torch.cuda.mem_get_info()[0] == free_before
        torch.testing.assert_close(ptraj[:, :, :3], traj[:, :, :3], rtol=1e-6, atol=1e-7)
        for k, rk in (("dK", "K"), ("duhat", "uhat"), ("dvel0", "vel0"), ("dpos0", "pos0")):
            a, r = out[k][:, :3], ref[rk][:, :3]
            scale = float(r.abs().max())
            assert torch.isfinite(a).all(), (call, k)
            assert float((a - r).abs().max()) <= 1e-5 * scale + 1e-30, (call, k)

    # requests beyond the static limit are refused before anything runs
    with pytest.raises(corde.CordeError) as e:
        corde.rod_adjoint_noalloc(params, inputs["pos"], inputs["quat"], n_steps=200000, ckpt_every=100000)
    assert e.value.code == corde.CORDE_ERR_ARG
