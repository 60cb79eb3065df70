"""Empty-barrier floors (block, warp, cluster, cooperative grid) measure and order sanely."""
import pytest

pytestmark = pytest.mark.gpu


def test_barrier_floors(cuda):
    from paper_2509_04277_gb300 import build, corde

    build.build()
    block = corde.rod_barrier_floor(0, threads=256, n_iters=20000)
    warp = corde.rod_barrier_floor(1, n_iters=20000)
    cl2 = corde.rod_barrier_floor(2, threads=128, cluster=2, n_iters=20000)
    grid = corde.rod_barrier_floor(3, threads=128, cluster=1, n_iters=2000)
    for v in (block, warp, cl2, grid):
        assert 0.0 < v < 1e6
    assert grid > block
    with pytest.raises(corde.CordeError):
        corde.rod_barrier_floor(7, threads=32)


def test_device_info_and_fp32_peak(cuda):
    """The SM count comes from the runtime (equal to torch's), and the FP32 FMA peak is
    bounded by the SM count x 128 lanes x 2 flops x the clock (4 flops with paired lanes):
    a measured rate above that bound would mean the kernel did not do the work."""
    import torch

    from paper_2509_04277_gb300 import build, corde

    build.build()
    info = corde.rod_device_info()
    assert info["n_sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = info["n_sms"] * 128 * 2 * 2.2e9 / 1e12  # no GB300 SM clock exceeds 2.2 GHz
    scalar = corde.rod_fp32_peak(False, n_iters=20000)
    packed = corde.rod_fp32_peak(True, n_iters=10000)
    assert 0.25 * ceiling < scalar <= ceiling, (scalar, ceiling)
    assert 0.25 * ceiling < packed <= 2 * ceiling, (packed, ceiling)
    with pytest.raises(corde.CordeError):
        corde.rod_fp32_peak(False, threads=33)
