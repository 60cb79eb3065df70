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
