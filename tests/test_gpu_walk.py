"""GPU parity of the random walks on the vertex graph (Section 2.3) with the
oracle: the same start vertices, seed and number of steps give the same
visited tuples and coordinates bit for bit (d = 2..6, the screened and the
binary64 RayCast paths, host and device buffers), also for sampled walkers of
a walk of 100,000 walkers at d = 5, N = 20,000; argument errors."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VD_TC16, Voronoi, synth, vd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,N", [(2, 300), (3, 400), (4, 200), (5, 150), (6, 60)])
def test_walk_parity(orc, d, N):
    need_cuda()
    X = synth.uniform(N, d, seed=120 + d)
    out = []
    for prec in (VD_FP32, VD_FP64, VD_TC16):
        vor = Voronoi(X, precision=prec)
        T, C, _ = vor.vertices()
        T = T.cpu().numpy()
        start = T[np.random.default_rng(d).choice(len(T), 64, replace=False)]
        PT, PC = vor.random_walk(start, 25, seed=9)
        out.append((PT.cpu().numpy(), PC.cpu().numpy()))
        vor.close()
    PT0, PC0 = orc.random_walk(X, start, 25, seed=9)
    for PT, PC in out:
        assert np.array_equal(PT, PT0) and np.array_equal(PC, PC0)


def test_walk_host_buffers_and_errors(orc):
    need_cuda()
    X = synth.uniform(200, 3, seed=2)
    vor = Voronoi(X)
    T, _, _ = vor.vertices()
    start = T.cpu().numpy()[:10]
    PT = np.empty((10, 7, 4), np.int32)
    PC = np.empty((10, 7, 3))
    vd.vd_random_walk(vor.ctx, start, 7, 4, PT, PC)
    PT0, PC0 = orc.random_walk(X, start, 7, seed=4)
    assert np.array_equal(PT, PT0) and np.array_equal(PC, PC0)
    st = vor.stats()
    assert st["rays"] == 70
    vor.close()
    vor7 = Voronoi(synth.uniform(40, 7, seed=1))
    with pytest.raises(vd.VDError):
        vd.vd_random_walk(vor7.ctx, np.zeros((1, 8), np.int32), 2, 1, np.empty((1, 2, 8), np.int32))
    vor7.close()
    vorb = Voronoi(X, box=False)
    with pytest.raises(vd.VDError):
        vd.vd_random_walk(vorb.ctx, start, 2, 1, np.empty((10, 2, 4), np.int32))
    vorb.close()


def test_walk_at_full_size(orc):
    """d = 5, N = 20,000: 100,000 walkers from vertices of the diagram, 6
    steps; 12 sampled walkers against the oracle (with their indices)."""
    torch = need_cuda()
    X = synth.uniform(20000, 5, seed=0)
    vor = Voronoi(X)
    T, _, _ = vor.vertices()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(T.shape[0], 100000, replace=False))
    start = T[torch.tensor(idx, device=T.device)]
    PT, PC = vor.random_walk(start, 6, seed=21)
    pick = np.sort(rng.choice(100000, 12, replace=False))
    PT0, PC0 = orc.random_walk(X, start.cpu().numpy()[pick], 6, seed=21, wid=pick)
    assert np.array_equal(PT.cpu().numpy()[pick], PT0) and np.array_equal(PC.cpu().numpy()[pick], PC0)
    vor.close()
