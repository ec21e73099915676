"""The allocation-free RayCast entry point (vd_raycast_noalloc).

It exists for callers that must not have the library call cudaMalloc while
they run (device memory owned by another allocator, or a steady-state loop
that must not pay cudaMalloc's synchronisation or risk an out-of-memory
error); its scratch is a fixed device array inside libvd.  This file is
collected last so that a run stopping at the first failure has run every
other test before it; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from gpu_util import clustered_fan, need_cuda, random_unit
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VDError, synth, vd

pytestmark = pytest.mark.gpu


def _ctx(torch, X, prec, knn_k=0):
    cfg = vd.vd_config_default()
    cfg.precision = prec
    cfg.knn_k = knn_k
    ctx = vd.vd_create(cfg, torch.cuda.current_stream().cuda_stream)
    vd.vd_set_nodes(ctx, torch.tensor(X, device="cuda"))
    return ctx


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32])
def test_noalloc_matches_vd_raycast_twice(prec):
    torch = need_cuda()
    d, N, R = 4, 3000, 20000
    X = synth.uniform(N, d, seed=31)
    rng = np.random.default_rng(5)
    cells = rng.integers(0, N, R).astype(np.int32)
    U = random_unit(rng, R, d)
    dev = torch.device("cuda")
    O = torch.tensor(X[cells], device=dev)
    Ud = torch.tensor(U, device=dev)
    E = torch.tensor(cells[:, None], device=dev)
    ctx = _ctx(torch, X, prec)
    try:
        h0 = torch.empty(R, dtype=torch.int32, device=dev)
        t0 = torch.empty(R, dtype=torch.float64, device=dev)
        vd.vd_raycast(ctx, O, Ud, E, h0, t0)
        for call in range(2):  # the scratch array keeps the previous call's contents
            h1 = torch.full((R,), -7, dtype=torch.int32, device=dev)
            t1 = torch.full((R,), -7.0, dtype=torch.float64, device=dev)
            vd.vd_raycast_noalloc(ctx, O, Ud, E, h1, t1)
            torch.cuda.synchronize()
            assert torch.equal(h1, h0), f"hit ids differ on call {call}"
            assert torch.equal(t1, t0), f"t differs on call {call}"
        # beyond the fixed scratch size the call is refused, not truncated
        big = 262144 + 1
        Ob = torch.zeros((big, d), dtype=torch.float64, device=dev)
        Eb = torch.zeros((big, 1), dtype=torch.int32, device=dev)
        with pytest.raises(VDError, match="scratch limit"):
            vd.vd_raycast_noalloc(ctx, Ob, Ob, Eb, torch.empty(big, dtype=torch.int32, device=dev),
                                  torch.empty(big, dtype=torch.float64, device=dev))
    finally:
        vd.vd_destroy(ctx)


def _noalloc_vs_oracle(orc, torch, X, O, U, E, prec, knn_k=0):
    """Two calls in a row against the oracle's brute force, bit for bit; the
    statistics of the last call."""
    h0, t0 = orc.raycast(X, O, U, E[:, 0])
    dev = torch.device("cuda")
    Od, Ud, Ed = (torch.tensor(a, device=dev) for a in (O, U, E))
    ctx = _ctx(torch, X, prec, knn_k)
    try:
        for call in range(2):
            h1 = torch.full((len(O),), -7, dtype=torch.int32, device=dev)
            t1 = torch.full((len(O),), -7.0, dtype=torch.float64, device=dev)
            vd.vd_raycast_noalloc(ctx, Od, Ud, Ed, h1, t1)
            torch.cuda.synchronize()
            assert np.array_equal(h1.cpu().numpy(), h0), f"hit ids differ from the oracle on call {call}"
            assert np.array_equal(t1.cpu().numpy(), t0), f"t differs from the oracle on call {call}"
            st = vd.vd_last_stats(ctx)
    finally:
        vd.vd_destroy(ctx)
    return st


def test_noalloc_tree_walk_rays_match_oracle(orc):
    """Short candidate lists (4 entries) leave most rays uncertified, so they
    go through the scratch array's tree-walk list: the hits still equal the
    oracle's."""
    torch = need_cuda()
    X = synth.uniform(3000, 4, seed=32)
    rng = np.random.default_rng(6)
    cells = rng.integers(0, 3000, 4000).astype(np.int32)
    st = _noalloc_vs_oracle(orc, torch, X, X[cells], random_unit(rng, 4000, 4), cells[:, None], VD_FP32, knn_k=4)
    assert st["fallback_rays"] > 0


def test_noalloc_overflow_rays_match_oracle(orc):
    """Clustered nodes overflow every ray's binary32 candidate buffer, so every
    ray goes through the scratch array's binary64 list: the hits still equal
    the oracle's."""
    torch = need_cuda()
    X, O, U, E = clustered_fan()
    st = _noalloc_vs_oracle(orc, torch, X, O, U, E, VD_FP32)
    assert st["overflow_rays"] > len(O) // 16
