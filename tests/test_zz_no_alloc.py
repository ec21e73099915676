"""The allocation-free RayCast entry point (vd_raycast_noalloc).

It exists for callers that must not have the library call cudaMalloc while
they run (device memory owned by another allocator, or a steady-state loop
that must not pay cudaMalloc's synchronisation or risk an out-of-memory
error); its scratch is a fixed device array inside libvd.  This file is
collected last so that a run stopping at the first failure has run every
other test before it; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from gpu_util import need_cuda, random_unit
from paper_2405_10050_gb300 import VD_FP32, VD_FP64, VDError, synth, vd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [VD_FP64, VD_FP32])
def test_noalloc_matches_vd_raycast_twice(prec):
    torch = need_cuda()
    d, N, R = 4, 3000, 20000
    X = synth.uniform(N, d, seed=31)
    rng = np.random.default_rng(5)
    cells = rng.integers(0, N, R).astype(np.int32)
    U = random_unit(rng, R, d)
    dev = torch.device("cuda")
    Xd = torch.tensor(X, device=dev)
    O = torch.tensor(X[cells], device=dev)
    Ud = torch.tensor(U, device=dev)
    E = torch.tensor(cells[:, None], device=dev)
    cfg = vd.vd_config_default()
    cfg.precision = prec
    ctx = vd.vd_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        vd.vd_set_nodes(ctx, Xd)
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
