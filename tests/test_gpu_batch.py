"""Batched Monte Carlo (many point sets of uneven N and d in one persistent,
graph-captured launch): every set matches the FP64 oracle run on that set
alone with its own Philox set id (Section 3.1, Algorithm 3)."""
import numpy as np
import pytest

from gpu_util import need_cuda
from paper_2405_10050_gb300 import synth, vd

pytestmark = pytest.mark.gpu


def _sets():
    rng = np.random.default_rng(4)
    out = []
    for s in range(10):
        N = int(rng.integers(40, 1500))
        d = int(rng.integers(2, 9))
        X = synth.uniform(N, d, seed=s) if s % 2 == 0 else synth.gaussian_mixture(N, d, 8, 0.05, seed=s)
        out.append(X)
    out.append(synth.uniform(1, 3, seed=99))   # a one-node set
    out.append(synth.uniform(33, 1, seed=98))  # d = 1
    return out


def test_batch_matches_oracle_per_set(orc):
    torch = need_cuda()
    Xs = _sets()
    R, seed = 24, 77
    ctx = vd.vd_create(None, torch.cuda.current_stream().cuda_stream)
    try:
        Xd = [torch.tensor(X, device="cuda") for X in Xs]
        mcs = vd.vd_mc_integrate_batch(ctx, Xd, R, seed)
        st = vd.vd_last_stats(ctx)
        assert st["rays"] == sum(X.shape[0] for X in Xs) * R
        ref_hits = []
        for s, (X, mc) in enumerate(zip(Xs, mcs)):
            N, d = X.shape
            ref = orc.mc_integrate(X, R, seed, set_id=s)
            ref_hits.append(ref.hit)
            hit = np.empty((N, R), np.int32)
            l = np.empty((N, R))
            vd.vd_mc_rays(mc, hit, l)
            assert np.array_equal(hit, ref.hit), f"set {s}"
            assert np.array_equal(l, ref.l), f"set {s}"
            V = np.empty(N)
            rowptr = np.empty(N + 1, np.int64)
            nnz = vd.vd_mc_get(mc, V=V, rowptr=rowptr)
            col = np.empty(nnz, np.int32)
            A = np.empty(nnz)
            vd.vd_mc_get(mc, col=col, A=A)
            assert np.array_equal(rowptr, ref.rowptr) and np.array_equal(col, ref.col)
            assert np.allclose(V, ref.V, rtol=1e-12, atol=0) and np.allclose(A, ref.A, rtol=1e-12, atol=0)
            if s < 3:  # the adjoint works on batched results too
                gV = np.linspace(-1, 1, N)
                gA = np.cos(np.arange(nnz))
                gX = np.empty((N, d))
                vd.vd_mc_adjoint(mc, gV, gA, gX)
                g0 = orc.mc_adjoint(X, R, seed, ref.hit, ref.l, ref.rowptr, ref.col, gV, gA, set_id=s)
                assert np.max(np.abs(gX - g0)) <= 1e-10 * max(np.max(np.abs(g0)), 1e-300)
            vd.vd_mc_free(mc)
        # a second call reuses the autotuned block size and the instantiated
        # graph (updated in place with this call's buffers): the same bits
        mcs2 = vd.vd_mc_integrate_batch(ctx, Xd, R, seed)
        for s, (X, mc) in enumerate(zip(Xs, mcs2)):
            h2 = np.empty((X.shape[0], R), np.int32)
            vd.vd_mc_rays(mc, h2, None)
            assert np.array_equal(h2, ref_hits[s]), f"set {s}, second call"
            vd.vd_mc_free(mc)
    finally:
        vd.vd_destroy(ctx)


def test_batch_rejects_high_dimension():
    torch = need_cuda()
    ctx = vd.vd_create(None)
    try:
        with pytest.raises(vd.VDError):
            vd.vd_mc_integrate_batch(ctx, [synth.uniform(10, 9, seed=0)], 8, 1)
    finally:
        vd.vd_destroy(ctx)


def test_batch_host_inputs_and_errors(orc):
    """Sets given as host arrays (copied on the preparation threads' own
    streams); a set with a non-finite coordinate fails the whole call with
    VD_EINVAL and leaves the context usable."""
    torch = need_cuda()
    Xs = [synth.uniform(300 + 37 * s, 2 + s % 5, seed=20 + s) for s in range(11)]
    R, seed = 16, 5
    ctx = vd.vd_create(None, torch.cuda.current_stream().cuda_stream)
    try:
        mcs = vd.vd_mc_integrate_batch(ctx, Xs, R, seed)
        for s in (0, 5, 10):
            X = Xs[s]
            hit = np.empty((X.shape[0], R), np.int32)
            l = np.empty((X.shape[0], R))
            vd.vd_mc_rays(mcs[s], hit, l)
            ref = orc.mc_integrate(X, R, seed, set_id=s)
            assert np.array_equal(hit, ref.hit) and np.array_equal(l, ref.l)
        for mc in mcs:
            vd.vd_mc_free(mc)
        bad = [X.copy() for X in Xs[:4]]
        bad[2][7, 1] = np.nan
        with pytest.raises(vd.VDError) as ei:
            vd.vd_mc_integrate_batch(ctx, bad, R, seed)
        assert ei.value.status == -1  # VD_EINVAL
        mcs = vd.vd_mc_integrate_batch(ctx, Xs[:3], R, seed)
        hit = np.empty((Xs[1].shape[0], R), np.int32)
        vd.vd_mc_rays(mcs[1], hit, None)
        assert np.array_equal(hit, orc.mc_integrate(Xs[1], R, seed, set_id=1).hit)
        for mc in mcs:
            vd.vd_mc_free(mc)
    finally:
        vd.vd_destroy(ctx)
