"""rxgs_render_csi_noalloc: the allocation-free CSI/RSSI entry point.

It exists for callers that must not allocate device memory while they render
(a serving thread with a hard latency budget, a program whose device memory
is owned by another allocator).  It keeps its partial sums in a fixed device
array inside the library, so these checks call it twice in a row with
different radiance (the second call finds the first call's leftovers in that
array) and compare both results with rxgs_render_views, which allocates its
scratch.  They also check the property the entry point exists for: across a
call, the library makes no device allocation, and neither the device's
default memory pool nor torch's caching allocator grows.  The file is named
to run last.
"""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, upload

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 4_194_304      # the fixed scratch size the header states


def alloc_state(torch, ctx):
    p = ctx.profile_read(reset=False)
    return (p["device_allocs"], p["pool_used_bytes"], p["pool_reserved_bytes"],
            torch.cuda.memory_reserved(), torch.cuda.memory_allocated())


def test_noalloc_matches_allocating_render_twice():
    import torch
    from paper_2605_24290_gb300 import rxgs

    assert torch.cuda.is_available(), "GPU tests need a GPU"
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    rng = np.random.default_rng(301)
    ctx = rxgs.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    tx = np.concatenate([w["tx"], S.draw_points(rng, 2)])
    M, N = tx.shape[0], 8
    views = ctx.prepare(h, dev(tx, torch))
    kind = rxgs.OUT_CSI | rxgs.OUT_RSSI
    for call in range(2):
        rad = S.draw_radiance(rng, N, sc.K, 1)
        radd = dev(rad, torch)
        ref_csi = torch.zeros((M, N, 1, 2), device="cuda")
        ref_rssi = torch.zeros((M, N), device="cuda")
        ctx.render_views(views, None, N, kind, radiance=radd, csi=ref_csi, rssi=ref_rssi)
        # scale: the same sums over absolute contributions
        abs_csi = torch.zeros((M, N, 1, 2), device="cuda")
        ctx.render_views(views, None, N, rxgs.OUT_CSI, radiance=dev(np.abs(rad), torch), csi=abs_csi)
        csi = torch.full((M, N, 1, 2), float("nan"), device="cuda")
        rssi = torch.full((M, N), float("nan"), device="cuda")
        ctx.sync()
        before = alloc_state(torch, ctx)
        ctx.render_csi_noalloc(views, radd, N, csi=csi, rssi=rssi)
        ctx.sync()
        after = alloc_state(torch, ctx)
        assert after == before, f"call {call} allocated: {before} -> {after}"
        a = abs_csi.cpu().numpy().sum(-1)[..., None]
        err = np.abs(csi.cpu().numpy() - ref_csi.cpu().numpy()) / (a + 1e-30)
        assert float(err.max()) <= TOL, (call, float(err.max()))
        err_r = np.abs(rssi.cpu().numpy() - ref_rssi.cpu().numpy()) / (a[..., 0, 0] + 1e-30)
        assert float(err_r.max()) <= TOL, (call, float(err_r.max()))
    # a request one receiver past the fixed scratch is refused before any
    # launch; its buffers are sized for that N, so even a launch would stay
    # inside them
    T = ((g.H + 15) // 16) * ((g.W + 15) // 16)
    n_big = SCRATCH_FLOATS // (M * T * 2) + 1
    big = torch.zeros((n_big, sc.K, 1, 2), device="cuda")
    out = torch.zeros((M, n_big, 1, 2), device="cuda")
    with pytest.raises(rxgs.RxgsError) as ei:
        ctx.render_csi_noalloc(views, big, n_big, csi=out)
    assert ei.value.status == rxgs.E_INVALID
    assert "scratch" in str(ei.value)
    del big, out
    ctx.release_views(views)
    ctx.close()


def test_noalloc_refuses_a_grid_too_wide():
    """One tile and one view: 2NC = 4,194,304 columns fit the scratch but need
    65,536 column blocks, one more than a launch grid holds; refused."""
    import torch
    from paper_2605_24290_gb300 import rxgs

    rng = np.random.default_rng(302)
    sc = S.draw_scene(rng, 4)
    ctx = rxgs.Context(H=8, W=16, step_deg=22.5)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(S.draw_points(rng, 1), torch))
    n = SCRATCH_FLOATS // 2
    rad = torch.zeros((n, sc.K, 1, 2), device="cuda")
    csi = torch.zeros((1, n, 1, 2), device="cuda")
    with pytest.raises(rxgs.RxgsError) as ei:
        ctx.render_csi_noalloc(views, rad, n, csi=csi)
    assert ei.value.status == rxgs.E_INVALID
    assert "grid" in str(ei.value)
    ctx.release_views(views)
    ctx.close()
