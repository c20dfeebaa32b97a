"""rxgs_render_csi_noalloc: the allocation-free CSI/RSSI entry point.

It exists for callers that must not allocate device memory while they render
(a serving thread with a hard latency budget, a program whose device memory
is owned by another allocator).  It keeps its partial sums in a fixed device
array inside the library, so these checks call it twice in a row with
different radiance (the second call finds the first call's leftovers in that
array) and compare both results with rxgs_render_views, which allocates its
scratch.  The file is named to run last.
"""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, upload

pytestmark = pytest.mark.gpu


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
        ctx.render_csi_noalloc(views, radd, N, csi=csi, rssi=rssi)
        ctx.sync()
        a = abs_csi.cpu().numpy().sum(-1)[..., None]
        err = np.abs(csi.cpu().numpy() - ref_csi.cpu().numpy()) / (a + 1e-30)
        assert float(err.max()) <= TOL, (call, float(err.max()))
        err_r = np.abs(rssi.cpu().numpy() - ref_rssi.cpu().numpy()) / (a[..., 0, 0] + 1e-30)
        assert float(err_r.max()) <= TOL, (call, float(err_r.max()))
    # a request larger than the fixed scratch is refused before any launch
    big = torch.zeros(4, device="cuda")
    with pytest.raises(rxgs.RxgsError) as ei:
        ctx.render_csi_noalloc(views, big, 20000, csi=torch.zeros(4, device="cuda"))
    assert ei.value.status == rxgs.E_INVALID
    ctx.release_views(views)
    ctx.close()
