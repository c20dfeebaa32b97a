"""CSI / RSSI through visibility weights (Eq. render_reorder) against the
per-pixel compositing path and the oracle, for explicit and MLP radiance,
alone and in uneven batches."""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, norm_err, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a GPU"
    return t


@pytest.fixture(scope="module")
def rx():
    from paper_2605_24290_gb300 import rxgs
    return rxgs


@pytest.mark.parametrize("C", [1, 2, 4])
def test_explicit_radiance_visibility_equals_oracle(torch, rx, oracle, C):
    rng = np.random.default_rng(601)
    sc = S.draw_scene(rng, 3000)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, C=C)
    tx = S.draw_points(rng, 3)
    rad = S.draw_radiance(rng, 7, sc.K, C)
    views = ctx.prepare(h, dev(tx, torch))
    kind = rx.OUT_CSI | (rx.OUT_RSSI if C == 1 else 0)
    csi = torch.zeros((3, 7, C, 2), device="cuda")
    rssi = torch.zeros((3, 7), device="cuda") if C == 1 else None
    ctx.render_views(views, None, 7, kind, radiance=dev(rad, torch), csi=csi, rssi=rssi,
                     reduce_path=1)
    ctx.sync()
    for v in range(3):
        o = oracle.render_view(g, sc, tx[v], rad.astype(np.float64))
        a = o["absacc"].sum(axis=(1, 2))
        assert norm_err(csi[v].cpu().numpy(), oracle.csi(o["spectra"]), a) <= TOL
        if C == 1:
            e = np.abs(rssi[v].cpu().numpy() - oracle.rssi(o["spectra"])) / (a[:, 0] + 1e-30)
            assert float(e.max()) <= TOL


@pytest.mark.parametrize("C", [1, 3])
def test_mlp_visibility_equals_oracle_and_batched(torch, rx, oracle, C):
    rng = np.random.default_rng(602 + C)
    K = 3000
    sc = S.draw_scene(rng, K)
    base = S.draw_base(rng, K, C)
    mlp = S.draw_mlp(rng, C)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, base=base, mlp_flat=S.flatten_mlp(mlp, C), C=C)
    tx = S.draw_points(rng, 2)
    rxp = S.draw_points(rng, 9)
    views = ctx.prepare(h, dev(tx, torch))
    csi = torch.zeros((2, 9, C, 2), device="cuda")
    ctx.render_views(views, dev(rxp, torch), 9, rx.OUT_CSI, csi=csi, reduce_path=1)
    ctx.sync()
    rad = oracle.mlp_radiance(mlp, rxp, sc.means, base)
    scales = []
    for v in range(2):
        o = oracle.render_view(g, sc, tx[v], rad)
        a = o["absacc"].sum(axis=(1, 2))
        scales.append(a)
        assert norm_err(csi[v].cpu().numpy(), oracle.csi(o["spectra"]), a) <= TOL
    # uneven batches through the graph: receivers 0..3 with tx 0, 4..8 with tx 1
    counts = [4, 5]
    bc = torch.zeros((9, C, 2), device="cuda")
    ctx.render_batched(h, dev(tx, torch), dev(rxp, torch), counts, rx.OUT_CSI, csi=bc)
    ctx.sync()
    ref = np.concatenate([csi[0, :4].cpu().numpy(), csi[1, 4:].cpu().numpy()])
    a = np.concatenate([scales[0][:4], scales[1][4:]])
    assert norm_err(bc.cpu().numpy(), ref, a) <= TOL


@pytest.mark.parametrize("C", [3, 8, 52])
def test_mlp_bf16_visibility_pixel_and_batched(torch, rx, oracle, C):
    """bf16 conditioning MLP: the per-pixel path, the visibility path (tensor
    cores for C > 4) and uneven batches, against the oracle's bf16 MLP."""
    rng = np.random.default_rng(640 + C)
    K = 3000
    sc = S.draw_scene(rng, K)
    base = S.draw_base(rng, K, C)
    mlp = S.draw_mlp(rng, C)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, base=base, mlp_flat=S.flatten_mlp(mlp, C), C=C, bf16=True)
    tx = S.draw_points(rng, 2)
    rxp = S.draw_points(rng, 9)
    views = ctx.prepare(h, dev(tx, torch))
    csi_v = torch.zeros((2, 9, C, 2), device="cuda")
    csi_p = torch.zeros((2, 9, C, 2), device="cuda")
    ctx.render_views(views, dev(rxp, torch), 9, rx.OUT_CSI, csi=csi_v, reduce_path=1)
    ctx.render_views(views, dev(rxp, torch), 9, rx.OUT_CSI, csi=csi_p, reduce_path=0)
    ctx.sync()
    rad = oracle.mlp_radiance(mlp, rxp, sc.means, base, bf16=True)
    scales = []
    for v in range(2):
        o = oracle.render_view(g, sc, tx[v], rad)
        a = o["absacc"].sum(axis=(1, 2))
        scales.append(a)
        ref = oracle.csi(o["spectra"])
        ev = norm_err(csi_v[v].cpu().numpy(), ref, a)
        ep = norm_err(csi_p[v].cpu().numpy(), ref, a)
        print(f"C={C} view {v}: visibility {ev:.3e}  per-pixel {ep:.3e}")
        assert ev <= TOL and ep <= TOL
    counts = [4, 5]
    bc = torch.zeros((9, C, 2), device="cuda")
    ctx.render_batched(h, dev(tx, torch), dev(rxp, torch), counts, rx.OUT_CSI, csi=bc)
    ctx.sync()
    ref = np.concatenate([csi_v[0, :4].cpu().numpy(), csi_v[1, 4:].cpu().numpy()])
    a = np.concatenate([scales[0][:4], scales[1][4:]])
    assert norm_err(bc.cpu().numpy(), ref, a) <= TOL


def test_visibility_many_views_and_backward(torch, rx, oracle):
    """18 transmitters (two passes of 16 views in the weighted sum, the gamma
    and the outer-product kernels), C = 2, an odd Gaussian count."""
    rng = np.random.default_rng(660)
    K, M, N, C = 1501, 18, 5, 2
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, C=C)
    tx = S.draw_points(rng, M)
    rad = S.draw_radiance(rng, N, K, C)
    views = ctx.prepare(h, dev(tx, torch))
    radd = dev(rad, torch)
    csi = torch.zeros((M, N, C, 2), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_CSI, radiance=radd, csi=csi, reduce_path=1)
    gc = rng.normal(size=(M, N, C, 2)).astype(np.float32)
    d_rad = torch.zeros_like(radd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_CSI, radiance=radd, grad_csi=dev(gc, torch),
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    ref_r = np.zeros(rad.shape)
    abs_r = np.zeros(rad.shape)
    ref_t = np.zeros(K)
    abs_t = np.zeros(K)
    for v in range(M):
        o = oracle.render_view(g, sc, tx[v], rad.astype(np.float64))
        a = o["absacc"].sum(axis=(1, 2))
        assert norm_err(csi[v].cpu().numpy(), oracle.csi(o["spectra"]), a) <= TOL, v
        gspec = np.broadcast_to(gc[v].astype(np.float64)[:, None, None, :, :], (N, g.H, g.W, C, 2))
        gr, gt, ar, at = oracle.backward_view(g, sc, tx[v], rad.astype(np.float64), gspec,
                                              want_abs=True)
        ref_r += gr
        abs_r += ar
        ref_t += gt
        abs_t += at
    assert float((np.abs(d_rad.cpu().numpy() - ref_r) / (abs_r + 1e-30)).max()) <= TOL
    assert float((np.abs(d_tau.cpu().numpy() - ref_t) / (abs_t + 1e-30)).max()) <= TOL
