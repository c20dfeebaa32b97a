"""Coverage map at full size: 1,000,000 Gaussians in a 40x30x4 m box,
16 transmitters x 1,024 receivers on a floor grid, 180x360 grid, explicit
radiance [1024, 1M, 1, 2] (8.2 GB, counter-based so that the oracle can draw
the rows it needs).  RSSI through the visibility path and the per-pixel path;
backward to radiance and opacity from an RSSI cotangent that is non-zero on
sampled (transmitter, receiver) pairs only, so that the oracle can compute
the exact gradients of the full-size launch."""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, upload

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


def test_coverage_map_full_size_sampled(torch, rx, oracle):
    w = S.workload_coverage(with_radiance=False)
    g, sc, tx, rxp = w["grid"], w["scene"], w["tx"], w["rx"]
    M, N, K = tx.shape[0], rxp.shape[0], sc.K
    ctx = rx.Context(H=g.H, W=g.W, theta0_deg=g.theta0_deg)
    h = upload(ctx, sc, torch)
    rad = S.hashed_radiance_torch(torch, N, K, "cuda")
    txd = dev(tx, torch)
    rssi_v = torch.zeros((M, N), device="cuda")
    csi_v = torch.zeros((M, N, 1, 2), device="cuda")
    rssi_p = torch.zeros((M, N), device="cuda")
    views = ctx.prepare(h, txd)
    ctx.render_views(views, None, N, rx.OUT_RSSI | rx.OUT_CSI, radiance=rad, rssi=rssi_v, csi=csi_v,
                     reduce_path=1)
    ctx.render_views(views, None, N, rx.OUT_RSSI, radiance=rad, rssi=rssi_p, reduce_path=0)
    ctx.sync()

    vs, js = [0, 11], [0, 517, 1023]
    rad_s = S.hashed_radiance_rows(js, K).astype(np.float64)
    rng = np.random.default_rng(S.SEED_BASE + 40)
    gsel = rng.normal(size=(len(vs), len(js))).astype(np.float32)
    grad_rssi = np.zeros((M, N), np.float32)
    # the forward CSI the backward takes for dRSSI/dCSI: the oracle's, rounded
    # to float32, on the sampled pairs (a near-cancelling CSI would make the
    # direction z/|z| ill-conditioned between two correct forwards)
    fwd_csi = np.zeros((M, N, 1, 2), np.float32)
    gspecs = []
    for a, v in enumerate(vs):
        o = oracle.render_view(g, sc, tx[v], rad_s)
        z = oracle.csi(o["spectra"])[:, 0, :]                # [3, 2]
        ref = np.sqrt((z ** 2).sum(axis=1))
        scale = o["absacc"].sum(axis=(1, 2))[:, 0]
        for got in (rssi_v, rssi_p):
            e = np.abs(got[v, js].cpu().numpy() - ref) / (scale + 1e-30)
            assert float(e.max()) <= TOL, (v, e)
        e = np.abs(csi_v[v, js, 0].cpu().numpy() - z) / (scale[:, None] + 1e-30)
        assert float(e.max()) <= TOL, (v, e)
        z32 = z.astype(np.float32)
        fwd_csi[v, js, 0] = z32
        grad_rssi[v, js] = gsel[a]
        z64 = z32.astype(np.float64)
        mag = np.sqrt((z64 ** 2).sum(axis=1))
        gpix = gsel[a].astype(np.float64)[:, None] * z64 / mag[:, None]   # [3, 2]
        gspecs.append(np.broadcast_to(gpix[:, None, None, None, :], (len(js), g.H, g.W, 1, 2)))

    d_rad = torch.zeros((N, K, 1, 2), device="cuda")
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_RSSI, radiance=rad, grad_rssi=dev(grad_rssi, torch),
                        fwd_csi=dev(fwd_csi, torch), grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    ref_r = ref_t = abs_r = abs_t = None
    for a, v in enumerate(vs):
        gr, gt, ar, at = oracle.backward_view(g, sc, tx[v], rad_s, gspecs[a], want_abs=True)
        ref_r = gr if ref_r is None else ref_r + gr
        ref_t = gt if ref_t is None else ref_t + gt
        abs_r = ar if abs_r is None else abs_r + ar
        abs_t = at if abs_t is None else abs_t + at
    got_r = d_rad[js].cpu().numpy().astype(np.float64)
    e_r = float((np.abs(got_r - ref_r) / (abs_r + 1e-30)).max())
    e_t = float((np.abs(d_tau.cpu().numpy() - ref_t) / (abs_t + 1e-30)).max())
    assert e_r <= TOL, e_r
    assert e_t <= TOL, e_t
    # receivers with a zero cotangent get exactly zero radiance gradient
    assert float(d_rad[[1, 300, 1000]].abs().max()) == 0.0
    ctx.release_views(views)
