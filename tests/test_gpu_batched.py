"""Uneven receiver batches in one persistent launch under a CUDA graph:
every batch's results equal those of rendering that batch alone, and a
second batch with other sizes replays the same graph correctly."""
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


def alone(ctx, rxm, torch, h, txv, rxv, rad, kind, C, H, W):
    n = rxv.shape[0] if rxv is not None else rad.shape[0]
    spec = torch.zeros((1, n, H, W, C, 2), device="cuda")
    csi = torch.zeros((1, n, C, 2), device="cuda")
    rssi = torch.zeros((1, n), device="cuda") if C == 1 else None
    ctx.render(h, dev(txv[None], torch), None if rxv is None else dev(rxv, torch), n, kind,
               radiance=None if rad is None else dev(rad, torch), spectra=spec, csi=csi, rssi=rssi)
    return spec[0], csi[0], (rssi[0] if rssi is not None else None)


@pytest.mark.parametrize("C", [1, 3])
def test_batched_explicit_radiance_matches_single_batches(torch, rx, C):
    rng = np.random.default_rng(401)
    sc = S.draw_scene(rng, 3000)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W, cols_per_cta=64)
    h = upload(ctx, sc, torch, C=C)
    kind = rx.OUT_SPECTRA | rx.OUT_CSI | (rx.OUT_RSSI if C == 1 else 0)
    for counts in ([5, 1, 9], [2, 7], [1, 1, 1, 12, 3]):
        B, R = len(counts), sum(counts)
        tx = S.draw_points(rng, B)
        rad = S.draw_radiance(rng, R, sc.K, C)
        spec = torch.zeros((R, g.H, g.W, C, 2), device="cuda")
        csi = torch.zeros((R, C, 2), device="cuda")
        rssi = torch.zeros((R,), device="cuda") if C == 1 else None
        ctx.render_batched(h, dev(tx, torch), None, counts, kind, radiance=dev(rad, torch),
                           spectra=spec, csi=csi, rssi=rssi)
        ctx.sync()
        off = 0
        for b, n in enumerate(counts):
            s1, c1, r1 = alone(ctx, rx, torch, h, tx[b], None, rad[off:off + n], kind, C, g.H, g.W)
            ctx.sync()
            np.testing.assert_array_equal(spec[off:off + n].cpu().numpy().view(np.uint32),
                                          s1.cpu().numpy().view(np.uint32))
            np.testing.assert_array_equal(csi[off:off + n].cpu().numpy(), c1.cpu().numpy())
            if C == 1:
                np.testing.assert_array_equal(rssi[off:off + n].cpu().numpy(), r1.cpu().numpy())
            off += n


def test_batched_mlp_matches_single_batches_and_oracle(torch, rx, oracle):
    rng = np.random.default_rng(402)
    K, C = 3000, 1
    sc = S.draw_scene(rng, K)
    base = S.draw_base(rng, K, C)
    mlp = S.draw_mlp(rng, C)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W, cols_per_cta=64)
    h = upload(ctx, sc, torch, base=base, mlp_flat=S.flatten_mlp(mlp, C), C=C)
    counts = [3, 6, 1]
    B, R = len(counts), sum(counts)
    tx, rxp = S.draw_points(rng, B), S.draw_points(rng, R)
    kind = rx.OUT_CSI | rx.OUT_RSSI
    csi = torch.zeros((R, C, 2), device="cuda")
    rssi = torch.zeros((R,), device="cuda")
    ctx.render_batched(h, dev(tx, torch), dev(rxp, torch), counts, kind, csi=csi, rssi=rssi,
                       reduce_path=0)
    ctx.sync()
    off = 0
    for b, n in enumerate(counts):
        _, c1, r1 = alone(ctx, rx, torch, h, tx[b], rxp[off:off + n], None, kind, C, g.H, g.W)
        ctx.sync()
        np.testing.assert_array_equal(csi[off:off + n].cpu().numpy(), c1.cpu().numpy())
        np.testing.assert_array_equal(rssi[off:off + n].cpu().numpy(), r1.cpu().numpy())
        rad = oracle.mlp_radiance(mlp, rxp[off:off + n], sc.means, base)
        o = oracle.render_view(g, sc, tx[b], rad)
        ref = oracle.csi(o["spectra"])
        a = o["absacc"].sum(axis=(1, 2))
        assert norm_err(csi[off:off + n].cpu().numpy(), ref, a) <= TOL
        off += n


def test_autotune_keeps_spectra(torch, rx, oracle):
    """The autotuner only moves work between CTAs: spectra after tuning equal
    those before (bit for bit when both runs composite on the CUDA cores;
    within the parity tolerance of the oracle's absolute chain when one of
    them takes the 128-column tensor-core product)."""
    rng = np.random.default_rng(403)
    sc = S.draw_scene(rng, 3000)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    tx = dev(S.draw_points(rng, 2), torch)
    rad = dev(S.draw_radiance(rng, 24, sc.K, 1), torch)
    before = torch.zeros((2, 24, g.H, g.W, 1, 2), device="cuda")
    ctx.render(h, tx, None, 24, rx.OUT_SPECTRA, radiance=rad, spectra=before)
    res = ctx.autotune(h, tx, None, 24, rx.OUT_SPECTRA, radiance=rad, iters=2)
    assert len(res["candidates"]) >= 6
    ch = res["chosen"]
    assert any(c["tile"] == ch["tile"] and c["cols"] == ch["cols"] for c in res["candidates"])
    after = torch.zeros_like(before)
    ctx.render(h, tx, None, 24, rx.OUT_SPECTRA, radiance=rad, spectra=after)
    ctx.sync()
    b_np, a_np = before.cpu().numpy(), after.cpu().numpy()
    if ch["cols"] < 128:
        np.testing.assert_array_equal(b_np.view(np.uint32), a_np.view(np.uint32))
    else:
        rad_np, tx_np = rad.cpu().numpy().astype(np.float64), tx.cpu().numpy()
        for v in range(2):
            o = oracle.render_view(g, sc, tx_np[v], rad_np)
            assert norm_err(a_np[v], b_np[v], o["absacc"]) <= TOL
