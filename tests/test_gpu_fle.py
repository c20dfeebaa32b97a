"""Fourier-Legendre directional radiance (App. E.2): per-receiver
coefficients [N,K,2,L] reduced against the transmitter-side basis, then
composited; forward spectra / CSI / RSSI and the backward to the
coefficients and the opacity, against the oracle."""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import TOL, dev, fle_abs_radiance, norm_err, upload

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


def draw_coeffs(rng, N, K, lmax):
    L = (lmax + 1) ** 2
    l_of = np.array([int(np.floor(np.sqrt(i))) for i in range(L)])
    c = rng.normal(size=(N, K, 2, L)) / (1.0 + l_of)[None, None, None, :]
    return c.astype(np.float32)


@pytest.mark.parametrize("lmax", [2, 9])
def test_fle_forward_and_backward_match_oracle(torch, rx, oracle, lmax):
    rng = np.random.default_rng(700 + lmax)
    K, M, N = 2000, 2, 5
    sc = S.draw_scene(rng, K)
    tx = S.draw_points(rng, M)
    coeffs = draw_coeffs(rng, N, K, lmax)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    cd = dev(coeffs, torch)
    spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    rssi = torch.zeros((M, N), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_SPECTRA | rx.OUT_CSI | rx.OUT_RSSI, spectra=spec,
                     csi=csi, rssi=rssi, fle_coeffs=cd, fle_lmax=lmax)
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    d_fle = torch.zeros_like(cd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_SPECTRA, grad_spectra=dev(gs, torch),
                        grad_opacity=d_tau, fle_coeffs=cd, fle_lmax=lmax, grad_fle=d_fle)
    ctx.sync()
    ref_c = np.zeros(coeffs.shape)
    scale_c = np.zeros(coeffs.shape)
    ref_t = np.zeros(K)
    abs_t = np.zeros(K)
    for v in range(M):
        rad = oracle.fle_radiance(coeffs, sc.means, tx[v], lmax)
        o = oracle.render_view(g, sc, tx[v], rad)
        a = oracle.render_view(g, sc, tx[v], fle_abs_radiance(oracle, coeffs, sc.means, tx[v],
                                                              lmax))["absacc"]
        assert norm_err(spec[v].cpu().numpy(), o["spectra"], a) <= TOL
        e = np.abs(csi[v].cpu().numpy() - oracle.csi(o["spectra"])) / (a.sum(axis=(1, 2))[..., None] + 1e-30)
        assert float(e.max()) <= TOL
        gr, gt, ar, at = oracle.backward_view(g, sc, tx[v], rad, gs[v].astype(np.float64),
                                              want_abs=True)
        ref_c += oracle.fle_backward(gr, sc.means, tx[v], lmax)
        Ya = np.abs(oracle.fle_basis(sc.means, tx[v], lmax))          # [K, L]
        sa = (ar[:, :, 0, 0] + ar[:, :, 0, 1])[:, :, None, None] * Ya[None, :, None, :]
        scale_c += sa
        ref_t += gt
        abs_t += at
    e_c = float((np.abs(d_fle.cpu().numpy() - ref_c) / (scale_c + 1e-30)).max())
    e_t = float((np.abs(d_tau.cpu().numpy() - ref_t) / (abs_t + 1e-30)).max())
    assert e_c <= TOL, e_c
    assert e_t <= TOL, e_t
    ctx.release_views(views)


def test_fle_arguments_are_checked(torch, rx):
    rng = np.random.default_rng(710)
    sc = S.draw_scene(rng, 500)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(S.draw_points(rng, 1), torch))
    cd = dev(draw_coeffs(rng, 3, sc.K, 2), torch)
    rssi = torch.zeros((1, 3), device="cuda")
    with pytest.raises(rx.RxgsError):      # the visibility path takes no FLE radiance
        ctx.render_views(views, None, 3, rx.OUT_RSSI, rssi=rssi, reduce_path=1, fle_coeffs=cd,
                         fle_lmax=2)
    with pytest.raises(rx.RxgsError):      # degree out of range
        ctx.render_views(views, None, 3, rx.OUT_RSSI, rssi=rssi, fle_coeffs=cd, fle_lmax=10)
    with pytest.raises(rx.RxgsError):      # radiance and coefficients together
        ctx.render_views(views, None, 3, rx.OUT_RSSI, rssi=rssi, fle_coeffs=cd, fle_lmax=2,
                         radiance=dev(S.draw_radiance(rng, 3, sc.K, 1), torch))
    ctx.render_views(views, None, 3, rx.OUT_RSSI, rssi=rssi, fle_coeffs=cd, fle_lmax=2)
    ctx.sync()
    assert bool(torch.isfinite(rssi).all())


def test_fle_view_and_receiver_groups(torch, rx, oracle):
    """33 transmitters and 65 receivers: the FLE kernels' second group of
    views (32 per pass) and of receivers (64 per pass)."""
    rng = np.random.default_rng(720)
    K, M, N, lmax = 300, 33, 65, 3
    sc = S.draw_scene(rng, K)
    tx = S.draw_points(rng, M)
    coeffs = draw_coeffs(rng, N, K, lmax)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    cd = dev(coeffs, torch)
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_CSI, csi=csi, fle_coeffs=cd, fle_lmax=lmax)
    gc = rng.normal(size=(M, N, 1, 2)).astype(np.float32)
    d_fle = torch.zeros_like(cd)
    ctx.render_backward(views, None, N, rx.OUT_CSI, grad_csi=dev(gc, torch), fle_coeffs=cd,
                        fle_lmax=lmax, grad_fle=d_fle)
    ctx.sync()
    ref_c = np.zeros(coeffs.shape)
    scale_c = np.zeros(coeffs.shape)
    for v in [0, 31, 32]:
        rad = oracle.fle_radiance(coeffs, sc.means, tx[v], lmax)
        o = oracle.render_view(g, sc, tx[v], rad)
        a = oracle.render_view(g, sc, tx[v], fle_abs_radiance(oracle, coeffs, sc.means, tx[v],
                                                              lmax))["absacc"].sum(axis=(1, 2))
        e = np.abs(csi[v].cpu().numpy() - oracle.csi(o["spectra"])) / (a[..., None] + 1e-30)
        assert float(e.max()) <= TOL, v
    # the coefficient gradient over all views (uniform cotangent per view)
    for v in range(M):
        rad = oracle.fle_radiance(coeffs, sc.means, tx[v], lmax)
        gspec = np.broadcast_to(gc[v].astype(np.float64)[:, None, None, :, :],
                                (N, g.H, g.W, 1, 2))
        gr, _, ar, _ = oracle.backward_view(g, sc, tx[v], rad, gspec, want_abs=True)
        ref_c += oracle.fle_backward(gr, sc.means, tx[v], lmax)
        Ya = np.abs(oracle.fle_basis(sc.means, tx[v], lmax))
        scale_c += (ar[:, :, 0, 0] + ar[:, :, 0, 1])[:, :, None, None] * Ya[None, :, None, :]
    e_c = float((np.abs(d_fle.cpu().numpy() - ref_c) / (scale_c + 1e-30)).max())
    assert e_c <= TOL, e_c
    ctx.release_views(views)
