"""Occlusion inputs of the local conditioning branch (App. E.5): occupancy
grid splat and 16 probes per (Gaussian, receiver) segment feed T and
rho_bar to the local MLP; forward spectra and the backward through the MLP
against the oracle, removal of the grid, and the paths that refuse it."""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.test_gpu_backward import check_mlp_grads
from tests.gpu_helpers import TOL, dev, norm_err, upload

pytestmark = pytest.mark.gpu
RES = 32


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a GPU"
    return t


@pytest.fixture(scope="module")
def rx():
    from paper_2605_24290_gb300 import rxgs
    return rxgs


def scene_with_occlusion(rng, K):
    # a small box and larger Gaussians, so that the probes see density
    sc = S.draw_scene(rng, K, box=(4.0, 4.0, 2.0), log_scale_mean=-1.2, log_scale_std=0.3)
    return sc


@pytest.mark.parametrize("C", [1, 3])
def test_occupancy_forward_and_backward_match_oracle(torch, rx, oracle, C):
    rng = np.random.default_rng(900 + C)
    K, M, N = 1500, 2, 6
    sc = scene_with_occlusion(rng, K)
    base, mlp = S.draw_base(rng, K, C), S.draw_mlp(rng, C)
    flat = S.flatten_mlp(mlp, C)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, base=base, mlp_flat=flat, C=C)
    ctx.build_occupancy(h, RES)
    tx = S.draw_points(rng, M, box=(4.0, 4.0, 2.0))
    rxp = S.draw_points(rng, N, box=(4.0, 4.0, 2.0))
    views = ctx.prepare(h, dev(tx, torch))
    rxd = dev(rxp, torch)
    spec = torch.zeros((M, N, g.H, g.W, C, 2), device="cuda")
    ctx.render_views(views, rxd, N, rx.OUT_SPECTRA, spectra=spec)
    gs = rng.normal(size=(M, N, g.H, g.W, C, 2)).astype(np.float32)
    d_tau = torch.zeros(K, device="cuda")
    d_base = torch.zeros((K, C, 2), device="cuda")
    d_mlp = torch.zeros(flat.shape[0], device="cuda")
    ctx.render_backward(views, rxd, N, rx.OUT_SPECTRA, grad_spectra=dev(gs, torch),
                        grad_opacity=d_tau, grad_base=d_base, grad_mlp=d_mlp)
    ctx.sync()
    occ = oracle.occupancy_grid(sc, RES)
    T, rb = oracle.occupancy_probes(occ, rxp, sc.means)
    assert T.min() < 0.5 and rb.max() > 0.05, "the probes should see occupancy"
    rad = oracle.mlp_radiance(mlp, rxp, sc.means, base, occ=occ)
    ref_r = np.zeros(rad.shape)
    abs_r = np.zeros(rad.shape)
    for v in range(M):
        o = oracle.render_view(g, sc, tx[v], rad)
        assert norm_err(spec[v].cpu().numpy(), o["spectra"], o["absacc"]) <= TOL
        gr, gt, ar, at = oracle.backward_view(g, sc, tx[v], rad, gs[v].astype(np.float64),
                                              want_abs=True)
        ref_r += gr
        abs_r += ar
    ref = oracle.mlp_backward(mlp, rxp, sc.means, base, ref_r, occ=occ)
    got = S.unflatten_mlp(d_mlp.cpu().numpy(), C)
    check_mlp_grads(oracle, mlp, rxp, sc.means, base, abs_r, ref, d_base.cpu().numpy(), got,
                    occ=occ)
    ctx.release_views(views)


def test_occupancy_removal_and_refusals(torch, rx):
    rng = np.random.default_rng(910)
    K, N = 800, 4
    sc = scene_with_occlusion(rng, K)
    base, mlp = S.draw_base(rng, K, 1), S.draw_mlp(rng, 1)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch, base=base, mlp_flat=S.flatten_mlp(mlp, 1), C=1)
    tx = dev(S.draw_points(rng, 1, box=(4.0, 4.0, 2.0)), torch)
    rxd = dev(S.draw_points(rng, N, box=(4.0, 4.0, 2.0)), torch)
    clear = torch.zeros((1, N), device="cuda")
    ctx.render(h, tx, rxd, N, rx.OUT_RSSI, rssi=clear)
    ctx.build_occupancy(h, RES)
    occl = torch.zeros((1, N), device="cuda")
    ctx.render(h, tx, rxd, N, rx.OUT_RSSI, rssi=occl)
    with pytest.raises(rx.RxgsError):
        ctx.render(h, tx, rxd, N, rx.OUT_RSSI, rssi=occl, reduce_path=1)
    with pytest.raises(rx.RxgsError):
        ctx.render_batched(h, tx, rxd, [N], rx.OUT_RSSI, rssi=occl)
    with pytest.raises(rx.RxgsError):
        ctx.serve_start(h, kind=rx.OUT_RSSI)
    ctx.build_occupancy(h, 0)
    again = torch.zeros((1, N), device="cuda")
    ctx.render(h, tx, rxd, N, rx.OUT_RSSI, rssi=again)
    ctx.sync()
    assert not torch.equal(clear, occl)
    assert torch.equal(clear, again)
    with pytest.raises(rx.RxgsError):
        ctx.build_occupancy(h, 1000)
