"""Stage II training step: the L1 loss against targets rendered from other
(phi_base, MLP) parameters falls under Adam, for spectra and for RSSI, and a
step's gradient equals the render backward's."""
import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S
from tests.gpu_helpers import dev, upload

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


def setup(torch, rx, seed):
    from paper_2605_24290_gb300 import autograd as AG
    rng = np.random.default_rng(seed)
    K, C = 2000, 1
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    true_base, true_mlp = S.draw_base(rng, K, C), S.draw_mlp(rng, C)
    h = upload(ctx, sc, torch, base=true_base, mlp_flat=S.flatten_mlp(true_mlp, C), C=C)
    tx, rxp = dev(S.draw_points(rng, 2), torch), dev(S.draw_points(rng, 4), torch)
    op = dev(sc.opacity, torch)
    with torch.no_grad():
        spec, rssi, _ = AG.render(ctx, h, tx, rxp, 4, op, base=dev(true_base, torch),
                                  mlp=dev(S.flatten_mlp(true_mlp, C), torch),
                                  kind=rx.OUT_SPECTRA | rx.OUT_RSSI)
        amp = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
    start_base = S.draw_base(rng, K, C)
    start_mlp = S.draw_mlp(rng, C)
    return ctx, h, op, tx, rxp, amp.clone(), rssi.clone(), dev(start_base, torch), \
        dev(S.flatten_mlp(start_mlp, C), torch)


@pytest.mark.parametrize("target_kind", ["spectra", "rssi"])
def test_stage2_loss_falls(torch, rx, target_kind):
    from paper_2605_24290_gb300.train import Stage2Trainer
    ctx, h, op, tx, rxp, amp, rssi, b0, m0 = setup(torch, rx, 801)
    tr = Stage2Trainer(ctx, h, op, b0, m0, lr_base=2e-2, lr_mlp=2e-3)
    kind = rx.OUT_SPECTRA if target_kind == "spectra" else rx.OUT_RSSI
    target = amp if target_kind == "spectra" else rssi
    losses = [float(tr.step(tx, rxp, target, kind)) for _ in range(25)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0], losses


def test_stage2_gradient_is_the_render_backward(torch, rx):
    """d(L1)/d(phi_base) from the trainer equals the render backward driven
    by the L1 loss's cotangent sign(|R| - y) d|R|/dR."""
    from paper_2605_24290_gb300.train import Stage2Trainer
    ctx, h, op, tx, rxp, amp, rssi, b0, m0 = setup(torch, rx, 802)
    tr = Stage2Trainer(ctx, h, op, b0, m0)
    loss = tr.loss(tx, rxp, amp)
    loss.backward()
    g_auto = tr.base.grad.detach().clone()
    # the same cotangent by hand, through the ABI
    from paper_2605_24290_gb300 import autograd as AG
    with torch.no_grad():
        spec, _, _ = AG.render(ctx, h, tx, rxp, 4, op, base=tr.base.detach(), mlp=tr.mlp.detach())
        a = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
        gs = (torch.sign(a - amp) / a.numel())[..., None] * spec / a[..., None]
    ctx.update_scene(h, opacity=op, base=tr.base.detach(), mlp=tr.mlp.detach())
    views = ctx.prepare(h, tx)
    d_base = torch.zeros_like(tr.base)
    d_op = torch.zeros_like(op)
    d_mlp = torch.zeros_like(tr.mlp)
    ctx.render_backward(views, rxp, 4, rx.OUT_SPECTRA, grad_spectra=gs.contiguous(),
                        grad_opacity=d_op, grad_base=d_base, grad_mlp=d_mlp)
    ctx.sync()
    ctx.release_views(views)
    torch.testing.assert_close(g_auto, d_base, rtol=1e-4, atol=1e-7)


def setup_fle(torch, rx, seed, lmax=3):
    """Targets rendered from a 'true' base / FiLM; training starts from other
    base coefficients and a FiLM whose final layer is zero (App. E.4)."""
    from paper_2605_24290_gb300 import autograd as AG
    rng = np.random.default_rng(seed)
    K = 1500
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    tx = dev(S.draw_points(rng, 2), torch)
    rxp = dev(S.f32(rng.uniform(-1.0, 1.0, size=(4, 3))), torch)
    op = dev(sc.opacity, torch)
    true_film = S.draw_film(rng, lmax, F=2, dc=4, D=16)
    dims = rx.film_sizes(true_film)
    with torch.no_grad():
        spec, rssi, _ = AG.render_fle_film(ctx, h, tx, rxp, 4, op,
                                           dev(S.draw_fle_base(rng, K, lmax), torch),
                                           dev(rx.pack_film(true_film), torch), dims, lmax,
                                           kind=rx.OUT_SPECTRA | rx.OUT_RSSI)
        amp = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
    start_film = S.draw_film(rng, lmax, F=2, dc=4, D=16)
    start_film["w3"][:] = 0.0
    start_film["b3"][:] = 0.0
    return (ctx, h, op, tx, rxp, amp.clone(), rssi.clone(),
            dev(S.draw_fle_base(rng, K, lmax), torch), dev(rx.pack_film(start_film), torch),
            dims, lmax)


def test_fle_stage2_loss_falls(torch, rx):
    from paper_2605_24290_gb300.train import FleStage2Trainer
    ctx, h, op, tx, rxp, amp, rssi, b0, f0, dims, lmax = setup_fle(torch, rx, 803)
    tr = FleStage2Trainer(ctx, h, op, b0, f0, dims, lmax, lr_base=2e-2, lr_film=2e-3)
    losses = [float(tr.step(tx, rxp, amp)) for _ in range(25)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.9 * losses[0], losses
    # the FiLM parameters moved off their zero final layer
    w3 = rx.unpack_film(tr.film.detach().cpu().numpy(), *dims, lmax)["w3"]
    assert float(np.abs(w3).max()) > 0.0


def test_fle_stage2_gradient_is_the_render_backward(torch, rx):
    """The trainer's gradients of the base coefficients and the FiLM
    parameters equal the render backward driven by the L1 cotangent."""
    from paper_2605_24290_gb300.train import FleStage2Trainer
    from paper_2605_24290_gb300 import autograd as AG
    ctx, h, op, tx, rxp, amp, rssi, b0, f0, dims, lmax = setup_fle(torch, rx, 804)
    f0 = f0 + 0.05 * torch.randn(f0.shape, device="cuda", generator=torch.Generator(
        device="cuda").manual_seed(5))                       # a non-zero final layer
    tr = FleStage2Trainer(ctx, h, op, b0, f0, dims, lmax)
    loss = tr.loss(tx, rxp, amp)
    loss.backward()
    g_base = torch.cat([tr.base_dc.grad, tr.base_rest.grad], dim=2)
    g_film = tr.film.grad.detach().clone()
    with torch.no_grad():
        spec, _, _ = AG.render_fle_film(ctx, h, tx, rxp, 4, op, tr.base().detach(),
                                        tr.film.detach(), dims, lmax)
        a = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
        gs = (torch.sign(a - amp) / a.numel())[..., None] * spec / a[..., None]
    views = ctx.prepare(h, tx)
    d_base = torch.zeros_like(g_base)
    d_film = torch.zeros_like(g_film)
    d_op = torch.zeros_like(op)
    ctx.render_backward(views, rxp, 4, rx.OUT_SPECTRA, grad_spectra=gs.contiguous(),
                        grad_opacity=d_op, fle_lmax=lmax, fle_base=tr.base().detach(),
                        film=tr.film.detach().contiguous(), film_dims=dims,
                        grad_fle_base=d_base, grad_film=d_film)
    ctx.sync()
    ctx.release_views(views)
    for got, ref in ((g_base, d_base), (g_film, d_film)):
        m = float(ref.abs().max())
        assert m > 0.0
        assert float((got - ref).abs().max()) <= 1e-5 * m
