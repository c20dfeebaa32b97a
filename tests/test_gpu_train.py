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


def test_stage2_step_matches_oracle(torch, rx, oracle):
    """One Stage2Trainer step (3,000 Gaussians, 2 transmitters x 4 receivers,
    MLP radiance, 90x360) against the oracle's Stage II step: the L1
    amplitude loss, the gradients of phi_base and of every MLP parameter
    (relative to their absolute chains), Adam's first moments and the
    updated parameters of both optimisers.

    The target is the oracle's starting amplitude scaled by 1 +- (0.3 ... 0.8)
    per element, so no element's |R| - y sign is within float32 reach of a
    flip.  Adam's first update is lr * g / (|g| + eps): where the oracle's
    gradient is larger than twice the admitted gradient error the update must
    agree to float32 rounding; elsewhere it must not exceed the step size."""
    from paper_2605_24290_gb300.train import Stage2Trainer
    from tests.test_gpu_backward import check_mlp_grads, oracle_grads, scaled_err
    from tests.gpu_helpers import TOL
    rng = np.random.default_rng(805)
    K, C, M, N = 3000, 1, 2, 4
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    tx, rxp = S.draw_points(rng, M), S.draw_points(rng, N)
    base0, mlp0 = S.draw_base(rng, K, C), S.draw_mlp(rng, C, final_scale=0.5)
    base64 = base0.astype(np.float64)
    mlp64 = {k: v.astype(np.float64) for k, v in mlp0.items()}
    rad0 = oracle.mlp_radiance(mlp64, rxp, sc.means, base64)
    views0 = [oracle.render_view(g, sc, tx[v], rad0) for v in range(M)]
    amp0 = oracle.amplitude(np.stack([o["spectra"] for o in views0]))
    sgn = np.where(rng.random(amp0.shape) < 0.5, -1.0, 1.0)
    target = S.f32(amp0 * (1.0 + sgn * rng.uniform(0.3, 0.8, size=amp0.shape)))
    lr_b, lr_m = 5e-3, 1e-3
    ref = oracle.stage2_step(g, sc, tx, rxp, base64, mlp64, target.astype(np.float64),
                             lr_base=lr_b, lr_mlp=lr_m)

    ctx = rx.Context(H=g.H, W=g.W)
    flat0 = S.flatten_mlp(mlp0, C)
    h = upload(ctx, sc, torch, base=base0, mlp_flat=flat0, C=C)
    tr = Stage2Trainer(ctx, h, dev(sc.opacity, torch), dev(base0, torch), dev(flat0, torch),
                       lr_base=lr_b, lr_mlp=lr_m)
    loss = float(tr.step(dev(tx, torch), dev(rxp, torch), dev(target, torch)))
    a_amp = np.stack([o["absacc"][..., 0] for o in views0])      # bounds |R| and its error
    assert abs(loss - ref["loss"]) <= TOL * a_amp.mean(), (loss, ref["loss"])

    # gradients: the render backward's absolute terms for the oracle's
    # cotangent, carried through the MLP backward's absolute chain
    _, gspec = oracle.l1_amplitude(ref["spectra"], target.astype(np.float64))
    ref_r, _, abs_r, _ = oracle_grads(oracle, g, sc, tx, rad0, gspec)
    got_gb = tr.base.grad.detach().cpu().numpy()
    got_gm = S.unflatten_mlp(tr.mlp.grad.detach().cpu().numpy(), C)
    check_mlp_grads(oracle, mlp64, rxp, sc.means, base64, abs_r,
                    dict(ref["grad_mlp"], base=ref["grad_base"]), got_gb, got_gm)
    chain, amb = oracle.mlp_backward_chain(mlp64, rxp, sc.means, base64, abs_r)

    def check_update(p0, p_got, p_ref, g_ref, dg, lr, m_got, name):
        p0, p_got, p_ref, g_ref, dg = (np.asarray(x, np.float64).reshape(-1)
                                       for x in (p0, p_got, p_ref, g_ref, dg))
        m_got = np.asarray(m_got, np.float64).reshape(-1)
        assert scaled_err(m_got, 0.1 * g_ref, 0.1 * dg / TOL) <= TOL, f"{name} first moment"
        sure = np.abs(g_ref) > 2.0 * dg
        # float32 rounding of the parameter and of the step, plus the step's
        # sensitivity to the admitted gradient error through Adam's eps:
        # d/dg [g / (|g| + eps)] = eps / (|g| + eps)^2
        eps = 1e-8
        tol = 2e-7 * np.maximum(np.abs(p0), lr) + \
            1.01 * lr * eps * dg / (np.maximum(np.abs(g_ref) - dg, 0.0) + eps) ** 2
        assert np.all(np.abs(p_got - p_ref)[sure] <= tol[sure]), f"{name} update"
        assert np.all(np.abs(p_got - p0)[~sure] <= lr * (1 + 1e-5) + tol[~sure]), f"{name} step"
        return int(sure.sum())

    st_b = tr.opt_base.state[tr.base]
    n_sure = check_update(base0, tr.base.detach().cpu().numpy(), ref["base"], ref["grad_base"],
                          TOL * chain["base"], lr_b, st_b["exp_avg"].cpu().numpy(), "phi_base")
    assert n_sure > 0.5 * base0.size
    st_m = tr.opt_mlp.state[tr.mlp]
    new_m = S.unflatten_mlp(tr.mlp.detach().cpu().numpy(), C)
    m1 = S.unflatten_mlp(st_m["exp_avg"].cpu().numpy(), C)
    for name in mlp0:
        check_update(mlp0[name], new_m[name], ref["params"][name], ref["grad_mlp"][name],
                     TOL * (chain[name] + amb[name] / TOL), lr_m, m1[name], name)


@pytest.mark.parametrize("kind_name", ["OUT_SPECTRA", "OUT_RSSI"])
def test_l1_loss_kernel_matches_oracle(torch, rx, oracle, kind_name):
    """rxgs_l1_loss (one pass: loss and cotangent) against the oracle's L1
    terms on 1,000,003 values, including exact zeros (an empty pixel has
    |R| = 1e-4) and ties |R| = y (sign 0)."""
    rng = np.random.default_rng(806)
    kind = getattr(rx, kind_name)
    n = 1_000_003
    ctx = rx.Context()
    if kind == rx.OUT_SPECTRA:
        vals = rng.normal(size=(n, 2)).astype(np.float32)
        vals[:1000] = 0.0
        y = np.abs(rng.normal(size=n)).astype(np.float32)
        y[:500] = np.sqrt(np.float32(1e-8))            # float32 |R| of an empty pixel
        L_ref, g_ref = oracle.l1_amplitude(vals.astype(np.float64), y.astype(np.float64))
        shape = (n, 2)
    else:
        vals = np.abs(rng.normal(size=n)).astype(np.float32)
        y = np.abs(rng.normal(size=n)).astype(np.float32)
        y[:700] = vals[:700]
        d = vals.astype(np.float64) - y
        L_ref, g_ref = float(np.abs(d).mean()), np.sign(d) / n
        shape = (n,)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(shape, device="cuda")
    ctx.l1_loss(kind, dev(vals, torch), dev(y, torch), loss, grad)
    ctx.sync()
    g = grad.cpu().numpy().astype(np.float64)
    # each |a - y| carries a float32 rounding of a; the mean of n terms in
    # float32 sums adds at most a few ulps per level of the block tree
    scale = np.abs(vals).sum(-1).mean() if kind == rx.OUT_SPECTRA else np.abs(vals).mean()
    assert abs(float(loss.item()) - L_ref) <= 1e-5 * scale + 1e-6 * L_ref
    if kind == rx.OUT_SPECTRA:
        # sign(|R| - y) is decided in float32 on the GPU: where |R| is within
        # float32 reach of y either sign is admitted (the cotangent is bounded)
        a = oracle.amplitude(vals.astype(np.float64))
        sure = np.abs(a - y) > 1e-5 * np.maximum(a, 1e-4)
        np.testing.assert_allclose(g[sure], g_ref[sure], rtol=1e-5, atol=1e-6 / n)
        assert np.all(np.abs(g[~sure]) <= (1 + 1e-5) / n)
    else:
        # float32 differences of float32 values have exact signs
        np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=0)
    ctx.close()
