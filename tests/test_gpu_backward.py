"""Backward parity of the CUDA path: gradients to radiance, opacity, phi_base
and the conditioning MLP against the float64 oracle, and directional finite
differences of the GPU forward itself.

Tolerance: |g_gpu - g_ref| <= TOL * A where A is the sum of the absolute
values of every term of the reference gradient (the oracle's abs_* scales):
the float32 error of a sum of terms is bounded by a small multiple of
2^-24 times that sum, so 1e-4 is far above it and far below any
structural mistake (a wrong sign, a missing term).
"""
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


def ctx_for(rx, g):
    return rx.Context(H=g.H, W=g.W, theta0_deg=g.theta0_deg, step_deg=g.step_deg, tile_h=g.tile_h,
                      tile_w=g.tile_w, eps_T=g.eps_T, q_max=g.q_max, r_near=g.r_near)


def scaled_err(got, ref, scale):
    got, ref, scale = (np.asarray(x, np.float64) for x in (got, ref, scale))
    return float((np.abs(got - ref) / (scale + 1e-30)).max())


def oracle_grads(oracle, g, sc, tx, rad, gspec):
    """Sum over views of the oracle backward: (grad_rad, grad_tau, abs_rad, abs_tau)."""
    tot = None
    for v in range(tx.shape[0]):
        r = oracle.backward_view(g, sc, tx[v], rad, gspec[v], want_abs=True)
        tot = list(r) if tot is None else [a + b for a, b in zip(tot, r)]
    return tot


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_backward_explicit_radiance(torch, rx, oracle, tile):
    """Cotangent on spectra, two transmitters, 8 receivers."""
    rng = np.random.default_rng(201)
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    g.tile_h, g.tile_w = tile
    tx = np.concatenate([w["tx"], S.draw_points(rng, 1)])
    rad = w["radiance"]
    M, N, K = tx.shape[0], rad.shape[0], sc.K
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    radd = dev(rad, torch)
    spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_SPECTRA, radiance=radd, spectra=spec)
    d_rad = torch.zeros_like(radd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_SPECTRA, radiance=radd, grad_spectra=dev(gs, torch),
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gs.astype(np.float64))
    e_r = scaled_err(d_rad.cpu().numpy(), ref_r, abs_r)
    e_t = scaled_err(d_tau.cpu().numpy(), ref_t, abs_t)
    assert e_r <= TOL, f"radiance gradient error {e_r}"
    assert e_t <= TOL, f"opacity gradient error {e_t}"
    assert np.abs(ref_t).max() > 0


@pytest.mark.parametrize("N", [64, 40, 100])
@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_backward_wide_blocks_tensor_cores(torch, rx, oracle, N, tile):
    """Column blocks of 128 (2NC > 64) take the tensor-core sweep: 64
    receivers fill one block exactly (the benchmark's width), 40 leave 48
    padding columns, 100 need two blocks (the second ragged).  Forward spectra
    (the tensor-core forward) and both gradients against the oracle."""
    rng = np.random.default_rng(206 + N)
    K = 2500
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    g.tile_h, g.tile_w = tile
    tx = S.draw_points(rng, 2)
    rad = S.draw_radiance(rng, N, K, 1)
    M = 2
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    radd = dev(rad, torch)
    spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_SPECTRA | rx.OUT_CSI, radiance=radd, spectra=spec,
                     csi=csi)
    d_rad = torch.zeros_like(radd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_SPECTRA, radiance=radd, grad_spectra=dev(gs, torch),
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    for v in range(M):
        o = oracle.render_view(g, sc, tx[v], rad.astype(np.float64))
        assert norm_err(spec[v].cpu().numpy(), o["spectra"], o["absacc"]) <= TOL
        a = o["absacc"].sum(axis=(1, 2))
        assert norm_err(csi[v].cpu().numpy(), oracle.csi(o["spectra"]), a) <= TOL
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gs.astype(np.float64))
    e_r = scaled_err(d_rad.cpu().numpy(), ref_r, abs_r)
    e_t = scaled_err(d_tau.cpu().numpy(), ref_t, abs_t)
    assert e_r <= TOL, f"radiance gradient error {e_r}"
    assert e_t <= TOL, f"opacity gradient error {e_t}"
    assert np.abs(ref_t).max() > 0 and np.abs(ref_r).max() > 0


def test_backward_reuses_the_forward_stops(torch, rx, oracle):
    """A 128-column forward leaves each pixel's stop and final transmittance
    on the views; the backward then skips its re-walk.  The gradients with
    that state equal, within float-atomic reordering, those of a backward on
    freshly prepared views that never saw a forward, and both match the
    oracle (two views, 64 receivers, 8x32 tiles, an early-stopping eps)."""
    rng = np.random.default_rng(231)
    K, N, M = 3000, 64, 2
    sc = S.draw_scene(rng, K)
    g = S.Grid()
    g.tile_h, g.tile_w = 8, 32
    g.eps_T = 0.05
    tx = S.draw_points(rng, M)
    rad = S.draw_radiance(rng, N, K, 1)
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch)
    radd, gsd = dev(rad, torch), dev(gs, torch)
    grads = []
    for with_forward in (True, False):
        views = ctx.prepare(h, dev(tx, torch))
        if with_forward:
            spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
            ctx.render_views(views, None, N, rx.OUT_SPECTRA, radiance=radd, spectra=spec)
        d_rad = torch.zeros_like(radd)
        d_tau = torch.zeros(K, device="cuda")
        ctx.render_backward(views, None, N, rx.OUT_SPECTRA, radiance=radd, grad_spectra=gsd,
                            grad_radiance=d_rad, grad_opacity=d_tau)
        ctx.sync()
        grads.append((d_rad.cpu().numpy(), d_tau.cpu().numpy()))
        ctx.release_views(views)
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gs.astype(np.float64))
    for d_r, d_t in grads:
        assert scaled_err(d_r, ref_r, abs_r) <= TOL
        assert scaled_err(d_t, ref_t, abs_t) <= TOL
    # the same stops: only the atomics' order differs
    assert scaled_err(grads[0][0], grads[1][0], abs_r) <= 1e-6
    assert scaled_err(grads[0][1], grads[1][1], abs_t) <= 1e-6


def test_backward_csi_and_rssi_cotangents(torch, rx, oracle):
    """dL/dCSI and dL/dRSSI act as pixel-uniform cotangents on the spectra."""
    rng = np.random.default_rng(202)
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    tx, rad = w["tx"], w["radiance"]
    M, N, K = 1, rad.shape[0], sc.K
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    radd = dev(rad, torch)
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    rssi = torch.zeros((M, N), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_CSI | rx.OUT_RSSI, radiance=radd, csi=csi, rssi=rssi)
    gc = rng.normal(size=(M, N, 1, 2)).astype(np.float32)
    gr = rng.normal(size=(M, N)).astype(np.float32)
    d_rad = torch.zeros_like(radd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_CSI | rx.OUT_RSSI, radiance=radd,
                        grad_csi=dev(gc, torch), grad_rssi=dev(gr, torch), fwd_csi=csi,
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    o = oracle.render_view(g, sc, tx[0], rad.astype(np.float64))
    S_ = oracle.csi(o["spectra"])[:, 0, :]                    # [N,2]
    mag = np.sqrt((S_ ** 2).sum(-1, keepdims=True))
    gu = gc[0, :, 0, :].astype(np.float64) + gr[0][:, None] * S_ / mag
    gspec = np.broadcast_to(gu[:, None, None, None, :], (N, g.H, g.W, 1, 2)).copy()
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gspec[None])
    assert scaled_err(d_rad.cpu().numpy(), ref_r, abs_r) <= TOL
    assert scaled_err(d_tau.cpu().numpy(), ref_t, abs_t) <= TOL


def test_backward_csi_wide_channels_odd_k(torch, rx, oracle):
    """CSI cotangent with C = 2 and an odd Gaussian count (the
    visibility-weight backward's scalar loads), two views."""
    rng = np.random.default_rng(205)
    K, N, C = 3001, 5, 2
    sc = S.draw_scene(rng, K)
    tx = S.draw_points(rng, 2)
    rad = S.draw_radiance(rng, N, K, C)
    g = S.Grid()
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch, C=C)
    views = ctx.prepare(h, dev(tx, torch))
    radd = dev(rad, torch)
    csi = torch.zeros((2, N, C, 2), device="cuda")
    ctx.render_views(views, None, N, rx.OUT_CSI, radiance=radd, csi=csi, reduce_path=1)
    gc = rng.normal(size=(2, N, C, 2)).astype(np.float32)
    d_rad = torch.zeros_like(radd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, None, N, rx.OUT_CSI, radiance=radd, grad_csi=dev(gc, torch),
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    gspec = np.broadcast_to(gc.astype(np.float64)[:, :, None, None, :, :],
                            (2, N, g.H, g.W, C, 2)).copy()
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gspec)
    assert scaled_err(d_rad.cpu().numpy(), ref_r, abs_r) <= TOL
    assert scaled_err(d_tau.cpu().numpy(), ref_t, abs_t) <= TOL
    for v in range(2):
        o = oracle.render_view(g, sc, tx[v], rad.astype(np.float64))
        a = o["absacc"].sum(axis=(1, 2))
        e = np.abs(csi[v].cpu().numpy() - oracle.csi(o["spectra"])) / (a[..., None] + 1e-30)
        assert float(e.max()) <= TOL


@pytest.mark.parametrize("N,C", [(8, 1), (8, 3), (40, 2), (6, 4), (5, 7), (3, 52)])
def test_backward_through_mlp(torch, rx, oracle, N, C):
    """Cotangent on spectra through the conditioning MLP to phi_base, the MLP
    parameters and the opacity (N * 2C columns: one or two column blocks)."""
    rng = np.random.default_rng(203 + 10 * C + N)
    K, M = 3000, 2
    sc = S.draw_scene(rng, K)
    tx, rxp = S.draw_points(rng, M), S.draw_points(rng, N)
    base = S.draw_base(rng, K, C)
    mlp = S.draw_mlp(rng, C)
    flat = S.flatten_mlp(mlp, C)
    g = S.Grid()
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch, base=base, mlp_flat=flat, C=C)
    views = ctx.prepare(h, dev(tx, torch))
    spec = torch.zeros((M, N, g.H, g.W, C, 2), device="cuda")
    rxd = dev(rxp, torch)
    ctx.render_views(views, rxd, N, rx.OUT_SPECTRA, spectra=spec)
    gs = rng.normal(size=(M, N, g.H, g.W, C, 2)).astype(np.float32)
    d_tau = torch.zeros(K, device="cuda")
    d_base = torch.zeros((K, C, 2), device="cuda")
    d_mlp = torch.zeros(flat.shape[0], device="cuda")
    ctx.render_backward(views, rxd, N, rx.OUT_SPECTRA, grad_spectra=dev(gs, torch),
                        grad_opacity=d_tau, grad_base=d_base, grad_mlp=d_mlp)
    ctx.sync()
    rad = oracle.mlp_radiance(mlp, rxp, sc.means, base)
    ref_r, ref_t, abs_r, abs_t = oracle_grads(oracle, g, sc, tx, rad, gs.astype(np.float64))
    assert scaled_err(d_tau.cpu().numpy(), ref_t, abs_t) <= TOL
    ref = oracle.mlp_backward(mlp, rxp, sc.means, base, ref_r)
    got_mlp = S.unflatten_mlp(d_mlp.cpu().numpy(), C)
    check_mlp_grads(oracle, mlp, rxp, sc.means, base, abs_r, ref, d_base.cpu().numpy(), got_mlp)


def check_mlp_grads(oracle, mlp, rxp, means, base, abs_r, ref, got_base, got_mlp, occ=None):
    """phi_base and MLP gradients against the oracle relative to the MLP
    backward's absolute chain (the actual ReLU activity, fed by the render
    backward's absolute radiance-gradient terms).  A hidden unit whose
    pre-activation float32 cannot place on one side of zero may be taken
    either way by the GPU: its whole first-layer term is admitted (scaled
    by 1 / TOL in the error scale).  Returns the number of such units."""
    chain, amb = oracle.mlp_backward_chain(mlp, rxp, means, base, abs_r, occ=occ)
    e = scaled_err(got_base, ref["base"], chain["base"])
    assert e <= TOL, f"phi_base gradient {e}"
    for name in mlp:
        e = scaled_err(got_mlp[name], ref[name], chain[name] + amb[name] / TOL)
        assert e <= TOL, f"{name} gradient {e}"
    return int(sum((v > 0).sum() for v in amb.values()))


def test_autograd_function_matches_abi(torch, rx):
    from paper_2605_24290_gb300 import autograd as AG
    rng = np.random.default_rng(204)
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch)
    tx = dev(w["tx"], torch)
    op = dev(sc.opacity, torch).requires_grad_(True)
    rad = dev(w["radiance"], torch).requires_grad_(True)
    spec, _, _ = AG.render(ctx, h, tx, None, 8, op, radiance=rad, kind=rx.OUT_SPECTRA)
    gs = torch.from_numpy(rng.normal(size=tuple(spec.shape)).astype(np.float32)).cuda()
    (spec * gs).sum().backward()
    views = ctx.prepare(h, tx)
    d_rad = torch.zeros_like(rad)
    d_tau = torch.zeros_like(op)
    ctx.render_backward(views, None, 8, rx.OUT_SPECTRA, radiance=rad.detach(), grad_spectra=gs,
                        grad_radiance=d_rad, grad_opacity=d_tau)
    ctx.sync()
    # both runs accumulate with float atomics, so only the rounding order differs
    torch.testing.assert_close(rad.grad, d_rad, rtol=1e-4, atol=1e-5)
    torch.testing.assert_close(op.grad, d_tau, rtol=1e-4, atol=1e-4)


def test_directional_finite_differences_on_gpu(torch, rx):
    """100,000 Gaussians (4 transmitters x 8 receivers), MLP radiance:
    central differences of the GPU forward along random directions over 1,000
    random parameters (400 opacities, 500 phi_base entries, 100 MLP weights)
    against the GPU backward.  L = sum(g * spectra) is evaluated in float64;
    the step sizes keep the float32 rounding of the forward well below the
    measured change."""
    w = S.workload_mlp(M=4, N=8)
    g, sc, C = w["grid"], w["scene"], w["C"]
    rng = np.random.default_rng(205)
    flat = S.flatten_mlp(w["mlp"], C)
    ctx = ctx_for(rx, g)
    h = upload(ctx, sc, torch, base=w["base"], mlp_flat=flat, C=C)
    txd, rxd = dev(w["tx"], torch), dev(w["rx"], torch)
    M, N, K = 4, 8, sc.K
    gs = torch.from_numpy(rng.normal(size=(M, N, g.H, g.W, C, 2)).astype(np.float32)).cuda()
    op0 = dev(sc.opacity, torch)
    base0 = dev(w["base"], torch)
    mlp0 = dev(flat, torch)

    def loss(op, base, mlp):
        ctx.update_scene(h, opacity=op, base=base, mlp=mlp)
        views = ctx.prepare(h, txd)
        spec = torch.zeros((M, N, g.H, g.W, C, 2), device="cuda")
        ctx.render_views(views, rxd, N, rx.OUT_SPECTRA, spectra=spec)
        ctx.release_views(views)
        return float((spec.double() * gs.double()).sum()), spec

    L0, spec0 = loss(op0, base0, mlp0)
    views = ctx.prepare(h, txd)
    d_tau = torch.zeros(K, device="cuda")
    d_base = torch.zeros((K, C, 2), device="cuda")
    d_mlp = torch.zeros_like(mlp0)
    ctx.render_backward(views, rxd, N, rx.OUT_SPECTRA, grad_spectra=gs,
                        grad_opacity=d_tau, grad_base=d_base, grad_mlp=d_mlp)
    ctx.sync()
    ctx.release_views(views)
    ip = torch.from_numpy(rng.choice(K, 400, replace=False)).cuda()
    ib = torch.from_numpy(rng.choice(K * C * 2, 500, replace=False)).cuda()
    # local-branch output weights and biases (they modulate every radiance)
    lw2 = S.mlp_shapes(C)
    off = 0
    offs = {}
    for name, shp in lw2:
        offs[name] = off
        off += int(np.prod(shp))
    cand = np.arange(offs["l_w2"], offs["l_b2"] + 4 * C)
    im = torch.from_numpy(rng.choice(cand, 100, replace=False)).cuda()
    for trial in range(4):
        dp = torch.from_numpy(rng.choice([-1.0, 1.0], 400).astype(np.float32)).cuda()
        db = torch.from_numpy(rng.choice([-1.0, 1.0], 500).astype(np.float32)).cuda()
        dm = torch.from_numpy(rng.choice([-1.0, 1.0], 100).astype(np.float32)).cuda()
        hp, hb, hm = 2e-3, 0.5, 2e-3
        an = (float((d_tau[ip] * dp).double().sum()) * hp + float((d_base.view(-1)[ib] * db).double().sum()) * hb
              + float((d_mlp[im] * dm).double().sum()) * hm)

        def shifted(sign):
            op = op0.clone()
            op[ip] += sign * hp * dp
            bs = base0.clone().view(-1)
            bs[ib] += sign * hb * db
            ml = mlp0.clone()
            ml[im] += sign * hm * dm
            return op, bs.view_as(base0), ml

        opp, bp, mp = shifted(+1)
        opm, bm, mm = shifted(-1)
        # the actual (float32-rounded) steps are what the forward saw
        an = (float((d_tau[ip].double() * (opp[ip] - op0[ip]).double()).sum())
              + float((d_base.view(-1)[ib].double() * (bp.view(-1)[ib] - base0.view(-1)[ib]).double()).sum())
              + float((d_mlp[im].double() * (mp[im] - mlp0[im]).double()).sum()))
        Lp, _ = loss(opp, bp, mp)
        Lm, _ = loss(opm, bm, mm)
        fd = (Lp - Lm) / 2.0
        noise = 64 * 2.0 ** -24 * float((spec0.double() * gs.double()).abs().sum())
        assert abs(fd - an) <= 2e-3 * abs(an) + noise, (trial, fd, an, noise)
    ctx.update_scene(h, opacity=op0, base=base0, mlp=mlp0)
