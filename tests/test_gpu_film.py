"""Global FiLM branch over the FLE components (Eq. rx_enc, film, film_apply):
the per-(receiver, component) modulation against the oracle, the
FiLM-conditioned FLE render (forward and backward to the base coefficients,
every FiLM parameter and the opacity) against the oracle, and the
zero-initialised final layer reproducing the unconditioned path bit for bit."""
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


def film_chain(oracle, film, r, lmax):
    """The absolute chain |W3| (|W2| (|W1| |x| + |b1|) + |b2|) + |b3| of every
    output, the scale of its float32 rounding.  With the frequency vectors at
    their initial values (one non-zero entry per vector, a power of two) the
    float32 phase w.r is exact, so the encoding carries only the rounding of
    sinf / cosf (a few 2^-24) and the error stays a small multiple of
    (din + 2 D) 2^-24 of this chain."""
    P = {k: np.asarray(v, np.float64) for k, v in film.items()}
    om = P["omega"]
    nz = (om != 0).sum(axis=1)
    mant = np.frexp(np.abs(om).max(axis=1))[0]
    assert bool(np.all(nz == 1) and np.all(mant == 0.5)), "phases are exact only for 2^f axis vectors"
    x = oracle.film_inputs(P, r, lmax)
    A1, A2, A3 = np.abs(P["w1"]), np.abs(P["w2"]), np.abs(P["w3"])
    return ((np.abs(x) @ A1.T + np.abs(P["b1"])) @ A2.T + np.abs(P["b2"])) @ A3.T + np.abs(P["b3"])


@pytest.mark.parametrize("F,dc,D,lmax", [(6, 16, 64, 9), (5, 16, 256, 4), (1, 0, 3, 0)])
def test_film_eval_matches_oracle(torch, rx, oracle, F, dc, D, lmax):
    """Receivers across the room (10 x 8 x 3 m) and the frequency vectors at
    their initial 2^f spacing (App. E.4 sizes: F = 6 or 5, d_c = 16, d = 64 or 256)."""
    rng = np.random.default_rng(800 + D)
    N = 64
    film = S.draw_film(rng, lmax, F=F, dc=dc, D=D, out_scale=1.0)
    r = S.draw_points(rng, N)
    ctx = rx.Context()
    dims = rx.film_sizes(film)
    L = (lmax + 1) ** 2
    ab = torch.zeros((N, L, 4), device="cuda")
    ctx.film_eval(dev(rx.pack_film(film), torch), dims, lmax, dev(r, torch), N, ab)
    ctx.sync()
    ref = oracle.film_global(film, r, lmax)
    chain = film_chain(oracle, film, r.astype(np.float64), lmax)
    err = float((np.abs(ab.cpu().numpy() - ref) / chain).max())
    assert err <= TOL, err


def _render_case(torch, rx, oracle, seed, K, M, N, lmax, F, dc, D, zero_final=False):
    rng = np.random.default_rng(seed)
    sc = S.draw_scene(rng, K)
    tx = S.draw_points(rng, M)
    r = S.f32(rng.uniform(-1.0, 1.0, size=(N, 3)))
    film = S.draw_film(rng, lmax, F=F, dc=dc, D=D, out_scale=1.0)
    if zero_final:
        film["w3"][:] = 0.0
        film["b3"][:] = 0.0
    base = S.draw_fle_base(rng, K, lmax)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    return rng, sc, tx, r, film, base, g, ctx, views


def test_film_render_forward_and_backward_match_oracle(torch, rx, oracle):
    K, M, N, lmax = 1500, 2, 5, 3
    rng, sc, tx, r, film, base, g, ctx, views = _render_case(torch, rx, oracle, 810, K, M, N,
                                                              lmax, F=2, dc=4, D=16)
    dims = rx.film_sizes(film)
    fd = dev(rx.pack_film(film), torch)
    bd, rd = dev(base, torch), dev(r, torch)
    spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    ctx.render_views(views, rd, N, rx.OUT_SPECTRA | rx.OUT_CSI, spectra=spec, csi=csi,
                     fle_lmax=lmax, fle_base=bd, film=fd, film_dims=dims)
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    d_base = torch.zeros_like(bd)
    d_film = torch.zeros_like(fd)
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, rd, N, rx.OUT_SPECTRA, grad_spectra=dev(gs, torch),
                        grad_opacity=d_tau, fle_lmax=lmax, fle_base=bd, film=fd, film_dims=dims,
                        grad_fle_base=d_base, grad_film=d_film)
    ctx.sync()
    coeffs = oracle.film_fle_coeffs(film, base, r, lmax)
    ab = oracle.film_global(film, r, lmax)
    amod = np.hypot(1.0 + ab[..., 0], ab[..., 1])                       # |1 + a| [N, L]
    gc = np.zeros(coeffs.shape)
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
        gc += oracle.fle_backward(gr, sc.means, tx[v], lmax)
        Ya = np.abs(oracle.fle_basis(sc.means, tx[v], lmax))
        scale_c += (ar[:, :, 0, 0] + ar[:, :, 0, 1])[:, :, None, None] * Ya[None, :, None, :]
        ref_t += gt
        abs_t += at
    ref = oracle.film_fle_backward(film, base, r, lmax, gc)
    # base: dL/dphi_kl = sum_j conj(1 + a_jl) G_jkl, scale sum_j |1 + a_jl| |G|-chain
    scale_b = (amod[:, None, None, :] * scale_c).sum(axis=0)
    e_b = float((np.abs(d_base.cpu().numpy() - ref["base"]) / (scale_b + 1e-30)).max())
    assert e_b <= TOL, e_b
    e_t = float((np.abs(d_tau.cpu().numpy() - ref_t) / (abs_t + 1e-30)).max())
    assert e_t <= TOL, e_t
    # FiLM parameters: relative to each tensor's largest entry
    got = rx.unpack_film(d_film.cpu().numpy(), *dims, lmax)
    for k in rx.FILM_FIELDS:
        m = float(np.abs(ref[k]).max())
        if m == 0.0:
            assert float(np.abs(got[k]).max()) == 0.0, k
            continue
        e = float(np.abs(got[k] - ref[k]).max()) / m
        assert e <= TOL, (k, e)
    ctx.release_views(views)


def test_film_paper_sizes_csi_gradients(torch, rx, oracle):
    """App. E.4 sizes (F = 6, d_c = 16, d = 64, lmax = 9) through a CSI
    cotangent, with 33 receivers (a second pass of 32 in the backward)."""
    K, M, N, lmax = 400, 2, 33, 9
    rng, sc, tx, r, film, base, g, ctx, views = _render_case(torch, rx, oracle, 820, K, M, N,
                                                              lmax, F=6, dc=16, D=64)
    dims = rx.film_sizes(film)
    fd = dev(rx.pack_film(film), torch)
    bd, rd = dev(base, torch), dev(r, torch)
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd, film=fd,
                     film_dims=dims)
    gcs = rng.normal(size=(M, N, 1, 2)).astype(np.float32)
    d_base = torch.zeros_like(bd)
    d_film = torch.zeros_like(fd)
    ctx.render_backward(views, rd, N, rx.OUT_CSI, grad_csi=dev(gcs, torch), fle_lmax=lmax,
                        fle_base=bd, film=fd, film_dims=dims, grad_fle_base=d_base,
                        grad_film=d_film)
    ctx.sync()
    coeffs = oracle.film_fle_coeffs(film, base, r, lmax)
    ab = oracle.film_global(film, r, lmax)
    amod = np.hypot(1.0 + ab[..., 0], ab[..., 1])
    gc = np.zeros(coeffs.shape)
    scale_c = np.zeros(coeffs.shape)
    for v in range(M):
        rad = oracle.fle_radiance(coeffs, sc.means, tx[v], lmax)
        o = oracle.render_view(g, sc, tx[v], rad)
        a = oracle.render_view(g, sc, tx[v], fle_abs_radiance(oracle, coeffs, sc.means, tx[v],
                                                              lmax))["absacc"].sum(axis=(1, 2))
        e = np.abs(csi[v].cpu().numpy() - oracle.csi(o["spectra"])) / (a[..., None] + 1e-30)
        assert float(e.max()) <= TOL, v
        gspec = np.broadcast_to(gcs[v].astype(np.float64)[:, None, None, :, :],
                                (N, g.H, g.W, 1, 2))
        gr, _, ar, _ = oracle.backward_view(g, sc, tx[v], rad, gspec, want_abs=True)
        gc += oracle.fle_backward(gr, sc.means, tx[v], lmax)
        Ya = np.abs(oracle.fle_basis(sc.means, tx[v], lmax))
        scale_c += (ar[:, :, 0, 0] + ar[:, :, 0, 1])[:, :, None, None] * Ya[None, :, None, :]
    ref = oracle.film_fle_backward(film, base, r, lmax, gc)
    scale_b = (amod[:, None, None, :] * scale_c).sum(axis=0)
    e_b = float((np.abs(d_base.cpu().numpy() - ref["base"]) / (scale_b + 1e-30)).max())
    assert e_b <= TOL, e_b
    got = rx.unpack_film(d_film.cpu().numpy(), *dims, lmax)
    for k in rx.FILM_FIELDS:
        m = float(np.abs(ref[k]).max())
        e = float(np.abs(got[k] - ref[k]).max()) / m
        assert e <= TOL, (k, e)
    ctx.release_views(views)


def test_film_zero_final_layer_equals_base_coefficients(torch, rx, oracle):
    """A zero final layer (the initialisation of App. E.4) makes the
    conditioned coefficients the base ones exactly: the spectra equal the
    explicit-coefficient path bit for bit."""
    K, M, N, lmax = 800, 2, 4, 4
    rng, sc, tx, r, film, base, g, ctx, views = _render_case(torch, rx, oracle, 830, K, M, N,
                                                              lmax, F=6, dc=16, D=64,
                                                              zero_final=True)
    dims = rx.film_sizes(film)
    a = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    b = torch.zeros_like(a)
    ctx.render_views(views, dev(r, torch), N, rx.OUT_SPECTRA, spectra=a, fle_lmax=lmax,
                     fle_base=dev(base, torch), film=dev(rx.pack_film(film), torch), film_dims=dims)
    coeffs = np.ascontiguousarray(np.broadcast_to(base[None], (N,) + base.shape))
    ctx.render_views(views, None, N, rx.OUT_SPECTRA, spectra=b, fle_coeffs=dev(coeffs, torch),
                     fle_lmax=lmax)
    ctx.sync()
    assert torch.equal(a, b)
    ctx.release_views(views)


def test_film_arguments_are_checked(torch, rx):
    rng = np.random.default_rng(840)
    sc = S.draw_scene(rng, 300)
    g = S.Grid()
    ctx = rx.Context(H=g.H, W=g.W)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(S.draw_points(rng, 1), torch))
    lmax, N = 2, 3
    film = S.draw_film(rng, lmax, F=2, dc=4, D=8)
    dims = rx.film_sizes(film)
    fd = dev(rx.pack_film(film), torch)
    bd = dev(S.draw_fle_base(rng, sc.K, lmax), torch)
    rd = dev(S.f32(rng.uniform(-1, 1, size=(N, 3))), torch)
    csi = torch.zeros((1, N, 1, 2), device="cuda")
    with pytest.raises(rx.RxgsError):      # no FiLM parameters
        ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd)
    with pytest.raises(rx.RxgsError):      # hidden width out of range
        ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd, film=fd,
                         film_dims=(dims[0], dims[1], 300))
    with pytest.raises(rx.RxgsError):      # explicit and conditioned coefficients together
        ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd, film=fd,
                         film_dims=dims, fle_coeffs=bd)
    with pytest.raises(rx.RxgsError):      # the visibility path takes no FLE radiance
        ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd, film=fd,
                         film_dims=dims, reduce_path=1)
    with pytest.raises(rx.RxgsError):      # receivers are needed for the encoding
        ctx.render_views(views, None, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd,
                         film=fd, film_dims=dims)
    ctx.render_views(views, rd, N, rx.OUT_CSI, csi=csi, fle_lmax=lmax, fle_base=bd, film=fd,
                     film_dims=dims)
    ctx.sync()
    assert bool(torch.isfinite(csi).all())
    ctx.release_views(views)


@pytest.mark.parametrize("occupancy", [False, True])
def test_film_local_branch_matches_oracle(torch, rx, oracle, occupancy):
    """Eq. combined_local over the FLE components: the global FiLM branch and
    the scene MLP's local branch (with the occlusion probes when the scene
    has an occupancy grid) composed per (receiver, Gaussian, component).
    Forward spectra and CSI, and the gradients of the base coefficients, the
    opacity, every FiLM parameter and the local branch against the oracle."""
    K, M, N, lmax = 1200, 2, 4, 3
    rng, sc, tx, r, film, base, g, ctx, views = _render_case(torch, rx, oracle, 820, K, M, N,
                                                              lmax, F=2, dc=4, D=16)
    ctx.release_views(views)
    mlp = S.draw_mlp(rng, 1, final_scale=0.5)
    flat = S.flatten_mlp(mlp, 1)
    h = upload(ctx, sc, torch, base=S.draw_base(rng, K, 1), mlp_flat=flat, C=1)
    occ = None
    if occupancy:
        ctx.build_occupancy(h, 64)
        occ = oracle.occupancy_grid(sc, 64)
    views = ctx.prepare(h, dev(tx, torch))
    dims = rx.film_sizes(film)
    fd = dev(rx.pack_film(film), torch)
    bd, rd = dev(base, torch), dev(r, torch)
    spec = torch.zeros((M, N, g.H, g.W, 1, 2), device="cuda")
    csi = torch.zeros((M, N, 1, 2), device="cuda")
    kw = dict(fle_lmax=lmax, fle_base=bd, film=fd, film_dims=dims, film_local=True)
    ctx.render_views(views, rd, N, rx.OUT_SPECTRA | rx.OUT_CSI, spectra=spec, csi=csi, **kw)
    gs = rng.normal(size=(M, N, g.H, g.W, 1, 2)).astype(np.float32)
    d_base = torch.zeros_like(bd)
    d_film = torch.zeros_like(fd)
    d_mlp = torch.zeros(flat.shape[0], device="cuda")
    d_tau = torch.zeros(K, device="cuda")
    ctx.render_backward(views, rd, N, rx.OUT_SPECTRA, grad_spectra=dev(gs, torch),
                        grad_opacity=d_tau, grad_fle_base=d_base, grad_film=d_film,
                        grad_mlp=d_mlp, **kw)
    ctx.sync()
    mlp64 = {k: v.astype(np.float64) for k, v in mlp.items()}
    coeffs = oracle.film_local_fle_coeffs(film, mlp64, base, r, sc.means, lmax, occ=occ)
    ab = oracle.film_global(film, r, lmax)
    alpha, _ = oracle.local_factors(mlp64, r, sc.means, occ)
    amod = np.hypot(1.0 + ab[..., 0], ab[..., 1])                       # |1 + a| [N, L]
    almod = np.abs(1.0 + alpha)                                          # |1 + alpha| [N, K]
    gc = np.zeros(coeffs.shape)
    scale_c = np.zeros(coeffs.shape)
    ref_t, abs_t = np.zeros(K), np.zeros(K)
    for v in range(M):
        rad = oracle.fle_radiance(coeffs, sc.means, tx[v], lmax)
        o = oracle.render_view(g, sc, tx[v], rad)
        a = oracle.render_view(g, sc, tx[v], fle_abs_radiance(oracle, coeffs, sc.means, tx[v],
                                                              lmax))["absacc"]
        assert norm_err(spec[v].cpu().numpy(), o["spectra"], a) <= TOL
        assert norm_err(csi[v].cpu().numpy(), oracle.csi(o["spectra"]), a.sum(axis=(1, 2))) <= TOL
        gr, gt, ar, at = oracle.backward_view(g, sc, tx[v], rad, gs[v].astype(np.float64),
                                              want_abs=True)
        gc += oracle.fle_backward(gr, sc.means, tx[v], lmax)
        Ya = np.abs(oracle.fle_basis(sc.means, tx[v], lmax))
        scale_c += (ar[:, :, 0, 0] + ar[:, :, 0, 1])[:, :, None, None] * Ya[None, :, None, :]
        ref_t += gt
        abs_t += at
    ref = oracle.film_local_fle_backward(film, mlp64, base, r, sc.means, lmax, gc, occ=occ)
    # base: dL/dphi = sum_j conj(1 + a) conj(1 + alpha) G', scaled by the |.| chain
    scale_b = (amod[:, None, None, :] * almod[:, :, None, None] * scale_c).sum(axis=0)
    e_b = float((np.abs(d_base.cpu().numpy() - ref["base"]) / (scale_b + 1e-30)).max())
    assert e_b <= TOL, e_b
    e_t = float((np.abs(d_tau.cpu().numpy() - ref_t) / (abs_t + 1e-30)).max())
    assert e_t <= TOL, e_t
    got_film = rx.unpack_film(d_film.cpu().numpy(), *dims, lmax)
    got_mlp = S.unflatten_mlp(d_mlp.cpu().numpy(), 1)
    checks = [(got_film[k], ref[k], k) for k in rx.FILM_FIELDS] + \
             [(got_mlp[k], ref[k], k) for k in ("l_w1", "l_b1", "l_w2", "l_b2")]
    for got, want, k in checks:
        m = float(np.abs(want).max())
        assert m > 0.0, k
        e = float(np.abs(got - want).max()) / m
        assert e <= TOL, (k, e)
    for k in ("g_w1", "g_b1", "g_w2", "g_b2"):            # the global MLP branch is not used
        assert float(np.abs(got_mlp[k]).max()) == 0.0, k
    with pytest.raises(rx.RxgsError):                      # film_local needs the FiLM path
        ctx.render_views(views, rd, N, rx.OUT_SPECTRA, spectra=spec, fle_lmax=lmax,
                         fle_coeffs=torch.zeros((N, K, 2, 16), device="cuda"), film_local=True)
    ctx.release_views(views)
