"""Forward parity of the CUDA path against the CPU oracle.

Index work (projection records, tile sets, sorted lists, tile ranges, the
number of Gaussians composited per pixel, the final transmittance) must be
bit-exact; composited values must be within the normalised tolerance of
gpu_helpers.TOL.
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


def make_ctx(rx, g, **kw):
    return rx.Context(H=g.H, W=g.W, theta0_deg=g.theta0_deg, step_deg=g.step_deg, tile_h=g.tile_h,
                      tile_w=g.tile_w, eps_T=g.eps_T, q_max=g.q_max, r_near=g.r_near, **kw)


def check_views(torch, ctx, oracle, g, scene, tx_np, views, which=None):
    """Records, tile counts, sorted (key, value) lists and tile ranges of the
    prepared views against the oracle's float32 shadow, bit for bit.  Keys:
    the whole array ascends; the low 31 bits of each key are the float32
    bits of the oracle's depth rho of the Gaussian it carries; the high bits
    are one value per (view, tile) list, increasing from list to list."""
    M, K = tx_np.shape[0], scene.K
    T = ((g.H + g.tile_h - 1) // g.tile_h) * ((g.W + g.tile_w - 1) // g.tile_w)
    rec, counts, keys, vals, ranges = ctx.views_export(views, M, K, T)
    torch.cuda.synchronize()
    rec, counts = rec.cpu().numpy(), counts.cpu().numpy()
    vals, ranges = vals.cpu().numpy(), ranges.cpu().numpy()
    keys = keys.cpu().numpy().view(np.uint64)
    assert np.all(keys[1:] >= keys[:-1]), "keys not sorted"
    hi_prev = -1
    for v in range(M):
        for t in range(T):
            s, e = ranges[v, t]
            if e > s:
                hi = keys[s:e] >> np.uint64(31)
                assert np.all(hi == hi[0]) and int(hi[0]) > hi_prev, f"key tile bits, view {v} tile {t}"
                hi_prev = int(hi[0])
    for v in (range(M) if which is None else which):
        _, orec, obox = oracle.project_view32(g, scene, tx_np[v])
        vr = ranges[v]
        used = vr[:, 1] > vr[:, 0]
        vs = int(vr[used, 0].min()) if used.any() else 0
        ve = int(vr[used, 1].max()) if used.any() else 0
        assert ve - vs == int((vr[used, 1] - vr[used, 0]).sum()), f"view {v} not contiguous"
        kv = keys[vs:ve] & np.uint64(0x7FFFFFFF)
        np.testing.assert_array_equal(kv.astype(np.uint32), orec[vals[vs:ve], 6].view(np.uint32),
                                      err_msg=f"depth bits of the keys, view {v}")
        ocnt, olists, ontiles = oracle.tile_lists(g, scene, tx_np[v])
        vis = orec[:, 7] > 0
        np.testing.assert_array_equal(counts[v] > 0, vis)
        np.testing.assert_array_equal(counts[v], ontiles)
        gb = rec[v].view(np.uint32)
        ob = orec.view(np.uint32)
        for f in range(6):           # theta, phi, conic a, 2b, c, tau: bit-exact
            np.testing.assert_array_equal(gb[vis, f], ob[vis, f], err_msg=f"record field {f}")
        rows = rec[v, :, 6].view(np.int32)
        cols = rec[v, :, 7].view(np.int32)
        np.testing.assert_array_equal(rows[vis] & 0xFFFF, obox[vis, 0])
        np.testing.assert_array_equal(rows[vis] >> 16, obox[vis, 1])
        np.testing.assert_array_equal(cols[vis] & 0xFFFF, obox[vis, 2])
        np.testing.assert_array_equal(cols[vis] >> 16, obox[vis, 3])
        # per-tile sorted lists and ranges
        off = np.concatenate([[0], np.cumsum(ocnt)])
        for t in range(T):
            s, e = ranges[v, t]
            got = vals[s:e] if e > s else np.zeros(0, np.int32)
            np.testing.assert_array_equal(got, olists[off[t]:off[t + 1]], err_msg=f"view {v} tile {t}")
    return int(vals.shape[0])


def render_all(torch, ctx, scene_h, tx_np, rad_np, kind, views=None, **kw):
    g_H, g_W = ctx.H, ctx.W
    M, N, K, C = tx_np.shape[0], rad_np.shape[0], rad_np.shape[1], rad_np.shape[2]
    spec = torch.zeros((M, N, g_H, g_W, C, 2), dtype=torch.float32, device="cuda")
    rssi = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    csi = torch.zeros((M, N, C, 2), dtype=torch.float32, device="cuda")
    ncon = torch.zeros((M, g_H, g_W), dtype=torch.int32, device="cuda")
    tfin = torch.zeros((M, g_H, g_W), dtype=torch.float32, device="cuda")
    rad = dev(rad_np, torch)
    txd = dev(tx_np, torch)
    if views is None:
        ctx.render(scene_h, txd, None, N, kind, radiance=rad, spectra=spec,
                   rssi=rssi if C == 1 else None, csi=csi, ncontrib=ncon, tfinal=tfin, **kw)
    else:
        ctx.render_views(views, None, N, kind, radiance=rad, spectra=spec,
                         rssi=rssi if C == 1 else None, csi=csi, ncontrib=ncon, tfinal=tfin, **kw)
    ctx.sync()
    return (spec.cpu().numpy(), rssi.cpu().numpy(), csi.cpu().numpy(), ncon.cpu().numpy(),
            tfin.cpu().numpy())


def compare_view(oracle, g, scene, txv, rad_np, spec, rssi, csi, ncon, tfin):
    o = oracle.render_view(g, scene, txv, rad_np.astype(np.float64))
    np.testing.assert_array_equal(ncon, o["ncontrib"])
    np.testing.assert_array_equal(tfin.view(np.uint32), o["Tfinal"].view(np.uint32))
    e = norm_err(spec, o["spectra"], o["absacc"])
    assert e <= TOL, f"spectra normalised error {e}"
    ref_csi = oracle.csi(o["spectra"])
    a_csi = o["absacc"].sum(axis=(1, 2))
    e = norm_err(csi, ref_csi, a_csi)
    assert e <= TOL, f"csi normalised error {e}"
    if rad_np.shape[2] == 1:
        ref = oracle.rssi(o["spectra"])
        e = float((np.abs(rssi - ref) / (a_csi[:, 0] + 1e-30)).max())
        assert e <= TOL, f"rssi normalised error {e}"
    return o


def test_small_scene_views_bitexact(torch, rx, oracle):
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    tx = np.concatenate([w["tx"], S.draw_points(np.random.default_rng(5), 2)])
    views = ctx.prepare(h, dev(tx, torch))
    n = check_views(torch, ctx, oracle, g, sc, tx, views)
    assert n > 10000
    ctx.release_views(views)


@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
@pytest.mark.parametrize("K", [48, 300])
def test_seam_pole_full_span_scene(torch, rx, oracle, tile, K):
    """The oracle's seam / pole / full-width-span scene (Gaussians straddling
    azimuth 0 = 360 deg and near the zenith, whose footprints cover every
    column) on the 18x36 grid at 10 deg: records, tile sets, sorted lists
    and ranges bit-exact; spectra, CSI and RSSI against the oracle."""
    from tests.test_oracle_pins import tiny_scene
    sc, tx = tiny_scene(60 + K, K=K)
    g = S.Grid(H=18, W=36, theta0_deg=-10.0, step_deg=10.0, tile_h=tile[0], tile_w=tile[1],
               eps_T=0.02)
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    txs = np.stack([tx, tx + S.f32([0.3, -0.2, 0.1])])
    views = ctx.prepare(h, dev(txs, torch))
    check_views(torch, ctx, oracle, g, sc, txs, views)
    _, orec, obox = oracle.project_view32(g, sc, txs[0])
    vis = orec[:, 7] > 0
    assert ((obox[vis, 3] + 1) >= g.W).any(), "no full-width span in the scene"
    assert (obox[vis, 2] + obox[vis, 3] >= g.W).any(), "no footprint across the seam"
    rad = S.draw_radiance(np.random.default_rng(K), 3, sc.K, 1)
    out = render_all(torch, ctx, h, txs, rad, rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI, views=views)
    for v in range(2):
        compare_view(oracle, g, sc, txs[v], rad, *[o[v] for o in out])
    ctx.release_views(views)


def test_full_size_sorted_lists_bitexact(torch, rx, oracle):
    """The sort at the benchmark's size (100,000 Gaussians, 32 transmitters,
    millions of instances, so thousands of radix-sort blocks and more than one
    pass of the block-offset carry loop): keys and values of two views bit
    for bit against the oracle's depth-sorted tile lists; sortedness and the
    list structure of the keys over all 32 views."""
    w = S.workload_mlp()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(w["tx"], torch))
    n = check_views(torch, ctx, oracle, g, sc, w["tx"], views, which=[0, 31])
    assert n > 256 * 2048, n              # past 256 sort blocks of 2,048 items
    ctx.release_views(views)


def test_lists_many_tiles_two_pass_path(torch, rx, oracle):
    """More than 512 tiles (a 360x720 grid at 0.5 deg: 1,035 tiles of 16x16)
    takes the two-pass (view | tile) instance sort and the ranges kernel in
    place of the one-pass sort per view: records, tile sets, sorted lists and
    ranges bit-exact for both views."""
    rng = np.random.default_rng(307)
    sc = S.draw_scene(rng, 1500)
    g = S.Grid(H=360, W=720, theta0_deg=-90.0, step_deg=0.5, tile_h=16, tile_w=16)
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    tx = S.draw_points(np.random.default_rng(308), 2)
    views = ctx.prepare(h, dev(tx, torch))
    n = check_views(torch, ctx, oracle, g, sc, tx, views)
    assert n > 0
    ctx.release_views(views)


def test_lists_narrow_depths_ties_empty_view(torch, rx, oracle):
    """Gaussians on a thin shell around the first transmitter (all depths
    within 0.3 % of each other, so the depth sort needs two 9-bit passes),
    fifty of them duplicated at other indices (equal depths and footprints:
    ties decided by the Gaussian index), and a middle view that sees nothing
    (an empty run between two non-empty ones in the per-view instance pass):
    lists and ranges bit-exact; spectra, CSI and RSSI of the first view
    against the oracle."""
    rng = np.random.default_rng(311)
    K = 600
    d = rng.normal(size=(K, 3))
    d[:, 2] = np.abs(d[:, 2]) + 0.2          # above the horizon
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tx0 = np.array([5.0, 4.0, 1.0])
    r = 3.0 + rng.uniform(-0.004, 0.004, K)
    means = tx0 + d * r[:, None]
    means[K - 50:] = means[:50]
    sc = S.Scene(S.f32(means), S.f32(rng.normal(-2.3, 0.3, size=(K, 3))),
                 S.f32(rng.normal(size=(K, 4))), S.f32(rng.uniform(0.2, 0.9, size=K)))
    g = S.Grid()
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    tx = S.f32([tx0, [5.0, 4.0, 50.0], tx0 + np.array([0.01, -0.01, 0.0])])
    views = ctx.prepare(h, dev(tx, torch))
    check_views(torch, ctx, oracle, g, sc, tx, views)
    _, orec, _ = oracle.project_view32(g, sc, tx[1])
    assert not (orec[:, 7] > 0).any(), "the middle view should see nothing"
    _, orec0, _ = oracle.project_view32(g, sc, tx[0])
    vis = orec0[:, 7] > 0
    assert vis[:50].any() and (vis[:50] == vis[K - 50:]).all()
    rad = S.draw_radiance(np.random.default_rng(312), 2, K, 1)
    out = render_all(torch, ctx, h, tx, rad, rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI,
                     views=views)
    compare_view(oracle, g, sc, tx[0], rad, *[o[0] for o in out])
    assert np.all(out[0][1] == 0)
    ctx.release_views(views)


def test_small_workload_forward_parity(torch, rx, oracle):
    """4,096 Gaussians, 1 transmitter, 8 receivers, 90x360, 16x16 tiles."""
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    out = render_all(torch, ctx, h, w["tx"], w["radiance"],
                     rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI)
    spec, rssi, csi, ncon, tfin = out
    o = compare_view(oracle, g, sc, w["tx"][0], w["radiance"], spec[0], rssi[0], csi[0], ncon[0],
                     tfin[0])
    assert (o["ncontrib"] > 0).mean() > 0.5          # the scene covers most of the grid
    assert (o["Tfinal"] < g.eps_T).any()             # and the stop is exercised


@pytest.mark.parametrize("cols", [16, 32, 64, 128])
def test_column_blocking(torch, rx, oracle, cols):
    """Column blocks of 16-64 composite on the CUDA cores in the same order:
    spectra bit-identical.  Blocks of 128 columns take the tensor-core
    product (split bf16, float32 accumulation): the same stop positions and
    final transmittances bit for bit, spectra within the parity tolerance of
    the oracle's absolute chain of the CUDA-core result."""
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g, cols_per_cta=cols)
    h = upload(ctx, sc, torch)
    spec, _, _, ncon, tfin = render_all(torch, ctx, h, w["tx"], w["radiance"], rx.OUT_SPECTRA)
    ctx2 = make_ctx(rx, g, cols_per_cta=64)
    h2 = upload(ctx2, sc, torch)
    ref, _, _, ncon2, tfin2 = render_all(torch, ctx2, h2, w["tx"], w["radiance"], rx.OUT_SPECTRA)
    np.testing.assert_array_equal(ncon, ncon2)
    np.testing.assert_array_equal(tfin.view(np.uint32), tfin2.view(np.uint32))
    if cols < 128:
        np.testing.assert_array_equal(spec.view(np.uint32), ref.view(np.uint32))
    else:
        o = oracle.render_view(g, sc, w["tx"][0], w["radiance"].astype(np.float64))
        assert norm_err(spec[0], ref[0], o["absacc"]) <= TOL


def test_ragged_sizes_and_channels(torch, rx, oracle):
    """Odd receiver count, 3 channels, 8x32 tiles, a 180x360 grid from -90 deg,
    two transmitters: ragged column blocks and partial tiles."""
    rng = np.random.default_rng(101)
    sc = S.draw_scene(rng, 3000)
    g = S.Grid(H=180, W=360, theta0_deg=-90.0, tile_h=8, tile_w=32)
    tx = S.draw_points(rng, 2)
    rad = S.draw_radiance(rng, 5, sc.K, 3)
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch, C=3)
    views = ctx.prepare(h, dev(tx, torch))
    check_views(torch, ctx, oracle, g, sc, tx, views)
    spec, rssi, csi, ncon, tfin = render_all(torch, ctx, h, tx, rad, rx.OUT_SPECTRA | rx.OUT_CSI,
                                             views=views)
    for v in range(2):
        compare_view(oracle, g, sc, tx[v], rad, spec[v], rssi[v], csi[v], ncon[v], tfin[v])


def test_coarse_grid_partial_tiles(torch, rx, oracle):
    """The 36x9 grid at 10 degrees (Table 5): one partial tile row, a partial
    last tile column."""
    rng = np.random.default_rng(102)
    sc = S.draw_scene(rng, 2000)
    g = S.Grid(H=9, W=36, step_deg=10.0)
    tx = S.draw_points(rng, 1)
    rad = S.draw_radiance(rng, 3, sc.K, 1)
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(tx, torch))
    check_views(torch, ctx, oracle, g, sc, tx, views)
    out = render_all(torch, ctx, h, tx, rad, rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI, views=views)
    compare_view(oracle, g, sc, tx[0], rad, *[o[0] for o in out])


def test_single_receiver_equals_batch(torch, rx):
    """N = 1 renders are bit-identical to the same receiver inside a batch."""
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g, cols_per_cta=16)
    h = upload(ctx, sc, torch)
    views = ctx.prepare(h, dev(w["tx"], torch))
    full = render_all(torch, ctx, h, w["tx"], w["radiance"], rx.OUT_SPECTRA, views=views)[0]
    for j in [0, 3, 7]:
        one = render_all(torch, ctx, h, w["tx"], w["radiance"][j:j + 1], rx.OUT_SPECTRA,
                         views=views)[0]
        np.testing.assert_array_equal(one[0, 0].view(np.uint32), full[0, j].view(np.uint32))


def test_empty_and_degenerate_views(torch, rx, oracle):
    """A transmitter above every Gaussian (nothing in the upper hemisphere),
    and a single-Gaussian scene."""
    rng = np.random.default_rng(103)
    sc = S.draw_scene(rng, 500)
    g = S.Grid()
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    tx = S.f32([[5.0, 4.0, 50.0]])
    rad = S.draw_radiance(rng, 2, sc.K, 1)
    spec, rssi, csi, ncon, tfin = render_all(torch, ctx, h, tx, rad,
                                             rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI)
    assert np.all(spec == 0) and np.all(rssi == 0) and np.all(ncon == 0) and np.all(tfin == 1.0)
    one = S.Scene(sc.means[:1].copy(), sc.log_scales[:1].copy(), sc.quats[:1].copy(),
                  sc.opacity[:1].copy())
    tx1 = S.f32(one.means[0] + np.array([0.5, 0.2, -0.4]))
    h1 = upload(ctx, one, torch)
    rad1 = rad[:, :1]
    out = render_all(torch, ctx, h1, tx1[None], rad1, rx.OUT_SPECTRA | rx.OUT_RSSI | rx.OUT_CSI)
    compare_view(oracle, g, one, tx1, rad1, *[o[0] for o in out])


def test_invalid_arguments_are_refused(torch, rx):
    w = S.workload_small()
    g, sc = w["grid"], w["scene"]
    ctx = make_ctx(rx, g)
    h = upload(ctx, sc, torch)
    tx = dev(w["tx"], torch)
    with pytest.raises(rx.RxgsError) as ei:
        ctx.render(h, tx, None, 8, rx.OUT_SPECTRA, radiance=dev(w["radiance"], torch), spectra=None)
    assert ei.value.status == rx.E_INVALID
    with pytest.raises(rx.RxgsError):
        ctx.render(h + 999, tx, None, 8, rx.OUT_RSSI, radiance=dev(w["radiance"], torch),
                   rssi=torch.zeros(8, device="cuda"))
    with pytest.raises(rx.RxgsError):          # no radiance and no MLP
        ctx.render(h, tx, dev(w["rx"], torch), 8, rx.OUT_RSSI, rssi=torch.zeros(8, device="cuda"))
    with pytest.raises(rx.RxgsError):
        rx.Context(tile_h=10, tile_w=10)
    with pytest.raises(rx.RxgsError):          # no bit-reproducible backward is offered
        rx.Context(deterministic=1)


def test_mlp_radiance_full_size_sampled(torch, rx, oracle):
    """100,000 Gaussians, 32 transmitters x 64 receivers with MLP radiance, in
    the launch configuration the benchmark times; sampled pixels of a few
    (transmitter, receiver) pairs against the oracle."""
    w = S.workload_mlp()
    g, sc, C = w["grid"], w["scene"], w["C"]
    ctx = make_ctx(rx, g)
    flat = S.flatten_mlp(w["mlp"], C)
    h = upload(ctx, sc, torch, base=w["base"], mlp_flat=flat, C=C)
    M, N = w["tx"].shape[0], w["rx"].shape[0]
    spec = torch.zeros((M, N, g.H, g.W, C, 2), dtype=torch.float32, device="cuda")
    ncon = torch.zeros((M, g.H, g.W), dtype=torch.int32, device="cuda")
    tfin = torch.zeros((M, g.H, g.W), dtype=torch.float32, device="cuda")
    ctx.render(h, dev(w["tx"], torch), dev(w["rx"], torch), N, rx.OUT_SPECTRA, spectra=spec,
               ncontrib=ncon, tfinal=tfin)
    ctx.sync()
    rng = np.random.default_rng(7)
    js = [0, 17, 63]
    rad = oracle.mlp_radiance(w["mlp"], w["rx"][js], sc.means, w["base"])
    for v in [0, 13, 31]:
        pix = rng.choice(g.H * g.W, size=96, replace=False).astype(np.int32)
        val, aab, nc, tf = oracle.render_pixels(g, sc, w["tx"][v], rad, pix)
        got = spec[v][js].reshape(len(js), g.H * g.W, C, 2)[:, torch.from_numpy(pix).long().cuda()]
        got = got.permute(1, 0, 2, 3).cpu().numpy()
        e = norm_err(got, val, aab)
        assert e <= TOL, f"view {v}: {e}"
        np.testing.assert_array_equal(ncon[v].reshape(-1).cpu().numpy()[pix], nc)
        np.testing.assert_array_equal(tfin[v].reshape(-1).cpu().numpy()[pix].view(np.uint32),
                                      tf.view(np.uint32))
