"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a library routine (scipy rotations, torch autograd, numpy complex
arithmetic), brute force, an identity of the method, or finite differences.
None needs a GPU.
"""
import math

import numpy as np
import pytest

from paper_2605_24290_gb300 import synthetic as S


def tiny_scene(seed=1, K=48, pole=True, seam=True):
    """K Gaussians around a transmitter at (5,4,1), including some near the
    azimuth seam (phi ~ 0 / 360 deg) and some near the zenith."""
    rng = np.random.default_rng(seed)
    tx = np.array([5.0, 4.0, 1.0])
    d = rng.uniform(1.0, 4.0, size=K)
    az = rng.uniform(0, 2 * math.pi, size=K)
    el = rng.uniform(-0.2, 1.4, size=K)
    if seam:
        az[:6] = rng.uniform(-0.15, 0.15, size=6)
    if pole:
        el[6:10] = rng.uniform(1.45, 1.56, size=4)
    p = tx + np.stack([d * np.cos(el) * np.cos(az), d * np.cos(el) * np.sin(az), d * np.sin(el)], -1)
    sc = S.Scene(S.f32(p), S.f32(rng.normal(-1.6, 0.4, size=(K, 3))), S.f32(rng.normal(size=(K, 4))),
                 S.f32(1 / (1 + np.exp(-rng.normal(size=K)))))
    return sc, S.f32(tx)


def tiny_grid(**kw):
    g = S.Grid(H=18, W=36, theta0_deg=-10.0, step_deg=10.0, tile_h=6, tile_w=6)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


# ------------------------------------------------------ float32 exp / atan2

def test_exp32_within_one_ulp(oracle):
    xs = np.concatenate([np.linspace(-86.9, 88.0, 40001),
                         np.random.default_rng(0).uniform(-4.5, 0.0, 40000)]).astype(np.float32)
    got = np.array([oracle.exp32(float(x)) for x in xs], np.float64)
    ref = np.exp(xs.astype(np.float64))
    ulp = np.abs(got - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert ulp.max() <= 1.0
    assert oracle.exp32(0.0) == 1.0


def test_atan2_32_within_four_ulp(oracle):
    rng = np.random.default_rng(2)
    ys = rng.normal(size=(20000, 2)).astype(np.float32)
    axes = np.array([[0, 1], [1, 0], [0, -1], [-1, 0], [1, 1], [-1, -1], [1, -1], [-1, 1],
                     [1e-7, 1], [1, 1e-7], [-1e-7, -1]], np.float32)
    ys = np.concatenate([ys, axes])
    got = np.array([oracle.atan2_32(float(y), float(x)) for y, x in ys], np.float64)
    ref = np.arctan2(ys[:, 0].astype(np.float64), ys[:, 1].astype(np.float64))
    ulp = np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 1e-30).astype(np.float32))
    assert ulp.max() <= 4.0


# ------------------------------------------------------------- covariance

def test_covariance_matches_rotation_library(oracle):
    """Sigma = R S S^T R^T (App. E.1) against scipy's quaternion rotation."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    s = S.f32(rng.normal(-2, 0.5, size=(50, 3)))
    q = S.f32(rng.normal(size=(50, 4)))
    c64 = oracle.cov64(s, q)
    c32 = oracle.cov32(s, q)
    for k in range(50):
        R = Rotation.from_quat(q[k].astype(np.float64), scalar_first=True).as_matrix()
        Sig = R @ np.diag(np.exp(2 * s[k].astype(np.float64))) @ R.T
        ref = Sig[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
        scale = np.abs(Sig).max()
        assert np.abs(c64[k] - ref).max() <= 1e-13 * scale
        assert np.abs(c32[k] - ref).max() <= 2e-6 * scale


# ------------------------------------------------------------- projection

def _angles(u):
    h = math.hypot(u[0], u[1])
    return np.array([math.atan2(u[2], h), math.atan2(u[1], u[0])])


def test_projection_isotropic_closed_form(oracle):
    """An isotropic Gaussian of std sigma at distance rho projects to
    Sigma2D = diag((sigma/(rho D))^2, (sigma/(h D))^2) in pixel units,
    h = horizontal distance: the elevation and azimuth axes are orthogonal
    with arc lengths rho*dtheta and h*dphi."""
    g = S.Grid(step_deg=1.0)
    D = math.radians(1.0)
    for u, sig in [((3.0, 0.0, 0.0), 0.2), ((1.0, -2.0, 1.5), 0.1), ((-0.5, 0.3, 2.0), 0.05)]:
        S6 = np.array([sig * sig, 0, 0, sig * sig, 0, sig * sig])
        out = oracle.sigma2d64(g, np.array(u, np.float32), S6, np.zeros(3, np.float32))
        uu = np.array(u, np.float32).astype(np.float64)
        rho, h = np.linalg.norm(uu), math.hypot(uu[0], uu[1])
        assert out[0] == pytest.approx((sig / (rho * D)) ** 2, rel=1e-12)
        assert out[2] == pytest.approx((sig / (h * D)) ** 2, rel=1e-12)
        assert abs(out[1]) <= 1e-12 * out[0]


def test_projection_matches_finite_difference_jacobian(oracle):
    """J Sigma J^T with J from central differences of the angle map."""
    g = S.Grid(step_deg=1.0)
    D = math.radians(1.0)
    rng = np.random.default_rng(4)
    for _ in range(20):
        u = rng.normal(size=3) * 3
        u32 = u.astype(np.float32)
        uu = u32.astype(np.float64)
        A = rng.normal(size=(3, 3)) * 0.2
        Sig = A @ A.T + 1e-3 * np.eye(3)
        J = np.zeros((2, 3))
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1e-6
            J[:, i] = (_angles(uu + e) - _angles(uu - e)) / 2e-6
        J /= D
        ref = J @ Sig @ J.T
        S6 = Sig[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
        out = oracle.sigma2d64(g, u32, S6, np.zeros(3, np.float32))
        np.testing.assert_allclose(out, [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-6,
                                   atol=1e-7 * abs(ref).max())


def test_projection_matches_monte_carlo(oracle):
    """A small Gaussian's samples, mapped to angles, have the projected
    covariance (the local linearisation the projection takes)."""
    g = S.Grid(step_deg=1.0)
    D = math.radians(1.0)
    rng = np.random.default_rng(5)
    u = np.array([2.0, 1.0, 0.7], np.float32)
    A = rng.normal(size=(3, 3)) * 0.02
    Sig = A @ A.T
    X = rng.multivariate_normal(u.astype(np.float64), Sig, size=200000)
    h = np.hypot(X[:, 0], X[:, 1])
    ang = np.stack([np.arctan2(X[:, 2], h), np.arctan2(X[:, 1], X[:, 0])], -1) / D
    emp = np.cov(ang.T)
    S6 = Sig[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    out = oracle.sigma2d64(g, u, S6, np.zeros(3, np.float32))
    np.testing.assert_allclose([emp[0, 0], emp[0, 1], emp[1, 1]], out, rtol=0.03,
                               atol=0.03 * max(out[0], out[2]))


# ------------------------------------------------------------- compositing

def _unit_radiance(N, K, C=1):
    r = np.zeros((N, K, C, 2))
    r[..., 0] = 1.0
    return r


def test_single_gaussian_closed_form(oracle):
    """One Gaussian: spectrum = tau exp(-q/2) s on the pixels it covers, q
    from the inverse of the finite-difference Sigma2D; zero elsewhere."""
    g = S.Grid(H=90, W=360)
    D = math.radians(1.0)
    tx = np.array([0.0, 0.0, 0.0], np.float32)
    p = np.array([[2.0, 1.0, 1.2]], np.float32)
    sc = S.Scene(p, S.f32([[-1.5, -1.9, -1.7]]), S.f32([[0.9, 0.2, -0.3, 0.1]]), S.f32([0.7]))
    s = np.array([[[[0.3, -1.1]]]])
    out = oracle.render_view(g, sc, tx, s)
    spec = out["spectra"][0, :, :, 0, :]
    Sig = oracle.cov64(sc.log_scales, sc.quats)[0]
    Sg = np.array([[Sig[0], Sig[1], Sig[2]], [Sig[1], Sig[3], Sig[4]], [Sig[2], Sig[4], Sig[5]]])
    uu = p[0].astype(np.float64)
    J = np.zeros((2, 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1e-6
        J[:, i] = (_angles(uu + e) - _angles(uu - e)) / 2e-6
    J /= D
    conic = np.linalg.inv(J @ Sg @ J.T)
    c_ang = _angles(uu) / D
    ii, jj = np.meshgrid(np.arange(90), np.arange(360), indexing="ij")
    dth = ii - c_ang[0]
    dph = (jj - c_ang[1] + 180) % 360 - 180
    q = conic[0, 0] * dth ** 2 + 2 * conic[0, 1] * dth * dph + conic[1, 1] * dph ** 2
    w = 0.7 * np.exp(-0.5 * q)
    covered = out["ncontrib"] == 1
    assert out["ncontrib"].max() == 1
    # the pixels the oracle composites are exactly those with q <= 9 (away from the edge)
    assert np.all(covered[q < 9 - 1e-4])
    assert not np.any(covered[q > 9 + 1e-4])
    ref = np.where(covered, w, 0.0)
    np.testing.assert_allclose(spec[..., 0], ref * 0.3, rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(spec[..., 1], ref * -1.1, rtol=1e-7, atol=1e-12)


def test_transmittance_telescoping_identity(oracle):
    """With s = 1 for every Gaussian, sum_k T_k w_k = 1 - prod_k (1 - w_k):
    the composited signal plus the final transmittance is exactly 1."""
    sc, tx = tiny_scene(7, K=64)
    g = tiny_grid(eps_T=0.0)
    out = oracle.render_view(g, sc, tx, _unit_radiance(1, sc.K), use_eps=False)
    tot = out["spectra"][0, :, :, 0, 0] + out["T64"]
    np.testing.assert_allclose(tot, 1.0, rtol=0, atol=1e-13)
    assert np.all(out["spectra"][0, :, :, 0, 1] == 0.0)
    # with the stop on, the final shadow transmittance is below eps exactly
    # where the loop stopped early
    g2 = tiny_grid(eps_T=0.5)
    o2 = oracle.render_view(g2, sc, tx, _unit_radiance(1, sc.K))
    stopped = o2["Tfinal"] < np.float32(0.5)
    assert stopped.any() and (~stopped).any()
    np.testing.assert_allclose(o2["spectra"][0, :, :, 0, 0] + o2["T64"], 1.0, atol=1e-13)


def test_linearity_in_radiance(oracle):
    sc, tx = tiny_scene(8)
    g = tiny_grid()
    rng = np.random.default_rng(9)
    r1 = rng.normal(size=(2, sc.K, 2, 2))
    r2 = rng.normal(size=(2, sc.K, 2, 2))
    a = oracle.render_view(g, sc, tx, r1)["spectra"]
    b = oracle.render_view(g, sc, tx, r2)["spectra"]
    c = oracle.render_view(g, sc, tx, 2.0 * r1 - 0.5 * r2)["spectra"]
    np.testing.assert_allclose(c, 2.0 * a - 0.5 * b, rtol=1e-12, atol=1e-12)


def test_two_gaussians_front_to_back_and_stop(oracle):
    """Two Gaussians on the same ray at q = 0: C = tau1 s1 + (1-tau1) tau2 s2;
    the stop comes after the contribution that crosses eps (Algorithm 1)."""
    tx = np.zeros(3, np.float32)
    p = S.f32([[4.0, 0.0, 0.0], [2.0, 0.0, 0.0]])     # index 1 is nearer
    sc = S.Scene(p, S.f32([[-2.0] * 3, [-2.0] * 3]), S.f32([[1, 0, 0, 0], [1, 0, 0, 0]]),
                 S.f32([0.6, 0.5]))
    rad = np.array([[[[1.0, 2.0]], [[-3.0, 0.5]]]])    # s_far, s_near
    g = S.Grid(H=90, W=360)
    out = oracle.render_view(g, sc, tx, rad)
    got = out["spectra"][0, 0, 0, 0]
    t_far, t_near = float(np.float32(0.6)), float(np.float32(0.5))
    ref = t_near * np.array([-3.0, 0.5]) + (1 - t_near) * t_far * np.array([1.0, 2.0])
    np.testing.assert_allclose(got, ref, rtol=1e-15)
    assert out["ncontrib"][0, 0] == 2
    g.eps_T = 0.6        # T after the near one is 0.5 < 0.6: stop there
    out = oracle.render_view(g, sc, tx, rad)
    np.testing.assert_allclose(out["spectra"][0, 0, 0, 0], t_near * np.array([-3.0, 0.5]), rtol=1e-15)
    assert out["ncontrib"][0, 0] == 1


def test_golden_two_gaussian_fixture(oracle):
    """tests/golden/two_gaussians.txt: hand-derived values of the case above
    (Algorithm 1, Stage 3)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "two_gaussians.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    tx = np.zeros(3, np.float32)
    p = S.f32([[4.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    sc = S.Scene(p, S.f32([[-2.0] * 3, [-2.0] * 3]), S.f32([[1, 0, 0, 0], [1, 0, 0, 0]]),
                 S.f32([0.75, 0.5]))
    rad = np.array([[[[1.0, 2.0]], [[-3.0, 0.5]]]])
    out = oracle.render_view(S.Grid(H=90, W=360), sc, tx, rad)
    assert out["spectra"][0, 0, 0, 0, 0] == pytest.approx(vals["re"], abs=1e-15)
    assert out["spectra"][0, 0, 0, 0, 1] == pytest.approx(vals["im"], abs=1e-15)
    assert out["T64"][0, 0] == pytest.approx(vals["T"], abs=1e-15)


def test_tiled_lists_equal_brute_force(oracle):
    """Per-tile lists hold exactly the Gaussians whose footprint meets the
    tile, in ascending (depth, index); walking a pixel's tile list gives the
    same sequence as walking all Gaussians in global depth order."""
    for seed in range(3):
        sc, tx = tiny_scene(10 + seed, K=64)
        g = tiny_grid()
        S6, rec, box = oracle.project_view32(g, sc, tx)
        counts, lists, ntiles = oracle.tile_lists(g, sc, tx)
        th, tw = 3, 6
        vis = rec[:, 7] > 0
        assert vis.sum() > 20

        def inside(k, i, j):
            if i < box[k, 0] or i > box[k, 1]:
                return False
            return (j - box[k, 2]) % g.W <= box[k, 3]

        # independent tile sets by enumeration
        sets = [set() for _ in range(th * tw)]
        for k in np.nonzero(vis)[0]:
            for i in range(g.H):
                for j in range(g.W):
                    if inside(k, i, j):
                        sets[(i // g.tile_h) * tw + j // g.tile_w].add(int(k))
        off = np.concatenate([[0], np.cumsum(counts)])
        for t in range(th * tw):
            lt = list(lists[off[t]:off[t + 1]])
            assert set(lt) == sets[t]
            assert lt == sorted(lt, key=lambda k: (rec[k, 6], k))
        for k in range(sc.K):
            assert ntiles[k] == sum(k in s_ for s_ in sets)
        # a Gaussian is kept only if its footprint holds at least one pixel
        assert np.all(ntiles[vis] >= 1)
        assert np.all((box[vis, 2] >= 0) & (box[vis, 2] < g.W))
        glob = sorted(np.nonzero(vis)[0], key=lambda k: (rec[k, 6], k))
        for i in range(g.H):
            for j in range(g.W):
                t = (i // g.tile_h) * tw + j // g.tile_w
                a = [k for k in lists[off[t]:off[t + 1]] if inside(k, i, j)]
                b = [k for k in glob if inside(k, i, j)]
                assert a == b
        # wrap and pole cases were exercised
        assert (box[vis, 3] == g.W - 1).any()
        assert ((box[vis, 2] + box[vis, 3]) >= g.W).any()


def test_footprint_column_start_wraps_into_grid(oracle):
    """A small Gaussian just below azimuth 360 deg whose only covered column
    is 0: its column range starts inside [0, W) and its tile is tile 0."""
    g = S.Grid(H=9, W=36, step_deg=10.0)
    rng = np.random.default_rng(102)
    sc = S.draw_scene(rng, 2000)
    tx = S.draw_points(rng, 1)
    _, rec, box = oracle.project_view32(g, sc, tx[0])
    counts, lists, ntiles = oracle.tile_lists(g, sc, tx[0])
    k = 6                                   # phi_px = 35.94, one column
    assert rec[k, 7] == 1 and rec[k, 1] > 35.5
    assert box[k, 2] == 0 and box[k, 3] == 0 and ntiles[k] == 1
    assert k in lists[:counts[0]]


def test_render_reorder_identity(oracle):
    """Eq. render_reorder: sum over directions of C^(j) = sum_k W_k s_kj with
    receiver-independent W_k = sum_omega T_k w_k."""
    sc, tx = tiny_scene(14, K=64)
    g = tiny_grid()
    rng = np.random.default_rng(15)
    rad = rng.normal(size=(3, sc.K, 2, 2))
    out = oracle.render_view(g, sc, tx, rad, want_w=True)
    lhs = oracle.csi(out["spectra"])
    rhs = np.einsum("k,nkcr->ncr", out["Wvis"], rad)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_amplitude_and_reductions(oracle):
    spec = np.zeros((1, 2, 2, 1, 2))
    spec[0, 0, 0, 0] = [3.0, 4.0]
    spec[0, 1, 1, 0] = [-1.0, 0.0]
    assert oracle.amplitude(spec)[0, 0, 0, 0] == pytest.approx(math.sqrt(25 + 1e-8))
    assert oracle.amplitude(spec)[0, 0, 1, 0] == pytest.approx(1e-4)
    assert oracle.rssi(spec)[0] == pytest.approx(math.sqrt(4 + 16))


# ------------------------------------------------------------------- MLP

def _torch_mlp(params, rx, means, base):
    torch = pytest.importorskip("torch")
    P = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in params.items()}
    rx_t = torch.tensor(np.asarray(rx, np.float64))
    p_t = torch.tensor(np.asarray(means, np.float64))
    b = torch.tensor(np.asarray(base, np.float64), requires_grad=True)
    C = base.shape[1]

    def mlp(x, pre):
        h = torch.relu(torch.nn.functional.linear(x, P[pre + "_w1"], P[pre + "_b1"]))
        return torch.nn.functional.linear(h, P[pre + "_w2"], P[pre + "_b2"])

    og = mlp(rx_t, "g").reshape(-1, 1, C, 4)
    v = rx_t[:, None, :] - p_t[None]
    d = torch.linalg.norm(v, dim=-1, keepdim=True)
    feat = torch.cat([v / d, d, torch.ones_like(d), torch.zeros_like(d)], -1)
    ol = mlp(feat, "l").reshape(rx_t.shape[0], -1, C, 4)
    cz = lambda a: torch.complex(a[..., 0], a[..., 1])
    phi = cz(b)[None]
    s = (1 + cz(ol[..., 0:2])) * ((1 + cz(og[..., 0:2])) * phi + cz(og[..., 2:4])) + cz(ol[..., 2:4])
    return torch.stack([s.real, s.imag], -1), P, b


def test_mlp_zero_init_is_identity(oracle):
    """Both branches zero-initialised: s = phi_base (Sec. 3.3.2)."""
    rng = np.random.default_rng(20)
    C = 3
    params = {k: np.zeros(v.shape) for k, v in S.draw_mlp(rng, C).items()}
    base = rng.normal(size=(10, C, 2))
    s = oracle.mlp_radiance(params, rng.normal(size=(4, 3)), rng.normal(size=(10, 3)), base)
    np.testing.assert_array_equal(s, np.broadcast_to(base[None], s.shape))


def test_mlp_affine_reproduces_propagation_factor(oracle):
    """Corollary 2: with alpha = eta_eff - 1 and beta = 0 the affine
    modulation is the complex product eta_eff * phi_base.  The MLP outputs
    are made constant (zero hidden weights, set biases) and compared with
    numpy complex arithmetic."""
    rng = np.random.default_rng(21)
    C = 2
    params = {k: np.zeros(v.shape) for k, v in S.draw_mlp(rng, C).items()}
    lam, d = 0.125, 3.7
    eta = lam / (4 * math.pi * d) * np.exp(-2j * math.pi / lam * d)
    params["l_b2"] = np.tile([eta.real - 1.0, eta.imag, 0.0, 0.0], C)
    base = rng.normal(size=(5, C, 2))
    s = oracle.mlp_radiance(params, rng.normal(size=(2, 3)), rng.normal(size=(5, 3)), base)
    ref = eta * (base[..., 0] + 1j * base[..., 1])
    np.testing.assert_allclose(s[..., 0], np.broadcast_to(ref.real, s.shape[:-1]), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(s[..., 1], np.broadcast_to(ref.imag, s.shape[:-1]), rtol=1e-13, atol=1e-15)
    # global branch alone: (1 + a_g) phi + b_g
    params = {k: np.zeros(v.shape) for k, v in S.draw_mlp(rng, C).items()}
    params["g_b2"] = np.tile([0.2, -0.3, 0.05, 0.4], C)
    s = oracle.mlp_radiance(params, rng.normal(size=(2, 3)), rng.normal(size=(5, 3)), base)
    ref = (1.2 - 0.3j) * (base[..., 0] + 1j * base[..., 1]) + (0.05 + 0.4j)
    np.testing.assert_allclose(s[0, ..., 0], ref.real, rtol=1e-13)
    np.testing.assert_allclose(s[0, ..., 1], ref.imag, rtol=1e-13)


def test_mlp_matches_torch(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(22)
    C = 3
    params = S.draw_mlp(rng, C, final_scale=1.0)
    rx, means, base = rng.normal(size=(4, 3)) * 3, rng.normal(size=(7, 3)) * 3, rng.normal(size=(7, C, 2))
    s = oracle.mlp_radiance(params, rx, means, base)
    st, _, _ = _torch_mlp(params, rx, means, base)
    np.testing.assert_allclose(s, st.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_mlp_backward_matches_torch_autograd(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(23)
    C = 2
    params = S.draw_mlp(rng, C, final_scale=1.0)
    rx, means, base = rng.normal(size=(3, 3)) * 3, rng.normal(size=(6, 3)) * 3, rng.normal(size=(6, C, 2))
    g = rng.normal(size=(3, 6, C, 2))
    st, P, b = _torch_mlp(params, rx, means, base)
    (st * torch.tensor(g)).sum().backward()
    got = oracle.mlp_backward(params, rx, means, base, g)
    np.testing.assert_allclose(got["base"], b.grad.numpy(), rtol=1e-11, atol=1e-12)
    for k in params:
        np.testing.assert_allclose(got[k], P[k].grad.numpy(), rtol=1e-11, atol=1e-12)


def test_mlp_bf16_rounding_matches_torch(oracle):
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(24).normal(size=1000) * 10
    got = oracle._bf16(x)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, ref)


def test_mlp_backward_chain_bounds_the_terms(oracle):
    """The absolute chain of the MLP backward bounds every gradient entry and,
    with every input, weight and incoming gradient positive and every complex
    quantity real (zero imaginary parts and zero weights into the imaginary
    outputs, so every unit is active and no term cancels), equals the
    gradient itself."""
    rng = np.random.default_rng(25)
    C = 2
    params = S.draw_mlp(rng, C, final_scale=1.0)
    rx, means, base = rng.normal(size=(3, 3)) * 3, rng.normal(size=(6, 3)) * 3, rng.normal(size=(6, C, 2))
    g = rng.normal(size=(3, 6, C, 2))
    got = oracle.mlp_backward(params, rx, means, base, g)
    chain, amb = oracle.mlp_backward_chain(params, rx, means, base, np.abs(g))
    for k in got:
        assert np.all(np.abs(got[k]) <= chain[k] * (1 + 1e-12) + 1e-300), k
        assert np.all(amb[k] == 0.0), k          # no unit near zero here
    pos = {k: np.abs(v) + 0.01 for k, v in params.items()}
    for k in ("g_w2", "g_b2", "l_w2", "l_b2"):    # outputs (a.re, a.im, b.re, b.im)
        pos[k][1::2] = 0.0
    means_p = rng.uniform(0.0, 1.0, size=(6, 3))
    rx_p = rng.uniform(2.0, 3.0, size=(3, 3))     # v_hat > 0 componentwise
    base_p, g_p = np.abs(base) + 0.1, np.abs(g) + 0.1
    base_p[..., 1] = 0.0
    g_p[..., 1] = 0.0
    got = oracle.mlp_backward(pos, rx_p, means_p, base_p, g_p)
    chain, _ = oracle.mlp_backward_chain(pos, rx_p, means_p, base_p, g_p)
    for k in got:
        np.testing.assert_allclose(chain[k], got[k], rtol=1e-12, err_msg=k)


def test_mlp_backward_chain_marks_units_at_zero(oracle):
    """A hidden unit whose pre-activation is exactly zero is a decision float32
    cannot settle: its first-layer terms are returned as ambiguous."""
    rng = np.random.default_rng(26)
    C = 1
    params = S.draw_mlp(rng, C, final_scale=1.0)
    rx = rng.normal(size=(2, 3)) * 3
    # unit 5 of the global branch: pre = w . x + b = 0 for receiver 0
    params["g_b1"][5] = -float(params["g_w1"][5] @ rx[0])
    means, base = rng.normal(size=(4, 3)), rng.normal(size=(4, C, 2))
    g = rng.normal(size=(2, 4, C, 2))
    _, amb = oracle.mlp_backward_chain(params, rx, means, base, np.abs(g))
    assert amb["g_b1"][5] > 0 and np.all(np.delete(amb["g_b1"], 5) == 0)
    assert np.all(amb["g_w1"][5] > 0)


# ------------------------------------------------------- Stage II step pins

def test_l1_amplitude_matches_torch_autograd(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(27)
    spec = rng.normal(size=(2, 3, 5, 7, 1, 2))
    spec[0, 0, 0, 0] = 0.0                        # an empty pixel: |R| = 1e-4
    y = np.abs(rng.normal(size=(2, 3, 5, 7, 1)))
    L, g = oracle.l1_amplitude(spec, y)
    st = torch.tensor(spec, requires_grad=True)
    amp = torch.sqrt(st[..., 0] ** 2 + st[..., 1] ** 2 + 1e-8)
    lt = (amp - torch.tensor(y)).abs().mean()
    lt.backward()
    assert L == pytest.approx(float(lt.detach()), rel=1e-14)
    np.testing.assert_allclose(g, st.grad.numpy(), rtol=1e-13, atol=1e-18)


def test_l1_rssi_matches_torch_autograd(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(28)
    c = rng.normal(size=(3, 4, 2))
    y = np.abs(rng.normal(size=(3, 4)))
    L, g = oracle.l1_rssi(c, y)
    ct = torch.tensor(c, requires_grad=True)
    lt = (torch.sqrt(ct[..., 0] ** 2 + ct[..., 1] ** 2) - torch.tensor(y)).abs().mean()
    lt.backward()
    assert L == pytest.approx(float(lt.detach()), rel=1e-14)
    np.testing.assert_allclose(g, ct.grad.numpy(), rtol=1e-13, atol=1e-18)


def test_adam_matches_torch_optimizer(oracle):
    """Three Adam steps on given gradients equal torch.optim.Adam's."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(29)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) * 10 ** rng.uniform(-6, 1, size=50) for _ in range(3)]
    pt = torch.nn.Parameter(torch.tensor(p0))
    opt = torch.optim.Adam([pt], lr=3e-3)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, gr in enumerate(grads, start=1):
        pt.grad = torch.tensor(gr)
        opt.step()
        p, m, v = oracle.adam(p, gr, m, v, t, 3e-3)
        np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(m, opt.state[pt]["exp_avg"].numpy(), rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(v, opt.state[pt]["exp_avg_sq"].numpy(), rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("kind", ["spectra", "rssi"])
def test_stage2_step_gradient_matches_finite_differences(oracle, kind):
    """The Stage II step's gradients (L1 loss -> render backward -> MLP
    backward) against central differences of its loss over phi_base and MLP
    entries on the seam / pole scene; the update is Adam's first step."""
    rng = np.random.default_rng(30)
    sc, tx = tiny_scene(31, K=40)
    g = tiny_grid(eps_T=0.02)
    txs = np.stack([tx, tx + S.f32([0.4, 0.1, -0.2])])
    rxp = S.f32(rng.uniform([3, 2, 0], [7, 6, 2], size=(2, 3)))
    C = 1
    base = rng.normal(size=(sc.K, C, 2))
    params = {k: v.astype(np.float64) for k, v in S.draw_mlp(rng, C, final_scale=0.5).items()}
    r0 = oracle.stage2_step(g, sc, txs, rxp, base, params,
                            np.zeros((2, 2, g.H, g.W, C)) if kind == "spectra" else np.zeros((2, 2)),
                            kind=kind)
    spec0 = r0["spectra"]
    if kind == "spectra":
        amp = oracle.amplitude(spec0)
        target = amp * (1 + np.where(rng.random(amp.shape) < 0.5, -0.5, 0.5))
    else:
        c = spec0.sum(axis=(2, 3))[..., 0, :]
        target = np.sqrt((c ** 2).sum(-1)) * (1 + np.where(rng.random((2, 2)) < 0.5, -0.5, 0.5))
    res = oracle.stage2_step(g, sc, txs, rxp, base, params, target, kind=kind, lr_base=1e-2,
                             lr_mlp=2e-3)

    def loss(b, P):
        return oracle.stage2_step(g, sc, txs, rxp, b, P, target, kind=kind)["loss"]

    h = 1e-6
    for idx in [(0, 0, 0), (7, 0, 1), (23, 0, 0)]:
        bp, bm = base.copy(), base.copy()
        bp[idx] += h
        bm[idx] -= h
        fd = (loss(bp, params) - loss(bm, params)) / (2 * h)
        assert fd == pytest.approx(res["grad_base"][idx], rel=1e-5, abs=1e-12)
    for name, idx in [("g_w1", (3, 1)), ("g_b2", (2,)), ("l_w1", (10, 3)), ("l_w2", (1, 7)),
                      ("l_b1", (4,))]:
        pp, pm = dict(params), dict(params)
        pp[name] = params[name].copy()
        pm[name] = params[name].copy()
        pp[name][idx] += h
        pm[name][idx] -= h
        fd = (loss(base, pp) - loss(base, pm)) / (2 * h)
        assert fd == pytest.approx(res["grad_mlp"][name][idx], rel=1e-5, abs=1e-12), name
    # Adam's first update: lr * g / (|g| + eps)
    gb = res["grad_base"]
    np.testing.assert_allclose(res["base"], base - 1e-2 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)
    assert res["state"]["t"] == 1


# -------------------------------------------------------------- backward

def test_render_backward_matches_finite_differences(oracle):
    """The oracle's analytic gradients against central differences of its
    own forward, with the early stop off so no decision can flip; q and the
    footprint do not depend on radiance or opacity."""
    sc, tx = tiny_scene(30, K=40)
    g = tiny_grid()
    rng = np.random.default_rng(31)
    N, C = 2, 2
    rad = rng.normal(size=(N, sc.K, C, 2))
    gs = rng.normal(size=(N, g.H, g.W, C, 2))
    gr, gt = oracle.backward_view(g, sc, tx, rad, gs, use_eps=False)

    def loss(scene, r):
        return float((oracle.render_view(g, scene, tx, r, use_eps=False, want_abs=False)["spectra"]
                      * gs).sum())

    # radiance: linear, so a unit step is exact
    for _ in range(12):
        idx = tuple(rng.integers(0, s_) for s_ in rad.shape)
        rp, rm = rad.copy(), rad.copy()
        rp[idx] += 0.5
        rm[idx] -= 0.5
        fd = loss(sc, rp) - loss(sc, rm)
        assert fd == pytest.approx(gr[idx], rel=1e-9, abs=1e-9)
    # opacity (float32 input): central difference over exactly representable steps
    vis = np.nonzero(np.abs(gt) > 0)[0]
    assert len(vis) > 10
    for k in vis[:15]:
        tp, tm = sc.opacity.copy(), sc.opacity.copy()
        tp[k] = np.float32(tp[k] + 1e-3)
        tm[k] = np.float32(tm[k] - 1e-3)
        sp = S.Scene(sc.means, sc.log_scales, sc.quats, tp)
        sm = S.Scene(sc.means, sc.log_scales, sc.quats, tm)
        fd = (loss(sp, rad) - loss(sm, rad)) / (float(tp[k]) - float(tm[k]))
        assert fd == pytest.approx(gt[k], rel=2e-5, abs=1e-7)


def test_render_backward_with_stop_matches_fd_of_fixed_sequence(oracle):
    """With the stop on, the gradient w.r.t. radiance is still exact (the
    sequence does not depend on radiance)."""
    sc, tx = tiny_scene(32, K=40)
    g = tiny_grid(eps_T=0.02)
    rng = np.random.default_rng(33)
    rad = rng.normal(size=(1, sc.K, 1, 2))
    gs = rng.normal(size=(1, g.H, g.W, 1, 2))
    gr, _ = oracle.backward_view(g, sc, tx, rad, gs, use_eps=True)
    base = oracle.render_view(g, sc, tx, rad)["spectra"]
    for _ in range(8):
        idx = tuple(rng.integers(0, s_) for s_ in rad.shape)
        rp = rad.copy()
        rp[idx] += 1.0
        d = ((oracle.render_view(g, sc, tx, rp)["spectra"] - base) * gs).sum()
        assert d == pytest.approx(gr[idx], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("case", ["seam_pole", "workload_small"])
def test_render_pixels_equals_render_view(oracle, case):
    """The pixel-list render (the checker of the full-size sampled GPU tests)
    returns, at every listed pixel and in any pixel order, exactly what the
    full-view render gives there: values, absolute chains, composited counts
    and the float32 final transmittance, bit for bit.  Cases: the seam, pole
    and full-width-span scene on the 18x36 grid (6x6 tiles), and the
    4,096-Gaussian workload on 90x360 with 8 receivers."""
    rng = np.random.default_rng(42)
    if case == "seam_pole":
        sc, tx = tiny_scene(43, K=48)
        g = tiny_grid(eps_T=0.6)        # a high threshold so that pixels stop
        rad = rng.normal(size=(3, sc.K, 2, 2))
        pix = rng.permutation(g.H * g.W).astype(np.int32)
    else:
        w = S.workload_small()
        g, sc, tx = w["grid"], w["scene"], w["tx"][0]
        rad = w["radiance"].astype(np.float64)
        pix = rng.choice(g.H * g.W, size=4000, replace=False).astype(np.int32)
    o = oracle.render_view(g, sc, tx, rad)
    val, aab, nc, tf = oracle.render_pixels(g, sc, tx, rad, pix)
    N, C = rad.shape[0], rad.shape[2]
    ref_val = o["spectra"].reshape(N, g.H * g.W, C, 2)[:, pix].transpose(1, 0, 2, 3)
    ref_aab = o["absacc"].reshape(N, g.H * g.W, C)[:, pix].transpose(1, 0, 2)
    np.testing.assert_array_equal(val.view(np.uint64), ref_val.view(np.uint64))
    np.testing.assert_array_equal(aab.view(np.uint64), ref_aab.view(np.uint64))
    np.testing.assert_array_equal(nc, o["ncontrib"].reshape(-1)[pix])
    np.testing.assert_array_equal(tf.view(np.uint32), o["Tfinal"].reshape(-1)[pix].view(np.uint32))
    # the case is not vacuous: many pixels composite, and some stop early
    assert (nc > 0).mean() > 0.3 and (tf < g.eps_T).any()


def test_backward_on_pixel_subsets_adds_up(oracle):
    """The pixel-list backward over a partition of the grid sums to the
    full-view backward (same per-pixel arithmetic, any pixel order)."""
    sc, tx = tiny_scene(40, K=40)
    g = tiny_grid(eps_T=0.02)
    rng = np.random.default_rng(41)
    rad = rng.normal(size=(2, sc.K, 1, 2))
    gs = rng.normal(size=(2, g.H, g.W, 1, 2))
    gr, gt = oracle.backward_view(g, sc, tx, rad, gs)
    perm = rng.permutation(g.H * g.W).astype(np.int32)
    acc_r, acc_t = np.zeros_like(gr), np.zeros_like(gt)
    for part in np.array_split(perm, 3):
        gp = gs.reshape(2, -1, 1, 2)[:, part].transpose(1, 0, 2, 3)
        r, t = oracle.backward_pixels(g, sc, tx, rad, part, gp)
        acc_r += r
        acc_t += t
    np.testing.assert_allclose(acc_r, gr, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(acc_t, gt, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------ FLE basis pins
def test_fle_legendre_closed_forms(oracle):
    """P_l^m for l <= 2 against the closed forms (no Condon-Shortley phase)."""
    x = np.linspace(-0.97, 0.97, 31)
    P = oracle.assoc_legendre(2, x)
    s = np.sqrt(1 - x * x)
    np.testing.assert_allclose(P[0, 0], 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(P[1, 0], x, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(P[1, 1], s, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(P[2, 0], 0.5 * (3 * x * x - 1), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(P[2, 1], 3 * x * s, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(P[2, 2], 3 * (1 - x * x), rtol=1e-14, atol=1e-15)


def test_fle_legendre_matches_scipy():
    """scipy's lpmv carries the Condon-Shortley phase (-1)^m."""
    sp = pytest.importorskip("scipy.special")
    from oracle import oracle as O
    x = np.linspace(-0.99, 0.99, 41)
    P = O.assoc_legendre(9, x)
    for l in range(10):
        for m in range(l + 1):
            np.testing.assert_allclose(P[l, m], (-1) ** m * sp.lpmv(m, l, x), rtol=1e-10,
                                       atol=1e-10 * max(1.0, np.abs(P[l, m]).max()))


def test_fle_basis_is_orthonormal_on_the_sphere(oracle):
    """Gauss-Legendre in cos(theta) x uniform azimuth integrates Y_a conj(Y_b)
    exactly for l <= 9: the Gram matrix is the identity."""
    lmax = 9
    xg, wg = np.polynomial.legendre.leggauss(24)
    nphi = 32
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct = np.repeat(xg, nphi)
    st = np.sqrt(1 - ct * ct)
    ph = np.tile(phi, xg.size)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    w = np.repeat(wg, nphi) * (2 * np.pi / nphi)
    Y = oracle.fle_basis(dirs, np.zeros(3), lmax)            # centre at the origin
    G = (Y * w[:, None]).T @ Y.conj()
    np.testing.assert_allclose(G, np.eye(Y.shape[1]), atol=1e-12)


def test_fle_radiance_special_cases(oracle):
    """Only a_00: s = a / sqrt(4 pi) in every direction; only a_10:
    s = sqrt(3 / (4 pi)) cos(theta); only b_11: s = i sqrt(3/(8 pi)) sin(theta) e^{i phi}."""
    rng = np.random.default_rng(5)
    means = rng.normal(size=(7, 3))
    tx = rng.normal(size=3)
    u = means - tx
    rho = np.linalg.norm(u, axis=1)
    L = oracle.fle_count(2)
    c = np.zeros((1, 7, 2, L))
    c[0, :, 0, 0] = 2.5
    s = oracle.fle_radiance(c, means, tx, 2)[0, :, 0]
    np.testing.assert_allclose(s[:, 0], 2.5 / np.sqrt(4 * np.pi), rtol=1e-14)
    np.testing.assert_allclose(s[:, 1], 0.0, atol=1e-15)
    c[:] = 0
    c[0, :, 0, 2] = 1.0                                       # (l, m) = (1, 0)
    s = oracle.fle_radiance(c, means, tx, 2)[0, :, 0]
    np.testing.assert_allclose(s[:, 0], np.sqrt(3 / (4 * np.pi)) * u[:, 2] / rho, rtol=1e-13)
    c[:] = 0
    c[0, :, 1, 3] = 1.0                                       # b_11: i * N11 P11 e^{i phi}
    s = oracle.fle_radiance(c, means, tx, 2)[0, :, 0]
    h = np.hypot(u[:, 0], u[:, 1])
    e = (u[:, 0] + 1j * u[:, 1]) / h
    ref = 1j * np.sqrt(3 / (8 * np.pi)) * (h / rho) * e
    np.testing.assert_allclose(s[:, 0], ref.real, atol=1e-14)
    np.testing.assert_allclose(s[:, 1], ref.imag, atol=1e-14)


def test_fle_backward_is_the_adjoint(oracle):
    """<g, J c> = <J^T g, c> for the linear map coefficients -> radiance."""
    rng = np.random.default_rng(6)
    lmax, N, K = 4, 3, 11
    means, tx = rng.normal(size=(K, 3)), rng.normal(size=3)
    c = rng.normal(size=(N, K, 2, oracle.fle_count(lmax)))
    g = rng.normal(size=(N, K, 1, 2))
    lhs = (g * oracle.fle_radiance(c, means, tx, lmax)).sum()
    rhs = (oracle.fle_backward(g, means, tx, lmax) * c).sum()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


# ---------------------------------------------- occupancy grid and probes
class _Sc:
    def __init__(self, means, log_scales, opacity):
        self.means, self.log_scales, self.opacity = means, log_scales, opacity
        self.quats = np.tile(np.array([1, 0, 0, 0], np.float32), (means.shape[0], 1))


def test_occupancy_single_gaussian_closed_form(oracle):
    """One isotropic Gaussian among two far corner anchors of zero opacity:
    every voxel within 2 sigma holds tau exp(-|c - p|^2 / (2 sigma^2))."""
    means = np.array([[0, 0, 0], [8, 8, 8], [4.01, 3.97, 4.02]], np.float32)
    ls = np.log(np.array([[0.1] * 3, [0.1] * 3, [0.5] * 3], np.float32))
    op = np.array([0.0, 0.0, 0.7], np.float32)
    grid, lo, D = oracle.occupancy_grid(_Sc(means, ls, op), res=32)
    idx = np.argwhere(grid > 0)
    c = lo.astype(np.float64) + (idx + 0.5) * D.astype(np.float64)
    r2 = ((c - means[2].astype(np.float64)) ** 2).sum(axis=1)
    np.testing.assert_allclose(grid[tuple(idx.T)], 0.7 * np.exp(-r2 / (2 * 0.5 ** 2)), rtol=1e-6)
    assert np.all(np.abs(c - means[2]) <= 2 * 0.5 + 1e-6)
    assert idx.shape[0] > 100


def test_occupancy_probes_clear_and_uniform_slab(oracle):
    """An empty grid gives T = 1, rho_bar = 0 (the clear features); a grid of
    uniform density rho0 gives T = (1 - rho0)^16 and rho_bar = rho0 for a
    receiver-Gaussian segment inside it."""
    rng = np.random.default_rng(3)
    means = rng.uniform(0, 5, size=(6, 3)).astype(np.float32)
    rx = rng.uniform(1, 4, size=(2, 3)).astype(np.float32)
    lo = np.zeros(3, np.float32)
    D = np.full(3, 5.0 / 16, np.float32)
    T, rb = oracle.occupancy_probes((np.zeros((16, 16, 16)), lo, D), rx, means)
    np.testing.assert_array_equal(T, 1.0)
    np.testing.assert_array_equal(rb, 0.0)
    T, rb = oracle.occupancy_probes((np.full((16, 16, 16), 0.2), lo, D), rx, means)
    np.testing.assert_allclose(T, 0.8 ** 16, rtol=1e-12)
    np.testing.assert_allclose(rb, 0.2, rtol=1e-12)
    T, rb = oracle.occupancy_probes((np.full((16, 16, 16), 3.0), lo, D), rx, means)
    np.testing.assert_array_equal(T, 0.0)        # densities clamp to 1
    np.testing.assert_allclose(rb, 1.0)


def test_mlp_with_empty_occupancy_equals_clear_features(oracle):
    rng = np.random.default_rng(4)
    from paper_2605_24290_gb300 import synthetic as S
    sc = S.draw_scene(rng, 20)
    mlp = S.draw_mlp(rng, 1)
    base = S.draw_base(rng, 20, 1)
    rx = S.draw_points(rng, 3)
    grid, lo, D = oracle.occupancy_grid(sc, res=16)
    a = oracle.mlp_radiance(mlp, rx, sc.means, base, occ=(np.zeros_like(grid), lo, D))
    b = oracle.mlp_radiance(mlp, rx, sc.means, base)
    np.testing.assert_array_equal(a, b)


def test_mlp_backward_with_occupancy_matches_finite_differences(oracle):
    """The occlusion inputs enter dW1 through columns 4 and 5 (T, rho_bar)."""
    rng = np.random.default_rng(8)
    from paper_2605_24290_gb300 import synthetic as S
    K, N = 40, 3
    sc = S.draw_scene(rng, K, box=(3.0, 3.0, 2.0))
    sc.log_scales[:] = np.log(0.4)
    sc.opacity[:] = 0.5
    mlp = S.draw_mlp(rng, 1)
    base = S.draw_base(rng, K, 1)
    rx = S.draw_points(rng, N, box=(3.0, 3.0, 2.0))
    occ = oracle.occupancy_grid(sc, res=16)
    T, rb = oracle.occupancy_probes(occ, rx, sc.means)
    assert T.min() < 0.99 and rb.max() > 0.01          # the probes see occupancy
    g = rng.normal(size=(N, K, 1, 2))
    grads = oracle.mlp_backward(mlp, rx, sc.means, base, g, occ=occ)
    for (u, i) in [(3, 4), (10, 5), (7, 4)]:
        h = 1e-6
        P1 = {k: v.copy() for k, v in mlp.items()}
        P2 = {k: v.copy() for k, v in mlp.items()}
        P1["l_w1"] = P1["l_w1"].astype(np.float64)
        P2["l_w1"] = P2["l_w1"].astype(np.float64)
        P1["l_w1"][u, i] += h
        P2["l_w1"][u, i] -= h
        f1 = (g * oracle.mlp_radiance(P1, rx, sc.means, base, occ=occ)).sum()
        f2 = (g * oracle.mlp_radiance(P2, rx, sc.means, base, occ=occ)).sum()
        fd = (f1 - f2) / (2 * h)
        assert abs(fd - grads["l_w1"][u, i]) <= 1e-6 * (1 + abs(fd)), (u, i, fd, grads["l_w1"][u, i])


# ------------- global FiLM over FLE components (Eq. rx_enc, film, film_apply)
def _tiny_film(lmax, nw, dc, D, w3, b3):
    din = 2 * nw + 2 + dc
    return {"omega": np.zeros((nw, 3)), "embed": np.zeros((oracle_L(lmax), dc)),
            "w1": np.zeros((D, din)), "b1": np.zeros(D), "w2": np.zeros((D, D)),
            "b2": np.zeros(D), "w3": np.asarray(w3, float), "b3": np.asarray(b3, float)}


def oracle_L(lmax):
    return (lmax + 1) ** 2


def test_rx_encoding_hand_values(oracle):
    """Interleaved [sin(w_1.r), cos(w_1.r), sin(w_2.r), cos(w_2.r)]."""
    om = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    r = np.array([[np.pi / 2, np.pi / 8, 5.0]])
    g = oracle.rx_encoding(r, om)[0]
    h = np.sqrt(0.5)
    np.testing.assert_allclose(g, [1.0, 0.0, h, h], atol=1e-15)


def test_film_component_features_index_map(oracle):
    """Component l*l + l + m carries (l, m) / lmax."""
    c = oracle.film_component_features(2)
    np.testing.assert_array_equal(c[0], [0.0, 0.0])
    np.testing.assert_array_equal(c[3], [0.5, 0.5])       # (1, 1)
    np.testing.assert_array_equal(c[5], [1.0, -0.5])      # (2, -1)
    np.testing.assert_array_equal(c[8], [1.0, 1.0])       # (2, 2)
    np.testing.assert_array_equal(oracle.film_component_features(0), [[0.0, 0.0]])


def test_film_zero_final_layer_is_identity(oracle):
    """Zero-initialised final layer (App. E.4): every receiver sees the base
    coefficients unchanged."""
    rng = np.random.default_rng(40)
    lmax, K, N = 3, 6, 4
    film = S.draw_film(rng, lmax, F=2, dc=3, D=8)
    film["w3"][:] = 0.0
    film["b3"][:] = 0.0
    base = S.draw_fle_base(rng, K, lmax)
    c = oracle.film_fle_coeffs(film, base, rng.normal(size=(N, 3)), lmax)
    for j in range(N):
        np.testing.assert_array_equal(c[j], base.astype(np.float64))


def test_film_apply_complex_affine_hand_value(oracle):
    """w3 = 0, b3 = (0.5, 0.25, 0.1, -0.2): (1.5 + 0.25i)(1 + 2i) + (0.1 - 0.2i)
    = 1.1 + 3.05i."""
    film = _tiny_film(0, 1, 1, 2, np.zeros((4, 2)), [0.5, 0.25, 0.1, -0.2])
    base = np.zeros((1, 2, 1))
    base[0, 0, 0], base[0, 1, 0] = 1.0, 2.0
    c = oracle.film_fle_coeffs(film, base, np.zeros((1, 3)), 0)
    np.testing.assert_allclose(c[0, 0, :, 0], [1.1, 3.05], rtol=1e-15)


def test_film_mlp_hand_network(oracle):
    """A hand-wired 3-layer network over x = [sin, cos, c_l, c_m, e_l]:
    h1 = relu(s), relu(-s), relu(c_m + e); h2 = w2 h1 with w2 not
    symmetric; outputs a.re = h2_0, a.im = h2_2, b.re = h2_1.  With
    s = sin(w.r) = +-1/2 and embeddings (0.5, 0.25, -0.5, 2) over lmax = 1."""
    w3 = np.zeros((4, 3))
    w3[0, 0], w3[1, 2], w3[2, 1] = 1.0, 1.0, 1.0
    film = _tiny_film(1, 1, 1, 3, w3, np.zeros(4))
    film["omega"][0] = (1.0, 0.0, 0.0)
    film["embed"][:, 0] = (0.5, 0.25, -0.5, 2.0)
    film["w1"][0, 0], film["w1"][1, 0] = 1.0, -1.0
    film["w1"][2, 3], film["w1"][2, 4] = 1.0, 1.0
    film["w2"][:] = [[1.0, 2.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]
    rx = np.array([[np.pi / 6, 0.0, 0.0], [-np.pi / 6, 0.0, 0.0]])
    ab = oracle.film_global(film, rx, 1)                       # [2, 4, 4]
    np.testing.assert_allclose(ab[0, :, 0], 0.5, rtol=1e-14)  # relu(s)
    np.testing.assert_allclose(ab[1, :, 0], 1.0, rtol=1e-14)  # 2 relu(-s)
    np.testing.assert_allclose(ab[0, :, 2], 0.0, atol=1e-15)
    np.testing.assert_allclose(ab[1, :, 2], 0.5, rtol=1e-14)
    for j in range(2):                                         # relu(m + e_l)
        np.testing.assert_allclose(ab[j, :, 1], [0.5, 0.0, 0.0, 3.0], atol=1e-15)
    np.testing.assert_array_equal(ab[..., 3], 0.0)


def test_film_backward_matches_finite_differences(oracle):
    """Every FiLM parameter and the base coefficients against central
    differences of film_fle_coeffs."""
    rng = np.random.default_rng(41)
    lmax, K, N = 2, 3, 3
    film = {k: v.astype(np.float64) for k, v in
            S.draw_film(rng, lmax, F=2, dc=3, D=5, out_scale=1.0).items()}
    base = S.draw_fle_base(rng, K, lmax).astype(np.float64)
    rx = rng.uniform(-1.0, 1.0, size=(N, 3))
    gc = rng.normal(size=(N, K, 2, oracle.fle_count(lmax)))
    got = oracle.film_fle_backward(film, base, rx, lmax, gc)

    def loss(f, b):
        return float((gc * oracle.film_fle_coeffs(f, b, rx, lmax)).sum())

    h = 1e-6
    for name in ["omega", "embed", "w1", "b1", "w2", "b2", "w3", "b3", "base"]:
        ref = np.zeros_like(got[name])
        src = base if name == "base" else film[name]
        for idx in np.ndindex(src.shape):
            keep = src[idx]
            src[idx] = keep + h
            lp = loss(film, base)
            src[idx] = keep - h
            lm = loss(film, base)
            src[idx] = keep
            ref[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(got[name], ref, rtol=1e-6, atol=1e-7, err_msg=name)


def test_film_degree_zero_radiance_closed_form(oracle):
    """lmax = 0: one component, Y_00 = 1/sqrt(4 pi) in every direction, so the
    conditioned radiance is ((1 + a) phi + b) / sqrt(4 pi) for each receiver."""
    rng = np.random.default_rng(42)
    film = {k: v.astype(np.float64) for k, v in S.draw_film(rng, 0, F=2, dc=3, D=6,
                                                             out_scale=1.0).items()}
    K, N = 5, 3
    base = S.draw_fle_base(rng, K, 0).astype(np.float64)
    r = rng.uniform(-1.0, 1.0, size=(N, 3))
    means, tx = rng.normal(size=(K, 3)), rng.normal(size=3)
    s = oracle.fle_radiance(oracle.film_fle_coeffs(film, base, r, 0), means, tx, 0)[:, :, 0]
    ab = oracle.film_global(film, r, 0)[:, 0]                         # [N, 4]
    a = (1.0 + ab[:, 0]) + 1j * ab[:, 1]
    b = ab[:, 2] + 1j * ab[:, 3]
    phi = base[:, 0, 0] + 1j * base[:, 1, 0]
    ref = (a[:, None] * phi[None] + b[:, None]) / np.sqrt(4 * np.pi)
    np.testing.assert_allclose(s[..., 0], ref.real, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(s[..., 1], ref.imag, rtol=1e-13, atol=1e-15)



# ------------------- Eq. combined_local over FLE components (Sec. 3.3.2)

def _film_local_case(rng, lmax=2, K=4, N=3, out_scale=1.0):
    film = {k: v.astype(np.float64) for k, v in
            S.draw_film(rng, lmax, F=2, dc=3, D=5, out_scale=out_scale).items()}
    params = {k: v.astype(np.float64) for k, v in S.draw_mlp(rng, 1, final_scale=0.5).items()}
    base = S.draw_fle_base(rng, K, lmax).astype(np.float64)
    rx = rng.uniform(-1.0, 1.0, size=(N, 3))
    means = rng.uniform(-2.0, 2.0, size=(K, 3))
    return film, params, base, rx, means


def test_film_local_zero_final_layer_is_film_only(oracle):
    """A local branch whose final layer is zero is the identity (Sec. 3.3.2:
    zero-initialised final layers): the composed coefficients equal the
    FiLM-modulated ones exactly."""
    rng = np.random.default_rng(50)
    lmax = 3
    film, params, base, rx, means = _film_local_case(rng, lmax=lmax)
    params["l_w2"][:] = 0.0
    params["l_b2"][:] = 0.0
    got = oracle.film_local_fle_coeffs(film, params, base, rx, means, lmax)
    ref = oracle.film_fle_coeffs(film, base, rx, lmax)
    np.testing.assert_array_equal(got, ref)


def test_film_local_complex_affine_hand_value(oracle):
    """With the local branch's output fixed by its bias (alpha = 0.3 - 0.2i,
    beta = -0.1 + 0.4i), one coefficient (1 + a) phi + b = 1.5 + 2i becomes
    (1.3 - 0.2i)(1.5 + 2i) + (-0.1 + 0.4i) = (1.95 + 0.4) + (2.6 - 0.3)i
    - 0.1 + 0.4i = 2.25 + 2.7i: a complex product, not an elementwise one
    (which would give 1.85 + 2.0i)."""
    rng = np.random.default_rng(51)
    lmax = 0
    film, params, base, rx, means = _film_local_case(rng, lmax=lmax, K=1, N=1)
    film["w3"][:] = 0.0
    film["b3"][:] = 0.0                                  # a = b = 0: c = phi_base
    base[0, :, 0] = [1.5, 2.0]
    params["l_w2"][:] = 0.0
    params["l_b2"][:] = [0.3, -0.2, -0.1, 0.4]           # (alpha.re, alpha.im, beta.re, beta.im)
    got = oracle.film_local_fle_coeffs(film, params, base, rx, means, lmax)
    assert got[0, 0, 0, 0] == pytest.approx(2.25, abs=1e-14)
    assert got[0, 0, 1, 0] == pytest.approx(2.7, abs=1e-14)


def test_film_local_backward_matches_finite_differences(oracle):
    """The local branch's parameters, the base coefficients and FiLM
    parameters against central differences of film_local_fle_coeffs."""
    rng = np.random.default_rng(52)
    lmax, K, N = 2, 4, 3
    film, params, base, rx, means = _film_local_case(rng, lmax=lmax, K=K, N=N)
    gc = rng.normal(size=(N, K, 2, oracle.fle_count(lmax)))
    got = oracle.film_local_fle_backward(film, params, base, rx, means, lmax, gc)

    def loss():
        return float((gc * oracle.film_local_fle_coeffs(film, params, base, rx, means,
                                                        lmax)).sum())

    h = 1e-6
    groups = [("l_w1", params), ("l_b1", params), ("l_w2", params), ("l_b2", params),
              ("base", None), ("w3", film), ("b1", film), ("omega", film)]
    for name, owner in groups:
        src = base if owner is None else owner[name]
        ref = np.zeros_like(got[name])
        for idx in np.ndindex(src.shape):
            keep = src[idx]
            src[idx] = keep + h
            lp = loss()
            src[idx] = keep - h
            lm = loss()
            src[idx] = keep
            ref[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(got[name], ref, rtol=1e-6, atol=1e-7, err_msg=name)
