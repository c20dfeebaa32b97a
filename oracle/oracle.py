"""Python face of the CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`.  The product library never
imports, links or executes anything in `oracle/`.

The render itself lives in `rxgs_oracle.c` (plain C, float64 values with a
float32 decision shadow); this module compiles it with gcc, loads it with
ctypes and adds, in float64 numpy, the conditioning MLP (Sec. 3.3.2), the
FLE directional basis (App. E.2), the occupancy grid and its probes
(App. E.5), the global FiLM branch over FLE components (Eq. rx_enc, film,
film_apply), its composition with the local branch (Eq. combined_local) and
the Stage II step (App. E.3 L1 term, Adam of App. E.5), each with its
backward where the path has one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rxgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Grid(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("theta0_deg", ctypes.c_double),
                ("step_deg", ctypes.c_double), ("TH", ctypes.c_int), ("TW", ctypes.c_int),
                ("eps_T", ctypes.c_float), ("q_max", ctypes.c_float), ("r_near", ctypes.c_float)]


def make_grid(g) -> Grid:
    """Accepts any object with the fields of `synthetic.Grid`."""
    return Grid(int(g.H), int(g.W), float(g.theta0_deg), float(g.step_deg), int(g.tile_h),
                int(g.tile_w), float(g.eps_T), float(g.q_max), float(g.r_near))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            _lib.or_exp32.restype = ctypes.c_float
            _lib.or_exp32.argtypes = [ctypes.c_float]
            _lib.or_atan2_32.restype = ctypes.c_float
            _lib.or_atan2_32.argtypes = [ctypes.c_float, ctypes.c_float]
            _lib.or_cov32.argtypes = [P, P, P]
            _lib.or_cov64.argtypes = [P, P, P]
            _lib.or_sigma2d64.argtypes = [P, P, P, P, P]
            _lib.or_project_view32.restype = ctypes.c_int
            _lib.or_project_view32.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, P]
            _lib.or_tile_lists.restype = ctypes.c_long
            _lib.or_tile_lists.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_long, P]
            _lib.or_render_view.restype = ctypes.c_int
            _lib.or_render_view.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                            ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int]
            _lib.or_render_pixels.restype = ctypes.c_int
            _lib.or_render_pixels.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                              ctypes.c_int, P, ctypes.c_int, P, P, P, P, P]
            _lib.or_backward_view.restype = ctypes.c_int
            _lib.or_backward_view.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                              ctypes.c_int, P, P, P, P, P, P, ctypes.c_int]
            _lib.or_backward_pixels.restype = ctypes.c_int
            _lib.or_backward_pixels.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_int,
                                                ctypes.c_int, P, ctypes.c_int, P, P, P, P]
            _lib.or_omp_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(lib().or_omp_threads())


def exp32(x: float) -> np.float32:
    return np.float32(lib().or_exp32(ctypes.c_float(x)))


def atan2_32(y: float, x: float) -> np.float32:
    return np.float32(lib().or_atan2_32(ctypes.c_float(y), ctypes.c_float(x)))


def cov32(log_scales, quats):
    s, q = _c32(log_scales), _c32(quats)
    out = np.zeros((s.shape[0], 6), np.float32)
    L = lib()
    for k in range(s.shape[0]):
        L.or_cov32(_p(s[k]), _p(q[k]), _p(out[k]))
    return out


def cov64(log_scales, quats):
    s, q = _c32(log_scales), _c32(quats)
    out = np.zeros((s.shape[0], 6), np.float64)
    L = lib()
    for k in range(s.shape[0]):
        L.or_cov64(_p(s[k]), _p(q[k]), _p(out[k]))
    return out


def sigma2d64(grid, mean, S6, centre):
    g = make_grid(grid)
    out = np.zeros(3, np.float64)
    lib().or_sigma2d64(ctypes.byref(g), _p(_c32(mean)), _p(_c64(S6)), _p(_c32(centre)), _p(out))
    return out


def project_view32(grid, scene, centre):
    """float32 shadow of the projection: (Sigma[K,6], rec[K,8], box[K,4])."""
    g = make_grid(grid)
    K = scene.K
    S6 = np.zeros((K, 6), np.float32)
    rec = np.zeros((K, 8), np.float32)
    box = np.zeros((K, 4), np.int32)
    lib().or_project_view32(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                            _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                            _p(S6), _p(rec), _p(box))
    return S6, rec, box


def tile_lists(grid, scene, centre, cap=None):
    """Per-tile depth-sorted lists: (counts[tiles], lists[total], ntiles[K])."""
    g = make_grid(grid)
    K = scene.K
    T = ((grid.H + grid.tile_h - 1) // grid.tile_h) * ((grid.W + grid.tile_w - 1) // grid.tile_w)
    counts = np.zeros(T, np.int32)
    ntiles = np.zeros(K, np.int32)
    cap = cap or max(1, K * 8)
    while True:
        lists = np.zeros(cap, np.int32)
        n = lib().or_tile_lists(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                                _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                                _p(counts), _p(lists), cap, _p(ntiles))
        if n == -1:
            cap *= 4
            continue
        if n < 0:
            raise MemoryError("oracle tile_lists failed")
        return counts, lists[:n].copy(), ntiles


def render_view(grid, scene, centre, radiance, use_eps=True, want_abs=True, want_w=False,
                want_spectra=True):
    """Render one view for all receivers of `radiance` [N,K,C,2].

    Returns dict(spectra[N,H,W,C,2] f64, absacc[N,H,W,C] f64,
    ncontrib[H,W] i32, Tfinal[H,W] f32, T64[H,W] f64, Wvis[K] f64 or None)."""
    g = make_grid(grid)
    rad = _c64(radiance)
    N, K, C = rad.shape[0], rad.shape[1], rad.shape[2]
    assert K == scene.K
    H, W = grid.H, grid.W
    spec = np.zeros((N, H, W, C, 2), np.float64) if want_spectra else None
    aab = np.zeros((N, H, W, C), np.float64) if want_abs else None
    ncon = np.zeros((H, W), np.int32)
    Tf = np.zeros((H, W), np.float32)
    T64 = np.zeros((H, W), np.float64)
    Wv = np.zeros(K, np.float64) if want_w else None
    rc = lib().or_render_view(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                              _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                              N, C, _p(rad), _p(spec), _p(aab), _p(ncon), _p(Tf), _p(T64), _p(Wv),
                              1 if use_eps else 0)
    if rc != 0:
        raise MemoryError("oracle render failed")
    return dict(spectra=spec, absacc=aab, ncontrib=ncon, Tfinal=Tf, T64=T64, Wvis=Wv)


def render_pixels(grid, scene, centre, radiance, pix):
    """Render only the pixels pix[np] (= i*W + jj).  Returns
    (values[np,N,C,2], absacc[np,N,C], ncontrib[np], Tfinal[np])."""
    g = make_grid(grid)
    rad = _c64(radiance)
    N, K, C = rad.shape[0], rad.shape[1], rad.shape[2]
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    npx = pix.shape[0]
    out = np.zeros((npx, N, C, 2), np.float64)
    aab = np.zeros((npx, N, C), np.float64)
    ncon = np.zeros(npx, np.int32)
    Tf = np.zeros(npx, np.float32)
    rc = lib().or_render_pixels(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                                _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                                N, C, _p(rad), npx, _p(pix), _p(out), _p(aab), _p(ncon), _p(Tf))
    if rc != 0:
        raise MemoryError("oracle render failed")
    return out, aab, ncon, Tf


def backward_view(grid, scene, centre, radiance, gspec, use_eps=True, want_abs=False):
    """dL/d radiance [N,K,C,2] and dL/d opacity [K] for cotangent gspec
    [N,H,W,C,2] on the spectra of one view.  With want_abs, also the sums of
    absolute terms (error scales) of both."""
    g = make_grid(grid)
    rad = _c64(radiance)
    N, K, C = rad.shape[0], rad.shape[1], rad.shape[2]
    gr = np.zeros_like(rad)
    gt = np.zeros(K, np.float64)
    ar = np.zeros_like(rad) if want_abs else None
    at = np.zeros(K, np.float64) if want_abs else None
    rc = lib().or_backward_view(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                                _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                                N, C, _p(rad), _p(_c64(gspec)), _p(gr), _p(gt), _p(ar), _p(at),
                                1 if use_eps else 0)
    if rc != 0:
        raise MemoryError("oracle backward failed")
    if want_abs:
        return gr, gt, ar, at
    return gr, gt


def backward_pixels(grid, scene, centre, radiance, pix, gpix):
    """Backward restricted to pixels pix[np] with cotangent gpix[np,N,C,2]:
    (dL/d radiance [N,K,C,2], dL/d opacity [K])."""
    g = make_grid(grid)
    rad = _c64(radiance)
    N, K, C = rad.shape[0], rad.shape[1], rad.shape[2]
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    gr = np.zeros_like(rad)
    gt = np.zeros(K, np.float64)
    rc = lib().or_backward_pixels(ctypes.byref(g), K, _p(_c32(scene.means)), _p(_c32(scene.log_scales)),
                                  _p(_c32(scene.quats)), _p(_c32(scene.opacity)), _p(_c32(centre)),
                                  N, C, _p(rad), int(pix.shape[0]), _p(pix), _p(_c64(gpix)), _p(gr),
                                  _p(gt))
    if rc != 0:
        raise MemoryError("oracle backward failed")
    return gr, gt


# ------------------------------------------------------------- reductions

def amplitude(spec):
    """|R| = sqrt(Re^2 + Im^2 + 1e-8)   (App. E.2)."""
    return np.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)


def csi(spec):
    """Coherent sum over all directions: [N,H,W,C,2] -> [N,C,2] (Def. 2)."""
    return spec.sum(axis=(1, 2))


def rssi(spec):
    """|sum over directions| of the single channel: [N,H,W,1,2] -> [N]."""
    s = csi(spec)[:, 0, :]
    return np.sqrt(s[:, 0] ** 2 + s[:, 1] ** 2)


# ------------------------------------------------- conditioning MLP (f64)

def _bf16(a):
    """Round float64 -> float32 -> bfloat16 (nearest even), back to float64."""
    x = np.ascontiguousarray(a, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _cmul(a, b):
    return np.stack([a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1],
                     a[..., 0] * b[..., 1] + a[..., 1] * b[..., 0]], axis=-1)


def _mlp(x, w1, b1, w2, b2, bf16):
    if bf16:
        x, w1, w2 = _bf16(x), _bf16(w1), _bf16(w2)
    h = np.maximum(x @ w1.T + b1, 0.0)
    if bf16:
        h = _bf16(h)
    return h @ w2.T + b2, h


def local_features(rx, means, occ=None):
    """[v_hat (3), d, T, rho_bar] per (receiver, Gaussian): v_hat points from
    the Gaussian to the receiver (Eq. local); T and rho_bar are the occlusion
    probes of `occ` (occupancy_probes), or 'clear' (T = 1, rho_bar = 0)."""
    r = np.asarray(rx, np.float64)[:, None, :]
    p = np.asarray(means, np.float64)[None, :, :]
    v = r - p
    d = np.sqrt((v ** 2).sum(-1, keepdims=True))
    vh = v / d
    if occ is None:
        T = np.ones_like(d)
        rb = np.zeros_like(d)
    else:
        T, rb = occupancy_probes(occ, rx, means)
        T, rb = T[..., None], rb[..., None]
    return np.concatenate([vh, d, T, rb], axis=-1)


# ------------------------- occupancy grid and occlusion probes (App. E.5)
# Grid: res^3 voxels over the bounding box [lo, hi] of the Gaussian means,
# voxel size D = (hi - lo) / res per axis (an axis of zero extent gets
# 1e-3 m), voxel centre lo + (i + 0.5) D.  Splat: Gaussian k adds
# tau_k exp(-1/2 sum_a ((c_a - p_a) / s_a)^2), s_a = sqrt(Sigma_aa) its
# standard deviation along axis a (from the float32 covariance of the
# decision specification), to every voxel centre within 2 s_a of p_a on
# every axis; densities are summed and clamped to [0, 1] when probed.  Probes:
# for Gaussian k and receiver j, x_s = p + t_s (r - p) at
# t_s = float32(0.05 + 0.06 s), s = 0..15; the voxel floor((x - lo) / D)
# (density 0 outside the grid); T = prod (1 - rho_s), rho_bar = mean rho_s.
# Every voxel range and index is decided in float32 with the written
# operation order (p - 2s - lo) / D - 0.5 and (x - lo) / D.

OCC_PROBES = 16


def occupancy_grid(scene, res: int = 128):
    """(grid [res,res,res] float64 densities, lo [3] f32, D [3] f32)."""
    f = np.float32
    p = np.asarray(scene.means, f)
    S32 = cov32(scene.log_scales, scene.quats)                # [K][00 01 02 11 12 22]
    s = np.sqrt(S32[:, [0, 3, 5]]).astype(f)
    tau = np.asarray(scene.opacity, np.float64)
    lo = p.min(axis=0).astype(f)
    hi = p.max(axis=0).astype(f)
    ext = (hi - lo).astype(f)
    ext = np.where(ext > f(0), ext, f(1e-3)).astype(f)
    D = (ext / f(res)).astype(f)
    two_s = (f(2) * s).astype(f)
    a_lo = ((p - two_s) - lo) / D - f(0.5)
    a_hi = ((p + two_s) - lo) / D - f(0.5)
    i_lo = np.maximum(np.ceil(a_lo).astype(np.int64), 0)
    i_hi = np.minimum(np.floor(a_hi).astype(np.int64), res - 1)
    grid = np.zeros((res, res, res), np.float64)
    for k in range(p.shape[0]):
        if np.any(i_lo[k] > i_hi[k]):
            continue
        axes = []
        for a in range(3):
            idx = np.arange(i_lo[k, a], i_hi[k, a] + 1)
            c = lo[a].astype(np.float64) + (idx + 0.5) * D[a].astype(np.float64)
            axes.append((idx, ((c - p[k, a]) / s[k, a]) ** 2))
        q = axes[0][1][:, None, None] + axes[1][1][None, :, None] + axes[2][1][None, None, :]
        grid[np.ix_(axes[0][0], axes[1][0], axes[2][0])] += tau[k] * np.exp(-0.5 * q)
    return grid, lo, D


def occupancy_probes(occ, rx, means):
    """(T [N,K], rho_bar [N,K]) of the occlusion probes (float64 values,
    float32 voxel decisions)."""
    grid, lo, D = occ
    f = np.float32
    res = grid.shape[0]
    p = np.asarray(means, f)[None, :, :]
    r = np.asarray(rx, f)[:, None, :]
    dvec = (r - p).astype(f)
    T = np.ones(dvec.shape[:2])
    acc = np.zeros(dvec.shape[:2])
    for s_ in range(OCC_PROBES):
        t = f(0.05 + 0.06 * s_)
        x = (p + (t * dvec).astype(f)).astype(f)
        u = (x - lo) / D
        idx = np.floor(u).astype(np.int64)
        inside = np.all((idx >= 0) & (idx < res), axis=-1)
        ic = np.clip(idx, 0, res - 1)
        rho = np.where(inside, np.minimum(grid[ic[..., 0], ic[..., 1], ic[..., 2]], 1.0), 0.0)
        T *= 1.0 - rho
        acc += rho
    return T, acc / OCC_PROBES


def mlp_radiance(params, rx, means, base, bf16=False, occ=None):
    """Receiver-conditioned radiance [N,K,C,2] (Eq. film, film_apply, local,
    combined_local): s = (1 + a_l) * ((1 + a_g) * phi_base + b_g) + b_l with
    complex products; each branch is Linear -> ReLU -> Linear with outputs
    (a.re, a.im, b.re, b.im) per channel."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    base = np.asarray(base, np.float64)
    K, C = base.shape[0], base.shape[1]
    rx = np.asarray(rx, np.float64)
    og, _ = _mlp(rx, P["g_w1"], P["g_b1"], P["g_w2"], P["g_b2"], bf16)        # [N,4C]
    ol, _ = _mlp(local_features(rx, means, occ), P["l_w1"], P["l_b1"], P["l_w2"], P["l_b2"], bf16)
    og = og.reshape(-1, 1, C, 4)
    ol = ol.reshape(rx.shape[0], K, C, 4)
    one = np.array([1.0, 0.0])
    u = _cmul(one + og[..., 0:2], base[None]) + og[..., 2:4]
    return _cmul(one + ol[..., 0:2], u) + ol[..., 2:4]


def mlp_backward(params, rx, means, base, grad_s, occ=None):
    """Gradients of sum(grad_s * s) w.r.t. phi_base [K,C,2] and every MLP
    parameter (float64, same names as `params`).

    With complex products z = a b, dL/da = g conj(b) and dL/db = g conj(a)."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    base = np.asarray(base, np.float64)
    rx = np.asarray(rx, np.float64)
    g = np.asarray(grad_s, np.float64)                       # [N,K,C,2]
    N, K, C = g.shape[0], g.shape[1], g.shape[2]
    xg = rx
    og, hg = _mlp(xg, P["g_w1"], P["g_b1"], P["g_w2"], P["g_b2"], False)
    xl = local_features(rx, means, occ)
    ol, hl = _mlp(xl, P["l_w1"], P["l_b1"], P["l_w2"], P["l_b2"], False)
    og4 = og.reshape(N, 1, C, 4)
    ol4 = ol.reshape(N, K, C, 4)
    one = np.array([1.0, 0.0])

    def conj(a):
        return np.stack([a[..., 0], -a[..., 1]], axis=-1)

    ag = one + og4[..., 0:2]
    al = one + ol4[..., 0:2]
    u = _cmul(ag, base[None]) + og4[..., 2:4]
    d_al = _cmul(g, conj(u))                  # dL/d a_l
    d_bl = g                                  # dL/d b_l
    d_u = _cmul(g, conj(al))
    d_ag = _cmul(d_u, conj(np.broadcast_to(base[None], d_u.shape))).sum(axis=1)   # [N,C,2]
    d_bg = d_u.sum(axis=1)
    d_base = _cmul(d_u, conj(np.broadcast_to(ag, d_u.shape))).sum(axis=0)         # [K,C,2]
    d_ol = np.concatenate([d_al, d_bl], axis=-1).reshape(N, K, 4 * C)
    d_og = np.concatenate([d_ag, d_bg], axis=-1).reshape(N, 4 * C)
    out = {"base": d_base}
    # local branch
    out["l_w2"] = np.einsum("nko,nkh->oh", d_ol, hl)
    out["l_b2"] = d_ol.sum(axis=(0, 1))
    d_hl = (d_ol @ P["l_w2"]) * (hl > 0)
    out["l_w1"] = np.einsum("nkh,nki->hi", d_hl, xl)
    out["l_b1"] = d_hl.sum(axis=(0, 1))
    # global branch
    out["g_w2"] = d_og.T @ hg
    out["g_b2"] = d_og.sum(axis=0)
    d_hg = (d_og @ P["g_w2"]) * (hg > 0)
    out["g_w1"] = d_hg.T @ xg
    out["g_b1"] = d_hg.sum(axis=0)
    return out


def _cmul_abs(A, B):
    """Bounds of |Re|, |Im| of a * b from bounds A, B of those of a and b."""
    return np.stack([A[..., 0] * B[..., 0] + A[..., 1] * B[..., 1],
                     A[..., 0] * B[..., 1] + A[..., 1] * B[..., 0]], axis=-1)


def mlp_backward_chain(params, rx, means, base, abs_grad_s, occ=None, amb=1e-5):
    """Error scales of `mlp_backward`: the same steps with every factor
    replaced by a bound of its absolute value (the absolute chain), so each
    returned entry bounds the sum of the absolute values of the terms that
    make up that gradient entry.  `abs_grad_s` [N,K,C,2] bounds the incoming
    gradient's terms.  ReLU units follow the forward's own activity.

    A unit whose pre-activation lies within `amb` of zero, relative to its
    own chain, is a decision float32 cannot settle: the GPU may take it either
    way, which adds or removes its whole term d_h * x in the first layer's
    gradients.  Such units count as active in the chain, and their first-layer
    terms are also returned apart, as the second dict, so that a comparison
    can admit both outcomes.  Returns (chain, ambiguous), keyed like
    `mlp_backward`."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    A = {k: np.abs(v) for k, v in P.items()}
    base = np.asarray(base, np.float64)
    G = np.abs(np.asarray(abs_grad_s, np.float64))
    N, K, C = G.shape[0], G.shape[1], G.shape[2]
    xg = np.asarray(rx, np.float64)
    xl = local_features(rx, means, occ)

    def layer(x, w1, b1, w2, b2, aw1, ab1, aw2, ab2):
        pre = x @ w1.T + b1
        cpre = np.abs(x) @ aw1.T + ab1
        amb_u = np.abs(pre) <= amb * cpre
        act = (pre > 0) | amb_u
        ch = cpre * act
        return ch @ aw2.T + ab2, ch, act, amb_u

    cog, chg, actg, ambg = layer(xg, P["g_w1"], P["g_b1"], P["g_w2"], P["g_b2"],
                                 A["g_w1"], A["g_b1"], A["g_w2"], A["g_b2"])
    col, chl, actl, ambl = layer(xl, P["l_w1"], P["l_b1"], P["l_w2"], P["l_b2"],
                                 A["l_w1"], A["l_b1"], A["l_w2"], A["l_b2"])
    cog4 = cog.reshape(N, 1, C, 4)
    col4 = col.reshape(N, K, C, 4)
    one = np.array([1.0, 0.0])
    AG = one + cog4[..., 0:2]
    AL = one + col4[..., 0:2]
    B = np.abs(base)[None]
    U = _cmul_abs(AG, B) + cog4[..., 2:4]
    D_al = _cmul_abs(G, U)
    D_u = _cmul_abs(G, AL)
    D_ag = _cmul_abs(D_u, np.broadcast_to(B, D_u.shape)).sum(axis=1)
    D_bg = D_u.sum(axis=1)
    out = {"base": _cmul_abs(D_u, np.broadcast_to(AG, D_u.shape)).sum(axis=0)}
    D_ol = np.concatenate([D_al, G], axis=-1).reshape(N, K, 4 * C)
    D_og = np.concatenate([D_ag, D_bg], axis=-1).reshape(N, 4 * C)
    amb_out = {k: np.zeros_like(v) for k, v in P.items()}
    amb_out["base"] = np.zeros_like(base)
    out["l_w2"] = np.einsum("nko,nkh->oh", D_ol, chl)
    out["l_b2"] = D_ol.sum(axis=(0, 1))
    D_hl = D_ol @ A["l_w2"]
    out["l_w1"] = np.einsum("nkh,nki->hi", D_hl * actl, np.abs(xl))
    out["l_b1"] = (D_hl * actl).sum(axis=(0, 1))
    amb_out["l_w1"] = np.einsum("nkh,nki->hi", D_hl * ambl, np.abs(xl))
    amb_out["l_b1"] = (D_hl * ambl).sum(axis=(0, 1))
    out["g_w2"] = D_og.T @ chg
    out["g_b2"] = D_og.sum(axis=0)
    D_hg = D_og @ A["g_w2"]
    out["g_w1"] = (D_hg * actg).T @ np.abs(xg)
    out["g_b1"] = (D_hg * actg).sum(axis=0)
    amb_out["g_w1"] = (D_hg * ambg).T @ np.abs(xg)
    amb_out["g_b1"] = (D_hg * ambg).sum(axis=0)
    return out, amb_out


# ----------------------------- Stage II step (Sec. 3.1; App. E.3, App. E.5)
# Geometry is frozen; phi_base and the conditioning MLP are trained against
# the L1 term of the loss (App. E.3) on the amplitude |R| (App. E.2) or on
# RSSI, each parameter group with its own Adam optimiser (App. E.5).  The
# SSIM and FFT terms of App. E.3 are not part of the path.

def l1_amplitude(spec, target):
    """L = mean over elements of | |R| - y | with |R| = sqrt(Re^2 + Im^2 +
    1e-8), spec [..., 2], target [...].  Returns (L, dL/dspec): the
    derivative of |R| is R / |R|, so dL/dspec = sign(|R| - y) / n * R / |R|."""
    spec = np.asarray(spec, np.float64)
    amp = amplitude(spec)
    diff = amp - np.asarray(target, np.float64)
    n = diff.size
    return float(np.abs(diff).mean()), (np.sign(diff) / n)[..., None] * spec / amp[..., None]


def l1_rssi(csi1, target):
    """L = mean | RSSI - y | with RSSI = |CSI| of a single channel, csi1
    [..., 2], target [...]; returns (L, dL/dcsi1) = sign(RSSI - y) / n *
    CSI / RSSI (zero where RSSI = 0)."""
    c = np.asarray(csi1, np.float64)
    r = np.sqrt(c[..., 0] ** 2 + c[..., 1] ** 2)
    diff = r - np.asarray(target, np.float64)
    n = diff.size
    safe = np.where(r > 0, r, 1.0)
    return float(np.abs(diff).mean()), ((np.sign(diff) / n) * (r > 0) / safe)[..., None] * c


def adam(p, g, m, v, t, lr, betas=(0.9, 0.999), eps=1e-8):
    """One update of Adam (Kingma & Ba, Algorithm 1), the optimiser App. E.5
    names, with PyTorch's default hyperparameters and no weight decay.  t is
    the 1-based step count.  Returns (p, m, v):
        m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
        p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    b1, b2 = betas
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def stage2_step(grid, scene, tx, rx, base, params, target, state=None, lr_base=5e-3,
                lr_mlp=1e-3, kind="spectra"):
    """One Stage II iteration: the receiver-conditioned radiance of every
    (receiver, Gaussian) pair (MLP), every transmitter's view rendered
    (brute force), the L1 loss against `target` (amplitude spectra
    [M,N,H,W,C] for kind "spectra", RSSI [M,N] for kind "rssi"), its
    gradient through the render backward (summed over views) and the MLP
    backward, then one Adam update of phi_base and one of the MLP parameters
    with separate optimiser states (App. E.5).

    `state` (None at the first step) is {"t": steps taken, name: (m, v)}.
    Returns dict(loss, grad_base, grad_mlp, base, params, state, spectra)."""
    M = tx.shape[0]
    rad = mlp_radiance(params, rx, scene.means, base)
    spec = np.stack([render_view(grid, scene, tx[v], rad, want_abs=False)["spectra"]
                     for v in range(M)])                                  # [M,N,H,W,C,2]
    if kind == "spectra":
        loss, gspec = l1_amplitude(spec, target)
    elif kind == "rssi":
        loss, gcsi = l1_rssi(csi(spec.reshape((-1,) + spec.shape[2:]))[:, 0].reshape(M, -1, 2),
                             target)
        gspec = np.broadcast_to(gcsi[:, :, None, None, None, :], spec.shape)
    else:
        raise ValueError(kind)
    grad_rad = None
    for v in range(M):
        gr, _ = backward_view(grid, scene, tx[v], rad, gspec[v])
        grad_rad = gr if grad_rad is None else grad_rad + gr
    grads = mlp_backward(params, rx, scene.means, base, grad_rad)
    st = {"t": 0} if state is None else dict(state)
    t = st["t"] + 1
    new_base, *mv = adam(base, grads["base"],
                         *st.get("base", (np.zeros_like(grads["base"]),) * 2), t, lr_base)
    st["base"] = tuple(mv)
    new_params = {}
    for k in params:
        new_params[k], *mv = adam(params[k], grads[k],
                                  *st.get(k, (np.zeros_like(grads[k]),) * 2), t, lr_mlp)
        st[k] = tuple(mv)
    st["t"] = t
    return dict(loss=loss, grad_base=grads["base"],
                grad_mlp={k: grads[k] for k in params}, base=new_base, params=new_params,
                state=st, spectra=spec)


# --------------------------------- FLE directional radiance (App. E.2, Alg. 1)
# For the direction from the transmitter to a Gaussian's centre, with polar
# angle theta (cos theta = u_z / |u|) and azimuth phi = atan2(u_y, u_x):
#   s = sum_{l <= lmax} sum_{|m| <= l} (a_lm + i b_lm) N_l|m| P_l^|m|(cos theta) e^{i m phi}
# i.e. Re s = sum [a cos(m phi) - b sin(m phi)] N P,  Im s = sum [a sin + b cos] N P,
# N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), P_l^m without the
# Condon-Shortley phase.  Component index of (l, m): l*l + l + m.

def fle_count(lmax: int) -> int:
    return (lmax + 1) ** 2


def assoc_legendre(lmax: int, x):
    """P_l^m(x), 0 <= m <= l <= lmax, no Condon-Shortley phase, by the
    three-term recurrence: P_m^m = (2m-1)!! (1-x^2)^(m/2),
    P_{m+1}^m = (2m+1) x P_m^m, (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m.
    Returns P[l, m, ...]."""
    x = np.asarray(x, np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = np.zeros((lmax + 1, lmax + 1) + x.shape, np.float64)
    pmm = np.ones_like(x)
    for m in range(lmax + 1):
        if m > 0:
            pmm = pmm * (2 * m - 1) * s
        P[m, m] = pmm
        if m + 1 <= lmax:
            P[m + 1, m] = (2 * m + 1) * x * pmm
        for l in range(m + 2, lmax + 1):
            P[l, m] = ((2 * l - 1) * x * P[l - 1, m] - (l + m - 1) * P[l - 2, m]) / (l - m)
    return P


def fle_norm(l: int, m: int) -> float:
    import math
    m = abs(m)
    return math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def fle_basis(means, centre, lmax: int):
    """Complex basis Y[K, L] of each Gaussian's direction from `centre`."""
    u = np.asarray(means, np.float64) - np.asarray(centre, np.float64)[None, :]
    rho = np.sqrt((u * u).sum(axis=1))
    ct = u[:, 2] / rho
    phi = np.arctan2(u[:, 1], u[:, 0])
    P = assoc_legendre(lmax, ct)
    Y = np.zeros((u.shape[0], fle_count(lmax)), np.complex128)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            Y[:, l * l + l + m] = fle_norm(l, m) * P[l, abs(m)] * np.exp(1j * m * phi)
    return Y


def fle_radiance(coeffs, means, centre, lmax: int):
    """Radiance [N,K,1,2] of one view from coefficients [N,K,2,L]."""
    c = np.asarray(coeffs, np.float64)
    Y = fle_basis(means, centre, lmax)                      # [K, L]
    s = ((c[:, :, 0, :] + 1j * c[:, :, 1, :]) * Y[None]).sum(axis=-1)   # [N, K]
    return np.stack([s.real, s.imag], axis=-1)[:, :, None, :]


def fle_backward(grad_rad, means, centre, lmax: int):
    """dL/dcoeffs [N,K,2,L] of one view from dL/dradiance [N,K,1,2]:
    dL/da = g_re Re Y + g_im Im Y, dL/db = -g_re Im Y + g_im Re Y."""
    g = np.asarray(grad_rad, np.float64)[:, :, 0, :]          # [N, K, 2]
    Y = fle_basis(means, centre, lmax)[None]                  # [1, K, L]
    da = g[..., 0:1] * Y.real + g[..., 1:2] * Y.imag
    db = -g[..., 0:1] * Y.imag + g[..., 1:2] * Y.real
    return np.stack([da, db], axis=2)


# ------------------ global branch over the FLE components (Eq. rx_enc, film, film_apply)
# Parameters (a dict of arrays; float64 inside):
#   omega [F, 3]   frequency vectors of the receiver encoding
#   embed [L, dc]  learnable component embeddings e_l
#   w1 [D, din], b1 [D], w2 [D, D], b2 [D], w3 [4, D], b3 [4],  din = 2F + 2 + dc
# The global MLP has three linear layers with ReLU between them (App. E.4);
# its four outputs per (receiver, component) are (a.re, a.im, b.re, b.im).
# Component l*l + l + m carries the degree/order feature c_l = (l, m) / max(lmax, 1).


def rx_encoding(rx, omega):
    """gamma(r) of Eq. rx_enc: [sin(w_1.r), cos(w_1.r), ..., sin(w_F.r), cos(w_F.r)]."""
    ph = np.asarray(rx, np.float64) @ np.asarray(omega, np.float64).T      # [N, F]
    out = np.empty(ph.shape[:-1] + (2 * ph.shape[-1],), np.float64)
    out[..., 0::2] = np.sin(ph)
    out[..., 1::2] = np.cos(ph)
    return out


def film_component_features(lmax: int):
    """c_l = (l, m) / max(lmax, 1) for component l*l + l + m: [L, 2]."""
    L = fle_count(lmax)
    c = np.zeros((L, 2), np.float64)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            c[l * l + l + m] = (l, m)
    return c / max(lmax, 1)


def film_inputs(film, rx, lmax: int):
    """x [N, L, din] = [gamma(r_j); c_l; e_l] (the input of Eq. film)."""
    g = rx_encoding(rx, film["omega"])                                    # [N, 2F]
    c = film_component_features(lmax)                                      # [L, 2]
    e = np.asarray(film["embed"], np.float64)                              # [L, dc]
    N, L = g.shape[0], c.shape[0]
    return np.concatenate([np.broadcast_to(g[:, None, :], (N, L, g.shape[1])),
                           np.broadcast_to(c[None], (N, L, 2)),
                           np.broadcast_to(e[None], (N, L, e.shape[1]))], axis=-1)


def _film_mlp(P, x):
    h1 = np.maximum(x @ P["w1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["w2"].T + P["b2"], 0.0)
    return h2 @ P["w3"].T + P["b3"], h1, h2


def film_global(film, rx, lmax: int):
    """(a_l, b_l) per receiver and component (Eq. film): [N, L, 4] =
    (a.re, a.im, b.re, b.im)."""
    P = {k: np.asarray(v, np.float64) for k, v in film.items()}
    out, _, _ = _film_mlp(P, film_inputs(P, rx, lmax))
    return out


def film_fle_coeffs(film, base, rx, lmax: int):
    """Per-receiver FLE coefficients [N,K,2,L] from the base coefficients
    base [K,2,L] (Eq. film_apply): (1 + a_l) phi_kl + b_l, complex, the same
    modulation for every Gaussian."""
    ab = film_global(film, rx, lmax)                                       # [N, L, 4]
    a = (1.0 + ab[..., 0]) + 1j * ab[..., 1]
    b = ab[..., 2] + 1j * ab[..., 3]
    base = np.asarray(base, np.float64)
    phi = base[:, 0, :] + 1j * base[:, 1, :]                               # [K, L]
    c = a[:, None, :] * phi[None] + b[:, None, :]                         # [N, K, L]
    return np.stack([c.real, c.imag], axis=2)


def film_fle_backward(film, base, rx, lmax: int, grad_coeffs):
    """Gradients of sum(grad_coeffs * coeffs) (coeffs = film_fle_coeffs)
    w.r.t. base [K,2,L] and every FiLM parameter (float64, same names as
    `film`).  With G = dL/dRe + i dL/dIm of a coefficient: dL/dphi = conj(1 + a) G,
    dL/da = conj(phi) G, dL/db = G."""
    P = {k: np.asarray(v, np.float64) for k, v in film.items()}
    base = np.asarray(base, np.float64)
    gc = np.asarray(grad_coeffs, np.float64)
    G = gc[:, :, 0, :] + 1j * gc[:, :, 1, :]                               # [N, K, L]
    x = film_inputs(P, rx, lmax)
    ab, h1, h2 = _film_mlp(P, x)
    a = (1.0 + ab[..., 0]) + 1j * ab[..., 1]                               # [N, L]
    phi = base[:, 0, :] + 1j * base[:, 1, :]
    d_phi = (np.conj(a)[:, None, :] * G).sum(axis=0)                        # [K, L]
    d_a = (np.conj(phi)[None] * G).sum(axis=1)                              # [N, L]
    d_b = G.sum(axis=1)
    d_out = np.stack([d_a.real, d_a.imag, d_b.real, d_b.imag], axis=-1)     # [N, L, 4]
    out = {"base": np.stack([d_phi.real, d_phi.imag], axis=1)}
    out["w3"] = np.einsum("nlo,nlh->oh", d_out, h2)
    out["b3"] = d_out.sum(axis=(0, 1))
    d_h2 = (d_out @ P["w3"]) * (h2 > 0)
    out["w2"] = np.einsum("nlo,nlh->oh", d_h2, h1)
    out["b2"] = d_h2.sum(axis=(0, 1))
    d_h1 = (d_h2 @ P["w2"]) * (h1 > 0)
    out["w1"] = np.einsum("nlo,nli->oi", d_h1, x)
    out["b1"] = d_h1.sum(axis=(0, 1))
    d_x = d_h1 @ P["w1"]                                                    # [N, L, din]
    F = P["omega"].shape[0]
    out["embed"] = d_x[..., 2 * F + 2:].sum(axis=0)
    d_g = d_x[..., :2 * F].sum(axis=1)                                      # [N, 2F]
    ph = np.asarray(rx, np.float64) @ P["omega"].T
    d_ph = d_g[:, 0::2] * np.cos(ph) - d_g[:, 1::2] * np.sin(ph)            # [N, F]
    out["omega"] = d_ph.T @ np.asarray(rx, np.float64)
    return out


# ------------------ Eq. combined_local over the FLE components (Sec. 3.3.2)
# The local branch (Eq. local) of the conditioning MLP gives one complex pair
# (alpha_loc, beta_loc) per (receiver j, Gaussian k) from [v_hat, d, T,
# rho_bar]; Eq. combined_local applies it to every component's coefficient
# after the global FiLM modulation (Eq. film_apply):
#   phi_jkl = (1 + alpha_jk) [(1 + a_jl) phi_base,kl + b_jl] + beta_jk.

def local_factors(params, rx, means, occ=None):
    """(alpha_loc, beta_loc): complex [N, K] each, the local branch's four
    outputs (alpha.re, alpha.im, beta.re, beta.im) for one channel."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    ol, _ = _mlp(local_features(rx, means, occ), P["l_w1"], P["l_b1"], P["l_w2"], P["l_b2"],
                 False)
    return ol[..., 0] + 1j * ol[..., 1], ol[..., 2] + 1j * ol[..., 3]


def film_local_fle_coeffs(film, params, base, rx, means, lmax: int, occ=None):
    """Per-receiver FLE coefficients [N,K,2,L] under both branches:
    (1 + alpha_jk) ((1 + a_jl) phi_kl + b_jl) + beta_jk."""
    c = film_fle_coeffs(film, base, rx, lmax)
    c = c[:, :, 0, :] + 1j * c[:, :, 1, :]                                 # [N, K, L]
    alpha, beta = local_factors(params, rx, means, occ)
    c2 = (1.0 + alpha)[..., None] * c + beta[..., None]
    return np.stack([c2.real, c2.imag], axis=2)


def film_local_fle_backward(film, params, base, rx, means, lmax: int, grad_coeffs, occ=None):
    """Gradients of sum(grad_coeffs * coeffs) (coeffs = film_local_fle_coeffs)
    w.r.t. base, every FiLM parameter (names of `film`) and the local branch
    (l_w1, l_b1, l_w2, l_b2).  With G' = dL/dRe + i dL/dIm of a coefficient:
    dL/dalpha_jk = sum_l conj(c_jkl) G'_jkl, dL/dbeta_jk = sum_l G'_jkl and
    the FiLM-modulated coefficient c gets conj(1 + alpha_jk) G'."""
    gc = np.asarray(grad_coeffs, np.float64)
    G2 = gc[:, :, 0, :] + 1j * gc[:, :, 1, :]                              # [N, K, L]
    c = film_fle_coeffs(film, base, rx, lmax)
    c = c[:, :, 0, :] + 1j * c[:, :, 1, :]
    alpha, _ = local_factors(params, rx, means, occ)
    d_alpha = (np.conj(c) * G2).sum(axis=-1)                               # [N, K]
    d_beta = G2.sum(axis=-1)
    G = np.conj(1.0 + alpha)[..., None] * G2
    out = film_fle_backward(film, base, rx, lmax, np.stack([G.real, G.imag], axis=2))
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    x = local_features(rx, means, occ)                                     # [N, K, 6]
    _, h = _mlp(x, P["l_w1"], P["l_b1"], P["l_w2"], P["l_b2"], False)      # h [N, K, H]
    d_ol = np.stack([d_alpha.real, d_alpha.imag, d_beta.real, d_beta.imag], axis=-1)
    out["l_w2"] = np.einsum("nko,nkh->oh", d_ol, h)
    out["l_b2"] = d_ol.sum(axis=(0, 1))
    d_h = (d_ol @ P["l_w2"]) * (h > 0)
    out["l_w1"] = np.einsum("nkh,nki->hi", d_h, x)
    out["l_b1"] = d_h.sum(axis=(0, 1))
    return out
