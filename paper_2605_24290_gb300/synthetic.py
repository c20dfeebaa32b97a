"""Seeded synthetic inputs shaped like indoor RF scenes.

This module only draws random numbers; it holds none of the renderer's
arithmetic.  It is the one module that both the CUDA path (tests, bench) and
the CPU oracle's tests take their inputs from.

Scene recipe (Sec. 2 scene representation; App. E.1 parameterisation):
  means        ~ U(box)                              [K,3]
  log-scales   ~ N(-2, 0.5) per axis                  [K,3]
  quaternions  = N(0,1)^4 (w,x,y,z), not normalised   [K,4]
  opacity      = sigmoid(N(0,1))                      [K]
  transmitters, receivers ~ U(box)                    [M,3], [N,3]
  radiance     = A(cos p, sin p), A ~ LogNormal(0,1), p ~ U(0, 2 pi)

Everything is drawn in float64 from numpy's PCG64 with a fixed draw order
and rounded once to float32.  The seed of a workload is 8371 + its index
(8371 is the paper's data-split seed, App. F).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 8371


@dataclasses.dataclass
class Scene:
    means: np.ndarray        # [K,3] float32
    log_scales: np.ndarray   # [K,3] float32
    quats: np.ndarray        # [K,4] float32, (w,x,y,z)
    opacity: np.ndarray      # [K]   float32 in (0,1)

    @property
    def K(self) -> int:
        return int(self.means.shape[0])


@dataclasses.dataclass
class Grid:
    H: int = 90
    W: int = 360
    theta0_deg: float = 0.0
    step_deg: float = 1.0
    tile_h: int = 16
    tile_w: int = 16
    eps_T: float = 1e-4
    q_max: float = 9.0
    r_near: float = 0.05


def f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def draw_scene(rng: np.random.Generator, K: int, box=(10.0, 8.0, 3.0),
               log_scale_mean: float = -2.0, log_scale_std: float = 0.5) -> Scene:
    box = np.asarray(box, dtype=np.float64)
    means = rng.uniform(0.0, 1.0, size=(K, 3)) * box
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(K, 3))
    quats = rng.normal(0.0, 1.0, size=(K, 4))
    logits = rng.normal(0.0, 1.0, size=(K,))
    opacity = 1.0 / (1.0 + np.exp(-logits))
    return Scene(f32(means), f32(log_scales), f32(quats), f32(opacity))


def draw_points(rng: np.random.Generator, n: int, box=(10.0, 8.0, 3.0)) -> np.ndarray:
    return f32(rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(box, dtype=np.float64))


def draw_radiance(rng: np.random.Generator, N: int, K: int, C: int = 1) -> np.ndarray:
    """Receiver-major complex radiance [N,K,C,2] (real, imag)."""
    amp = rng.lognormal(0.0, 1.0, size=(N, K, C))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(N, K, C))
    return f32(np.stack([amp * np.cos(ph), amp * np.sin(ph)], axis=-1))


def draw_base(rng: np.random.Generator, K: int, C: int = 1) -> np.ndarray:
    """Base coefficients phi_base [K,C,2] drawn like the radiance above."""
    return draw_radiance(rng, 1, K, C)[0]


MLP_HIDDEN = 64


def mlp_shapes(C: int, hidden: int = MLP_HIDDEN):
    """Parameter shapes of the two conditioning MLPs, in the flat order used
    everywhere (torch Linear convention: weight [out, in])."""
    return [
        ("g_w1", (hidden, 3)), ("g_b1", (hidden,)),
        ("g_w2", (4 * C, hidden)), ("g_b2", (4 * C,)),
        ("l_w1", (hidden, 6)), ("l_b1", (hidden,)),
        ("l_w2", (4 * C, hidden)), ("l_b2", (4 * C,)),
    ]


def draw_mlp(rng: np.random.Generator, C: int, hidden: int = MLP_HIDDEN,
             final_scale: float = 0.1) -> dict:
    """U(+-1/sqrt(fan_in)) init; the output layers are scaled by `final_scale`
    so that the modulation is small but not the identity."""
    out = {}
    fan_in_of = {"g_w1": 3, "g_b1": 3, "l_w1": 6, "l_b1": 6,
                 "g_w2": hidden, "g_b2": hidden, "l_w2": hidden, "l_b2": hidden}
    for name, shape in mlp_shapes(C, hidden):
        bound = 1.0 / math.sqrt(fan_in_of[name])
        a = rng.uniform(-bound, bound, size=shape)
        if name.endswith("w2") or name.endswith("b2"):
            a = a * final_scale
        out[name] = f32(a)
    return out


def flatten_mlp(params: dict, C: int, hidden: int = MLP_HIDDEN) -> np.ndarray:
    return f32(np.concatenate([params[n].reshape(-1) for n, _ in mlp_shapes(C, hidden)]))


def unflatten_mlp(flat: np.ndarray, C: int, hidden: int = MLP_HIDDEN) -> dict:
    out, o = {}, 0
    for name, shape in mlp_shapes(C, hidden):
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n]).reshape(shape)
        o += n
    return out


# ---------------------------------------------------------------- workloads

def workload_small(seed: int = SEED_BASE + 0, K: int = 4096, M: int = 1, N: int = 8):
    """4,096 Gaussians in a 10x8x3 m box, 1 transmitter, 8 receivers,
    explicit radiance [8,4096,1,2], 90x360 grid, 16x16 tiles."""
    rng = np.random.default_rng(seed)
    scene = draw_scene(rng, K)
    tx = draw_points(rng, M)
    rx = draw_points(rng, N)
    rad = draw_radiance(rng, N, K, 1)
    return dict(scene=scene, tx=tx, rx=rx, radiance=rad, grid=Grid())


def workload_mlp(seed: int = SEED_BASE + 1, K: int = 100_000, M: int = 32, N: int = 64,
                 C: int = 1):
    """100,000 Gaussians, 32 transmitters x 64 receivers, radiance from the
    2-layer 64-wide conditioning MLP, 90x360 grid, cotangent N(0,1) on
    spectra."""
    rng = np.random.default_rng(seed)
    scene = draw_scene(rng, K)
    tx = draw_points(rng, M)
    rx = draw_points(rng, N)
    base = draw_base(rng, K, C)
    mlp = draw_mlp(rng, C)
    return dict(scene=scene, tx=tx, rx=rx, base=base, mlp=mlp, C=C, grid=Grid())


def ragged_batches(rng: np.random.Generator, total: int = 256, lo: int = 1, hi: int = 64):
    sizes, s = [], 0
    while s < total:
        b = int(rng.integers(lo, hi + 1))
        b = min(b, total - s)
        sizes.append(b)
        s += b
    return sizes


def workload_csi(seed: int = SEED_BASE + 2, K: int = 300_000, total_rx: int = 256, C: int = 52):
    """300,000 Gaussians; 256 receivers in batches of U{1..64}, one
    transmitter per batch; CSI over 52 subcarriers; BF16 MLP."""
    rng = np.random.default_rng(seed)
    scene = draw_scene(rng, K)
    sizes = ragged_batches(rng, total_rx)
    tx = draw_points(rng, len(sizes))
    rx = draw_points(rng, total_rx)
    base = draw_base(rng, K, C)
    mlp = draw_mlp(rng, C)
    return dict(scene=scene, tx=tx, rx=rx, sizes=sizes, base=base, mlp=mlp, C=C, grid=Grid())


def serve_requests(rng: np.random.Generator, n_req: int, rate_hz: float, max_rx: int = 1024,
                   box=(10.0, 8.0, 3.0)):
    """Poisson arrivals; n = floor(exp(U(0, ln(max_rx+1)))) clipped to [1, max_rx]."""
    gaps = rng.exponential(1.0 / rate_hz, size=n_req)
    t = np.cumsum(gaps)
    reqs = []
    for i in range(n_req):
        n = int(math.floor(math.exp(rng.uniform(0.0, math.log(max_rx + 1)))))
        n = max(1, min(max_rx, n))
        reqs.append(dict(t=float(t[i]), tx=draw_points(rng, 1, box)[0], rx=draw_points(rng, n, box)))
    return reqs


def workload_coverage(seed: int = SEED_BASE + 4, K: int = 1_000_000, M: int = 16, side: int = 32,
                      with_radiance: bool = True):
    """1,000,000 Gaussians in a 40x30x4 m box, 16 transmitters, 1,024
    receivers at floor-grid cell centres 1 m high, 180x360 grid.  The
    [1024, K, 1, 2] radiance (8.2 GB at full size) is drawn here only when
    asked; `hashed_radiance_rows` / `hashed_radiance_torch` give a
    counter-based stand-in that can be produced on either side."""
    rng = np.random.default_rng(seed)
    box = (40.0, 30.0, 4.0)
    scene = draw_scene(rng, K, box)
    tx = draw_points(rng, M, box)
    a, b = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    rx = f32(np.stack([(a.reshape(-1) + 0.5) * 40.0 / side, (b.reshape(-1) + 0.5) * 30.0 / side,
                       np.ones(side * side)], axis=-1))
    rad = draw_radiance(rng, side * side, K, 1) if with_radiance else None
    return dict(scene=scene, tx=tx, rx=rx, radiance=rad,
                grid=Grid(H=180, W=360, theta0_deg=-90.0))


# ---------------------------------------------- counter-based radiance
# SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) applied to the counter
# i = j*K + k + 1: z = i * 0x9E3779B97F4A7C15, then the three xor-shift /
# multiply rounds.  The real part takes bits 40..63 and the imaginary part
# bits 16..39 of z, each mapped to m / 2^23 - 1 in [-1, 1): exact in
# float32, so the numpy and the torch versions agree bit for bit.
_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB


def _splitmix64_np(i: np.ndarray) -> np.ndarray:
    z = i.astype(np.uint64) * np.uint64(_SM_GAMMA)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
    return z ^ (z >> np.uint64(31))


def hashed_radiance_rows(js, K: int) -> np.ndarray:
    """Rows js of the counter-based radiance, [len(js), K, 1, 2] float32."""
    js = np.asarray(js, np.uint64)
    out = np.empty((js.shape[0], K, 1, 2), np.float32)
    k = np.arange(K, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for r, j in enumerate(js):
            z = _splitmix64_np(j * np.uint64(K) + k + np.uint64(1))
            re = ((z >> np.uint64(40)) & np.uint64(0xFFFFFF)).astype(np.float64) / 8388608.0 - 1.0
            im = ((z >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) / 8388608.0 - 1.0
            out[r, :, 0, 0] = re
            out[r, :, 0, 1] = im
    return out


def _i64(c: int) -> int:
    """The int64 with the bit pattern of the 64-bit constant c."""
    return c - (1 << 64) if c >= (1 << 63) else c


def hashed_radiance_torch(torch, N: int, K: int, device, rows_per_pass: int = 32):
    """The same counter-based radiance for rows 0..N-1, [N, K, 1, 2] float32,
    built on `device` with int64 arithmetic (wrapping products; logical
    right shifts by masking)."""
    out = torch.empty((N, K, 1, 2), dtype=torch.float32, device=device)
    k = torch.arange(K, dtype=torch.int64, device=device)

    def srl(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    for j0 in range(0, N, rows_per_pass):
        j1 = min(N, j0 + rows_per_pass)
        j = torch.arange(j0, j1, dtype=torch.int64, device=device)[:, None]
        z = (j * K + k[None, :] + 1) * _i64(_SM_GAMMA)
        z = (z ^ srl(z, 30)) * _i64(_SM_M1)
        z = (z ^ srl(z, 27)) * _i64(_SM_M2)
        z = z ^ srl(z, 31)
        re = (srl(z, 40) & 0xFFFFFF).to(torch.float64) / 8388608.0 - 1.0
        im = (srl(z, 16) & 0xFFFFFF).to(torch.float64) / 8388608.0 - 1.0
        out[j0:j1, :, 0, 0] = re.to(torch.float32)
        out[j0:j1, :, 0, 1] = im.to(torch.float32)
    return out


# --------------------------- global FiLM over FLE components (App. E.4 sizes)
FILM_BANDS = 6      # Fourier bands per spatial dimension
FILM_EMBED = 16     # component embedding width d_c
FILM_HIDDEN = 64    # hidden width d of the 3-layer global MLP


def film_frequencies(F: int = FILM_BANDS) -> np.ndarray:
    """The receiver encoding's frequency vectors at their initial values:
    2^f along each axis, f = 0 .. F-1 (3F vectors, x bands first)."""
    w = np.zeros((3 * F, 3), np.float64)
    for d in range(3):
        for f in range(F):
            w[d * F + f, d] = 2.0 ** f
    return f32(w)


def draw_film(rng: np.random.Generator, lmax: int, F: int = FILM_BANDS, dc: int = FILM_EMBED,
              D: int = FILM_HIDDEN, out_scale: float = 0.3) -> dict:
    """Parameters of the global FiLM MLP over L = (lmax+1)^2 components:
    frequencies at their initial spacing, random embeddings and weights.
    The final layer is drawn non-zero (a trained state, not the identity
    of the zero initialisation)."""
    L = (lmax + 1) ** 2
    nw = 3 * F
    din = 2 * nw + 2 + dc
    return {
        "omega": film_frequencies(F),
        "embed": f32(0.5 * rng.normal(size=(L, dc))),
        "w1": f32(rng.normal(size=(D, din)) * np.sqrt(2.0 / din)),
        "b1": f32(0.1 * rng.normal(size=D)),
        "w2": f32(rng.normal(size=(D, D)) * np.sqrt(2.0 / D)),
        "b2": f32(0.1 * rng.normal(size=D)),
        "w3": f32(rng.normal(size=(4, D)) * out_scale / np.sqrt(D)),
        "b3": f32(0.1 * out_scale * rng.normal(size=4)),
    }


def draw_fle_base(rng: np.random.Generator, K: int, lmax: int) -> np.ndarray:
    """Base FLE coefficients [K, 2, L], decaying with the degree l."""
    L = (lmax + 1) ** 2
    l_of = np.floor(np.sqrt(np.arange(L)))
    return f32(rng.normal(size=(K, 2, L)) / (1.0 + l_of)[None, None, :])
