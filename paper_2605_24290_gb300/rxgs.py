"""Python binding of librxgs (include/rxgs.h): argument marshalling only.

Every step of the renderer runs in the CUDA library; this module turns torch
tensors into device pointers and the current torch stream into the call's
stream.  There is no CPU path: without the compiled library (or without a
GPU) every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librxgs.so")

OUT_SPECTRA, OUT_RSSI, OUT_CSI = 1, 2, 4
STATUS = {0: "OK", 1: "E_INVALID", 2: "E_OOM", 3: "E_CUDA", 4: "E_ADMISSION", 5: "E_NOT_READY",
          6: "E_TIMEOUT", 7: "E_DEVICE", 8: "E_CANCELLED"}
OK, E_INVALID, E_OOM, E_CUDA, E_ADMISSION, E_NOT_READY, E_TIMEOUT, E_DEVICE, E_CANCELLED = range(9)


class RxgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rxgs {STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("theta0_deg", ctypes.c_float),
                ("step_deg", ctypes.c_float), ("tile_h", ctypes.c_int), ("tile_w", ctypes.c_int),
                ("eps_T", ctypes.c_float), ("q_max", ctypes.c_float), ("r_near", ctypes.c_float),
                ("cols_per_cta", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("mem_budget", ctypes.c_size_t)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("C", ctypes.c_int), ("means", ctypes.c_void_p),
                ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("base_radiance", ctypes.c_void_p),
                ("mlp_params", ctypes.c_void_p), ("mlp_hidden", ctypes.c_int),
                ("mlp_bf16", ctypes.c_int), ("on_device", ctypes.c_int)]


class RenderDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("radiance", ctypes.c_void_p), ("reduce_path", ctypes.c_int),
                ("fle_coeffs", ctypes.c_void_p), ("fle_lmax", ctypes.c_int),
                ("fle_base", ctypes.c_void_p), ("film", ctypes.c_void_p),
                ("film_nfreq", ctypes.c_int), ("film_embed", ctypes.c_int),
                ("film_hidden", ctypes.c_int), ("film_local", ctypes.c_int)]


class Outputs(ctypes.Structure):
    _fields_ = [("spectra", ctypes.c_void_p), ("rssi", ctypes.c_void_p), ("csi", ctypes.c_void_p),
                ("ncontrib", ctypes.c_void_p), ("tfinal", ctypes.c_void_p)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("max_batch_receivers", ctypes.c_int),
                ("max_batch_views", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("slots", ctypes.c_int)]


class Cotangents(ctypes.Structure):
    _fields_ = [("grad_spectra", ctypes.c_void_p), ("grad_csi", ctypes.c_void_p),
                ("grad_rssi", ctypes.c_void_p), ("fwd_csi", ctypes.c_void_p)]


class Grads(ctypes.Structure):
    _fields_ = [("grad_radiance", ctypes.c_void_p), ("grad_opacity", ctypes.c_void_p),
                ("grad_base", ctypes.c_void_p), ("grad_mlp", ctypes.c_void_p),
                ("grad_fle", ctypes.c_void_p), ("grad_fle_base", ctypes.c_void_p),
                ("grad_film", ctypes.c_void_p)]


P = ctypes.c_void_p
U64 = ctypes.c_uint64
I = ctypes.c_int
# name -> (restype, argtypes); the exported symbols of include/rxgs.h
SIGNATURES = {
    "rxgs_default_options": (None, [P]),
    "rxgs_create": (I, [P, I, P]),
    "rxgs_destroy": (I, [P]),
    "rxgs_last_error": (ctypes.c_char_p, [P]),
    "rxgs_upload_scene": (I, [P, P, P]),
    "rxgs_release_scene": (I, [P, U64]),
    "rxgs_update_scene": (I, [P, U64, P, P, P, P]),
    "rxgs_build_occupancy": (I, [P, U64, I, P]),
    "rxgs_prepare": (I, [P, U64, P, I, P, P]),
    "rxgs_release_views": (I, [P, U64, P]),
    "rxgs_render_views": (I, [P, U64, P, I, P, P, P]),
    "rxgs_render": (I, [P, U64, P, I, P, I, P, P, P]),
    "rxgs_render_backward": (I, [P, U64, P, I, P, P, P, P]),
    "rxgs_views_info": (I, [P, U64, P]),
    "rxgs_views_export": (I, [P, U64, P, P, P, P, P, P]),
    "rxgs_profile": (I, [P, I]),
    "rxgs_profile_read": (I, [P, ctypes.c_char_p, ctypes.c_size_t, I]),
    "rxgs_render_csi_noalloc": (I, [P, U64, P, I, P, P, P]),
    "rxgs_render_batched": (I, [P, U64, P, I, P, P, P, P, P]),
    "rxgs_autotune": (I, [P, U64, P, I, P, I, P, I, ctypes.c_char_p, ctypes.c_size_t]),
    "rxgs_serve_default_options": (None, [P]),
    "rxgs_serve_start": (I, [P, U64, P]),
    "rxgs_serve_submit": (I, [P, P, P, I, P]),
    "rxgs_serve_poll": (I, [P, U64, P, I]),
    "rxgs_serve_cancel": (I, [P, U64]),
    "rxgs_serve_stats": (I, [P, ctypes.c_char_p, ctypes.c_size_t]),
    "rxgs_serve_reset_stats": (I, [P]),
    "rxgs_serve_inject_fault": (I, [P, I]),
    "rxgs_serve_stop": (I, [P]),
    "rxgs_sync": (I, [P, P]),
    "rxgs_l1_loss": (I, [P, I, P, P, ctypes.c_size_t, P, P, P]),
    "rxgs_film_param_count": (ctypes.c_int64, [I, I, I, I]),
    "rxgs_film_eval": (I, [P, P, I, I, I, I, P, I, P, P]),
}

# Packed order of the global FiLM parameters (rxgs_film_eval).
FILM_FIELDS = ("omega", "embed", "w1", "b1", "w2", "b2", "w3", "b3")


def film_shapes(nfreq: int, embed: int, hidden: int, lmax: int) -> dict:
    L = (lmax + 1) ** 2
    din = 2 * nfreq + 2 + embed
    return {"omega": (nfreq, 3), "embed": (L, embed), "w1": (hidden, din), "b1": (hidden,),
            "w2": (hidden, hidden), "b2": (hidden,), "w3": (4, hidden), "b3": (4,)}


def film_param_count(nfreq: int, embed: int, hidden: int, lmax: int) -> int:
    """Length of the packed FiLM parameters (rxgs_film_param_count)."""
    n = 0
    for shp in film_shapes(nfreq, embed, hidden, lmax).values():
        k = 1
        for d in shp:
            k *= d
        n += k
    return n


def check_film_length(numel: int, nfreq: int, embed: int, hidden: int, lmax: int) -> None:
    """Raises ValueError when sizes the library accepts (nfreq 1..32, embed
    0..64, hidden 1..256, lmax 0..9) do not match the packed length; sizes
    out of range are left to the library, which refuses them."""
    if not (1 <= nfreq <= 32 and 0 <= embed <= 64 and 1 <= hidden <= 256 and 0 <= lmax <= 9):
        return
    need = film_param_count(nfreq, embed, hidden, lmax)
    if int(numel) != need:
        raise ValueError(f"film holds {int(numel)} floats; sizes ({nfreq}, {embed}, {hidden}) "
                         f"and lmax {lmax} need {need}")


def film_sizes(params: dict):
    """(nfreq, embed, hidden) of a FiLM parameter dict."""
    return (int(params["omega"].shape[0]), int(params["embed"].shape[1]),
            int(params["w1"].shape[0]))


def pack_film(params: dict):
    """Concatenates the FiLM parameters (numpy arrays or tensors) in the
    packed order, flattened."""
    parts = [params[k].reshape(-1) for k in FILM_FIELDS]
    if hasattr(parts[0], "detach"):
        import torch
        return torch.cat(parts)
    import numpy as np
    return np.concatenate(parts).astype(np.float32)


def unpack_film(flat, nfreq: int, embed: int, hidden: int, lmax: int) -> dict:
    """The inverse of pack_film (views into `flat`)."""
    out, o = {}, 0
    for k, shp in film_shapes(nfreq, embed, hidden, lmax).items():
        n = 1
        for d in shp:
            n *= d
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    return out

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Loads librxgs.so (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                from . import build as _b
                _b.build()
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t):
    import torch
    if t is not None and t.dtype != torch.float32:
        raise TypeError("expected float32")
    return _ptr(t)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One rxgs context on one CUDA device (argument marshalling only)."""

    def __init__(self, H=90, W=360, theta0_deg=0.0, step_deg=1.0, tile_h=16, tile_w=16,
                 eps_T=1e-4, q_max=9.0, r_near=0.05, cols_per_cta=0, deterministic=0,
                 mem_budget=0, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("rxgs needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        o = Options(H, W, theta0_deg, step_deg, tile_h, tile_w, eps_T, q_max, r_near, cols_per_cta,
                    deterministic, mem_budget)
        self.opts = o
        h = ctypes.c_void_p()
        st = self.lib.rxgs_create(ctypes.byref(o), self.device, ctypes.byref(h))
        if st != OK:
            raise RxgsError(st, "rxgs_create failed (bad options or CUDA error)")
        self.h = h
        self.H, self.W = H, W

    def close(self):
        if getattr(self, "h", None):
            self.lib.rxgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise RxgsError(st, self.lib.rxgs_last_error(self.h).decode())

    # --------------------------------------------------------------- scene
    def upload_scene(self, means, log_scales, quats, opacity, base=None, mlp=None, C=1,
                     hidden=64, bf16=False):
        """Device tensors (float32).  Returns a scene handle."""
        d = SceneDesc(int(means.shape[0]), int(C), _f32(means), _f32(log_scales), _f32(quats),
                      _f32(opacity), _f32(base), _f32(mlp), int(hidden), int(bool(bf16)), 1)
        out = ctypes.c_uint64()
        import torch
        torch.cuda.synchronize()
        self._check(self.lib.rxgs_upload_scene(self.h, ctypes.byref(d), ctypes.byref(out)))
        return out.value

    def release_scene(self, scene):
        self._check(self.lib.rxgs_release_scene(self.h, U64(scene)))

    def update_scene(self, scene, opacity=None, base=None, mlp=None, stream=None):
        self._check(self.lib.rxgs_update_scene(self.h, U64(scene), _f32(opacity), _f32(base),
                                               _f32(mlp), _stream(stream)))

    def build_occupancy(self, scene, res=128, stream=None):
        """Occupancy grid for the local branch's occlusion inputs (res = 0
        removes it)."""
        self._check(self.lib.rxgs_build_occupancy(self.h, U64(scene), int(res), _stream(stream)))

    # --------------------------------------------------------------- views
    def prepare(self, scene, tx, stream=None):
        out = ctypes.c_uint64()
        self._check(self.lib.rxgs_prepare(self.h, U64(scene), _f32(tx), int(tx.shape[0]),
                                          ctypes.byref(out), _stream(stream)))
        return out.value

    def release_views(self, views, stream=None):
        self._check(self.lib.rxgs_release_views(self.h, U64(views), _stream(stream)))

    @staticmethod
    def _desc(kind, radiance, reduce_path, fle_coeffs, fle_lmax, fle_base, film, film_dims,
              film_local=False):
        nf, ne, nh = film_dims if film_dims is not None else (0, 0, 0)
        if film is not None and film_dims is not None:
            check_film_length(film.numel(), int(nf), int(ne), int(nh), int(fle_lmax))
        return RenderDesc(int(kind), _f32(radiance), int(reduce_path), _f32(fle_coeffs),
                          int(fle_lmax), _f32(fle_base), _f32(film), int(nf), int(ne), int(nh),
                          1 if film_local else 0)

    def film_eval(self, film, film_dims, lmax, rx, N, ab, stream=None):
        """ab[N, L, 4] = (a.re, a.im, b.re, b.im) of the global FiLM branch."""
        nf, ne, nh = film_dims
        check_film_length(film.numel(), int(nf), int(ne), int(nh), int(lmax))
        L = (int(lmax) + 1) ** 2
        if ab.numel() != int(N) * L * 4 or rx.numel() != int(N) * 3:
            raise ValueError("ab must hold [N, L, 4] and rx [N, 3] floats")
        self._check(self.lib.rxgs_film_eval(self.h, _f32(film), int(nf), int(ne), int(nh),
                                            int(lmax), _f32(rx), int(N), _f32(ab),
                                            _stream(stream)))

    def render_views(self, views, rx, N, kind, radiance=None, spectra=None, rssi=None, csi=None,
                     ncontrib=None, tfinal=None, reduce_path=0, fle_coeffs=None, fle_lmax=0,
                     fle_base=None, film=None, film_dims=None, film_local=False, stream=None):
        d = self._desc(kind, radiance, reduce_path, fle_coeffs, fle_lmax, fle_base, film, film_dims,
                       film_local)
        o = Outputs(_f32(spectra), _f32(rssi), _f32(csi), _ptr(ncontrib), _f32(tfinal))
        self._check(self.lib.rxgs_render_views(self.h, U64(views), _f32(rx), int(N),
                                               ctypes.byref(d), ctypes.byref(o), _stream(stream)))

    def render(self, scene, tx, rx, N, kind, radiance=None, spectra=None, rssi=None, csi=None,
               ncontrib=None, tfinal=None, reduce_path=0, fle_coeffs=None, fle_lmax=0,
               fle_base=None, film=None, film_dims=None, film_local=False, stream=None):
        d = self._desc(kind, radiance, reduce_path, fle_coeffs, fle_lmax, fle_base, film, film_dims,
                       film_local)
        o = Outputs(_f32(spectra), _f32(rssi), _f32(csi), _ptr(ncontrib), _f32(tfinal))
        self._check(self.lib.rxgs_render(self.h, U64(scene), _f32(tx), int(tx.shape[0]),
                                         _f32(rx), int(N), ctypes.byref(d), ctypes.byref(o),
                                         _stream(stream)))

    def render_backward(self, views, rx, N, kind, radiance=None, grad_spectra=None,
                        grad_csi=None, grad_rssi=None, fwd_csi=None,
                        grad_radiance=None, grad_opacity=None, grad_base=None, grad_mlp=None,
                        fle_coeffs=None, fle_lmax=0, grad_fle=None, fle_base=None, film=None,
                        film_dims=None, grad_fle_base=None, grad_film=None, film_local=False,
                        stream=None):
        d = self._desc(kind, radiance, 0, fle_coeffs, fle_lmax, fle_base, film, film_dims,
                       film_local)
        c = Cotangents(_f32(grad_spectra), _f32(grad_csi), _f32(grad_rssi), _f32(fwd_csi))
        g = Grads(_f32(grad_radiance), _f32(grad_opacity), _f32(grad_base), _f32(grad_mlp),
                  _f32(grad_fle), _f32(grad_fle_base), _f32(grad_film))
        self._check(self.lib.rxgs_render_backward(self.h, U64(views), _f32(rx), int(N),
                                                  ctypes.byref(d), ctypes.byref(c),
                                                  ctypes.byref(g), _stream(stream)))

    def views_info(self, views):
        n = ctypes.c_int64()
        self._check(self.lib.rxgs_views_info(self.h, U64(views), ctypes.byref(n)))
        return n.value

    def views_export(self, views, M, K, T, stream=None):
        """Copies the transmitter-side state into new tensors:
        (rec[M,K,8] f32, counts[M,K] i32, keys[I] i64, vals[I] i32, ranges[M,T,2] i32)."""
        import torch
        n = self.views_info(views)
        dev = torch.device("cuda", self.device)
        rec = torch.empty((M, K, 8), dtype=torch.float32, device=dev)
        counts = torch.empty((M, K), dtype=torch.int32, device=dev)
        keys = torch.empty((max(n, 1),), dtype=torch.int64, device=dev)
        vals = torch.empty((max(n, 1),), dtype=torch.int32, device=dev)
        ranges = torch.empty((M, T, 2), dtype=torch.int32, device=dev)
        self._check(self.lib.rxgs_views_export(self.h, U64(views), _ptr(rec), _ptr(counts),
                                               _ptr(keys), _ptr(vals), _ptr(ranges),
                                               _stream(stream)))
        return rec, counts, keys[:n], vals[:n], ranges

    def profile(self, enable=True):
        self._check(self.lib.rxgs_profile(self.h, 1 if enable else 0))

    def profile_read(self, reset=True):
        """Per-stage CUDA-event totals and the library's kernel launch count."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.lib.rxgs_profile_read(self.h, buf, len(buf), 1 if reset else 0))
        return json.loads(buf.value.decode())

    @staticmethod
    def mlp_numel(C, hidden=64):
        """Number of float32 parameters of the two conditioning MLPs."""
        return hidden * 3 + hidden + 4 * C * hidden + 4 * C + hidden * 6 + hidden + 4 * C * hidden + 4 * C

    def render_batched(self, scene, tx, rx, counts, kind, radiance=None, spectra=None, rssi=None,
                       csi=None, reduce_path=None, stream=None):
        """Ragged batches: tx[B,3], rx[R,3], counts = list of B receiver counts.
        reduce_path defaults to the visibility path for CSI/RSSI-only MLP renders."""
        cnt = (ctypes.c_int32 * len(counts))(*[int(c) for c in counts])
        if reduce_path is None:
            reduce_path = 1 if (radiance is None and not (kind & OUT_SPECTRA)) else 0
        d = RenderDesc(int(kind), _f32(radiance), int(reduce_path))
        o = Outputs(_f32(spectra), _f32(rssi), _f32(csi), None, None)
        self._check(self.lib.rxgs_render_batched(self.h, U64(scene), _f32(tx), int(tx.shape[0]),
                                                 _f32(rx), cnt, ctypes.byref(d), ctypes.byref(o),
                                                 _stream(stream)))

    def autotune(self, scene, tx, rx, N, kind, radiance=None, iters=3):
        """Times tile shapes x column blocks on this workload and keeps the
        fastest in the context; returns the timings."""
        import json
        d = RenderDesc(int(kind), _f32(radiance), 0)
        buf = ctypes.create_string_buffer(8192)
        self._check(self.lib.rxgs_autotune(self.h, U64(scene), _f32(tx), int(tx.shape[0]),
                                           _f32(rx), int(N), ctypes.byref(d), int(iters), buf,
                                           len(buf)))
        return json.loads(buf.value.decode())

    # ------------------------------------------------------------- serving
    def serve_start(self, scene, kind=OUT_RSSI, max_batch_receivers=4096, max_batch_views=64,
                    mem_budget=16 << 30, slots=2):
        o = ServeOptions(int(kind), int(max_batch_receivers), int(max_batch_views),
                         int(mem_budget), int(slots))
        self._check(self.lib.rxgs_serve_start(self.h, U64(scene), ctypes.byref(o)))

    def serve_submit(self, tx, rx):
        """tx: 3 floats, rx: [n,3] float32 numpy array (host).  Returns a ticket."""
        import numpy as np
        t = np.ascontiguousarray(tx, dtype=np.float32)
        r = np.ascontiguousarray(rx, dtype=np.float32).reshape(-1, 3)
        out = ctypes.c_uint64()
        self._check(self.lib.rxgs_serve_submit(self.h, t.ctypes.data_as(P), r.ctypes.data_as(P),
                                               int(r.shape[0]), ctypes.byref(out)))
        return out.value

    def serve_poll(self, ticket, n_out, timeout_us=-1):
        """Returns the result (numpy float32, n_out values) or raises RxgsError
        (E_NOT_READY / E_TIMEOUT keep the ticket)."""
        import numpy as np
        out = np.empty(int(n_out), np.float32)
        st = self.lib.rxgs_serve_poll(self.h, U64(ticket), out.ctypes.data_as(P), int(timeout_us))
        if st != OK:
            raise RxgsError(st, self.lib.rxgs_last_error(self.h).decode())
        return out

    def serve_cancel(self, ticket):
        self._check(self.lib.rxgs_serve_cancel(self.h, U64(ticket)))

    def serve_stats(self):
        import json
        buf = ctypes.create_string_buffer(1024)
        self._check(self.lib.rxgs_serve_stats(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def serve_reset_stats(self):
        self._check(self.lib.rxgs_serve_reset_stats(self.h))

    def serve_inject_fault(self, batches=1):
        self._check(self.lib.rxgs_serve_inject_fault(self.h, int(batches)))

    def serve_stop(self):
        self._check(self.lib.rxgs_serve_stop(self.h))

    def render_csi_noalloc(self, views, radiance, N, csi=None, rssi=None, stream=None):
        """CSI / RSSI of prepared views with no device allocation (the
        library's fixed scratch array holds the partial sums)."""
        self._check(self.lib.rxgs_render_csi_noalloc(self.h, U64(views), _f32(radiance), int(N),
                                                     _f32(csi), _f32(rssi), _stream(stream)))

    def l1_loss(self, kind, values, target, loss, grad, stream=None):
        """Stage II L1 term and its cotangent in one pass (device tensors):
        kind OUT_SPECTRA: values = spectra [..., 2], target = amplitudes [...];
        kind OUT_RSSI: values = RSSI, target the same shape.  Writes the mean
        absolute difference into loss[0] and its gradient into grad (the
        shape of values)."""
        n = int(target.numel())
        self._check(self.lib.rxgs_l1_loss(self.h, int(kind), _f32(values), _f32(target), n,
                                          _f32(loss), _f32(grad), _stream(stream)))

    def sync(self, stream=None):
        self._check(self.lib.rxgs_sync(self.h, _stream(stream)))
