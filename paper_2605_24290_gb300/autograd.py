"""torch.autograd.Function over rxgs_render_views / rxgs_render_backward.

Geometry is frozen (App. D; Sec. 3.1 Stage II): gradients flow to the
opacity, to the radiance (explicit) or to phi_base and the conditioning MLP.
The forward writes the new opacity / phi_base / MLP parameters into the
library's scene, prepares the transmitter-side state, renders and releases
it; the backward prepares it again (the per-tile lists are recomputed, not
stored) and runs the backward kernels.  Everything runs on the current torch
stream.
"""
from __future__ import annotations

import torch

from . import rxgs


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(fctx, opacity, base, mlp, radiance, rctx, scene, tx, rx, N, kind):
        rctx.update_scene(scene, opacity=opacity.detach().contiguous(),
                          base=None if base is None else base.detach().contiguous(),
                          mlp=None if mlp is None else mlp.detach().contiguous())
        M = tx.shape[0]
        dev = tx.device
        C = (base.shape[1] if base is not None else radiance.shape[2])
        spec = torch.empty((M, N, rctx.H, rctx.W, C, 2), device=dev) \
            if kind & rxgs.OUT_SPECTRA else None
        rssi = torch.empty((M, N), device=dev) if kind & rxgs.OUT_RSSI else None
        want_csi = bool(kind & (rxgs.OUT_CSI | rxgs.OUT_RSSI))
        csi = torch.empty((M, N, C, 2), device=dev) if want_csi else None
        kk = kind | (rxgs.OUT_CSI if want_csi else 0)
        rad = None if radiance is None else radiance.detach().contiguous()
        views = rctx.prepare(scene, tx)
        try:
            rctx.render_views(views, rx, N, kk, radiance=rad, spectra=spec, rssi=rssi, csi=csi)
        finally:
            rctx.release_views(views)
        fctx.rctx, fctx.scene, fctx.N, fctx.kind, fctx.C = rctx, scene, N, kind, C
        fctx.has = (base is not None, mlp is not None, radiance is not None)
        fctx.save_for_backward(tx, rx, rad, csi, opacity)
        outs = (spec, rssi, csi if kind & rxgs.OUT_CSI else None)
        return tuple(o if o is not None else torch.empty(0, device=dev) for o in outs)

    @staticmethod
    def backward(fctx, g_spec, g_rssi, g_csi):
        tx, rx, rad, csi, opacity = fctx.saved_tensors
        rctx, scene, N, kind = fctx.rctx, fctx.scene, fctx.N, fctx.kind
        has_base, has_mlp, has_rad = fctx.has
        gs = g_spec.contiguous() if (kind & rxgs.OUT_SPECTRA and g_spec is not None
                                     and g_spec.numel()) else None
        gr = g_rssi.contiguous() if (kind & rxgs.OUT_RSSI and g_rssi is not None
                                     and g_rssi.numel()) else None
        gc = g_csi.contiguous() if (kind & rxgs.OUT_CSI and g_csi is not None
                                    and g_csi.numel()) else None
        d_op = torch.zeros_like(opacity)
        d_rad = torch.zeros_like(rad) if has_rad else None
        d_base = d_mlp = None
        if not has_rad:
            K = opacity.shape[0]
            C = fctx.C
            d_base = torch.zeros((K, C, 2), device=opacity.device)
            d_mlp = torch.zeros((rctx.mlp_numel(C),), device=opacity.device)
        if gs is None and gr is None and gc is None:
            return (d_op, d_base, d_mlp, d_rad) + (None,) * 6
        views = rctx.prepare(scene, tx)
        try:
            rctx.render_backward(views, rx, N, kind, radiance=rad, grad_spectra=gs, grad_csi=gc,
                                 grad_rssi=gr, fwd_csi=csi, grad_radiance=d_rad, grad_opacity=d_op,
                                 grad_base=d_base, grad_mlp=d_mlp)
        finally:
            rctx.release_views(views)
        return (d_op, d_base if has_base else None, d_mlp if has_mlp else None,
                d_rad) + (None,) * 6


def render(rctx: "rxgs.Context", scene: int, tx: torch.Tensor, rx: torch.Tensor, N: int,
           opacity: torch.Tensor, base=None, mlp=None, radiance=None,
           kind: int = rxgs.OUT_SPECTRA):
    """Differentiable render.  Returns (spectra, rssi, csi); outputs that
    `kind` does not ask for are empty tensors."""
    return _Render.apply(opacity, base, mlp, radiance, rctx, scene, tx, rx, N, kind)


class _RenderFleFilm(torch.autograd.Function):
    """The same over the FLE radiance whose base coefficients are conditioned
    by the global FiLM branch (Eq. film, film_apply): gradients flow to the
    opacity, the base coefficients [K,2,L] and the packed FiLM parameters."""

    @staticmethod
    def forward(fctx, opacity, base, film, rctx, scene, tx, rx, N, kind, lmax, dims):
        rctx.update_scene(scene, opacity=opacity.detach().contiguous())
        M = tx.shape[0]
        dev = tx.device
        spec = torch.empty((M, N, rctx.H, rctx.W, 1, 2), device=dev) \
            if kind & rxgs.OUT_SPECTRA else None
        rssi = torch.empty((M, N), device=dev) if kind & rxgs.OUT_RSSI else None
        want_csi = bool(kind & (rxgs.OUT_CSI | rxgs.OUT_RSSI))
        csi = torch.empty((M, N, 1, 2), device=dev) if want_csi else None
        kk = kind | (rxgs.OUT_CSI if want_csi else 0)
        b, f = base.detach().contiguous(), film.detach().contiguous()
        views = rctx.prepare(scene, tx)
        try:
            rctx.render_views(views, rx, N, kk, spectra=spec, rssi=rssi, csi=csi, fle_lmax=lmax,
                              fle_base=b, film=f, film_dims=dims)
        finally:
            rctx.release_views(views)
        fctx.rctx, fctx.scene, fctx.N, fctx.kind = rctx, scene, N, kind
        fctx.lmax, fctx.dims = lmax, dims
        fctx.save_for_backward(tx, rx, b, f, csi, opacity)
        outs = (spec, rssi, csi if kind & rxgs.OUT_CSI else None)
        return tuple(o if o is not None else torch.empty(0, device=dev) for o in outs)

    @staticmethod
    def backward(fctx, g_spec, g_rssi, g_csi):
        tx, rx, b, f, csi, opacity = fctx.saved_tensors
        rctx, scene, N, kind = fctx.rctx, fctx.scene, fctx.N, fctx.kind
        gs = g_spec.contiguous() if (kind & rxgs.OUT_SPECTRA and g_spec is not None
                                     and g_spec.numel()) else None
        gr = g_rssi.contiguous() if (kind & rxgs.OUT_RSSI and g_rssi is not None
                                     and g_rssi.numel()) else None
        gc = g_csi.contiguous() if (kind & rxgs.OUT_CSI and g_csi is not None
                                    and g_csi.numel()) else None
        d_op = torch.zeros_like(opacity)
        d_base = torch.zeros_like(b)
        d_film = torch.zeros_like(f)
        if gs is None and gr is None and gc is None:
            return (d_op, d_base, d_film) + (None,) * 8
        views = rctx.prepare(scene, tx)
        try:
            rctx.render_backward(views, rx, N, kind, grad_spectra=gs, grad_csi=gc, grad_rssi=gr,
                                 fwd_csi=csi, grad_opacity=d_op, fle_lmax=fctx.lmax, fle_base=b,
                                 film=f, film_dims=fctx.dims, grad_fle_base=d_base,
                                 grad_film=d_film)
        finally:
            rctx.release_views(views)
        return (d_op, d_base, d_film) + (None,) * 8


def render_fle_film(rctx: "rxgs.Context", scene: int, tx: torch.Tensor, rx: torch.Tensor,
                    N: int, opacity: torch.Tensor, base: torch.Tensor, film: torch.Tensor,
                    film_dims, lmax: int, kind: int = rxgs.OUT_SPECTRA):
    """Differentiable render of the FiLM-conditioned FLE radiance (C = 1).
    `film` is packed (rxgs.pack_film); film_dims = (nfreq, embed, hidden).
    Returns (spectra, rssi, csi) as `render` does."""
    return _RenderFleFilm.apply(opacity, base, film, rctx, scene, tx, rx, N, kind, int(lmax),
                                tuple(int(x) for x in film_dims))
