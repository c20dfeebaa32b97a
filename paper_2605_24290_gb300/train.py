"""Stage II training step (Sec. 3.1; App. E.3-E.5) on top of the
differentiable render: geometry frozen, the base radiance phi_base and the
conditioning MLP trained with Adam against an L1 reconstruction loss on the
rendered amplitude spectra |R| = sqrt(Re^2 + Im^2 + 1e-8) (App. E.2) or on
RSSI.  The loss's SSIM and FFT terms and Stage I geometry learning are not
included.

A training step runs in the library's kernels from end to end: the
transmitter-side state is prepared once, the render writes the spectra (or
RSSI), one pass of rxgs_l1_loss forms the loss and its cotangent, and the
backward writes the parameter gradients; only the two Adam updates (small
tensors) are torch operations.  `loss()` is the same loss through the
differentiable render (autograd.py), for checking the step's gradients.
"""
from __future__ import annotations

import torch

from . import autograd, rxgs


class Stage2Trainer:
    """Holds the trainable phi_base [K,C,2] and MLP parameters of one scene.

    `target` of a step is either amplitude spectra [M,N,H,W,C] (kind
    OUT_SPECTRA) or RSSI [M,N] (kind OUT_RSSI)."""

    def __init__(self, rctx: "rxgs.Context", scene: int, opacity: torch.Tensor,
                 base: torch.Tensor, mlp: torch.Tensor, lr_base: float = 5e-3,
                 lr_mlp: float = 1e-3):
        self.rctx, self.scene = rctx, scene
        self.opacity = opacity.detach().contiguous()          # geometry frozen
        self.base = torch.nn.Parameter(base.detach().clone().contiguous())
        self.mlp = torch.nn.Parameter(mlp.detach().clone().contiguous())
        # separate optimisers for the radiance coefficients and the
        # conditioning modules (App. E.5)
        self.opt_base = torch.optim.Adam([self.base], lr=lr_base)
        self.opt_mlp = torch.optim.Adam([self.mlp], lr=lr_mlp)

    def loss(self, tx, rx, target, kind=rxgs.OUT_SPECTRA):
        N = rx.shape[0]
        spec, rssi, _ = autograd.render(self.rctx, self.scene, tx, rx, N, self.opacity,
                                        base=self.base, mlp=self.mlp, kind=kind)
        if kind == rxgs.OUT_SPECTRA:
            amp = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
            return (amp - target).abs().mean()
        if kind == rxgs.OUT_RSSI:
            return (rssi - target).abs().mean()
        raise ValueError("kind must be OUT_SPECTRA or OUT_RSSI")

    def _buffers(self, M, N, kind):
        key = (M, N, kind)
        if getattr(self, "_bkey", None) != key:
            dev, c = self.base.device, self.rctx
            C = self.base.shape[1]
            spectra = kind == rxgs.OUT_SPECTRA
            self._buf = dict(
                out=torch.empty((M, N, c.H, c.W, C, 2) if spectra else (M, N), device=dev),
                csi=None if spectra else torch.empty((M, N, C, 2), device=dev),
                grad=torch.empty((M, N, c.H, c.W, C, 2) if spectra else (M, N), device=dev),
                loss=torch.empty(1, device=dev),
                d_op=torch.empty_like(self.opacity))
            self._bkey = key
        return self._buf

    def step(self, tx, rx, target, kind=rxgs.OUT_SPECTRA) -> torch.Tensor:
        """One iteration: render, L1 loss and its cotangent (one kernel pass),
        backward, Adam.  Returns the loss (a device scalar, before the
        update)."""
        if kind not in (rxgs.OUT_SPECTRA, rxgs.OUT_RSSI):
            raise ValueError("kind must be OUT_SPECTRA or OUT_RSSI")
        c = self.rctx
        M, N = tx.shape[0], rx.shape[0]
        b = self._buffers(M, N, kind)
        c.update_scene(self.scene, opacity=self.opacity, base=self.base.detach(),
                       mlp=self.mlp.detach())
        d_base = torch.zeros_like(self.base)
        d_mlp = torch.zeros_like(self.mlp)
        views = c.prepare(self.scene, tx)
        try:
            if kind == rxgs.OUT_SPECTRA:
                c.render_views(views, rx, N, kind, spectra=b["out"])
                c.l1_loss(kind, b["out"], target.contiguous(), b["loss"], b["grad"])
                c.render_backward(views, rx, N, kind, grad_spectra=b["grad"],
                                  grad_opacity=b["d_op"].zero_(), grad_base=d_base, grad_mlp=d_mlp)
            else:
                c.render_views(views, rx, N, kind | rxgs.OUT_CSI, rssi=b["out"], csi=b["csi"])
                c.l1_loss(kind, b["out"], target.contiguous(), b["loss"], b["grad"])
                c.render_backward(views, rx, N, kind, grad_rssi=b["grad"], fwd_csi=b["csi"],
                                  grad_opacity=b["d_op"].zero_(), grad_base=d_base, grad_mlp=d_mlp)
        finally:
            c.release_views(views)
        self.base.grad = d_base
        self.mlp.grad = d_mlp
        self.opt_base.step()
        self.opt_mlp.step()
        return b["loss"][0].clone()


class FleStage2Trainer:
    """Stage II over the FLE representation (App. E.4): the base FLE
    coefficients [K,2,L] and the global FiLM branch trained with separate
    Adam optimisers; the coefficients of degree l > 0 take the learning rate
    lr_base * rest_ratio (the paper's "rest" ratio, 0.16-0.8; Adam is
    invariant to a gradient scale, so the degree-0 and higher-degree
    coefficients are separate tensors).  Geometry frozen; loss as
    Stage2Trainer."""

    def __init__(self, rctx: "rxgs.Context", scene: int, opacity: torch.Tensor,
                 base: torch.Tensor, film: torch.Tensor, film_dims, lmax: int,
                 lr_base: float = 5e-3, rest_ratio: float = 0.2, lr_film: float = 1e-3):
        self.rctx, self.scene, self.lmax = rctx, scene, int(lmax)
        self.dims = tuple(int(x) for x in film_dims)
        self.opacity = opacity.detach().contiguous()
        b = base.detach()
        self.base_dc = torch.nn.Parameter(b[:, :, :1].clone().contiguous())
        self.base_rest = torch.nn.Parameter(b[:, :, 1:].clone().contiguous())
        self.film = torch.nn.Parameter(film.detach().clone().contiguous())
        groups = [{"params": [self.base_dc], "lr": lr_base}]
        if self.base_rest.shape[2]:
            groups.append({"params": [self.base_rest], "lr": lr_base * rest_ratio})
        self.opt_base = torch.optim.Adam(groups)
        self.opt_film = torch.optim.Adam([self.film], lr=lr_film)

    def base(self) -> torch.Tensor:
        return torch.cat([self.base_dc, self.base_rest], dim=2).contiguous()

    def loss(self, tx, rx, target, kind=rxgs.OUT_SPECTRA):
        N = rx.shape[0]
        spec, rssi, _ = autograd.render_fle_film(self.rctx, self.scene, tx, rx, N, self.opacity,
                                                 self.base(), self.film, self.dims, self.lmax,
                                                 kind=kind)
        if kind == rxgs.OUT_SPECTRA:
            amp = torch.sqrt(spec[..., 0] ** 2 + spec[..., 1] ** 2 + 1e-8)
            return (amp - target).abs().mean()
        if kind == rxgs.OUT_RSSI:
            return (rssi - target).abs().mean()
        raise ValueError("kind must be OUT_SPECTRA or OUT_RSSI")

    def step(self, tx, rx, target, kind=rxgs.OUT_SPECTRA) -> torch.Tensor:
        """One iteration through the library's kernels (as Stage2Trainer.step):
        render, rxgs_l1_loss, backward to the base coefficients and the FiLM
        parameters, then the two Adam updates.  Returns the loss."""
        if kind not in (rxgs.OUT_SPECTRA, rxgs.OUT_RSSI):
            raise ValueError("kind must be OUT_SPECTRA or OUT_RSSI")
        c = self.rctx
        M, N = tx.shape[0], rx.shape[0]
        dev = self.film.device
        spectra = kind == rxgs.OUT_SPECTRA
        out = torch.empty((M, N, c.H, c.W, 1, 2) if spectra else (M, N), device=dev)
        csi = None if spectra else torch.empty((M, N, 1, 2), device=dev)
        grad = torch.empty_like(out)
        loss = torch.empty(1, device=dev)
        base = self.base().detach()
        film = self.film.detach().contiguous()
        d_base = torch.zeros_like(base)
        d_film = torch.zeros_like(film)
        d_op = torch.zeros_like(self.opacity)
        fle = dict(fle_lmax=self.lmax, fle_base=base, film=film, film_dims=self.dims)
        c.update_scene(self.scene, opacity=self.opacity)
        views = c.prepare(self.scene, tx)
        try:
            if spectra:
                c.render_views(views, rx, N, kind, spectra=out, **fle)
                c.l1_loss(kind, out, target.contiguous(), loss, grad)
                c.render_backward(views, rx, N, kind, grad_spectra=grad, grad_opacity=d_op,
                                  grad_fle_base=d_base, grad_film=d_film, **fle)
            else:
                c.render_views(views, rx, N, kind | rxgs.OUT_CSI, rssi=out, csi=csi, **fle)
                c.l1_loss(kind, out, target.contiguous(), loss, grad)
                c.render_backward(views, rx, N, kind, grad_rssi=grad, fwd_csi=csi,
                                  grad_opacity=d_op, grad_fle_base=d_base, grad_film=d_film, **fle)
        finally:
            c.release_views(views)
        self.base_dc.grad = d_base[:, :, :1].contiguous()
        self.base_rest.grad = d_base[:, :, 1:].contiguous()
        self.film.grad = d_film
        self.opt_base.step()
        self.opt_film.step()
        return loss[0].clone()
