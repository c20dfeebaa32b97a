"""Stage II training step (Sec. 3.1; App. E.3-E.5) on top of the
differentiable render: geometry frozen, the base radiance phi_base and the
conditioning MLP trained with Adam against an L1 reconstruction loss on the
rendered amplitude spectra |R| = sqrt(Re^2 + Im^2 + 1e-8) (App. E.2) or on
RSSI.  The loss's SSIM and FFT terms and Stage I geometry learning are not
included.

The render and its backward run in the library's kernels (autograd.py);
the loss and the optimiser update are ordinary torch operations on the
rendered outputs and the parameters.
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

    def step(self, tx, rx, target, kind=rxgs.OUT_SPECTRA) -> torch.Tensor:
        """One iteration: render, L1 loss, backward, Adam.  Returns the loss
        (a device scalar, before the update)."""
        self.opt_base.zero_grad(set_to_none=True)
        self.opt_mlp.zero_grad(set_to_none=True)
        loss = self.loss(tx, rx, target, kind)
        loss.backward()
        self.opt_base.step()
        self.opt_mlp.step()
        return loss.detach()


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
        self.opt_base.zero_grad(set_to_none=True)
        self.opt_film.zero_grad(set_to_none=True)
        loss = self.loss(tx, rx, target, kind)
        loss.backward()
        self.opt_base.step()
        self.opt_film.step()
        return loss.detach()
