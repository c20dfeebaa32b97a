"""Helpers shared by the GPU tests: device copies of synthetic inputs and the
normalised error used for every floating-point comparison.

Tolerance.  For a composited value x (one real or imaginary part of one
pixel, receiver and channel), err = |x_gpu - x_ref| / (A_ref + 1e-30) where
A_ref = sum_k T_k w_k |s_kj| is the sum of the absolute contributions the
oracle composited for that element (summed over pixels for RSSI / CSI).
float32 accumulation of n terms bounds err by about n * 2^-24 plus the
float32 error of each weight (a few ulp from exp and the conic), so 1e-4
leaves a wide margin for n up to several hundred.
"""
import numpy as np

TOL = 1e-4


def dev(a, torch, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def upload(ctx, scene, torch, base=None, mlp_flat=None, C=1, bf16=False):
    return ctx.upload_scene(dev(scene.means, torch), dev(scene.log_scales, torch),
                            dev(scene.quats, torch), dev(scene.opacity, torch),
                            None if base is None else dev(base, torch),
                            None if mlp_flat is None else dev(mlp_flat, torch), C=C, bf16=bf16)


def norm_err(x_gpu, x_ref, a_ref):
    """max over elements of |x_gpu - x_ref| / A_ref (A_ref broadcast over the
    trailing real/imag axis)."""
    x_gpu = np.asarray(x_gpu, np.float64)
    x_ref = np.asarray(x_ref, np.float64)
    a = np.asarray(a_ref, np.float64)[..., None]
    d = np.abs(x_gpu - x_ref)
    zero = a[..., 0] == 0
    if zero.any():
        assert np.all(d[zero] == 0.0), "non-zero output where nothing was composited"
    return float((d / (a + 1e-30)).max()) if d.size else 0.0


def fle_abs_radiance(oracle, coeffs, means, centre, lmax):
    """The absolute chain of the FLE radiance, sum_l (|Re Y_l| + |Im Y_l|)
    (|Re c_l| + |Im c_l|) as a real radiance [N,K,1,2]: the tensor-core
    contraction rounds each real product of Y and c (split bf16 terms), so its
    error scales with this sum, not with |sum_l Y_l c_l|.  Rendered with
    oracle.render_view, its "absacc" is the error scale of the spectra."""
    c = np.asarray(coeffs, np.float64)
    Y = oracle.fle_basis(means, centre, lmax)                       # [K, L]
    ya = np.abs(Y.real) + np.abs(Y.imag)
    ca = np.abs(c[:, :, 0, :]) + np.abs(c[:, :, 1, :])              # [N, K, L]
    chain = (ca * ya[None]).sum(axis=-1)
    out = np.zeros(c.shape[:2] + (1, 2))
    out[..., 0, 0] = chain
    return out
