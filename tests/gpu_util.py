"""Helpers for the GPU tests: run the CUDA path through the C ABI on torch
device memory and compare with the float64 oracle."""

import numpy as np

import oracle as o
import paper_2206_04681_gb300 as pkg


def gpu_filter(img, levels, K, m, sigma_r, T=2.0, precision="fp32", runs=1):
    """Filter a (C, H, W) float32 image on cuda:0; returns (outputs, a_k float64)."""
    import torch
    img = np.ascontiguousarray(img, dtype=np.float32)
    if img.ndim == 2:
        img = img[None]
    C, H, W = img.shape
    p = pkg.make_params(H, W, C, levels, K, m, sigma_r, T, precision)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        outs = []
        for _ in range(runs):
            y = torch.full_like(x, float("nan"))
            pkg.run_tensor(plan, x, y)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
    finally:
        pkg.fllf_plan_destroy(plan)
    a = np.array(o.coeffs_quadrature(m, sigma_r, T, K))  # the oracle's own a_k
    return (outs[0] if runs == 1 else outs), a


def psnr(x, ref):
    mse = float(np.mean((np.asarray(x, np.float64) - ref) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
