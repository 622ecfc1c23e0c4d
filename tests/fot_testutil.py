"""Comparison helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

# FP32 tolerance for potentials, normwise relative over finite entries (the bound the
# method's FP32 path is held to).
POT_RTOL = 1e-6


def solve_rtol(iters):
    """Normwise bound for potentials after `iters` full iterations in FP32.

    Every half-step rounds the stored potential once (<= 2^-24 |pot|) and rounds the
    potential/eps product it reads (<= 2^-24 |pot|/eps in the exponent, i.e. <= 2^-24 |pot|
    after the update); the iteration neither amplifies nor (at small eps) noticeably damps
    these, so they add like a random walk over the 2 * iters half-steps.  Bound: a safety
    factor 4 on sqrt(2 iters) * 2 * 2^-24, and never below the single-step bound."""
    return max(POT_RTOL, 4.0 * (2.0 * iters) ** 0.5 * 2.0 * 2.0 ** -24)


def f32(a):
    """Round an FP64 array to FP32 and back: the exact values the GPU receives."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_np(t):
    return t.detach().cpu().double().numpy()


def assert_pot_close(gpu, ref, rtol=POT_RTOL, what="potential"):
    """-inf pattern identical (index work: exact); finite entries normwise relative."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    fin_r = np.isfinite(ref)
    assert np.array_equal(np.isneginf(gpu), np.isneginf(ref)), f"{what}: -inf pattern differs"
    assert np.all(np.isfinite(gpu[fin_r])), f"{what}: non-finite GPU value"
    scale = np.abs(ref[fin_r]).max() if fin_r.any() else 1.0
    err = np.abs(gpu[fin_r] - ref[fin_r]).max() / max(scale, 1e-30)
    assert err <= rtol, f"{what}: normwise relative error {err:.3e} > {rtol:.1e}"
    return err


def normwise(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    fin = np.isfinite(ref)
    return np.abs(gpu[fin] - ref[fin]).max() / max(np.abs(ref[fin]).max(), 1e-30)
