"""Comparison helpers shared by the GPU parity tests (no method arithmetic here beyond the
oracle calls that size an error bound)."""
import numpy as np
import torch

from oracle import fot

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


def phase_step_bound(psi, S_last, eps, dx, phi_ref, rounding=8):
    """A-priori bound on |phi_gpu - phi_ref| when both take the phase step (Eqs. 9-10, then
    the trapezoid rule) from the same (psi, S_last) and the GPU works in FP32.

    Every moment weight is exp of a log value of magnitude <= lmax (psi/eps, the Gaussian
    exponent, S_last); `rounding` FP32 roundings of such values change it by a relative
    d <= rounding * 2^-24 * lmax.  The first moments then move by at most (e^(2d) - 1) max|X| W,
    W = sum of the weights = exp(S(psi) - S_last), and the trapezoid steps add these along
    their path (the centre column, then the row), plus FP32 rounding of the running sums."""
    n_r, n_c = psi.shape
    fin_p = np.isfinite(psi)
    S_psi = fot.log_kernel_apply(psi, eps)
    fin_w = np.isfinite(S_psi) & np.isfinite(S_last)
    W = np.where(fin_w, np.exp(np.where(fin_w, S_psi - S_last, 0.0)), 0.0)
    lmax = np.abs(S_last[fin_w]).max() + np.abs(psi[fin_p]).max() / eps
    d = rounding * 2.0 ** -24 * lmax
    Xmax = max(n_r, n_c) // 2 / (max(n_r, n_c) * dx)
    Bd = np.expm1(2 * d) * Xmax * W
    cr, cc = n_r // 2, n_c // 2
    seg_c = dx * 0.5 * (Bd[1:, cc] + Bd[:-1, cc])
    col = np.zeros(n_r)
    col[cr + 1:] = np.cumsum(seg_c[cr:])
    col[:cr] = np.cumsum(seg_c[:cr][::-1])[::-1]
    seg_r = dx * 0.5 * (Bd[:, 1:] + Bd[:, :-1])
    row = np.zeros((n_r, n_c))
    row[:, cc + 1:] = np.cumsum(seg_r[:, cc:], axis=1)
    row[:, :cc] = np.cumsum(seg_r[:, :cc][:, ::-1], axis=1)[:, ::-1]
    return col[:, None] + row + (n_r + n_c) * 2.0 ** -23 * np.abs(phi_ref).max(), Bd
