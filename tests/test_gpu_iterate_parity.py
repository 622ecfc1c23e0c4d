"""The benchmark workload's own iterates against the oracle, at full size.

A full 200-iteration solve at 1024^2 or 2048^2 is far beyond the FP64 oracle, so the solve is
checked step by step instead:
  * a half-step (Algorithm 1, Eqs. 7-8) taken from the GPU's actual iterate (f, psi after the
    benchmark's 200 iterations, FP32 and mixed) is compared with the oracle's half-step from
    the same iterate on 64 sampled outputs, each computed one by one;
  * the phase step (Eqs. 9-10 and the trapezoid rule) at 1024^2 is compared over the whole
    image with the oracle's phase computed from the GPU's own potentials, against an a-priori
    bound on the FP32 rounding of that step alone.
Together with the element-wise solves at 256^2 (FP32 and mixed) these cover the iteration and
the phase of the benchmark workload."""
import math

import numpy as np
import pytest
import torch

from oracle import fot
from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, f32, phase_step_bound, solve_rtol, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:invalid value encountered"),
              pytest.mark.filterwarnings("ignore:divide by zero")]

# split-BF16 products (hi*hi + hi*lo + lo*hi) miss < 2^-16 relative per term: each of the two
# passes of a half-step adds < 2^-16 / ln 2 to a log2 output, i.e. |df| <= 2^-15 eps
MIXED_HALF_STEP = 2.0 ** -15
# single BF16 operands (FOT_BF16): each operand rounded to 8 significant bits (relative error
# <= 2^-8), a product within 2^-7 + 2^-16 relative, so each window sum within delta = 2^-7
# (1 + 2^-9) relative; each of the two passes of a half-step moves S by at most delta (natural
# log units): |df| <= 2 delta eps = 2^-6 (1 + 2^-9) eps
BF16_HALF_STEP = 2.0 ** -6 * (1 + 2.0 ** -9)


def _sampled_lse(pot, eps, samples):
    """S_jk = log sum_LM exp(pot_LM/eps - ((j-L)^2 + (k-M)^2)/(2 eps)) at the sampled (j, k),
    straight from the definition (the row sums for one output column k at a time)."""
    n_r, n_c = pot.shape
    M = np.arange(n_c, dtype=np.float64)
    L = np.arange(n_r, dtype=np.float64)
    out = {}
    for k in sorted({k for _, k in samples}):
        Rk = torch.logsumexp(torch.from_numpy(pot / eps - ((k - M) ** 2 / (2 * eps))[None, :]), dim=1).numpy()
        for j, kk in samples:
            if kk == k:
                out[(j, k)] = float(torch.logsumexp(torch.from_numpy(Rk - (j - L) ** 2 / (2 * eps)), dim=0))
    return out


def _solve(B, n, prec):
    w = inputs.config3(n)
    g, G = f32(w.g), f32(w.G)
    ctx = B.fot_create(n, n, prec)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    return w, g, G, ctx


def _prec(B, name):
    return {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED, "bf16": B.FOT_BF16}[name]


@pytest.mark.parametrize("prec", ["fp32", "mixed", "bf16"])
@pytest.mark.parametrize("n", [1024, 2048])
def test_iterate_half_steps_sampled(fot_lib, n, prec):
    B = fot_lib
    w, g, G, ctx = _solve(B, n, _prec(B, prec))
    eps = float(w.eps[-1])
    f_it, psi_it = (to_np(t) for t in B.fot_potentials(ctx))
    # one more u-half from the iterate's psi, and one more v-half from its f
    f_gpu, S_gpu = (to_np(t) for t in B.fot_u_update(ctx, to_dev(psi_it), eps, with_logsum=True))
    psi_gpu, T_gpu = (to_np(t) for t in B.fot_v_update(ctx, to_dev(f_it), eps, with_logsum=True))
    B.fot_sync(ctx)
    ctx.close()
    la, lb = fot.log0(fot.marginal(g)), fot.log0(fot.marginal(G))
    rng = np.random.default_rng(10 * n + (prec == "mixed"))
    samples = [(int(rng.integers(n)), int(k)) for k in rng.integers(0, n, size=16) for _ in range(4)]
    for pot_in, out_gpu, lse_gpu, lmarg in ((psi_it, f_gpu, S_gpu, la), (f_it, psi_gpu, T_gpu, lb)):
        ref = _sampled_lse(pot_in, eps, samples)
        lse_scale = max(abs(v) for v in ref.values())
        out_scale = np.abs(out_gpu[np.isfinite(out_gpu)]).max()
        for (j, k), S in ref.items():
            o_ref = eps * (lmarg[j, k] - S)
            if prec == "fp32":
                assert abs(lse_gpu[j, k] - S) <= POT_RTOL * lse_scale, ((j, k), lse_gpu[j, k], S)
                tol = POT_RTOL * out_scale
            else:
                tol = POT_RTOL * out_scale + (MIXED_HALF_STEP if prec == "mixed" else BF16_HALF_STEP) * eps
            if np.isfinite(o_ref):
                assert abs(out_gpu[j, k] - o_ref) <= tol, ((j, k), out_gpu[j, k], o_ref, tol)
            else:
                assert out_gpu[j, k] == -np.inf


@pytest.mark.parametrize("prec", ["mixed"])
def test_full_size_phase_from_gpu_potentials(fot_lib, prec):
    """1024^2, 200 iterations: the GPU phase against the oracle's phase step from the GPU's
    potentials (the potentials themselves are covered by the half-step checks above; the
    phase step is the same FP32 kernel pair in both precisions, so the benchmark's mixed form
    is taken)."""
    B = fot_lib
    n = 1024
    w, g, G, ctx = _solve(B, n, _prec(B, prec))
    eps = float(w.eps[-1])
    dx = 1.0 / math.sqrt(n)
    f_gpu, psi_gpu = (to_np(t) for t in B.fot_potentials(ctx))
    phi, Dx, Dy = (to_np(t) for t in B.fot_phase(ctx))
    ctx.close()
    la = fot.log0(fot.marginal(g))
    with np.errstate(invalid="ignore"):
        S_last = np.where(np.isfinite(f_gpu), la - f_gpu / eps, -np.inf)
    phi_ref, Dx_ref, Dy_ref = fot.phase(psi_gpu, S_last, eps, dx)
    bound, Bd = phase_step_bound(psi_gpu, S_last, eps, dx, phi_ref)
    live = np.isfinite(Dx_ref)
    assert (np.abs(Dx - Dx_ref)[live] <= Bd[live] + 1e-6 * np.abs(Dx_ref[live]).max()).all()
    assert (np.abs(Dy - Dy_ref)[live] <= Bd[live] + 1e-6 * np.abs(Dy_ref[live]).max()).all()
    err = np.abs(phi - phi_ref)
    assert (err <= bound).all(), (err.max(), bound[err > bound].min())


@pytest.fixture(scope="module")
def c3_256_ref():
    w = inputs.config3(256)
    g, G = f32(w.g), f32(w.G)
    return w, g, G, fot.fot_iterate(g, G, w.eps, w.iters)


@pytest.mark.parametrize("prec", ["mixed", "bf16"])
def test_tensor_solve_256_matches_oracle(fot_lib, c3_256_ref, prec):
    """Config 3 at 256^2, 200 iterations, tensor-core forms, against the oracle's FP64 iterate.

    Each update is 1-Lipschitz in the sup norm (a log-sum-exp of its input plus a constant), so
    the operand rounding error of each half-step (2^-15 eps for split BF16, 2^-7 eps for single
    BF16) adds at most linearly over the 2T half-steps; the FP32 rounding adds as in the FP32
    solve (solve_rtol)."""
    B = fot_lib
    w, g, G, r = c3_256_ref
    step = MIXED_HALF_STEP if prec == "mixed" else BF16_HALF_STEP
    ctx = B.fot_create(256, 256, _prec(B, prec))
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    f, psi = (to_np(t) for t in B.fot_potentials(ctx))
    _, tensor_terms = B.fot_work_count(ctx, tensor=True)
    assert tensor_terms > 0
    for gpu, ref, what in ((f, r["f"], "f"), (psi, r["psi"], "psi")):
        fin = np.isfinite(ref)
        assert np.array_equal(np.isneginf(gpu), np.isneginf(ref)), what
        scale = np.abs(ref[fin]).max()
        tol = 2 * w.iters * step * float(np.max(w.eps)) + solve_rtol(w.iters) * scale
        err = np.abs(gpu[fin] - ref[fin]).max()
        assert err <= tol, (what, err, tol)
    l1, _ = B.fot_marginal_error(ctx)
    l1_ref = fot.marginal_l1(r["f"], r["psi"], r["a"], r["b"], r["eps_last"])
    assert abs(l1 - l1_ref) <= (1e-3 if prec == "mixed" else 2e-2) + 1e-2 * l1_ref
    ctx.close()
