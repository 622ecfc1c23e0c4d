"""Hand-written adjoint (fot_backward / the FOTPhase autograd function) against the dense
FP64 autograd oracle (tiny grids) and against finite differences of the GPU forward
(benchmark-size backward workload: 512^2, 100 iterations, eps 4 px^2, checkpoint every 10)."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint
from paper_2512_19072_gb300 import inputs
from fot_testutil import f32, to_dev

pytestmark = pytest.mark.gpu


def _loss_seed(phi, w, phi_t):
    # L = sum w phi + sum (phi - phi*)^2  ->  dL/dphi = w + 2 (phi - phi*)
    return w + 2.0 * (phi - phi_t)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_adjoint_matches_dense_oracle(fot_lib, prec):
    B = fot_lib
    P = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED}[prec]
    rng = np.random.default_rng(40)
    n_r, n_c = 24, 20
    g = f32(rng.uniform(0.3, 1.0, size=(n_r, n_c)))
    G = f32(rng.uniform(0.3, 1.0, size=(n_r, n_c)))
    eps, iters, dx = 30.0, 12, 1 / math.sqrt(24)
    w = f32(rng.uniform(0, 1, size=(n_r, n_c)))
    phi_t = f32(rng.normal(0, 0.1, size=(n_r, n_c)))
    L_ref, dg_ref, dG_ref = adjoint.gradients(g, G, eps, iters, w, phi_t, dx)
    gt, Gt = to_dev(g), to_dev(G)
    ctx = B.fot_create(n_r, n_c, P)
    B.fot_solve(ctx, gt, Gt, [eps], iters, dx=dx)
    phi, _, _ = B.fot_phase(ctx)
    seed = _loss_seed(phi, to_dev(w), to_dev(phi_t))
    dg, dG = B.fot_backward(ctx, gt, Gt, dL_dphi=seed, checkpoint_every=5)
    dg, dG = dg.double().cpu().numpy(), dG.double().cpu().numpy()
    for got, ref in ((dg, dg_ref), (dG, dG_ref)):
        assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_backward_workload_at_32_matches_dense_oracle(fot_lib, prec):
    """The backward workload's construction at 32 x 32 (two-Gaussian beam, ring/rectangle
    target with zero-mass background, eps 4 px^2, 100 iterations, checkpoint every 10)
    against the dense FP64 autograd gradient."""
    B = fot_lib
    P = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED}[prec]
    n = 32
    w4 = inputs.config4(n=n)
    g, G = f32(w4.g), f32(w4.G)
    w, phi_t = f32(w4.extra["w"]), f32(w4.extra["phi_target"])
    dx = 1 / math.sqrt(n)
    L_ref, dg_ref, dG_ref = adjoint.gradients(g, G, 4.0, w4.iters, w, phi_t, dx)
    ctx = B.fot_create(n, n, P)
    gt, Gt = to_dev(g), to_dev(G)
    B.fot_solve(ctx, gt, Gt, w4.eps, w4.iters, dx=dx)
    phi, _, _ = B.fot_phase(ctx)
    dg, dG = B.fot_backward(ctx, gt, Gt, dL_dphi=_loss_seed(phi, to_dev(w), to_dev(phi_t)),
                            checkpoint_every=10)
    dg, dG = dg.double().cpu().numpy(), dG.double().cpu().numpy()
    for got, ref in ((dg, dg_ref), (dG, dG_ref)):
        assert np.isfinite(got).all()
        assert (got[ref == 0] == 0).all()          # zero-mass pixels: derivative 0
        assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    ctx.close()


def test_autograd_function_and_checkpoint_invariance(fot_lib):
    B = fot_lib
    rng = np.random.default_rng(41)
    g = to_dev(f32(rng.uniform(0.3, 1.0, size=(40, 48))))
    G = to_dev(f32(rng.uniform(0.3, 1.0, size=(40, 48))))
    w = torch.rand(40, 48, device="cuda")
    g.requires_grad_(True)
    G.requires_grad_(True)
    phi, f, psi = B.fot_phase_fn(g, G, [8.0], 15, checkpoint_every=4)
    L = (w * phi).sum() + (phi ** 2).sum() + 1e-3 * (f * torch.isfinite(f)).nan_to_num().sum()
    dg, dG = torch.autograd.grad(L, (g, G))
    # same gradient through the C entry point with another checkpoint interval
    ctx = B.fot_create(40, 48)
    B.fot_solve(ctx, g.detach(), G.detach(), [8.0], 15)
    phi2, _, _ = B.fot_phase(ctx)
    df = 1e-3 * torch.isfinite(f).float()
    dg2, dG2 = B.fot_backward(ctx, g.detach(), G.detach(), dL_dphi=w + 2 * phi2, dL_df=df, checkpoint_every=15)
    assert torch.allclose(dg, dg2, rtol=1e-5, atol=1e-6 * dg.abs().max().item())
    assert torch.allclose(dG, dG2, rtol=1e-5, atol=1e-6 * dG.abs().max().item())
    ctx.close()


def test_adjoint_backward_workload_directional_fd(fot_lib):
    """512^2, 100 iterations at eps = 4 px^2, checkpoint every 10: the adjoint gradients of a
    phase loss and of a potentials loss agree with central differences of the GPU forward
    along seeded smooth directions.  (At this eps the 100 iterations are far from converged and
    the moment weights' row sums are far from 1, so the phase loss is large; its central
    differences are stable from h = 1e-2 down to 1e-4.)"""
    B = fot_lib
    w4 = inputs.config4()
    n = 512
    g, G = f32(w4.g), f32(w4.G)
    wt, phit = to_dev(f32(w4.extra["w"])), to_dev(f32(w4.extra["phi_target"]))
    w2 = to_dev(f32(np.random.default_rng(45).uniform(0, 1, size=(n, n))))
    ctx = B.fot_create(n, n)
    gt, Gt = to_dev(g), to_dev(G)

    def run(gg, GG):
        B.fot_solve(ctx, gg, GG, w4.eps, w4.iters)
        phi, _, _ = B.fot_phase(ctx)
        f, psi = B.fot_potentials(ctx)
        return phi.double(), f.double(), psi.double()

    def losses(r):
        phi, f, psi = r
        fin_f = torch.where(torch.isfinite(f), f, torch.zeros_like(f))
        fin_p = torch.where(torch.isfinite(psi), psi, torch.zeros_like(psi))
        Lph = (wt.double() * phi).sum().item() + ((phi - phit.double()) ** 2).sum().item()
        Lpo = (w2.double() * fin_p).sum().item() + (wt.double() * fin_f).sum().item()
        return Lph, Lpo

    phi, f, psi = run(gt, Gt)
    grads = {}
    grads["phase"] = B.fot_backward(ctx, gt, Gt, dL_dphi=_loss_seed(phi.float(), wt, phit),
                                    checkpoint_every=10)
    dL_df = torch.where(torch.isfinite(f), wt.double(), torch.zeros_like(f)).float().contiguous()
    dL_dpsi = torch.where(torch.isfinite(psi), w2.double(), torch.zeros_like(psi)).float().contiguous()
    grads["pot"] = B.fot_backward(ctx, gt, Gt, dL_df=dL_df, dL_dpsi=dL_dpsi, checkpoint_every=10)
    for dg, dG in grads.values():
        assert torch.isfinite(dg).all() and torch.isfinite(dG).all()
    rng = np.random.default_rng(44)
    x = np.linspace(-1, 1, n)
    h = 1e-2
    for which in ("g", "G"):
        base = g if which == "g" else G
        for _ in range(2):
            a = rng.normal(size=3)
            v = base * (a[0] + a[1] * x[:, None] + a[2] * x[None, :])      # smooth relative direction
            p, m = to_dev(base + h * v), to_dev(base - h * v)
            Lp = losses(run(p, Gt) if which == "g" else run(gt, p))
            Lm = losses(run(m, Gt) if which == "g" else run(gt, m))
            for k, kind in enumerate(("phase", "pot")):
                grad = grads[kind][0 if which == "g" else 1].double().cpu().numpy()
                fd = (Lp[k] - Lm[k]) / (2 * h)
                ad = float((grad * v).sum())
                assert abs(fd - ad) <= 2e-2 * abs(ad), (which, kind, fd, ad)
    ctx.close()
