"""Batched solves (many problems of their own sizes in multi-problem launches replayed as one
CUDA graph) against single-problem solves of the same problems, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, f32, to_dev, to_np

pytestmark = pytest.mark.gpu


def _problems():
    rng = np.random.default_rng(55)
    out = []
    for (n_r, n_c) in [(64, 64), (96, 96), (48, 80), (128, 128), (200, 200), (33, 65)]:
        g = f32(inputs.normalise_power(inputs.gauss(n_r, n_c, 0.15 * min(n_r, n_c))))
        G = f32(inputs.normalise_power(np.maximum(inputs.disk(n_r, n_c, 0.25 * min(n_r, n_c)),
                                                  inputs.rect(n_r, n_c, 0.1 * n_r, 0.2 * n_c,
                                                              rng.uniform(-5, 5), rng.uniform(-5, 5)))))
        out.append((g, G))
    return out


def _single(B, prec, g, G, eps, iters):
    ctx = B.fot_create(*g.shape, prec)
    B.fot_solve(ctx, to_dev(g), to_dev(G), eps, iters)
    f, psi = B.fot_potentials(ctx)
    ctx.close()
    return f, psi


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_batch_equals_single_solves(fot_lib, prec):
    B = fot_lib
    P = {"fp32": B.FOT_FP32, "mixed": B.FOT_MIXED}[prec]
    probs = _problems()
    iters = 30
    eps = np.stack([inputs.geometric_eps(0.05 * max(g.shape) ** 2, 2.0, iters) for g, _ in probs])
    batch = B.fot_batch_create([g.shape for g, _ in probs], P)
    gs = [to_dev(g) for g, _ in probs]
    Gs = [to_dev(G) for _, G in probs]
    B.fot_batch_solve(batch, gs, Gs, eps, iters)
    kernels, tensor = B.fot_batch_info(batch)
    # problem setup (3 kernels each), then per axis pass and per group of problems sharing a
    # kernel (FP32: one group; mixed: one per tensor tile width in use, at most 4, each split
    # into the problems the tensor kernel takes and the others) the window plan and one
    # window-sum kernel; the mixed form also writes a problem's B-operand table when its eps
    # changes (at most once per iteration and problem)
    base = 3 * len(probs) + iters * 4 * 2
    if prec == "fp32":
        assert kernels == base
    else:
        assert base <= kernels <= 3 * len(probs) + iters * 4 * 2 * 4 * 2 + iters * len(probs)
    assert tensor == (prec == "mixed")
    for q, (g, G) in enumerate(probs):
        f, psi = B.fot_potentials(B.fot_batch_context(batch, q))
        f1, psi1 = _single(B, P, g, G, eps[q], iters)
        # identical arithmetic in the multi-problem kernels: bitwise equal
        assert torch.equal(f, f1) and torch.equal(psi, psi1), q
    # replaying the captured graph reproduces the solve
    B.fot_batch_solve(batch, gs, Gs, eps, iters)
    f2, _ = B.fot_potentials(B.fot_batch_context(batch, 0))
    f1, _ = _single(B, P, probs[0][0], probs[0][1], eps[0], iters)
    assert torch.equal(f2, f1)
    batch.close()


def test_batch_auto_and_phase(fot_lib):
    B = fot_lib
    probs = _problems()[:3]
    iters = 20
    eps = np.full((len(probs), 1), 6.0)
    batch = B.fot_batch_create([g.shape for g, _ in probs], B.FOT_AUTO)
    B.fot_batch_solve(batch, [to_dev(g) for g, _ in probs], [to_dev(G) for _, G in probs], eps, iters)
    _, tensor = B.fot_batch_info(batch)
    for q, (g, G) in enumerate(probs):
        ctx = B.fot_batch_context(batch, q)
        f, psi = B.fot_potentials(ctx)
        f1, psi1 = _single(B, B.FOT_MIXED if tensor else B.FOT_FP32, g, G, [6.0], iters)
        assert torch.equal(f, f1)
        phi, Dx, Dy = B.fot_phase(ctx)
        assert torch.isfinite(phi).all()
        l1, _ = B.fot_marginal_error(ctx)
        assert np.isfinite(l1)
    batch.close()
