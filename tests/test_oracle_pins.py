"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute force (dense N x N cost, the LP), a closed form (Gaussian -> Gaussian entropic
transport), an independent 1-D recursion for product inputs, the literal exponential
form of Algorithm 1, and invariants of the iteration (marginals, dual ascent, symmetry).
CPU only."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore:invalid value encountered")

from oracle import fot, lp, onedim
from paper_2512_19072_gb300 import inputs


def _rand_masses(rng, n_r, n_c, zero_frac=0.0):
    g = rng.uniform(0.2, 1.0, size=(n_r, n_c))
    G = rng.uniform(0.2, 1.0, size=(n_r, n_c))
    if zero_frac:
        G[rng.uniform(size=G.shape) < zero_frac] = 0.0
    return g, G


# P1: separable factorisation of exp(-C/eps) (Sec. 3) equals the dense N x N cost
@pytest.mark.parametrize("shape,eps", [((6, 7), 0.7), ((8, 8), 3.0), ((12, 11), 25.0)])
def test_p1_dense_equals_separable(shape, eps):
    rng = np.random.default_rng(1)
    pot = rng.normal(0, 5.0, size=shape)
    pot[0, 0] = -np.inf
    S_sep = fot.log_kernel_apply(pot, eps)
    S_den = fot.log_kernel_apply_dense(pot, eps)
    assert np.allclose(S_sep, S_den, rtol=1e-12, atol=1e-12)
    g, G = _rand_masses(rng, *shape, zero_frac=0.2)
    r1 = fot.fot_iterate(g, G, eps, 6)
    r2 = fot.fot_iterate(g, G, eps, 6, dense=True)
    fin = np.isfinite(r2["psi"])
    assert np.array_equal(fin, np.isfinite(r1["psi"]))
    assert np.allclose(r1["f"], r2["f"], rtol=1e-12, atol=1e-11)
    assert np.allclose(r1["psi"][fin], r2["psi"][fin], rtol=1e-12, atol=1e-11)


# P2: the log-domain restatement equals Algorithm 1 as printed (exp domain, Eqs. 7-8)
def test_p2_expdomain_algorithm1():
    rng = np.random.default_rng(2)
    n_r, n_c = 16, 14
    g, G = _rand_masses(rng, n_r, n_c)
    eps = 12.0
    u, V, Lr, Lc = fot.fot_iterate_expdomain(g, G, eps, 25)
    r = fot.fot_iterate(g, G, eps, 25)
    assert np.allclose(eps * np.log(u), r["f"], rtol=1e-10, atol=1e-10)
    assert np.allclose(eps * np.log(V), r["psi"], rtol=1e-10, atol=1e-10)
    # Lambda is the Toeplitz matrix of the sampled Gaussian lambda_d (Sec. 3.1)
    d = np.arange(-(n_r - 1), n_r)
    lam = np.exp(-d.astype(float) ** 2 / (2 * eps))
    for j in range(n_r):
        assert np.allclose(Lr[j], lam[n_r - 1 - j: 2 * n_r - 1 - j])


# P3: product inputs -> every 2-D iterate is the outer sum of two 1-D iterates
def test_p3_separable_inputs_match_1d():
    w = inputs.separable_workload(24, 20, inputs.geometric_eps(30.0, 2.0, 12), 12)
    r = fot.fot_iterate(w.g, w.G, w.eps, w.iters)
    p, q, rr, s = (w.extra[k] for k in ("p", "q", "r", "s"))
    f1, psi1, _ = onedim.sinkhorn_1d(p * p, rr * rr, w.eps, w.iters)
    f2, psi2, _ = onedim.sinkhorn_1d(q * q, s * s, w.eps, w.iters)
    f_exp = f1[:, None] + f2[None, :]
    psi_exp = psi1[:, None] + psi2[None, :]
    fin = np.isfinite(psi_exp)
    assert np.array_equal(fin, np.isfinite(r["psi"]))
    assert np.allclose(r["f"], f_exp, rtol=1e-12, atol=1e-10)
    assert np.allclose(r["psi"][fin], psi_exp[fin], rtol=1e-12, atol=1e-10)


# P4: Gaussian -> Gaussian closed form.  Intensities with variance A, B per axis; the
# entropic plan (entropy w.r.t. the unit pixel measure) is Gaussian with covariance
# C = (sqrt(eps^2 + 4AB) - eps)/2, so E[L | j] - c = (C/A)(j - c): Dx is linear in j,
# and the trapezoid phase is exactly quadratic, phi = (C/A)((j-c)^2 + (k-c)^2)/(2n).
def test_p4_gaussian_closed_form():
    n, sg, sG, eps = 128, 6.0, 9.0, 8.0
    g, G = inputs.gaussian_pair(n, sg, sG)
    A, B = sg * sg / 2, sG * sG / 2
    slope = (math.sqrt(eps * eps + 4 * A * B) - eps) / 2 / A
    r = fot.fot_iterate(g, G, eps, 60)
    dx = 1 / math.sqrt(n)
    phi, Dx, Dy = fot.phase(r["psi"], r["S_last"], eps, dx)
    j = (np.arange(n) - n // 2).astype(float)
    mask = r["a"] > 1e-8 * r["a"].max()
    Dx_exp = np.broadcast_to(slope * j[:, None] / (n * dx), (n, n))
    Dy_exp = np.broadcast_to(slope * j[None, :] / (n * dx), (n, n))
    assert np.abs(Dx - Dx_exp)[mask].max() <= 1e-9 * np.abs(Dx_exp).max()
    assert np.abs(Dy - Dy_exp)[mask].max() <= 1e-9 * np.abs(Dy_exp).max()
    phi_exp = slope * (j[:, None] ** 2 + j[None, :] ** 2) / (2 * n)
    assert np.abs(phi - phi_exp)[mask].max() <= 1e-9 * np.abs(phi_exp).max()
    # converged: dual potentials quadratic too -> marginal error at round-off
    assert fot.marginal_l1(r["f"], r["psi"], r["a"], r["b"], eps) < 1e-12


# P5: eps -> infinity: the plan is the product a (x) b, so the phase gradient is the
# target centroid everywhere
def test_p5_large_eps_product_plan():
    rng = np.random.default_rng(5)
    n_r, n_c = 10, 12
    g, G = _rand_masses(rng, n_r, n_c, zero_frac=0.3)
    eps = 1e12
    r = fot.fot_iterate(g, G, eps, 2)
    dx = 0.37
    Dx, Dy = fot.moments(r["psi"], r["S_last"], eps, dx)
    b = r["b"]
    cx = (b.sum(1) * fot.target_coords(n_r, dx)).sum()
    cy = (b.sum(0) * fot.target_coords(n_c, dx)).sum()
    assert np.allclose(Dx, cx, atol=1e-8) and np.allclose(Dy, cy, atol=1e-8)


# P6: LP brute force (Eqs. 2-3 without entropy): 0 <= <C, Gamma_eps> - OT <= eps log(Na Nb);
# the c-transform dual of any psi is a lower bound of OT (weak duality)
def test_p6_lp_bounds():
    rng = np.random.default_rng(6)
    n = 5
    g, G = _rand_masses(rng, n, n, zero_frac=0.2)
    a, b = fot.marginal(g), fot.marginal(G)
    ot, plan, C = lp.ot_lp(a, b)
    eps = 0.3
    r = fot.fot_iterate(g, G, eps, 3000)
    f, psi = r["f"], r["psi"]
    # entropic plan Gamma = exp((f + psi - C)/eps), dense
    Gam = np.exp((f.ravel()[:, None] + psi.ravel()[None, :] - C) / eps)
    assert np.abs(Gam.sum(1) - a.ravel()).sum() < 1e-10
    cost_eps = float((Gam * C).sum())
    Na, Nb = (a > 0).sum(), (b > 0).sum()
    assert -1e-9 <= cost_eps - ot <= eps * (math.log(Na) + math.log(Nb))
    psic = fot.c_transform(psi)
    dual = float(np.where(a > 0, psic * a, 0).sum() + np.where(b > 0, psi * b, 0).sum())
    assert dual <= ot + 1e-9
    # and it is close for small eps (c-transform of the entropic potential)
    assert ot - dual < 3 * eps * math.log(Nb)


# P7: each half-step is an exact block-coordinate ascent of the entropic dual (fixed eps)
def test_p7_dual_ascent():
    rng = np.random.default_rng(7)
    g, G = _rand_masses(rng, 12, 12, zero_frac=0.15)
    a, b = fot.marginal(g), fot.marginal(G)
    vals = []

    def rec(t, stage, f, psi, eps):
        vals.append(fot.dual_objective(f, psi, a, b, eps))

    fot.fot_iterate(g, G, 2.0, 15, record=rec)
    d = np.diff(vals[1:])
    assert np.all(d >= -1e-13 * max(1.0, abs(vals[-1])))


# P8: after every V-update the column marginal of Gamma is exactly b (Eq. 8)
def test_p8_column_marginal_after_v():
    rng = np.random.default_rng(8)
    g, G = _rand_masses(rng, 9, 13, zero_frac=0.25)
    a, b = fot.marginal(g), fot.marginal(G)
    errs = []

    def rec(t, stage, f, psi, eps):
        if stage == "v":
            _, col = fot.plan_marginals(f, psi, eps)
            errs.append(np.abs(col - b).sum())

    fot.fot_iterate(g, G, inputs.geometric_eps(20.0, 1.0, 8), record=rec)
    assert max(errs) < 1e-13


# Eqs. 4-5 literally (plan formed, moments taken, divided by g^2) == separable moments
def test_moments_separable_equals_dense_plan():
    rng = np.random.default_rng(9)
    g, G = _rand_masses(rng, 7, 9, zero_frac=0.2)
    eps, dx = 1.7, 0.41
    r = fot.fot_iterate(g, G, eps, 5)
    Dx, Dy = fot.moments(r["psi"], r["S_last"], eps, dx)
    Dxd, Dyd = fot.moments_dense(r["f"], r["psi"], r["a"], eps, dx)
    assert np.allclose(Dx, Dxd, rtol=1e-11, atol=1e-12)
    assert np.allclose(Dy, Dyd, rtol=1e-11, atol=1e-12)


# trapezoid rule: exact for a linear gradient field; second order for smooth fields
def test_trapezoid_exact_and_order():
    n_r, n_c, dx = 9, 12, 0.25
    j = (np.arange(n_r) - n_r // 2)[:, None] * dx
    k = (np.arange(n_c) - n_c // 2)[None, :] * dx
    Dx = np.broadcast_to(3.0 * j + 1.5, (n_r, n_c))
    Dy = np.broadcast_to(-2.0 * k + 0.5, (n_r, n_c))
    phi = fot.integrate_trapezoid(Dx, Dy, dx)
    assert np.allclose(phi, 1.5 * j ** 2 + 1.5 * j - k ** 2 + 0.5 * k, atol=1e-13)
    errs = []
    for n in (33, 65):
        h = 2.0 / (n - 1)
        x = (np.arange(n) - n // 2)[:, None] * h
        y = (np.arange(n) - n // 2)[None, :] * h
        ph = fot.integrate_trapezoid(np.cos(x) * np.cos(y) + 0 * y, -np.sin(x) * np.sin(y), h)
        errs.append(np.abs(ph - np.sin(x) * np.cos(y)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


# P10: index conventions -- transposing both images transposes every output, and
# mirroring both along an axis mirrors the potentials
def test_p10_symmetry():
    rng = np.random.default_rng(10)
    g, G = _rand_masses(rng, 8, 11, zero_frac=0.2)
    eps = 1.5
    r = fot.fot_iterate(g, G, eps, 7)
    rt = fot.fot_iterate(g.T, G.T, eps, 7)
    assert np.allclose(rt["f"], r["f"].T, atol=1e-11)
    assert np.array_equal(np.isfinite(rt["psi"]), np.isfinite(r["psi"]).T)
    fin = np.isfinite(r["psi"])
    assert np.allclose(rt["psi"].T[fin], r["psi"][fin], atol=1e-11)
    rf = fot.fot_iterate(g[::-1], G[::-1], eps, 7)
    assert np.allclose(rf["f"][::-1], r["f"], atol=1e-11)
    # square grid: transposed problem swaps the two phase-gradient components
    g2, G2 = _rand_masses(rng, 9, 9)
    r2 = fot.fot_iterate(g2, G2, eps, 4)
    r2t = fot.fot_iterate(g2.T, G2.T, eps, 4)
    Dx, Dy = fot.moments(r2["psi"], r2["S_last"], eps, 0.3)
    Dxt, Dyt = fot.moments(r2t["psi"], r2t["S_last"], eps, 0.3)
    assert np.allclose(Dxt, Dy.T, atol=1e-12) and np.allclose(Dyt, Dx.T, atol=1e-12)


# c-transform: separable == dense brute force; entropic half-step -> c-transform as eps -> 0
# with 0 <= eps*LSE - max <= eps log(#terms)
def test_c_transform_pins():
    rng = np.random.default_rng(12)
    pot = rng.normal(0, 10.0, size=(7, 9))
    pot[2, 3] = -np.inf
    ct = fot.c_transform(pot)
    assert np.allclose(ct, fot.c_transform_dense(pot), atol=1e-12)
    N = np.isfinite(pot).sum()
    for eps in (1.0, 0.1, 0.01):
        soft = -eps * fot.log_kernel_apply(pot, eps)
        gap = ct - soft
        assert np.all(gap >= -1e-9) and np.all(gap <= eps * math.log(N) + 1e-9)


def test_marginal_l1_matches_dense_plan():
    rng = np.random.default_rng(13)
    g, G = _rand_masses(rng, 5, 6, zero_frac=0.2)
    eps = 0.9
    r = fot.fot_iterate(g, G, eps, 3)
    n_r, n_c = 5, 6
    jj, kk = np.meshgrid(np.arange(n_r), np.arange(n_c), indexing="ij")
    P = np.stack([jj.ravel(), kk.ravel()], 1).astype(float)
    C = ((P[:, None] - P[None]) ** 2).sum(-1) / 2
    Gam = np.exp((r["f"].ravel()[:, None] + r["psi"].ravel()[None, :] - C) / eps)
    l1 = np.abs(Gam.sum(1) - r["a"].ravel()).sum() + np.abs(Gam.sum(0) - r["b"].ravel()).sum()
    assert abs(fot.marginal_l1(r["f"], r["psi"], r["a"], r["b"], eps) - l1) < 1e-14
    D = (np.where(r["a"] > 0, r["f"] * r["a"], 0).sum() + np.where(r["b"] > 0, r["psi"] * r["b"], 0).sum()
         - eps * Gam.sum() + eps)
    assert abs(fot.dual_objective(r["f"], r["psi"], r["a"], r["b"], eps) - D) < 1e-12


# P13: the convergence stop (Sec. 3).  The source violation against the row sums of the dense
# plan Gamma = exp((f + psi - C)/eps) (the target half vanishing after a V-half), and the stop
# against the violations of the dense plan at the checks before and at it.
def _dense_violation(f, psi, a, b, eps):
    n_r, n_c = f.shape
    jj, kk = np.meshgrid(np.arange(n_r), np.arange(n_c), indexing="ij")
    P = np.stack([jj.ravel(), kk.ravel()], 1).astype(float)
    C = ((P[:, None] - P[None]) ** 2).sum(-1) / 2
    Gam = np.exp((f.ravel()[:, None] + psi.ravel()[None, :] - C) / eps)
    return np.abs(Gam.sum(1) - a.ravel()).sum(), np.abs(Gam.sum(0) - b.ravel()).sum()


def test_p13_source_violation_matches_dense_plan():
    rng = np.random.default_rng(17)
    g, G = _rand_masses(rng, 6, 5, zero_frac=0.2)
    g[0, 0] = 0.0
    for eps, iters in ((0.8, 2), (2.5, 4)):
        r = fot.fot_iterate(g, G, eps, iters)
        src, tgt = _dense_violation(r["f"], r["psi"], r["a"], r["b"], eps)
        assert tgt < 1e-13                      # the V-half left the column sums at b
        assert src > 1e-4                       # not yet converged: the check is not vacuous
        assert abs(fot.source_violation(r["f"], r["psi"], r["a"], eps) - src) < 1e-13


def test_p13_stop_rule_against_dense_plan():
    rng = np.random.default_rng(19)
    g, G = _rand_masses(rng, 5, 6, zero_frac=0.15)
    eps, k, max_iters = 1.2, 3, 30
    # the violations of the dense plan at every check, by brute force
    tvs = []
    for t in range(k, max_iters + 1, k):
        r = fot.fot_iterate(g, G, eps, t)
        tvs.append(sum(_dense_violation(r["f"], r["psi"], r["a"], r["b"], eps)))
    assert all(x > y for x, y in zip(tvs, tvs[1:]))          # decreasing here: a clean test
    i = 3
    tol = (tvs[i] * tvs[i - 1]) ** 0.5                       # between the checks i-1 and i
    r = fot.fot_iterate_tol(g, G, eps, max_iters, tol, k)
    assert r["iters"] == (i + 1) * k
    assert abs(r["tv"] - tvs[i]) < 1e-12 and r["tv"] <= tol
    ref = fot.fot_iterate(g, G, eps, (i + 1) * k)
    assert np.array_equal(r["f"], ref["f"]) and np.array_equal(r["psi"], ref["psi"])
    assert np.array_equal(r["S_last"], ref["S_last"])
    # never below tol: every check runs, the last one at max_iters (not a multiple of k here)
    r = fot.fot_iterate_tol(g, G, eps, 28, 0.0, k)
    assert r["iters"] == 28
    ref = fot.fot_iterate(g, G, eps, 28)
    assert abs(r["tv"] - sum(_dense_violation(ref["f"], ref["psi"], ref["a"], ref["b"], eps))) < 1e-12
    # already below tol at the first check
    assert fot.fot_iterate_tol(g, G, eps, max_iters, 10.0, k)["iters"] == k


# P14: the L1 intensity loss (Sec. 5).  The centred DFT against numpy's FFT with the centring
# done by index shifts, Parseval, and plane waves whose far field is one pixel.
def test_p14_intensity_loss():
    rng = np.random.default_rng(23)
    for n_r, n_c in ((8, 8), (6, 9), (16, 12)):
        g = rng.uniform(0.0, 1.0, size=(n_r, n_c))
        phi = rng.normal(0.0, 2.0, size=(n_r, n_c))
        G = rng.uniform(0.0, 1.0, size=(n_r, n_c))
        loss, inten = fot.intensity_loss(g, phi, G)
        field = g * np.exp(2j * np.pi * phi)
        X = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(field)))
        ref = np.abs(X) ** 2
        assert np.abs(inten - ref / ref.sum()).max() < 1e-13
        assert abs(ref.sum() - n_r * n_c * (g ** 2).sum()) < 1e-9 * ref.sum()      # Parseval
        b = G ** 2 / (G ** 2).sum()
        assert abs(loss - np.abs(ref / ref.sum() - b).sum()) < 1e-13
    # a uniform beam with the linear phase x . X0 lands on the single target pixel X0
    n = 16
    j = np.arange(n) - n // 2
    for L0, M0 in ((3, -5), (0, 0), (-8, 7)):
        phi = (np.add.outer(j * L0, j * M0)) / n          # cycles: (x X0) with dx dX = 1/n
        G = np.zeros((n, n))
        G[L0 + n // 2, M0 + n // 2] = 1.0
        loss, inten = fot.intensity_loss(np.ones((n, n)), phi, G)
        assert loss < 1e-12 and abs(inten[L0 + n // 2, M0 + n // 2] - 1.0) < 1e-12
    # and misses a target one pixel away entirely: the loss is the maximum, 2
    G = np.zeros((n, n))
    G[n // 2 + 1, n // 2] = 1.0
    assert abs(fot.intensity_loss(np.ones((n, n)), np.zeros((n, n)), G)[0] - 2.0) < 1e-12


# P15: cFOT (Sec. 3.1).  The linear convolutions against the Toeplitz products of the literal
# exponential-domain Algorithm 1, and against the log-domain iterate (same iteration, so same
# potentials, f = eps log u, psi = eps log V, and the same S_last).
def test_p15_cfot_equals_toeplitz_products():
    rng = np.random.default_rng(29)
    for (n_r, n_c), eps, iters in (((6, 9), 4.0, 5), ((12, 10), 20.0, 8)):
        g, G = _rand_masses(rng, n_r, n_c)
        u, V, S = fot.cfot_iterate(g, G, eps, iters)
        u2, V2, _, _ = fot.fot_iterate_expdomain(g, G, eps, iters)
        assert np.abs(u / u2 - 1).max() < 1e-12 and np.abs(V / V2 - 1).max() < 1e-12
        r = fot.fot_iterate(g, G, eps, iters)
        assert np.abs(eps * np.log(u) - r["f"]).max() < 1e-9 * np.abs(r["f"]).max()
        assert np.abs(eps * np.log(V) - r["psi"]).max() < 1e-9 * np.abs(r["psi"]).max()
        assert np.abs(S - r["S_last"]).max() < 1e-10


# P12: the dense autograd gradient of the phase loss (an independent dense implementation)
# against central finite differences, and its phase against the separable oracle
def test_p12_adjoint_oracle_vs_finite_differences():
    from oracle import adjoint
    rng = np.random.default_rng(12)
    n_r, n_c = 7, 8
    g = rng.uniform(0.3, 1.0, size=(n_r, n_c))
    G = rng.uniform(0.3, 1.0, size=(n_r, n_c))
    eps, iters, dx = 1.5, 6, 1 / math.sqrt(8)
    w = rng.uniform(0, 1, size=(n_r, n_c))
    phi_t = rng.normal(0, 0.1, size=(n_r, n_c))
    # the dense chain reproduces the separable oracle's phase
    import torch as _t
    _, phi_dense = adjoint.phase_loss(_t.tensor(g), _t.tensor(G), eps, iters, _t.tensor(w), _t.tensor(phi_t), dx)
    r = fot.fot_iterate(g, G, eps, iters)
    phi_sep, _, _ = fot.phase(r["psi"], r["S_last"], eps, dx)
    assert np.allclose(phi_dense.detach().numpy(), phi_sep, atol=1e-12)
    L, dg, dG = adjoint.gradients(g, G, eps, iters, w, phi_t, dx)
    h = 1e-3
    for (arr, grad) in ((g, dg), (G, dG)):
        for idx in [(0, 0), (3, 4), (6, 7), (2, 5)]:
            p = arr.copy(); p[idx] += h
            m = arr.copy(); m[idx] -= h
            if arr is g:
                fd = (adjoint.loss_value(p, G, eps, iters, w, phi_t, dx)
                      - adjoint.loss_value(m, G, eps, iters, w, phi_t, dx)) / (2 * h)
            else:
                fd = (adjoint.loss_value(g, p, eps, iters, w, phi_t, dx)
                      - adjoint.loss_value(g, m, eps, iters, w, phi_t, dx)) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-4 * max(1.0, abs(grad[idx])), (idx, fd, grad[idx])


# P12b: zero-mass pixels.  The loss sees a pixel of zero mass only through exp(f/eps) =
# a exp(-S), linear in a = amp^2 / sum amp^2, so its one-sided derivative at amp = 0 is 0;
# elsewhere the gradient still matches central differences, and nothing is NaN.
def test_p12b_adjoint_oracle_with_zero_masses():
    from oracle import adjoint
    rng = np.random.default_rng(13)
    n_r, n_c = 6, 7
    g = rng.uniform(0.3, 1.0, size=(n_r, n_c))
    G = rng.uniform(0.3, 1.0, size=(n_r, n_c))
    g[1, 2] = g[4, 6] = 0.0
    G[0, 0] = G[3, 3] = G[5, 1] = 0.0
    eps, iters, dx = 1.5, 6, 1 / math.sqrt(7)
    w = rng.uniform(0, 1, size=(n_r, n_c))
    phi_t = rng.normal(0, 0.1, size=(n_r, n_c))
    L, dg, dG = adjoint.gradients(g, G, eps, iters, w, phi_t, dx)
    assert np.isfinite(dg).all() and np.isfinite(dG).all()
    assert dg[1, 2] == 0.0 and dg[4, 6] == 0.0
    assert dG[0, 0] == 0.0 and dG[3, 3] == 0.0 and dG[5, 1] == 0.0
    h = 1e-3
    for (arr, grad) in ((g, dg), (G, dG)):
        for idx in [(0, 1), (2, 2), (5, 6)]:
            p = arr.copy(); p[idx] += h
            m = arr.copy(); m[idx] -= h
            args_p = (p, G) if arr is g else (g, p)
            args_m = (m, G) if arr is g else (g, m)
            fd = (adjoint.loss_value(*args_p, eps, iters, w, phi_t, dx)
                  - adjoint.loss_value(*args_m, eps, iters, w, phi_t, dx)) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-4 * max(1.0, abs(grad[idx])), (idx, fd, grad[idx])
    # one-sided difference at a zero-mass pixel: L(h) - L(0) = O(h^2)
    p = g.copy(); p[1, 2] = h
    d1 = adjoint.loss_value(p, G, eps, iters, w, phi_t, dx) - L
    assert abs(d1) <= 10 * h * h * max(1.0, abs(L)), d1
