"""CUDA path (through the C ABI) vs the FP64 oracle on seeded inputs.

Small and mid sizes: element by element against the oracle (several tiles and ragged
tails).  Full sizes (1024^2, 2048^2, the benchmark configuration): against the 1-D
oracle for product inputs (every element), and single half-steps checked on sampled
outputs that the oracle computes one by one.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fot, onedim
from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, assert_pot_close, f32, normwise, phase_step_bound, solve_rtol, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:invalid value encountered")]


def _masses(rng, shape, zero_frac):
    g = rng.uniform(0.05, 1.0, size=shape)
    G = rng.uniform(0.05, 1.0, size=shape)
    g[rng.uniform(size=shape) < zero_frac] = 0.0
    G[rng.uniform(size=shape) < zero_frac] = 0.0
    return f32(g), f32(G)


# ---------------------------------------------------------------------------------------
# single half-steps (Eqs. 7-8), all shapes and eps regimes
# ---------------------------------------------------------------------------------------
SHAPES = [(1, 1), (1, 37), (29, 1), (8, 8), (33, 47), (64, 64), (100, 130), (257, 200)]
EPSS = [0.3, 4.0, 60.0, 3000.0]


@pytest.mark.parametrize("prec", ["banded", "dense"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("eps", EPSS)
def test_half_steps_match_oracle(fot_lib, shape, eps, prec):
    """Both FP32 kernels (banded windows with the tilted GEMM or exact windowed sums, and
    the dense exact pass) against the oracle's half-step."""
    B = fot_lib
    rng = np.random.default_rng(hash((shape, eps)) % 2**32)
    g, G = _masses(rng, shape, 0.15)
    if g.sum() == 0:
        g[0, 0] = 1.0
    if G.sum() == 0:
        G[-1, -1] = 1.0
    n = max(shape)
    psi = f32(inputs.random_potential(*shape, scale=0.3 * n * n + 5 * eps, seed=3, zero_frac=0.1))
    ctx = B.fot_create(*shape, B.FOT_FP32 if prec == "banded" else B.FOT_FP32_DENSE)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    f_gpu, S_gpu = B.fot_u_update(ctx, to_dev(psi), eps, with_logsum=True)
    psi_gpu, T_gpu = B.fot_v_update(ctx, f_gpu, eps, with_logsum=True)
    B.fot_sync(ctx)
    la, lb = fot.log0(fot.marginal(g)), fot.log0(fot.marginal(G))
    f_ref, S_ref = fot.u_update(psi, la, eps)
    assert_pot_close(to_np(f_gpu), f_ref, what="f")
    assert normwise(to_np(S_gpu), S_ref) <= POT_RTOL
    # the GPU's v-update continues from its own f; the oracle from its own f_ref
    psi_ref, _ = fot.v_update(f_ref, lb, eps)
    assert_pot_close(to_np(psi_gpu), psi_ref, rtol=4 * POT_RTOL, what="psi")
    ctx.close()


# ---------------------------------------------------------------------------------------
# full solves against the oracle
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1_ref():
    w = inputs.config1()
    g, G = f32(w.g), f32(w.G)
    r = fot.fot_iterate(g, G, w.eps, w.iters)
    dx = 1 / math.sqrt(64)
    r["phi"], r["Dx"], r["Dy"] = fot.phase(r["psi"], r["S_last"], r["eps_last"], dx)
    r["l1"] = fot.marginal_l1(r["f"], r["psi"], r["a"], r["b"], r["eps_last"])
    return w, g, G, r


def test_config1_solve_and_phase(fot_lib, c1_ref):
    B = fot_lib
    w, g, G, r = c1_ref
    ctx = B.fot_create(64, 64)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    f, psi = B.fot_potentials(ctx)
    tol = solve_rtol(w.iters)
    assert_pot_close(to_np(f), r["f"], rtol=tol, what="f")
    assert_pot_close(to_np(psi), r["psi"], rtol=tol, what="psi")
    phi, Dx, Dy = (to_np(t) for t in B.fot_phase(ctx))
    # the phase step against the oracle's phase step from the GPU's own potentials (those are
    # checked against the oracle's iterate just above), within the a-priori FP32 bound of that
    # step alone
    f_np, psi_np = to_np(f), to_np(psi)
    eps, dx = r["eps_last"], 1 / math.sqrt(64)
    la = fot.log0(fot.marginal(g))
    with np.errstate(invalid="ignore"):
        S_last = np.where(np.isfinite(f_np), la - f_np / eps, -np.inf)
    phi_ref, Dx_ref, Dy_ref = fot.phase(psi_np, S_last, eps, dx)
    bound, Bd = phase_step_bound(psi_np, S_last, eps, dx, phi_ref)
    live = np.isfinite(Dx_ref)
    assert (np.abs(Dx - Dx_ref)[live] <= Bd[live] + 1e-6 * np.abs(Dx_ref[live]).max()).all()
    assert (np.abs(Dy - Dy_ref)[live] <= Bd[live] + 1e-6 * np.abs(Dy_ref[live]).max()).all()
    assert (np.abs(phi - phi_ref) <= bound).all()
    l1, dual = B.fot_marginal_error(ctx)
    assert abs(l1 - r["l1"]) <= 1e-6 + 1e-3 * r["l1"]
    ctx.close()


@pytest.mark.parametrize("cfg", ["c2", "c3_256"])
def test_annealed_and_composite_solves_256(fot_lib, cfg):
    B = fot_lib
    w = inputs.config2() if cfg == "c2" else inputs.config3(256)
    g, G = f32(w.g), f32(w.G)
    r = fot.fot_iterate(g, G, w.eps, w.iters)
    ctx = B.fot_create(256, 256)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    f, psi = B.fot_potentials(ctx)
    assert_pot_close(to_np(f), r["f"], rtol=solve_rtol(w.iters), what="f")
    assert_pot_close(to_np(psi), r["psi"], rtol=solve_rtol(w.iters), what="psi")
    l1, _ = B.fot_marginal_error(ctx)
    l1_ref = fot.marginal_l1(r["f"], r["psi"], r["a"], r["b"], r["eps_last"])
    assert abs(l1 - l1_ref) <= 2e-5 + 1e-2 * l1_ref
    ctx.close()


@pytest.mark.parametrize("shape,eps", [((9, 7), 0.8), ((64, 64), 3.0), ((130, 97), 40.0)])
def test_moments_kernel_matches_oracle(fot_lib, shape, eps):
    """Eqs. 9-10 and the trapezoid step on seeded (psi, S) inputs, element by element."""
    B = fot_lib
    n = max(shape)
    psi = f32(inputs.random_potential(*shape, scale=0.2 * n * n + 5 * eps, seed=21, zero_frac=0.15))
    S = f32(fot.log_kernel_apply(psi, eps) + np.random.default_rng(5).normal(0, 0.3, size=shape))
    dx = 0.37
    ctx = B.fot_create(*shape)
    phi, Dx, Dy = (to_np(t) for t in B.fot_moments(ctx, to_dev(psi), to_dev(S), eps, dx))
    Dx_r, Dy_r = fot.moments(psi, S, eps, dx)
    phi_r = fot.integrate_trapezoid(Dx_r, Dy_r, dx)
    # FP32 log-domain values of magnitude |v| carry absolute errors of 2^-24 |v|, which become
    # relative errors of the exponential weights: bound from the largest log value involved
    # (S and psi/eps, in log2 units), times the largest coordinate.
    lmax = (np.abs(S).max() + np.abs(psi[np.isfinite(psi)]).max() / eps) / np.log(2)
    cmax = max(shape) / 2 / (min(shape) * dx)
    tol = 4 * 2.0 ** -24 * lmax * cmax + 1e-6 * max(np.abs(Dx_r).max(), 1e-3)
    assert np.abs(Dx - Dx_r).max() <= tol and np.abs(Dy - Dy_r).max() <= tol
    assert np.abs(phi - phi_r).max() <= tol * max(shape) * dx
    ctx.close()


def test_work_counter(fot_lib):
    B = fot_lib
    ctx = B.fot_create(40, 56, B.FOT_FP32_DENSE)
    g = torch.rand(40, 56, device="cuda") + 0.1
    B.fot_solve(ctx, g, g, [2.0], 3)
    assert B.fot_work_count(ctx) == 3 * 2 * (40 * 56 * 56 + 56 * 40 * 40)
    ctx2 = B.fot_create(40, 56, B.FOT_FP32)
    B.fot_solve(ctx2, g, g, [2.0], 3)
    t = B.fot_work_count(ctx2)
    assert 0 < t <= 3 * 2 * (40 * 56 * 56 + 56 * 40 * 40) * 2
    ctx.close()
    ctx2.close()


def test_gaussian_closed_form_phase(fot_lib):
    """Gaussian -> Gaussian: Dx linear with slope C/A (closed form), phi quadratic."""
    B = fot_lib
    n, sg, sG, eps = 128, 6.0, 9.0, 8.0
    g, G = inputs.gaussian_pair(n, sg, sG)
    A, Bv = sg * sg / 2, sG * sG / 2
    slope = (math.sqrt(eps * eps + 4 * A * Bv) - eps) / 2 / A
    ctx = B.fot_create(n, n)
    B.fot_solve(ctx, to_dev(g), to_dev(G), [eps], 60)
    phi, Dx, Dy = (to_np(t) for t in B.fot_phase(ctx))
    j = (np.arange(n) - n // 2).astype(float)
    dx = 1 / math.sqrt(n)
    mask = fot.marginal(g) > 1e-6 * fot.marginal(g).max()
    Dx_exp = np.broadcast_to(slope * j[:, None] / (n * dx), (n, n))
    assert np.abs(Dx - Dx_exp)[mask].max() <= 2e-5 * np.abs(Dx_exp).max()
    phi_exp = slope * (j[:, None] ** 2 + j[None, :] ** 2) / (2 * n)
    assert np.abs(phi - phi_exp)[mask].max() <= 2e-5 * np.abs(phi_exp).max()
    ctx.close()


def test_resume_equals_uninterrupted(fot_lib):
    B = fot_lib
    w = inputs.config2(n=96, iters=40)
    g, G = to_dev(f32(w.g)), to_dev(f32(w.G))
    ctx = B.fot_create(96, 96)
    B.fot_solve(ctx, g, G, w.eps, w.iters)
    f1, p1 = B.fot_potentials(ctx)
    B.fot_solve(ctx, g, G, w.eps[:25], 25)
    f0, p0 = B.fot_potentials(ctx)
    B.fot_set_potentials(ctx, f0, p0)
    B.fot_resume(ctx, w.eps[25:], 15)
    f2, p2 = B.fot_potentials(ctx)
    assert torch.equal(f1, f2) and torch.equal(p1, p2)   # deterministic: bitwise
    ctx.close()


# ---------------------------------------------------------------------------------------
# full size: product inputs vs the 1-D oracle, element by element
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1024, 2048])
def test_full_size_separable_matches_1d_oracle(fot_lib, n):
    B = fot_lib
    iters = 200 if n == 1024 else 60
    w = inputs.separable_workload(n, n, 2e-4 * n * n, iters)
    p, q, r_, s_ = (f32(w.extra[k]) for k in ("p", "q", "r", "s"))
    g = np.outer(p, q)
    G = np.outer(r_, s_)
    ctx = B.fot_create(n, n)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, iters)
    f, psi = (to_np(t) for t in B.fot_potentials(ctx))
    # product of FP32-rounded factors: the 1-D problems are p*p etc. up to FP32 rounding
    f1, psi1, _ = onedim.sinkhorn_1d(p * p, r_ * r_, w.eps, iters)
    f2, psi2, _ = onedim.sinkhorn_1d(q * q, s_ * s_, w.eps, iters)
    assert_pot_close(f, f1[:, None] + f2[None, :], rtol=solve_rtol(iters), what="f")
    assert_pot_close(psi, psi1[:, None] + psi2[None, :], rtol=solve_rtol(iters), what="psi")
    ctx.close()


def _sampled_S(psi, eps, samples):
    """S_jk = log sum_LM exp(psi/eps - C/eps) for sampled (j, k), one column at a time."""
    n_r, n_c = psi.shape
    M = np.arange(n_c, dtype=np.float64)
    L = np.arange(n_r, dtype=np.float64)
    out = {}
    for k in sorted({k for _, k in samples}):
        E = torch.from_numpy(psi / eps - ((k - M) ** 2 / (2 * eps))[None, :])
        Rk = torch.logsumexp(E, dim=1).numpy()                     # R[L, k]
        for j, kk in samples:
            if kk == k:
                out[(j, k)] = float(torch.logsumexp(
                    torch.from_numpy(Rk - (j - L) ** 2 / (2 * eps)), dim=0))
    return out


@pytest.mark.parametrize("n", [1024, 2048])
def test_full_size_half_step_sampled(fot_lib, n):
    """Benchmark-size single u-update from a seeded potential: 64 sampled outputs vs the
    oracle computed one by one (eps = 2e-4 n^2, the benchmark value)."""
    B = fot_lib
    w = inputs.config3(n)
    eps = float(w.eps[0])
    g, G = f32(w.g), f32(w.G)
    psi = f32(inputs.random_potential(n, n, scale=0.3 * n * n, seed=7))
    psi[f32(w.G) == 0] = -np.inf
    ctx = B.fot_create(n, n)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    f_gpu, S_gpu = B.fot_u_update(ctx, to_dev(psi), eps, with_logsum=True)
    f_gpu, S_gpu = to_np(f_gpu), to_np(S_gpu)
    rng = np.random.default_rng(n)
    samples = [(int(rng.integers(n)), int(k)) for k in rng.integers(0, n, size=16) for _ in range(4)]
    ref = _sampled_S(psi, eps, samples)
    la = fot.log0(fot.marginal(g))
    S_scale = max(abs(v) for v in ref.values())
    f_scale = np.abs(f_gpu[np.isfinite(f_gpu)]).max()
    for (j, k), S in ref.items():
        assert abs(S_gpu[j, k] - S) <= POT_RTOL * S_scale
        f_ref = eps * (la[j, k] - S)
        if np.isfinite(f_ref):
            assert abs(f_gpu[j, k] - f_ref) <= POT_RTOL * f_scale
        else:
            assert f_gpu[j, k] == -np.inf
    ctx.close()


def test_full_size_transpose_symmetry(fot_lib):
    """Benchmark workload (1024^2, 200 its): transposing both images transposes f."""
    B = fot_lib
    w = inputs.config3(1024)
    g, G = f32(w.g), f32(w.G)
    ctx = B.fot_create(1024, 1024)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    f, psi = (to_np(t) for t in B.fot_potentials(ctx))
    l1, _ = B.fot_marginal_error(ctx)
    B.fot_solve(ctx, to_dev(np.ascontiguousarray(g.T)), to_dev(np.ascontiguousarray(G.T)),
                w.eps, w.iters)
    ft, psit = (to_np(t) for t in B.fot_potentials(ctx))
    assert_pot_close(ft.T, f, rtol=4 * POT_RTOL, what="f^T")
    assert_pot_close(psit.T, psi, rtol=4 * POT_RTOL, what="psi^T")
    assert np.isfinite(l1) and 0.0 <= l1 <= 2.0
    ctx.close()


# ---------------------------------------------------------------------------------------
# c-transform (eps -> 0 limit) against brute force
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1), (7, 9), (64, 64), (130, 97), (300, 257)])
def test_c_transform_matches_oracle(fot_lib, shape):
    B = fot_lib
    n = max(shape)
    pot = f32(inputs.random_potential(*shape, scale=0.3 * n * n + 10, seed=11, zero_frac=0.2))
    ctx = B.fot_create(*shape)
    out = to_np(B.fot_c_transform(ctx, to_dev(pot)))
    ref = fot.c_transform(pot)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.abs(out[fin] - ref[fin]).max() <= 1e-6 * max(1.0, np.abs(ref[fin]).max())
    ctx.close()


# ---------------------------------------------------------------------------------------
# errors found on the device are latched and reported, never faulting
# ---------------------------------------------------------------------------------------
def test_device_error_reporting(fot_lib):
    B = fot_lib
    ctx = B.fot_create(16, 16)
    ok = torch.ones(16, 16, device="cuda")
    zero = torch.zeros(16, 16, device="cuda")
    with pytest.raises(B.FotError) as e:
        B.fot_phase(ctx)
    assert e.value.status == 8                       # FOT_ESTATE
    B.fot_solve(ctx, ok, zero, [1.0], 3)
    with pytest.raises(B.FotError) as e:
        B.fot_sync(ctx)
    assert e.value.status == 6                       # FOT_EMASS
    bad = ok.clone()
    bad[3, 4] = float("nan")
    B.fot_solve(ctx, bad, ok, [1.0], 3)
    with pytest.raises(B.FotError) as e:
        B.fot_sync(ctx)
    assert e.value.status == 1                       # FOT_EINVAL
    neg = ok.clone()
    neg[0, 0] = -1.0
    B.fot_solve(ctx, ok, neg, [1.0], 3)
    with pytest.raises(B.FotError) as e:
        B.fot_potentials(ctx)
    assert e.value.status == 1
    # the latch clears on the next solve
    B.fot_solve(ctx, ok, ok, [1.0], 3)
    B.fot_sync(ctx)
    with pytest.raises(B.FotError):
        B.fot_solve(ctx, ok, ok, [1.0, 2.0], 3)    # schedule length mismatch (host-side)
    ctx.close()


def test_host_buffer_entry_point(fot_lib, c1_ref):
    B = fot_lib
    w, g, G, r = c1_ref
    ctx = B.fot_create(64, 64)
    gh = torch.from_numpy(g.astype(np.float32)).pin_memory()
    Gh = torch.from_numpy(G.astype(np.float32)).pin_memory()
    phi = B.fot_solve_phase_host(ctx, gh, Gh, w.eps, w.iters)
    assert normwise(phi.double().numpy(), r["phi"]) <= 2e-6
    assert B.fot_launch_count(ctx) > 4 * w.iters
    ctx.close()


# ---------------------------------------------------------------------------------------
# mixed precision: the banded GEMM on tcgen05 tensor cores with split-BF16 operands
# ---------------------------------------------------------------------------------------
# Bound: every product is hi*hi + hi*lo + lo*hi of two-part BF16 operands, missing lo*lo and
# the rounding of the lo parts, i.e. < 2^-16 relative; all terms are positive, so each window
# sum is within 2^-16 relative and each pass adds < 2^-16 / ln 2 to a log2 output.  Two passes
# per half-step: |df| <= eps * ln 2 * 2 * 2^-16 / ln 2 = 2^-15 eps, plus FP32 rounding.
def mixed_atol(eps):
    return 2.0 ** -15 * eps


@pytest.mark.parametrize("shape", [(64, 64), (100, 130), (257, 200), (300, 300)])
@pytest.mark.parametrize("eps", [4.0, 12.0, 60.0, 300.0, 3000.0])
def test_mixed_half_steps_match_oracle(fot_lib, shape, eps):
    """eps 4: no tile can meet the tensor kernel's tilt bound (the pass runs the CUDA-core
    kernels); eps 12: 16-wide tensor tiles, and the tiles the kernel declines are computed
    with the CUDA-core window sums inside the same launch; eps 60: 16-wide tensor tiles;
    eps 300: 64-wide tensor tiles, the noisy potential's long windows declining some of them
    (exact window sums over the 64-wide tile's window); eps 3000: 64-wide tensor tiles."""
    B = fot_lib
    rng = np.random.default_rng(hash((shape, eps, "mixed")) % 2**32)
    g, G = _masses(rng, shape, 0.15)
    n = max(shape)
    psi = f32(inputs.random_potential(*shape, scale=0.3 * n * n + 5 * eps, seed=3, zero_frac=0.1))
    ctx = B.fot_create(*shape, B.FOT_MIXED)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    f_gpu, S_gpu = B.fot_u_update(ctx, to_dev(psi), eps, with_logsum=True)
    B.fot_sync(ctx)
    _, tensor_terms = B.fot_work_count(ctx, tensor=True)
    split = B.fot_work_split(ctx)
    la = fot.log0(fot.marginal(g))
    f_ref, S_ref = fot.u_update(psi, la, eps)
    f_np = to_np(f_gpu)
    fin = np.isfinite(f_ref)
    assert np.array_equal(np.isneginf(f_np), np.isneginf(f_ref))
    err = np.abs(f_np[fin] - f_ref[fin]).max()
    assert err <= POT_RTOL * np.abs(f_ref[fin]).max() + mixed_atol(eps), (err, mixed_atol(eps))
    if eps >= 3000.0:
        assert tensor_terms > 0          # these tiles satisfy the tilt bounds: tensor cores used
    if eps == 4.0 or (eps == 12.0 and n > 64):
        assert split[0] + split[1] > 0, split   # CUDA-core window sums ran (at 64^2 and eps 12
                                                # every tile meets the tensor kernel's bound)
    if eps == 4.0:
        assert split[2] == 0, split            # no tile can meet the tilt bound at eps 4
    ctx.close()


@pytest.mark.parametrize("n", [1024, 2048])
def test_mixed_full_size_half_step_sampled(fot_lib, n):
    B = fot_lib
    w = inputs.config3(n)
    eps = float(w.eps[0])
    g, G = f32(w.g), f32(w.G)
    psi = f32(inputs.random_potential(n, n, scale=0.3 * n * n, seed=7))
    psi[f32(w.G) == 0] = -np.inf
    ctx = B.fot_create(n, n, B.FOT_MIXED)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    f_gpu = to_np(B.fot_u_update(ctx, to_dev(psi), eps))
    # (the noisy potential's windows are long: many wide tensor tiles are declined here and
    # take the exact window sums, so both forms are checked)
    rng = np.random.default_rng(n + 1)
    samples = [(int(rng.integers(n)), int(k)) for k in rng.integers(0, n, size=16) for _ in range(4)]
    ref = _sampled_S(psi, eps, samples)
    la = fot.log0(fot.marginal(g))
    f_scale = np.abs(f_gpu[np.isfinite(f_gpu)]).max()
    for (j, k), S in ref.items():
        f_ref = eps * (la[j, k] - S)
        if np.isfinite(f_ref):
            assert abs(f_gpu[j, k] - f_ref) <= POT_RTOL * f_scale + mixed_atol(eps)
        else:
            assert f_gpu[j, k] == -np.inf
    ctx.close()


def test_mixed_solve_marginal_matches_fp32(fot_lib):
    """Benchmark workload at 1024^2, 200 iterations: the mixed iterate's marginal L1 equals
    the FP32 iterate's to within 1e-4 (the marginal-error requirement of the mixed form)."""
    B = fot_lib
    w = inputs.config3(1024)
    g, G = to_dev(f32(w.g)), to_dev(f32(w.G))
    out = {}
    for name, prec in (("fp32", B.FOT_FP32), ("mixed", B.FOT_MIXED)):
        ctx = B.fot_create(1024, 1024, prec)
        B.fot_solve(ctx, g, G, w.eps, w.iters)
        out[name] = B.fot_marginal_error(ctx)[0]
        if name == "mixed":
            split = B.fot_work_split(ctx)
            assert split[2] >= 0.9 * (split[0] + split[1] + split[2]), split   # tensor cores did the work
        ctx.close()
    assert abs(out["mixed"] - out["fp32"]) <= 1e-4, out
