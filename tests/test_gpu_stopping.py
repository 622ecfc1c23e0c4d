"""Convergence stop (Sec. 3: total variation of the marginal violation) through the C ABI,
against the oracle's fot_iterate_tol on the same seeded inputs.

The tolerances sit between the oracle's violations at two consecutive checks, with a margin
far above the FP32 (and split-BF16) error of the measured violation, so the iteration count
where the GPU stops is compared exactly.
"""
import numpy as np
import pytest

from oracle import fot
from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, assert_pot_close, f32, solve_rtol, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:invalid value encountered")]

K = 5            # iterations between checks


def _c1():
    w = inputs.config1()
    return f32(w.g), f32(w.G)


def _check_violations(g, G, eps, iters, k):
    """The oracle's violation of the iterate at every check (iterations k, 2k, ...)."""
    a = fot.marginal(g)
    out = []

    def rec(t, stage, f, psi, e):
        if stage == "v" and (t + 1) % k == 0:
            out.append(fot.source_violation(f, psi, a, e))
    fot.fot_iterate(g, G, eps, iters, record=rec)
    return out


def _pot_errors(r, eps, iters, mixed):
    """Bounds on |f_gpu - f| and |psi_gpu - psi| after `iters` iterations: the FP32 solve bound,
    or for the mixed form 2 iters half-steps of POT_RTOL |pot| + 2^-15 eps each (every
    half-step is 1-Lipschitz in the sup norm, so per-step errors add up)."""
    fmax = np.abs(r["f"][np.isfinite(r["f"])]).max()
    pmax = np.abs(r["psi"][np.isfinite(r["psi"])]).max()
    if not mixed:
        return solve_rtol(iters) * fmax, solve_rtol(iters) * pmax
    return (2 * iters * (POT_RTOL * fmax + 2.0 ** -15 * eps),
            2 * iters * (POT_RTOL * pmax + 2.0 ** -15 * eps))


def _tv_bound(r, eps, iters, mixed):
    """Bound on |tv_gpu - tv|: every row sum exp(f/eps + S(psi)) carries a log error of at most
    d = (df + dpsi)/eps plus the FP32 rounding of f/eps and S (and for the mixed form the
    2^-15 eps of its extra u-half), so the violation moves by at most (1 + tv)(e^d - 1)."""
    df, dp = _pot_errors(r, eps, iters, mixed)
    S = fot.log_kernel_apply(r["psi"], eps)
    lmax = np.abs(r["f"][np.isfinite(r["f"])]).max() / eps + np.abs(S[np.isfinite(S)]).max()
    d = (df + dp) / eps + 4 * 2.0 ** -24 * lmax + (2.0 ** -15 if mixed else 0.0)
    return (1.0 + r["tv"]) * np.expm1(d)


@pytest.mark.parametrize("form,eps,i", [("fp32", 1.0, 4), ("mixed", 12.0, 1)])
def test_stop_matches_oracle(fot_lib, form, eps, i):
    """eps 1: the banded FP32 passes; eps 12: 16-wide tensor tiles (mixed form).  The stop
    is set between the checks i - 1 and i."""
    B = fot_lib
    g, G = _c1()
    tvs = _check_violations(g, G, eps, (i + 1) * K, K)
    assert tvs[i] < tvs[i - 1] / 1.1
    tol = (tvs[i - 1] * tvs[i]) ** 0.5
    r = fot.fot_iterate_tol(g, G, eps, 60, tol, K)
    assert r["iters"] == (i + 1) * K
    ctx = B.fot_create(64, 64, B.FOT_FP32 if form == "fp32" else B.FOT_MIXED)
    iters, tv = B.fot_solve_tol(ctx, to_dev(g), to_dev(G), eps, 60, tol, K)
    assert iters == r["iters"]
    mixed = form == "mixed"
    bound = _tv_bound(r, eps, iters, mixed)
    assert bound < min(tvs[i - 1] - tol, tol - tvs[i])       # the stop cannot move
    assert abs(tv - r["tv"]) <= bound, (tv, r["tv"], bound)
    f, psi = B.fot_potentials(ctx)
    df, dp = _pot_errors(r, eps, iters, mixed)
    for gpu, ref, d, what in ((f, r["f"], df, "f"), (psi, r["psi"], dp, "psi")):
        gpu = to_np(gpu)
        assert np.array_equal(np.isneginf(gpu), np.isneginf(ref)), what
        fin = np.isfinite(ref)
        assert np.abs(gpu[fin] - ref[fin]).max() <= d, what
    ctx.close()


def test_stop_edges_and_schedule(fot_lib):
    B = fot_lib
    g, G = _c1()
    ctx = B.fot_create(64, 64)
    # tol 0: every check runs, the last after max_iters (a partial block of 3)
    iters, tv = B.fot_solve_tol(ctx, to_dev(g), to_dev(G), 1.0, 23, 0.0, K)
    r = fot.fot_iterate_tol(g, G, 1.0, 23, 0.0, K)
    assert iters == 23 == r["iters"]
    assert abs(tv - r["tv"]) <= _tv_bound(r, 1.0, 23, False)
    f, _ = B.fot_potentials(ctx)
    assert_pot_close(to_np(f), r["f"], rtol=solve_rtol(23), what="f")
    # a loose tolerance stops at the first check; check_every beyond max_iters checks once
    assert B.fot_solve_tol(ctx, to_dev(g), to_dev(G), 1.0, 60, 10.0, K)[0] == K
    assert B.fot_solve_tol(ctx, to_dev(g), to_dev(G), 1.0, 7, 0.0, 100)[0] == 7
    # an annealing schedule (one eps per iteration): stop and state as the oracle's
    sched = list(np.geomspace(4.0, 1.0, 30))
    r = fot.fot_iterate_tol(g, G, sched, 30, 0.3, K)
    iters, tv = B.fot_solve_tol(ctx, to_dev(g), to_dev(G), sched, 30, 0.3, K)
    assert iters == r["iters"] == 10
    f, psi = B.fot_potentials(ctx)
    assert_pot_close(to_np(psi), r["psi"], rtol=solve_rtol(iters), what="psi")
    # argument errors are reported before any work (FOT_EINVAL)
    for args in ((1.0, 10, -1.0, K), (1.0, 10, float("nan"), K), (1.0, 10, 0.1, 0),
                 (1.0, 0, 0.1, K), ([1.0, 2.0], 10, 0.1, K)):
        with pytest.raises(B.FotError) as e:
            B.fot_solve_tol(ctx, to_dev(g), to_dev(G), *args)
        assert e.value.status == 1
    ctx.close()
