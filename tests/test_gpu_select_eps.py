"""Automatic eps selection (fot_select_eps): the smallest candidate whose probe stays finite and
reduces the marginal violation by the requested fraction.  The rule is replayed through the
public entry points (fot_solve_tol measures the same violation after a fixed number of
iterations when its tolerance is 0)."""
import numpy as np
import pytest

from paper_2512_19072_gb300 import inputs
from fot_testutil import f32, to_dev

pytestmark = pytest.mark.gpu

N = 128


def _problem():
    w = inputs.config3(N)
    return to_dev(f32(w.g)), to_dev(f32(w.G))


def test_select_eps_fot_follows_its_rule(fot_lib):
    B = fot_lib
    g, G = _problem()
    cand = [2e-5, 5e-5, 1e-4, 2e-4, 5e-4, 1e-3]          # paper units (eps_px = n^2 eps)
    probe, check, dec = 60, 20, 0.3
    ctx = B.fot_create(N, N, B.FOT_MIXED)
    idx, tv = B.fot_select_eps(ctx, g, G, cand, probe, check, min_decrease=dec,
                               eps_units=B.FOT_EPS_PAPER)

    def violations(e):
        _, t1 = B.fot_solve_tol(ctx, g, G, [e], check, 0.0, check, eps_units=B.FOT_EPS_PAPER)
        _, t2 = B.fot_solve_tol(ctx, g, G, [e], probe, 0.0, probe, eps_units=B.FOT_EPS_PAPER)
        return t1, t2

    tvs = [violations(e) for e in cand]
    stable = [t2 <= (1 - dec) * t1 for t1, t2 in tvs]
    expect = next((i for i, s in enumerate(stable) if s), -1)
    assert idx == expect, (idx, tvs)
    assert idx >= 0                                        # some candidate converges here
    assert tv == pytest.approx(tvs[idx][1], rel=1e-9)
    ctx.close()


def test_select_eps_cfot_rejects_unstable_small_eps(fot_lib):
    """cFOT iterates in the FP32 exponential domain: at small eps u and V leave its range (the
    instability Sec. 5 describes), so the selection must skip those candidates."""
    B = fot_lib
    g, G = _problem()
    cand = [0.25, 1.0, 4.0, 16.0, 64.0, 256.0]             # px^2
    probe, check, dec = 40, 10, 0.05
    ctx = B.fot_create(N, N, B.FOT_FP32)
    idx, _ = B.fot_select_eps(ctx, g, G, cand, probe, check, min_decrease=dec, use_cfot=True)
    assert idx >= 0
    B.fot_cfot_solve(ctx, g, G, [cand[idx]], probe)        # the chosen eps runs through
    l1, _ = B.fot_marginal_error(ctx)
    assert np.isfinite(l1)
    smaller = [e for e in cand if e < cand[idx]]
    for e in smaller:
        # each smaller candidate fails: non-finite within the probe, or too little progress
        try:
            B.fot_cfot_solve(ctx, g, G, [e], check)
            l1_a, _ = B.fot_marginal_error(ctx)
            B.fot_cfot_solve(ctx, g, G, [e], probe)
            l1_b, _ = B.fot_marginal_error(ctx)
            assert not (l1_b <= (1 - dec) * l1_a * (1 - 1e-3)), (e, l1_a, l1_b)
        except B.FotError as err:
            assert B.STATUS[err.status] == "FOT_ENONFINITE", err
    ctx.close()


def test_select_eps_arguments(fot_lib):
    B = fot_lib
    g, G = _problem()
    ctx = B.fot_create(N, N)
    with pytest.raises(B.FotError):
        B.fot_select_eps(ctx, g, G, [1.0, -2.0], 40, 10)   # a candidate <= 0
    with pytest.raises(B.FotError):
        B.fot_select_eps(ctx, g, G, [1.0], 10, 10)         # probe not longer than the first part
    with pytest.raises(B.FotError):
        B.fot_select_eps(ctx, g, G, [1.0], 40, 10, min_decrease=1.0)
    ctx.close()
