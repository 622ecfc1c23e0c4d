"""Failure detection on the GPU without a fault: the tensor pass's bounded barrier waits.

Every mbarrier wait of the tensor-core kernel gives up after a poll limit, latches
FOT_ETIMEOUT, waits (again bounded) for the copies and MMAs already issued, frees its tensor
memory and returns.  The test-only variable FOT_TEST_WAIT_LIMIT, read when a context is
created, shortens the limit to a few polls without sleeping, so that the first wait on a copy
still in flight runs out.  The call must then fail with FOT_ETIMEOUT (not hang), and a fresh
context on the same device must give the oracle's result."""
import numpy as np
import pytest

from oracle import fot
from paper_2512_19072_gb300 import inputs
from fot_testutil import POT_RTOL, f32, to_dev, to_np

pytestmark = pytest.mark.gpu

N = 256
EPS = 13.1072          # 0.0002 * 256^2 px^2: 16-wide tensor tiles at this size


def _problem():
    rng = np.random.default_rng(77)
    g = f32(inputs.normalise_power(inputs.gauss(N, N, 0.15 * N)))
    G = f32(inputs.normalise_power(inputs.disk(N, N, 0.3 * N)))
    psi = f32(inputs.random_potential(N, N, scale=0.3 * N * N, seed=int(rng.integers(1 << 30))))
    return g, G, psi


def test_wait_limit_runs_out_then_context_recovers(fot_lib, monkeypatch):
    B = fot_lib
    g, G, psi = _problem()
    monkeypatch.setenv("FOT_TEST_WAIT_LIMIT", "1")
    short = B.fot_create(N, N, B.FOT_MIXED)
    monkeypatch.delenv("FOT_TEST_WAIT_LIMIT")
    B.fot_set_problem(short, to_dev(g), to_dev(G))
    with pytest.raises(B.FotError) as err:
        B.fot_u_update(short, to_dev(psi), EPS)
        B.fot_sync(short)
    assert B.STATUS[err.value.status] == "FOT_ETIMEOUT"
    short.close()

    # the device is usable and a context with the normal limit computes the right result
    ctx = B.fot_create(N, N, B.FOT_MIXED)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    f_gpu = to_np(B.fot_u_update(ctx, to_dev(psi), EPS))
    B.fot_sync(ctx)
    _, tensor_terms = B.fot_work_count(ctx, tensor=True)
    assert tensor_terms > 0                      # the tensor kernel did the work
    ctx.close()
    f_ref, _ = fot.u_update(psi, fot.log0(fot.marginal(g)), EPS)
    fin = np.isfinite(f_ref)
    assert np.array_equal(np.isneginf(f_gpu), np.isneginf(f_ref))
    err = np.abs(f_gpu[fin] - f_ref[fin]).max()
    # split-BF16 bound of the mixed form (2^-15 eps per half-step) plus FP32 rounding
    assert err <= POT_RTOL * np.abs(f_ref[fin]).max() + 2.0 ** -15 * EPS, err
