"""cFOT (Sec. 3.1) through the C ABI against the oracle's cfot_iterate (FP64 linear
convolutions) on the same FP32 inputs, on beams over a flat floor: the regime where an
exponential-domain FP32 iteration holds its accuracy."""
import math

import numpy as np
import pytest

from oracle import fot
from fot_testutil import f32, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:divide by zero")]


def _beam(n_r, n_c, cy, cx, s, floor):
    j = np.arange(n_r)[:, None]
    k = np.arange(n_c)[None, :]
    return f32(np.exp(-((j - cy) ** 2 + (k - cx) ** 2) / (2 * s * s)) + floor)


def _fft_eps(n):
    """Normwise error of one FP32 radix-2 FFT of the padded length P >= 2n - 1 (7 log2(P)
    2^-24, the standard floating-point FFT bound) plus the rounding of the stored spectrum."""
    P = 1
    while P < 2 * n - 1:
        P *= 2
    return 7 * math.log2(P) * 2.0 ** -24 + 2.0 ** -24


def _conv_rel_error(x, eps):
    """Bound on the relative error of every entry of lambda * x * lambda computed as the GPU
    does (rows, then columns, each by a forward FFT, the product with lambda's spectrum and an
    inverse FFT): per line ||dy||_inf <= e (sum(lambda) ||x_line||_2 + ||y_line||_2), divided by
    each entry of y; the two passes add."""
    n_r, n_c = x.shape
    lam_c = np.exp(-np.arange(-(n_c - 1), n_c) ** 2 / (2 * eps))
    lam_r = np.exp(-np.arange(-(n_r - 1), n_r) ** 2 / (2 * eps))
    Y = np.stack([np.convolve(x[j], lam_c)[n_c - 1:2 * n_c - 1] for j in range(n_r)])
    Z = np.stack([np.convolve(Y[:, k], lam_r)[n_r - 1:2 * n_r - 1] for k in range(n_c)], 1)
    dY = np.array([_fft_eps(n_c) * (lam_c.sum() * np.linalg.norm(x[j]) + np.linalg.norm(Y[j]))
                   for j in range(n_r)])
    dZ = np.array([_fft_eps(n_r) * (lam_r.sum() * np.linalg.norm(Y[:, k]) + np.linalg.norm(Z[:, k]))
                   for k in range(n_c)])
    return (dY[:, None] / Y).max() + (dZ[None, :] / Z).max()


@pytest.mark.parametrize("shape,eps,iters", [((32, 32), 200.0, 10), ((32, 32), 60.0, 10),
                                             ((16, 64), 100.0, 10), ((64, 64), 300.0, 8)])
def test_cfot_matches_oracle(fot_lib, shape, eps, iters):
    B = fot_lib
    n_r, n_c = shape
    g = _beam(n_r, n_c, 0.45 * n_r, 0.55 * n_c, n_r / 5, 1.0)
    G = _beam(n_r, n_c, 0.55 * n_r, 0.40 * n_c, n_r / 4, 1.0)
    u, V, S = fot.cfot_iterate(g, G, eps, iters)
    # the largest per-half-step log error over the whole run (each half-step's own input)
    d = 0.0
    for t in range(1, iters + 1):
        ut, Vt, _ = fot.cfot_iterate(g, G, eps, t)
        d = max(d, _conv_rel_error(ut, eps), _conv_rel_error(Vt, eps))
    Vprev = fot.cfot_iterate(g, G, eps, iters - 1)[1] if iters > 1 else np.full(shape, 1.0 / (n_r * n_c))
    d = max(d, _conv_rel_error(Vprev, eps), _conv_rel_error(np.full(shape, 1.0 / (n_r * n_c)), eps))
    # each half-step is 1-Lipschitz in the sup norm of the log values, so errors add: its
    # convolution's d, the FP32 log marginal (2^-24 |log a|) and the exp / division (2 ulp);
    # then the final eps log u (2^-24 |log u|)
    a, b = fot.marginal(g), fot.marginal(G)
    lm = max(np.abs(np.log(a)).max(), np.abs(np.log(b)).max())
    lu = max(np.abs(np.log(u)).max(), np.abs(np.log(V)).max())
    bound = 2 * iters * (d + 2.0 ** -24 * (lm + 4)) + 2.0 ** -24 * (lu + 1)
    ctx = B.fot_create(n_r, n_c)
    B.fot_cfot_solve(ctx, to_dev(g), to_dev(G), eps, iters)
    f, psi = B.fot_potentials(ctx)
    assert np.abs(to_np(f) - eps * np.log(u)).max() <= eps * bound
    assert np.abs(to_np(psi) - eps * np.log(V)).max() <= eps * bound
    assert bound < 1e-2                                      # the comparison is not vacuous
    phi, _, _ = B.fot_phase(ctx)                             # the phase step applies
    assert np.isfinite(to_np(phi)).all()
    ctx.close()


def test_cfot_errors_and_instability(fot_lib):
    B = fot_lib
    g = _beam(16, 16, 7, 8, 3, 0.2)
    G = _beam(16, 16, 8, 7, 4, 0.2)
    ctx = B.fot_create(16, 16)
    with pytest.raises(B.FotError) as e:
        B.fot_cfot_solve(ctx, to_dev(g), to_dev(G), 10.0, 0)
    assert e.value.status == 1                           # FOT_EINVAL: no iteration
    B.fot_cfot_solve(ctx, to_dev(g), to_dev(G), 10.0, 3)
    with pytest.raises(B.FotError) as e:                 # no schedule recorded for the adjoint
        B.fot_backward(ctx, to_dev(g), to_dev(G), dL_dphi=ctx.empty().zero_())
    assert e.value.status == 8                           # FOT_ESTATE
    # a one-pixel target at eps 0.01 px^2: after the first V-half, V is zero but at that pixel,
    # and lambda * V * lambda (a delta through an FFT round trip) is rounding noise of both
    # signs, or zero, at every other pixel, where the source has mass: the iteration has left
    # what FP32 represents, and the convolution reports it
    G2 = np.zeros((16, 16))
    G2[8, 8] = 1.0
    B.fot_cfot_solve(ctx, to_dev(g), to_dev(G2), 0.01, 3)
    with pytest.raises(B.FotError) as e:
        B.fot_sync(ctx)
    assert e.value.status == 4                           # FOT_ENONFINITE
    ctx.close()
    ctx = B.fot_create(2, 3000)
    with pytest.raises(B.FotError) as e:
        B.fot_cfot_solve(ctx, to_dev(np.ones((2, 3000))), to_dev(np.ones((2, 3000))), 10.0, 2)
    assert e.value.status == 7                           # FOT_EUNSUPPORTED: FFT length > 4096
    ctx.close()
