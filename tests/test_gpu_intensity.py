"""L1 intensity loss of a phase solution (Sec. 5) through the C ABI, against the oracle's
intensity_loss (the centred 2-D DFT written with DFT matrices) on the same FP32 inputs."""
import math

import numpy as np
import pytest

from oracle import fot
from paper_2512_19072_gb300 import inputs
from fot_testutil import f32, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:divide by zero")]


def _bound(shape, g):
    """Bound on |loss_gpu - loss| (and on every |I_gpu - I|).  A radix-2 FFT in FP32 with
    twiddles good to an ulp has a normwise error below 7 log2(n) 2^-24 per 1-D transform (the
    standard floating-point FFT bound); the 2-D transform adds the two, and the input field
    e^{log a / 2 + 2 pi i phi} carries 2^-24 (|log a|/2 + 4) relative error.  With e_X that total,
    sum |dI| <= (2 e_X + e_X^2) P, and dividing by a P with the same error doubles it."""
    a = g ** 2 / (g ** 2).sum()
    la = np.abs(np.log(a[a > 0])).max()
    ex = 7 * math.log2(shape[0] * shape[1]) * 2.0 ** -24 + 2.0 ** -24 * (la / 2 + 4)
    return 2 * (2 * ex + ex * ex)


@pytest.mark.parametrize("shape", [(2, 2), (8, 8), (16, 64), (128, 32), (256, 256), (1024, 1024)])
def test_intensity_loss_matches_oracle(fot_lib, shape):
    B = fot_lib
    rng = np.random.default_rng(31)
    g = f32(rng.uniform(0.0, 1.0, shape))
    g[rng.uniform(size=shape) < 0.1] = 0.0
    g[0, 0] = 0.5
    G = f32(rng.uniform(0.0, 1.0, shape))
    phi = f32(rng.normal(0.0, 3.0, shape))
    ctx = B.fot_create(*shape)
    B.fot_set_problem(ctx, to_dev(g), to_dev(G))
    loss, inten = B.fot_intensity_loss(ctx, to_dev(phi), with_intensity=True)
    ref, iref = fot.intensity_loss(g, phi, G)
    tol = _bound(shape, g)
    assert abs(loss - ref) <= tol, (loss, ref, tol)
    assert np.abs(to_np(inten) - iref).max() <= tol
    assert abs(to_np(inten).sum() - 1.0) <= 1e-5
    ctx.close()


def test_intensity_loss_of_a_solved_phase(fot_lib):
    """The phase fot_phase returns for the 64^2 workload, evaluated by both sides."""
    B = fot_lib
    w = inputs.config1()
    g, G = f32(w.g), f32(w.G)
    ctx = B.fot_create(64, 64)
    B.fot_solve(ctx, to_dev(g), to_dev(G), w.eps, w.iters)
    phi, _, _ = B.fot_phase(ctx)
    loss = B.fot_intensity_loss(ctx, phi)
    ref, _ = fot.intensity_loss(g, to_np(phi), G)
    assert abs(loss - ref) <= _bound((64, 64), g), (loss, ref)
    assert 0.0 < loss < 2.0
    ctx.close()


def test_plane_wave_and_errors(fot_lib):
    B = fot_lib
    n = 64
    j = np.arange(n) - n // 2
    ctx = B.fot_create(n, n)
    for L0, M0 in ((5, -9), (-32, 31)):
        G = np.zeros((n, n))
        G[L0 + n // 2, M0 + n // 2] = 1.0
        B.fot_set_problem(ctx, to_dev(np.ones((n, n))), to_dev(G))
        phi = np.add.outer(j * L0, j * M0) / n          # x . X0 in cycles (exact in FP32)
        loss, inten = B.fot_intensity_loss(ctx, to_dev(phi), with_intensity=True)
        assert loss <= _bound((n, n), np.ones((n, n))), loss        # no sidelobes up to rounding
        assert abs(to_np(inten)[L0 + n // 2, M0 + n // 2] - 1.0) < 1e-4
    with pytest.raises(B.FotError) as e:
        B.fot_intensity_loss(ctx, None)
    assert e.value.status == 1                           # FOT_EINVAL
    ctx.close()
    ctx = B.fot_create(12, 16)
    with pytest.raises(B.FotError) as e:
        B.fot_intensity_loss(ctx, to_dev(np.zeros((12, 16))))
    assert e.value.status == 8                           # FOT_ESTATE: no problem loaded
    B.fot_set_problem(ctx, to_dev(np.ones((12, 16))), to_dev(np.ones((12, 16))))
    with pytest.raises(B.FotError) as e:
        B.fot_intensity_loss(ctx, to_dev(np.zeros((12, 16))))
    assert e.value.status == 7                           # FOT_EUNSUPPORTED: 12 rows
    ctx.close()
