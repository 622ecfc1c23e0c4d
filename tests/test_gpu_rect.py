"""fot_solve_rect (Algorithm 1 between grids of different sizes, dense FP32 passes) against the
FP64 oracle of oracle/rect.py, element by element."""
import numpy as np
import pytest

from oracle import rect
from paper_2512_19072_gb300 import inputs
from fot_testutil import assert_pot_close, f32, solve_rtol, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:invalid value encountered")]


def _amp(rng, shape, kind, zero_frac=0.0):
    n_r, n_c = shape
    if kind == "gauss":
        a = inputs.gauss(n_r, n_c, 0.2 * min(n_r, n_c))
    else:
        a = np.maximum(inputs.disk(n_r, n_c, 0.3 * min(n_r, n_c)), 0.05)
    a = np.asarray(a, dtype=np.float64) * rng.uniform(0.8, 1.2, size=shape)
    a[rng.uniform(size=shape) < zero_frac] = 0.0
    return f32(a)


@pytest.mark.parametrize("shapes", [((40, 50), (56, 36)), ((33, 65), (64, 64)), ((48, 48), (48, 48)),
                                    ((17, 130), (96, 23))])
@pytest.mark.parametrize("eps", [4.0, 25.0])
def test_rect_solve_matches_oracle(fot_lib, shapes, eps):
    B = fot_lib
    (si, so) = shapes
    rng = np.random.default_rng(hash((shapes, eps)) % 2**32)
    g = _amp(rng, si, "gauss", 0.05)
    G = _amp(rng, so, "disk", 0.05)
    iters = 60
    f, psi = B.fot_solve_rect(to_dev(g), to_dev(G), [eps], iters)
    r = rect.fot_iterate_rect(g, G, eps, iters)
    assert_pot_close(to_np(f), r["f"], rtol=solve_rtol(iters), what="f")
    assert_pot_close(to_np(psi), r["psi"], rtol=solve_rtol(iters), what="psi")


def test_rect_schedule_and_marginal(fot_lib):
    """A per-iteration eps schedule; the GPU iterate's column sums equal b (exact after a
    V-update up to FP32 rounding of the potentials)."""
    B = fot_lib
    rng = np.random.default_rng(7)
    g = _amp(rng, (36, 44), "gauss")
    G = _amp(rng, (52, 30), "disk")
    eps = np.geomspace(30.0, 3.0, 40)
    f, psi = B.fot_solve_rect(to_dev(g), to_dev(G), eps, 40)
    r = rect.fot_iterate_rect(g, G, eps, 40)
    assert_pot_close(to_np(f), r["f"], rtol=solve_rtol(40), what="f")
    assert_pot_close(to_np(psi), r["psi"], rtol=solve_rtol(40), what="psi")
    _, cols = rect.marginals_rect(to_np(f), to_np(psi), float(eps[-1]))
    assert np.abs(cols - r["b"]).sum() <= 1e-4


def test_rect_arguments(fot_lib):
    B = fot_lib
    rng = np.random.default_rng(3)
    g = to_dev(_amp(rng, (8, 8), "gauss"))
    with pytest.raises(B.FotError):
        B.fot_solve_rect(g, to_dev(np.zeros((6, 6))), [2.0], 5)            # no target mass
    with pytest.raises(B.FotError):
        B.fot_solve_rect(g, to_dev(_amp(rng, (6, 6), "gauss")), [-1.0], 5)  # eps <= 0
    with pytest.raises(B.FotError):
        B.fot_solve_rect(g, to_dev(_amp(rng, (6, 6), "gauss")), [2.0, 3.0], 5)   # n_eps mismatch


@pytest.mark.parametrize("shapes", [((40, 50), (56, 36)), ((64, 64), (64, 64))])
def test_rect_fp64_reference_matches_oracle(fot_lib, shapes):
    """The FP64 GPU reference form: the oracle's FP64 iterate to ~1e-12 (both compute the same
    sums in double precision; only the order of additions and the library exp / log differ)."""
    import torch
    B = fot_lib
    si, so = shapes
    rng = np.random.default_rng(11)
    g = _amp(rng, si, "gauss", 0.05)
    G = _amp(rng, so, "disk", 0.05)
    eps = [6.0]
    f, psi = B.fot_solve_rect_fp64(torch.from_numpy(g).cuda(), torch.from_numpy(G).cuda(), eps, 50)
    r = rect.fot_iterate_rect(g, G, eps, 50)
    assert_pot_close(f.cpu().numpy(), r["f"], rtol=1e-11, what="f")
    assert_pot_close(psi.cpu().numpy(), r["psi"], rtol=1e-11, what="psi")
