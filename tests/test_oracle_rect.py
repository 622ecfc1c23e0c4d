"""Pins of the unequal-grid oracle (oracle/rect.py), CPU only."""
import numpy as np

from oracle import fot, rect


def _amps(rng, shape, zero_frac=0.1):
    a = rng.uniform(0.05, 1.0, size=shape)
    a[rng.uniform(size=shape) < zero_frac] = 0.0
    return a


def test_p16a_separable_equals_dense_four_index():
    rng = np.random.default_rng(16)
    pot = rng.normal(size=(5, 7)) * 3.0
    pot[1, 2] = -np.inf
    for out_shape in [(6, 4), (3, 9), (5, 7)]:
        for eps in (0.7, 4.0):
            s = rect.log_kernel_apply_rect(pot, eps, out_shape)
            d = rect.log_kernel_apply_rect_dense(pot, eps, out_shape)
            assert np.allclose(s, d, rtol=1e-12, atol=1e-12)


def test_p16b_equal_grids_reduce_to_the_square_oracle():
    rng = np.random.default_rng(17)
    g, G = _amps(rng, (9, 11)), _amps(rng, (9, 11))
    r = rect.fot_iterate_rect(g, G, 3.0, 12)
    q = fot.fot_iterate(g, G, 3.0, 12)
    for k in ("f", "psi", "S_last"):
        fin = np.isfinite(q[k])
        assert np.array_equal(fin, np.isfinite(r[k]))
        assert np.allclose(r[k][fin], q[k][fin], rtol=1e-12, atol=1e-9)


def test_p16c_marginals_and_convergence_on_unequal_grids():
    rng = np.random.default_rng(18)
    g, G = _amps(rng, (7, 10)), _amps(rng, (12, 6))
    eps = 6.0
    l1 = []
    for T in (5, 20, 80):
        r = rect.fot_iterate_rect(g, G, eps, T)
        rows, cols = rect.marginals_rect(r["f"], r["psi"], eps)
        assert np.allclose(cols, r["b"], rtol=1e-12, atol=1e-15)   # exact after a V-update
        l1.append(np.abs(rows - r["a"]).sum())
    assert l1[0] > l1[1] > l1[2] and l1[2] < 1e-3 * max(l1[0], 1e-12) + 1e-9


def test_p16d_dense_iterate_equals_separable_iterate():
    rng = np.random.default_rng(19)
    g, G = _amps(rng, (4, 5)), _amps(rng, (6, 3))
    r = rect.fot_iterate_rect(g, G, [5.0, 3.0, 2.0], 3)
    d = rect.fot_iterate_rect(g, G, [5.0, 3.0, 2.0], 3, dense=True)
    for k in ("f", "psi"):
        fin = np.isfinite(d[k])
        assert np.allclose(r[k][fin], d[k][fin], rtol=1e-12, atol=1e-10)


def test_p16e_transposing_both_planes_transposes_the_potentials():
    rng = np.random.default_rng(20)
    g, G = _amps(rng, (6, 9)), _amps(rng, (10, 5))
    r = rect.fot_iterate_rect(g, G, 4.0, 15)
    t = rect.fot_iterate_rect(g.T, G.T, 4.0, 15)
    for k in ("f", "psi"):
        fin = np.isfinite(r[k])
        assert np.allclose(t[k].T[fin], r[k][fin], rtol=1e-12, atol=1e-9)
