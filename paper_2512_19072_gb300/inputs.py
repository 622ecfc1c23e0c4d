"""Seeded synthetic beam-shaping workloads.

This module only builds input and target amplitude images (and the scalar
schedules that go with them). It holds none of the transport arithmetic, so
both the FP64 oracle tests and the CUDA path may draw their inputs from it.

The paper's own images (the two-Gaussian beam and composite target of Fig. 1,
the targets of Fig. 4) are not published; these generators stand in for them
with the same kind of content: smooth Gaussian input beams and flat-top
targets (rectangles, disks, rings) with smoothed edges and zero background.

Amplitude primitives live on the pixel grid (j, k), centre c = floor(n/2):
  gauss(sigma, dj, dk) = exp(-((j-c-dj)^2 + (k-c-dk)^2) / (2 sigma^2))
  edge(d) = 1 (d <= 0), (1 + cos(pi d / 2)) / 2 (0 < d < 2), 0 (d >= 2)
with d the signed distance to a shape boundary (2-px cosine edge).
Every image is normalised to unit power, sum(amp^2) = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "gauss", "disk", "ring", "rect", "normalise_power",
    "config1", "config2", "config3", "config4", "config5",
    "separable_workload", "gaussian_pair", "random_potential", "geometric_eps",
]


@dataclass
class Workload:
    """One beam-shaping problem: amplitudes g (input plane) and G (target plane)."""
    name: str
    g: np.ndarray
    G: np.ndarray
    eps: np.ndarray          # per-iteration entropic parameter, px^2 (len == iters)
    iters: int
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.g.shape


def _grid(n_r: int, n_c: int):
    j = np.arange(n_r, dtype=np.float64)[:, None] - (n_r // 2)
    k = np.arange(n_c, dtype=np.float64)[None, :] - (n_c // 2)
    return j, k


def _edge(d):
    d = np.asarray(d, dtype=np.float64)
    out = np.where(d <= 0.0, 1.0, 0.0)
    mid = (d > 0.0) & (d < 2.0)
    return np.where(mid, 0.5 * (1.0 + np.cos(np.pi * d / 2.0)), out)


def gauss(n_r, n_c, sigma, dj=0.0, dk=0.0):
    j, k = _grid(n_r, n_c)
    return np.exp(-((j - dj) ** 2 + (k - dk) ** 2) / (2.0 * sigma * sigma))


def disk(n_r, n_c, R, cj=0.0, ck=0.0):
    j, k = _grid(n_r, n_c)
    r = np.sqrt((j - cj) ** 2 + (k - ck) ** 2)
    return _edge(r - R)


def ring(n_r, n_c, R, W, cj=0.0, ck=0.0):
    j, k = _grid(n_r, n_c)
    r = np.sqrt((j - cj) ** 2 + (k - ck) ** 2)
    return _edge(np.abs(r - R) - W / 2.0)


def rect(n_r, n_c, hj, hk, cj=0.0, ck=0.0):
    j, k = _grid(n_r, n_c)
    return _edge(np.maximum(np.abs(j - cj) - hj, np.abs(k - ck) - hk))


def normalise_power(a):
    a = np.asarray(a, dtype=np.float64)
    return a / math.sqrt(float((a * a).sum()))


def geometric_eps(eps_start, eps_end, iters):
    """eps_t = eps_s (eps_e/eps_s)^(t/(T-1)); both half-steps of iteration t use eps_t."""
    if iters == 1:
        return np.array([float(eps_start)])
    t = np.arange(iters, dtype=np.float64)
    return eps_start * (eps_end / eps_start) ** (t / (iters - 1))


def _two_gauss(n, rng, scale):
    d = rng.uniform(-4.0, 4.0, size=4) * scale
    return (0.6 * gauss(n, n, 40.0 * scale, 20.0 * scale + d[0], d[1])
            + 0.4 * gauss(n, n, 25.0 * scale, -20.0 * scale + d[2], d[3]))


def config1():
    """64x64: Gaussian (sigma 10 px) -> flat-top disk R = 20 px, eps 1 px^2, 200 iterations."""
    n = 64
    g = normalise_power(gauss(n, n, 10.0))
    G = normalise_power(disk(n, n, 20.0))
    T = 200
    return Workload("c1_64_gauss_to_disk", g, G, np.full(T, 1.0), T)


def _c2_target(n, rng, scale, pedestal=True):
    shapes = []
    for _ in range(4):
        hj, hk = rng.uniform(8.0, 30.0, size=2) * scale
        cj, ck = rng.uniform(-80.0, 80.0, size=2) * scale
        shapes.append(rect(n, n, hj, hk, cj, ck))
    for _ in range(2):
        R = rng.uniform(20.0, 60.0) * scale
        W = rng.uniform(4.0, 8.0) * scale
        cj, ck = rng.uniform(-80.0, 80.0, size=2) * scale
        shapes.append(ring(n, n, R, W, cj, ck))
    G = np.max(np.stack(shapes), axis=0)
    if pedestal:
        # 0.02 amplitude pedestal everywhere except an exactly-zero 7-px frame
        frame = int(round(7 * scale))
        ped = np.full((n, n), 0.02)
        ped[:frame, :] = 0.0
        ped[-frame:, :] = 0.0
        ped[:, :frame] = 0.0
        ped[:, -frame:] = 0.0
        G = np.maximum(G, ped)
        G[ped == 0.0] = 0.0
    return G


def config2(n=256, iters=300):
    """256x256: two-Gaussian input, 4 rectangles + 2 rings target, eps 64 -> 1 px^2 over 300 its."""
    rng = np.random.default_rng(2)
    scale = n / 256.0
    g = normalise_power(_two_gauss(n, rng, scale))
    G = normalise_power(_c2_target(n, rng, scale))
    return Workload(f"c2_{n}_twogauss_to_rects_rings", g, G,
                    geometric_eps(64.0 * scale * scale, 1.0 * scale * scale, iters), iters)


def _c3_shapes(n, rng, scale):
    specs = []
    for i in range(12):
        kind = ("rect", "disk", "ring")[i % 3]
        cj, ck = rng.uniform(-80.0, 80.0, size=2) * scale * 1.6
        if kind == "rect":
            specs.append((kind, rng.uniform(8.0, 30.0, size=2) * scale, cj, ck))
        elif kind == "disk":
            specs.append((kind, rng.uniform(20.0, 45.0) * scale, cj, ck))
        else:
            specs.append((kind, (rng.uniform(20.0, 60.0) * scale, rng.uniform(4.0, 8.0) * scale), cj, ck))
    return specs


def _c3_render(n, specs, s, f=1.0):
    """Render the shapes on an n x n grid with sizes times s; f rescales every length
    (positions included) to render the same composite at another resolution."""
    out = np.zeros((n, n))
    for kind, p, cj, ck in specs:
        if kind == "rect":
            img = rect(n, n, p[0] * s * f, p[1] * s * f, cj * f, ck * f)
        elif kind == "disk":
            img = disk(n, n, p * s * f, cj * f, ck * f)
        else:
            img = ring(n, n, p[0] * s * f, p[1] * s * f, cj * f, ck * f)
        out = np.maximum(out, img)
    return out


def config3(n=1024, iters=200, eps_paper=2e-4):
    """n x n (1024 or 2048; 256 for the downsampled oracle case): two-Gaussian beam scaled by n/256,
    target = 12 seeded flat-tops/disks/rings whose sizes are bisected to ~30% coverage.
    Fixed eps = eps_paper * n^2 px^2 (the paper's working value 0.0002), 200 iterations."""
    rng = np.random.default_rng(3)
    scale = n / 256.0
    g = normalise_power(_two_gauss(n, rng, scale))
    specs = _c3_shapes(n, rng, scale)
    nb = min(n, 256)                          # bisect the size factor on a coarse copy
    lo, hi = 0.2, 4.0
    for _ in range(24):
        mid = 0.5 * (lo + hi)
        cov = float((_c3_render(nb, specs, mid, nb / n) > 0).mean())
        if cov < 0.30:
            lo = mid
        else:
            hi = mid
    if nb < n:                                # refine at full resolution (edges are 2 px)
        lo, hi = 0.5 * (lo + hi), 0.5 * (lo + hi) * 1.6
        for _ in range(10):
            mid = 0.5 * (lo + hi)
            if float((_c3_render(n, specs, mid) > 0).mean()) < 0.30:
                lo = mid
            else:
                hi = mid
    G = normalise_power(_c3_render(n, specs, 0.5 * (lo + hi)))
    eps = eps_paper * n * n
    return Workload(f"c3_{n}_twogauss_to_12shapes", g, G, np.full(iters, eps), iters,
                    extra={"coverage": float((G > 0).mean()), "eps_paper": eps_paper})


def config4(n=512, iters=100):
    """512x512 backward case: config-2 construction scaled x2, eps 4 px^2, 100 iterations,
    loss weights w ~ U[0,1] and a smooth Legendre target phase."""
    rng = np.random.default_rng(4)
    scale = n / 256.0
    g = normalise_power(_two_gauss(n, rng, scale))
    G = normalise_power(_c2_target(n, rng, scale))
    w = rng.uniform(0.0, 1.0, size=(n, n))
    x = np.linspace(-1.0, 1.0, n)
    P = [np.ones_like(x), x, 0.5 * (3 * x * x - 1), 0.5 * (5 * x ** 3 - 3 * x)]
    phi_t = np.zeros((n, n))
    for p in range(4):
        for q in range(4 - p):
            phi_t += rng.normal(0.0, 0.1) * P[p][:, None] * P[q][None, :]
    return Workload(f"c4_{n}_backward", g, G, np.full(iters, 4.0), iters,
                    extra={"w": w, "phi_target": phi_t, "checkpoint": 10})


def config5(count=64, iters=200):
    """64 independent problems, n_i ~ U{128,192,256,384,512}; Gaussian or two-Gaussian inputs,
    2-6 seeded shapes per target, eps geometric 32 -> 1 px^2 over 200 iterations."""
    rng = np.random.default_rng(5)
    sizes = rng.choice([128, 192, 256, 384, 512], size=count)
    out = []
    for i, n in enumerate(sizes):
        n = int(n)
        scale = n / 256.0
        if rng.uniform() < 0.5:
            g = gauss(n, n, 40.0 * scale, *(rng.uniform(-4, 4, size=2) * scale))
        else:
            g = _two_gauss(n, rng, scale)
        shapes = []
        for s in range(int(rng.integers(2, 7))):
            kind = s % 3
            cj, ck = rng.uniform(-60.0, 60.0, size=2) * scale
            if kind == 0:
                shapes.append(rect(n, n, *(rng.uniform(8.0, 30.0, size=2) * scale), cj, ck))
            elif kind == 1:
                shapes.append(disk(n, n, rng.uniform(15.0, 40.0) * scale, cj, ck))
            else:
                shapes.append(ring(n, n, rng.uniform(20.0, 50.0) * scale,
                                   rng.uniform(4.0, 8.0) * scale, cj, ck))
        G = np.max(np.stack(shapes), axis=0)
        out.append(Workload(f"c5_{i}_{n}", normalise_power(g), normalise_power(G),
                            geometric_eps(32.0, 1.0, iters), iters))
    return out


def separable_workload(n_r, n_c, eps, iters, seed=11):
    """Product-form input and target, g = p(j) q(k), G = r(L) s(M): the 2-D iterate then splits
    into two 1-D iterates, which gives a full-size elementwise check."""
    rng = np.random.default_rng(seed)

    def prof1d(n, sig, off):
        x = np.arange(n, dtype=np.float64) - n // 2
        return 0.6 * np.exp(-((x - off) ** 2) / (2 * sig * sig)) + 0.4 * np.exp(-((x + off) ** 2) / (2 * (0.6 * sig) ** 2))

    def flat1d(n, parts):
        x = np.arange(n, dtype=np.float64) - n // 2
        out = np.zeros(n)
        for c, h in parts:
            out = np.maximum(out, _edge(np.abs(x - c) - h))
        return out

    p = prof1d(n_r, n_r / 6.4, n_r / 12.8 + rng.uniform(-2, 2))
    q = prof1d(n_c, n_c / 6.4, n_c / 12.8 + rng.uniform(-2, 2))
    r = flat1d(n_r, [(rng.uniform(-0.25, 0.25) * n_r, rng.uniform(0.04, 0.12) * n_r) for _ in range(3)])
    s = flat1d(n_c, [(rng.uniform(-0.25, 0.25) * n_c, rng.uniform(0.04, 0.12) * n_c) for _ in range(3)])
    g = normalise_power(np.outer(p, q))
    G = normalise_power(np.outer(r, s))
    eps_arr = np.full(iters, float(eps)) if np.isscalar(eps) else np.asarray(eps, dtype=np.float64)
    return Workload(f"sep_{n_r}x{n_c}", g, G, eps_arr, iters,
                    extra={"p": p, "q": q, "r": r, "s": s})


def gaussian_pair(n, sig_g, sig_G, shift_g=(0.0, 0.0), shift_G=(0.0, 0.0)):
    """Gaussian amplitude -> Gaussian amplitude (the entropic closed-form case)."""
    g = normalise_power(gauss(n, n, sig_g, *shift_g))
    G = normalise_power(gauss(n, n, sig_G, *shift_G))
    return g, G


def random_potential(n_r, n_c, scale, seed, zero_frac=0.0):
    """Seeded smooth-plus-noise potential image (px^2) for single half-step checks,
    with an optional fraction of -inf (zero-mass) pixels."""
    rng = np.random.default_rng(seed)
    j, k = _grid(n_r, n_c)
    a2 = rng.uniform(0.1, 0.45)
    pot = scale * (a2 * (j * j + k * k) / max(n_r, n_c) ** 2 + 0.05 * rng.standard_normal((n_r, n_c)))
    if zero_frac > 0:
        pot[rng.uniform(size=(n_r, n_c)) < zero_frac] = -np.inf
    return pot
