"""Seeded synthetic inputs for the Dirichlet-cavity Helmholtz workloads.

This module only *draws* data: grid coordinates, sources f and boundary data g
on the host, in numpy complex128, from ``numpy.random.default_rng(seed)`` with a
fixed draw order.  It contains none of the solver's arithmetic (no stencil, no
residual, no Poisson solve, no iteration).  Both the CPU oracle and the CUDA path
receive exactly the arrays built here.

Layouts (the same memory layout as ``torch.complex128``):

* ``f``: interior values, shape ``(n,)*D``, index order ``[z, y, x]`` (x fastest);
  interior node ``(i, j[, l])`` sits at ``x = i*h`` for ``i = 1..n``.
* ``g``: a padded array of shape ``(n+2,)*D``; only its boundary ring is data
  (the Dirichlet values of the cavity wall), its interior is ignored.

Workloads (the cavity problem of Section 2.2 with ``p = 0`` and a Dirichlet-only
wall, on the unit square / cube, ``h = 1/(n+1)``):

* ``plane_wave_cavity_2d``: 63x63, f = 0, g = exp(i k (cos t x + sin t y)), t = pi/6.
* ``gaussian_cavity_2d``: 1023x1023, g = 0, f = sum of 8 Gaussians of width 0.02
  with centres uniform in [0.2, 0.8]^2 and amplitudes N(0,1) + i N(0,1).
* ``plane_wave_sine_cube``: 255^3, g = plane wave along a seeded unit direction,
  f = sin(pi x) sin(2 pi y) sin(pi z).
* ``batched_instances``: N in {63, 127, 255, 511} with probabilities
  {0.4, 0.3, 0.2, 0.1}, k uniform in [0.5, 0.9 k_max(N)], Gaussian sources.
* ``served_stream``: Poisson arrivals of mixed 2D / 3D requests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAUSS_WIDTH = 0.02
N_GAUSS = 8


def node_coords(D: int, n: int, h: float):
    """Coordinates of the padded grid, as broadcastable arrays in [z, y, x] order.

    Returns a list ``[x, y]`` (2D) or ``[x, y, z]`` (3D) of arrays of shape
    ``(n+2,)*D`` broadcast-ready; node ``i`` of an axis sits at ``i*h``.
    """
    t = np.arange(n + 2, dtype=np.float64) * h
    if D == 2:
        y, x = np.meshgrid(t, t, indexing="ij")
        return [x, y]
    if D == 3:
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        return [x, y, z]
    raise ValueError("D must be 2 or 3")


def interior(a: np.ndarray) -> np.ndarray:
    """View of the interior of a padded array."""
    return a[(slice(1, -1),) * a.ndim]


def plane_wave(D: int, n: int, h: float, kappa: float, direction) -> np.ndarray:
    """Padded array exp(i kappa d.x) at every node (ring and interior)."""
    d = np.asarray(direction, dtype=np.float64)
    xs = node_coords(D, n, h)
    phase = sum(kappa * d[a] * xs[a] for a in range(D))
    return np.exp(1j * phase)


def zero_ring(D: int, n: int) -> np.ndarray:
    return np.zeros((n + 2,) * D, dtype=np.complex128)


def draw_gaussian_params(D: int, rng: np.random.Generator, n_gauss: int = N_GAUSS,
                         lo: float = 0.2, hi: float = 0.8):
    """Draw order: all centres (n_gauss x D uniforms in [lo, hi]), then the real parts
    of the amplitudes (n_gauss normals), then the imaginary parts (n_gauss normals)."""
    centres = rng.uniform(lo, hi, size=(n_gauss, D))
    a_re = rng.standard_normal(n_gauss)
    a_im = rng.standard_normal(n_gauss)
    return centres, a_re + 1j * a_im


def gaussian_from_params(D: int, n: int, h: float, centres, amps,
                         width: float = GAUSS_WIDTH) -> np.ndarray:
    """Sum of Gaussians a_j exp(-|x - c_j|^2 / (2 width^2)) on the interior nodes."""
    xs = [interior(c) for c in node_coords(D, n, h)]
    f = np.zeros((n,) * D, dtype=np.complex128)
    for j in range(len(amps)):
        r2 = sum((xs[a] - centres[j, a]) ** 2 for a in range(D))
        f += amps[j] * np.exp(-r2 / (2.0 * width * width))
    return f


def gaussian_source(D: int, n: int, h: float, rng: np.random.Generator,
                    n_gauss: int = N_GAUSS, width: float = GAUSS_WIDTH,
                    lo: float = 0.2, hi: float = 0.8) -> np.ndarray:
    """Seeded Gaussian source: draws its parameters, then evaluates them."""
    centres, amps = draw_gaussian_params(D, rng, n_gauss, lo, hi)
    return gaussian_from_params(D, n, h, centres, amps, width)


def sine_source(D: int, n: int, h: float, modes) -> np.ndarray:
    """prod_d sin(m_d pi x_d) on the interior (real, stored as complex128)."""
    xs = [interior(c) for c in node_coords(D, n, h)]
    f = np.ones((n,) * D, dtype=np.float64)
    for a in range(D):
        f = f * np.sin(modes[a] * math.pi * xs[a])
    return f.astype(np.complex128)


@dataclass
class Problem:
    """One Dirichlet-cavity Helmholtz problem: (Delta_h + k^2) u = f, u = g on the wall."""
    D: int
    n: int
    h: float
    k: float
    f: np.ndarray          # (n,)*D complex128
    g: np.ndarray          # (n+2,)*D complex128, ring = Dirichlet data
    meta: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.n ** self.D


def plane_wave_cavity_2d(k: float, n: int = 63, theta: float = math.pi / 6) -> Problem:
    """63x63 unit-square cavity, f = 0, g = exp(i k (cos(theta) x + sin(theta) y))."""
    h = 1.0 / (n + 1)
    d = (math.cos(theta), math.sin(theta))
    g = plane_wave(2, n, h, k, d)
    f = np.zeros((n, n), dtype=np.complex128)
    return Problem(2, n, h, k, f, g, {"theta": theta, "direction": d})


def gaussian_cavity_2d(k: float, seed: int = 2, n: int = 1023) -> Problem:
    """1023x1023 unit-square cavity, g = 0, f = 8 seeded Gaussians of width 0.02."""
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(seed)
    f = gaussian_source(2, n, h, rng)
    return Problem(2, n, h, k, f, zero_ring(2, n), {"seed": seed})


def random_direction(D: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(D)
    return v / np.linalg.norm(v)


def plane_wave_sine_cube(k: float = 4.0, seed: int = 3, n: int = 255) -> Problem:
    """255^3 unit-cube cavity: plane-wave wall data along a seeded direction plus
    the source sin(pi x) sin(2 pi y) sin(pi z)."""
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(seed)
    d = random_direction(3, rng)
    g = plane_wave(3, n, h, k, d)
    f = sine_source(3, n, h, (1, 2, 1))
    return Problem(3, n, h, k, f, g, {"seed": seed, "direction": tuple(d)})


def dirichlet_kmax(D: int, n: int, h: float) -> float:
    """Square root of the smallest eigenvalue of the Dirichlet 2nd-order FD Laplacian
    on an n^D grid of spacing h (textbook eigenpairs of the 1D [1,-2,1] matrix).
    Used here only to set the sampling range of k for the batched and served
    workloads."""
    return math.sqrt(D * 4.0 / (h * h) * math.sin(math.pi / (2.0 * (n + 1))) ** 2)


def batched_instances(count: int = 512, seed: int = 4,
                      sizes=(63, 127, 255, 511), probs=(0.4, 0.3, 0.2, 0.1),
                      k_lo: float = 0.5, k_frac: float = 0.9) -> list[Problem]:
    """Independent 2D cavities of uneven size with Gaussian sources and g = 0.

    Draw order: all sizes, then all k fractions, then each instance's source in
    instance order (8 centres, 8 real amplitudes, 8 imaginary amplitudes).
    """
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count, p=np.asarray(probs))
    us = rng.uniform(0.0, 1.0, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        h = 1.0 / (n + 1)
        kmax = dirichlet_kmax(2, n, h)
        k = k_lo + us[i] * (k_frac * kmax - k_lo)
        f = gaussian_source(2, n, h, rng)
        out.append(Problem(2, n, h, float(k), f, zero_ring(2, n), {"seed": seed, "index": i}))
    return out


@dataclass
class Request:
    t_arrival: float
    problem: Problem


def served_stream(rate: float, count: int, seed: int = 5,
                  sizes_2d=(127, 255, 511, 1023, 2047), sizes_3d=(63, 127, 255),
                  p_2d: float = 0.7, p_gauss: float = 0.5,
                  k_lo: float = 0.5, k_frac: float = 0.9,
                  materialise: bool = True) -> list[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate) of mixed 2D / 3D requests.

    Each request: dimension (2D with probability p_2d), size uniform over that
    dimension's list, k uniform in [k_lo, k_frac k_max], then either Gaussian
    sources with g = 0 (probability p_gauss) or f = 0 and a plane wave of wave
    number k on the wall along a random direction.  Draw order per request:
    gap, dimension, size, k fraction, source kind, then the source's own draws.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        D = 2 if rng.uniform() < p_2d else 3
        sizes = sizes_2d if D == 2 else sizes_3d
        n = int(sizes[rng.integers(len(sizes))])
        h = 1.0 / (n + 1)
        kmax = dirichlet_kmax(D, n, h)
        k = k_lo + rng.uniform() * (k_frac * kmax - k_lo)
        gauss = rng.uniform() < p_gauss
        if gauss:
            centres, amps = draw_gaussian_params(D, rng)
            f = gaussian_from_params(D, n, h, centres, amps) if materialise else None
            g = zero_ring(D, n) if materialise else None
            meta = {"index": i, "kind": "gauss", "centres": centres, "amps": amps}
        else:
            d = random_direction(D, rng)
            f = np.zeros((n,) * D, dtype=np.complex128) if materialise else None
            g = plane_wave(D, n, h, k, d) if materialise else None
            meta = {"index": i, "kind": "plane", "direction": tuple(d)}
        reqs.append(Request(t, Problem(D, n, h, float(k), f, g, meta)))
    return reqs


def materialise(p: Problem) -> Problem:
    """Build f and g of a request drawn with ``materialise=False``."""
    if p.f is not None:
        return p
    if p.meta["kind"] == "gauss":
        f = gaussian_from_params(p.D, p.n, p.h, p.meta["centres"], p.meta["amps"])
        g = zero_ring(p.D, p.n)
    else:
        f = np.zeros((p.n,) * p.D, dtype=np.complex128)
        g = plane_wave(p.D, p.n, p.h, p.k, p.meta["direction"])
    return Problem(p.D, p.n, p.h, p.k, f, g, p.meta)


def annulus_scattering(N: int, k: float, side: float = 1.0, hole: float = 0.15) -> np.ndarray:
    """Data array of the annular problem's scattering case (Section 2.3): g = -exp(-i k x_1) on
    the nodes of the closed hole |x|, |y| <= hole of the (N+1)^2 grid on [-side/2, side/2]^2
    (node (i, j) at (-side/2 + i h, -side/2 + j h), h = side / N); f = 0 and q = 0 elsewhere."""
    h = side / N
    x = -0.5 * side + h * np.arange(N + 1)
    X, Y = np.meshgrid(x, x, indexing="ij")
    eps = 1e-9 * side
    hole_nodes = (np.abs(X) <= hole + eps) & (np.abs(Y) <= hole + eps)
    data = np.zeros((N + 1, N + 1), dtype=np.complex128)
    data[hole_nodes] = -np.exp(-1j * k * X[hole_nodes])
    return data
