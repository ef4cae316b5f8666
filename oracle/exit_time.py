"""Mean exit time and the sufficient wavenumber bound k_*^C of the cavity iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Source: Section 2.2.  The iteration converges when (alpha + p) E[tau^y] < 1 for every
start y (the theorem after Eq. (2.8)); since alpha >= k^2, no alpha qualifies once k
exceeds k_*^C = sqrt(1 / max_y E[tau^y] - p) (Eq. (2.9)).  By the Feynman-Kac formula
the mean exit time E(x) = E[tau^x] of the process with generator Delta solves Eq. (2.10):
Delta E = -1 in Omega, E = 0 on the Dirichlet wall.  Discretised as in Section 2.4:
Delta_h E_h = -1 on the interior nodes, E_h = 0 on the wall; E_h is a plain Poisson
solve (sine basis here).

Continuum references for the unit square / cube (textbook torsion-function series, used
only to pin the discrete values' O(h^2) convergence):

* square, separating one variable:  E(x, y) = x(1-x)/2
  - sum_{m odd} 4 sin(m pi x) cosh(m pi (y - 1/2)) / (pi^3 m^3 cosh(m pi / 2));
* square, the double sine series:  E = sum_{m,n odd} 16 sin(m pi x) sin(n pi y)
  / (pi^4 m n (m^2 + n^2));
* cube, separating z:  E(x, y, z) = E_square(x, y)
  - sum_{m,n odd} 16 sin(m pi x) sin(n pi y) cosh(q (z - 1/2)) / (pi^4 m n (m^2 + n^2) cosh(q / 2)),
  q = pi sqrt(m^2 + n^2).
"""
from __future__ import annotations

import math

import numpy as np

from . import fd


def exit_time(D: int, n: int, h: float) -> np.ndarray:
    """E_h on the interior nodes: Delta_h E_h = -1, E_h = 0 on the wall."""
    return np.real(fd.dst_poisson(-np.ones((n,) * D), h))


def max_exit_time(D: int, n: int, h: float) -> float:
    return float(np.max(exit_time(D, n, h)))


def k_star_c(D: int, n: int, h: float, p: float = 0.0) -> float:
    """Eq. (2.9) with the discrete exit time: sqrt(1 / max E_h - p) (0 if negative)."""
    q = 1.0 / max_exit_time(D, n, h) - p
    return math.sqrt(q) if q > 0 else 0.0


def square_center_cosh_series(terms: int = 40) -> float:
    """max E on the unit square (attained at the centre), one-variable series."""
    s = 0.125
    for j in range(terms):
        m = 2 * j + 1
        s -= 4.0 * (-1) ** j / (math.pi ** 3 * m ** 3 * math.cosh(m * math.pi / 2))
    return s


def square_center_sine_series(terms: int = 400) -> float:
    """max E on the unit square from the double sine series (slower, independent form)."""
    m = 2 * np.arange(terms) + 1.0
    sg = (-1.0) ** np.arange(terms)
    M, N = np.meshgrid(m, m, indexing="ij")
    S = np.outer(sg, sg)
    return float(np.sum(16.0 * S / (math.pi ** 4 * M * N * (M * M + N * N))))


def cube_center_series(terms: int = 40) -> float:
    """max E on the unit cube (at the centre), separating z."""
    s = square_center_cosh_series()
    for a in range(terms):
        for b in range(terms):
            m, n = 2 * a + 1, 2 * b + 1
            q = math.pi * math.sqrt(m * m + n * n)
            sg = (-1) ** (a + b)
            s -= 16.0 * sg / (math.pi ** 4 * m * n * (m * m + n * n) * math.cosh(q / 2))
    return s
