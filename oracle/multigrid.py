"""Textbook geometric-multigrid components for Delta_h e = r with e = 0 on the wall.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves each Poisson iterate with an exact solver (it names probabilistic
domain decomposition, finite elements and direct solvers, Section 3); it prescribes no
multigrid.  This module restates, in the plainest numpy, the V-cycle the CUDA library
uses as its inner Poisson solver, so single sweeps and single cycles can be checked
element by element.  Its pins are mathematical facts (exact local solves at updated
points, exactness of the transfer operators on (multi)linear data, the adjoint relation
R = P^T / 2^D, convergence to the direct solve) -- see tests/test_oracle_multigrid.py.

Components (levels have n_l = 2^(m-l) - 1 interior nodes per axis, h_l = 2^l h):

* red-black Gauss-Seidel: a node with padded indices (i_x, i_y[, i_z]) is *red* when
  their sum is even; a half-sweep of one colour sets, at each node of that colour,
  e = (sum of the 2D neighbours - h^2 r) / (2D), i.e. solves that node's equation;
* residual r - Delta_h e;
* full-weighting restriction: the tensor product of [1, 2, 1]/4 along every axis,
  sampled at the even fine nodes (coarse node I <-> fine node 2I);
* multilinear prolongation: along every axis, fine 2I <- coarse I and
  fine 2I+1 <- (coarse I + coarse I+1)/2, added to the fine iterate;
* coarsest level n = 1: the exact solve e = -h^2 r / (2D);
* V(nu1, nu2)-cycle: nu1 x (red, black) half-sweeps, residual, restriction, recursive
  cycle on the coarse level from a zero guess, prolongation + correction,
  nu2 x (red, black) half-sweeps;
* optionally (``exact_n``) a direct coarse-grid solver: the level with n == exact_n is
  not cycled but solved exactly (sine-basis solve of Delta_h e = r, zero walls), as the
  CUDA library does for its 2D complex64 hierarchies.

``sigma`` >= 0 selects the shifted operator Delta_h - sigma of the general cavity
iteration (Section 2.2, sigma = alpha - k^2; see ``general``) on every level: the local
solve becomes e = (sum of neighbours - h^2 r) / (2D + sigma h^2), the residual
r - (Delta_h - sigma) e, the one-node solve e = -h^2 r / (2D + sigma h^2).
"""
from __future__ import annotations

import numpy as np

from . import fd


def color_mask(D: int, n: int, color: int) -> np.ndarray:
    """Boolean interior mask of the nodes whose padded index sum has parity `color`
    (0 = red, 1 = black)."""
    i = np.arange(1, n + 1)
    if D == 2:
        s = i[:, None] + i[None, :]
    else:
        s = i[:, None, None] + i[None, :, None] + i[None, None, :]
    return (s % 2) == color


def rbgs_half_sweep(E: np.ndarray, r: np.ndarray, h: float, color: int,
                    sigma: float = 0.0) -> None:
    """In-place half-sweep on the padded iterate E for the interior right-hand side r."""
    D = E.ndim
    n = E.shape[0] - 2
    nbr = np.zeros(r.shape, dtype=E.dtype)
    for a in range(D):
        nbr = nbr + fd._shift(E, a, +1) + fd._shift(E, a, -1)
    new = (nbr - (h * h) * r) / (2.0 * D + sigma * h * h)
    mask = color_mask(D, n, color)
    inner = E[(slice(1, -1),) * D]
    inner[mask] = new[mask]


def rbgs_sweep(E: np.ndarray, r: np.ndarray, h: float, sigma: float = 0.0) -> None:
    rbgs_half_sweep(E, r, h, 0, sigma)
    rbgs_half_sweep(E, r, h, 1, sigma)


def poisson_residual(E: np.ndarray, r: np.ndarray, h: float, sigma: float = 0.0) -> np.ndarray:
    """r - (Delta_h - sigma) E on the interior."""
    return r - (fd.apply_laplacian(E, h) - sigma * fd.interior(E))


def restrict_fw(rf: np.ndarray) -> np.ndarray:
    """Full weighting of the interior fine array rf (n_f = 2 n_c + 1) to n_c^D."""
    D = rf.ndim
    P = np.zeros(tuple(s + 2 for s in rf.shape), dtype=rf.dtype)
    P[(slice(1, -1),) * D] = rf
    for a in range(D):
        lo = [slice(None)] * D
        mid = [slice(None)] * D
        hi = [slice(None)] * D
        lo[a] = slice(0, -2)
        mid[a] = slice(1, -1)
        hi[a] = slice(2, None)
        S = np.zeros_like(P)
        sm = [slice(None)] * D
        sm[a] = slice(1, -1)
        S[tuple(sm)] = (P[tuple(lo)] + 2.0 * P[tuple(mid)] + P[tuple(hi)]) / 4.0
        P = S
    # coarse interior I = 1..n_c sits at fine padded index 2I
    return P[(slice(2, -2, 2),) * D]


def prolong_add(Ef: np.ndarray, Ec: np.ndarray) -> None:
    """Ef (padded fine) += multilinear interpolation of Ec (padded coarse, ring used)."""
    D = Ec.ndim
    Q = Ec
    for a in range(D):
        nc2 = Q.shape[a]                  # n_c + 2
        shape = list(Q.shape)
        shape[a] = 2 * nc2 - 1            # n_f + 2
        R = np.zeros(shape, dtype=Q.dtype)
        ev = [slice(None)] * D
        od = [slice(None)] * D
        q0 = [slice(None)] * D
        q1 = [slice(None)] * D
        ev[a] = slice(0, None, 2)
        od[a] = slice(1, None, 2)
        q0[a] = slice(0, -1)
        q1[a] = slice(1, None)
        R[tuple(ev)] = Q
        R[tuple(od)] = (Q[tuple(q0)] + Q[tuple(q1)]) / 2.0
        Q = R
    Ef[(slice(1, -1),) * D] += Q[(slice(1, -1),) * D]


def coarse_solve(E: np.ndarray, r: np.ndarray, h: float, sigma: float = 0.0) -> None:
    """Exact solve on a single interior node (n = 1): -(2D / h^2 + sigma) e = r."""
    D = E.ndim
    E[(slice(1, 2),) * D] = -(h * h) * r / (2.0 * D + sigma * h * h)


def vcycle(E: np.ndarray, r: np.ndarray, h: float, nu1: int = 2, nu2: int = 2,
           exact_n: int | None = None, sigma: float = 0.0) -> None:
    """One V(nu1, nu2)-cycle on the padded iterate E (in place); a level with
    n == exact_n is solved exactly instead (whatever E held there)."""
    D = E.ndim
    n = E.shape[0] - 2
    if exact_n is not None and n == exact_n:
        if sigma == 0.0:
            E[(slice(1, -1),) * D] = fd.dst_poisson(r, h)
        else:
            from .general import dst_shifted_poisson
            E[(slice(1, -1),) * D] = dst_shifted_poisson(r, h, sigma)
        return
    if n == 1:
        coarse_solve(E, r, h, sigma)
        return
    for _ in range(nu1):
        rbgs_sweep(E, r, h, sigma)
    rc = restrict_fw(poisson_residual(E, r, h, sigma))
    nc = rc.shape[0]
    Ec = np.zeros((nc + 2,) * D, dtype=E.dtype)
    vcycle(Ec, rc, 2.0 * h, nu1, nu2, exact_n, sigma)
    prolong_add(E, Ec)
    for _ in range(nu2):
        rbgs_sweep(E, r, h, sigma)
