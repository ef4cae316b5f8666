"""The paper's nested Poisson iteration for the Dirichlet cavity, with exact inner solves.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Source: Section 2.2, the iteration Eq. (2.6) with boundary conditions Eq. (2.7)-(2.8),
taken with alpha = k^2 (the choice Section 2.4 makes for its FD analysis) and p = 0,
on a wall that is Dirichlet everywhere.  In the paper's notation, with f = f^Re + i f^Im
and g = g^Re + i g^Im:

    Delta v_0 = f^Re,             v_0 = g^Re on the wall,
    Delta w_0 = f^Im,             w_0 = g^Im on the wall,
    Delta v_n = -k^2 v_{n-1},     v_n = 0 on the wall   (n >= 1),
    Delta w_n = -k^2 w_{n-1},     w_n = 0 on the wall   (n >= 1),

and the solution is the sum u = sum_n (v_n + i w_n) (the theorem of Section 2.2).
Each v_n, w_n is a *real* Poisson problem: with p = 0 the real and imaginary chains do
not couple (Eq. (2.5)).  Discretised (Section 2.4) every iterate is an exact solve with
the real matrix Delta_h, and the increments obey u_n = G u_{n-1} with
G = -k^2 Delta_h^{-1}, so the partial sums are the matrix geometric series.

Bookkeeping used throughout this project (readings of points the paper leaves open):

* u^(0) = 0 inside, g on the wall; u^(N) = sum_{n < N} (v_n + i w_n) for N >= 1.
  ``iters`` counts the increments added, so u^(iters) is returned and the residual
  history has iters + 1 entries.
* relres_N = ||f - (Delta_h + k^2) u^(N)||_2 / ||f - (Delta_h + k^2) u^(0)||_2 over the
  interior nodes (unweighted 2-norm; the h^(D/2) weights cancel).  With u^(0) as above
  the denominator is ||b||_2, b the lifted right-hand side of Section 2.4.
* The increment sup-norm ||v_n + i w_n||_inf is recorded too: Section 3 proposes
  truncating on the size of successive iterates.
* Status (the paper only reports "converges" / "diverges"): CONVERGED when relres <= tol;
  DIVERGED when relres > 1e4, or when N >= 20, relres has not decreased for 10
  consecutive steps and has grown to at least twice its smallest value so far (so that
  stagnation at the rounding floor is not taken for divergence); NONFINITE on a NaN /
  Inf; MAXITER when N reaches max_outer.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import fd

CONVERGED = 0
MAXITER = 1
DIVERGED = 2
NONFINITE = -4

DIVERGE_RELRES = 1e4
DIVERGE_MIN_STEPS = 20
DIVERGE_RUN = 10
DIVERGE_GROWTH = 2.0


@dataclass
class IterationResult:
    u: np.ndarray                  # padded complex128, u^(iters)
    iters: int
    relres: list = field(default_factory=list)    # iters + 1 entries
    einf: list = field(default_factory=list)      # iters entries, ||increment||_inf
    status: int = MAXITER
    iterates: list | None = None   # optional padded u^(N), N = 0..iters


class StatusRule:
    """Incremental form of the convergence / divergence rule above."""

    def __init__(self, tol: float, max_outer: int):
        self.tol = tol
        self.max_outer = max_outer
        self.prev = None
        self.run = 0
        self.rmin = math.inf

    def __call__(self, N: int, relres: float) -> int | None:
        if not math.isfinite(relres):
            return NONFINITE
        if relres <= self.tol:
            return CONVERGED
        if relres > DIVERGE_RELRES:
            return DIVERGED
        if self.prev is not None:
            self.run = self.run + 1 if relres >= self.prev else 0
        self.prev = relres
        self.rmin = min(self.rmin, relres)
        if (N >= DIVERGE_MIN_STEPS and self.run >= DIVERGE_RUN
                and relres >= DIVERGE_GROWTH * self.rmin):
            return DIVERGED
        if N >= self.max_outer:
            return MAXITER
        return None


def paper_iteration(f: np.ndarray, g: np.ndarray, h: float, k: float,
                    tol: float = 1e-8, max_outer: int = 1000, poisson: str = "splu",
                    keep_iterates: bool = False, workers: int | None = None) -> IterationResult:
    """Run the alpha = k^2, p = 0 cavity iteration of Section 2.2 with exact Poisson solves.

    f: interior (n,)*D complex128; g: padded (n+2,)*D complex128 (ring = wall data).
    poisson: "splu" (sparse LU of the real Delta_h) or "dst" (sine-basis solve).
    """
    D, n = f.ndim, f.shape[0]
    f = np.asarray(f, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    solve = fd.SparsePoisson(D, n, h) if poisson == "splu" else fd.DSTPoisson(D, n, h, workers)
    G0 = fd.ring_only(g)

    def relres_of(U):
        return float(np.linalg.norm(fd.residual(U, f, h, k)))

    rule = StatusRule(tol, max_outer)
    U = G0.copy()                                   # u^(0)
    r0 = relres_of(U)
    res = IterationResult(u=U, iters=0, relres=[], einf=[],
                          iterates=[U.copy()] if keep_iterates else None)
    if r0 == 0.0:
        res.relres.append(0.0)
        res.status = CONVERGED
        return res
    res.relres.append(1.0)
    st = rule(0, 1.0)
    if st is not None:
        res.status = st
        return res

    # v_0, w_0: Delta v_0 = f^Re with v_0 = g^Re on the wall.  With the wall data moved
    # to the right-hand side (Section 2.4) the interior solve is Delta_h v = f^Re - Delta_h(G0^Re).
    Lg = fd.apply_laplacian(G0, h)
    v = solve((f.real - Lg.real))
    w = solve((f.imag - Lg.imag))
    N = 0
    while True:
        inc = v + 1j * w                             # interior values of v_N + i w_N
        if N == 0:
            U = fd.padded_from(inc, g)               # u^(1) = v_0 + i w_0 (carries the wall data)
        else:
            U = U.copy()
            U[(slice(1, -1),) * D] += inc            # u^(N+1) = u^(N) + v_N + i w_N
        N += 1
        res.einf.append(float(np.max(np.abs(inc))))
        rr = relres_of(U) / r0
        res.relres.append(rr)
        if keep_iterates:
            res.iterates.append(U.copy())
        st = rule(N, rr)
        if st is not None:
            res.status = st
            break
        # next increments: Delta v_N = -k^2 v_{N-1}, v_N = 0 on the wall (likewise w_N)
        v = solve(-(k * k) * v)
        w = solve(-(k * k) * w)
    res.u = U
    res.iters = N
    return res


def predicted_status(D: int, n: int, h: float, k: float) -> int:
    """CONVERGED when the spectral radius k^2 / lambda_min of G is below one."""
    return CONVERGED if fd.rho_pred(D, n, h, k) < 1.0 else DIVERGED
