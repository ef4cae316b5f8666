"""The general cavity iteration: shift alpha >= k^2 and damping p >= 0, Dirichlet wall.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Source: Section 2.2.  The cavity problem Eq. (2.4) with a wall that is Dirichlet
everywhere,

    Delta u + (i p + k^2) u = f in Omega,   u = g on the wall,

splits into the real pair Eq. (2.5), and the iteration Eq. (2.6) with the boundary
conditions Eq. (2.7) reads, with sigma = alpha - k^2 >= 0,

    (Delta - sigma) v_0 = f^Re,                   v_0 = g^Re on the wall,
    (Delta - sigma) w_0 = f^Im,                   w_0 = g^Im on the wall,
    (Delta - sigma) v_n = -alpha v_{n-1} + p w_{n-1},   v_n = 0 on the wall (n >= 1),
    (Delta - sigma) w_n = -alpha w_{n-1} - p v_{n-1},   w_n = 0 on the wall (n >= 1),

and u = sum_n (v_n + i w_n) when the sums converge (the theorem that follows Eq. (2.8)).
Discretised as in Section 2.4 (Delta -> Delta_h, wall nodes moved to the right-hand
side).  In complex form z_n = v_n + i w_n obeys (Delta_h - sigma) z_n = -(alpha + i p)
z_{n-1}: the iteration matrix is G = -(alpha + i p)(Delta_h - sigma)^{-1}, normal, with
eigenvalues (alpha + i p) / (lambda_m + sigma) (lambda_m > 0 the eigenvalues of -Delta_h),
so rho(G) = sqrt(alpha^2 + p^2) / (lambda_min + sigma) and the partial sums converge iff
rho < 1, i.e. k^2 < lambda_min + alpha - sqrt(alpha^2 + p^2).  With alpha = k^2 and
p = 0 everything reduces to ``iteration.paper_iteration``.

Bookkeeping (start, iteration count, relres, status rule) is that of ``iteration``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fd
from .iteration import CONVERGED, DIVERGED, IterationResult, StatusRule


def apply_damped_helmholtz(U: np.ndarray, h: float, k: float, p: float) -> np.ndarray:
    """(Delta_h + k^2 + i p) U at every interior node (U padded)."""
    return fd.apply_laplacian(U, h) + (k * k + 1j * p) * fd.interior(U)


def residual(U: np.ndarray, f: np.ndarray, h: float, k: float, p: float) -> np.ndarray:
    """r = f - (Delta_h + k^2 + i p) U on the interior."""
    return f - apply_damped_helmholtz(U, h, k, p)


def shifted_laplacian_matrix(D: int, n: int, h: float, sigma: float) -> sp.csr_matrix:
    """Delta_h - sigma I on the interior unknowns (real)."""
    return (fd.laplacian_matrix(D, n, h) - sigma * sp.identity(n ** D, format="csr")).tocsr()


def dst_shifted_poisson(r: np.ndarray, h: float, sigma: float,
                        workers: int | None = None) -> np.ndarray:
    """Exact e of (Delta_h - sigma) e = r, e = 0 on the wall: e^ = r^ / (-lambda_m - sigma)."""
    lam = fd._dst_eigs(r.ndim, r.shape[0], h)
    rh = scipy.fft.dstn(r, type=1, workers=workers)
    return scipy.fft.idstn(rh / (-lam - sigma), type=1, workers=workers)


def solve_exact(f: np.ndarray, g: np.ndarray, h: float, k: float, p: float,
                workers: int | None = None) -> np.ndarray:
    """Unique solution of (Delta_h + k^2 + i p) u = f, u = g on the wall (sine basis:
    u^ = b^ / (k^2 + i p - lambda_m)); padded."""
    lam = fd._dst_eigs(f.ndim, f.shape[0], h)
    b = fd.lifted_rhs(f, g, h)
    bh = scipy.fft.dstn(b, type=1, workers=workers)
    x = scipy.fft.idstn(bh / (k * k + 1j * p - lam), type=1, workers=workers)
    return fd.padded_from(x, g.astype(np.complex128))


def rho_pred(D: int, n: int, h: float, k: float, alpha: float, p: float) -> float:
    """Spectral radius of G = -(alpha + i p)(Delta_h - sigma)^{-1}, sigma = alpha - k^2."""
    return math.hypot(alpha, p) / (fd.lambda_min(D, n, h) + alpha - k * k)


def k_limit(D: int, n: int, h: float, alpha: float, p: float) -> float:
    """Supremum of the k (with alpha >= k^2 fixed) for which rho < 1:
    k^2 < lambda_min + alpha - sqrt(alpha^2 + p^2) (0 when no k qualifies)."""
    q = fd.lambda_min(D, n, h) + alpha - math.hypot(alpha, p)
    return math.sqrt(q) if q > 0 else 0.0


def predicted_status(D: int, n: int, h: float, k: float, alpha: float, p: float) -> int:
    return CONVERGED if rho_pred(D, n, h, k, alpha, p) < 1.0 else DIVERGED


class ShiftedSolver:
    """Direct solver of (Delta_h - sigma) e = r (hom. Dirichlet) for real right-hand
    sides: one sparse LU of the real matrix, reused for every solve."""

    def __init__(self, D: int, n: int, h: float, sigma: float):
        self.shape = (n,) * D
        self.lu = spla.splu(shifted_laplacian_matrix(D, n, h, sigma).tocsc())

    def __call__(self, r: np.ndarray) -> np.ndarray:
        assert np.isrealobj(r)
        return self.lu.solve(np.ascontiguousarray(r, dtype=np.float64).reshape(-1)).reshape(self.shape)


def general_iteration(f: np.ndarray, g: np.ndarray, h: float, k: float, alpha: float,
                      p: float, tol: float = 1e-8, max_outer: int = 1000,
                      keep_iterates: bool = False) -> IterationResult:
    """The iteration Eq. (2.6)-(2.8) in its own notation (v_n, w_n; exact shifted solves).

    f: interior (n,)*D complex128; g: padded (n+2,)*D complex128 (ring = wall data).
    Requires alpha >= k^2 (Section 2.2) and p >= 0."""
    if alpha < k * k or p < 0:
        raise ValueError("the iteration needs alpha >= k^2 and p >= 0")
    D, n = f.ndim, f.shape[0]
    f = np.asarray(f, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    sigma = alpha - k * k
    solve = ShiftedSolver(D, n, h, sigma)
    G0 = fd.ring_only(g)

    def relres_of(U):
        return float(np.linalg.norm(residual(U, f, h, k, p)))

    rule = StatusRule(tol, max_outer)
    U = G0.copy()
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
    # v_0, w_0: (Delta_h - sigma) v_0 = f^Re with v_0 = g^Re on the wall; the wall nodes
    # moved to the right-hand side (sigma acts on interior nodes only)
    Lg = fd.apply_laplacian(G0, h)
    v = solve(f.real - Lg.real)
    w = solve(f.imag - Lg.imag)
    N = 0
    while True:
        inc = v + 1j * w
        if N == 0:
            U = fd.padded_from(inc, g)
        else:
            U = U.copy()
            U[(slice(1, -1),) * D] += inc
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
        # Eq. (2.6), n >= 1: the real and imaginary chains couple through p
        v, w = solve(-alpha * v + p * w), solve(-alpha * w - p * v)
    res.u = U
    res.iters = N
    return res
