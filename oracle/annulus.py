"""The annular problem: a square with a square hole, Dirichlet on the hole, Robin on the
outer edge (Section 2.3, the FD discussion of Section 2.4 and its figure).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Problem (Section 2.3, written for a general source and data):

    Delta u + k^2 u = f in Omega,   u = g on the hole's edge (d Omega_1),
    du/dn - i k u = q on the outer edge (d Omega_2),

with the paper's scattering data f = 0, g = -exp(-i k x_1), q = 0.  The iteration of
Section 2.3 (its real pair v_n, w_n), for alpha >= k^2 and sigma = alpha - k^2:

    (Delta - sigma) v_0 = f^Re, v_0 = g^Re on d Omega_1, dv_0/dn = q^Re on d Omega_2
    (Delta - sigma) v_n = -alpha v_{n-1}, v_n = 0 on d Omega_1, dv_n/dn = -k w_{n-1}
    (Delta - sigma) w_n = -alpha w_{n-1}, w_n = 0 on d Omega_1, dw_n/dn = +k v_{n-1}

(w_0 likewise with the imaginary parts), and u = sum_n (v_n + i w_n) when the sums
converge.  In complex form z_n = v_n + i w_n solves A z_n = M z_{n-1}, with A the real
FD matrix of the Laplacian rows and of the normal-derivative rows, and M diagonal:
-alpha on the PDE rows, +i k on the outer-edge rows (Section 2.4 with alpha = k^2); G =
A^{-1} M is the iteration matrix whose spectral radius decides convergence.

Discretisation (this project's reading; the paper prints no stencil):
  * square [-side/2, side/2]^2, N intervals per axis, h = side / N, nodes x_i = -side/2 + i h;
  * hole nodes: |x| <= hole and |y| <= hole (the closed hole; its outer layer carries g);
  * outer-edge nodes: i or j in {0, N} (outside the hole): their row is the outward normal
    derivative, the one-sided difference (u_b - u_in) / h towards the inward neighbour,
    averaged over the two normals at a corner;
  * every other node is a PDE node with the 5-point Delta_h (hole neighbours moved to the
    right-hand side as data).

Mean exit time and expected local time (Section 2.3's remarks, Eq. for k_*^A):
    Delta E = -c_tau in Omega, E = 0 on d Omega_1, dE/dn = 0 on d Omega_2,
    Delta L = 0,               L = 0 on d Omega_1, dL/dn = 1 on d Omega_2,
    k_*^A = min_x (-L + sqrt(L^2 + 4 E)) / (2 E).
c_tau = 1 is the normalisation of the cavity's Eq. (2.10); c_tau = 2 that of Section 3
(Delta E + 2 = 0).

Bookkeeping (start, relres, status rule) is that of ``iteration``: U_0 carries the hole
data and zero elsewhere, relres_N = ||b - B U_N|| / ||b - B U_0||, b the lifted
right-hand side and B the FD Helmholtz operator (PDE rows Delta_h + k^2, outer rows the
normal derivative minus i k).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .iteration import CONVERGED, IterationResult, StatusRule

PDE, EDGE, HOLE = 0, 1, 2
_NB = ((1, 0), (-1, 0), (0, 1), (0, -1))


@dataclass
class Geometry:
    N: int
    side: float
    hole: float
    h: float
    typ: np.ndarray          # (N+1, N+1) int: PDE / EDGE / HOLE, index [i, j] = (x_i, y_j)
    idx: np.ndarray          # unknown number of a node, -1 on hole nodes
    nodes: np.ndarray        # (M, 2) the unknown nodes (i, j)

    @property
    def x(self) -> np.ndarray:
        return -0.5 * self.side + self.h * np.arange(self.N + 1)


def geometry(N: int, side: float = 1.0, hole: float = 0.15) -> Geometry:
    """Node types of the square with a square hole (reading in the module docstring)."""
    h = side / N
    x = -0.5 * side + h * np.arange(N + 1)
    X, Y = np.meshgrid(x, x, indexing="ij")
    eps = 1e-9 * side
    typ = np.zeros((N + 1, N + 1), dtype=np.int64)
    i, j = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    typ[(i == 0) | (i == N) | (j == 0) | (j == N)] = EDGE
    typ[(np.abs(X) <= hole + eps) & (np.abs(Y) <= hole + eps)] = HOLE
    if (typ[:2, :] == HOLE).any() or (typ[-2:, :] == HOLE).any() or (typ[:, :2] == HOLE).any() \
            or (typ[:, -2:] == HOLE).any() or not (typ == HOLE).any():
        raise ValueError("the hole must hold a node and stay off the outer edge and its first layer")
    nodes = np.argwhere(typ != HOLE)
    idx = -np.ones((N + 1, N + 1), dtype=np.int64)
    idx[nodes[:, 0], nodes[:, 1]] = np.arange(len(nodes))
    return Geometry(N, side, hole, h, typ, idx, nodes)


def inward_offsets(geo: Geometry, i: int, j: int) -> list:
    """Offsets from an outer-edge node to its inward neighbour(s) (two at a corner)."""
    N, out = geo.N, []
    if i == 0:
        out.append((1, 0))
    if i == N:
        out.append((-1, 0))
    if j == 0:
        out.append((0, 1))
    if j == N:
        out.append((0, -1))
    return out


def operator(geo: Geometry, sigma: float = 0.0, k: float | None = None) -> sp.csr_matrix:
    """The FD operator on the unknowns.  k is None: A_sigma (PDE rows Delta_h - sigma, edge
    rows the normal derivative; real).  k given: the Helmholtz operator B (PDE rows
    Delta_h + k^2, edge rows the normal derivative - i k; sigma ignored)."""
    h, M = geo.h, len(geo.nodes)
    rows, cols, vals = [], [], []
    for q, (i, j) in enumerate(geo.nodes):
        if geo.typ[i, j] == PDE:
            diag = -4.0 / (h * h) + (k * k if k is not None else -sigma)
            rows.append(q); cols.append(q); vals.append(diag)
            for di, dj in _NB:
                t = geo.idx[i + di, j + dj]
                if t >= 0:
                    rows.append(q); cols.append(t); vals.append(1.0 / (h * h))
        else:
            offs = inward_offsets(geo, i, j)
            w = 1.0 / len(offs)
            rows.append(q); cols.append(q); vals.append(1.0 / h + (-1j * k if k is not None else 0.0))
            for di, dj in offs:
                rows.append(q); cols.append(geo.idx[i + di, j + dj]); vals.append(-w / h)
    dtype = np.complex128 if k is not None else np.float64
    return sp.csr_matrix((np.asarray(vals, dtype=dtype), (rows, cols)), shape=(M, M))


def lifted_rhs(geo: Geometry, data: np.ndarray) -> np.ndarray:
    """b on the unknowns from the (N+1)^2 data array (f on PDE nodes, q on outer-edge nodes,
    g on hole nodes): PDE rows f - (hole neighbours' g) / h^2, edge rows q."""
    h = geo.h
    b = np.zeros(len(geo.nodes), dtype=np.complex128)
    for q, (i, j) in enumerate(geo.nodes):
        b[q] = data[i, j]
        if geo.typ[i, j] == PDE:
            for di, dj in _NB:
                if geo.typ[i + di, j + dj] == HOLE:
                    b[q] -= data[i + di, j + dj] / (h * h)
    return b


def scatter(geo: Geometry, z: np.ndarray, data: np.ndarray | None = None) -> np.ndarray:
    """Unknown vector -> (N+1)^2 array (hole nodes from data, else 0)."""
    U = np.zeros((geo.N + 1,) * 2, dtype=np.complex128)
    if data is not None:
        U[geo.typ == HOLE] = data[geo.typ == HOLE]
    U[geo.nodes[:, 0], geo.nodes[:, 1]] = z
    return U


def scattering_data(geo: Geometry, k: float) -> np.ndarray:
    """The paper's data: f = 0, g = -exp(-i k x_1) on the hole, q = 0."""
    X = np.broadcast_to(geo.x[:, None], (geo.N + 1, geo.N + 1))
    data = np.zeros((geo.N + 1,) * 2, dtype=np.complex128)
    hole = geo.typ == HOLE
    data[hole] = -np.exp(-1j * k * X[hole])
    return data


def solve_direct(geo: Geometry, k: float, data: np.ndarray) -> np.ndarray:
    """The FD solution of the Robin problem, B u = b (sparse LU)."""
    B = operator(geo, k=k).tocsc()
    return scatter(geo, spla.spsolve(B, lifted_rhs(geo, data)), data)


def annulus_iteration(geo: Geometry, k: float, data: np.ndarray, alpha: float | None = None,
                      tol: float = 1e-8, max_outer: int = 1000,
                      keep_iterates: bool = False) -> IterationResult:
    """Section 2.3's iteration in its own notation (v_n, w_n; exact sparse solves of A_sigma).
    Returns the partial sums U_N = sum_{n<N} (v_n + i w_n) on the (N+1)^2 grid."""
    alpha = k * k if alpha is None else alpha
    if alpha < k * k:
        raise ValueError("the iteration needs alpha >= k^2")
    sigma = alpha - k * k
    lu = spla.splu(operator(geo, sigma=sigma).tocsc())
    B = operator(geo, k=k)
    b = lifted_rhs(geo, data)
    edge = geo.typ[geo.nodes[:, 0], geo.nodes[:, 1]] == EDGE
    solve = lambda r: lu.solve(np.ascontiguousarray(r, dtype=np.float64))

    rule = StatusRule(tol, max_outer)
    z = np.zeros(len(geo.nodes), dtype=np.complex128)
    r0 = float(np.linalg.norm(b - B @ z))
    U = scatter(geo, z, data)
    res = IterationResult(u=U, iters=0, relres=[], einf=[], iterates=[U.copy()] if keep_iterates else None)
    if r0 == 0.0:
        res.relres.append(0.0)
        res.status = CONVERGED
        return res
    res.relres.append(1.0)
    st = rule(0, 1.0)
    if st is not None:
        res.status = st
        return res
    # v_0, w_0: the PDE rows carry f and the hole data, the edge rows q (zero for the paper)
    v, w = solve(b.real), solve(b.imag)
    N = 0
    while True:
        z = z + (v + 1j * w)
        N += 1
        res.einf.append(float(np.max(np.abs(v + 1j * w))))
        rr = float(np.linalg.norm(b - B @ z)) / r0
        res.relres.append(rr)
        if keep_iterates:
            res.iterates.append(scatter(geo, z, data))
        st = rule(N, rr)
        if st is not None:
            res.status = st
            break
        # n >= 1: PDE rows -alpha times the previous increment; edge rows the Neumann data
        # -k w_{n-1} (for v) and +k v_{n-1} (for w)
        rv = np.where(edge, -k * w, -alpha * v)
        rw = np.where(edge, k * v, -alpha * w)
        v, w = solve(rv), solve(rw)
    res.u = scatter(geo, z, data)
    res.iters = N
    return res


def iteration_matrix(geo: Geometry, k: float, alpha: float | None = None) -> np.ndarray:
    """Dense G = A_sigma^{-1} M (M = -alpha on PDE rows, +i k on edge rows)."""
    alpha = k * k if alpha is None else alpha
    A = operator(geo, sigma=alpha - k * k).toarray()
    edge = geo.typ[geo.nodes[:, 0], geo.nodes[:, 1]] == EDGE
    m = np.where(edge, 1j * k, -alpha + 0j)
    return np.linalg.solve(A, np.diag(m))


def spectral_radius(geo: Geometry, k: float, alpha: float | None = None) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(iteration_matrix(geo, k, alpha)))))


def singular_extremes(geo: Geometry, k: float, alpha: float | None = None):
    """(sigma_max, sigma_min) of the dense G (its 2-norm and the inverse's 2-norm
    reciprocal), from the singular values of G."""
    sv = np.linalg.svd(iteration_matrix(geo, k, alpha), compute_uv=False)
    return float(sv[0]), float(sv[-1])


def condition_number(geo: Geometry, k: float, alpha: float | None = None) -> float:
    """2-norm condition number sigma_max / sigma_min of G, the quantity plotted against k
    beside the spectral radius in Section 2.4's figure (this project's reading: of the
    matrices A^{-1} and G only G depends on k)."""
    smax, smin = singular_extremes(geo, k, alpha)
    return smax / smin


def exit_times(geo: Geometry, c_tau: float = 1.0):
    """(E, L) on the (N+1)^2 grid: Delta E = -c_tau, dE/dn = 0; Delta L = 0, dL/dn = 1; both
    zero on the hole."""
    A = operator(geo, sigma=0.0).tocsc()
    edge = geo.typ[geo.nodes[:, 0], geo.nodes[:, 1]] == EDGE
    E = spla.spsolve(A, np.where(edge, 0.0, -c_tau))
    L = spla.spsolve(A, np.where(edge, 1.0, 0.0))
    return scatter(geo, E).real, scatter(geo, L).real


def k_star_A(geo: Geometry, c_tau: float = 1.0) -> float:
    """min over the PDE nodes of (-L + sqrt(L^2 + 4 E)) / (2 E)."""
    E, L = exit_times(geo, c_tau)
    pde = geo.typ == PDE
    kh = (-L[pde] + np.sqrt(L[pde] ** 2 + 4.0 * E[pde])) / (2.0 * E[pde])
    return float(kh.min())
