"""Finite-difference operator, lifting, exact discrete solutions and closed forms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Problem (Section 2.2, the cavity problem Eq. (2.4) with damping p = 0 and a wall that
is Dirichlet everywhere, i.e. the reflecting part of the wall is empty):

    Delta u + k^2 u = f in Omega = (0, l)^D,   u = g on the wall,

discretised as in Section 2.4: second-order central differences on the nodes
x_i = i h, i = 0..n+1, with the Dirichlet nodes eliminated and moved to the
right-hand side, giving the system B(k) u = b on the n^D interior nodes.

Array conventions: a *padded* array has shape (n+2,)*D (ring = wall nodes), an
*interior* array has shape (n,)*D; index order [z, y, x], x fastest.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# The stencil (definition of Delta_h, Section 2.4)
# ---------------------------------------------------------------------------

def _shift(U: np.ndarray, axis: int, off: int) -> np.ndarray:
    """Interior-sized view of the padded array U shifted by `off` along `axis`."""
    idx = []
    for a in range(U.ndim):
        if a == axis:
            idx.append(slice(1 + off, U.shape[a] - 1 + off))
        else:
            idx.append(slice(1, U.shape[a] - 1))
    return U[tuple(idx)]


def interior(U: np.ndarray) -> np.ndarray:
    return U[(slice(1, -1),) * U.ndim]


def apply_laplacian(U: np.ndarray, h: float) -> np.ndarray:
    """Delta_h U at every interior node: sum over axes of (U[+1] - 2 U + U[-1]) / h^2.

    U is padded; the ring values enter as the wall data."""
    c = interior(U)
    out = np.zeros(c.shape, dtype=np.result_type(U.dtype, np.float64))
    for a in range(U.ndim):
        out += (_shift(U, a, +1) - 2.0 * c + _shift(U, a, -1))
    return out / (h * h)


def apply_helmholtz(U: np.ndarray, h: float, k: float) -> np.ndarray:
    """(Delta_h + k^2) U at every interior node (U padded)."""
    return apply_laplacian(U, h) + (k * k) * interior(U)


def residual(U: np.ndarray, f: np.ndarray, h: float, k: float) -> np.ndarray:
    """r = f - (Delta_h + k^2) U on the interior."""
    return f - apply_helmholtz(U, h, k)


def padded_from(interior_vals: np.ndarray, ring: np.ndarray | None = None) -> np.ndarray:
    """Padded array with the given interior and ring (zero ring if `ring` is None)."""
    D = interior_vals.ndim
    n = interior_vals.shape[0]
    dtype = np.result_type(interior_vals.dtype, ring.dtype if ring is not None else np.float64)
    U = np.zeros((n + 2,) * D, dtype=dtype) if ring is None else ring.astype(dtype, copy=True)
    U[(slice(1, -1),) * D] = interior_vals
    return U


def ring_only(g: np.ndarray) -> np.ndarray:
    """Copy of the padded array g with its interior zeroed (the lifting of the wall data)."""
    G = g.copy()
    G[(slice(1, -1),) * g.ndim] = 0
    return G


def lifted_rhs(f: np.ndarray, g: np.ndarray, h: float) -> np.ndarray:
    """b of B(k) u = b (Section 2.4): the Dirichlet nodes are moved to the right-hand
    side, b = f - Delta_h(G0) with G0 = the wall data on the ring and 0 inside."""
    return f - apply_laplacian(ring_only(g), h)


# ---------------------------------------------------------------------------
# Sparse matrices (Dirichlet nodes eliminated)
# ---------------------------------------------------------------------------

def laplacian_1d(n: int, h: float) -> sp.csr_matrix:
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr") / (h * h)


def laplacian_matrix(D: int, n: int, h: float) -> sp.csr_matrix:
    """Delta_h on the n^D interior unknowns (x fastest), as a Kronecker sum."""
    T = laplacian_1d(n, h)
    I = sp.identity(n, format="csr")
    if D == 1:
        return T
    if D == 2:
        return (sp.kron(I, T) + sp.kron(T, I)).tocsr()
    if D == 3:
        return (sp.kron(I, sp.kron(I, T)) + sp.kron(I, sp.kron(T, I))
                + sp.kron(T, sp.kron(I, I))).tocsr()
    raise ValueError("D must be 1, 2 or 3")


def helmholtz_matrix(D: int, n: int, h: float, k: float) -> sp.csr_matrix:
    """B(k) = Delta_h + k^2 I on the interior unknowns (Dirichlet case of Section 2.4)."""
    return (laplacian_matrix(D, n, h) + (k * k) * sp.identity(n ** D, format="csr")).tocsr()


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------

def dirichlet_eigenvalues_1d(n: int, h: float) -> np.ndarray:
    """Eigenvalues lambda_m (m = 1..n) of -[1, -2, 1]/h^2 with Dirichlet ends:
    (4/h^2) sin^2(m pi / (2 (n+1))); eigenvector i -> sin(m pi i / (n+1))."""
    m = np.arange(1, n + 1, dtype=np.float64)
    return (4.0 / (h * h)) * np.sin(m * math.pi / (2.0 * (n + 1))) ** 2


def lambda_min(D: int, n: int, h: float) -> float:
    """Smallest eigenvalue of -Delta_h (all D modes at m = 1)."""
    return D * (4.0 / (h * h)) * math.sin(math.pi / (2.0 * (n + 1))) ** 2


def k_max(D: int, n: int, h: float) -> float:
    """Largest k for which the alpha = k^2 iteration converges (Section 2.4): the
    iteration matrix for the Dirichlet cavity is G = -k^2 Delta_h^{-1}, symmetric with
    spectral radius k^2 / lambda_min, and the geometric series converges iff < 1."""
    return math.sqrt(lambda_min(D, n, h))


def rho_pred(D: int, n: int, h: float, k: float) -> float:
    """Spectral radius of G = -k^2 Delta_h^{-1}."""
    return k * k / lambda_min(D, n, h)


def discrete_wavenumber(k: float, h: float, direction) -> float:
    """kappa with sum_d (4/h^2) sin^2(kappa d_d h / 2) = k^2, so that exp(i kappa d.x)
    satisfies (Delta_h + k^2) u = 0 exactly at every node.  Solved by bisection on
    [0, k * pi/2] (the left side is increasing there and exceeds k^2 at the right end
    for the resolutions used, kappa h d_d < pi)."""
    d = np.asarray(direction, dtype=np.float64)

    def F(kap):
        return np.sum((4.0 / (h * h)) * np.sin(kap * d * h / 2.0) ** 2) - k * k

    lo, hi = 0.0, k * math.pi / 2.0
    if F(hi) < 0:
        raise ValueError("k too large for the grid")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if F(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def sine_mode(D: int, n: int, modes) -> np.ndarray:
    """Interior array prod_d sin(m_d pi i_d / (n+1)) (a discrete Dirichlet eigenvector)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    vecs = [np.sin(m * math.pi * i / (n + 1)) for m in modes]
    if D == 2:
        return np.einsum("y,x->yx", vecs[1], vecs[0])
    return np.einsum("z,y,x->zyx", vecs[2], vecs[1], vecs[0])


def sine_mode_eigenvalue(D: int, n: int, h: float, modes) -> float:
    """lambda_h(m) = sum_d (4/h^2) sin^2(m_d pi / (2(n+1))); Delta_h mode = -lambda mode."""
    return float(sum((4.0 / (h * h)) * math.sin(m * math.pi / (2.0 * (n + 1))) ** 2 for m in modes))


# ---------------------------------------------------------------------------
# Exact discrete solutions
# ---------------------------------------------------------------------------

def solve_exact_splu(f: np.ndarray, g: np.ndarray, h: float, k: float) -> np.ndarray:
    """Unique solution of B(k) u = b by sparse LU; returns the padded u (ring = g)."""
    D, n = f.ndim, f.shape[0]
    b = lifted_rhs(f, g, h).reshape(-1)
    A = helmholtz_matrix(D, n, h, k).astype(np.complex128).tocsc()
    x = spla.splu(A).solve(b)
    return padded_from(x.reshape(f.shape), g.astype(np.complex128))


def _dst_eigs(D: int, n: int, h: float) -> np.ndarray:
    lam = dirichlet_eigenvalues_1d(n, h)
    if D == 2:
        return lam[:, None] + lam[None, :]
    return lam[:, None, None] + lam[None, :, None] + lam[None, None, :]


def dst_poisson(r: np.ndarray, h: float, workers: int | None = None) -> np.ndarray:
    """Exact solution e of Delta_h e = r with e = 0 on the wall (interior arrays),
    through the sine basis that diagonalises Delta_h: e^ = r^ / (-lambda_m)."""
    lam = _dst_eigs(r.ndim, r.shape[0], h)
    rh = scipy.fft.dstn(r, type=1, workers=workers)
    return scipy.fft.idstn(rh / (-lam), type=1, workers=workers)


def solve_exact_dst(f: np.ndarray, g: np.ndarray, h: float, k: float,
                    workers: int | None = None) -> np.ndarray:
    """Unique solution of B(k) u = b through the sine basis: u^ = b^ / (k^2 - lambda_m)."""
    D = f.ndim
    lam = _dst_eigs(D, f.shape[0], h)
    b = lifted_rhs(f, g, h)
    bh = scipy.fft.dstn(b, type=1, workers=workers)
    x = scipy.fft.idstn(bh / (k * k - lam), type=1, workers=workers)
    return padded_from(x, g.astype(np.complex128))


class SparsePoisson:
    """Direct solver of Delta_h e = r (hom. Dirichlet) for real right-hand sides:
    one sparse LU factorisation of the real matrix, reused for every solve."""

    def __init__(self, D: int, n: int, h: float):
        self.shape = (n,) * D
        self.lu = spla.splu(laplacian_matrix(D, n, h).tocsc())

    def __call__(self, r: np.ndarray) -> np.ndarray:
        assert np.isrealobj(r)
        return self.lu.solve(np.ascontiguousarray(r, dtype=np.float64).reshape(-1)).reshape(self.shape)


class DSTPoisson:
    """Direct solver of Delta_h e = r (hom. Dirichlet) through the sine basis."""

    def __init__(self, D: int, n: int, h: float, workers: int | None = None):
        self.h = h
        self.workers = workers

    def __call__(self, r: np.ndarray) -> np.ndarray:
        return dst_poisson(r, self.h, self.workers)
