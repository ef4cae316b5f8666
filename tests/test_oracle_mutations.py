"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case monkeypatches one plausible slip into oracle code -- a dropped term, a wrong
sign, a wrong scale, a swapped axis -- and checks that at least one of the pin checks
below fails, while all of them pass on the unmodified oracle.
"""
import math

import numpy as np
import pytest

from oracle import exit_time as ex, fd, general as gen, iteration as it, multigrid as mg
from paper_2308_11469_gb300 import inputs


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def pin_quadratic():
    n, h = 7, 0.13
    xs = inputs.node_coords(3, n, h)
    L = fd.apply_laplacian(xs[0] ** 2 + 3 * xs[1] ** 2 - xs[2] ** 2, h)
    return np.allclose(L, 6.0, atol=1e-10)


def pin_plane_wave():
    D, n, k = 2, 31, 3.0
    h = 1.0 / (n + 1)
    d = (0.6, 0.8)
    kap = fd.discrete_wavenumber(k, h, d)
    w = inputs.plane_wave(D, n, h, kap, d)
    u = fd.solve_exact_splu(np.zeros((n, n), complex), w, h, k)
    return (np.max(np.abs(u - w)) < 1e-12
            and np.max(np.abs(fd.apply_helmholtz(w, h, k))) < 1e-9 * k * k)


def pin_hand_relres():
    # one interior node, worked by hand: relres_N = 16^-N, u^(1) = (11 + 10i)/16
    f = np.full((1, 1), 1 + 2j)
    g = np.zeros((3, 3), complex)
    g[1, 0], g[1, 2], g[0, 1], g[2, 1] = 1, 2j, -1, 3 + 1j
    res = it.paper_iteration(f, g, 0.5, 1.0, tol=1e-300, max_outer=3, keep_iterates=True)
    return (abs(res.iterates[1][1, 1] - (11 + 10j) / 16) < 1e-15
            and np.allclose(res.relres, [1, 1 / 16, 1 / 256, 1 / 4096], rtol=1e-14, atol=0))


def pin_partial_sums():
    D, n = 2, 5
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    f = _rand_c(rng, (n, n))
    g = _rand_c(rng, (n + 2, n + 2))
    k = 0.8 * math.sqrt(2 * 4 / h ** 2 * math.sin(math.pi / (2 * (n + 1))) ** 2)
    # the matrix series built from scratch here (no oracle helper)
    A = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            p = j * n + i
            A[p, p] = -4 / h ** 2
            for jj, ii in [(j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)]:
                if 0 <= ii < n and 0 <= jj < n:
                    A[p, jj * n + ii] = 1 / h ** 2
    b = f.copy()
    b[:, 0] -= g[1:-1, 0] / h ** 2
    b[:, -1] -= g[1:-1, -1] / h ** 2
    b[0, :] -= g[0, 1:-1] / h ** 2
    b[-1, :] -= g[-1, 1:-1] / h ** 2
    Ainv = np.linalg.inv(A)
    term = Ainv @ b.reshape(-1)
    partial = np.zeros_like(term)
    res = it.paper_iteration(f, g, h, k, tol=1e-300, max_outer=6, keep_iterates=True)
    for N in range(1, 7):
        partial = partial + term
        term = -(k * k) * (Ainv @ term)
        if np.linalg.norm(fd.interior(res.iterates[N]).reshape(-1) - partial) > 1e-12 * np.linalg.norm(partial):
            return False
    return True


def pin_sine_eigen():
    n = 9
    h = 1.0 / (n + 1)
    s = fd.sine_mode(2, n, (2, 5))
    lam = (4 / h ** 2) * (math.sin(2 * math.pi / 20) ** 2 + math.sin(5 * math.pi / 20) ** 2)
    return np.allclose(fd.apply_laplacian(fd.padded_from(s), h), -lam * s, atol=1e-9 * lam)


def pin_vcycle():
    n = 31
    h = 1.0 / (n + 1)
    r = _rand_c(np.random.default_rng(4), (n, n))
    exact = fd.dst_poisson(r, h)
    E = np.zeros((n + 2, n + 2), complex)
    for _ in range(14):
        mg.vcycle(E, r, h)
    return np.linalg.norm(fd.interior(E) - exact) < 1e-10 * np.linalg.norm(exact)


def pin_kmax():
    return abs(fd.k_max(2, 2 ** 12 - 1, 2.0 ** -12) - math.pi * math.sqrt(2)) < 1e-6


def pin_general_hand():
    # one interior node, alpha = 3, p = 2, k = 1, h = 1/2 (worked by hand):
    # u^(1) = (6 + 5i)/18, relres_N = (sqrt(13)/18)^N, rho = sqrt(13)/18
    f = np.full((1, 1), 2 - 1j)
    g = np.full((3, 3), 0.5 + 0.25j)
    res = gen.general_iteration(f, g, 0.5, 1.0, 3.0, 2.0, tol=1e-300, max_outer=3, keep_iterates=True)
    q = math.sqrt(13) / 18
    return (abs(res.iterates[1][1, 1] - (6 + 5j) / 18) < 1e-15
            and np.allclose(res.relres, [1, q, q * q, q ** 3], rtol=1e-13, atol=0)
            and abs(gen.rho_pred(2, 1, 0.5, 1.0, 3.0, 2.0) - q) < 1e-15)


def pin_general_series():
    # partial sums of G = -(alpha + i p)(Delta_h - sigma)^{-1}, matrices built here
    n, h, k, alpha, p = 4, 0.2, 1.0, 4.0, 3.0
    rng = np.random.default_rng(6)
    f = _rand_c(rng, (n, n))
    g = fd.padded_from(np.zeros((n, n), complex), _rand_c(rng, (n + 2, n + 2)))
    T = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2
    M = np.kron(np.eye(n), T) + np.kron(T, np.eye(n)) - (alpha - k * k) * np.eye(n * n)
    Minv = np.linalg.inv(M)
    b = fd.lifted_rhs(f, g, h).reshape(-1)
    res = gen.general_iteration(f, g, h, k, alpha, p, tol=1e-300, max_outer=5, keep_iterates=True)
    term, acc = Minv @ b, 0
    for N in range(1, 6):
        acc = acc + term
        term = -(alpha + 1j * p) * (Minv @ term)
        if np.linalg.norm(fd.interior(res.iterates[N]).reshape(-1) - acc) > 1e-12 * np.linalg.norm(acc):
            return False
    return True


def pin_exit_time():
    # one node by hand (E = h^2/4 = 1/16 -> k_*^C = 4) and the square's continuum maximum
    # 0.0736713... (torsion series, written out here) approached at O(h^2)
    s = 0.125 - sum(4.0 * (-1) ** j / (math.pi ** 3 * (2 * j + 1) ** 3 * math.cosh((2 * j + 1) * math.pi / 2))
                    for j in range(20))
    e1 = abs(ex.max_exit_time(2, 63, 1 / 64) - s)
    e2 = abs(ex.max_exit_time(2, 127, 1 / 128) - s)
    return (abs(ex.k_star_c(2, 1, 0.5) - 4.0) < 1e-14 and 3.5 < e1 / e2 < 4.5 and e2 < 5e-6)


PINS = [pin_quadratic, pin_plane_wave, pin_hand_relres, pin_partial_sums, pin_sine_eigen,
        pin_vcycle, pin_kmax, pin_general_hand, pin_general_series, pin_exit_time]


def test_pins_pass_on_the_oracle():
    assert all(p() for p in PINS)


def _laplacian_no_minus_two(U, h):
    c = fd.interior(U)
    out = np.zeros(c.shape, dtype=np.result_type(U.dtype, np.float64))
    for a in range(U.ndim):
        out += (fd._shift(U, a, +1) - c + fd._shift(U, a, -1))
    return out / (h * h)


def _laplacian_one_axis_dropped(U, h):
    c = fd.interior(U)
    out = np.zeros(c.shape, dtype=np.result_type(U.dtype, np.float64))
    for a in range(U.ndim - 1):
        out += (fd._shift(U, a, +1) - 2 * c + fd._shift(U, a, -1))
    return out / (h * h)


def _helmholtz_wrong_sign(U, h, k):
    return fd.apply_laplacian(U, h) - (k * k) * fd.interior(U)


def _lifting_wrong_sign(f, g, h):
    return f + fd.apply_laplacian(fd.ring_only(g), h)


def _lambda_min_wrong_scale(D, n, h):
    return D * (4.0 / (h * h)) * math.sin(math.pi / (n + 1)) ** 2


def _eigenvalues_off_by_one(n, h):
    m = np.arange(0, n, dtype=np.float64)
    return (4.0 / (h * h)) * np.sin(m * math.pi / (2.0 * (n + 1))) ** 2


def _restrict_unweighted(rf):
    D = rf.ndim
    return rf[(slice(1, None, 2),) * D].copy()


def _half_sweep_wrong_h(E, r, h, color, sigma=0.0):
    D = E.ndim
    n = E.shape[0] - 2
    nbr = np.zeros(r.shape, dtype=E.dtype)
    for a in range(D):
        nbr = nbr + fd._shift(E, a, +1) + fd._shift(E, a, -1)
    new = (nbr - h * r) / (2.0 * D + sigma * h * h)
    mask = mg.color_mask(D, n, color)
    E[(slice(1, -1),) * D][mask] = new[mask]


def _damping_wrong_sign(U, h, k, p):
    return fd.apply_laplacian(U, h) + (k * k - 1j * p) * fd.interior(U)


def _shift_dropped(D, n, h, sigma):
    return fd.laplacian_matrix(D, n, h)


def _rho_without_hypot(D, n, h, k, alpha, p):
    return (alpha + p) / (fd.lambda_min(D, n, h) + alpha - k * k)


def _exit_time_wrong_source(D, n, h):
    return np.real(fd.dst_poisson(-2.0 * np.ones((n,) * D), h))


def _k_star_without_inverse(D, n, h, p=0.0):
    q = ex.max_exit_time(D, n, h) - p
    return math.sqrt(q) if q > 0 else 0.0


MUTATIONS = [
    (ex, "exit_time", _exit_time_wrong_source),
    (ex, "k_star_c", _k_star_without_inverse),
    (gen, "apply_damped_helmholtz", _damping_wrong_sign),
    (gen, "shifted_laplacian_matrix", _shift_dropped),
    (gen, "rho_pred", _rho_without_hypot),
    (fd, "apply_laplacian", _laplacian_no_minus_two),
    (fd, "apply_laplacian", _laplacian_one_axis_dropped),
    (fd, "apply_helmholtz", _helmholtz_wrong_sign),
    (fd, "lifted_rhs", _lifting_wrong_sign),
    (fd, "lambda_min", _lambda_min_wrong_scale),
    (fd, "dirichlet_eigenvalues_1d", _eigenvalues_off_by_one),
    (mg, "restrict_fw", _restrict_unweighted),
    (mg, "rbgs_half_sweep", _half_sweep_wrong_h),
]


@pytest.mark.parametrize("mod,name,bad", MUTATIONS, ids=[m[2].__name__ for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, mod, name, bad):
    monkeypatch.setattr(mod, name, bad)
    results = []
    for p in PINS:
        try:
            results.append(bool(p()))
        except Exception:
            results.append(False)
    assert not all(results), f"mutation {bad.__name__} escaped every pin"


def test_planted_iteration_sign_is_caught(monkeypatch):
    # v_n = Delta^{-1}(+k^2 v_{n-1}) instead of -k^2: the iterates stop matching the series
    orig = it.paper_iteration

    def wrong(f, g, h, k, **kw):
        return orig(f, g, h, 1j * k, **kw)   # k^2 -> -k^2 everywhere in the recursion
    monkeypatch.setattr(it, "paper_iteration", wrong)
    try:
        ok = pin_partial_sums()
    except Exception:
        ok = False
    assert not ok
