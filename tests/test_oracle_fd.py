"""Pins for oracle/fd.py against facts fixed by mathematics and the paper.

None of these re-types the oracle's formula: each compares it with an independent
route (exact polynomial identities, dense eigen-decomposition, a second exact solver,
the discrete plane wave, hand-worked examples, brute-force loops).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fd
from paper_2308_11469_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("D", [2, 3])
def test_stencil_exact_on_quadratics(D):
    # The 2nd-order central difference is exact on quadratics:
    # Delta(x^2 + 3 y^2 [- z^2]) = 2 + 6 [- 2].
    n, h = 7, 0.13
    xs = inputs.node_coords(D, n, h)
    if D == 2:
        U = xs[0] ** 2 + 3 * xs[1] ** 2
        expect = 8.0
    else:
        U = xs[0] ** 2 + 3 * xs[1] ** 2 - xs[2] ** 2
        expect = 6.0
    L = fd.apply_laplacian(U, h)
    assert np.allclose(L, expect, rtol=0, atol=1e-10)


@pytest.mark.parametrize("D", [2, 3])
def test_sine_modes_are_eigenvectors(D):
    n = 9
    h = 1.0 / (n + 1)
    for modes in [(1,) * D, (2, 5, 3)[:D], (n,) * D, (4, 1, 7)[:D]]:
        s = fd.sine_mode(D, n, modes)
        lam = fd.sine_mode_eigenvalue(D, n, h, modes)
        L = fd.apply_laplacian(fd.padded_from(s), h)
        assert np.allclose(L, -lam * s, rtol=0, atol=1e-9 * lam)


@pytest.mark.parametrize("D,n", [(2, 7), (3, 5), (2, 6)])
def test_lambda_min_against_dense_eigensolver(D, n):
    h = 1.0 / (n + 1)
    A = -fd.laplacian_matrix(D, n, h).toarray()
    ev = np.linalg.eigvalsh(A)
    assert abs(ev[0] - fd.lambda_min(D, n, h)) < 1e-10 * ev[-1]
    # every eigenvalue is a sum of 1D Dirichlet eigenvalues
    lam1 = fd.dirichlet_eigenvalues_1d(n, h)
    grids = np.meshgrid(*([lam1] * D), indexing="ij")
    sums = np.sort(sum(grids).ravel())
    assert np.allclose(np.sort(ev), sums, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("D", [2, 3])
def test_matrix_matches_stencil(D):
    n, h = 6, 0.2
    x = _rand_c(_rng(1), (n,) * D)
    M = fd.laplacian_matrix(D, n, h)
    via_matrix = (M @ x.reshape(-1)).reshape(x.shape)
    via_stencil = fd.apply_laplacian(fd.padded_from(x), h)
    assert np.allclose(via_matrix, via_stencil, rtol=1e-13, atol=1e-12)


def test_lifting_brute_force_2d():
    # b = f - (sum of wall neighbours)/h^2, by explicit loops
    n, h = 4, 0.2
    rng = _rng(2)
    f = _rand_c(rng, (n, n))
    g = _rand_c(rng, (n + 2, n + 2))
    b = fd.lifted_rhs(f, g, h)
    for j in range(1, n + 1):
        for i in range(1, n + 1):
            acc = f[j - 1, i - 1]
            for (jj, ii) in [(j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)]:
                if ii in (0, n + 1) or jj in (0, n + 1):
                    acc -= g[jj, ii] / (h * h)
            assert abs(acc - b[j - 1, i - 1]) < 1e-12 * (1 + abs(acc))


@pytest.mark.parametrize("D,n", [(2, 15), (3, 7), (2, 16)])
def test_splu_and_dst_agree(D, n):
    h = 1.0 / (n + 1)
    rng = _rng(3)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    k = 0.7 * fd.k_max(D, n, h)
    u1 = fd.solve_exact_splu(f, g, h, k)
    u2 = fd.solve_exact_dst(f, g, h, k)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u1)
    r = fd.residual(u1, f, h, k)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(f)


@pytest.mark.parametrize("D,n,k", [(2, 63, 2.0), (2, 31, 4.0), (3, 15, 4.0), (3, 15, 9.0)])
def test_discrete_plane_wave_is_reproduced(D, n, k):
    # exp(i kappa d.x) with the discrete dispersion relation solves (Delta_h + k^2) u = 0
    # at every node, so with f = 0 and that wall data the exact solution is the wave
    # itself (k = 9 > k_max on 15^3 still has a unique solution: the system is
    # uniquely solvable away from resonances, the iteration is not needed here).
    h = 1.0 / (n + 1)
    rng = _rng(4)
    d = inputs.random_direction(D, rng)
    kap = fd.discrete_wavenumber(k, h, d)
    w = inputs.plane_wave(D, n, h, kap, d)
    assert np.max(np.abs(fd.apply_helmholtz(w, h, k))) < 1e-9 * k * k
    f = np.zeros((n,) * D, dtype=np.complex128)
    u = fd.solve_exact_dst(f, w, h, k)
    assert np.max(np.abs(u - w)) < 1e-12


def test_continuum_plane_wave_second_order():
    # Unit square, f = 0, g = exp(i k (cos pi/6 x + sin pi/6 y)), k = 2 (the 63^2 case):
    # the FD solution approaches the continuum wave at O(h^2).
    errs = []
    for n in (63, 127):
        p = inputs.plane_wave_cavity_2d(2.0, n=n)
        u = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
        exact = inputs.plane_wave(2, n, p.h, p.k, p.meta["direction"])
        errs.append(np.max(np.abs(u - exact)))
    ratio = errs[0] / errs[1]
    assert 3.5 <= ratio <= 4.5, ratio
    assert 1e-5 < errs[0] < 3e-5


@pytest.mark.parametrize("D,n,modes", [(2, 31, (1, 2)), (3, 15, (1, 2, 1)), (2, 20, (3, 5))])
def test_manufactured_sine(D, n, modes):
    h = 1.0 / (n + 1)
    k = 3.3
    f = fd.sine_mode(D, n, modes).astype(np.complex128)
    g = np.zeros((n + 2,) * D, dtype=np.complex128)
    lam = fd.sine_mode_eigenvalue(D, n, h, modes)
    u = fd.solve_exact_splu(f, g, h, k)
    assert np.max(np.abs(fd.interior(u) - f / (k * k - lam))) < 1e-12 * np.max(np.abs(f / (k * k - lam)))


def test_kmax_values_and_limits():
    assert abs(fd.k_max(2, 63, 1 / 64) - 4.442437) < 2e-6
    assert abs(fd.k_max(2, 1023, 1 / 1024) - 4.442881) < 2e-6
    assert abs(fd.k_max(3, 255, 1 / 256) - 5.441364) < 2e-6
    # continuum limits pi*sqrt(D) of the unit square / cube (first Dirichlet eigenvalue)
    assert abs(fd.k_max(2, 2 ** 14 - 1, 2.0 ** -14) - math.pi * math.sqrt(2)) < 1e-7
    assert abs(fd.k_max(3, 2 ** 14 - 1, 2.0 ** -14) - math.pi * math.sqrt(3)) < 1e-7
    # scaling with the domain side l (Section 3: first-exit times scale with l^2, so the
    # admissible wave numbers scale with 1/l); exact for the discrete operator
    for l in (0.5, 2.0, 3.7):
        assert abs(fd.k_max(2, 63, l / 64) - fd.k_max(2, 63, 1 / 64) / l) < 1e-12
    # rho for the config-1 wave numbers
    assert abs(fd.rho_pred(2, 63, 1 / 64, 2.0) - 0.2027) < 1e-4
    assert abs(fd.rho_pred(2, 63, 1 / 64, 5.0) - 1.2667) < 1e-4


def _golden_case(c):
    D, n, h = c["D"], c["n"], c["h"]
    f = np.full((1,) * D, complex(*c["f"]))
    g = np.zeros((3,) * D, dtype=np.complex128)
    if D == 2:
        g[1, 0] = complex(*c["ring"]["west"])
        g[1, 2] = complex(*c["ring"]["east"])
        g[0, 1] = complex(*c["ring"]["south"])
        g[2, 1] = complex(*c["ring"]["north"])
    else:
        v = complex(*c["ring"]["all_faces"])
        for idx in [(1, 1, 0), (1, 1, 2), (1, 0, 1), (1, 2, 1), (0, 1, 1), (2, 1, 1)]:
            g[idx] = v
    return D, n, h, c["k"], f, g


def test_hand_worked_one_node_examples():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        D, n, h, k, f, g = _golden_case(c)
        for solver in (fd.solve_exact_splu, fd.solve_exact_dst):
            u = solver(f, g, h, k)
            assert abs(u[(1,) * D] - complex(*c["u_exact"])) < 1e-14
        assert abs(fd.rho_pred(D, n, h, k) - c["rho"]) < 1e-15
