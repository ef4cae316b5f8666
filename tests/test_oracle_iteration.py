"""Pins for oracle/iteration.py: the paper's nested iteration with exact inner solves.

Independent routes: the dense matrix geometric series of Section 2.4 built with
numpy's dense inverse, hand-worked one-node examples, the k_max invariant, the
discrete plane wave, and the exact discrete solution.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fd, iteration as it
from paper_2308_11469_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("D,n", [(2, 3), (2, 5), (2, 7), (3, 3), (3, 5)])
def test_iterates_are_partial_sums_of_the_geometric_series(D, n):
    # Section 2.4: increments obey u_n = G u_{n-1}, G = -k^2 A^{-1} (A = Delta_h with the
    # Dirichlet nodes eliminated), u_0 = A^{-1} b, so u^(N) = sum_{j<N} G^j A^{-1} b.
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(10 + n + D)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    k = 0.8 * fd.k_max(D, n, h)
    A = fd.laplacian_matrix(D, n, h).toarray()
    Ainv = np.linalg.inv(A)
    G = -(k * k) * Ainv
    b = fd.lifted_rhs(f, g, h).reshape(-1)
    res = it.paper_iteration(f, g, h, k, tol=1e-300, max_outer=12, keep_iterates=True)
    assert res.status == it.MAXITER and res.iters == 12
    term = Ainv @ b
    partial = np.zeros_like(term)
    for N in range(1, 13):
        partial = partial + term
        term = G @ term
        got = fd.interior(res.iterates[N]).reshape(-1)
        assert np.linalg.norm(got - partial) <= 1e-13 * np.linalg.norm(partial), N
        # the wall ring always carries g
        ring = res.iterates[N].copy()
        ring[(slice(1, -1),) * D] = 0
        assert np.array_equal(ring, fd.ring_only(g))


def test_residual_contracts_by_rho():
    # r_{N+1} = G r_N with G symmetric, so ||r_{N+1}|| <= rho ||r_N||, ratio -> rho.
    D, n = 2, 31
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(5)
    f = _rand_c(rng, (n, n))
    g = np.zeros((n + 2, n + 2), dtype=np.complex128)
    k = 0.9 * fd.k_max(D, n, h)
    rho = fd.rho_pred(D, n, h, k)
    res = it.paper_iteration(f, g, h, k, tol=1e-300, max_outer=80)
    rr = np.asarray(res.relres)
    ratios = rr[1:] / rr[:-1]
    # the residual of the partial sum is evaluated in floating point; keep to steps whose
    # residual is far above its rounding floor (|Delta_h u| ~ 8/h^2 |u|)
    clean = rr[1:] > 1e-6
    assert clean.sum() > 40
    assert np.all(ratios[clean] <= rho * (1 + 1e-6))
    assert abs(ratios[clean][-1] - rho) < 1e-4


@pytest.mark.parametrize("D,n", [(2, 15), (3, 7)])
def test_converges_below_kmax_diverges_above(D, n):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(6)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    km = fd.k_max(D, n, h)
    lo = it.paper_iteration(f, g, h, 0.95 * km, tol=1e-8, max_outer=2000)
    hi = it.paper_iteration(f, g, h, 1.05 * km, tol=1e-8, max_outer=2000)
    assert lo.status == it.CONVERGED == it.predicted_status(D, n, h, 0.95 * km)
    assert hi.status == it.DIVERGED == it.predicted_status(D, n, h, 1.05 * km)


def test_plane_wave_cavity_63():
    # The 63^2 unit-square cavity: k = 2 converges (rho = 0.203), reproducing the
    # continuum plane wave to O(h^2); k = 5 > k_max = 4.4424 diverges.
    p = inputs.plane_wave_cavity_2d(2.0)
    res = it.paper_iteration(p.f, p.g, p.h, p.k, tol=1e-10, max_outer=200)
    assert res.status == it.CONVERGED
    assert res.iters == 12
    exact_cont = inputs.plane_wave(2, p.n, p.h, p.k, p.meta["direction"])
    err = np.max(np.abs(res.u - exact_cont))
    assert 1.5e-5 < err < 2.0e-5
    # relres 5e-11 leaves an error ~65x larger (the low modes of A_H^{-1} amplify it)
    ex = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
    assert np.linalg.norm(res.u - ex) <= 1e-8 * np.linalg.norm(ex)
    tight = it.paper_iteration(p.f, p.g, p.h, p.k, tol=1e-14, max_outer=200)
    assert np.linalg.norm(tight.u - ex) <= 1e-12 * np.linalg.norm(ex)
    p5 = inputs.plane_wave_cavity_2d(5.0)
    res5 = it.paper_iteration(p5.f, p5.g, p5.h, p5.k, tol=1e-10, max_outer=400)
    assert res5.status == it.DIVERGED
    # caught by the growth rule: ten non-decreasing steps once N >= 20 (rho = 1.267)
    assert res5.iters == 20
    assert all(b >= a for a, b in zip(res5.relres[-11:-1], res5.relres[-10:]))


def test_discrete_plane_wave_fixed_point():
    D, n, k = 2, 31, 3.0
    h = 1.0 / (n + 1)
    d = (0.6, 0.8)
    kap = fd.discrete_wavenumber(k, h, d)
    w = inputs.plane_wave(D, n, h, kap, d)
    f = np.zeros((n, n), dtype=np.complex128)
    res = it.paper_iteration(f, w, h, k, tol=1e-14, max_outer=500)
    assert res.status == it.CONVERGED
    assert np.max(np.abs(res.u - w)) < 1e-12


def test_real_data_gives_real_iterates_and_linearity():
    D, n = 2, 15
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(7)
    fr = rng.standard_normal((n, n)).astype(np.complex128)
    gr = rng.standard_normal((n + 2, n + 2)).astype(np.complex128)
    k = 2.5
    a = it.paper_iteration(fr, gr, h, k, tol=1e-300, max_outer=6)
    assert np.max(np.abs(a.u.imag)) == 0.0
    f2 = _rand_c(rng, (n, n))
    g2 = _rand_c(rng, (n + 2, n + 2))
    b = it.paper_iteration(f2, g2, h, k, tol=1e-300, max_outer=6)
    c = it.paper_iteration(fr + 2j * f2, gr + 2j * g2, h, k, tol=1e-300, max_outer=6)
    assert np.linalg.norm(c.u - (a.u + 2j * b.u)) <= 1e-12 * np.linalg.norm(c.u)


def test_splu_and_dst_iterations_agree():
    D, n = 3, 7
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(8)
    f = _rand_c(rng, (n,) * D)
    g = _rand_c(rng, (n + 2,) * D)
    a = it.paper_iteration(f, g, h, 3.0, tol=1e-10, poisson="splu")
    b = it.paper_iteration(f, g, h, 3.0, tol=1e-10, poisson="dst")
    assert a.iters == b.iters
    assert np.linalg.norm(a.u - b.u) <= 1e-12 * np.linalg.norm(a.u)
    assert np.allclose(a.relres, b.relres, rtol=1e-6, atol=1e-13)


def test_hand_worked_iterates():
    from tests.test_oracle_fd import _golden_case
    for c in json.load(open(GOLDEN))["cases"]:
        D, n, h, k, f, g = _golden_case(c)
        res = it.paper_iteration(f, g, h, k, tol=1e-300, max_outer=3, keep_iterates=True)
        ctr = (1,) * D
        assert abs(res.iterates[1][ctr] - complex(*c["u1"])) < 1e-15
        assert abs(res.iterates[2][ctr] - complex(*c["u2"])) < 1e-15
        for N, rr in enumerate(c["relres_first"]):
            assert abs(res.relres[N] - rr) < 1e-15 * max(1.0, rr) + 1e-17


def test_status_rule():
    r = it.StatusRule(1e-8, 50)
    assert r(0, 1.0) is None
    assert r(1, float("nan")) == it.NONFINITE
    r = it.StatusRule(1e-8, 50)
    assert r(0, 1.0) is None and r(1, 1e-9) == it.CONVERGED
    r = it.StatusRule(1e-8, 50)
    assert r(0, 1.0) is None and r(1, 2e4) == it.DIVERGED
    # slow growth: ten non-decreasing steps after step 20
    r = it.StatusRule(1e-8, 1000)
    out = [r(N, 0.5 * 1.001 ** N if N > 5 else 1.0 / (N + 1)) for N in range(40)]
    first = next(i for i, s in enumerate(out) if s is not None)
    assert out[first] == it.DIVERGED and first == 20
    r = it.StatusRule(1e-8, 3)
    assert [r(N, 0.5 ** N) for N in range(4)] == [None, None, None, it.MAXITER]
    # stagnation at a floor (non-decreasing, but within 2x of the minimum) is not divergence
    r = it.StatusRule(1e-12, 100)
    vals = [1.0, 1e-3, 1e-6, 1e-9] + [1.1e-9 + 1e-12 * N for N in range(4, 101)]
    out = [r(N, v) for N, v in enumerate(vals)]
    assert [s for s in out if s is not None] == [it.MAXITER]


def test_zero_data_is_converged_immediately():
    n = 7
    f = np.zeros((n, n), dtype=np.complex128)
    g = np.zeros((n + 2, n + 2), dtype=np.complex128)
    res = it.paper_iteration(f, g, 1 / 8, 2.0)
    assert res.status == it.CONVERGED and res.iters == 0 and res.relres == [0.0]
