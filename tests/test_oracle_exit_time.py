"""Pins of the mean-exit-time oracle (Eq. (2.10)) and of k_*^C (Eq. (2.9)).

Fixed by: the one-node grids worked by hand, the continuum torsion-function series
(two independent forms for the square) with O(h^2) convergence of the discrete maxima,
the maximum principle against the strip / prism solutions, exactness of Delta_h on the
1D quadratic, scaling with the domain side, and k_*^C <= k_max (1/lambda_min <= max E).
"""
import math

import numpy as np
import pytest

from oracle import exit_time as ex, fd


def test_one_node_grids_by_hand():
    # n = 1, h = 1/2: -(2D/h^2) E = -1 -> E = h^2/(2D): 1/16 (square), 1/24 (cube)
    assert ex.max_exit_time(2, 1, 0.5) == pytest.approx(1 / 16, abs=1e-16)
    assert ex.max_exit_time(3, 1, 0.5) == pytest.approx(1 / 24, abs=1e-16)
    assert ex.k_star_c(2, 1, 0.5) == pytest.approx(4.0, rel=1e-15)
    assert ex.k_star_c(2, 1, 0.5, p=7.0) == pytest.approx(3.0, rel=1e-15)
    assert ex.k_star_c(3, 1, 0.5, p=30.0) == 0.0


def test_the_two_square_series_agree():
    a = ex.square_center_cosh_series()
    b = ex.square_center_sine_series(600)
    assert a == pytest.approx(b, abs=2e-6)          # the double series converges slowly
    assert 0.0736 < a < 0.0738


@pytest.mark.parametrize("D,ref", [(2, ex.square_center_cosh_series), (3, ex.cube_center_series)])
def test_discrete_maximum_converges_at_second_order(D, ref):
    ns = (63, 127) if D == 2 else (31, 63)
    E = ref()
    errs = [abs(ex.max_exit_time(D, n, 1.0 / (n + 1)) - E) for n in ns]
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio
    assert errs[1] < (5e-6 if D == 2 else 3e-5)
    # k_*^C of the unit square and cube
    kc = ex.k_star_c(D, ns[1], 1.0 / (ns[1] + 1))
    assert kc == pytest.approx(1 / math.sqrt(E), rel=2e-4)
    assert kc == pytest.approx(3.684 if D == 2 else 4.218, abs=2e-3)


def test_maximum_principle_bounds():
    # the square's E lies below the strip solution x(1-x)/2 (max 1/8), the cube's below
    # the square prism's (its 2D maximum), all three being positive inside
    n = 31
    h = 1.0 / (n + 1)
    E2 = ex.exit_time(2, n, h)
    E3 = ex.exit_time(3, n, h)
    assert np.all(E2 > 0) and np.all(E3 > 0)
    assert np.max(E2) < 0.125
    assert np.max(E3) < np.max(E2)


def test_strip_solution_is_exact_in_1d():
    # Delta_h is exact on quadratics: in 1D E_h(x_i) = x_i (1 - x_i) / 2 to rounding
    n = 15
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    T = fd.laplacian_1d(n, h).toarray()
    E = np.linalg.solve(T, -np.ones(n))
    assert np.allclose(E, x * (1 - x) / 2, atol=1e-14)


def test_symmetric_and_maximal_at_the_centre():
    n = 31
    h = 1.0 / (n + 1)
    E = ex.exit_time(2, n, h)
    assert np.allclose(E, E[::-1, :], atol=1e-15) and np.allclose(E, E.T, atol=1e-15)
    c = n // 2
    assert E[c, c] == np.max(E)


def test_scaling_with_the_domain_side():
    # side l: E scales by l^2, k_*^C by 1/l
    n, l = 31, 2.5
    h = 1.0 / (n + 1)
    assert ex.max_exit_time(2, n, l * h) == pytest.approx(l * l * ex.max_exit_time(2, n, h), rel=1e-12)
    assert ex.k_star_c(2, n, l * h) == pytest.approx(ex.k_star_c(2, n, h) / l, rel=1e-12)


@pytest.mark.parametrize("D,n", [(2, 31), (2, 127), (3, 31)])
def test_sufficient_bound_is_below_k_max(D, n):
    # ||(-Delta_h)^{-1}||_inf = max E >= its spectral radius 1/lambda_min
    h = 1.0 / (n + 1)
    assert ex.k_star_c(D, n, h) <= fd.k_max(D, n, h)
