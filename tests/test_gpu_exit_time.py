"""GPU parity of the mean exit time (Eq. (2.10)) and k_*^C (Eq. (2.9)) against the oracle."""
import math

import numpy as np
import pytest

from oracle import exit_time as ex, fd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11469_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("D,n", [(2, 127), (2, 1023), (3, 31), (3, 63)])
@pytest.mark.parametrize("prec", [0, 1])
def test_exit_time_field_and_maximum(B, D, n, prec):
    h = 1.0 / (n + 1)
    plan = B.helm_plan_create(D, n, h, 1.0, prec=prec)
    E = torch.empty((n + 2,) * D, dtype=torch.complex128, device=DEV)
    tol = 1e-12 if prec == 0 else 1e-8
    if D == 2 and n == 1023 and prec == 0:
        tol = 1e-10                        # the FP64 relres floor at 1023^2 is ~1e-10
    st, emax, kstar = B.helm_exit_time(plan, tol, 200, E)
    B.helm_plan_destroy(plan)
    assert st == B.HELM_CONVERGED
    want = ex.exit_time(D, n, h)
    got = E.cpu().numpy()
    assert np.all(got.imag == 0) and np.all(fd.ring_only(got) == 0)
    err = np.linalg.norm(fd.interior(got).real - want) / np.linalg.norm(want)
    assert err <= (1e-9 if prec == 0 else 1e-6), err
    assert emax == pytest.approx(float(np.max(want)), rel=(1e-9 if prec == 0 else 1e-6))
    assert emax == np.max(fd.interior(got).real)           # the maximum of the returned field
    assert kstar == pytest.approx(ex.k_star_c(D, n, h), rel=(1e-9 if prec == 0 else 1e-6))


def test_unit_square_bound(B):
    # 1023^2: k_*^C of the unit square, 3.684 (the continuum torsion maximum 0.0736713...)
    n = 1023
    plan = B.helm_plan_create(2, n, 1.0 / (n + 1), 1.0, prec=1)
    st, emax, kstar = B.helm_exit_time(plan, 1e-8, 200)
    B.helm_plan_destroy(plan)
    assert emax == pytest.approx(ex.square_center_cosh_series(), rel=1e-5)
    assert kstar == pytest.approx(3.684, abs=1e-3)


def test_damping_lowers_the_bound(B):
    n = 63
    h = 1.0 / (n + 1)
    plan = B.helm_plan_create(2, n, h, 2.0, prec=0)
    B.helm_plan_set_cavity(plan, 4.0, 5.0)
    st, emax, kstar = B.helm_exit_time(plan, 1e-12, 200)
    B.helm_plan_destroy(plan)
    assert kstar == pytest.approx(ex.k_star_c(2, n, h, p=5.0), rel=1e-9)
    assert kstar == pytest.approx(math.sqrt(1.0 / emax - 5.0), rel=1e-14)


def test_one_node_grid(B):
    plan = B.helm_plan_create(2, 1, 0.5, 1.0, prec=0)
    st, emax, kstar = B.helm_exit_time(plan, 1e-14, 20)
    B.helm_plan_destroy(plan)
    assert emax == pytest.approx(1 / 16, rel=1e-14) and kstar == pytest.approx(4.0, rel=1e-14)


def test_bad_arguments(B):
    plan = B.helm_plan_create(2, 31, 1 / 32, 1.0)
    with pytest.raises(B.HelmError):
        B.helm_exit_time(plan, -1.0)
    with pytest.raises(B.HelmError):
        B.helm_exit_time(plan, 1e-8, 0)
    B.helm_plan_destroy(plan)
