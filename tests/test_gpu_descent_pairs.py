"""Whole outer steps whose descent restricts two levels per launch (cycles without
pre-smoothing from a zero inner iterate: level l+1's and level l+2's rhs from level l's in
one kernel), against the oracle: with u_0 = 0 and zero wall data the first iterate is one
V(0, nu2)-cycle of f from zero, element by element.  The 3D case runs the z-marching
restriction of the rhs and half-sweeps (levels 127 and up) on the same path."""
import numpy as np
import pytest
import torch

from oracle import fd
from oracle import multigrid as mg

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None


@pytest.fixture(scope="module")
def B():
    from paper_2308_11469_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("D,n,prec", [(2, 255, 0), (2, 255, 1), (2, 511, 0), (2, 1023, 1), (3, 127, 1)])
@pytest.mark.parametrize("nu2", [1, 2])
def test_first_iterate_is_one_vcycle(B, D, n, prec, nu2):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(900 + n + nu2)
    f = rng.standard_normal((n,) * D) + 1j * rng.standard_normal((n,) * D)
    plan = B.helm_plan_create(D, n, h, 2.0, prec=prec)
    B.helm_plan_set_cycle(plan, 0, nu2, 1)
    _, exact_n = B.helm_plan_coarse(plan)
    ft = torch.from_numpy(f).to(DEV)
    g = torch.zeros((n + 2,) * D, dtype=torch.complex128, device=DEV)
    u = torch.zeros_like(g)
    st, it, _ = B.helm_solve(plan, ft, g, u, 0.0, 1)
    B.helm_plan_destroy(plan)
    assert st == B.HELM_MAXITER and it == 1
    E = fd.padded_from(np.zeros((n,) * D, complex))
    mg.vcycle(E, f, h, 0, nu2, exact_n=exact_n or None)
    want = fd.interior(E)
    got = fd.interior(u.cpu().numpy())
    scale = np.max(np.abs(want))
    tol = 1e-12 if prec == 0 else 1e-4 * max(1.0, (n + 1) / 256)
    assert np.max(np.abs(got - want)) <= tol * scale
