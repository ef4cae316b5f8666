"""The cluster tail (levels 255, 127, 63 and the exact level 31 of 2D complex64 cycles in
one 8-CTA cluster per solve) against the oracle's V-cycle and against the one-CTA tail.

Single V(0, nu2) cycles from a nonzero starting iterate (the finest level then carries an
iterate, the cluster's levels start from zero), element by element against
``oracle.multigrid.vcycle``; whole 1023^2 Gaussian-cavity solves with both coarse forms
against each other and against the relres target.
"""
import numpy as np
import pytest
import torch

from oracle import fd
from oracle import multigrid as mg
from paper_2308_11469_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None


@pytest.fixture(scope="module")
def B():
    from paper_2308_11469_gb300 import binding
    binding.load()
    return binding


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _vcycle(B, n, nus, mode, r, e0):
    plan = B.helm_plan_create(2, n, 1.0 / (n + 1), 1.0, prec=B.HELM_PREC_MIXED)
    B.helm_plan_set_coarse_mode(plan, mode)
    et = torch.from_numpy(e0).to(DEV).to(torch.complex64)
    B.poisson_vcycle(plan, torch.from_numpy(r).to(DEV).to(torch.complex64), et, *nus)
    used = B.helm_plan_coarse_mode(plan)[1]
    _, exact_n = B.helm_plan_coarse(plan)
    B.helm_plan_destroy(plan)
    return et.cpu().numpy().astype(np.complex128), used, exact_n


@pytest.mark.parametrize("n", [511, 1023])
@pytest.mark.parametrize("nus", [(0, 1), (0, 2)])
def test_cluster_vcycle_elementwise(B, n, nus):
    rng = np.random.default_rng(500 + n + nus[1])
    r = _rand_c(rng, (n, n))
    e0 = 0.01 * _rand_c(rng, (n, n))
    got, used, exact_n = _vcycle(B, n, nus, B.HELM_COARSE_CLUSTER, r, e0)
    assert used == 1
    ref, used_cta, _ = _vcycle(B, n, nus, B.HELM_COARSE_CTA, r, e0)
    assert used_cta == 0
    E = fd.padded_from(e0.copy())
    mg.vcycle(E, r, 1.0 / (n + 1), *nus, exact_n=exact_n)
    want = fd.interior(E)
    scale = np.max(np.abs(want))
    tol = 1e-4 * (n + 1) / 256
    assert np.max(np.abs(got - want)) <= tol * scale
    # same operations in the same order: the two coarse forms agree to FP32 rounding
    dev = float(np.max(np.abs(got - ref)) / scale)
    print(f"n={n} V{nus}: cluster vs one-CTA tail max dev {dev:.3e}, vs oracle "
          f"{float(np.max(np.abs(got - want)) / scale):.3e}")
    assert dev <= 1e-5


def test_cluster_not_used_where_it_does_not_apply(B):
    rng = np.random.default_rng(3)
    for n, nus in ((255, (0, 1)), (1023, (1, 1)), (1023, (0, 3))):
        r = _rand_c(rng, (n, n))
        e0 = np.zeros((n, n), complex)
        _, used, _ = _vcycle(B, n, nus, B.HELM_COARSE_CLUSTER, r, e0)
        assert used == 0, (n, nus)
    with pytest.raises(B.HelmError):
        plan = B.helm_plan_create(2, 63, 1 / 64, 1.0, prec=B.HELM_PREC_MIXED)
        try:
            B.helm_plan_set_coarse_mode(plan, 3)
        finally:
            B.helm_plan_destroy(plan)


@pytest.mark.parametrize("k", [1.0, 4.0])
def test_cluster_gaussian_cavity_1023_solve(B, k):
    p = inputs.gaussian_cavity_2d(k)
    f = torch.from_numpy(p.f).to(DEV)
    g = torch.from_numpy(p.g).to(DEV)
    out = {}
    for mode in (B.HELM_COARSE_CLUSTER, B.HELM_COARSE_AUTO, B.HELM_COARSE_CTA):
        plan = B.helm_plan_create(2, p.n, p.h, p.k, prec=B.HELM_PREC_MIXED)
        B.helm_plan_set_cycle(plan, 0, 1, 1)
        B.helm_plan_set_coarse_mode(plan, mode)
        u = torch.zeros_like(g)
        st, it, hist = B.helm_solve(plan, f, g, u, 1e-8, 400)
        out[mode] = (st, it, hist, u.cpu().numpy(), B.helm_plan_coarse_mode(plan)[1])
        B.helm_plan_destroy(plan)
    st, it, hist, uc, used = out[B.HELM_COARSE_CLUSTER]
    st2, it2, hist2, ut, used2 = out[B.HELM_COARSE_CTA]
    st3, it3, hist3, ua, used3 = out[B.HELM_COARSE_AUTO]
    assert used == 1 and used2 == 0 and used3 == 1
    assert it3 == it and np.array_equal(hist3, hist) and np.array_equal(ua, uc)
    assert st == B.HELM_CONVERGED and st2 == B.HELM_CONVERGED
    assert hist[-1] <= 1e-8
    dev = float(np.linalg.norm(uc - ut) / np.linalg.norm(ut))
    print(f"k={k}: cluster {it} steps, one-CTA tail {it2} steps, solutions differ by {dev:.3e}")
    # the same operations either way (cluster tail and level 1's ascent inside the finest
    # kernel, or the one-CTA tail and per-level launches): the same bits
    assert it == it2 and np.array_equal(hist, hist2) and np.array_equal(uc, ut)
