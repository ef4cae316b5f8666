"""The allocation-free V-cycle entry point against the plan-based one.

poisson_vcycle_noalloc is meant for callers that cannot call cudaMalloc (a host framework
that owns the device memory, or a latency-critical loop that cannot take the device
synchronisation of an allocation): it runs the same multigrid cycle as poisson_vcycle on
the library's static scratch array.  This file is collected last so that, when it fails,
a run that stops at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest

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


def _rand(rng, shape, dt):
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(a).to(DEV).to(dt)


def _tol(prec, n):
    # the element-wise V-cycle tolerance of the parity tests, relative to the array's max
    return 1e-12 if prec == 0 else 1e-4 * max(1.0, (n + 1) / 256)


@pytest.mark.parametrize("D,n,prec", [(2, 255, 1), (2, 255, 0), (2, 511, 1), (2, 31, 0),
                                      (3, 31, 1), (3, 63, 0)])
def test_noalloc_vcycle_matches_plan_vcycle(B, D, n, prec):
    h = 1.0 / (n + 1)
    dt = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(7 + n + D)
    plan = B.helm_plan_create(D, n, h, 1.0, prec=prec)
    # two calls in a row with different data: the second must not see the first's state
    for call in range(2):
        rhs = _rand(rng, (n,) * D, dt)
        e0 = _rand(rng, (n,) * D, dt) * 0.01
        want = e0.clone()
        B.poisson_vcycle(plan, rhs, want, 2, 2)
        got = e0.clone()
        st = B.poisson_vcycle_noalloc(D, n, h, prec, rhs, got, 2, 2)
        torch.cuda.synchronize()
        assert st == B.HELM_OK, (call, B.helm_status_str(st))
        w = want.cpu().numpy().astype(np.complex128)
        g = got.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(g - w)) <= _tol(prec, n) * np.max(np.abs(w)), call
    B.helm_plan_destroy(plan)


def test_noalloc_rejects_grids_beyond_the_scratch_array(B):
    n = 1023                                   # complex64 hierarchy > 16 MiB
    rhs = torch.ones((n, n), dtype=torch.complex64, device=DEV)
    e = torch.zeros((n, n), dtype=torch.complex64, device=DEV)
    st = B.poisson_vcycle_noalloc(2, n, 1.0 / (n + 1), 1, rhs, e, 2, 2)
    torch.cuda.synchronize()
    assert st == B.HELM_EUNSUPPORTED
    assert torch.count_nonzero(e).item() == 0  # nothing was done
