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


def _compare(B, D, n, prec, nus, seed):
    h = 1.0 / (n + 1)
    dt = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(seed)
    plan = B.helm_plan_create(D, n, h, 1.0, prec=prec)
    # two calls in a row with different data: the second must not see the first's state
    for call in range(2):
        rhs = _rand(rng, (n,) * D, dt)
        e0 = _rand(rng, (n,) * D, dt) * 0.01
        want = e0.clone()
        B.poisson_vcycle(plan, rhs, want, *nus)
        got = e0.clone()
        st = B.poisson_vcycle_noalloc(D, n, h, prec, rhs, got, *nus)
        torch.cuda.synchronize()
        assert st == B.HELM_OK, (call, B.helm_status_str(st))
        w = want.cpu().numpy().astype(np.complex128)
        g = got.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(g - w)) <= _tol(prec, n) * np.max(np.abs(w)), (call, nus)
    B.helm_plan_destroy(plan)


@pytest.mark.parametrize("D,n,prec", [(2, 255, 1), (2, 255, 0), (2, 511, 1), (2, 31, 0),
                                      (3, 31, 1), (3, 63, 0)])
def test_noalloc_vcycle_matches_plan_vcycle(B, D, n, prec):
    _compare(B, D, n, prec, (2, 2), 7 + n + D)


# schedules whose launch sequences differ from V(2,2): no pre-smoothing (zero coarse
# iterates on the way down), no post-smoothing, and the generic 2D kernels (nu > 4)
@pytest.mark.parametrize("D,n,prec,nus", [(2, 127, 1, (0, 2)), (2, 127, 0, (2, 0)),
                                          (2, 127, 1, (5, 1)), (2, 63, 0, (1, 6)),
                                          (3, 31, 1, (0, 2)), (3, 31, 0, (0, 2))])
def test_noalloc_other_schedules_match_plan_vcycle(B, D, n, prec, nus):
    _compare(B, D, n, prec, nus, 11 + n + D + 10 * nus[0] + nus[1])


def test_noalloc_returns_before_queued_work_ends(B):
    """The call only enqueues: with a long sleep kernel queued ahead of it on the stream,
    it returns long before the sleep ends, and the result is still the plan's cycle."""
    n, h, prec = 127, 1.0 / 128, 1
    rng = np.random.default_rng(3)
    rhs = _rand(rng, (n, n), torch.complex64)
    e0 = _rand(rng, (n, n), torch.complex64) * 0.01
    plan = B.helm_plan_create(2, n, h, 1.0, prec=prec)
    want = e0.clone()
    B.poisson_vcycle(plan, rhs, want, 2, 2)
    B.helm_plan_destroy(plan)
    got = e0.clone()
    assert B.poisson_vcycle_noalloc(2, n, h, prec, rhs, got, 2, 2) == B.HELM_OK   # set-up call
    torch.cuda.synchronize()
    got.copy_(e0)
    torch.cuda.synchronize()
    import time
    t0 = time.perf_counter()
    torch.cuda._sleep(200_000_000)            # ~0.1 s at 2 GHz
    st = B.poisson_vcycle_noalloc(2, n, h, prec, rhs, got, 2, 2)
    t_call = time.perf_counter() - t0
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    assert st == B.HELM_OK
    assert t_all > 0.02, t_all                # the sleep did hold the stream
    assert t_call < 0.25 * t_all, (t_call, t_all)
    w = want.cpu().numpy().astype(np.complex128)
    g = got.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(g - w)) <= _tol(prec, n) * np.max(np.abs(w))


def test_noalloc_rejects_grids_beyond_the_library_bounds(B):
    """A hierarchy too deep for the descriptor (or beyond the plan's grid bounds) is
    refused before anything is enqueued; e is left as it was."""
    import ctypes
    rhs = torch.ones((31, 31), dtype=torch.complex64, device=DEV)
    e = torch.zeros((31, 31), dtype=torch.complex64, device=DEV)
    lib = B.load()
    for D, n in ((2, (1 << 20) - 1), (2, (1 << 22) - 1), (3, (1 << 19) - 1), (3, 4095), (2, 65535)):
        for prec in (0, 1):
            st = lib.poisson_vcycle_noalloc(D, n, 1.0 / (n + 1), prec, ctypes.c_void_p(rhs.data_ptr()),
                                            ctypes.c_void_p(e.data_ptr()), 2, 2, None)
            assert st in (B.HELM_EINVAL, B.HELM_EUNSUPPORTED), (D, n, prec, st)
    torch.cuda.synchronize()
    assert torch.count_nonzero(e).item() == 0


def test_noalloc_rejects_grids_beyond_the_scratch_array(B):
    n = 1023                                   # complex64 hierarchy > 16 MiB
    rhs = torch.ones((n, n), dtype=torch.complex64, device=DEV)
    e = torch.zeros((n, n), dtype=torch.complex64, device=DEV)
    st = B.poisson_vcycle_noalloc(2, n, 1.0 / (n + 1), 1, rhs, e, 2, 2)
    torch.cuda.synchronize()
    assert st == B.HELM_EUNSUPPORTED
    assert torch.count_nonzero(e).item() == 0  # nothing was done
