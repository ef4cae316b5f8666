"""Served stream on the GPU: Poisson arrivals of mixed 2D / 3D solves through the
continuous-batching server; every result is the same alone and in the mix, admission
respects the memory cap, every solve converges to its exact discrete solution."""
import numpy as np
import pytest

from oracle import fd
from paper_2308_11469_gb300 import inputs

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


def test_served_stream_equals_solo(B):
    from paper_2308_11469_gb300 import serve
    reqs = inputs.served_stream(rate=400.0, count=24, seed=11, sizes_2d=(31, 63, 127, 255),
                                sizes_3d=(15, 31))
    jobs = []
    for i, r in enumerate(reqs):
        p = r.problem
        f = torch.from_numpy(p.f).to(DEV)
        g = torch.from_numpy(p.g).to(DEV)
        jobs.append(serve.Job(i, p.D, p.n, p.h, p.k, f, g, torch.zeros_like(g), r.t_arrival))
    cap = 48 << 20                       # small cap: admissions must wait for retirements
    srv = serve.Server(cap, chunk=3)
    done = srv.run(jobs, realtime=True)
    assert len(done) == len(jobs)
    assert srv.max_in_use <= cap
    stats = serve.latency_stats(done)
    assert stats["count"] == len(jobs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    srv.close()
    for j in done:
        p = reqs[j.rid].problem
        assert j.status == B.HELM_CONVERGED
        plan = B.helm_plan_create(p.D, p.n, p.h, p.k, prec=B.HELM_PREC_MIXED)
        u = torch.zeros_like(j.g)
        st, iters, hist = B.helm_solve(plan, j.f, j.g, u, 1e-8, 2000)
        B.helm_plan_destroy(plan)
        assert st == j.status and iters == j.iters
        assert np.array_equal(hist, j.hist)
        assert torch.equal(u, j.u)
        exact = fd.solve_exact_dst(p.f, p.g, p.h, p.k)
        ref = np.linalg.norm(exact)
        # relres 1e-8 against ||b|| bounds the error by ||r|| / (lambda_min - k^2)
        lam = fd.lambda_min(p.D, p.n, p.h)
        bound = max(1e-6, 2 * hist[-1] * np.linalg.norm(fd.lifted_rhs(p.f, p.g, p.h)) / (lam - p.k ** 2) / ref)
        assert np.linalg.norm(j.u.cpu().numpy() - exact) / ref <= bound


@pytest.mark.parametrize("pinned", [True, False])
def test_host_batch_equals_solo(B, pinned):
    # problems in host memory through the library's host entry point (uploads in submission
    # order, the longest solve first): results and histories equal each solve alone
    from paper_2308_11469_gb300 import serve
    probs = [inputs.gaussian_cavity_2d(k, seed=2, n=n) for k, n in ((1.0, 127), (3.0, 255), (4.0, 127))]
    plans = [B.helm_plan_create(2, p.n, p.h, p.k, prec=1) for p in probs]
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    fh = [pin(torch.from_numpy(p.f)) for p in probs]
    gh = [pin(torch.from_numpy(p.g)) for p in probs]
    uh = [pin(torch.full_like(g, 7.0)) for g in gh]        # overwritten by the results
    batch = B.helm_batch_create(0)
    for rep in range(2):                       # the second pass reuses the batch's plans
        out = serve.solve_host_batch(batch, plans, fh, gh, uh, 1e-8, 2000)
        assert B.helm_batch_info(batch) == (0, 0)
        for i, p in enumerate(probs):
            u = torch.zeros((p.n + 2,) * 2, dtype=torch.complex128, device=DEV)
            st, it, hist = B.helm_solve(plans[i], torch.from_numpy(p.f).to(DEV),
                                        torch.from_numpy(p.g).to(DEV), u, 1e-8, 2000)
            assert out[i][0] == st == B.HELM_CONVERGED and out[i][1] == it
            assert np.array_equal(out[i][2], hist)
            assert np.array_equal(uh[i].numpy(), u.cpu().numpy())
    with pytest.raises(ValueError):
        B.helm_batch_submit_host(batch, plans[0], fh[0].to(DEV), gh[0], uh[0], 1e-8, 10)
    B.helm_batch_destroy(batch)
    for pl in plans:
        B.helm_plan_destroy(pl)

