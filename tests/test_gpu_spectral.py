"""rho(G) measured by GPU power iteration (the operator the solver applies) against the
closed form rho = sqrt(alpha^2 + p^2) / (lambda_min + alpha - k^2) (Section 2.4 / 2.2)."""
import pytest

from oracle import fd, general as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_11469_gb300 import binding, build
    build.build()
    binding.load()
    return binding


CASES = [(2.0, 0.0, 0.0), (3.0, 6.0, 0.0), (2.0, 1.0, 5.0), (1.0, 30.0, 20.0)]


@pytest.mark.parametrize("D,n", [(2, 63), (2, 255), (3, 31)])
@pytest.mark.parametrize("prec", [0, 1])
def test_power_iteration_matches_the_closed_form(B, D, n, prec):
    h = 1.0 / (n + 1)
    for k, dalpha, p in CASES:
        alpha = k * k + dalpha
        plan = B.helm_plan_create(D, n, h, k, prec=prec)
        B.helm_plan_set_cavity(plan, alpha, p)
        B.helm_plan_set_cycle(plan, 2, 2, 1)
        st, rho, its = B.helm_spectral_radius(plan, 300, 1e-12 if prec == 0 else 1e-7, 12)
        info_rho = B.helm_plan_info(plan)[2]
        B.helm_plan_destroy(plan)
        want = gen.rho_pred(D, n, h, k, alpha, p)
        assert st == B.HELM_OK, (k, alpha, p, its)
        # complex64 cycles: M^{-1} carries rounding ~1e-4 (n+1)/256 of its largest terms
        # (as single cycles do), which bounds the power iteration's accuracy
        assert rho == pytest.approx(want, rel=1e-9 if prec == 0 else 1e-4 * max(1.0, (n + 1) / 256)), (k, alpha, p)
        assert info_rho == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_rho_crosses_one_at_k_max(B, prec):
    D, n = 2, 127
    h = 1.0 / (n + 1)
    km = fd.k_max(D, n, h)
    out = []
    for frac in (0.95, 1.05):
        plan = B.helm_plan_create(D, n, h, frac * km, prec=prec)
        B.helm_plan_set_cycle(plan, 2, 2, 1)
        st, rho, its = B.helm_spectral_radius(plan, 300, 1e-10, 12)
        B.helm_plan_destroy(plan)
        out.append(rho)
    assert out[0] < 1.0 < out[1]
    assert out[0] == pytest.approx(0.95 ** 2, rel=1e-4) and out[1] == pytest.approx(1.05 ** 2, rel=1e-4)


def test_bad_arguments(B):
    plan = B.helm_plan_create(2, 31, 1 / 32, 1.0)
    for args in [(0, 1e-8, 4), (10, -1.0, 4), (10, 1e-8, 0)]:
        with pytest.raises(B.HelmError):
            B.helm_spectral_radius(plan, *args)
    B.helm_plan_destroy(plan)
