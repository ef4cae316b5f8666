"""Pins for oracle/multigrid.py (the textbook V-cycle used for element-wise kernel checks)."""
import numpy as np
import pytest

from oracle import fd, multigrid as mg
from paper_2308_11469_gb300 import inputs


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("D,n", [(2, 7), (2, 15), (3, 7)])
@pytest.mark.parametrize("color", [0, 1])
def test_half_sweep_solves_its_nodes_exactly(D, n, color):
    # after a half-sweep of one colour, each node of that colour satisfies its own
    # equation (Delta_h e)(x) = r(x) exactly: the neighbours all have the other colour.
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(1)
    E = fd.padded_from(_rand(rng, (n,) * D))
    r = _rand(rng, (n,) * D)
    before = E.copy()
    mg.rbgs_half_sweep(E, r, h, color)
    res = mg.poisson_residual(E, r, h)
    mask = mg.color_mask(D, n, color)
    assert np.max(np.abs(res[mask])) < 1e-12 * np.max(np.abs(r)) * 10
    # the other colour is untouched, the ring stays zero
    assert np.array_equal(fd.interior(E)[~mask], fd.interior(before)[~mask])
    ring = E.copy()
    ring[(slice(1, -1),) * D] = 0
    assert not ring.any()


def test_colours_alternate_like_a_checkerboard():
    m = mg.color_mask(2, 5, 0)
    assert m[0, 0]              # padded (1,1): sum 2 -> red
    assert not m[0, 1] and not m[1, 0] and m[1, 1]
    m3 = mg.color_mask(3, 3, 0)
    # padded (1,1,1) has an odd sum: black in 3D
    assert not m3[0, 0, 0] and m3[0, 0, 1] and not m3[1, 1, 0] and m3[1, 1, 1]
    assert m3.sum() == 13 and mg.color_mask(3, 3, 1).sum() == 14


@pytest.mark.parametrize("D", [2, 3])
def test_prolongation_exact_on_multilinear_data(D):
    nc = 7
    nf = 2 * nc + 1
    hc = 1.0 / (nc + 1)
    hf = hc / 2
    rng = np.random.default_rng(2)
    a = rng.standard_normal(2 ** D)

    def multilinear(xs):
        # sum over subsets of axes of a_S prod_{d in S} x_d
        out = 0.0
        for s in range(2 ** D):
            term = a[s]
            for d in range(D):
                if s >> d & 1:
                    term = term * xs[d]
            out = out + term
        return out

    Ec = multilinear(inputs.node_coords(D, nc, hc)).astype(np.complex128)
    Ef = np.zeros((nf + 2,) * D, dtype=np.complex128)
    mg.prolong_add(Ef, Ec)
    expect = fd.interior(multilinear(inputs.node_coords(D, nf, hf)))
    assert np.allclose(fd.interior(Ef), expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3])
def test_restriction_exact_on_linear_data(D):
    nc = 7
    nf = 2 * nc + 1
    hf = 1.0 / (nf + 1)
    hc = 2 * hf
    c = np.array([0.3, -1.2, 2.0, 0.7])[: D + 1]
    lin = lambda xs: c[0] + sum(c[d + 1] * xs[d] for d in range(D))
    rf = fd.interior(lin(inputs.node_coords(D, nf, hf)))
    rc = mg.restrict_fw(rf)
    assert np.allclose(rc, fd.interior(lin(inputs.node_coords(D, nc, hc))), rtol=0, atol=1e-12)


@pytest.mark.parametrize("D,nc", [(2, 3), (2, 7), (3, 3)])
def test_restriction_is_scaled_adjoint_of_prolongation(D, nc):
    nf = 2 * nc + 1
    P = np.zeros((nf ** D, nc ** D))
    for j in range(nc ** D):
        ec = np.zeros(nc ** D)
        ec[j] = 1.0
        Ef = np.zeros((nf + 2,) * D)
        mg.prolong_add(Ef, fd.padded_from(ec.reshape((nc,) * D)))
        P[:, j] = fd.interior(Ef).reshape(-1)
    R = np.zeros((nc ** D, nf ** D))
    for i in range(nf ** D):
        ef = np.zeros(nf ** D)
        ef[i] = 1.0
        R[:, i] = mg.restrict_fw(ef.reshape((nf,) * D)).reshape(-1)
    assert np.allclose(R, P.T / 2 ** D, rtol=0, atol=1e-15)


def test_coarse_solve_is_exact():
    for D in (2, 3):
        h = 0.5
        r = np.array([1.5 - 2j]).reshape((1,) * D)
        E = np.zeros((3,) * D, dtype=np.complex128)
        mg.coarse_solve(E, r, h)
        assert np.allclose(mg.poisson_residual(E, r, h), 0, atol=1e-15)


@pytest.mark.parametrize("D,n,bound", [(2, 63, 0.1), (3, 15, 0.15), (2, 31, 0.1)])
def test_vcycle_contracts_and_converges_to_direct_solve(D, n, bound):
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    r = _rand(rng, (n,) * D)
    exact = fd.dst_poisson(r, h)
    E = np.zeros((n + 2,) * D, dtype=np.complex128)
    errs = []
    for _ in range(14):
        mg.vcycle(E, r, h, 2, 2)
        errs.append(np.linalg.norm(fd.interior(E) - exact) / np.linalg.norm(exact))
    factors = np.asarray(errs[1:6]) / np.asarray(errs[0:5])
    assert np.all(factors < bound), factors
    assert errs[-1] < 1e-12


@pytest.mark.parametrize("D,n", [(2, 31), (3, 7)])
def test_exact_level_is_the_direct_solve(D, n):
    # a cycle whose top level is the exactly solved one returns the sparse-LU solution
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(11)
    r = _rand(rng, (n,) * D)
    E = fd.padded_from(_rand(rng, (n,) * D))        # the guess is discarded
    mg.vcycle(E, r, h, 1, 1, exact_n=n)
    lu = fd.SparsePoisson(D, n, h)
    want = lu(r.real) + 1j * lu(r.imag)
    assert np.allclose(fd.interior(E), want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("nus", [(2, 2), (1, 1)])
def test_exact_coarse_level_contracts_at_least_as_well(nus):
    # 2D n = 127 with the n = 31 level solved exactly (the CUDA complex64 hierarchy):
    # a better coarse solve cannot slow the cycle down, and it still converges to the
    # direct solve of the fine system
    n = 127
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(12)
    r = _rand(rng, (n, n))
    exact = fd.dst_poisson(r, h)
    errs = {}
    for xn in (None, 31):
        E = np.zeros((n + 2, n + 2), dtype=np.complex128)
        e = []
        for _ in range(10):
            mg.vcycle(E, r, h, *nus, exact_n=xn)
            e.append(np.linalg.norm(fd.interior(E) - exact) / np.linalg.norm(exact))
        errs[xn] = np.asarray(e)
    assert np.all(errs[31] <= errs[None] * 1.02)
    f = errs[31][1:6] / errs[31][:5]
    assert np.all(f < (0.1 if nus == (2, 2) else 0.2)), f
    assert errs[31][-1] < 1e-8
