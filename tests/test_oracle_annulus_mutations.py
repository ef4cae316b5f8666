"""Planted mistakes in the annulus oracle (on the CPU) must be caught by its pins.

Each case monkeypatches one plausible slip into ``oracle.annulus`` -- a wrong sign, a
dropped scale, a wrong corner rule, an open instead of a closed hole -- and checks that at
least one of the pins below fails (or the oracle raises), while all of them pass on the
unmodified oracle.  The series pin builds its matrices here, from the stated stencils,
without the oracle's operator.
"""
import math

import numpy as np
import pytest

from oracle import annulus as an


def pin_counts():
    g = an.geometry(10)
    g2 = an.geometry(20)
    return ((g.typ == an.HOLE).sum() == 9 and (g.typ == an.EDGE).sum() == 40
            and (g2.typ == an.HOLE).sum() == 49)


def pin_plane_wave():
    k, th = 2.0, 0.7
    a, b = k * math.cos(th), k * math.sin(th)
    errs = []
    for N in (20, 40):
        g = an.geometry(N)
        X, Y = np.meshgrid(g.x, g.x, indexing="ij")
        u = np.exp(1j * (a * X + b * Y))
        data = np.zeros_like(u)
        hole = g.typ == an.HOLE
        data[hole] = u[hole]
        for i, j in g.nodes:
            if g.typ[i, j] == an.EDGE:
                outs = []
                if i == 0: outs.append((-1, 0))
                if i == N: outs.append((1, 0))
                if j == 0: outs.append((0, -1))
                if j == N: outs.append((0, 1))
                dn = np.mean([1j * (a * ox + b * oy) * u[i, j] for ox, oy in outs])
                data[i, j] = dn - 1j * k * u[i, j]
        errs.append(np.max(np.abs(an.solve_direct(g, k, data) - u)))
    return errs[1] < 0.7 * errs[0] and errs[1] < 0.1


def _matrices_from_scratch(N, alpha, k):
    # the stated rows, built here: PDE (sum - 4u)/h^2 - sigma u, edge mean (u - u_in)/h
    h = 1.0 / N
    x = -0.5 + h * np.arange(N + 1)
    typ = {}
    for i in range(N + 1):
        for j in range(N + 1):
            if abs(x[i]) <= 0.15 + 1e-12 and abs(x[j]) <= 0.15 + 1e-12:
                typ[i, j] = "H"
            elif i in (0, N) or j in (0, N):
                typ[i, j] = "E"
            else:
                typ[i, j] = "P"
    unk = [(i, j) for i in range(N + 1) for j in range(N + 1) if typ[i, j] != "H"]
    pos = {p: q for q, p in enumerate(unk)}
    M = len(unk)
    A = np.zeros((M, M))
    m = np.zeros(M, dtype=complex)
    for q, (i, j) in enumerate(unk):
        if typ[i, j] == "P":
            A[q, q] = -4 / h ** 2 - (alpha - k * k)
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if typ[i + di, j + dj] != "H":
                    A[q, pos[i + di, j + dj]] += 1 / h ** 2
            m[q] = -alpha
        else:
            ins = [(i + 1, j)] * (i == 0) + [(i - 1, j)] * (i == N) + [(i, j + 1)] * (j == 0) + [(i, j - 1)] * (j == N)
            A[q, q] = 1 / h
            for p in ins:
                A[q, pos[p]] -= 1 / (h * len(ins))
            m[q] = 1j * k
    return A, m, unk


def pin_series():
    N, k = 10, 0.9
    alpha = k * k + 1.5
    rng = np.random.default_rng(11)
    data = rng.standard_normal((N + 1, N + 1)) + 1j * rng.standard_normal((N + 1, N + 1))
    g = an.geometry(N)
    res = an.annulus_iteration(g, k, data, alpha=alpha, tol=1e-300, max_outer=4, keep_iterates=True)
    A, m, unk = _matrices_from_scratch(N, alpha, k)
    h = 1.0 / N
    b = np.array([data[i, j] for i, j in unk])
    for q, (i, j) in enumerate(unk):      # the hole's data moved to the PDE rows
        if 0 < i < N and 0 < j < N:
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if (i + di, j + dj) not in set(unk):
                    b[q] -= data[i + di, j + dj] / h ** 2
    term = np.linalg.solve(A, b)
    acc = np.zeros_like(term)
    G = np.linalg.solve(A, np.diag(m))
    for n in range(1, 5):
        acc = acc + term
        term = G @ term
        got = np.array([res.iterates[n][i, j] for i, j in unk])
        if not np.allclose(got, acc, atol=1e-10 * np.max(np.abs(acc))):
            return False
    return True


def pin_threshold():
    g = an.geometry(10)
    ks = np.arange(0.9, 1.5, 0.02)
    cross = next((k for k in ks if an.spectral_radius(g, k) > 1), None)
    return cross is not None and 1.05 <= cross <= 1.3


def pin_exit():
    g = an.geometry(20)
    E, L = an.exit_times(g)
    ok = bool(np.all(E[g.typ != an.HOLE] > 0) and np.all(L[g.typ != an.HOLE] > 0))
    for i, j in g.nodes:
        if g.typ[i, j] == an.EDGE:
            ins = an.inward_offsets(g, i, j)
            ok &= abs(L[i, j] - np.mean([L[i + a, j + b] for a, b in ins]) - g.h) < 1e-12
    ok &= abs(an.k_star_A(an.geometry(40), c_tau=2.0) - 0.81) < 0.08
    return ok


PINS = [pin_counts, pin_plane_wave, pin_series, pin_threshold, pin_exit]


def test_annulus_pins_pass_on_the_oracle():
    assert all(p() for p in PINS)


# ---- the planted mistakes -------------------------------------------------------------
_orig_operator = an.operator
_orig_geometry = an.geometry
_orig_iteration = an.annulus_iteration
_orig_exit = an.exit_times


def _edge_rows_unscaled(geo, sigma=0.0, k=None):
    A = _orig_operator(geo, sigma=sigma, k=k).tolil()
    edge = geo.typ[geo.nodes[:, 0], geo.nodes[:, 1]] == an.EDGE
    for q in np.where(edge)[0]:
        A[q, :] = A[q, :] * geo.h          # (u_b - u_in) without the 1/h
    return A.tocsr()


def _robin_sign(geo, sigma=0.0, k=None):
    return _orig_operator(geo, sigma=sigma, k=None if k is None else -k) if k is not None else \
        _orig_operator(geo, sigma=sigma)


def _shift_dropped(geo, sigma=0.0, k=None):
    return _orig_operator(geo, sigma=0.0, k=k)


def _open_hole(N, side=1.0, hole=0.15):
    return _orig_geometry(N, side, hole - 1e-6)


def _lifting_wrong_sign(geo, data):
    h = geo.h
    b = np.zeros(len(geo.nodes), dtype=np.complex128)
    for q, (i, j) in enumerate(geo.nodes):
        b[q] = data[i, j]
        if geo.typ[i, j] == an.PDE:
            for di, dj in an._NB:
                if geo.typ[i + di, j + dj] == an.HOLE:
                    b[q] += data[i + di, j + dj] / (h * h)
    return b


def _corner_single_normal(geo, i, j):
    out = []
    if i == 0:
        out.append((1, 0))
    elif i == geo.N:
        out.append((-1, 0))
    elif j == 0:
        out.append((0, 1))
    elif j == geo.N:
        out.append((0, -1))
    return out


def _neumann_coupling_sign(geo, k, data, alpha=None, tol=1e-8, max_outer=1000, keep_iterates=False):
    # k's sign flipped in the Neumann coupling of the increments (-k w_{n-1}, +k v_{n-1})
    # and in the Robin term, k^2 unchanged
    return _orig_iteration(geo, -k, data, alpha=alpha if alpha is not None else k * k,
                           tol=tol, max_outer=max_outer, keep_iterates=keep_iterates)


def _local_time_wrong_sign(geo, c_tau=1.0):
    E, L = _orig_exit(geo, c_tau)
    return E, -L


MUTATIONS = [
    ("operator", _edge_rows_unscaled),
    ("operator", _robin_sign),
    ("operator", _shift_dropped),
    ("geometry", _open_hole),
    ("lifted_rhs", _lifting_wrong_sign),
    ("inward_offsets", _corner_single_normal),
    ("annulus_iteration", _neumann_coupling_sign),
    ("exit_times", _local_time_wrong_sign),
]


@pytest.mark.parametrize("name,bad", MUTATIONS, ids=[m[1].__name__ for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, bad):
    monkeypatch.setattr(an, name, bad)
    caught = False
    for p in PINS:
        try:
            if not p():
                caught = True
                break
        except Exception:
            caught = True
            break
    assert caught, name
