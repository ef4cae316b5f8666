"""ctypes binding of the C ABI in include/helm.h (argument marshalling only).

Every function of the ABI appears here under the same name.  Arrays are torch tensors on
the plan's CUDA device (PyTorch supplies device memory and streams); each call checks
dtype / shape / contiguity, passes raw pointers, and raises ``HelmError`` on a negative
status.  All arithmetic runs in the CUDA library: there is no fallback, and loading
fails loudly when ``libhelm.so`` has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhelm.so")

HELM_OK = 0
HELM_CONVERGED = 0
HELM_MAXITER = 1
HELM_DIVERGED = 2
HELM_EINVAL = -1
HELM_ENOMEM = -2
HELM_ECUDA = -3
HELM_ENONFINITE = -4
HELM_ETIMEOUT = -5
HELM_EUNSUPPORTED = -6
HELM_BC_DIRICHLET = 0
HELM_PREC_FP64 = 0
HELM_PREC_MIXED = 1

# every symbol the header declares, with (restype, argtypes)
_vp = C.c_void_p
_SIGS = {
    "helm_status_str": (C.c_char_p, [C.c_int]),
    "helm_last_error": (C.c_char_p, []),
    "helm_launch_count": (C.c_uint64, []),
    "helm_selftest_conversions": (C.c_int, [C.c_int, C.c_uint64, C.POINTER(C.c_uint64)]),
    "helm_measure_fp64_rate": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "helm_plan_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(C.c_int), C.c_double,
                                   C.c_double, C.c_int, C.c_int, _vp]),
    "helm_plan_destroy": (C.c_int, [_vp]),
    "helm_plan_info": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_size_t)]),
    "helm_plan_set_cycle": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "helm_plan_coarse": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "helm_plan_set_cavity": (C.c_int, [_vp, C.c_double, C.c_double]),
    "helm_plan_set_tiles": (C.c_int, [_vp, C.c_int]),
    "helm_plan_tiles": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "helm_batch_set_tiles": (C.c_int, [_vp, C.c_int]),
    "helm_plan_set_coarse_mode": (C.c_int, [_vp, C.c_int]),
    "helm_plan_coarse_mode": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "helm_batch_set_coarse_mode": (C.c_int, [_vp, C.c_int]),
    "helm_batch_set_cycle_class": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "helm_batch_submit_many": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                         C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.c_double, C.c_int,
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_int)]),
    "helm_batch_poll_many": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "helm_exit_time": (C.c_int, [_vp, C.c_double, C.c_int, _vp, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "helm_spectral_radius": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_int)]),
    "helm_solve": (C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                             C.POINTER(C.c_double)]),
    "helm_solve_ex": (C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "poisson_vcycle": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int]),
    "poisson_vcycle_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_int, _vp, _vp, C.c_int,
                                         C.c_int, _vp]),
    "helm_annulus_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_double, C.c_double, C.c_double, C.c_int]),
    "helm_annulus_spectral_radius": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                                 C.POINTER(C.c_double), C.POINTER(C.c_double),
                                                 C.POINTER(C.c_int)]),
    "helm_annulus_condition": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "helm_annulus_destroy": (C.c_int, [_vp]),
    "helm_annulus_set_shift": (C.c_int, [_vp, C.c_double]),
    "helm_annulus_set_cycle": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "helm_annulus_solve": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_double)]),
    "helm_annulus_exit_times": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, _vp, _vp,
                                          C.POINTER(C.c_double)]),
    "helm_batch_create": (C.c_int, [C.POINTER(_vp), C.c_size_t, _vp]),
    "helm_batch_destroy": (C.c_int, [_vp]),
    "helm_batch_submit": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_double, C.c_int,
                                    C.POINTER(C.c_uint64)]),
    "helm_batch_step": (C.c_int, [_vp, C.c_int]),
    "helm_batch_submit_geom": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _vp,
                                         _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_uint64)]),
    "helm_batch_set_cycle": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "helm_batch_set_lanes": (C.c_int, [_vp, C.c_int]),
    "helm_plan_autotune": (C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "helm_batch_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "helm_batch_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
    "helm_batch_set_host_result": (C.c_int, [_vp, C.c_uint64, _vp]),
    "helm_batch_submit_host": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_double, C.c_int, C.POINTER(C.c_uint64)]),
    "helm_batch_profile": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.c_int]),
}

KERNEL_KINDS = ["rbgs_half_sweep", "residual_restrict", "prolong_correct", "zero",
                "coarse_tail", "helmholtz_residual_update", "convergence_check",
                "smooth_restrict_2d", "prolong_smooth_2d", "ascent_residual_update_2d",
                "cluster_tail", "restrict_two_levels_2d", "ascent_l1_residual_update_2d"]

_lib = None


class HelmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = ""
        if _lib is not None:
            detail = _lib.helm_last_error().decode()
        super().__init__(f"{where}: {status_name(status)}" + (f" ({detail})" if detail else ""))


def load(path: str = LIB_PATH):
    """Load libhelm.so and declare the ABI.  Raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(s: int) -> str:
    if _lib is None:
        return str(s)
    return _lib.helm_status_str(int(s)).decode()


def _check(status: int, where: str) -> int:
    if status < 0 and status != HELM_ENONFINITE:
        raise HelmError(status, where)
    return status


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    return C.c_void_p(t.data_ptr())


def helm_status_str(status: int) -> str:
    return load().helm_status_str(int(status)).decode()


def helm_last_error() -> str:
    return load().helm_last_error().decode()


def helm_launch_count() -> int:
    return int(load().helm_launch_count())


def helm_measure_fp64_rate():
    """(TFLOP/s, ms of the best launch) of the device's FP64 FMA rate."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().helm_measure_fp64_rate(C.byref(tf), C.byref(ms)), "helm_measure_fp64_rate")
    return tf.value, ms.value


def helm_selftest_conversions(count: int = 1 << 20, seed: int = 1) -> int:
    bad = C.c_uint64()
    _check(load().helm_selftest_conversions(int(count), C.c_uint64(seed), C.byref(bad)),
           "helm_selftest_conversions")
    return int(bad.value)


class _Plan:
    """Handle returned by helm_plan_create (owns the C plan)."""

    def __init__(self, handle, D, n, h, k, prec):
        self.handle = handle
        self.D, self.n, self.h, self.k, self.prec = D, n, h, k, prec

    @property
    def inner_dtype(self):
        import torch
        return torch.complex128 if self.prec == HELM_PREC_FP64 else torch.complex64

    def __del__(self):
        if self.handle is not None and _lib is not None:
            _lib.helm_plan_destroy(self.handle)
            self.handle = None


def helm_plan_create(ndim: int, n: int, h: float, k: float, bc: int = HELM_BC_DIRICHLET,
                     prec: int = HELM_PREC_MIXED, stream=None) -> _Plan:
    lib = load()
    out = C.c_void_p()
    arr = (C.c_int * ndim)(*([n] * ndim))
    st = lib.helm_plan_create(C.byref(out), ndim, arr, float(h), float(k), int(bc), int(prec),
                              _stream_handle(stream))
    _check(st, "helm_plan_create")
    return _Plan(out, ndim, n, h, k, prec)


def helm_plan_destroy(plan: _Plan) -> None:
    if plan.handle is not None:
        _check(load().helm_plan_destroy(plan.handle), "helm_plan_destroy")
        plan.handle = None


def helm_plan_info(plan: _Plan):
    lm, km, rho = C.c_double(), C.c_double(), C.c_double()
    ws = C.c_size_t()
    _check(load().helm_plan_info(plan.handle, C.byref(lm), C.byref(km), C.byref(rho), C.byref(ws)),
           "helm_plan_info")
    return lm.value, km.value, rho.value, ws.value


def helm_plan_coarse(plan: _Plan):
    """(tail_n, exact_n): where the one-CTA coarse tail starts, and the level it solves
    exactly in the sine basis (0: none)."""
    t, x = C.c_int(), C.c_int()
    _check(load().helm_plan_coarse(plan.handle, C.byref(t), C.byref(x)), "helm_plan_coarse")
    return t.value, x.value


def helm_plan_set_cavity(plan: _Plan, alpha: float, p: float) -> None:
    """General cavity iteration: shift alpha >= k^2 and damping p >= 0."""
    _check(load().helm_plan_set_cavity(plan.handle, float(alpha), float(p)), "helm_plan_set_cavity")


def helm_exit_time(plan: _Plan, tol: float = 1e-10, max_outer: int = 200, E_out=None):
    """Mean exit time (Delta_h E = -1, E = 0 on the wall) and k_*^C = sqrt(1/max E - p).
    E_out: optional padded complex128 device tensor receiving E.  Returns
    (status, max E, k_*^C)."""
    import torch
    D, n = plan.D, plan.n
    pe = None if E_out is None else _ptr(E_out, torch.complex128, (n + 2,) * D, "E_out")
    em, ks = C.c_double(), C.c_double()
    st = _check(load().helm_exit_time(plan.handle, float(tol), int(max_outer), pe, C.byref(em),
                                      C.byref(ks)), "helm_exit_time")
    return st, em.value, ks.value


def helm_spectral_radius(plan: _Plan, max_iters: int = 200, tol: float = 1e-10, cycles: int = 8):
    """rho(G) by GPU power iteration; returns (status, rho, iterations)."""
    r, n = C.c_double(), C.c_int()
    st = _check(load().helm_spectral_radius(plan.handle, int(max_iters), float(tol), int(cycles),
                                            C.byref(r), C.byref(n)), "helm_spectral_radius")
    return st, r.value, n.value


def helm_plan_set_cycle(plan: _Plan, nu1: int, nu2: int, cycles: int = 1) -> None:
    _check(load().helm_plan_set_cycle(plan.handle, nu1, nu2, cycles), "helm_plan_set_cycle")


HELM_TILES_AUTO = 0
HELM_TILES_LARGE = 1
HELM_TILES_SMALL = 2


def helm_plan_set_tiles(plan: _Plan, policy: int) -> None:
    _check(load().helm_plan_set_tiles(plan.handle, int(policy)), "helm_plan_set_tiles")


def helm_plan_tiles(plan: _Plan) -> int:
    v = C.c_int()
    _check(load().helm_plan_tiles(plan.handle, C.byref(v)), "helm_plan_tiles")
    return v.value


HELM_COARSE_AUTO = 0
HELM_COARSE_CTA = 1
HELM_COARSE_CLUSTER = 2


def helm_plan_set_coarse_mode(plan: _Plan, mode: int) -> None:
    _check(load().helm_plan_set_coarse_mode(plan.handle, int(mode)), "helm_plan_set_coarse_mode")


def helm_plan_coarse_mode(plan: _Plan) -> tuple[int, int]:
    """(policy, whether the last built outer step used the cluster tail)."""
    m, used = C.c_int(), C.c_int()
    _check(load().helm_plan_coarse_mode(plan.handle, C.byref(m), C.byref(used)), "helm_plan_coarse_mode")
    return m.value, used.value


def helm_batch_submit_many(batch, jobs, prec: int, tol: float, max_outer: int):
    """jobs: sequence of (ndim, n, h, k, f, g, u) with complex128 contiguous device tensors
    (f interior n^D, g and u padded (n+2)^D).  Returns the tickets of the admitted prefix
    (shorter than jobs when the memory cap stopped the submission)."""
    import torch
    m = len(jobs)
    nd = (C.c_int * m)()
    nn = (C.c_int * m)()
    hh = (C.c_double * m)()
    kk = (C.c_double * m)()
    pf, pg, pu = (_vp * m)(), (_vp * m)(), (_vp * m)()
    for i, (d, n, h, k, f, g, u) in enumerate(jobs):
        for t, cnt, name in ((f, n ** d, "f"), (g, (n + 2) ** d, "g"), (u, (n + 2) ** d, "u")):
            if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() != cnt:
                raise HelmError(HELM_EINVAL, f"helm_batch_submit_many: job {i}: bad {name}")
        nd[i], nn[i], hh[i], kk[i] = int(d), int(n), float(h), float(k)
        pf[i], pg[i], pu[i] = f.data_ptr(), g.data_ptr(), u.data_ptr()
    tk = (C.c_uint64 * m)()
    adm = C.c_int(0)
    st = load().helm_batch_submit_many(batch.handle, m, nd, nn, hh, kk, int(prec), pf, pg, pu, float(tol),
                                       int(max_outer), tk, C.byref(adm))
    if st != HELM_ENOMEM:
        _check(st, "helm_batch_submit_many")
    return [tk[i] for i in range(adm.value)]


def helm_batch_poll_many(batch, tickets, release: bool = True):
    """Returns [(done, status, iters)] for the tickets (status / iters valid when done);
    release=False keeps the finished solves' records (helm_batch_poll then returns the
    history)."""
    m = len(tickets)
    tk = (C.c_uint64 * m)(*tickets)
    dn, stt, its = (C.c_int * m)(), (C.c_int * m)(), (C.c_int * m)()
    _check(load().helm_batch_poll_many(batch.handle, m, tk, 1 if release else 0, dn, stt, its),
           "helm_batch_poll_many")
    return [(dn[i], stt[i], its[i]) for i in range(m)]


def helm_batch_set_cycle_class(batch, ndim: int, prec: int, nu1: int, nu2: int, cycles: int = 1) -> None:
    _check(load().helm_batch_set_cycle_class(batch.handle, int(ndim), int(prec), int(nu1), int(nu2), int(cycles)),
           "helm_batch_set_cycle_class")


def helm_batch_set_tiles(batch, policy: int) -> None:
    _check(load().helm_batch_set_tiles(batch.handle, int(policy)), "helm_batch_set_tiles")


def helm_batch_set_coarse_mode(batch, mode: int) -> None:
    _check(load().helm_batch_set_coarse_mode(batch.handle, int(mode)), "helm_batch_set_coarse_mode")


def helm_plan_autotune(plan: _Plan, f, g, u, tol: float, max_outer: int):
    """Returns (nu1, nu2, cycles, best ms); the plan keeps the fastest schedule."""
    import torch
    D, n = plan.D, plan.n
    pf = _ptr(f, torch.complex128, (n,) * D, "f")
    pg = _ptr(g, torch.complex128, (n + 2,) * D, "g")
    pu = _ptr(u, torch.complex128, (n + 2,) * D, "u")
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    ms = C.c_double()
    _check(load().helm_plan_autotune(plan.handle, pf, pg, pu, float(tol), int(max_outer), C.byref(a),
                                     C.byref(b), C.byref(c), C.byref(ms)), "helm_plan_autotune")
    return a.value, b.value, c.value, ms.value


def helm_solve_ex(plan: _Plan, f, g, u, tol: float, max_outer: int):
    """Returns (status, iters, relres history, increment sup-norm history)."""
    import torch
    D, n = plan.D, plan.n
    pf = _ptr(f, torch.complex128, (n,) * D, "f")
    pg = _ptr(g, torch.complex128, (n + 2,) * D, "g")
    pu = _ptr(u, torch.complex128, (n + 2,) * D, "u")
    iters = C.c_int()
    hist = np.zeros(max_outer + 1, dtype=np.float64)
    einf = np.zeros(max(max_outer, 1), dtype=np.float64)
    st = load().helm_solve_ex(plan.handle, pf, pg, pu, float(tol), int(max_outer), C.byref(iters),
                              hist.ctypes.data_as(C.POINTER(C.c_double)),
                              einf.ctypes.data_as(C.POINTER(C.c_double)))
    _check(st, "helm_solve")
    it = iters.value
    return st, it, hist[: it + 1].copy(), einf[:it].copy()


def helm_solve(plan: _Plan, f, g, u, tol: float, max_outer: int):
    """Returns (status, iters, relres history)."""
    st, it, hist, _ = helm_solve_ex(plan, f, g, u, tol, max_outer)
    return st, it, hist


def poisson_vcycle(plan: _Plan, rhs, e, nu1: int = 2, nu2: int = 2) -> None:
    D, n = plan.D, plan.n
    pr = _ptr(rhs, plan.inner_dtype, (n,) * D, "rhs")
    pe = _ptr(e, plan.inner_dtype, (n,) * D, "e")
    _check(load().poisson_vcycle(plan.handle, pr, pe, int(nu1), int(nu2)), "poisson_vcycle")


def poisson_vcycle_noalloc(ndim: int, n: int, h: float, prec: int, rhs, e, nu1: int = 2,
                           nu2: int = 2, stream=None) -> int:
    """One V-cycle without a plan or any device allocation (the library's static scratch
    array); asynchronous on the stream.  Returns the status (HELM_EUNSUPPORTED when the
    grid does not fit the scratch array)."""
    import torch
    dt = torch.complex128 if prec == HELM_PREC_FP64 else torch.complex64
    pr = _ptr(rhs, dt, (n,) * ndim, "rhs")
    pe = _ptr(e, dt, (n,) * ndim, "e")
    st = load().poisson_vcycle_noalloc(int(ndim), int(n), float(h), int(prec), pr, pe, int(nu1),
                                       int(nu2), _stream_handle(stream))
    if st != HELM_EUNSUPPORTED:
        _check(st, "poisson_vcycle_noalloc")
    return st


class _Annulus:
    """Handle returned by helm_annulus_create (owns the C plan)."""

    def __init__(self, handle, n, side, hole, k, prec):
        self.handle = handle
        self.n, self.side, self.hole, self.k, self.prec = n, side, hole, k, prec

    def __del__(self):
        if self.handle is not None and _lib is not None:
            _lib.helm_annulus_destroy(self.handle)
            self.handle = None


def helm_annulus_create(n: int, side: float = 1.0, hole: float = 0.15, k: float = 0.0,
                        prec: int = HELM_PREC_MIXED) -> _Annulus:
    out = C.c_void_p()
    _check(load().helm_annulus_create(C.byref(out), int(n), float(side), float(hole), float(k), int(prec)),
           "helm_annulus_create")
    return _Annulus(out, n, side, hole, k, prec)


def helm_annulus_destroy(plan: _Annulus) -> None:
    if plan.handle is not None:
        _check(load().helm_annulus_destroy(plan.handle), "helm_annulus_destroy")
        plan.handle = None


def helm_annulus_set_shift(plan: _Annulus, alpha: float) -> None:
    _check(load().helm_annulus_set_shift(plan.handle, float(alpha)), "helm_annulus_set_shift")


def helm_annulus_set_cycle(plan: _Annulus, nu1: int, nu2: int, cycles: int = 1) -> None:
    _check(load().helm_annulus_set_cycle(plan.handle, nu1, nu2, cycles), "helm_annulus_set_cycle")


def helm_annulus_solve(plan: _Annulus, data, u, tol: float, max_outer: int):
    """data, u: (n+1, n+1) complex128 device tensors.  Returns (status, iters, relres history)."""
    import torch
    n = plan.n
    pd = _ptr(data, torch.complex128, (n + 1, n + 1), "data")
    pu = _ptr(u, torch.complex128, (n + 1, n + 1), "u")
    iters = C.c_int()
    hist = np.zeros(max_outer + 1, dtype=np.float64)
    st = _check(load().helm_annulus_solve(plan.handle, pd, pu, float(tol), int(max_outer), C.byref(iters),
                                          hist.ctypes.data_as(C.POINTER(C.c_double))), "helm_annulus_solve")
    return st, iters.value, hist[: iters.value + 1].copy()


def helm_annulus_exit_times(plan: _Annulus, E, L, c_tau: float = 1.0, tol: float = 1e-10,
                            max_outer: int = 200):
    """E, L: (n+1, n+1) float64 device tensors (outputs).  Returns (status, k_*^A); the status
    is HELM_CONVERGED when both solves reached tol (else E, L and k_*^A are not valid)."""
    import torch
    n = plan.n
    pe = _ptr(E, torch.float64, (n + 1, n + 1), "E")
    pl = _ptr(L, torch.float64, (n + 1, n + 1), "L")
    ks = C.c_double(0.0)
    st = _check(load().helm_annulus_exit_times(plan.handle, float(c_tau), float(tol), int(max_outer), pe, pl,
                                               C.byref(ks)), "helm_annulus_exit_times")
    return st, ks.value


def helm_annulus_spectral_radius(plan: _Annulus, max_iters: int = 300, tol: float = 1e-10, cycles: int = 16):
    """Returns (status, rho, complex dominant eigenvalue, iterations) of G by power
    iteration (status HELM_OK when converged, HELM_MAXITER otherwise)."""
    r, lr, li = C.c_double(), C.c_double(), C.c_double()
    it = C.c_int()
    st = _check(load().helm_annulus_spectral_radius(plan.handle, int(max_iters), float(tol), int(cycles),
                                                    C.byref(r), C.byref(lr), C.byref(li), C.byref(it)),
                "helm_annulus_spectral_radius")
    return st, r.value, complex(lr.value, li.value), it.value


def helm_annulus_condition(plan: _Annulus, max_iters: int = 400, tol: float = 1e-10, cycles: int = 16):
    """Returns (status, sigma_max, sigma_min, cond, iterations) of G."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    it = C.c_int()
    st = _check(load().helm_annulus_condition(plan.handle, int(max_iters), float(tol), int(cycles), C.byref(a),
                                              C.byref(b), C.byref(c), C.byref(it)), "helm_annulus_condition")
    return st, a.value, b.value, c.value, it.value


class _Batch:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if self.handle is not None and _lib is not None:
            _lib.helm_batch_destroy(self.handle)
            self.handle = None


def helm_batch_create(hbm_cap_bytes: int = 0, stream=None) -> _Batch:
    out = C.c_void_p()
    _check(load().helm_batch_create(C.byref(out), int(hbm_cap_bytes), _stream_handle(stream)),
           "helm_batch_create")
    return _Batch(out)


def helm_batch_destroy(batch: _Batch) -> None:
    if batch.handle is not None:
        _check(load().helm_batch_destroy(batch.handle), "helm_batch_destroy")
        batch.handle = None


def helm_batch_submit(batch: _Batch, plan: _Plan, f, g, u, tol: float, max_outer: int):
    """Returns a ticket, or None when the memory cap does not admit the solve yet."""
    import torch
    D, n = plan.D, plan.n
    pf = _ptr(f, torch.complex128, (n,) * D, "f")
    pg = _ptr(g, torch.complex128, (n + 2,) * D, "g")
    pu = _ptr(u, torch.complex128, (n + 2,) * D, "u")
    t = C.c_uint64()
    st = load().helm_batch_submit(batch.handle, plan.handle, pf, pg, pu, float(tol), int(max_outer),
                                  C.byref(t))
    if st == HELM_ENOMEM:
        return None
    _check(st, "helm_batch_submit")
    return t.value


def helm_batch_submit_geom(batch: _Batch, ndim: int, n: int, h: float, k: float, prec: int, f, g, u,
                           tol: float, max_outer: int):
    """As helm_batch_submit without a plan.  Returns a ticket, or None over the memory cap."""
    import torch
    pf = _ptr(f, torch.complex128, (n,) * ndim, "f")
    pg = _ptr(g, torch.complex128, (n + 2,) * ndim, "g")
    pu = _ptr(u, torch.complex128, (n + 2,) * ndim, "u")
    t = C.c_uint64()
    st = load().helm_batch_submit_geom(batch.handle, int(ndim), int(n), float(h), float(k), int(prec),
                                       pf, pg, pu, float(tol), int(max_outer), C.byref(t))
    if st == HELM_ENOMEM:
        return None
    _check(st, "helm_batch_submit_geom")
    return t.value


def helm_batch_step(batch: _Batch, max_steps: int = 0) -> None:
    _check(load().helm_batch_step(batch.handle, int(max_steps)), "helm_batch_step")


def helm_batch_set_cycle(batch: _Batch, nu1: int, nu2: int, cycles: int = 1) -> None:
    _check(load().helm_batch_set_cycle(batch.handle, nu1, nu2, cycles), "helm_batch_set_cycle")


def helm_batch_set_lanes(batch: _Batch, lanes: int) -> None:
    _check(load().helm_batch_set_lanes(batch.handle, int(lanes)), "helm_batch_set_lanes")


def helm_batch_poll(batch: _Batch, ticket: int, max_outer: int):
    """Returns None while running, else (status, iters, relres history)."""
    done, status, iters = C.c_int(), C.c_int(), C.c_int()
    hist = np.zeros(max_outer + 1, dtype=np.float64)
    _check(load().helm_batch_poll(batch.handle, C.c_uint64(ticket), C.byref(done), C.byref(status),
                                  C.byref(iters), hist.ctypes.data_as(C.POINTER(C.c_double))),
           "helm_batch_poll")
    if not done.value:
        return None
    return status.value, iters.value, hist[: iters.value + 1].copy()


def helm_batch_set_host_result(batch: _Batch, ticket: int, u_host) -> None:
    """Also copy the solve's result (padded complex128, the device u's layout) into the
    contiguous host tensor u_host (pinned for an asynchronous copy) once it finishes."""
    import torch
    if u_host.device.type != "cpu" or not u_host.is_contiguous() or u_host.dtype != torch.complex128:
        raise ValueError("u_host: a contiguous complex128 CPU tensor")
    _check(load().helm_batch_set_host_result(batch.handle, C.c_uint64(ticket), C.c_void_p(u_host.data_ptr())),
           "helm_batch_set_host_result")


def helm_batch_submit_host(batch: _Batch, plan: _Plan, f_host, g_host, u_host, tol: float, max_outer: int):
    """Submit a solve from host tensors (contiguous complex128 CPU tensors; page-locked for
    asynchronous copies): f_host interior n^D, g_host the padded wall data, u_host receives
    the padded solution.  The library uploads, solves from zero and copies the result back.
    Returns a ticket, or None when the memory cap does not admit the solve yet."""
    import torch
    D, n = plan.D, plan.n
    for t, shape, name in ((f_host, (n,) * D, "f_host"), (g_host, (n + 2,) * D, "g_host"),
                           (u_host, (n + 2,) * D, "u_host")):
        if (t.device.type != "cpu" or not t.is_contiguous() or t.dtype != torch.complex128
                or tuple(t.shape) != shape):
            raise ValueError(f"{name}: a contiguous complex128 CPU tensor of shape {shape}")
    tk = C.c_uint64()
    st = load().helm_batch_submit_host(batch.handle, plan.handle, C.c_void_p(f_host.data_ptr()),
                                       C.c_void_p(g_host.data_ptr()), C.c_void_p(u_host.data_ptr()),
                                       float(tol), int(max_outer), C.byref(tk))
    if st == HELM_ENOMEM:
        return None
    _check(st, "helm_batch_submit_host")
    return tk.value


def helm_batch_info(batch: _Batch):
    a = C.c_int()
    b = C.c_size_t()
    _check(load().helm_batch_info(batch.handle, C.byref(a), C.byref(b)), "helm_batch_info")
    return a.value, b.value


def helm_batch_profile(batch: _Batch, max_steps: int = 0):
    """Per kernel kind: {name: (launches, device ms, algorithmic bytes)}."""
    nk = len(KERNEL_KINDS)
    la = (C.c_uint64 * nk)()
    ms = (C.c_double * nk)()
    by = (C.c_double * nk)()
    _check(load().helm_batch_profile(batch.handle, int(max_steps), la, ms, by, nk),
           "helm_batch_profile")
    return {KERNEL_KINDS[i]: (int(la[i]), float(ms[i]), float(by[i])) for i in range(nk)}
