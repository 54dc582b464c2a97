"""Plain FP64 CPU oracle for PRIEST (arXiv 2309.08235).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` leg may import this
package.  The product path (the CUDA library and its binding) never imports,
links or executes anything here, and this package shares no code with it.

The arithmetic lives in ``priest_oracle.c`` (plain C, FP64, built with
``-O2 -ffp-contract=off``, single-threaded); this module only compiles it and
marshals numpy arrays through ctypes.  A problem is the plain dict produced by
``paper_2309_08235_gb300.workloads`` (obstacles, boundary values, sizes); that
module holds inputs only, none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "priest_oracle.c")
_HDR = os.path.join(_HERE, "priest_oracle.h")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("dims", C.c_int), ("degree", C.c_int), ("n_p", C.c_int),
        ("horizon", C.c_double), ("rho", C.c_double),
        ("vmax", C.c_double), ("amax", C.c_double),
        ("use_bounds", C.c_int), ("smin", C.c_double * 3), ("smax", C.c_double * 3),
        ("bc_final_mask", C.c_int),
        ("b0", (C.c_double * 3) * 3), ("bf", (C.c_double * 3) * 3),
        ("n_obs", C.c_int),
        ("center", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
        ("semi", C.POINTER(C.c_double)),
        ("cost_kind", C.c_int), ("w_acc", C.c_double), ("w_curv", C.c_double), ("w_path", C.c_double),
        ("curv_eps", C.c_double),
    ]


class _Cem(C.Structure):
    _fields_ = [
        ("proj_iters", C.c_int), ("cem_iters", C.c_int), ("n_samples", C.c_int),
        ("n_proj", C.c_int), ("n_elite", C.c_int),
        ("sigma_lr", C.c_double), ("gamma", C.c_double), ("chol_eps", C.c_double),
        ("init_std", C.c_double),
    ]


_P = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_basis": (C.c_int, [C.c_int, C.c_int, C.c_double, _P, _P, _P]),
                "orc_equality": (C.c_int, [C.POINTER(_Problem), _P, _P]),
                "orc_kkt_matrix": (C.c_int, [C.POINTER(_Problem), _P]),
                "orc_obstacle_polar": (None, [C.c_int, _P, _P, C.c_double, C.c_double,
                                              _P, _P, _P, _P]),
                "orc_bound_polar": (None, [C.c_int, _P, C.c_double, _P, _P, _P, _P]),
                "orc_project": (C.c_int, [C.POINTER(_Problem), C.c_int, C.c_int, _P, _P, _P, _P]),
                "orc_project_eq": (C.c_int, [C.POINTER(_Problem), C.c_int, _P, _P]),
                "orc_residual_cost": (C.c_int, [C.POINTER(_Problem), C.c_int, _P, _P, _P]),
                "orc_residual_stacked": (C.c_int, [C.POINTER(_Problem), C.c_int, _P, _P]),
                "orc_select": (C.c_int, [C.c_int, _P, _P, C.c_int, C.c_int, _PI, _PI]),
                "orc_refit": (C.c_int, [C.c_int, C.c_int, _P, _P, C.c_double, C.c_double, _P, _P]),
                "orc_cholesky": (C.c_int, [C.c_int, _P, _P]),
                "orc_rng_normal": (None, [C.c_uint64, C.c_int64, _P]),
                "orc_default_mean": (C.c_int, [C.POINTER(_Problem), _P]),
                "orc_plan": (C.c_int, [C.POINTER(_Problem), C.POINTER(_Cem), _P, _P, _P,
                                       C.c_uint64, _P, _P, _P, _P, _P, _PI]),
                "orc_plan_warm": (C.c_int, [C.POINTER(_Problem), C.POINTER(_Cem), _P, _P, _P, _P,
                                            C.c_uint64, _P, _P, _P, _P, _P, _PI, _P]),
                "orc_multi_default_means": (C.c_int, [C.POINTER(_Problem), C.c_int, C.c_double, _P]),
                "orc_plan_multi": (C.c_int, [C.POINTER(_Problem), C.POINTER(_Cem), C.c_int, _P, _P, _P,
                                             C.c_uint64, _P, _P, _PI, _P, _P, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def _problem(p):
    """Build the C struct from a problem dict; returns (struct, keepalive)."""
    dims = int(p["dims"])
    n_obs = int(p.get("n_obs", len(p["center"])))
    center = _f64(p["center"], (n_obs, dims)) if n_obs else np.zeros((1, dims))
    vel = _f64(p.get("vel", np.zeros((n_obs, dims))), (n_obs, dims)) if n_obs else np.zeros((1, dims))
    semi = _f64(p["semi"], (n_obs, 2)) if n_obs else np.ones((1, 2))
    s = _Problem()
    s.dims = dims
    s.degree = int(p.get("degree", 10))
    s.n_p = int(p["n_p"])
    s.horizon = float(p["horizon"])
    s.rho = float(p.get("rho", 1.0))
    s.vmax = float(p["vmax"])
    s.amax = float(p["amax"])
    s.use_bounds = int(bool(p.get("use_bounds", False)))
    smin = np.zeros(3)
    smax = np.zeros(3)
    smin[:dims] = np.asarray(p.get("smin", np.zeros(dims)), dtype=float)[:dims]
    smax[:dims] = np.asarray(p.get("smax", np.zeros(dims)), dtype=float)[:dims]
    for ax in range(3):
        s.smin[ax] = smin[ax]
        s.smax[ax] = smax[ax]
    s.bc_final_mask = int(p.get("bc_final_mask", 7))
    b0 = np.zeros((3, 3))
    bf = np.zeros((3, 3))
    b0[:dims] = np.asarray(p["b0"], dtype=float).reshape(dims, 3)
    bf[:dims] = np.asarray(p["bf"], dtype=float).reshape(dims, 3)
    for ax in range(3):
        for q in range(3):
            s.b0[ax][q] = b0[ax, q]
            s.bf[ax][q] = bf[ax, q]
    s.n_obs = n_obs
    s.center = _dptr(center)
    s.vel = _dptr(vel)
    s.semi = _dptr(semi)
    s.cost_kind = int(p.get("cost_kind", 0))
    s.w_acc = float(p.get("w_acc", 1.0))
    s.w_curv = float(p.get("w_curv", 0.0))
    s.w_path = float(p.get("w_path", 0.0))
    s.curv_eps = float(p.get("curv_eps", 0.1))
    return s, (center, vel, semi)


def n_coeffs(p):
    return int(p["dims"]) * (int(p.get("degree", 10)) + 1)


def basis(degree, n_p, horizon):
    nv = degree + 1
    P = np.zeros((n_p, nv))
    Pd = np.zeros((n_p, nv))
    Pdd = np.zeros((n_p, nv))
    _check(_load().orc_basis(degree, n_p, horizon, _dptr(P), _dptr(Pd), _dptr(Pdd)), "orc_basis")
    return P, Pd, Pdd


def equality(p):
    s, keep = _problem(p)
    nv = int(p.get("degree", 10)) + 1
    A = np.zeros((6, nv))
    b = np.zeros((3, 6))
    n = _load().orc_equality(C.byref(s), _dptr(A), _dptr(b))
    if n < 0:
        raise OracleError(f"orc_equality failed with {n}")
    dims = int(p["dims"])
    return A[:n].copy(), b.reshape(-1)[: dims * n].reshape(dims, n).copy()


def kkt_matrix(p):
    s, keep = _problem(p)
    nv = int(p.get("degree", 10)) + 1
    K = np.zeros((nv + 6) * (nv + 6))
    n = _load().orc_kkt_matrix(C.byref(s), _dptr(K))
    if n < 0:
        raise OracleError(f"orc_kkt_matrix failed with {n}")
    return K[: n * n].reshape(n, n).copy()


def obstacle_polar(dims, pos, o, a, b):
    pos = _f64(pos)
    o = _f64(o)
    al = C.c_double()
    be = C.c_double()
    d = C.c_double()
    e = np.zeros(3)
    _load().orc_obstacle_polar(dims, _dptr(pos), _dptr(o), float(a), float(b),
                               C.byref(al), C.byref(be), C.byref(d), _dptr(e))
    return al.value, be.value, d.value, e[:dims].copy()


def bound_polar(dims, v, vmax):
    v = _f64(v)
    al = C.c_double()
    be = C.c_double()
    d = C.c_double()
    e = np.zeros(3)
    _load().orc_bound_polar(dims, _dptr(v), float(vmax), C.byref(al), C.byref(be), C.byref(d), _dptr(e))
    return al.value, be.value, d.value, e[:dims].copy()


def project(p, xi, K, lam=None, xi_bar0=None):
    """K AM iterations from xi_bar0 (default Pi_A(xi)); returns (xi_bar, lambda)."""
    s, keep = _problem(p)
    D = n_coeffs(p)
    xi = _f64(xi).reshape(-1, D)
    N = xi.shape[0]
    lam = np.zeros((N, D)) if lam is None else _f64(lam, (N, D)).copy()
    xb0 = None if xi_bar0 is None else _f64(xi_bar0, (N, D))
    out = np.zeros((N, D))
    _check(_load().orc_project(C.byref(s), int(K), N, _dptr(xi), _dptr(xb0), _dptr(lam), _dptr(out)),
           "orc_project")
    return out, lam


def project_eq(p, xi):
    s, keep = _problem(p)
    D = n_coeffs(p)
    xi = _f64(xi).reshape(-1, D)
    out = np.zeros_like(xi)
    _check(_load().orc_project_eq(C.byref(s), xi.shape[0], _dptr(xi), _dptr(out)), "orc_project_eq")
    return out


def residual_cost(p, xi_bar):
    s, keep = _problem(p)
    D = n_coeffs(p)
    xb = _f64(xi_bar).reshape(-1, D)
    r = np.zeros(xb.shape[0])
    c1 = np.zeros(xb.shape[0])
    _check(_load().orc_residual_cost(C.byref(s), xb.shape[0], _dptr(xb), _dptr(r), _dptr(c1)),
           "orc_residual_cost")
    return r, c1


def residual_stacked(p, xi_bar):
    s, keep = _problem(p)
    D = n_coeffs(p)
    xb = _f64(xi_bar).reshape(-1, D)
    r = np.zeros(xb.shape[0])
    _check(_load().orc_residual_stacked(C.byref(s), xb.shape[0], _dptr(xb), _dptr(r)),
           "orc_residual_stacked")
    return r


def select(r, c_aug, n_proj, n_elite):
    r = _f64(r)
    c_aug = _f64(c_aug)
    pi = np.zeros(n_proj, dtype=np.int32)
    ei = np.zeros(n_elite, dtype=np.int32)
    _check(_load().orc_select(len(r), _dptr(r), _dptr(c_aug), n_proj, n_elite,
                              pi.ctypes.data_as(_PI), ei.ctypes.data_as(_PI)), "orc_select")
    return pi, ei


def refit(elites, c_aug, mu, cov, sigma_lr, gamma):
    el = _f64(elites)
    m, D = el.shape
    mu = _f64(mu).copy()
    cov = _f64(cov, (D, D)).copy()
    _check(_load().orc_refit(D, m, _dptr(el), _dptr(_f64(c_aug)), float(sigma_lr), float(gamma),
                             _dptr(mu), _dptr(cov)), "orc_refit")
    return mu, cov


def cholesky(S):
    S = _f64(S)
    D = S.shape[0]
    L = np.zeros_like(S)
    _check(_load().orc_cholesky(D, _dptr(S), _dptr(L)), "orc_cholesky")
    return L


def rng_normal(seed, count):
    out = np.zeros(int(count))
    _load().orc_rng_normal(C.c_uint64(int(seed) & (2**64 - 1)), int(count), _dptr(out))
    return out


def default_mean(p):
    s, keep = _problem(p)
    mu = np.zeros(n_coeffs(p))
    _check(_load().orc_default_mean(C.byref(s), _dptr(mu)), "orc_default_mean")
    return mu


def plan(p, cem, mu0=None, cov0=None, z=None, seed=None, lam0=None, want_lam=False):
    """Alg. 1.  cem: dict with proj_iters, cem_iters, n_samples, n_proj,
    n_elite, sigma_lr, gamma, chol_eps, init_std.  lam0 (N x D): lambda^0 of
    the first CEM iteration's projection (multiplier warm start); want_lam:
    also return the multipliers after the last CEM iteration's projection.
    Returns a dict."""
    s, keep = _problem(p)
    c = _Cem()
    for name, _ in _Cem._fields_:
        setattr(c, name, type(getattr(c, name))(cem[name]))
    D = n_coeffs(p)
    N = int(cem["n_samples"])
    mu0 = _f64(mu0)
    cov0 = _f64(cov0)
    lam0 = None if lam0 is None else _f64(lam0, (N, D))
    if z is not None:
        z = _f64(z)
        assert z.size == cem["cem_iters"] * cem["n_samples"] * D
    best = np.zeros(D)
    br = C.c_double()
    bc = C.c_double()
    mu = np.zeros(D)
    cov = np.zeros((D, D))
    el = np.zeros(cem["n_elite"], dtype=np.int32)
    lam_out = np.zeros((N, D)) if want_lam else None
    seed = int(p.get("seed", 0) if seed is None else seed)
    rc = _load().orc_plan_warm(C.byref(s), C.byref(c), _dptr(mu0), _dptr(cov0), _dptr(lam0), _dptr(z),
                               C.c_uint64(seed & (2**64 - 1)), _dptr(best), C.byref(br), C.byref(bc),
                               _dptr(mu), _dptr(cov), el.ctypes.data_as(_PI), _dptr(lam_out))
    _check(rc, "orc_plan_warm")
    out = {"best": best, "r": br.value, "c_aug": bc.value, "mu": mu, "cov": cov, "elites": el}
    if want_lam:
        out["lam"] = lam_out
    return out


def multi_default_means(p, M, spread):
    """D-PRIEST default means (M x D): the straight line bowed sideways."""
    s, keep = _problem(p)
    out = np.zeros((M, n_coeffs(p)))
    _check(_load().orc_multi_default_means(C.byref(s), int(M), float(spread), _dptr(out)), "orc_multi_default_means")
    return out


def plan_multi(p, cem, M, mu0=None, cov0=None, z=None, seed=None):
    """D-PRIEST (Sec. D-PRIEST): M distributions refined in parallel on one
    stacked projection; returns the best over the M and each distribution's
    best elite."""
    s, keep = _problem(p)
    c = _Cem()
    for name, _ in _Cem._fields_:
        setattr(c, name, type(getattr(c, name))(cem[name]))
    D = n_coeffs(p)
    mu0 = None if mu0 is None else _f64(mu0, (M, D))
    cov0 = None if cov0 is None else _f64(cov0, (M, D, D))
    z = None if z is None else _f64(z)
    best = np.zeros(D)
    bc = C.c_double()
    bd = C.c_int()
    db = np.zeros((M, D))
    dr = np.zeros(M)
    dc = np.zeros(M)
    mu = np.zeros((M, D))
    seed = int(p.get("seed", 0) if seed is None else seed)
    rc = _load().orc_plan_multi(C.byref(s), C.byref(c), int(M), _dptr(mu0), _dptr(cov0), _dptr(z),
                                C.c_uint64(seed & (2**64 - 1)), _dptr(best), C.byref(bc), C.byref(bd), _dptr(db),
                                _dptr(dr), _dptr(dc), _dptr(mu))
    _check(rc, "orc_plan_multi")
    return {"best": best, "c_aug": bc.value, "dist": bd.value, "dist_best": db, "dist_r": dr, "dist_c_aug": dc,
            "mu": mu}
