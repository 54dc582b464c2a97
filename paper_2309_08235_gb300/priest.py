"""Thin ctypes binding of libpriest.so, the C ABI declared in include/priest.h.

Argument marshalling only: every step of the PRIEST path runs in the
library's CUDA kernels.  The functions below carry the C names; the
``Context`` class is a convenience wrapper over them that takes the plain
problem / CEM dicts of ``paper_2309_08235_gb300.workloads``.

If libpriest.so has not been built (``paper_2309_08235_gb300.build.build()``)
every call raises ``PriestError``: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PRIEST_OK, PRIEST_PENDING = 0, 1
PRIEST_ERR_INVALID, PRIEST_ERR_NOMEM, PRIEST_ERR_BUDGET = -1, -2, -3
PRIEST_ERR_CUDA, PRIEST_ERR_TIMEOUT, PRIEST_ERR_NUMERIC = -4, -5, -6
PRIEST_FP64_CHECK, PRIEST_FP32, PRIEST_MIXED_BF16 = 0, 1, 2
MAX_D = 48

STATUS_NAMES = {0: "PRIEST_OK", 1: "PRIEST_PENDING", -1: "PRIEST_ERR_INVALID", -2: "PRIEST_ERR_NOMEM",
                -3: "PRIEST_ERR_BUDGET", -4: "PRIEST_ERR_CUDA", -5: "PRIEST_ERR_TIMEOUT",
                -6: "PRIEST_ERR_NUMERIC"}

# Every symbol include/priest.h declares.
EXPORTS = ["priest_create", "priest_destroy", "priest_last_error", "priest_project", "priest_plan",
           "priest_plan_z", "priest_submit", "priest_poll", "priest_rng_normal", "priest_load",
           "priest_unload", "priest_plan_device", "priest_project_device", "priest_sync",
           "priest_kernel_launches", "priest_profile_enable", "priest_profile_read",
           "priest_project_noalloc", "priest_plan_batch", "priest_wait", "priest_serve_stats_get",
           "priest_rng_normal_device", "priest_plan_plain", "priest_plan_plain_device",
           "priest_project_plain", "priest_tc_selftest", "priest_plan_multi", "priest_chol_selftest",
           "priest_plan_batch_host", "priest_project_batch", "priest_read_elites", "priest_last_kernel",
           "priest_grid_info"]


class PriestError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


class priest_config(C.Structure):
    _fields_ = [
        ("dims", C.c_int), ("degree", C.c_int), ("n_p", C.c_int), ("horizon", C.c_double),
        ("rho", C.c_double), ("proj_iters", C.c_int), ("cem_iters", C.c_int), ("n_samples", C.c_int),
        ("n_proj", C.c_int), ("n_elite", C.c_int), ("sigma_lr", C.c_double), ("gamma", C.c_double),
        ("chol_eps", C.c_double), ("init_std", C.c_double), ("vmax", C.c_double), ("amax", C.c_double),
        ("use_bounds", C.c_int), ("smin", C.c_double * 3), ("smax", C.c_double * 3),
        ("precision", C.c_int), ("hbm_budget", C.c_size_t), ("autotune", C.c_int), ("serve_slots", C.c_int),
    ]


class priest_problem(C.Structure):
    _fields_ = [
        ("n_obs", C.c_int), ("center", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
        ("semi", C.POINTER(C.c_double)), ("b0", (C.c_double * 3) * 3), ("bf", (C.c_double * 3) * 3),
        ("bc_final_mask", C.c_int), ("seed", C.c_uint64), ("robot_id", C.c_int64),
        ("dims", C.c_int), ("n_p", C.c_int), ("n_samples", C.c_int), ("n_proj", C.c_int),
        ("n_elite", C.c_int), ("horizon", C.c_double), ("vmax", C.c_double), ("amax", C.c_double),
        ("cost_kind", C.c_int), ("w_acc", C.c_double), ("w_curv", C.c_double), ("w_path", C.c_double),
        ("curv_eps", C.c_double),
    ]


class priest_result(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("D", C.c_int), ("best_index", C.c_int), ("xi_best", C.c_double * MAX_D),
        ("resid", C.c_double), ("cost", C.c_double), ("c_aug", C.c_double), ("mu", C.c_double * MAX_D),
        ("latency_ms", C.c_double),
    ]


class priest_serve_stats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64), ("completed", C.c_int64), ("steps", C.c_int64), ("slot_steps", C.c_int64),
        ("max_active", C.c_int64), ("warm_starts", C.c_int64), ("deferred", C.c_int64), ("evictions", C.c_int64),
        ("budget_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
    ]


_P = C.POINTER(C.c_double)
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libpriest.so; raises PriestError when it is not built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise PriestError(PRIEST_ERR_CUDA, f"CUDA extension missing: {path} is not built "
                                               "(run paper_2309_08235_gb300.build.build())")
        L = C.CDLL(path)
        vp = C.c_void_p
        sig = {
            "priest_create": (C.c_int, [C.POINTER(priest_config), vp, C.POINTER(vp)]),
            "priest_destroy": (C.c_int, [vp]),
            "priest_last_error": (C.c_char_p, [vp]),
            "priest_project": (C.c_int, [vp, C.POINTER(priest_problem), C.c_int, _P, _P, _P, _P, _P]),
            "priest_plan": (C.c_int, [vp, C.POINTER(priest_problem), _P, _P, C.POINTER(priest_result)]),
            "priest_plan_z": (C.c_int, [vp, C.POINTER(priest_problem), _P, _P, _P, C.POINTER(priest_result)]),
            "priest_submit": (C.c_int, [vp, C.POINTER(priest_problem), C.POINTER(C.c_uint64)]),
            "priest_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(priest_result)]),
            "priest_rng_normal": (C.c_int, [C.c_uint64, C.c_int64, _P]),
            "priest_load": (C.c_int, [vp, C.POINTER(priest_problem), C.POINTER(vp)]),
            "priest_unload": (C.c_int, [vp, vp]),
            "priest_plan_device": (C.c_int, [vp, vp, vp, vp]),
            "priest_project_device": (C.c_int, [vp, vp, C.c_int, vp, vp, vp, vp, vp]),
            "priest_sync": (C.c_int, [vp]),
            "priest_kernel_launches": (C.c_int64, [vp]),
            "priest_profile_enable": (C.c_int, [vp, C.c_int]),
            "priest_profile_read": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
            "priest_project_noalloc": (C.c_int, [C.POINTER(priest_config), C.POINTER(priest_problem), C.c_int,
                                                 vp, vp, vp, vp, vp, vp]),
            "priest_plan_batch": (C.c_int, [vp, C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
            "priest_plan_batch_host": (C.c_int, [vp, C.c_int, C.POINTER(priest_problem), C.POINTER(vp),
                                                 C.POINTER(priest_result)]),
            "priest_project_batch": (C.c_int, [vp, C.c_int, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp),
                                               C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
            "priest_read_elites": (C.c_int, [vp, vp, C.POINTER(C.c_int), _P, _P]),
            "priest_last_kernel": (C.c_int, [vp]),
            "priest_grid_info": (C.c_int, [vp, vp, C.POINTER(C.c_int)]),
            "priest_wait": (C.c_int, [vp, C.c_uint64, C.c_double, C.POINTER(priest_result)]),
            "priest_serve_stats_get": (C.c_int, [vp, C.POINTER(priest_serve_stats)]),
            "priest_rng_normal_device": (C.c_int, [C.c_uint64, C.c_int64, vp, vp]),
            "priest_plan_plain": (C.c_int, [vp, C.POINTER(priest_problem), _P, _P, _P, C.POINTER(priest_result)]),
            "priest_plan_plain_device": (C.c_int, [vp, vp, vp, vp]),
            "priest_project_plain": (C.c_int, [vp, C.POINTER(priest_problem), C.c_int, _P, _P, _P, _P, _P]),
            "priest_tc_selftest": (C.c_int, [C.c_int, C.c_int, C.c_int, vp, vp, vp]),
            "priest_chol_selftest": (C.c_int, [C.c_int, C.c_int, vp, vp]),
            "priest_plan_multi": (C.c_int, [vp, C.POINTER(priest_problem), C.c_int, _P, _P, _P,
                                            C.POINTER(priest_result), C.POINTER(C.c_int), C.POINTER(priest_result)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _arr(a, n=None):
    if a is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a, a.ctypes.data_as(_P)


def make_config(problem=None, cem=None, precision=PRIEST_FP32, hbm_budget=0, **over):
    """priest_config from a workloads problem dict (context-level fields) and
    a CEM dict; keyword arguments override any field."""
    p = problem or {}
    c = cem or {}
    cfg = priest_config()
    dims = int(p.get("dims", 2))
    vals = {
        "dims": dims, "degree": int(p.get("degree", 10)), "n_p": int(p.get("n_p", 100)),
        "horizon": float(p.get("horizon", 8.0)), "rho": float(p.get("rho", 1.0)),
        "proj_iters": int(c.get("proj_iters", 50)), "cem_iters": int(c.get("cem_iters", 4)),
        "n_samples": int(c.get("n_samples", 200)), "n_proj": int(c.get("n_proj", 0)),
        "n_elite": int(c.get("n_elite", 0)), "sigma_lr": float(c.get("sigma_lr", 0.5)),
        "gamma": float(c.get("gamma", 1.0)), "chol_eps": float(c.get("chol_eps", 1e-8)),
        "init_std": float(c.get("init_std", 2.0)), "vmax": float(p.get("vmax", 1.0)),
        "amax": float(p.get("amax", 1.0)), "use_bounds": int(bool(p.get("use_bounds", False))),
        "precision": int(precision), "hbm_budget": int(hbm_budget), "autotune": 1,
    }
    vals.update(over)
    for k, v in vals.items():
        setattr(cfg, k, v)
    smin = np.zeros(3)
    smax = np.zeros(3)
    smin[:dims] = np.asarray(p.get("smin", np.zeros(dims)), dtype=float)[:dims]
    smax[:dims] = np.asarray(p.get("smax", np.zeros(dims)), dtype=float)[:dims]
    for ax in range(3):
        cfg.smin[ax] = smin[ax]
        cfg.smax[ax] = smax[ax]
    return cfg


def make_problem(p, cem=None, robot_id=-1, seed=None, per_problem_shape=False):
    """priest_problem from a workloads problem dict; returns (struct, keepalive)."""
    dims = int(p["dims"])
    n_obs = int(p.get("n_obs", len(p["center"])))
    keep = []
    s = priest_problem()
    s.n_obs = n_obs
    if n_obs:
        c, cp = _arr(p["center"], n_obs * dims)
        v, vp = _arr(p.get("vel", np.zeros((n_obs, dims))), n_obs * dims)
        m, mp = _arr(p["semi"], n_obs * 2)
        keep += [c, v, m]
        s.center, s.vel, s.semi = cp, vp, mp
    b0 = np.zeros((3, 3))
    bf = np.zeros((3, 3))
    b0[:dims] = np.asarray(p["b0"], dtype=float).reshape(dims, 3)
    bf[:dims] = np.asarray(p["bf"], dtype=float).reshape(dims, 3)
    for ax in range(3):
        for q in range(3):
            s.b0[ax][q] = b0[ax, q]
            s.bf[ax][q] = bf[ax, q]
    s.bc_final_mask = int(p.get("bc_final_mask", 7))
    s.seed = int(p.get("seed", 0) if seed is None else seed) & (2**64 - 1)
    s.robot_id = int(robot_id)
    s.cost_kind = int(p.get("cost_kind", 0))
    s.w_acc = float(p.get("w_acc", 1.0))
    s.w_curv = float(p.get("w_curv", 0.0))
    s.w_path = float(p.get("w_path", 0.0))
    s.curv_eps = float(p.get("curv_eps", 0.1))
    if per_problem_shape:
        s.dims = dims
        s.n_p = int(p["n_p"])
        s.horizon = float(p["horizon"])
        s.vmax = float(p["vmax"])
        s.amax = float(p["amax"])
        if cem:
            s.n_samples = int(cem["n_samples"])
            s.n_proj = int(cem.get("n_proj", 0))
            s.n_elite = int(cem.get("n_elite", 0))
    return s, keep


def _check(ctx, st):
    if st not in (PRIEST_OK, PRIEST_PENDING):
        msg = lib().priest_last_error(ctx)
        raise PriestError(st, msg.decode() if msg else "")
    return st


# ---- the C names --------------------------------------------------------

def priest_create(cfg, stream=None):
    h = C.c_void_p()
    st = lib().priest_create(C.byref(cfg), stream, C.byref(h))
    if st != PRIEST_OK:
        raise PriestError(st, "priest_create failed")
    return h


def priest_destroy(ctx):
    return lib().priest_destroy(ctx)


def priest_last_error(ctx):
    m = lib().priest_last_error(ctx)
    return m.decode() if m else ""


def priest_rng_normal(seed, count):
    out = np.zeros(int(count))
    st = lib().priest_rng_normal(C.c_uint64(int(seed) & (2**64 - 1)), int(count), out.ctypes.data_as(_P))
    if st != PRIEST_OK:
        raise PriestError(st, "priest_rng_normal failed")
    return out


def priest_project(ctx, prob, n, xi, lambda_io, xi_bar_out, resid_out, cost_out):
    return _check(ctx, lib().priest_project(ctx, C.byref(prob), int(n), *(
        None if a is None else a.ctypes.data_as(_P) for a in (xi, lambda_io, xi_bar_out, resid_out, cost_out))))


def priest_plan(ctx, prob, mu0, cov0, res):
    return _check(ctx, lib().priest_plan(ctx, C.byref(prob), _arr(mu0)[1], _arr(cov0)[1], C.byref(res)))


def priest_plan_z(ctx, prob, mu0, cov0, z, res):
    return _check(ctx, lib().priest_plan_z(ctx, C.byref(prob), _arr(mu0)[1], _arr(cov0)[1], z.ctypes.data_as(_P),
                                           C.byref(res)))


def priest_plan_plain(ctx, prob, mu0, cov0, z, res):
    zp = None if z is None else z.ctypes.data_as(_P)
    return _check(ctx, lib().priest_plan_plain(ctx, C.byref(prob), _arr(mu0)[1], _arr(cov0)[1], zp, C.byref(res)))


def priest_plan_plain_device(ctx, h, z_ptr, out_ptr):
    return _check(ctx, lib().priest_plan_plain_device(ctx, h, C.c_void_p(z_ptr), C.c_void_p(out_ptr)))


def priest_project_plain(ctx, prob, n, xi, lambda_io, xi_bar_out, resid_out, cost_out):
    return _check(ctx, lib().priest_project_plain(ctx, C.byref(prob), int(n), *(
        None if a is None else a.ctypes.data_as(_P) for a in (xi, lambda_io, xi_bar_out, resid_out, cost_out))))


def priest_tc_selftest(a_bf16, b_bf16, swap=0):
    """D = A B^T on the tensor core; a_bf16 (128 x k) and b_bf16 (n x k) are
    uint16 BF16 bit patterns.  Returns (status, D)."""
    a = np.ascontiguousarray(a_bf16, dtype=np.uint16)
    b = np.ascontiguousarray(b_bf16, dtype=np.uint16)
    n, k = b.shape
    d = np.zeros((128, n), dtype=np.float32)
    st = lib().priest_tc_selftest(int(n), int(k), int(swap), a.ctypes.data_as(C.c_void_p),
                                  b.ctypes.data_as(C.c_void_p), d.ctypes.data_as(C.c_void_p))
    return st, d


def priest_chol_selftest(a, threads=256):
    """The device Cholesky of the symmetric matrix a (D x D, FP64) on one CTA
    of `threads` threads.  Returns (status, L)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    D = a.shape[0]
    out = np.zeros((D, D), dtype=np.float64)
    st = lib().priest_chol_selftest(int(D), int(threads), a.ctypes.data_as(C.c_void_p),
                                    out.ctypes.data_as(C.c_void_p))
    return st, out


def priest_plan_multi(ctx, prob, M, mu0, cov0, z):
    """D-PRIEST; returns (best result, best distribution, list of M per-distribution results)."""
    best = priest_result()
    per = (priest_result * int(M))()
    bd = C.c_int()
    zp = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
    _check(ctx, lib().priest_plan_multi(ctx, C.byref(prob), int(M), _arr(mu0)[1], _arr(cov0)[1],
                                        None if zp is None else zp.ctypes.data_as(_P), C.byref(best), C.byref(bd),
                                        per))
    return best, bd.value, [per[j] for j in range(int(M))]


def priest_submit(ctx, prob):
    t = C.c_uint64()
    _check(ctx, lib().priest_submit(ctx, C.byref(prob), C.byref(t)))
    return t.value


def priest_poll(ctx, ticket, res):
    return _check(ctx, lib().priest_poll(ctx, C.c_uint64(ticket), C.byref(res)))


def priest_wait(ctx, ticket, res, timeout_ms=-1.0):
    """Blocks until the ticket's result is there (PRIEST_OK) or the timeout
    passes (PriestError with PRIEST_ERR_TIMEOUT)."""
    return _check(ctx, lib().priest_wait(ctx, C.c_uint64(ticket), float(timeout_ms), C.byref(res)))


def priest_serve_stats_get(ctx):
    s = priest_serve_stats()
    _check(ctx, lib().priest_serve_stats_get(ctx, C.byref(s)))
    return {name: getattr(s, name) for name, _ in priest_serve_stats._fields_}


def priest_rng_normal_device(seed, count, out_ptr, stream=None):
    """The standard-normal stream computed on the device into out_ptr (int)."""
    st = lib().priest_rng_normal_device(C.c_uint64(int(seed) & (2**64 - 1)), int(count), C.c_void_p(out_ptr),
                                        stream)
    if st != PRIEST_OK:
        raise PriestError(st, "priest_rng_normal_device failed")
    return st


def priest_load(ctx, prob):
    h = C.c_void_p()
    _check(ctx, lib().priest_load(ctx, C.byref(prob), C.byref(h)))
    return h


def priest_unload(ctx, h):
    return lib().priest_unload(ctx, h)


def priest_plan_device(ctx, h, z_ptr, out_ptr):
    return _check(ctx, lib().priest_plan_device(ctx, h, C.c_void_p(z_ptr), C.c_void_p(out_ptr)))


def priest_plan_batch(ctx, handles, z_ptrs, out_ptrs):
    """Batched solve; handles from priest_load, device pointers as ints."""
    n = len(handles)
    arr = C.c_void_p * n
    hs = arr(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    zs = arr(*[int(z) for z in z_ptrs])
    os_ = arr(*[int(o) for o in out_ptrs])
    return _check(ctx, lib().priest_plan_batch(ctx, n, hs, zs, os_))


def priest_plan_batch_host(ctx, problems, z_list, results):
    """Batched solve through host buffers.  problems: priest_problem structs,
    or a ctypes array of them (passed as is); z_list: host float64 arrays
    (L x N_i x D, pinned or pageable) or their addresses, or a ctypes array of
    c_void_p (passed as is); results: a ctypes array of priest_result
    (len(problems)), written.  A caller repeating a batch can keep the two
    ctypes arrays (priest_problem_array, pointer_array) and skip rebuilding
    them on every call."""
    n = len(problems)
    parr = problems if isinstance(problems, C.Array) else priest_problem_array(problems)
    zs = z_list if isinstance(z_list, C.Array) else pointer_array(z_list)
    return _check(ctx, lib().priest_plan_batch_host(ctx, n, parr, zs, results))


def priest_problem_array(problems):
    """A ctypes array of the given priest_problem structs."""
    return (priest_problem * len(problems))(*problems)


def pointer_array(arrays):
    """A ctypes array of the host addresses of numpy arrays (or ints)."""
    return (C.c_void_p * len(arrays))(*[a.__array_interface__["data"][0] if hasattr(a, "__array_interface__")
                                         else int(a) for a in arrays])


def priest_project_batch(ctx, handles, rows, xi_ptrs, lam_ptrs, xb_ptrs, r_ptrs, c1_ptrs):
    """Batched projection of caller samples; device pointers as ints (lam_ptrs
    may be None or hold 0 entries)."""
    n = len(handles)
    arr = C.c_void_p * n
    hs = arr(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    rr = (C.c_int * n)(*[int(x) for x in rows])
    lam = None if lam_ptrs is None else arr(*[int(x) if x else None for x in lam_ptrs])
    return _check(ctx, lib().priest_project_batch(ctx, n, hs, rr, arr(*[int(x) for x in xi_ptrs]), lam,
                                                  arr(*[int(x) for x in xb_ptrs]), arr(*[int(x) for x in r_ptrs]),
                                                  arr(*[int(x) for x in c1_ptrs])))


def priest_read_elites(ctx, h, n_elite, n):
    """(EliteSet indices, r, c_1) of the last CEM iteration of a solve; h a
    loaded handle or None for the context's last host-buffer solve."""
    el = np.zeros(int(n_elite), dtype=np.int32)
    r = np.zeros(int(n))
    c1 = np.zeros(int(n))
    _check(ctx, lib().priest_read_elites(ctx, h, el.ctypes.data_as(C.POINTER(C.c_int)), r.ctypes.data_as(_P),
                                         c1.ctypes.data_as(_P)))
    return el, r, c1


def priest_last_kernel(ctx):
    return int(lib().priest_last_kernel(ctx))


def priest_grid_info(ctx, h=None):
    """(cells in x, cells in y, entries) of the static-obstacle grid of a
    loaded problem's FP32 tables (h None: the context's last host-buffer
    solve); zeros without a grid."""
    out = (C.c_int * 3)()
    _check(ctx, lib().priest_grid_info(ctx, h, out))
    return int(out[0]), int(out[1]), int(out[2])


def priest_project_device(ctx, h, n, xi_ptr, lam_ptr, xb_ptr, r_ptr, c1_ptr):
    return _check(ctx, lib().priest_project_device(ctx, h, int(n), C.c_void_p(xi_ptr), C.c_void_p(lam_ptr),
                                                   C.c_void_p(xb_ptr), C.c_void_p(r_ptr), C.c_void_p(c1_ptr)))


def priest_sync(ctx):
    return _check(ctx, lib().priest_sync(ctx))


def priest_kernel_launches(ctx):
    return int(lib().priest_kernel_launches(ctx))


def priest_profile_enable(ctx, enable):
    return _check(ctx, lib().priest_profile_enable(ctx, int(bool(enable))))


def priest_profile_read(ctx):
    n = C.c_int64()
    ms = C.c_double()
    _check(ctx, lib().priest_profile_read(ctx, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def priest_project_noalloc(cfg, prob, n, xi_ptr, lam_ptr, xb_ptr, r_ptr, c1_ptr, stream=None):
    """Projection without device allocation; device pointers as ints.  Returns
    the status code (no context, so no message)."""
    return lib().priest_project_noalloc(C.byref(cfg), C.byref(prob), int(n), C.c_void_p(xi_ptr),
                                        C.c_void_p(lam_ptr), C.c_void_p(xb_ptr), C.c_void_p(r_ptr),
                                        C.c_void_p(c1_ptr), stream)


# ---- convenience wrapper ---------------------------------------------------

def result_dict(res):
    D = res.D
    return {"status": res.status, "D": D, "best_index": res.best_index,
            "best": np.array(res.xi_best[:D]), "r": res.resid, "c1": res.cost, "c_aug": res.c_aug,
            "mu": np.array(res.mu[:D]), "latency_ms": res.latency_ms}


class Context:
    """A priest_ctx bound to a workloads problem / CEM description."""

    def __init__(self, problem=None, cem=None, precision=PRIEST_FP32, stream=None, hbm_budget=0, **over):
        self.cfg = make_config(problem, cem, precision, hbm_budget, **over)
        self.h = priest_create(self.cfg, stream)

    def close(self):
        if self.h:
            priest_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def project(self, p, xi, lam=None):
        D = int(p["dims"]) * (self.cfg.degree + 1)
        xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(-1, D))
        n = xi.shape[0]
        lam_io = None if lam is None else np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(n, D)).copy()
        xb = np.zeros((n, D))
        r = np.zeros(n)
        c1 = np.zeros(n)
        prob, keep = make_problem(p)
        priest_project(self.h, prob, n, xi, lam_io, xb, r, c1)
        return xb, lam_io, r, c1

    def project_plain(self, p, xi, lam=None):
        """As project, through the plain per-problem FP32 path."""
        D = int(p["dims"]) * (self.cfg.degree + 1)
        xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(-1, D))
        n = xi.shape[0]
        lam_io = None if lam is None else np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(n, D)).copy()
        xb = np.zeros((n, D))
        r = np.zeros(n)
        c1 = np.zeros(n)
        prob, keep = make_problem(p)
        priest_project_plain(self.h, prob, n, xi, lam_io, xb, r, c1)
        return xb, lam_io, r, c1

    def plan_plain(self, p, z=None, mu0=None, cov0=None, cem=None):
        """As plan, through the plain per-problem FP32 path."""
        prob, keep = make_problem(p, cem, per_problem_shape=cem is not None)
        res = priest_result()
        z = None if z is None else np.ascontiguousarray(np.asarray(z, dtype=np.float64))
        priest_plan_plain(self.h, prob, mu0, cov0, z, res)
        return result_dict(res)

    def plan_multi(self, p, M, z=None, mu0=None, cov0=None, cem=None):
        """D-PRIEST over M distributions: dict with the best result, its
        distribution and every distribution's result."""
        prob, keep = make_problem(p, cem, per_problem_shape=cem is not None)
        best, bd, per = priest_plan_multi(self.h, prob, M, mu0, cov0, z)
        return {"best": result_dict(best), "dist": bd, "per_dist": [result_dict(r) for r in per]}

    def plan(self, p, z=None, mu0=None, cov0=None, cem=None):
        """Alg. 1 on p; with cem given, the problem's own sizes (dims, n_p,
        horizon, bounds, sample counts) override the context defaults."""
        prob, keep = make_problem(p, cem, per_problem_shape=cem is not None)
        res = priest_result()
        if z is None:
            priest_plan(self.h, prob, mu0, cov0, res)
        else:
            z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
            priest_plan_z(self.h, prob, mu0, cov0, z, res)
        return result_dict(res)

    def submit(self, p, cem=None, robot_id=-1, seed=None):
        """Queues a solve on the serving loop; returns the ticket."""
        prob, keep = make_problem(p, cem, robot_id=robot_id, seed=seed, per_problem_shape=True)
        return priest_submit(self.h, prob)

    def poll(self, ticket):
        """The result dict, or None while the solve is pending."""
        res = priest_result()
        st = priest_poll(self.h, ticket, res)
        return None if st == PRIEST_PENDING else result_dict(res)

    def wait(self, ticket, timeout_ms=-1.0):
        res = priest_result()
        priest_wait(self.h, ticket, res, timeout_ms)
        return result_dict(res)

    def serve_stats(self):
        return priest_serve_stats_get(self.h)

    def launches(self):
        return priest_kernel_launches(self.h)
