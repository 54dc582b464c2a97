"""Seeded synthetic inputs shaped like PRIEST's navigation scenes.

This module produces INPUTS only: obstacle lists, boundary values, problem
sizes, CEM settings and standard-normal draws.  It holds none of the method's
arithmetic, and it is the one module that both the CUDA path's tests/bench and
the CPU oracle's tests read from.

The paper's benchmark scenes (BARN, its point-to-point rooms, its dynamic
scene; Sec. IV-A) are not available, so these seeded scenes stand in for them
with the paper's shapes: 2-D circles / 3-D axis-aligned ellipsoids (a, a, b)
of 0.2-0.8 m, some moving at constant velocity (Sec. IV-A, dynamic
environment), a start and a goal "at rest" (zero velocity and acceleration).

A problem is a plain dict:
  dims, degree, n_p, horizon, rho, vmax, amax, use_bounds, smin, smax,
  bc_final_mask, b0 (dims x 3: pos, vel, acc at t0), bf (dims x 3 at tf),
  center (n_obs x dims, at t = 0), vel (n_obs x dims), semi (n_obs x 2: a, b),
  n_obs, seed.
A CEM setting is a dict: proj_iters, cem_iters, n_samples, n_proj, n_elite,
  sigma_lr, gamma, chol_eps, init_std.
"""
from __future__ import annotations

import math

import numpy as np

DEGREE = 10

# Constants the paper leaves open; both the oracle and the CUDA path receive
# them as inputs.
SIGMA_LR = 0.5
GAMMA = 1.0
CHOL_EPS = 1e-8
INIT_STD_2D = 2.0
INIT_STD_3D = 1.5

# Velocity / acceleration bounds for the 2-D scenes whose description gives
# none (the 30 x 30 m scene and the batched / serving mixes).
VMAX_2D = 12.0
AMAX_2D = 14.0


def default_counts(n_samples: int) -> tuple[int, int]:
    """N_proj = floor(80 N / 110) (the paper's 110 / 80 ratio) and N_elite = N / 10."""
    n_proj = max(1, (80 * n_samples) // 110)
    n_elite = max(1, min(n_proj, n_samples // 10))
    return n_proj, n_elite


def cem_settings(n_samples, proj_iters, cem_iters, n_proj=None, n_elite=None, dims=2):
    dp, de = default_counts(n_samples)
    return {
        "proj_iters": int(proj_iters),
        "cem_iters": int(cem_iters),
        "n_samples": int(n_samples),
        "n_proj": int(dp if n_proj is None else n_proj),
        "n_elite": int(de if n_elite is None else n_elite),
        "sigma_lr": SIGMA_LR,
        "gamma": GAMMA,
        "chol_eps": CHOL_EPS,
        "init_std": INIT_STD_2D if dims == 2 else INIT_STD_3D,
    }


def _at_rest(p):
    p = np.asarray(p, dtype=float)
    out = np.zeros((len(p), 3))
    out[:, 0] = p
    return out


def _place(rng, n, lo, hi, radii, keep_clear, dims):
    """Uniform centres in [lo, hi]^dims, rejecting those within r + 0.5 m of
    any point in keep_clear."""
    lo = np.broadcast_to(np.asarray(lo, dtype=float), (dims,))
    hi = np.broadcast_to(np.asarray(hi, dtype=float), (dims,))
    out = np.zeros((n, dims))
    for j in range(n):
        for _ in range(1000):
            c = lo + (hi - lo) * rng.random(dims)
            if all(np.linalg.norm(c - k) > radii[j] + 0.5 for k in keep_clear):
                break
        out[j] = c
    return out


def problem(dims, n_p, horizon, start, goal, center, vel, semi, vmax, amax, seed=0,
            rho=1.0, use_bounds=False, smin=None, smax=None, bc_final_mask=7, degree=DEGREE):
    center = np.asarray(center, dtype=float).reshape(-1, dims)
    n_obs = center.shape[0]
    return {
        "dims": int(dims), "degree": int(degree), "n_p": int(n_p), "horizon": float(horizon),
        "rho": float(rho), "vmax": float(vmax), "amax": float(amax),
        "use_bounds": bool(use_bounds),
        "smin": np.zeros(dims) if smin is None else np.asarray(smin, dtype=float),
        "smax": np.zeros(dims) if smax is None else np.asarray(smax, dtype=float),
        "bc_final_mask": int(bc_final_mask),
        "b0": _at_rest(start), "bf": _at_rest(goal),
        "center": center,
        "vel": np.zeros_like(center) if vel is None else np.asarray(vel, dtype=float).reshape(n_obs, dims),
        "semi": np.asarray(semi, dtype=float).reshape(n_obs, 2),
        "n_obs": n_obs, "seed": int(seed),
    }


def scene_small_2d(seed=0, n_obs=20, n_p=100, horizon=5.0, vmax=1.4, amax=1.5):
    """20 static circles, r ~ U[0.3, 0.6], centres U[2, 16]^2; (0,0) -> (18,18)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.3, 0.6, n_obs)
    start, goal = np.array([0.0, 0.0]), np.array([18.0, 18.0])
    c = _place(rng, n_obs, 2.0, 16.0, r, [start, goal], 2)
    return problem(2, n_p, horizon, start, goal, c, None, np.stack([r, r], 1), vmax, amax, seed)


def scene_clutter_2d(seed=1, n_static=90, n_dyn=10, n_p=100, horizon=8.0, size=30.0,
                     vmax=VMAX_2D, amax=AMAX_2D):
    """n_static circles r ~ U[0.2, 0.5] plus n_dyn moving ones (v ~ U[-1, 1]^2)
    in a size x size box; start (1,1) -> goal (size-1, size-1); centres
    U[2, size-2]^2 kept r + 0.5 m clear of start and goal."""
    rng = np.random.default_rng(seed)
    n = n_static + n_dyn
    r = rng.uniform(0.2, 0.5, n)
    start, goal = np.array([1.0, 1.0]), np.array([size - 1.0, size - 1.0])
    c = _place(rng, n, 2.0, size - 2.0, r, [start, goal], 2)
    v = np.zeros((n, 2))
    v[n_static:] = rng.uniform(-1.0, 1.0, (n_dyn, 2))
    return problem(2, n_p, horizon, start, goal, c, v, np.stack([r, r], 1), vmax, amax, seed)


def scene_ellipsoids_3d(seed=2, n_obs=200, n_p=150, horizon=10.0, vmax=2.0, amax=3.0):
    """n_obs static ellipsoids, a, b ~ U[0.3, 0.8], in 20 x 20 x 8 m;
    (1,1,1) -> (19,19,7)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.3, 0.8, n_obs)
    b = rng.uniform(0.3, 0.8, n_obs)
    start, goal = np.array([1.0, 1.0, 1.0]), np.array([19.0, 19.0, 7.0])
    c = _place(rng, n_obs, [0.0, 0.0, 0.0], [20.0, 20.0, 8.0], np.maximum(a, b), [start, goal], 3)
    return problem(3, n_p, horizon, start, goal, c, None, np.stack([a, b], 1), vmax, amax, seed)


# BARN-style cost weights (chosen: the paper names the three terms but gives
# no weights) and the curvature regularisation of rest states.
BARN_WEIGHTS = {"w_acc": 1.0, "w_curv": 0.1, "w_path": 1.0, "curv_eps": 0.1}


def with_barn_cost(p, **w):
    """The problem with the BARN-style cost c_1: acceleration, curvature and
    path-following (distance to the straight start-goal segment) penalties."""
    q = dict(p)
    q["cost_kind"] = 1
    q.update(BARN_WEIGHTS)
    q.update(w)
    return q


def scene_dynamic_2d(seed=3, n_obs=10, n_p=100, horizon=10.0):
    """Dynamic environment: n_obs circles r = 0.3 m moving at 0.1 m/s against
    the robot's direction, start (0, 0) -> goal (8, 0), v_max 1 m/s, a_max
    1 m/s^2 (chosen), centres U[2, 7] x U[-1.5, 1.5], BARN-style cost."""
    rng = np.random.default_rng(seed)
    r = np.full(n_obs, 0.3)
    start, goal = np.array([0.0, 0.0]), np.array([8.0, 0.0])
    c = np.stack([rng.uniform(2.0, 7.0, n_obs), rng.uniform(-1.5, 1.5, n_obs)], 1)
    v = np.tile(np.array([[-0.1, 0.0]]), (n_obs, 1))
    p = problem(2, n_p, horizon, start, goal, c, v, np.stack([r, r], 1), 1.0, 1.0, seed)
    return with_barn_cost(p)


def scene_p2p_2d(seed=4, n_obs=50, n_p=100, horizon=8.0):
    """Point-to-point 2-D: n_obs circles r = 0.4 m, centres U[1, 19]^2 kept
    clear of start (0, 0) and goal (20, 20); v_max 5, a_max 5 (chosen)."""
    rng = np.random.default_rng(seed)
    r = np.full(n_obs, 0.4)
    start, goal = np.array([0.0, 0.0]), np.array([20.0, 20.0])
    c = _place(rng, n_obs, 1.0, 19.0, r, [start, goal], 2)
    return problem(2, n_p, horizon, start, goal, c, None, np.stack([r, r], 1), 5.0, 5.0, seed)


def scene_p2p_3d(seed=5, n_obs=25, n_p=100, horizon=6.0):
    """Point-to-point 3-D room of 7 x 7 x 3 m: n_obs spheres r = 0.68 m,
    start (0.5, 0.5, 0.5) -> goal (6.5, 6.5, 2.5); v_max 3, a_max 3 (chosen)."""
    rng = np.random.default_rng(seed)
    r = np.full(n_obs, 0.68)
    start, goal = np.array([0.5, 0.5, 0.5]), np.array([6.5, 6.5, 2.5])
    c = _place(rng, n_obs, [0.0, 0.0, 0.0], [7.0, 7.0, 3.0], r, [start, goal], 3)
    return problem(3, n_p, horizon, start, goal, c, None, np.stack([r, r], 1), 3.0, 3.0, seed)


# The paper's solver settings for its benchmarks: N = 13 CEM iterations,
# N_b = 110 samples, N_proj = 80, N_elite = 20 (projection iterations not
# given: 50 chosen).
PAPER_CEM = {"n_samples": 110, "cem_iters": 13, "n_proj": 80, "n_elite": 20, "proj_iters": 50}


def batched_problems(n_problems=256, seed0=100):
    """Uneven 2-D problems: n_obs log-uniform in [10, 400], N in
    {256, 512, 1024, 2048}, n_p in {60, 100, 150}, horizon = 0.08 s * n_p,
    scene as the 30 x 30 m clutter (90 % static, 10 % moving)."""
    out = []
    for k in range(n_problems):
        seed = seed0 + k
        rng = np.random.default_rng(10_000 + seed)
        n_obs = int(round(math.exp(rng.uniform(math.log(10), math.log(400)))))
        n_samples = int(rng.choice([256, 512, 1024, 2048]))
        n_p = int(rng.choice([60, 100, 150]))
        n_dyn = n_obs // 10
        p = scene_clutter_2d(seed=seed, n_static=n_obs - n_dyn, n_dyn=n_dyn, n_p=n_p,
                             horizon=0.08 * n_p)
        out.append((p, n_samples))
    return out


def _place_fast(rng, n, lo, hi, radii, keep_clear, dims):
    """As _place, vectorised: rejected centres are redrawn together."""
    lo = np.broadcast_to(np.asarray(lo, dtype=float), (dims,))
    hi = np.broadcast_to(np.asarray(hi, dtype=float), (dims,))
    out = lo + (hi - lo) * rng.random((n, dims))
    keep = np.asarray(keep_clear, dtype=float).reshape(-1, dims)
    for _ in range(1000):
        d = np.linalg.norm(out[:, None, :] - keep[None, :, :], axis=2).min(axis=1)
        bad = d <= radii + 0.5
        if not bad.any():
            break
        out[bad] = lo + (hi - lo) * rng.random((int(bad.sum()), dims))
    return out


def serving_requests(rate=500.0, duration=60.0, seed=7, frac_3d=0.2, frac_warm=0.3, shift_s=0.5,
                     sizes=None):
    """A Poisson stream of planning requests (arrival time, problem, CEM
    overrides, robot id), sizes as in batched_problems: n_obs log-uniform in
    [10, 400], N in {256, 512, 1024, 2048}, n_p in {60, 100, 150},
    horizon 0.08 s * n_p.  A fraction frac_3d are 3-D (ellipsoids in
    20 x 20 x 8 m, v_max 2, a_max 3); a fraction frac_warm are replans of an
    earlier robot: same goal, obstacles and sizes, the start moved shift_s
    seconds along the straight start-goal line at the previous request's mean
    speed and moving obstacles advanced by shift_s.  sizes: optional list of
    (n_obs, N, n_p) choices that replaces the ranges (small test streams)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    robots = []  # (robot id, last problem)
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        k = len(out)
        if robots and rng.random() < frac_warm:
            j = int(rng.integers(max(0, len(robots) - 64), len(robots)))
            rid, prev, n_samples = robots[j]
            p = dict(prev)
            b0 = np.array(prev["b0"], dtype=float)
            bf = np.array(prev["bf"], dtype=float)
            step = (bf[:, 0] - b0[:, 0]) * (shift_s / prev["horizon"])
            b0[:, 0] = b0[:, 0] + step
            p["b0"] = b0
            p["center"] = np.asarray(prev["center"]) + shift_s * np.asarray(prev["vel"])
            p["seed"] = int(rng.integers(0, 2**62))
            robots[j] = (rid, p, n_samples)
            out.append((t, p, n_samples, rid))
            continue
        if sizes is not None:
            n_obs, n_samples, n_p = sizes[int(rng.integers(0, len(sizes)))]
        else:
            n_obs = int(round(math.exp(rng.uniform(math.log(10), math.log(400)))))
            n_samples = int(rng.choice([256, 512, 1024, 2048]))
            n_p = int(rng.choice([60, 100, 150]))
        horizon = 0.08 * n_p
        pseed = int(rng.integers(0, 2**62))
        if rng.random() < frac_3d:
            a = rng.uniform(0.3, 0.8, n_obs)
            b = rng.uniform(0.3, 0.8, n_obs)
            start, goal = np.array([1.0, 1.0, 1.0]), np.array([19.0, 19.0, 7.0])
            c = _place_fast(rng, n_obs, [0.0, 0.0, 0.0], [20.0, 20.0, 8.0], np.maximum(a, b), [start, goal], 3)
            p = problem(3, n_p, horizon, start, goal, c, None, np.stack([a, b], 1), 2.0, 3.0, pseed)
        else:
            r = rng.uniform(0.2, 0.5, n_obs)
            start, goal = np.array([1.0, 1.0]), np.array([29.0, 29.0])
            c = _place_fast(rng, n_obs, 2.0, 28.0, r, [start, goal], 2)
            v = np.zeros((n_obs, 2))
            n_dyn = n_obs // 10
            if n_dyn:
                v[n_obs - n_dyn:] = rng.uniform(-1.0, 1.0, (n_dyn, 2))
            p = problem(2, n_p, horizon, start, goal, c, v, np.stack([r, r], 1), VMAX_2D, AMAX_2D, pseed)
        rid = k
        robots.append((rid, p, n_samples))
        out.append((t, p, n_samples, rid))
    return out


def normals(seed, shape):
    """Standard normal draws for the sampling step (passed to both sides)."""
    return np.random.default_rng(seed).standard_normal(shape)


def workload(name: str):
    """The named benchmark / parity configurations.  Returns (problem, cem)."""
    if name == "small_fp64":
        p = scene_small_2d()
        return p, cem_settings(200, 50, 4, n_elite=20, dims=2)
    if name == "clutter2d_fp32":
        p = scene_clutter_2d()
        return p, cem_settings(1000, 100, 5, n_elite=100, dims=2)
    if name == "ellipsoid3d_mixed":
        p = scene_ellipsoids_3d()
        return p, cem_settings(2000, 100, 4, n_elite=200, dims=3)
    if name == "clutter2d_bounds":
        # the 2-D clutter workload with the workspace rows G = [-P; P] on
        # (tau = [-s_min; s_max], the 30 x 30 m box) and the paper's four
        # boundary rows per axis (end position only: final mask 1)
        p = dict(scene_clutter_2d())
        p.update(use_bounds=True, smin=np.zeros(2), smax=np.full(2, 30.0), bc_final_mask=1)
        return p, cem_settings(1000, 100, 5, n_elite=100, dims=2)
    c = PAPER_CEM
    if name == "p2p2d":
        return scene_p2p_2d(), cem_settings(c["n_samples"], c["proj_iters"], c["cem_iters"], c["n_proj"],
                                            c["n_elite"], dims=2)
    if name == "p2p3d":
        return scene_p2p_3d(), cem_settings(c["n_samples"], c["proj_iters"], c["cem_iters"], c["n_proj"],
                                            c["n_elite"], dims=3)
    if name == "dynamic2d":
        return scene_dynamic_2d(), cem_settings(c["n_samples"], c["proj_iters"], c["cem_iters"], c["n_proj"],
                                                c["n_elite"], dims=2)
    raise KeyError(name)
