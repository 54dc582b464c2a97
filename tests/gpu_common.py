"""Shared helpers of the GPU parity tests: scenes, tolerances, error norms."""
import numpy as np

from paper_2309_08235_gb300 import workloads as W

# Tolerances (relative, see rel_err): FP64 check mode and the FP32 fast path.
TOL_FP64 = 1e-9
TOL_FP32 = 1e-4


def rel_err(x, ref, scale=1.0):
    """||x - ref||_inf / max(||ref||_inf, scale)."""
    x = np.asarray(x, dtype=float)
    ref = np.asarray(ref, dtype=float)
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), scale)) if ref.size else 0.0


def scale_of(p):
    return float(np.linalg.norm(np.asarray(p["bf"])[:, 0] - np.asarray(p["b0"])[:, 0]))


def scene(dims=2, n_obs=24, n_dyn=3, n_p=50, horizon=6.0, seed=5, bounds=False, mask=7, radius=(0.4, 1.2),
          vmax=None, amax=None):
    """Obstacles scattered along the start-goal diagonal so samples hit them."""
    rng = np.random.default_rng(seed)
    start = np.zeros(dims)
    goal = np.array([12.0, 9.0, 4.0][:dims])
    t = rng.uniform(0.1, 0.9, n_obs)
    c = start + t[:, None] * (goal - start) + rng.normal(0, 1.0, (n_obs, dims))
    a = rng.uniform(*radius, n_obs)
    b = rng.uniform(*radius, n_obs)
    v = np.zeros((n_obs, dims))
    if n_dyn:
        v[-n_dyn:] = rng.uniform(-0.8, 0.8, (n_dyn, dims))
    p = W.problem(dims, n_p, horizon, start, goal, c, v, np.stack([a, b], 1),
                  vmax=vmax or (4.0 if dims == 2 else 3.5), amax=amax or (4.0 if dims == 2 else 3.0),
                  seed=seed, use_bounds=bounds, smin=np.full(dims, -0.5), smax=goal + 0.5,
                  bc_final_mask=mask)
    return p


def samples(oracle, p, n, seed=0, std=1.5):
    rng = np.random.default_rng(seed)
    mu = oracle.default_mean(p)
    return mu + std * rng.normal(size=(n, len(mu)))
