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


# Elite sets of Alg. 1 under FP32: the selections must match the oracle's
# whenever the oracle's sorted keys around each cut differ by more than this
# (relative to max(|key|, 1)); closer keys may swap order under FP32 rounding.
GAP_FP32 = 1e-3


def alg1_iterations(oracle, p, cem, z, mu0=None, cov0=None):
    """Alg. 1 assembled from the oracle's stage functions (sample, project,
    residual / cost, ConstraintEliteSet, EliteSet, refit), one dict per CEM
    iteration with that iteration's input distribution (mu, cov), r, c_1 and
    both selections; returns (iterations, final mu, final cov)."""
    D = int(p["dims"]) * (int(p.get("degree", 10)) + 1)
    mu = oracle.default_mean(p) if mu0 is None else np.asarray(mu0, dtype=float)
    cov = np.eye(D) * cem["init_std"] ** 2 if cov0 is None else np.asarray(cov0, dtype=float)
    its = []
    for l in range(cem["cem_iters"]):
        S = cov + cem["chol_eps"] * np.trace(cov) / D * np.eye(D)
        xi = mu + z[l] @ oracle.cholesky(S).T
        xb, _ = oracle.project(p, xi, cem["proj_iters"])
        r, c1 = oracle.residual_cost(p, xb)
        pi, ei = oracle.select(r, c1 + r, cem["n_proj"], cem["n_elite"])
        its.append({"mu": mu, "cov": cov, "xb": xb, "r": r, "c1": c1, "proj": pi, "elite": ei})
        mu, cov = oracle.refit(xb[ei], (c1 + r)[ei], mu, cov, cem["sigma_lr"], cem["gamma"])
    return its, mu, cov


def cut_gaps(r, c1, proj, n_elite):
    """Relative gaps of the sorted keys at the two cuts of Alg. 1: r at the
    N_proj-th least sample (ConstraintEliteSet = proj), c_aug = c_1 + r at the
    N_elite-th least member of that set (EliteSet); inf for a cut that keeps
    every candidate."""
    def gap(keys, m):
        k = np.sort(np.asarray(keys, dtype=float))
        if m >= len(k):
            return np.inf
        return (k[m] - k[m - 1]) / max(abs(k[m]), 1.0)

    c_aug = np.asarray(c1) + np.asarray(r)
    return gap(r, len(proj)), gap(c_aug[np.asarray(proj)], n_elite)


def elites_match_or_flip(it, got_elite, got_r, got_c1, n_elite, oracle):
    """The gap rule for one CEM iteration.  got_*: the GPU's EliteSet and its
    r, c_1 of every sample (same iteration, same input distribution and
    draws).  Returns True when the oracle's gaps at both cuts exceed GAP_FP32
    and the GPU's ConstraintEliteSet (the N_proj least of its own r) and
    EliteSet equal the oracle's; False (a reported flip) when a gap is
    smaller; raises AssertionError when the gaps are large and a set differs."""
    g_proj, g_elite = cut_gaps(it["r"], it["c1"], it["proj"], n_elite)
    gpu_proj, gpu_elite = oracle.select(got_r, got_c1 + got_r, len(it["proj"]), n_elite)
    # the device selection is the selection of its own keys
    np.testing.assert_array_equal(np.asarray(got_elite), gpu_elite)
    if g_proj <= GAP_FP32 or g_elite <= GAP_FP32:
        print(f"elite flip allowed: cut gaps {g_proj:.2e} (r) / {g_elite:.2e} (c_aug)")
        return False
    assert set(np.asarray(gpu_proj).tolist()) == set(np.asarray(it["proj"]).tolist()), "ConstraintEliteSet differs"
    np.testing.assert_array_equal(np.asarray(got_elite), np.asarray(it["elite"]))
    return True


def plan_under_gap_rule(oracle, p, cem, z, got, tol, mu0=None, cov0=None):
    """A full FP32 solve against Alg. 1 assembled from the oracle's stages:
    when every cut of every iteration has a gap above GAP_FP32, the returned
    sample must be the oracle's (same index, coefficients within tol) and
    True is returned; otherwise the flip is reported and False returned."""
    its, _, _ = alg1_iterations(oracle, p, cem, z, mu0, cov0)
    g = min(min(cut_gaps(it["r"], it["c1"], it["proj"], cem["n_elite"])) for it in its)
    if g <= GAP_FP32:
        print(f"elite flip allowed: smallest cut gap {g:.2e}")
        return False
    best = its[-1]["elite"][0]
    assert got["best_index"] == best
    assert rel_err(got["best"], its[-1]["xb"][best], scale_of(p)) < tol
    return True
