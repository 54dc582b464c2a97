"""GPU parity of the FP32 point-owner projection kernel (threads own time
stamps of one sample for all iterations; segmented reductions, state lanes)
against the FP64 oracle, through the C ABI.  The autotuner is off, so the
default tiling runs: the point-owner kernel with two time stamps per thread
for every shape here (degree 10, at rest at both ends or, in 2-D, the end
position only; enough time stamps).
Cases: warm-start multipliers over many iterations (the fixed-column
multipliers come from the summed residual rows), workspace bounds, moving
obstacles, 2-D and 3-D, a ragged last CTA and samples of several CTAs
whose warps straddle two samples."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, rel_err, samples, scale_of, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def project(P, p, xi, K, lam0):
    with P.Context(p, {"proj_iters": K}, precision=P.PRIEST_FP32, autotune=0) as ctx:
        return ctx.project(p, xi, lam=lam0)


@pytest.mark.parametrize("dims,bounds,n_dyn,mask", [(2, False, 4, 7), (3, False, 3, 7), (2, True, 2, 7), (2, True, 2, 1)])
def test_k_steps_with_warm_multipliers(P, oracle, dims, bounds, n_dyn, mask):
    p = scene(dims=dims, n_obs=40, n_p=100, n_dyn=n_dyn, bounds=bounds, mask=mask)
    xi = samples(oracle, p, 300, seed=11 + dims)
    lam0 = np.random.default_rng(3).normal(0.0, 0.2, xi.shape)
    K = 30
    xb, lam, r, c1 = project(P, p, xi, K, lam0)
    xb_o, lam_o = oracle.project(p, xi, K, lam=lam0)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    # every column, the fixed ones included
    assert rel_err(lam, lam_o, 1.0) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    assert np.count_nonzero(r_o > 1e-6) > 10  # obstacles are active


def test_ragged_last_cta_sampled(P, oracle):
    """1003 samples (seven per CTA, the last CTA holds two): every 59th
    sample and the last one against the oracle."""
    p = scene(dims=2, n_obs=30, n_p=100, n_dyn=3)
    xi = samples(oracle, p, 1003, seed=21)
    K = 20
    xb, lam, r, c1 = project(P, p, xi, K, None)
    idx = np.r_[np.arange(0, 1003, 59), 1001, 1002]
    xb_o, _ = oracle.project(p, xi[idx], K)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    assert rel_err(xb[idx], xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(r[idx], r_o, 1.0) < TOL_FP32
    assert rel_err(c1[idx], c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32


def test_same_result_alone_and_in_a_larger_launch(P, oracle):
    """A sample's result does not depend on which CTA or warp position holds
    it: the first 7 samples alone (one per CTA) and inside 700 (five per CTA,
    warps shared by two samples) agree to well within the FP32 tolerance."""
    p = scene(dims=2, n_obs=25, n_p=100, n_dyn=2)
    xi = samples(oracle, p, 700, seed=31)
    a = project(P, p, xi[:7], 25, None)
    b = project(P, p, xi, 25, None)
    assert rel_err(a[0], b[0][:7], scale_of(p)) < TOL_FP32 / 10
    assert rel_err(a[2], b[2][:7], 1.0) < TOL_FP32 / 10


@pytest.mark.parametrize("case", ["no_obstacles", "moving_only", "one_sample", "long_horizon"])
def test_edge_shapes(P, oracle, case):
    """Degenerate and extreme shapes through the point-owner kernel: no
    obstacles (the projection is the equality projection at every iteration),
    moving obstacles only (no static quads), a single sample (one CTA with
    one partial warp), and 400 time stamps (200 threads per sample)."""
    if case == "no_obstacles":
        p = scene(dims=2, n_obs=0, n_dyn=0, n_p=100, vmax=1e6, amax=1e6)
        n, K = 64, 15
    elif case == "moving_only":
        p = scene(dims=2, n_obs=8, n_dyn=8, n_p=100)
        n, K = 64, 15
    elif case == "one_sample":
        p = scene(dims=3, n_obs=20, n_dyn=2, n_p=100)
        n, K = 1, 15
    else:
        p = scene(dims=2, n_obs=30, n_dyn=3, n_p=400, horizon=12.0)
        n, K = 40, 15
    xi = samples(oracle, p, n, seed=51)
    # zero multipliers without obstacles (the equality-projection pin), warm ones otherwise
    lam0 = np.zeros_like(xi) if case == "no_obstacles" else np.random.default_rng(5).normal(0.0, 0.1, xi.shape)
    xb, lam, r, c1 = project(P, p, xi, K, lam0)
    xb_o, lam_o = oracle.project(p, xi, K, lam=lam0)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(lam, lam_o, 1.0) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    if case == "no_obstacles":
        assert rel_err(xb, oracle.project_eq(p, xi), scale_of(p)) < TOL_FP32


@pytest.mark.parametrize("dims", [2, 3])
def test_list_overflow_falls_back_to_full_screening(P, oracle, dims):
    """Neighbour lists hold at most 8 (2-D) / 6 (3-D) obstacles per point:
    twelve coincident obstacles on the start-goal line overflow the lists of
    every point near them, and those warps screen every obstacle exactly in
    every iteration until their next rebuild.  The results still equal the
    oracle's (and multipliers, residuals and costs with them)."""
    # 3-D needs n_p >= 64: a warp may touch two samples only (dims x 5 state lanes each)
    p = scene(dims=dims, n_obs=24, n_p=60 if dims == 2 else 100, n_dyn=2)
    c = np.asarray(p["center"], dtype=float).copy()
    semi = np.asarray(p["semi"], dtype=float).copy()
    mid = 0.5 * (np.asarray(p["b0"])[:, 0] + np.asarray(p["bf"])[:, 0])
    c[:12] = mid  # twelve obstacles with one centre, on the straight line
    semi[:12] = 0.8
    p = dict(p, center=c, semi=semi)
    xi = samples(oracle, p, 150, seed=31 + dims)
    lam0 = np.random.default_rng(4).normal(0.0, 0.1, xi.shape)
    K = 25
    with P.Context(p, {"proj_iters": K}, precision=P.PRIEST_FP32, autotune=0) as ctx:
        xb, lam, r, c1 = ctx.project(p, xi, lam=lam0)
        assert P.priest_last_kernel(ctx.h) == 1
    xb_o, lam_o = oracle.project(p, xi, K, lam=lam0)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(lam, lam_o, 1.0) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    assert np.count_nonzero(r_o > 1e-6) > 10


def test_dense_scene_keeps_lists(P, oracle):
    """1,500 circles in the 30 x 30 m box (the list margin shrinks with the
    density so that the lists stay short): sampled rows against the oracle,
    on the point-owner kernel."""
    from paper_2309_08235_gb300 import workloads as W

    p = W.scene_clutter_2d(seed=9, n_static=1350, n_dyn=150, n_p=60, horizon=4.8)
    xi = oracle.default_mean(p) + 2.0 * W.normals(12, (400, 22))
    K = 20
    with P.Context(p, {"proj_iters": K}, precision=P.PRIEST_FP32, autotune=0) as ctx:
        xb, _, r, c1 = ctx.project(p, xi)
        assert P.priest_last_kernel(ctx.h) == 1
    idx = np.r_[0:400:53, 399]
    xb_o, _ = oracle.project(p, xi[idx], K)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    assert rel_err(xb[idx], xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(r[idx], r_o, 1.0) < TOL_FP32
    assert rel_err(c1[idx], c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
