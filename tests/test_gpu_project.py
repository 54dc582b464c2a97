"""GPU parity of the fused projection (priest_project, through the C ABI)
against the FP64 oracle.  Sizes span several CTAs, several obstacle chunks
and a ragged last CTA; both precisions, 2-D / 3-D, moving obstacles,
workspace bounds and every supported end-condition mask."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, rel_err, samples, scale_of, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def run_both(P, oracle, p, xi, K, precision, lam=None):
    with P.Context(p, {"proj_iters": K}, precision=precision) as ctx:
        xb, lam_g, r, c1 = ctx.project(p, xi, lam=np.zeros_like(xi) if lam is None else lam)
    xb_o, lam_o = oracle.project(p, xi, K, lam=lam)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    return (xb, lam_g, r, c1), (xb_o, lam_o, r_o, c1_o)


@pytest.mark.parametrize("dims,bounds,mask,n_dyn", [
    (2, False, 7, 3), (3, False, 7, 2), (2, True, 1, 0), (3, True, 3, 1), (2, False, 0, 2)])
def test_fp64_check_mode_matches_oracle(P, oracle, dims, bounds, mask, n_dyn):
    p = scene(dims=dims, bounds=bounds, mask=mask, n_dyn=n_dyn, n_obs=17, n_p=40)
    xi = samples(oracle, p, 301, seed=dims)
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, 20, P.PRIEST_FP64_CHECK)
    s = scale_of(p)
    assert rel_err(xb, xb_o, s) < TOL_FP64
    assert rel_err(lam, lam_o, 1.0) < TOL_FP64
    assert rel_err(r, r_o, 1.0) < TOL_FP64
    assert rel_err(c1, c1_o, 1.0) < TOL_FP64
    assert np.count_nonzero(r_o) > 10  # the scene is active


@pytest.mark.parametrize("dims", [2, 3])
def test_fp64_converged_projection_matches_oracle(P, oracle, dims):
    """Thousands of iterations on the scenes of the oracle's converged-
    projection pin (fixed points on the constraint boundary: obstacle contact,
    a moving circle, an active acceleration bound): the FP64 check mode
    reaches the oracle's fixed points, and its own output satisfies the
    fixed-point identity xi_bar_F = xi_F + lambda_F."""
    from paper_2309_08235_gb300 import workloads as W

    if dims == 2:
        centre = np.array([[4.0, 0.4], [8.0, -0.5], [12.0, 0.3], [6.0, 3.0]])
        vel = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [0.3, -0.6]])
        a = np.array([0.9, 0.8, 0.9, 0.6])
        p = W.problem(2, 50, 8.0, np.zeros(2), np.array([16.0, 0.0]), centre, vel, np.stack([a, a], 1), 3.0, 2.0,
                      seed=1)
        xi = oracle.default_mean(p)[None] + np.random.default_rng(5).normal(0.0, 0.4, (6, 22))
        K = 8000
    else:
        centre = np.array([[4.0, 0.3, 0.8], [8.0, -0.4, 1.2], [10.0, 0.2, 1.8]])
        semi = np.array([[0.9, 0.6], [0.8, 1.0], [0.7, 0.5]])
        p = W.problem(3, 50, 8.0, np.zeros(3), np.array([14.0, 0.0, 2.0]), centre, None, semi, 3.0, 1.6, seed=1)
        xi = oracle.default_mean(p)[None] + np.random.default_rng(7).normal(0.0, 0.4, (4, 33))
        K = 2000
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, K, P.PRIEST_FP64_CHECK)
    s = scale_of(p)
    assert rel_err(xb, xb_o, s) < TOL_FP64
    assert rel_err(lam, lam_o, 1.0) < TOL_FP64
    assert np.abs(r).max() < 1e-9 and np.abs(r_o).max() < 1e-9  # feasible fixed points
    nv = 11
    free = np.concatenate([ax * nv + np.r_[3:nv - 3] for ax in range(dims)])
    assert np.abs(xb[:, free] - xi[:, free] - lam[:, free]).max() < 1e-10 * s


def test_k0_is_equality_projection(P, oracle):
    p = scene(dims=3, mask=7)
    xi = samples(oracle, p, 50, seed=1)
    for prec, tol in ((P.PRIEST_FP64_CHECK, 1e-12), (P.PRIEST_FP32, 1e-6)):
        with P.Context(p, {"proj_iters": 0}, precision=prec) as ctx:
            xb, _, r, c1 = ctx.project(p, xi)
        pa = oracle.project_eq(p, xi)
        assert rel_err(xb, pa, scale_of(p)) < tol
        r_o, c1_o = oracle.residual_cost(p, pa)
        assert rel_err(r, r_o, 1.0) < max(tol, 1e-6)


def test_fp32_one_step_map(P, oracle):
    """Same xi_bar^k in: one iteration agrees to the FP32 tolerance."""
    p = scene(dims=2, n_obs=30, n_p=60)
    xi = samples(oracle, p, 200, seed=3)
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, 1, P.PRIEST_FP32)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(lam, lam_o, 1.0) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32


@pytest.mark.parametrize("dims", [2, 3])
def test_fp32_k_steps(P, oracle, dims):
    p = scene(dims=dims, n_obs=20, n_p=50, n_dyn=2)
    xi = samples(oracle, p, 257, seed=4)
    K = 40
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, K, P.PRIEST_FP32)
    s = scale_of(p)
    err = np.abs(xb - xb_o).max(1) / max(np.abs(xb_o).max(), s)
    # The residual map is continuous at the active-set switch, so no flip
    # margin is needed here: every sample is held to the FP32 tolerance.
    assert err.max() < TOL_FP32, (err.max(), np.argmax(err))
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32


def test_many_samples_per_cta_against_sampled_oracle(P, oracle):
    """4096 samples (many per CTA): every 97th is checked against the oracle."""
    p = scene(dims=2, n_obs=12, n_p=30, n_dyn=2)
    xi = samples(oracle, p, 4096, seed=6)
    with P.Context(p, {"proj_iters": 15}, precision=P.PRIEST_FP32) as ctx:
        xb, lam, r, c1 = ctx.project(p, xi, lam=np.zeros_like(xi))
    idx = np.arange(0, 4096, 97)
    xb_o, lam_o = oracle.project(p, xi[idx], 15)
    r_o, _ = oracle.residual_cost(p, xb_o)
    assert rel_err(xb[idx], xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(r[idx], r_o, 1.0) < TOL_FP32


def test_warm_start_multipliers(P, oracle):
    p = scene(dims=2, n_obs=10, n_p=30)
    xi = samples(oracle, p, 40, seed=7)
    lam0 = np.random.default_rng(1).normal(0, 0.3, xi.shape)
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, 10, P.PRIEST_FP64_CHECK, lam=lam0)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP64
    assert rel_err(lam, lam_o, 1.0) < TOL_FP64


def test_degenerate_sample_at_obstacle_centre(P, oracle):
    """A trajectory point exactly on an obstacle centre (alpha = atan2(0, 0))."""
    from paper_2309_08235_gb300 import workloads as W

    p0 = W.problem(2, 11, 5.0, [0, 0], [10, 0], [[5.0, 0.0]], None, [[1.0, 1.0]], vmax=50, amax=50)
    xi = oracle.project_eq(p0, oracle.default_mean(p0)[None])  # straight line through (5, 0) at t = 2.5
    P0 = oracle.basis(10, 11, 5.0)[0]
    assert np.isclose((P0 @ xi[0, :11])[5], 5.0) and abs((P0 @ xi[0, 11:])[5]) < 1e-15
    for prec, tol in ((P.PRIEST_FP64_CHECK, TOL_FP64), (P.PRIEST_FP32, TOL_FP32)):
        (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p0, xi, 3, prec)
        assert rel_err(xb, xb_o, 10.0) < tol
        assert rel_err(r, r_o, 1.0) < tol


def test_zero_obstacles_and_empty_batch(P, oracle):
    from paper_2309_08235_gb300 import workloads as W

    p = W.problem(3, 25, 4.0, [0, 0, 0], [3, 1, 2], np.zeros((0, 3)), None, np.zeros((0, 2)), vmax=1e6,
                  amax=1e6)
    xi = samples(oracle, p, 9, seed=2)
    with P.Context(p, {"proj_iters": 12}, precision=P.PRIEST_FP64_CHECK) as ctx:
        xb, lam, r, c1 = ctx.project(p, xi)
        assert rel_err(xb, oracle.project_eq(p, xi), scale_of(p)) < 1e-12
        assert np.all(r == 0.0)
        out = ctx.project(p, np.zeros((0, 33)))
        assert out[0].shape == (0, 33)


def test_invalid_inputs_are_rejected(P, oracle):
    p = scene(dims=2, n_obs=4)
    xi = samples(oracle, p, 3)
    with P.Context(p, {"proj_iters": 2}) as ctx:
        for bad in ({"semi": -np.abs(p["semi"])}, {"dims": 4}, {"bc_final_mask": 5},
                    {"center": np.full_like(p["center"], np.nan)}):
            q = dict(p, **{k: v for k, v in bad.items() if k != "dims"})
            prob, keep = P.make_problem(q)
            if "dims" in bad:
                prob.dims = bad["dims"]
            out = np.zeros_like(xi)
            with pytest.raises(P.PriestError) as e:
                P.priest_project(ctx.h, prob, 3, xi, None, out, None, None)
            assert e.value.status == P.PRIEST_ERR_INVALID
        xi_nan = xi.copy()
        xi_nan[1, 4] = np.nan
        with pytest.raises(P.PriestError):
            ctx.project(p, xi_nan)


def test_fp32_bounded_four_row_workload(P, oracle):
    """The measured bounded workload's shape (workspace rows on, the paper's
    four boundary rows per axis: end position only), 2-D clutter scene, FP32
    against the oracle on 150 samples over 20 iterations."""
    from paper_2309_08235_gb300 import workloads as W

    p, _ = W.workload("clutter2d_bounds")
    xi = samples(oracle, p, 150, seed=41, std=2.0)
    (xb, lam, r, c1), (xb_o, lam_o, r_o, c1_o) = run_both(P, oracle, p, xi, 20, P.PRIEST_FP32)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
