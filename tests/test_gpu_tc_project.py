"""GPU parity of PRIEST_MIXED_BF16: the fused projection whose (point,
obstacle) tests run as one BF16 tensor-core product per CTA (split
high / low operands, FP32 accumulation in tensor memory) selecting the pairs
for the exact FP32 test.  Against the FP64 oracle to the FP32 tolerance, and
against the FP32 kernel on the same inputs; sizes span several CTAs,
tensor-memory waves, column segments, static and moving obstacles, more
than 256 obstacle columns, and no obstacles at all."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, plan_under_gap_rule, rel_err, samples, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def project(P, p, xi, K, precision, lam=None):
    # autotune off: PRIEST_MIXED_BF16 runs the tensor-core kernel (no timed routing)
    mixed = precision == P.PRIEST_MIXED_BF16
    with P.Context(p, {"proj_iters": K}, precision=precision, autotune=0 if mixed else 1) as ctx:
        out = ctx.project(p, xi, lam=lam)
        if mixed and xi.shape[0] > 0:
            assert P.priest_last_kernel(ctx.h) == 2
        return out


@pytest.mark.parametrize("dims,n_obs,n_dyn,n_p,N,bounds", [
    (2, 19, 3, 40, 133, False), (3, 19, 2, 41, 133, False), (2, 30, 0, 60, 300, True),
    (3, 24, 0, 37, 257, True), (2, 300, 20, 50, 180, False), (2, 12, 2, 30, 2100, False)])
def test_mixed_projection_matches_oracle(P, oracle, dims, n_obs, n_dyn, n_p, N, bounds):
    p = scene(dims=dims, n_obs=n_obs, n_dyn=n_dyn, n_p=n_p, bounds=bounds, radius=(0.4, 1.2))
    xi = samples(oracle, p, N, seed=dims + n_obs)
    lam0 = np.random.default_rng(7).normal(0, 0.2, xi.shape)
    K = 20
    xb, lam, r, c1 = project(P, p, xi, K, P.PRIEST_MIXED_BF16, lam=lam0)
    idx = np.arange(0, N, max(1, N // 97))  # the oracle on a sample of rows for the large cases
    xb_o, lam_o = oracle.project(p, xi[idx], K, lam=lam0[idx])
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    s = scale_of(p)
    assert rel_err(xb[idx], xb_o, s) < TOL_FP32
    assert rel_err(lam[idx], lam_o, 1.0) < TOL_FP32
    assert rel_err(r[idx], r_o, 1.0) < TOL_FP32
    assert rel_err(c1[idx], c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    assert np.count_nonzero(r_o) > 5  # the scene is active
    # and the FP32 kernel on the same inputs
    xb32, lam32, r32, _ = project(P, p, xi, K, P.PRIEST_FP32, lam=lam0)
    assert rel_err(xb, xb32, s) < TOL_FP32
    assert rel_err(r, r32, 1.0) < TOL_FP32


def test_mixed_without_obstacles(P, oracle):
    p = W.problem(2, 25, 4.0, [0, 0], [3, 1], np.zeros((0, 2)), None, np.zeros((0, 2)), vmax=2.0, amax=2.0)
    xi = samples(oracle, p, 40, seed=2)
    xb, lam, r, c1 = project(P, p, xi, 12, P.PRIEST_MIXED_BF16)
    xb_o, _ = oracle.project(p, xi, 12)
    r_o, _ = oracle.residual_cost(p, xb_o)
    assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32


def test_mixed_plan_close_to_oracle(P, oracle):
    p = scene(dims=3, n_obs=20, n_dyn=2, n_p=40)
    cem = W.cem_settings(96, 20, 3, dims=3)
    z = W.normals(23, (3, 96, 33))  # every elite cut of this draw has a gap > 1e-3
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_MIXED_BF16, autotune=0) as ctx:
        got = ctx.plan(p, z=z)
        assert P.priest_last_kernel(ctx.h) == 2
    r_o, c1_o = oracle.residual_cost(p, got["best"][None])
    assert abs(got["r"] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
    assert abs(got["c_aug"] - (r_o[0] + c1_o[0])) < TOL_FP32 * max(1.0, c1_o[0])
    assert plan_under_gap_rule(oracle, p, cem, z, got, 10 * TOL_FP32)
    assert rel_err(got["best"], want["best"], scale_of(p)) < 10 * TOL_FP32


def test_mixed_routes_to_the_faster_kernel(P, oracle):
    """With the autotuner on, PRIEST_MIXED_BF16 times the tensor-core kernel
    and the FP32 kernel once per shape and runs the faster one; either way the
    result is the FP32 result up to summation order."""
    p = scene(dims=2, n_obs=40, n_dyn=4, n_p=50)
    xi = samples(oracle, p, 300, seed=4)
    with P.Context(p, {"proj_iters": 15}, precision=P.PRIEST_MIXED_BF16) as ctx:
        xb, _, r, _ = ctx.project(p, xi)
        kind = P.priest_last_kernel(ctx.h)
        xb2, _, _, _ = ctx.project(p, xi)  # the decision is kept for the shape
        assert P.priest_last_kernel(ctx.h) == kind
    assert kind in (1, 2)
    xb32, _, r32, _ = project(P, p, xi, 15, P.PRIEST_FP32)
    assert rel_err(xb, xb32, scale_of(p)) < TOL_FP32
    assert rel_err(r, r32, 1.0) < TOL_FP32
    np.testing.assert_array_equal(xb, xb2)
