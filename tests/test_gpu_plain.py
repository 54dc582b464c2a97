"""GPU parity of the plain per-problem FP32 path (priest_project_plain /
priest_plan_plain: one kernel per step, HBM intermediates) against the FP64
oracle, to the FP32 tolerance, and its agreement with the fused path on the
same draws."""
import numpy as np
import pytest

from gpu_common import plan_under_gap_rule, TOL_FP32, rel_err, samples, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


@pytest.mark.parametrize("dims,bounds,mask,n_dyn,n_p", [
    (2, False, 7, 3, 50), (3, False, 7, 2, 41), (2, True, 1, 0, 37), (3, True, 3, 1, 30)])
def test_plain_projection_matches_oracle(P, oracle, dims, bounds, mask, n_dyn, n_p):
    p = scene(dims=dims, bounds=bounds, mask=mask, n_dyn=n_dyn, n_obs=19, n_p=n_p)
    xi = samples(oracle, p, 133, seed=dims + 3)
    lam0 = np.random.default_rng(5).normal(0, 0.2, xi.shape)
    K = 25
    with P.Context(p, {"proj_iters": K}, precision=P.PRIEST_FP32) as ctx:
        xb, lam, r, c1 = ctx.project_plain(p, xi, lam=lam0)
    xb_o, lam_o = oracle.project(p, xi, K, lam=lam0)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    s = scale_of(p)
    assert rel_err(xb, xb_o, s) < TOL_FP32
    assert rel_err(lam, lam_o, 1.0) < TOL_FP32
    assert rel_err(r, r_o, 1.0) < TOL_FP32
    assert rel_err(c1, c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    assert np.count_nonzero(r_o) > 10


def test_plain_and_fused_agree(P, oracle):
    p = scene(dims=2, n_obs=30, n_p=60, n_dyn=3)
    xi = samples(oracle, p, 300, seed=8)
    with P.Context(p, {"proj_iters": 30}, precision=P.PRIEST_FP32) as ctx:
        a = ctx.project_plain(p, xi)
        b = ctx.project(p, xi)
    assert rel_err(a[0], b[0], scale_of(p)) < TOL_FP32
    assert rel_err(a[2], b[2], 1.0) < TOL_FP32


def test_plain_plan_close_to_oracle(P, oracle):
    p = scene(dims=2, n_obs=16, n_dyn=2, n_p=50)
    cem = W.cem_settings(128, 25, 3, dims=2)
    z = W.normals(10, (3, 128, 22))  # every elite cut of this draw has a gap > 1e-3
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP32) as ctx:
        got = ctx.plan_plain(p, z=z)
        fused = ctx.plan(p, z=z)
    r_o, c1_o = oracle.residual_cost(p, got["best"][None])
    assert abs(got["r"] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
    assert abs(got["c_aug"] - (r_o[0] + c1_o[0])) < TOL_FP32 * max(1.0, c1_o[0])
    # the gap rule holds at every cut, so both paths return the oracle's sample
    assert plan_under_gap_rule(oracle, p, cem, z, got, 10 * TOL_FP32)
    assert plan_under_gap_rule(oracle, p, cem, z, fused, 10 * TOL_FP32)
    assert rel_err(got["best"], want["best"], scale_of(p)) < 10 * TOL_FP32
    assert rel_err(got["best"], fused["best"], scale_of(p)) < 10 * TOL_FP32


def test_plain_rejects_fp64_context(P, oracle):
    p = scene(dims=2, n_obs=4)
    xi = samples(oracle, p, 3)
    with P.Context(p, {"proj_iters": 2}, precision=P.PRIEST_FP64_CHECK) as ctx:
        with pytest.raises(P.PriestError) as e:
            ctx.project_plain(p, xi)
        assert e.value.status == P.PRIEST_ERR_INVALID
