"""GPU parity of the full solve (Alg. 1: sample, project, residual / cost,
ConstraintEliteSet, EliteSet, refit, Cholesky) through the C ABI against the
FP64 oracle, with the same standard-normal draws on both sides."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, plan_under_gap_rule, rel_err, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


@pytest.mark.parametrize("dims,N,n_proj,n_elite", [(2, 64, 45, 7), (3, 50, 50, 1), (2, 33, 20, 20), (2, 2500, 1300, 300)])
def test_fp64_plan_matches_oracle(P, oracle, dims, N, n_proj, n_elite):
    p = scene(dims=dims, n_obs=10, n_dyn=2, n_p=40)
    cem = W.cem_settings(N, 15, 3, n_proj=n_proj, n_elite=n_elite, dims=dims)
    z = W.normals(11, (cem["cem_iters"], N, dims * 11))
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        got = ctx.plan(p, z=z)
    s = scale_of(p)
    assert got["best_index"] == want["elites"][0]
    assert rel_err(got["best"], want["best"], s) < TOL_FP64
    assert rel_err(got["mu"], want["mu"], s) < TOL_FP64
    assert abs(got["r"] - want["r"]) < TOL_FP64 * max(1.0, want["r"])
    assert abs(got["c_aug"] - want["c_aug"]) < TOL_FP64 * max(1.0, want["c_aug"])


def test_plan_seeded_stream_matches_explicit_draws(P, oracle):
    p = scene(dims=2, n_obs=8, n_p=30)
    cem = W.cem_settings(40, 10, 2, dims=2)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        a = ctx.plan(p)  # draws from the host stream seeded by p["seed"]
        z = oracle.rng_normal(p["seed"], 2 * 40 * 22)
        b = ctx.plan(p, z=z)
    assert np.array_equal(a["best"], b["best"])
    want = oracle.plan(p, cem, seed=p["seed"])
    assert rel_err(a["best"], want["best"], scale_of(p)) < TOL_FP64


def test_fp64_plan_with_ties_at_zero_residual(P, oracle):
    """Far obstacles and loose bounds: every sample has r = 0 exactly, so
    ConstraintEliteSet is decided by the sample index on both sides."""
    p = W.problem(2, 30, 10.0, [0, 0], [5, 5], [[100, 100]], None, [[0.5, 0.5]], vmax=1e3, amax=1e3)
    cem = W.cem_settings(48, 5, 2, n_proj=17, n_elite=5, dims=2)
    cem["init_std"] = 0.3
    z = W.normals(3, (2, 48, 22))
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        got = ctx.plan(p, z=z)
    assert want["r"] == 0.0 and got["r"] == 0.0
    assert got["best_index"] == want["elites"][0]
    assert rel_err(got["mu"], want["mu"], 7.0) < TOL_FP64


def test_fp32_plan_close_to_oracle(P, oracle):
    p = scene(dims=2, n_obs=16, n_dyn=2, n_p=50)
    cem = W.cem_settings(128, 25, 3, dims=2)
    z = W.normals(10, (3, 128, 22))  # every elite cut of this draw has a gap > 1e-3
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP32) as ctx:
        got = ctx.plan(p, z=z)
    # the returned trajectory's residual / cost, re-evaluated by the oracle
    r_o, c1_o = oracle.residual_cost(p, got["best"][None])
    assert abs(got["r"] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
    assert abs(got["c_aug"] - (r_o[0] + c1_o[0])) < TOL_FP32 * max(1.0, c1_o[0])
    # the gap rule: large gaps at every cut, so the oracle's sample is returned
    assert plan_under_gap_rule(oracle, p, cem, z, got, 10 * TOL_FP32)
    assert rel_err(got["best"], want["best"], scale_of(p)) < 10 * TOL_FP32


def test_plan_rejects_bad_counts(P, oracle):
    p = scene(dims=2, n_obs=4)
    with P.Context(p, W.cem_settings(10, 2, 1)) as ctx:
        prob, keep = P.make_problem(p)
        prob.n_samples, prob.n_proj, prob.n_elite = 10, 12, 2
        res = P.priest_result()
        with pytest.raises(P.PriestError) as e:
            P.priest_plan(ctx.h, prob, None, None, res)
        assert e.value.status == P.PRIEST_ERR_INVALID


def test_non_pd_initial_covariance_reports_numeric(P, oracle):
    p = scene(dims=2, n_obs=4, n_p=20)
    cem = W.cem_settings(16, 2, 1, dims=2)
    cov0 = -np.eye(22)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        with pytest.raises(P.PriestError) as e:
            ctx.plan(p, cov0=cov0)
        assert e.value.status == P.PRIEST_ERR_NUMERIC
        # the context stays usable
        ok = ctx.plan(p)
        assert ok["status"] == 0
