"""GPU parity of the BARN-style cost c_1 (acceleration, curvature and
path-following penalties) in every path that evaluates it: the fused
projection (FP64 check mode to 1e-9, FP32 and MIXED_BF16 to 1e-4), the plain
path, and a full solve on the dynamic scene against the oracle."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, rel_err, samples, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


@pytest.mark.parametrize("dims", [2, 3])
def test_projection_cost_matches_oracle(P, oracle, dims):
    p = W.with_barn_cost(scene(dims=dims, n_obs=14, n_dyn=2, n_p=45), w_curv=0.3, w_path=0.7)
    xi = samples(oracle, p, 150, seed=dims)
    K = 15
    xb_o, _ = oracle.project(p, xi, K)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    cs = max(1.0, np.abs(c1_o).max())
    for prec, tol in ((P.PRIEST_FP64_CHECK, TOL_FP64), (P.PRIEST_FP32, TOL_FP32), (P.PRIEST_MIXED_BF16, TOL_FP32)):
        with P.Context(p, {"proj_iters": K}, precision=prec) as ctx:
            xb, _, r, c1 = ctx.project(p, xi)
            if prec == P.PRIEST_FP32:
                _, _, _, c1p = ctx.project_plain(p, xi)
                assert rel_err(c1p, c1_o, cs) < TOL_FP32
        assert rel_err(xb, xb_o, scale_of(p)) < tol
        assert rel_err(c1, c1_o, cs) < tol


def test_dynamic_scene_plan_matches_oracle(P, oracle):
    p, cem = W.workload("dynamic2d")
    cem = dict(cem, cem_iters=3, proj_iters=20)
    z = W.normals(91, (3, cem["n_samples"], 22))
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        got = ctx.plan(p, z=z)
    assert got["best_index"] == want["elites"][0]
    assert rel_err(got["best"], want["best"], scale_of(p)) < TOL_FP64
    assert abs(got["c_aug"] - want["c_aug"]) < TOL_FP64 * max(1.0, want["c_aug"])


def test_bad_cost_rejected(P, oracle):
    p = W.with_barn_cost(scene(dims=2, n_obs=4), curv_eps=0.0)
    xi = samples(oracle, p, 3)
    with P.Context(p, {"proj_iters": 2}) as ctx:
        with pytest.raises(P.PriestError) as e:
            ctx.project(p, xi)
        assert e.value.status == P.PRIEST_ERR_INVALID
