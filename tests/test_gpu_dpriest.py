"""GPU parity of D-PRIEST (priest_plan_multi: M distributions on one stacked
projection launch, segmented selections and refits, best of M) against the
FP64 oracle's orc_plan_multi, with the same standard-normal draws."""
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


@pytest.mark.parametrize("dims,M,nj", [(2, 3, 40), (3, 2, 33), (2, 5, 16)])
def test_fp64_dpriest_matches_oracle(P, oracle, dims, M, nj):
    p = scene(dims=dims, n_obs=12, n_dyn=2, n_p=36)
    D = dims * 11
    cem = W.cem_settings(M * nj, 12, 3, n_proj=M * (nj * 3 // 4), n_elite=M * 4, dims=dims)
    z = W.normals(41 + M, (3, M * nj, D))
    want = oracle.plan_multi(p, cem, M, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        got = ctx.plan_multi(p, M, z=z)
    s = scale_of(p)
    assert got["dist"] == want["dist"]
    assert rel_err(got["best"]["best"], want["best"], s) < TOL_FP64
    for j in range(M):
        assert rel_err(got["per_dist"][j]["best"], want["dist_best"][j], s) < TOL_FP64
        assert rel_err(got["per_dist"][j]["mu"], want["mu"][j], s) < TOL_FP64
        assert abs(got["per_dist"][j]["c_aug"] - want["dist_c_aug"][j]) < TOL_FP64 * max(1.0, want["dist_c_aug"][j])


def test_one_distribution_equals_plan(P, oracle):
    p = scene(dims=2, n_obs=10, n_p=30)
    cem = W.cem_settings(64, 10, 2, dims=2)
    z = W.normals(5, (2, 64, 22))
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        a = ctx.plan_multi(p, 1, z=z)
        b = ctx.plan(p, z=z)
    assert a["dist"] == 0
    np.testing.assert_array_equal(a["best"]["best"], b["best"])


def test_fp32_dpriest_close_to_oracle(P, oracle):
    p = scene(dims=2, n_obs=16, n_dyn=2, n_p=40)
    M, nj = 4, 64
    cem = W.cem_settings(M * nj, 20, 3, dims=2)
    z = W.normals(49, (3, M * nj, 22))
    want = oracle.plan_multi(p, cem, M, z=z)
    # each distribution is Alg. 1 on its own rows (pinned on the oracle side)
    sub = dict(cem, n_samples=nj, n_proj=cem["n_proj"] // M, n_elite=max(1, cem["n_elite"] // M))
    means = oracle.multi_default_means(p, M, 2.0 * cem["init_std"])
    for prec in (P.PRIEST_FP32, P.PRIEST_MIXED_BF16):
        # autotune off: the mixed pass runs the tensor-core kernel
        with P.Context(p, cem, precision=prec, autotune=0 if prec == P.PRIEST_MIXED_BF16 else 1) as ctx:
            got = ctx.plan_multi(p, M, z=z)
        best = got["best"]
        checked = 0
        for j, res in enumerate(got["per_dist"]):
            # every distribution's answer re-evaluated by the oracle
            r_o, c1_o = oracle.residual_cost(p, res["best"][None])
            assert abs(res["r"] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
            assert abs(res["c_aug"] - (r_o[0] + c1_o[0])) < TOL_FP32 * max(1.0, c1_o[0])
            # the gap rule per distribution: the oracle's sample where every cut has a large gap
            if plan_under_gap_rule(oracle, p, sub, z[:, j * nj:(j + 1) * nj], res, 10 * TOL_FP32, mu0=means[j]):
                assert rel_err(res["best"], want["dist_best"][j], scale_of(p)) < 10 * TOL_FP32
                checked += 1
        assert checked >= 3  # distributions 0, 1 and 3 of this draw have large gaps at every cut
        assert best["c_aug"] == min(r["c_aug"] for r in got["per_dist"])
        assert best["c_aug"] <= want["c_aug"] * (1 + 1e-3) + 1e-3


def test_dpriest_rejects_uneven_split(P, oracle):
    p = scene(dims=2, n_obs=4, n_p=20)
    cem = W.cem_settings(30, 4, 1, dims=2)
    with P.Context(p, cem) as ctx:
        with pytest.raises(P.PriestError) as e:
            ctx.plan_multi(p, 4)
        assert e.value.status == P.PRIEST_ERR_INVALID
