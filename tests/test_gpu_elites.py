"""Elite-set parity of the FP32 solvers (Alg. 1, ConstraintEliteSet /
EliteSet) against the FP64 oracle under the gap rule: whenever the oracle's
sorted keys around a cut (r at N_proj, c_aug at N_elite) differ by more than
1e-3 relative, the GPU's sets must equal the oracle's; closer keys may swap
under FP32 rounding and are reported.  Each CEM iteration is run on the GPU
from the oracle's own input distribution (mu_l, Sigma_l) and draws, so every
iteration is compared on identical inputs; the scenes and seeds are chosen
so that every cut of every iteration has a large gap, which makes the
comparison unconditional there."""
import numpy as np
import pytest

from gpu_common import (TOL_FP32, alg1_iterations, cut_gaps, elites_match_or_flip, rel_err, scale_of, scene,
                        GAP_FP32)
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


# (scene, CEM settings, draw seed) whose oracle cuts all have gaps > 1e-3
CASES = {
    "2d": (lambda: scene(dims=2, n_obs=16, n_dyn=2, n_p=50), lambda: W.cem_settings(128, 25, 3, dims=2), 10),
    "3d": (lambda: scene(dims=3, n_obs=20, n_dyn=2, n_p=40), lambda: W.cem_settings(96, 20, 3, dims=3), 23),
}


def one_iteration(P, ctx, path, p, it, z_l, cem):
    """One CEM iteration on the GPU from the oracle's input distribution;
    returns (result, EliteSet, r, c_1)."""
    z1 = np.ascontiguousarray(z_l[None])
    got = ctx.plan_plain(p, z=z1, mu0=it["mu"], cov0=it["cov"]) if path == "plain" else \
        ctx.plan(p, z=z1, mu0=it["mu"], cov0=it["cov"])
    el, r, c1 = P.priest_read_elites(ctx.h, None, cem["n_elite"], cem["n_samples"])
    return got, el, r, c1


@pytest.mark.parametrize("case,path", [("2d", "fp32"), ("2d", "plain"), ("3d", "mixed"), ("3d", "fp32")])
def test_elites_match_oracle_every_iteration(P, oracle, case, path):
    mk_p, mk_c, zseed = CASES[case]
    p, cem = mk_p(), mk_c()
    D = p["dims"] * 11
    z = W.normals(zseed, (cem["cem_iters"], cem["n_samples"], D))
    its, _, _ = alg1_iterations(oracle, p, cem, z)
    for it in its:  # the precondition that makes every comparison below active
        assert min(cut_gaps(it["r"], it["c1"], it["proj"], cem["n_elite"])) > GAP_FP32
    prec = P.PRIEST_MIXED_BF16 if path == "mixed" else P.PRIEST_FP32
    # autotune off: the mixed path runs the tensor-core kernel
    with P.Context(p, dict(cem, cem_iters=1), precision=prec, autotune=0 if path == "mixed" else 1) as ctx:
        for l, it in enumerate(its):
            got, el, r, c1 = one_iteration(P, ctx, path, p, it, z[l], cem)
            # r and c_1 of every projected sample against the oracle's
            assert rel_err(r, it["r"], 1.0) < TOL_FP32
            assert rel_err(c1, it["c1"], 1.0) < TOL_FP32
            assert elites_match_or_flip(it, el, r, c1, cem["n_elite"], oracle)
            assert got["best_index"] == it["elite"][0]
            assert rel_err(got["best"], it["xb"][it["elite"][0]], scale_of(p)) < TOL_FP32


@pytest.mark.parametrize("case,path", [("2d", "fp32"), ("2d", "plain"), ("3d", "mixed")])
def test_full_plan_matches_oracle_when_gaps_are_large(P, oracle, case, path):
    """All L iterations on the GPU in one solve: with every cut's gap large,
    the FP32 differences carried from one iteration to the next stay far
    below the gaps, so the answer is the oracle's sample."""
    mk_p, mk_c, zseed = CASES[case]
    p, cem = mk_p(), mk_c()
    D = p["dims"] * 11
    z = W.normals(zseed, (cem["cem_iters"], cem["n_samples"], D))
    want = oracle.plan(p, cem, z=z)
    prec = P.PRIEST_MIXED_BF16 if path == "mixed" else P.PRIEST_FP32
    with P.Context(p, cem, precision=prec, autotune=0 if path == "mixed" else 1) as ctx:
        got = ctx.plan_plain(p, z=z) if path == "plain" else ctx.plan(p, z=z)
        el, _, _ = P.priest_read_elites(ctx.h, None, cem["n_elite"], cem["n_samples"])
    np.testing.assert_array_equal(el, want["elites"])
    assert got["best_index"] == want["elites"][0]
    assert rel_err(got["best"], want["best"], scale_of(p)) < 10 * TOL_FP32
    assert rel_err(got["mu"], want["mu"], scale_of(p)) < 10 * TOL_FP32
    assert abs(got["c_aug"] - want["c_aug"]) < 10 * TOL_FP32 * max(1.0, want["c_aug"])
