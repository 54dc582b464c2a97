"""GPU parity of the point-to-point benchmark workloads (Sec. V-B scene
shapes: 2-D with 50 circles r = 0.4, 3-D room 7 x 7 x 3 m with 25 spheres
r = 0.68; the paper's N_b = 110 samples and 13 CEM iterations) in FP64 check
mode against the oracle's Alg. 1: identical elite sets, the same returned
sample and final mean."""
import numpy as np
import pytest

from gpu_common import TOL_FP64, rel_err, scale_of
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


@pytest.mark.parametrize("name", ["p2p2d", "p2p3d"])
def test_p2p_fp64_plan_matches_oracle(P, oracle, name):
    p, cem = W.workload(name)
    assert cem["n_samples"] == 110 and cem["cem_iters"] == 13
    D = p["dims"] * 11
    z = W.normals(61, (cem["cem_iters"], cem["n_samples"], D))
    want = oracle.plan(p, cem, z=z)
    with P.Context(p, cem, precision=P.PRIEST_FP64_CHECK) as ctx:
        got = ctx.plan(p, z=z, cem=cem)
        el, _, _ = P.priest_read_elites(ctx.h, None, cem["n_elite"], cem["n_samples"])
    np.testing.assert_array_equal(el, want["elites"])
    assert got["best_index"] == want["elites"][0]
    s = scale_of(p)
    assert rel_err(got["best"], want["best"], s) < TOL_FP64
    assert rel_err(got["mu"], want["mu"], s) < TOL_FP64
    assert abs(got["c_aug"] - want["c_aug"]) < TOL_FP64 * max(1.0, want["c_aug"])
