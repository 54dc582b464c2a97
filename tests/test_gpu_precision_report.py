"""Error of the FP32 and the BF16-tensor-core (PRIEST_MIXED_BF16) paths
against the FP64 oracle on the 3-D ellipsoid workload's shapes (200
ellipsoids, n_p = 150, K = 100): coefficients, constraint residual r and
cost c_1 of a sample of projected trajectories.  Prints the figures (run
with -s) and holds them to the FP32 tolerance of the projection (1e-4 on
coefficients) and 1e-3 on the residual / cost."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, rel_err, scale_of
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


@pytest.mark.parametrize("name", ["ellipsoid3d_mixed", "clutter2d_fp32"])
def test_error_against_oracle(P, oracle, name):
    p, cem = W.workload(name)
    K = cem["proj_iters"]
    D = p["dims"] * 11
    n = 12
    xi = oracle.default_mean(p) + cem["init_std"] * W.normals(77, (n, D))
    xb_o, _ = oracle.project(p, xi, K)
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    s = scale_of(p)
    for prec, label in ((P.PRIEST_FP32, "fp32"), (P.PRIEST_MIXED_BF16, "mixed_bf16")):
        # autotune off: the mixed label measures the tensor-core kernel itself
        with P.Context(p, cem, precision=prec, autotune=0 if prec == P.PRIEST_MIXED_BF16 else 1) as ctx:
            xb, _, r, c1 = ctx.project(p, xi)
        e_xi = rel_err(xb, xb_o, s)
        e_r = float(np.abs(r - r_o).max())
        e_c = float(np.abs(c1 - c1_o).max() / max(1.0, np.abs(c1_o).max()))
        print(f"\n{name} {label}: coefficients {e_xi:.2e} (rel), residual {e_r:.2e} (abs, max r {r_o.max():.3f}), "
              f"cost {e_c:.2e} (rel)")
        assert e_xi < TOL_FP32
        assert e_r < 1e-3 and e_c < 1e-3
