"""priest_project_noalloc, the projection entry point that allocates no device
memory (for callers that cannot call cudaMalloc, e.g. real-time loops with a
fixed memory budget), checked through the C ABI against the regular
priest_project and against the FP64 oracle on the same inputs, on two calls
in a row with different problems so that state left in the shared scratch by
the first call cannot leak into the second.  Collected last on purpose."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, rel_err, scale_of, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def inputs(p, n, seed):
    rng = np.random.default_rng(seed)
    D = p["dims"] * 11
    mu = np.concatenate([np.linspace(p["b0"][a][0], p["bf"][a][0], 11) for a in range(p["dims"])])
    return mu + 1.5 * rng.normal(size=(n, D)), 0.1 * rng.normal(size=(n, D))


@pytest.mark.parametrize("precision,tol", [(1, TOL_FP32), (0, TOL_FP64)])
def test_noalloc_matches_priest_project_twice(P, oracle, precision, tol):
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    problems = [scene(dims=2, n_obs=21, n_dyn=3, n_p=50, seed=1),
                scene(dims=3, n_obs=9, n_dyn=2, n_p=37, seed=2, mask=3)]
    for call, p in enumerate(problems):
        n = 203 if call == 0 else 77
        xi, lam0 = inputs(p, n, seed=10 + call)
        cem = {"proj_iters": 25}
        # reference: the existing entry point
        with P.Context(p, cem, precision=precision) as ctx:
            xb_ref, lam_ref, r_ref, c1_ref = ctx.project(p, xi, lam=lam0)
        # allocation-free entry point on caller-owned device buffers
        cfg = P.make_config(p, cem, precision)
        prob, keep = P.make_problem(p, per_problem_shape=True)
        t_xi = torch.from_numpy(xi).to(dev)
        t_lam = torch.from_numpy(lam0).to(dev)
        t_xb = torch.full_like(t_xi, float("nan"))
        t_r = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        t_c = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        st = P.priest_project_noalloc(cfg, prob, n, t_xi.data_ptr(), t_lam.data_ptr(), t_xb.data_ptr(),
                                      t_r.data_ptr(), t_c.data_ptr(), stream.cuda_stream)
        assert st == P.PRIEST_OK, st
        torch.cuda.synchronize()
        s = scale_of(p)
        assert rel_err(t_xb.cpu().numpy(), xb_ref, s) < tol
        assert rel_err(t_lam.cpu().numpy(), lam_ref, 1.0) < tol
        assert rel_err(t_r.cpu().numpy(), r_ref, 1.0) < tol
        assert rel_err(t_c.cpu().numpy(), c1_ref, max(1.0, np.abs(c1_ref).max())) < tol
        # and against the oracle (Sec. III-A, Appendix eqs. comp_alpha .. comp_zeta)
        xb_o, lam_o = oracle.project(p, xi, cem["proj_iters"], lam=lam0)
        r_o, c1_o = oracle.residual_cost(p, xb_o)
        assert rel_err(t_xb.cpu().numpy(), xb_o, s) < tol
        assert rel_err(t_lam.cpu().numpy(), lam_o, 1.0) < tol
        assert rel_err(t_r.cpu().numpy(), r_o, 1.0) < tol
        assert rel_err(t_c.cpu().numpy(), c1_o, max(1.0, np.abs(c1_o).max())) < tol


def test_noalloc_rejects_bad_sizes(P):
    p = scene(dims=2, n_obs=4, n_p=20)
    cfg = P.make_config(p, {"proj_iters": 3}, P.PRIEST_FP32)
    prob, keep = P.make_problem(p, per_problem_shape=True)
    prob.n_p = 100000
    assert P.priest_project_noalloc(cfg, prob, 4, 1, 0, 1, 1, 1) == P.PRIEST_ERR_INVALID
    prob.n_p = 20
    assert P.priest_project_noalloc(cfg, prob, -1, 0, 0, 0, 0, 0) == P.PRIEST_ERR_INVALID
    assert P.priest_project_noalloc(cfg, prob, 0, 0, 0, 0, 0, 0) == P.PRIEST_OK
