"""GPU parity of the batched solve (priest_plan_batch: one persistent
projection launch over uneven problems per CEM iteration, replayed as a CUDA
graph) against the FP64 oracle and against single-problem solves."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, rel_err, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def uneven_problems(dims=2, n=5):
    rng = np.random.default_rng(42)
    out = []
    for i in range(n):
        p = scene(dims=dims, n_obs=int(rng.integers(3, 30)), n_dyn=int(rng.integers(0, 3)),
                  n_p=int(rng.choice([20, 37, 50])), seed=100 + i)
        N = int(rng.choice([17, 40, 64, 150]))
        cem = W.cem_settings(N, 12, 2, dims=dims)
        out.append((p, cem))
    return out


def run_batch(P, probs, precision, repeats=2):
    import torch

    dev = torch.device("cuda", 0)
    p0, c0 = probs[0]
    K, L = c0["proj_iters"], c0["cem_iters"]
    stream = torch.cuda.current_stream(dev)
    with P.Context(p0, c0, precision=precision, stream=stream.cuda_stream) as ctx:
        handles, zs, outs, keep = [], [], [], []
        for i, (p, cem) in enumerate(probs):
            prob, kp = P.make_problem(p, cem, per_problem_shape=True)
            keep.append(kp)
            handles.append(P.priest_load(ctx.h, prob))
            z = torch.from_numpy(W.normals(500 + i, (L, cem["n_samples"], p["dims"] * 11))).to(dev)
            zs.append(z)
            outs.append(torch.zeros(p["dims"] * 11 + 4, dtype=torch.float64, device=dev))
        results = []
        for _ in range(repeats):
            for o in outs:
                o.zero_()
            P.priest_plan_batch(ctx.h, handles, [z.data_ptr() for z in zs], [o.data_ptr() for o in outs])
            P.priest_sync(ctx.h)
            results.append([o.cpu().numpy() for o in outs])
        for h in handles:
            P.priest_unload(ctx.h, h)
        return results, [z.cpu().numpy() for z in zs]


@pytest.mark.parametrize("dims", [2, 3])
def test_fp64_batch_matches_oracle(P, oracle, dims):
    probs = uneven_problems(dims=dims)
    results, zs = run_batch(P, probs, P.PRIEST_FP64_CHECK)
    for run in results:  # direct launch, then the recorded graph
        for (p, cem), z, out in zip(probs, zs, run):
            want = oracle.plan(p, cem, z=z)
            D = p["dims"] * 11
            assert int(out[D + 3]) == want["elites"][0]
            assert rel_err(out[:D], want["best"], scale_of(p)) < TOL_FP64
            assert abs(out[D] - want["r"]) < TOL_FP64 * max(1.0, want["r"])


def test_fp32_batch_matches_single_solves(P, oracle):
    probs = uneven_problems(dims=2, n=6)
    results, zs = run_batch(P, probs, P.PRIEST_FP32)
    for (p, cem), z, out in zip(probs, zs, results[1]):
        with P.Context(p, cem, precision=P.PRIEST_FP32) as ctx:
            got = ctx.plan(p, z=z, cem=cem)
        D = p["dims"] * 11
        # same draws, same kernels: the two paths agree to the FP32 tolerance
        r_o, c1_o = oracle.residual_cost(p, out[:D][None])
        assert abs(out[D] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
        if int(out[D + 3]) == got["best_index"]:
            assert rel_err(out[:D], got["best"], scale_of(p)) < 10 * TOL_FP32
