"""GPU parity of the batched solve (priest_plan_batch: one persistent
projection launch over uneven problems per CEM iteration, replayed as a CUDA
graph) against the FP64 oracle and against single-problem solves."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, plan_under_gap_rule, rel_err, samples, scale_of, scene
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


def run_batch(P, probs, precision, repeats=2, **over):
    import torch

    dev = torch.device("cuda", 0)
    p0, c0 = probs[0]
    K, L = c0["proj_iters"], c0["cem_iters"]
    stream = torch.cuda.current_stream(dev)
    with P.Context(p0, c0, precision=precision, stream=stream.cuda_stream, **over) as ctx:
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


def test_fp32_batch_under_gap_rule(P, oracle):
    """FP32 batched solves against Alg. 1 assembled from the oracle's stages:
    every returned trajectory's r and c_aug re-evaluated by the oracle, and
    for the problems whose elite cuts all have large gaps, the oracle's
    sample itself."""
    probs = uneven_problems(dims=2, n=6)
    results, zs = run_batch(P, probs, P.PRIEST_FP32)
    checked = 0
    for (p, cem), z, out in zip(probs, zs, results[1]):
        D = p["dims"] * 11
        r_o, c1_o = oracle.residual_cost(p, out[:D][None])
        assert abs(out[D] - r_o[0]) < TOL_FP32 * max(1.0, r_o[0])
        assert abs(out[D + 2] - (r_o[0] + c1_o[0])) < TOL_FP32 * max(1.0, c1_o[0])
        got = {"best_index": int(out[D + 3]), "best": out[:D]}
        checked += plan_under_gap_rule(oracle, p, cem, z, got, 10 * TOL_FP32)
    assert checked >= 5  # all problems but the last have large gaps at every cut of these draws


# Problems of the 256-problem batched workload spanning its sizes: obstacles
# up to 400, samples up to 2048, every time-stamp count (60, 100, 150).
BATCH_PICK = [25, 54, 41, 8, 4, 56, 28]


def test_fp32_project_batch_matches_oracle_at_batched_sizes(P, oracle):
    """priest_project_batch (the persistent point-owner launch of the batched
    solves) against the oracle element by element: xi_bar, lambda, r and c_1
    of sampled rows of every problem (first, middle, last -- the last one in
    a ragged final item -- and a random one), K = 60."""
    import torch

    dev = torch.device("cuda", 0)
    every = W.batched_problems(64)
    probs = [every[i] for i in BATCH_PICK]
    K = 60
    p0, n0 = probs[0]
    with P.Context(p0, W.cem_settings(n0, K, 1), precision=P.PRIEST_FP32) as ctx:
        handles, keep, rows, ins, lams, outs = [], [], [], [], [], []
        for i, (p, N) in enumerate(probs):
            prob, kp = P.make_problem(p, W.cem_settings(N, K, 1), per_problem_shape=True)
            keep.append(kp)
            handles.append(P.priest_load(ctx.h, prob))
            xi = oracle.default_mean(p) + 2.0 * W.normals(700 + i, (N, 22))
            lam = 0.3 * W.normals(800 + i, (N, 22)) if i % 3 == 0 else None
            rows.append(N)
            ins.append((xi, lam))
            lams.append(None if lam is None else torch.from_numpy(lam).to(dev))
            outs.append((torch.from_numpy(xi).to(dev), torch.full((N, 22), float("nan"), dtype=torch.float64, device=dev),
                         torch.full((N,), float("nan"), dtype=torch.float64, device=dev),
                         torch.full((N,), float("nan"), dtype=torch.float64, device=dev)))
        P.priest_project_batch(ctx.h, handles, rows, [o[0].data_ptr() for o in outs],
                               [0 if l is None else l.data_ptr() for l in lams], [o[1].data_ptr() for o in outs],
                               [o[2].data_ptr() for o in outs], [o[3].data_ptr() for o in outs])
        P.priest_sync(ctx.h)
        assert P.priest_last_kernel(ctx.h) == 1  # the point-owner kernel ran the launch
        for h in handles:
            P.priest_unload(ctx.h, h)
    rng = np.random.default_rng(5)
    for i, ((p, N), (xi, lam), o, l) in enumerate(zip(probs, ins, outs, lams)):
        sel = sorted({0, N // 2 + 1, N - 1, int(rng.integers(N))})
        xb_o, lam_o = oracle.project(p, xi[sel], K, lam=None if lam is None else lam[sel])
        r_o, c1_o = oracle.residual_cost(p, xb_o)
        xb = o[1].cpu().numpy()[sel]
        assert rel_err(xb, xb_o, scale_of(p)) < TOL_FP32, (i, p["n_p"], p["n_obs"], N)
        assert rel_err(o[2].cpu().numpy()[sel], r_o, 1.0) < TOL_FP32
        assert rel_err(o[3].cpu().numpy()[sel], c1_o, 1.0) < TOL_FP32
        if l is not None:
            assert rel_err(l.cpu().numpy()[sel], lam_o, 1.0) < TOL_FP32
        # every row written
        assert np.isfinite(o[1].cpu().numpy()).all() and np.isfinite(o[2].cpu().numpy()).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plan_batch_host_matches_device_batch_and_oracle(P, oracle, precision):
    """priest_plan_batch_host (host problems, host draws, host results):
    the same answers as priest_plan_batch on device buffers; in FP64 the
    oracle's.  A second call with moved obstacles and a new goal (same
    layout) runs the resident plan on the new data; a third call with a
    different obstacle count replaces it."""
    prec = P.PRIEST_FP64_CHECK if precision == "fp64" else P.PRIEST_FP32
    probs = uneven_problems(dims=2, n=5)
    # cost-model tilings on both sides (no timing), so the FP32 kernels match bit for bit
    dev_results, zs = run_batch(P, probs, prec, repeats=1, autotune=0)
    p0, c0 = probs[0]

    def host_call(ctx, plist):
        structs, keep = [], []
        for p, cem in plist:
            s, k = P.make_problem(p, cem, per_problem_shape=True)
            structs.append(s)
            keep.append(k)
        res = (P.priest_result * len(plist))()
        P.priest_plan_batch_host(ctx.h, structs, zs[:len(plist)], res)
        return [P.result_dict(res[i]) for i in range(len(plist))]

    def moved(p, dx):
        q = dict(p)
        q["center"] = np.asarray(p["center"]) + dx
        q["bf"] = [list(r) for r in p["bf"]]
        q["bf"][0][0] += 0.5
        return q

    with P.Context(p0, c0, precision=prec, autotune=0) as ctx:
        first = host_call(ctx, probs)
        again = host_call(ctx, probs)  # replay of the resident plan
        shifted = [(moved(p, 0.3), cem) for p, cem in probs]
        second = host_call(ctx, shifted)
        fewer = [(dict(p, center=p["center"][:-1], vel=p["vel"][:-1], semi=p["semi"][:-1], n_obs=p["n_obs"] - 1), cem)
                 for p, cem in probs[:3]]
        third = host_call(ctx, fewer)
    for (p, cem), got, again_i, dv in zip(probs, first, again, dev_results[0]):
        D = p["dims"] * 11
        assert got["status"] == 0
        assert got["best_index"] == int(dv[D + 3])
        np.testing.assert_array_equal(got["best"], dv[:D])
        np.testing.assert_array_equal(got["best"], again_i["best"])
    if precision == "fp64":
        for plist, res in ((probs, first), (shifted, second), (fewer, third)):
            for (p, cem), got, z in zip(plist, res, zs):
                want = oracle.plan(p, cem, z=z)
                assert got["best_index"] == want["elites"][0]
                assert rel_err(got["best"], want["best"], scale_of(p)) < TOL_FP64
                assert rel_err(got["mu"], want["mu"], scale_of(p)) < TOL_FP64
                assert abs(got["c_aug"] - want["c_aug"]) < TOL_FP64 * max(1.0, want["c_aug"])


def test_plan_batch_host_after_tuned_device_batch(P, oracle):
    """The benchmark's order in one context: a device-buffer batch tunes the
    tilings and records its graph, then the host-buffer path loads its own
    resident copies of the same problems (every class already tuned, so no
    set-up runs before its recording) and must reproduce the device answers
    bit for bit, on its first call and on replays."""
    import torch

    dev = torch.device("cuda", 0)
    probs = uneven_problems(dims=2, n=5)
    p0, c0 = probs[0]
    K, L = c0["proj_iters"], c0["cem_iters"]
    stream = torch.cuda.current_stream(dev)
    with P.Context(p0, c0, precision=P.PRIEST_FP32, stream=stream.cuda_stream) as ctx:
        handles, structs, keep, zs, outs = [], [], [], [], []
        for i, (p, cem) in enumerate(probs):
            prob, kp = P.make_problem(p, cem, per_problem_shape=True)
            keep.append(kp)
            structs.append(prob)
            handles.append(P.priest_load(ctx.h, prob))
            zs.append(W.normals(900 + i, (L, cem["n_samples"], 22)))
            outs.append(torch.zeros(26, dtype=torch.float64, device=dev))
        zd = [torch.from_numpy(z).to(dev) for z in zs]
        for _ in range(2):
            P.priest_plan_batch(ctx.h, handles, [z.data_ptr() for z in zd], [o.data_ptr() for o in outs])
        P.priest_sync(ctx.h)
        want = [o.cpu().numpy() for o in outs]
        for call in range(3):
            res = (P.priest_result * len(probs))()
            P.priest_plan_batch_host(ctx.h, structs, zs, res)
            for i, w in enumerate(want):
                got = P.result_dict(res[i])
                assert got["best_index"] == int(w[25]), (call, i)
                np.testing.assert_array_equal(got["best"], w[:22])
                assert got["c_aug"] == w[24]
        for h in handles:
            P.priest_unload(ctx.h, h)


@pytest.mark.parametrize("mode", ["pinned", "mixed"])
def test_plan_batch_host_pinned_draws(P, oracle, mode):
    """Draws in page-locked host memory are read in place by the transfer
    kernel (16-byte aligned buffers, buffers at an 8-byte offset, and, in
    "mixed", pageable ones copied by DMA beside them): the answers equal
    those of pageable draws bit for bit, on the first call and on a replay."""
    import torch

    probs = uneven_problems(dims=2, n=5)
    p0, c0 = probs[0]
    L = c0["cem_iters"]
    zs = [W.normals(700 + i, (L, cem["n_samples"], 22)) for i, (p, cem) in enumerate(probs)]
    keep_t = []

    def pinned(z, shift):
        t = torch.empty(z.size + shift, dtype=torch.float64).pin_memory()
        t[shift:] = torch.from_numpy(z.ravel())
        keep_t.append(t)
        return t.data_ptr() + 8 * shift

    if mode == "pinned":
        zp = [pinned(z, 0) for z in zs]
    else:
        zp = [pinned(z, 1) if i % 2 == 0 else z for i, z in enumerate(zs)]
    structs, keep = [], []
    for p, cem in probs:
        s, k = P.make_problem(p, cem, per_problem_shape=True)
        structs.append(s)
        keep.append(k)

    def call(ctx, z_list):
        res = (P.priest_result * len(probs))()
        P.priest_plan_batch_host(ctx.h, structs, z_list, res)
        return [P.result_dict(res[i]) for i in range(len(probs))]

    with P.Context(p0, c0, precision=P.PRIEST_FP32, autotune=0) as ctx:
        want = call(ctx, zs)
        got = [call(ctx, zp), call(ctx, zp)]
    for g in got:
        for w, x in zip(want, g):
            assert x["status"] == 0 and x["best_index"] == w["best_index"]
            np.testing.assert_array_equal(x["best"], w["best"])
            np.testing.assert_array_equal(x["mu"], w["mu"])
            assert x["c_aug"] == w["c_aug"]


def project_batch_numpy(P, oracle, probs, K, env, **over):
    """priest_project_batch on the given problems with env set; returns
    (xi_bar, lambda or None, r, c_1) per problem as host arrays and the kernel
    kind of the launch."""
    import os

    import torch

    dev = torch.device("cuda", 0)
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        p0, n0 = probs[0]
        with P.Context(p0, W.cem_settings(n0, K, 1), precision=P.PRIEST_FP32, **over) as ctx:
            handles, keep, rows, lams, outs = [], [], [], [], []
            for i, (p, N) in enumerate(probs):
                prob, kp = P.make_problem(p, W.cem_settings(N, K, 1), per_problem_shape=True)
                keep.append(kp)
                handles.append(P.priest_load(ctx.h, prob))
                xi = oracle.default_mean(p) + 2.0 * W.normals(700 + i, (N, 22))
                lam = 0.3 * W.normals(800 + i, (N, 22)) if i % 3 == 0 else None
                rows.append(N)
                lams.append(None if lam is None else torch.from_numpy(lam).to(dev))
                outs.append((torch.from_numpy(xi).to(dev), torch.zeros((N, 22), dtype=torch.float64, device=dev),
                             torch.zeros((N,), dtype=torch.float64, device=dev),
                             torch.zeros((N,), dtype=torch.float64, device=dev)))
            P.priest_project_batch(ctx.h, handles, rows, [o[0].data_ptr() for o in outs],
                                   [0 if l is None else l.data_ptr() for l in lams], [o[1].data_ptr() for o in outs],
                                   [o[2].data_ptr() for o in outs], [o[3].data_ptr() for o in outs])
            P.priest_sync(ctx.h)
            kind = P.priest_last_kernel(ctx.h)
            for h in handles:
                P.priest_unload(ctx.h, h)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [(o[1].cpu().numpy(), None if l is None else l.cpu().numpy(), o[2].cpu().numpy(), o[3].cpu().numpy())
            for o, l in zip(outs, lams)], kind


def test_project_batch_lists_equal_full_screening(P, oracle):
    """The persistent point-owner launch (its own compilation of the kernel
    source, at 128 registers) gives bitwise the same outputs with its
    neighbour lists and grid, with the lists rebuilt from every static
    obstacle (PRIEST_LIST_GRID=0), and with every obstacle screened in every
    iteration (PRIEST_NEIGHBOUR_LISTS=0), on problems of the batched workload
    (cost-model tilings, so the three launches share their layout)."""
    every = W.batched_problems(64)
    probs = [every[i] for i in BATCH_PICK[:4]]
    a, ka = project_batch_numpy(P, oracle, probs, 60, {}, autotune=0)
    b, kb = project_batch_numpy(P, oracle, probs, 60, {"PRIEST_LIST_GRID": "0"}, autotune=0)
    c, kc = project_batch_numpy(P, oracle, probs, 60, {"PRIEST_NEIGHBOUR_LISTS": "0"}, autotune=0)
    assert ka == kb == kc == 1
    for x, y, z in zip(a, b, c):
        for u, v, w in zip(x, y, z):  # xi_bar, lambda, r, c_1
            if u is None:
                continue
            np.testing.assert_array_equal(u, v)
            np.testing.assert_array_equal(u, w)


def test_project_batch_edge_cases(P, oracle):
    """priest_project_batch with a problem of zero rows among others, no
    multiplier lists at all, a single-row problem, and rows beyond a loaded
    problem's sample count rejected."""
    import torch

    dev = torch.device("cuda", 0)
    probs = uneven_problems(dims=2, n=3)
    K = 12
    p0, c0 = probs[0]
    with P.Context(p0, dict(c0, proj_iters=K), precision=P.PRIEST_FP32) as ctx:
        handles, keep, bufs, xis = [], [], [], []
        rows = [0, 1, probs[2][1]["n_samples"]]
        for i, ((p, cem), n) in enumerate(zip(probs, rows)):
            prob, kp = P.make_problem(p, cem, per_problem_shape=True)
            keep.append(kp)
            handles.append(P.priest_load(ctx.h, prob))
            xi = samples(oracle, p, max(n, 1), seed=60 + i)
            xis.append(xi)
            bufs.append([torch.from_numpy(xi).to(dev), torch.zeros_like(torch.from_numpy(xi)).to(dev),
                         torch.zeros(max(n, 1), dtype=torch.float64, device=dev),
                         torch.zeros(max(n, 1), dtype=torch.float64, device=dev)])
        P.priest_project_batch(ctx.h, handles, rows, [b[0].data_ptr() for b in bufs], None,
                               [b[1].data_ptr() for b in bufs], [b[2].data_ptr() for b in bufs],
                               [b[3].data_ptr() for b in bufs])
        P.priest_sync(ctx.h)
        for (p, cem), n, xi, b in zip(probs, rows, xis, bufs):
            if n == 0:
                assert not b[1].abs().sum().item()  # nothing written
                continue
            xb_o, _ = oracle.project(p, xi[:n], K)
            assert rel_err(b[1].cpu().numpy()[:n], xb_o, scale_of(p)) < TOL_FP32
        with pytest.raises(P.PriestError) as e:
            P.priest_project_batch(ctx.h, handles[:1], [probs[0][1]["n_samples"] + 1], [bufs[0][0].data_ptr()],
                                   None, [bufs[0][1].data_ptr()], [bufs[0][2].data_ptr()], [bufs[0][3].data_ptr()])
        assert e.value.status == P.PRIEST_ERR_INVALID
        for h in handles:
            P.priest_unload(ctx.h, h)
