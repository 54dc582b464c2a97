"""GPU tests of the serving loop (priest_submit / priest_poll / priest_wait):
continuous batching of uneven 2-D / 3-D requests at CEM-iteration
granularity, admission by HBM budget, device-resident warm starts, and the
device copy of the standard-normal stream.  Parity is against the FP64 oracle
(Alg. 1, with the multiplier warm start for replans) and against the same
request solved alone."""
import numpy as np
import pytest

from gpu_common import TOL_FP32, TOL_FP64, rel_err, scale_of, scene
from paper_2309_08235_gb300 import workloads as W

pytestmark = pytest.mark.gpu

L_ITERS, K_ITERS = 3, 12


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def _cem(n_samples, dims=2):
    cem = W.cem_settings(n_samples, K_ITERS, L_ITERS, dims=dims)
    cem["init_std"] = W.INIT_STD_2D  # one context serves both dims with its own Sigma_0
    return cem


def _requests():
    """Uneven requests: 2-D and 3-D, different n_p, N, n_obs, horizons."""
    reqs = []
    shapes = [(2, 12, 40, 64), (3, 9, 30, 48), (2, 30, 60, 128), (2, 5, 24, 33), (3, 20, 50, 96),
              (2, 18, 36, 80), (2, 0, 20, 40), (3, 4, 28, 17)]
    for k, (dims, n_obs, n_p, N) in enumerate(shapes):
        p = scene(dims=dims, n_obs=max(n_obs, 1), n_dyn=2 if n_obs > 4 else 0, n_p=n_p, horizon=4.0 + 0.5 * k,
                  seed=40 + k)
        if n_obs == 0:
            p = W.problem(dims, n_p, p["horizon"], np.zeros(dims), np.array([12.0, 9.0, 4.0][:dims]),
                          np.zeros((0, dims)), None, np.zeros((0, 2)), p["vmax"], p["amax"], seed=40 + k)
        p["seed"] = 1000 + k
        reqs.append((p, _cem(N, dims)))
    return reqs


def _ctx(P, precision, **over):
    p0 = scene(dims=2, n_obs=4)
    return P.Context(p0, _cem(32), precision=precision, **over)


def _oracle_z(oracle, p, cem):
    D = p["dims"] * 11
    return oracle.rng_normal(p["seed"], cem["cem_iters"] * cem["n_samples"] * D).reshape(
        cem["cem_iters"], cem["n_samples"], D)


def test_device_normal_stream_matches_host(P, oracle):
    import torch

    for seed, n in [(0, 1), (7, 100_001), (2**63 + 5, 4096)]:
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        P.priest_rng_normal_device(seed, n, out.data_ptr())
        torch.cuda.synchronize()
        host = oracle.rng_normal(seed, n)
        got = out.cpu().numpy()
        assert np.abs(got - host).max() < 1e-13, (seed, n)


def test_served_fp64_matches_oracle(P, oracle):
    reqs = _requests()
    with _ctx(P, P.PRIEST_FP64_CHECK) as ctx:
        tickets = [ctx.submit(p, cem) for p, cem in reqs]
        got = [ctx.wait(t) for t in tickets]
        stats = ctx.serve_stats()
    assert stats["completed"] == len(reqs) and stats["max_active"] > 1
    for (p, cem), g in zip(reqs, got):
        want = oracle.plan(p, cem, z=_oracle_z(oracle, p, cem))
        s = scale_of(p)
        assert g["status"] == 0
        assert g["best_index"] == want["elites"][0]
        assert rel_err(g["best"], want["best"], s) < TOL_FP64
        assert rel_err(g["mu"], want["mu"], s) < TOL_FP64
        assert abs(g["c_aug"] - want["c_aug"]) < TOL_FP64 * max(1.0, want["c_aug"])


def _serve(P, reqs, precision, robot_ids=None, alone=False, **over):
    with _ctx(P, precision, **over) as ctx:
        out = [None] * len(reqs)
        if alone:
            for i, (p, cem) in enumerate(reqs):
                rid = -1 if robot_ids is None else robot_ids[i]
                out[i] = ctx.wait(ctx.submit(p, cem, robot_id=rid))
        else:
            ts = [ctx.submit(p, cem, robot_id=-1 if robot_ids is None else robot_ids[i])
                  for i, (p, cem) in enumerate(reqs)]
            out = [ctx.wait(t) for t in ts]
        return out, ctx.serve_stats()


def _replans(reqs, robots):
    """Replans of the given requests: start moved along the start-goal line."""
    out = []
    for i in robots:
        p, cem = reqs[i]
        q = dict(p)
        b0 = np.array(p["b0"], dtype=float)
        b0[:, 0] += 0.1 * (np.asarray(p["bf"])[:, 0] - b0[:, 0])
        q["b0"] = b0
        q["seed"] = p["seed"] + 500
        out.append((q, cem))
    return out


def test_mix_equals_alone_fp32(P):
    """Each request's result is the same solved alone and in the mix (shared
    launches with other requests, admitted while others run), including warm
    replans of two robots."""
    base = _requests()
    reqs = base + _replans(base, [0, 4])
    robot_ids = [100 + i for i in range(len(base))] + [100, 104]
    alone, st_a = _serve(P, reqs, P.PRIEST_FP32, robot_ids, alone=True)
    mix, st_m = _serve(P, reqs, P.PRIEST_FP32, robot_ids)
    assert st_a["max_active"] == 1 and st_m["max_active"] > 1
    assert st_a["warm_starts"] == 2 and st_m["warm_starts"] == 2
    for (p, _), a, m in zip(reqs, alone, mix):
        assert a["status"] == 0 and m["status"] == 0
        assert a["best_index"] == m["best_index"]
        assert rel_err(m["best"], a["best"], scale_of(p)) <= TOL_FP32
        assert abs(m["c_aug"] - a["c_aug"]) <= TOL_FP32 * max(1.0, a["c_aug"])


def test_budget_admission_defers_and_matches(P):
    """A budget that holds about two requests at once: the rest wait for
    memory, every result is produced, peak memory stays within the budget,
    and results equal an unconstrained run."""
    reqs = _requests()
    free, _ = _serve(P, reqs, P.PRIEST_FP32)
    budget = 450 << 10
    tight, st = _serve(P, reqs, P.PRIEST_FP32, hbm_budget=budget)
    assert st["deferred"] > 0 and st["peak_bytes"] <= budget and st["completed"] == len(reqs)
    for (p, _), a, b in zip(reqs, free, tight):
        assert rel_err(b["best"], a["best"], scale_of(p)) <= TOL_FP32


def test_slot_limit(P):
    reqs = _requests()
    out, st = _serve(P, reqs, P.PRIEST_FP32, serve_slots=2)
    assert st["max_active"] <= 2 and all(o["status"] == 0 for o in out)


def test_warm_replan_matches_oracle_fp64(P, oracle):
    """A replan of a robot starts from the previous plan's final mean,
    covariance and multipliers kept on the device (oracle: Alg. 1 with
    mu0 / cov0 and the multiplier warm start)."""
    p1 = scene(dims=2, n_obs=14, n_dyn=2, n_p=40, seed=61)
    p1["seed"] = 321
    cem = _cem(48)
    (p2, _), = _replans([(p1, cem)], [0])
    with _ctx(P, P.PRIEST_FP64_CHECK) as ctx:
        g1 = ctx.wait(ctx.submit(p1, cem, robot_id=9))
        g2 = ctx.wait(ctx.submit(p2, cem, robot_id=9))
        assert ctx.serve_stats()["warm_starts"] == 1
    w1 = oracle.plan(p1, cem, z=_oracle_z(oracle, p1, cem), want_lam=True)
    w2 = oracle.plan(p2, cem, mu0=w1["mu"], cov0=w1["cov"], z=_oracle_z(oracle, p2, cem), lam0=w1["lam"])
    cold = oracle.plan(p2, cem, z=_oracle_z(oracle, p2, cem))
    s = scale_of(p1)
    assert rel_err(g1["best"], w1["best"], s) < TOL_FP64
    assert g2["best_index"] == w2["elites"][0]
    assert rel_err(g2["best"], w2["best"], s) < TOL_FP64
    assert rel_err(g2["mu"], w2["mu"], s) < TOL_FP64
    assert rel_err(cold["mu"], w2["mu"], s) > 1e-6  # the warm start mattered


def test_ticket_semantics(P):
    p, cem = _requests()[0]
    with _ctx(P, P.PRIEST_FP32) as ctx:
        res = P.priest_result()
        with pytest.raises(P.PriestError) as e:
            P.priest_poll(ctx.h, 12345, res)
        assert e.value.status == P.PRIEST_ERR_INVALID
        t = ctx.submit(p, cem)
        r = ctx.wait(t, timeout_ms=60_000)
        assert r["status"] == 0 and r["latency_ms"] > 0
        with pytest.raises(P.PriestError) as e:
            P.priest_poll(ctx.h, t, res)  # already released
        assert e.value.status == P.PRIEST_ERR_INVALID


def test_request_over_budget_rejected(P):
    p, cem = _requests()[2]
    with _ctx(P, P.PRIEST_FP32, hbm_budget=1 << 16) as ctx:
        with pytest.raises(P.PriestError) as e:
            ctx.submit(p, cem)
        assert e.value.status == P.PRIEST_ERR_BUDGET


def test_wait_timeout_leaves_ticket_pending(P):
    """priest_wait with a limit shorter than the solve returns
    PRIEST_ERR_TIMEOUT and leaves the ticket pending; a later wait returns
    the result (failure detection of the serving loop by its bounded wait)."""
    p = scene(dims=2, n_obs=120, n_dyn=10, n_p=100, seed=77)
    cem = W.cem_settings(1024, 60, 3, dims=2)
    with _ctx(P, P.PRIEST_FP64_CHECK) as ctx:  # an FP64 solve of this size takes far longer than 1 ms
        t = ctx.submit(p, cem)
        res = P.priest_result()
        with pytest.raises(P.PriestError) as e:
            P.priest_wait(ctx.h, t, res, timeout_ms=1.0)
        assert e.value.status == P.PRIEST_ERR_TIMEOUT
        r = ctx.wait(t)  # no limit
        assert r["status"] == 0 and r["latency_ms"] > 1.0
