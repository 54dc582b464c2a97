"""Pins of the oracle's projection (Sec. III-A, Appendix eqs. lagrange,
comp_alpha..comp_zeta) and of its residual / cost (Alg. 1), no GPU.

  * zero obstacles, inactive bounds: every iterate equals Pi_A(xi);
  * a feasible sample is a fixed point;
  * an explicit dense restatement of eqs. f_e, lag, matrix_vec, affine_trans
    (F with F_o replicated n_o times, M the inverse of the full KKT matrix,
    targets e from the ray geometry rather than the trigonometric form);
  * each xi_bar update is the constrained minimiser of the Lagrangian;
  * boundary conditions hold to rounding after any number of iterations;
  * the closed-form residual equals ||F xi_bar - e(xi_bar)|| of the
    trigonometric form;
  * the paper's simple benchmark (Fig. teaser): projection lowers r.
"""
import json
import os

import numpy as np
import pytest

from paper_2309_08235_gb300 import workloads as W
from test_oracle_basis_kkt import dense_F, small_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def traj(P, c):
    return P @ c


def ray_targets(p, P, Pd, Pdd, xb):
    """e of eq. f_e written from the geometry: each obstacle target is the point
    itself when outside, else the surface point on the ray from the centre;
    velocity / acceleration targets are v * min(1, vmax/||v||); bound targets
    tau - max(0, tau - G xi_bar)."""
    dims, nv, n_p = p["dims"], 11, p["n_p"]
    t = np.linspace(0, p["horizon"], n_p)
    C = xb.reshape(dims, nv)
    pos = np.stack([P @ C[a] for a in range(dims)], 1)
    vel = np.stack([Pd @ C[a] for a in range(dims)], 1)
    acc = np.stack([Pdd @ C[a] for a in range(dims)], 1)
    blocks = []  # list of (n_p x dims) target blocks, in the stacking order of dense_F
    for j in range(p["n_obs"]):
        o = p["center"][j] + np.outer(t, p["vel"][j])
        sc = np.array([p["semi"][j, 0]] * 2 + [p["semi"][j, 1]])[:dims]
        dl = pos - o
        rs = np.linalg.norm(dl / sc, axis=1)
        blocks.append(o + dl * (np.maximum(1.0, rs) / rs)[:, None])
    for v, m in ((vel, p["vmax"]), (acc, p["amax"])):
        n = np.linalg.norm(v, axis=1)
        blocks.append(v * np.minimum(1.0, m / np.maximum(n, 1e-300))[:, None])
    if p["use_bounds"]:
        lo, hi = -np.asarray(p["smin"]), np.asarray(p["smax"])
        blocks.append(lo - np.maximum(0.0, lo + pos))   # rows -P: tau = -s_min
        blocks.append(hi - np.maximum(0.0, hi - pos))   # rows +P: tau = +s_max
    # per axis: stack the blocks' column for that axis
    return np.concatenate([np.concatenate([b[:, a] for b in blocks]) for a in range(dims)])


def dense_step(p, P, Pd, Pdd, xi, xb, lam):
    """One iteration of eqs. lag, obtain_e, matrix_vec, affine_trans with
    explicit matrices."""
    dims, nv = p["dims"], 11
    F, _ = dense_F(p, P, Pd, Pdd)
    A1 = np.vstack([P[0], Pd[0], Pdd[0]] + [[P[-1], Pd[-1], Pdd[-1]][q] for q in range(3)
                                            if p["bc_final_mask"] >> q & 1])
    neq = A1.shape[0]
    A = np.zeros((dims * neq, dims * nv))
    b = np.zeros(dims * neq)
    for a in range(dims):
        A[a * neq:(a + 1) * neq, a * nv:(a + 1) * nv] = A1
        b[a * neq:(a + 1) * neq] = list(p["b0"][a]) + [p["bf"][a][q] for q in range(3)
                                                       if p["bc_final_mask"] >> q & 1]
    e = ray_targets(p, P, Pd, Pdd, xb)
    lam_new = lam - p["rho"] * F.T @ (F @ xb - e)
    D = dims * nv
    K = np.zeros((D + dims * neq, D + dims * neq))
    K[:D, :D] = np.eye(D) + p["rho"] * F.T @ F
    K[:D, D:] = A.T
    K[D:, :D] = A
    M = np.linalg.inv(K)
    eta = np.concatenate([p["rho"] * F.T @ e + lam_new + xi, b])
    return (M @ eta)[:D], lam_new


@pytest.mark.parametrize("dims,bounds,mask", [(2, False, 7), (3, False, 7), (2, True, 1), (3, True, 3)])
def test_dense_restatement(oracle, dims, bounds, mask):
    p = small_problem(dims=dims, n_obs=3, n_p=8, bounds=bounds, mask=mask)
    P, Pd, Pdd = oracle.basis(10, p["n_p"], p["horizon"])
    rng = np.random.default_rng(11)
    D = dims * 11
    xi = rng.normal(2.5, 2.0, (4, D))
    xb = oracle.project_eq(p, xi)
    lam = rng.normal(0, 0.1, (4, D))
    for k in range(6):
        want = [dense_step(p, P, Pd, Pdd, xi[i], xb[i], lam[i]) for i in range(4)]
        got_xb, got_lam = oracle.project(p, xi, 1, lam=lam, xi_bar0=xb)
        wxb = np.stack([w[0] for w in want])
        wlam = np.stack([w[1] for w in want])
        np.testing.assert_allclose(got_xb, wxb, rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(got_lam, wlam, rtol=1e-11, atol=1e-11)
        xb, lam = got_xb, got_lam


def test_update_minimises_lagrangian(oracle):
    """xi_bar^{k+1} minimises 1/2||x - xi||^2 - <lambda^{k+1}, x> + rho/2 ||F x - e^{k+1}||^2
    over {A x = b}: no feasible direction lowers it."""
    p = small_problem(dims=2, n_obs=3, n_p=8)
    P, Pd, Pdd = oracle.basis(10, p["n_p"], p["horizon"])
    F, _ = dense_F(p, P, Pd, Pdd)
    A, _ = oracle.equality(p)
    rng = np.random.default_rng(3)
    xi = rng.normal(2.5, 2.0, 22)
    xb0 = oracle.project_eq(p, xi[None])[0]
    e = ray_targets(p, P, Pd, Pdd, xb0)
    xb1, lam1 = oracle.project(p, xi[None], 1, xi_bar0=xb0[None])
    Lag = lambda x: 0.5 * np.sum((x - xi) ** 2) - lam1[0] @ x + 0.5 * p["rho"] * np.sum((F @ x - e) ** 2)
    # null space of the per-axis equality block
    _, _, vt = np.linalg.svd(A)
    N1 = vt[A.shape[0]:].T
    base = Lag(xb1[0])
    for _ in range(30):
        dvec = np.concatenate([N1 @ rng.normal(size=N1.shape[1]) for _ in range(2)])
        for h in (1e-3, -1e-3):
            assert Lag(xb1[0] + h * dvec) >= base - 1e-12


def test_zero_obstacles_is_equality_projection(oracle):
    p = W.problem(2, 50, 6.0, [0, 0], [10, 4], np.zeros((0, 2)), None, np.zeros((0, 2)),
                  vmax=1e6, amax=1e6)
    rng = np.random.default_rng(1)
    xi = rng.normal(3, 4, (6, 22))
    pa = oracle.project_eq(p, xi)
    for K in (1, 5, 20):
        xb, lam = oracle.project(p, xi, K)
        np.testing.assert_allclose(xb, pa, atol=1e-12 * np.abs(pa).max())
        np.testing.assert_allclose(lam, 0.0, atol=1e-12)


def test_feasible_sample_is_fixed_point(oracle):
    # slow straight line in an empty corridor, obstacles far away
    p = W.problem(3, 40, 10.0, [0, 0, 0], [3, 2, 1], [[50, 50, 50], [-40, 10, 3]], None,
                  [[0.5, 0.4], [0.6, 0.6]], vmax=5.0, amax=5.0)
    mu = oracle.default_mean(p)
    xi = oracle.project_eq(p, mu[None])
    r, _ = oracle.residual_cost(p, xi)
    assert r[0] == 0.0
    for K in (1, 10, 40):
        xb, lam = oracle.project(p, xi, K)
        np.testing.assert_allclose(xb, xi, atol=1e-13 * np.abs(xi).max())
        np.testing.assert_allclose(lam, 0.0, atol=1e-12)


@pytest.mark.parametrize("mask", [1, 3, 7])
def test_boundary_conditions_hold(oracle, mask):
    p = small_problem(dims=3, n_obs=5, n_p=30, mask=mask, horizon=4.0)
    A, b = oracle.equality(p)
    rng = np.random.default_rng(4)
    xi = rng.normal(2.5, 3.0, (5, 33))
    xb, _ = oracle.project(p, xi, 25)
    for ax in range(3):
        np.testing.assert_allclose(xb[:, ax * 11:(ax + 1) * 11] @ A.T, np.broadcast_to(b[ax], (5, len(b[ax]))),
                                   atol=1e-12 * max(1.0, np.abs(xb).max()))


@pytest.mark.parametrize("dims,bounds", [(2, False), (3, False), (2, True)])
def test_residual_closed_form_matches_stacked(oracle, dims, bounds):
    p = small_problem(dims=dims, n_obs=6, n_p=40, bounds=bounds)
    p["semi"][:, :] *= 3.0   # big obstacles so many rows are active
    rng = np.random.default_rng(8)
    xi = rng.normal(2.5, 2.0, (20, dims * 11))
    xb = oracle.project_eq(p, xi)
    r, c1 = oracle.residual_cost(p, xb)
    rs = oracle.residual_stacked(p, xb)
    assert np.count_nonzero(r) > 10
    np.testing.assert_allclose(r, rs, rtol=1e-10, atol=1e-12)
    # c_1: summed squared acceleration
    P, Pd, Pdd = oracle.basis(10, p["n_p"], p["horizon"])
    acc = np.stack([(Pdd @ xb[:, a * 11:(a + 1) * 11].T) for a in range(dims)])
    np.testing.assert_allclose(c1, (acc ** 2).sum((0, 1)), rtol=1e-12)


def teaser_problem(n_p=80):
    g = json.load(open(os.path.join(GOLDEN, "teaser_scene.json")))
    r = g["radius"]
    return W.problem(2, n_p, g["horizon_chosen"], g["start"], g["goal"], [g["center_chosen"]], None,
                     [[r, r]], vmax=g["vmax"], amax=g["amax"])


def test_teaser_projection_pushes_samples_out(oracle):
    """Fig. teaser: every sample starts inside the 7 m obstacle; projection
    lowers the residual and pushes most samples out."""
    p = teaser_problem()
    mu = oracle.default_mean(p)
    rng = np.random.default_rng(0)
    xi = mu + 0.5 * rng.normal(size=(16, 22))
    r0, _ = oracle.residual_cost(p, oracle.project_eq(p, xi))
    assert np.all(r0 > 1.0)
    rs = []
    for K in (10, 40, 120):
        xb, _ = oracle.project(p, xi, K)
        rs.append(oracle.residual_cost(p, xb)[0])
    assert np.median(rs[0]) < np.median(r0)
    assert np.median(rs[2]) < np.median(rs[0])
    assert np.median(rs[2]) < 0.1 * np.median(r0)


def test_converged_projection_on_a_two_variable_case(oracle):
    """Degree 6 with both ends at rest leaves one free coefficient per axis
    (c_3), so the projection of Sec. III-A is a two-variable problem that
    brute force can check.  One circle of radius 1 at the middle of the
    straight start-goal line (0, 0) -> (10, 0), horizon 4 s, 41 time stamps,
    velocity / acceleration bounds inactive; the sample's free coefficients
    are (5, 0.3).  At convergence the method fixes:
      * feasibility at every time stamp, checked here from the basis and the
        circle directly;
      * the mirror symmetry of the scene (t -> T - t, x -> 10 - x): c_3,x
        stays 5;
      * xi_bar = Pi_A(xi + lambda): with r = 0 the targets equal F xi_bar, so
        the minimiser of eq. lagrange under A xi_bar = b (eq. comp_zeta) is the
        equality projection of xi + lambda.
    The alpha / d steps (eqs. comp_alpha .. comp_d) do not involve lambda, so
    every feasible xi_bar with that property is a fixed point: the method
    stops at a feasible point, farther from xi than the Euclidean projection
    found by brute force (distance 2.90 at c_3,y = 3.2; the method stops near
    c_3,y = 3.94)."""
    p = W.problem(2, 41, 4.0, [0, 0], [10, 0], [[5.0, 0.0]], None, [[1.0, 1.0]], vmax=1e6, amax=1e6, degree=6)
    P, _, _ = oracle.basis(6, 41, 4.0)
    xi = np.array([0, 0, 0, 5.0, 10, 10, 10, 0, 0, 0, 0.3, 0, 0, 0])
    xb, lam = oracle.project(p, xi[None], 2000)
    r, _ = oracle.residual_cost(p, xb)
    xb, lam = xb[0], lam[0]
    x, y = P @ xb[:7], P @ xb[7:]
    assert r[0] == 0.0
    assert ((x - 5.0) ** 2 + y ** 2).min() >= 1.0 - 1e-9
    assert abs(xb[3] - 5.0) < 1e-9
    assert np.abs(xb - oracle.project_eq(p, (xi + lam)[None])[0]).max() < 1e-10
    # brute force: the nearest feasible (c_3,x, c_3,y) to (5, 0.3), coarse grid then fine
    B3, xfix = P[:, 3], P[:, 4:] @ np.array([10.0, 10.0, 10.0])

    def nearest(cx, cy):
        CX, CY = np.meshgrid(cx, cy, indexing="ij")
        X = np.multiply.outer(CX, B3) + xfix
        Y = np.multiply.outer(CY, B3)
        d2 = (CX - 5.0) ** 2 + (CY - 0.3) ** 2
        d2[((X - 5.0) ** 2 + Y ** 2 < 1.0).any(axis=-1)] = np.inf
        i = np.unravel_index(np.argmin(d2), d2.shape)
        return CX[i], CY[i], np.sqrt(d2[i])

    cx, cy, _ = nearest(np.arange(3.0, 7.0, 0.01), np.arange(0.0, 6.0, 0.01))
    cx, cy, dmin = nearest(np.arange(cx - 0.01, cx + 0.01, 1e-4), np.arange(cy - 0.01, cy + 0.01, 1e-4))
    assert abs(cy - 3.2) < 2e-4 and abs(dmin - 2.9) < 2e-4
    d_am = np.hypot(xb[3] - 5.0, xb[10] - 0.3)
    assert d_am >= dmin - 1e-3
    assert d_am > dmin + 0.5
