"""The oracle's converged multi-obstacle projection (Sec. III-A, eqs.
fixed_point_1, lag, affine_trans) against what the iteration fixes once it
has converged, with nothing taken from the oracle but its output.  A
strictly feasible iterate makes every residual row zero, so the multipliers
stop moving and the iteration rests at the feasible point
xi_bar = Pi_A(xi + lambda): a fixed point of the method, not the nearest
feasible point (which one depends on the multipliers accumulated while the
sample was infeasible).  Checked here:

* feasibility at every time stamp, evaluated with a Bernstein basis written
  in this file (binomial form, derivatives by the degree-lowering identity):
  scaled obstacle distance >= 1 (moving obstacles at their position at the
  time stamp), |v| <= v_max, |a| <= a_max;
* the equality rows held exactly (both ends at rest: the three end
  coefficients per axis equal the end positions);
* the fixed-point identity on the free coefficients, xi_bar_F = xi_F + lambda_F;
* boundary fixed points: the scenes make obstacle contact (2-D) and the
  acceleration bound (2-D, 3-D) active at convergence, so the checks are not
  met trivially in the interior.
"""
from math import comb

import numpy as np

from paper_2309_08235_gb300 import workloads as W

DEG = 10  # degree of the workloads' Bernstein basis


def bernstein_rows(n, n_p, horizon):
    """Position, velocity and acceleration rows at tau_k = k / (n_p - 1)."""
    tau = np.linspace(0.0, 1.0, n_p)

    def b(m, k):
        return comb(m, k) * tau ** k * (1.0 - tau) ** (m - k) if 0 <= k <= m else 0.0 * tau

    B0 = np.stack([b(n, k) for k in range(n + 1)], 1)
    B1 = np.stack([n * (b(n - 1, k - 1) - b(n - 1, k)) for k in range(n + 1)], 1) / horizon
    B2 = np.stack([n * (n - 1) * (b(n - 2, k - 2) - 2.0 * b(n - 2, k - 1) + b(n - 2, k)) for k in range(n + 1)],
                  1) / horizon ** 2
    return B0, B1, B2, tau * horizon


def test_bernstein_rows_are_the_basis():
    """The rows written here: partition of unity, and the velocity / acceleration
    rows as finite differences of the position rows."""
    B0, B1, B2, t = bernstein_rows(DEG, 4001, 8.0)
    np.testing.assert_allclose(B0.sum(1), 1.0, atol=1e-13)
    h = t[1] - t[0]  # central differences: error h^2 / 6 x the third derivative, about 5e-6 here
    np.testing.assert_allclose((B0[2:] - B0[:-2]) / (2 * h), B1[1:-1], atol=1e-5)
    np.testing.assert_allclose((B1[2:] - B1[:-2]) / (2 * h), B2[1:-1], atol=1e-5)


def converged_checks(oracle, p, xi, K, centre, vel, semi, start, goal):
    dims, n_p, T = p["dims"], p["n_p"], p["horizon"]
    nv = DEG + 1
    B0, B1, B2, t = bernstein_rows(DEG, n_p, T)
    xb, lam = oracle.project(p, xi, K)
    free = np.r_[3:nv - 3]
    out = []
    for s in range(xb.shape[0]):
        cf = [xb[s, ax * nv:(ax + 1) * nv] for ax in range(dims)]
        for ax in range(dims):
            # equality rows: at rest at both ends
            np.testing.assert_allclose(cf[ax][:3], start[ax], atol=1e-12)
            np.testing.assert_allclose(cf[ax][-3:], goal[ax], atol=1e-12)
            # fixed point on the free coefficients
            d = xb[s, ax * nv + free] - xi[s, ax * nv + free] - lam[s, ax * nv + free]
            assert np.abs(d).max() < 1e-10 * max(1.0, np.abs(xb[s]).max())
        pos = [B0 @ c for c in cf]
        v = np.sqrt(sum((B1 @ c) ** 2 for c in cf))
        acc = np.sqrt(sum((B2 @ c) ** 2 for c in cf))
        d2 = np.zeros((n_p, len(semi)))
        for ax in range(dims):
            o = centre[None, :, ax] + t[:, None] * vel[None, :, ax]
            s_ax = semi[None, :, 1] if (dims == 3 and ax == 2) else semi[None, :, 0]
            d2 += ((pos[ax][:, None] - o) / s_ax) ** 2
        out.append((d2.min(), v.max() / p["vmax"], acc.max() / p["amax"]))
    out = np.array(out)
    assert out[:, 0].min() >= 1.0 - 1e-9  # outside every obstacle
    assert out[:, 1].max() <= 1.0 + 1e-9 and out[:, 2].max() <= 1.0 + 1e-9  # within the bounds
    return out


def test_converged_2d_projection_with_contact(oracle):
    """Four circles along a 16 m line, one of them moving; a_max 2 m/s^2 makes
    the acceleration bound bind.  Six perturbed samples, K = 8000."""
    centre = np.array([[4.0, 0.4], [8.0, -0.5], [12.0, 0.3], [6.0, 3.0]])
    vel = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [0.3, -0.6]])
    a = np.array([0.9, 0.8, 0.9, 0.6])
    semi = np.stack([a, a], 1)
    start, goal = np.array([0.0, 0.0]), np.array([16.0, 0.0])
    p = W.problem(2, 50, 8.0, start, goal, centre, vel, semi, 3.0, 2.0, seed=1)
    xi = oracle.default_mean(p)[None] + np.random.default_rng(5).normal(0.0, 0.4, (6, 22))
    out = converged_checks(oracle, p, xi, 8000, centre, vel, semi, start, goal)
    assert np.count_nonzero(np.abs(out[:, 0] - 1.0) < 1e-6) >= 1  # obstacle contact
    assert np.count_nonzero(np.abs(out[:, 2] - 1.0) < 1e-6) >= 1  # acceleration bound active


def test_converged_3d_projection(oracle):
    """Three ellipsoids (a != b) along a rising 14 m line, a_max 1.6 m/s^2.
    Four perturbed samples, K = 2000."""
    centre = np.array([[4.0, 0.3, 0.8], [8.0, -0.4, 1.2], [10.0, 0.2, 1.8]])
    semi = np.array([[0.9, 0.6], [0.8, 1.0], [0.7, 0.5]])
    vel = np.zeros_like(centre)
    start, goal = np.zeros(3), np.array([14.0, 0.0, 2.0])
    p = W.problem(3, 50, 8.0, start, goal, centre, None, semi, 3.0, 1.6, seed=1)
    xi = oracle.default_mean(p)[None] + np.random.default_rng(7).normal(0.0, 0.4, (4, 33))
    out = converged_checks(oracle, p, xi, 2000, centre, vel, semi, start, goal)
    assert np.count_nonzero(np.abs(out[:, 2] - 1.0) < 1e-6) >= 1  # acceleration bound active


def test_fixed_point_identity_is_not_vacuous(oracle):
    """On a sample the projection had to move, the multipliers carry the move:
    xi_bar_F - xi_F is far from zero, so the identity above tests lambda."""
    centre = np.array([[4.0, 0.4], [8.0, -0.5]])
    a = np.array([0.9, 0.8])
    p = W.problem(2, 50, 8.0, np.zeros(2), np.array([16.0, 0.0]), centre, None, np.stack([a, a], 1), 3.0, 2.0)
    xi = oracle.default_mean(p)[None]
    xb, lam = oracle.project(p, xi, 2000)
    free = np.r_[3:8, 14:19]
    assert np.abs(xb[0, free] - xi[0, free]).max() > 1e-2
    np.testing.assert_allclose(xb[0, free] - xi[0, free], lam[0, free], atol=1e-10)
