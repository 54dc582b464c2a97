"""Pins of the oracle's BARN-style cost c_1 (acceleration, curvature and
path-following penalties; Sec. Baselines and Benchmarks) against geometry
that fixes each term: a trajectory on the start-goal line has no curvature
and no path error, a parallel offset has path error = offset, a circular arc
has curvature 1 / R, points past the goal measure to the goal."""
import numpy as np
import pytest

from paper_2309_08235_gb300 import workloads as W


def _traj_coeffs(oracle, p, fn, n_fit=400):
    """Least-squares Bernstein coefficients (degree 10) of a path fn(tau)."""
    tau = np.linspace(0.0, 1.0, n_fit)
    P, _, _ = oracle.basis(10, n_fit, p["horizon"])
    pts = fn(tau)  # n_fit x dims
    c, *_ = np.linalg.lstsq(P, pts, rcond=None)
    return c.T.reshape(-1)  # axis-major


def _cost(oracle, p, xi):
    return oracle.residual_cost(p, np.asarray(xi)[None])[1][0]


def test_acceleration_only_weights_reduce_to_default(oracle):
    p = W.scene_small_2d(n_obs=3, n_p=40)
    xi = oracle.default_mean(p) + 0.7 * W.normals(2, 22)
    a = _cost(oracle, p, xi)
    b = _cost(oracle, W.with_barn_cost(p, w_acc=1.0, w_curv=0.0, w_path=0.0), xi)
    assert b == pytest.approx(a, rel=1e-14)


def test_straight_line_has_only_acceleration(oracle):
    p = W.scene_small_2d(n_obs=3, n_p=40)
    xi = oracle.project_eq(p, oracle.default_mean(p)[None])[0]  # on the start-goal line, rest-to-rest
    acc_only = _cost(oracle, p, xi)
    assert acc_only > 0.0
    q = W.with_barn_cost(p, w_acc=1.0, w_curv=5.0, w_path=5.0)
    assert _cost(oracle, q, xi) == pytest.approx(acc_only, rel=1e-9, abs=1e-12)


def test_parallel_offset_path_error(oracle):
    p = W.scene_small_2d(n_obs=3, n_p=50)
    s, g = np.asarray(p["b0"])[:, 0], np.asarray(p["bf"])[:, 0]
    n = np.array([-(g - s)[1], (g - s)[0]]) / np.linalg.norm(g - s)
    delta = 0.37
    xi = oracle.default_mean(p).reshape(2, 11)
    xi = (xi + delta * n[:, None]).reshape(-1)  # every coefficient moved: the whole path is offset
    q = W.with_barn_cost(p, w_acc=0.0, w_curv=0.0, w_path=1.0)
    assert _cost(oracle, q, xi) == pytest.approx(p["n_p"] * delta ** 2, rel=1e-12)


def test_points_past_the_goal_measure_to_the_goal(oracle):
    p = W.problem(2, 30, 5.0, [0, 0], [4, 0], np.zeros((0, 2)), None, np.zeros((0, 2)), vmax=10, amax=10)
    # a path along the x axis from 5 to 6 (beyond the goal at x = 4)
    xi = _traj_coeffs(oracle, p, lambda tau: np.stack([5.0 + tau, 0.0 * tau], 1))
    q = W.with_barn_cost(p, w_acc=0.0, w_curv=0.0, w_path=1.0)
    tt = np.linspace(0, 1, 30)
    want = np.sum((1.0 + tt) ** 2)
    assert _cost(oracle, q, xi) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("R", [2.0, 5.0])
def test_circular_arc_curvature(oracle, R):
    T = 4.0
    p = W.problem(2, 60, T, [R, 0], [0, R], np.zeros((0, 2)), None, np.zeros((0, 2)), vmax=10, amax=10)
    # quarter circle at constant angular rate: speed V = R (pi / 2) / T
    xi = _traj_coeffs(oracle, p, lambda tau: np.stack([R * np.cos(0.5 * np.pi * tau), R * np.sin(0.5 * np.pi * tau)], 1))
    eps = 0.1
    q = W.with_barn_cost(p, w_acc=0.0, w_curv=1.0, w_path=0.0, curv_eps=eps)
    V = R * 0.5 * np.pi / T
    # |v x a| = V^3 / R on a circle
    kappa = (V ** 3 / R) / (V ** 2 + eps ** 2) ** 1.5
    assert _cost(oracle, q, xi) == pytest.approx(p["n_p"] * kappa ** 2, rel=2e-4)
