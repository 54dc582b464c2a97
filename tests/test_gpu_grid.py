"""The static-obstacle grid of the neighbour-list builds (Sec. III-A, eq.
comp_d: only obstacles near a point can be active there).  A grid cell holds
every static obstacle whose inflated pre-filter can accept a point in the
cell, in obstacle order, so the lists, and with them every output, are
bitwise the same as with every static obstacle screened at each rebuild
(PRIEST_LIST_GRID=0) and as with every obstacle screened exactly in every
iteration (PRIEST_NEIGHBOUR_LISTS=0); the outputs also match the FP64
oracle.  Scenes: the 2-D clutter and 3-D ellipsoid workloads, the dense
1,500-circle box, radii from 5 cm to 2.5 m along a 150 m start-goal line
(obstacles 75 m from the frame origin: the pre-filter's rounding margin and
the grid's slack), and a pile of 80 coincident obstacles that turns the grid
off."""
import os

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


def far_mixed():
    """60 obstacles (6 moving), radii U[0.05, 2.5], along (0, 0) -> (120, 90)."""
    rng = np.random.default_rng(17)
    start, goal = np.array([0.0, 0.0]), np.array([120.0, 90.0])
    t = rng.uniform(0.05, 0.95, 60)
    c = start + t[:, None] * (goal - start) + rng.normal(0.0, 3.0, (60, 2))
    r = rng.uniform(0.05, 2.5, 60)
    v = np.zeros((60, 2))
    v[54:] = rng.uniform(-1.0, 1.0, (6, 2))
    return W.problem(2, 100, 40.0, start, goal, c, v, np.stack([r, r], 1), 4.0, 4.0, seed=17)


def pile():
    """The clutter scene plus 80 circles on one centre (the start-goal midpoint)."""
    p = W.scene_clutter_2d(seed=4, n_static=90, n_dyn=10, n_p=100)
    c = np.asarray(p["center"], dtype=float)
    s = np.asarray(p["semi"], dtype=float)
    v = np.asarray(p["vel"], dtype=float)
    mid = 0.5 * (np.asarray(p["b0"])[:, 0] + np.asarray(p["bf"])[:, 0])
    c = np.vstack([c[:90], np.repeat(mid[None], 80, 0), c[90:]])
    s = np.vstack([s[:90], np.full((80, 2), 0.4), s[90:]])
    v = np.vstack([v[:90], np.zeros((80, 2)), v[90:]])
    return dict(p, center=c, semi=s, vel=v, n_obs=c.shape[0])


# scene, samples, K, draw std, expect a grid
SCENES = {
    "clutter2d": (lambda: W.scene_clutter_2d(seed=3, n_static=90, n_dyn=10, n_p=100), 300, 40, 2.0, True),
    "ellipsoid3d": (lambda: W.scene_ellipsoids_3d(seed=2, n_obs=200, n_p=150), 150, 30, 1.5, True),
    "dense": (lambda: W.scene_clutter_2d(seed=9, n_static=1350, n_dyn=150, n_p=60, horizon=4.8), 200, 20, 2.0,
              True),
    "far_mixed": (far_mixed, 200, 30, 6.0, True),
    "pile": (pile, 200, 30, 2.0, False),
}


def run(P, p, xi, K, lam0, env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        with P.Context(p, {"proj_iters": K}, precision=P.PRIEST_FP32, autotune=0) as ctx:
            out = ctx.project(p, xi, lam=lam0)
            kind = P.priest_last_kernel(ctx.h)
            grid = P.priest_grid_info(ctx.h)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out, kind, grid


@pytest.mark.parametrize("name", list(SCENES))
def test_grid_lists_equal_full_screening(P, oracle, name):
    mk, n, K, std, want_grid = SCENES[name]
    p = mk()
    D = p["dims"] * 11
    xi = oracle.default_mean(p) + std * W.normals(40 + len(name), (n, D))
    lam0 = np.random.default_rng(6).normal(0.0, 0.1, xi.shape)
    a, kind_a, grid = run(P, p, xi, K, lam0, {})
    b, kind_b, grid_b = run(P, p, xi, K, lam0, {"PRIEST_LIST_GRID": "0"})
    c, kind_c, _ = run(P, p, xi, K, lam0, {"PRIEST_NEIGHBOUR_LISTS": "0"})
    assert kind_a == kind_b == kind_c == 1  # the point-owner kernel
    assert grid == grid_b  # the tables carry the grid either way
    if want_grid:
        nx, ny, ent = grid
        n_static = int(np.count_nonzero(np.all(np.asarray(p["vel"]) == 0.0, axis=1)))
        assert nx > 0 and ny > 0 and n_static <= ent <= 4 * n_static
    else:
        assert grid == (0, 0, 0)
    for x, y, z in zip(a, b, c):  # xi_bar, lambda, r, c_1
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
    idx = np.r_[0:n:23, n - 1]
    xb_o, lam_o = oracle.project(p, xi[idx], K, lam=lam0[idx])
    r_o, c1_o = oracle.residual_cost(p, xb_o)
    xb, lam, r, c1 = a
    assert rel_err(xb[idx], xb_o, scale_of(p)) < TOL_FP32
    assert rel_err(lam[idx], lam_o, 1.0) < TOL_FP32
    assert rel_err(r[idx], r_o, 1.0) < TOL_FP32
    assert rel_err(c1[idx], c1_o, max(1.0, np.abs(c1_o).max())) < TOL_FP32
    assert np.count_nonzero(r_o > 1e-6) > 0  # obstacles are active


def test_list_margin_does_not_change_results(P, oracle):
    """Any positive list margin gives bitwise the same outputs: the lists hold
    every obstacle that can be active while a point stays within 7/8 of the
    margin of its rebuild position.  0.35, 0.75 (the default) and 1.5 mean
    semi-axes (PRIEST_LIST_MARGIN) on the 2-D clutter scene: the smallest
    rebuilds most often, the largest keeps the longest lists."""
    p = W.scene_clutter_2d(seed=3, n_static=90, n_dyn=10, n_p=100)
    xi = oracle.default_mean(p) + 2.0 * W.normals(77, (300, 22))
    lam0 = np.random.default_rng(8).normal(0.0, 0.1, xi.shape)
    outs = []
    for m in ("0.35", "0.75", "1.5"):
        out, kind, grid = run(P, p, xi, 40, lam0, {"PRIEST_LIST_MARGIN": m})
        assert kind == 1 and grid[0] > 0
        outs.append(out)
    for o in outs[1:]:
        for x, y in zip(outs[0], o):  # xi_bar, lambda, r, c_1
            np.testing.assert_array_equal(x, y)
