"""Geometric pins of the oracle's closed-form alpha / beta / d updates
(Appendix, eqs. collision_avoidance_proposed, fv, fa and the AM steps
comp_alpha, comp_beta, comp_d), against textbook geometry and 1-D searches.
No GPU."""
import math

import numpy as np
import pytest


def golden_min(f, lo, hi, iters=200):
    g = (math.sqrt(5) - 1) / 2
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(iters):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def rand_cases(dims, n=300, seed=0):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        a = rng.uniform(0.2, 1.0)
        b = rng.uniform(0.2, 1.0) if dims == 3 else a
        o = rng.uniform(-5, 5, dims)
        pos = o + rng.normal(0, 1.0, dims) * rng.uniform(0.05, 2.0)
        yield pos, o, a, b


@pytest.mark.parametrize("dims", [2, 3])
def test_obstacle_target_geometry(oracle, dims):
    n_in = 0
    for pos, o, a, b in rand_cases(dims):
        al, be, d, e = oracle.obstacle_polar(dims, pos, o, a, b)
        assert d >= 1.0
        scale = np.array([a, a, b][:dims])
        rs = np.linalg.norm((pos - o) / scale)
        if rs >= 1.0:
            # outside the ellipsoid: the target is the point itself (zero residual)
            np.testing.assert_allclose(e, pos, atol=1e-12)
            assert d == pytest.approx(rs, rel=1e-12)
        else:
            n_in += 1
            # inside: target on the surface, on the ray from the centre through the point
            assert np.linalg.norm((e - o) / scale) == pytest.approx(1.0, abs=1e-12)
            u, w = pos - o, e - o
            cos = u @ w / (np.linalg.norm(u) * np.linalg.norm(w))
            assert cos == pytest.approx(1.0, abs=1e-12)
            if dims == 2 or abs(a - b) < 1e-15:
                # circle / sphere: the textbook nearest surface point
                np.testing.assert_allclose(e, o + a * u / np.linalg.norm(u), atol=1e-12)
    assert n_in > 30


@pytest.mark.parametrize("dims", [2, 3])
def test_alpha_and_d_are_argmins(oracle, dims):
    """alpha minimises ||Delta - d u(alpha, beta)||^2 for fixed (beta, d); d is
    the minimiser over d >= 1 for fixed angles (golden-section search)."""
    for pos, o, a, b in list(rand_cases(dims, n=40, seed=1)):
        al, be, d, e = oracle.obstacle_polar(dims, pos, o, a, b)
        dl = pos - o

        def u(alpha, beta):
            if dims == 2:
                return np.array([a * math.cos(alpha), a * math.sin(alpha)])
            return np.array([a * math.cos(alpha) * math.sin(beta), a * math.sin(alpha) * math.sin(beta),
                             b * math.cos(beta)])

        f_al = lambda x: np.sum((dl - d * u(x, be)) ** 2)
        best = golden_min(f_al, al - 1.0, al + 1.0)
        assert f_al(al) <= f_al(best) + 1e-10
        f_d = lambda x: np.sum((dl - x * u(al, be)) ** 2)
        dbest = max(1.0, golden_min(f_d, 0.0, 20.0))
        assert d == pytest.approx(dbest, abs=1e-6)


def test_beta_is_polar_angle_for_spheres(oracle):
    rng = np.random.default_rng(5)
    for _ in range(50):
        o = rng.uniform(-3, 3, 3)
        pos = o + rng.normal(size=3)
        al, be, d, e = oracle.obstacle_polar(3, pos, o, 0.7, 0.7)
        dl = pos - o
        # spherical coordinates: polar angle from +z, azimuth in the xy plane
        assert be == pytest.approx(math.acos(dl[2] / np.linalg.norm(dl)), abs=1e-12)
        assert al == pytest.approx(math.atan2(dl[1], dl[0]), abs=1e-15)


def test_degenerate_direction(oracle):
    o = np.array([1.0, 2.0, 3.0])
    al, be, d, e = oracle.obstacle_polar(2, o[:2], o[:2], 0.5, 0.5)
    assert al == 0.0 and d == 1.0
    np.testing.assert_array_equal(e, o[:2] + [0.5, 0.0])
    al, be, d, e = oracle.obstacle_polar(3, o, o, 0.5, 0.4)
    assert al == 0.0 and be == 0.0 and d == 1.0
    np.testing.assert_allclose(e, o + [0.0, 0.0, 0.4], atol=1e-16)


@pytest.mark.parametrize("dims", [2, 3])
def test_velocity_bound_target(oracle, dims):
    rng = np.random.default_rng(2)
    for _ in range(200):
        v = rng.normal(0, 2.0, dims)
        vmax = rng.uniform(0.5, 3.0)
        al, be, d, e = oracle.bound_polar(dims, v, vmax)
        assert 0.0 <= d <= 1.0
        # ||e|| = min(||v||, vmax) and e parallel to v
        assert np.linalg.norm(e) == pytest.approx(min(np.linalg.norm(v), vmax), rel=1e-12)
        assert e @ v == pytest.approx(np.linalg.norm(e) * np.linalg.norm(v), rel=1e-12)
    al, be, d, e = oracle.bound_polar(dims, np.zeros(dims), 1.0)
    assert d == 0.0 and np.all(e == 0.0)
