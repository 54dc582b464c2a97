"""Pins of the oracle's D-PRIEST (Sec. D-PRIEST, Fig. fig_decentralized): M
distributions refined in parallel on one stacked projection, best of M.
Pinned by reduction (M = 1 is Alg. 1), by decomposition (each distribution
is an independent Alg. 1 on its rows, because the stacked projection never
mixes rows), and by the geometry of the default means."""
import numpy as np
import pytest

from paper_2309_08235_gb300 import workloads as W


def test_single_distribution_is_alg1(oracle):
    p = W.scene_small_2d(n_obs=6, n_p=30)
    cem = W.cem_settings(24, 8, 3, n_proj=16, n_elite=5)
    z = W.normals(31, (3, 24, 22))
    a = oracle.plan_multi(p, cem, 1, z=z)
    b = oracle.plan(p, cem, z=z)
    np.testing.assert_array_equal(a["best"], b["best"])
    np.testing.assert_array_equal(a["mu"][0], b["mu"])
    assert a["dist"] == 0 and a["c_aug"] == b["c_aug"]


@pytest.mark.parametrize("dims", [2, 3])
def test_distributions_are_independent_alg1_runs(oracle, dims):
    if dims == 2:
        p = W.scene_small_2d(n_obs=8, n_p=30)
    else:
        p = W.scene_ellipsoids_3d(n_obs=10, n_p=25)
    M, nj = 3, 12
    D = dims * 11
    cem = W.cem_settings(M * nj, 6, 2, n_proj=M * 8, n_elite=M * 3, dims=dims)
    z = W.normals(32, (2, M * nj, D))
    means = oracle.multi_default_means(p, M, 2.0 * cem["init_std"])
    got = oracle.plan_multi(p, cem, M, z=z)
    sub = dict(cem, n_samples=nj, n_proj=8, n_elite=3)
    caugs = []
    for j in range(M):
        want = oracle.plan(p, sub, mu0=means[j], z=z[:, j * nj:(j + 1) * nj])
        np.testing.assert_allclose(got["dist_best"][j], want["best"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(got["mu"][j], want["mu"], rtol=0, atol=1e-12)
        assert got["dist_c_aug"][j] == pytest.approx(want["c_aug"], abs=1e-12)
        caugs.append(want["c_aug"])
    assert got["dist"] == int(np.argmin(caugs))
    np.testing.assert_array_equal(got["best"], got["dist_best"][got["dist"]])


def test_default_means_geometry(oracle):
    p = W.scene_small_2d(n_obs=2)
    M, spread = 4, 1.5
    mus = oracle.multi_default_means(p, M, spread)
    base = oracle.default_mean(p)
    d = np.asarray(p["bf"])[:, 0] - np.asarray(p["b0"])[:, 0]
    for j in range(M):
        off = (mus[j] - base).reshape(2, 11)
        # end coefficients untouched, interior moved by one vector normal to the line
        assert np.all(off[:, 0] == 0) and np.all(off[:, 10] == 0)
        v = off[:, 5]
        np.testing.assert_allclose(off[:, 1:10], np.repeat(v[:, None], 9, 1), atol=1e-14)
        assert abs(v @ d) < 1e-12
        assert np.linalg.norm(v) == pytest.approx(abs(j - (M - 1) / 2) * spread, abs=1e-12)
    # symmetric about the straight line
    np.testing.assert_allclose(mus[0] - base, -(mus[-1] - base), atol=1e-12)
