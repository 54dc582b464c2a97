"""Pins of the oracle's basis, equality block and KKT system against textbook
identities and an explicit dense restatement (no GPU).

Paper: Sec. II-A.2 (eq. parametrized, A xi = b_eq), Sec. III-A (eqs.
affine_trans / matrix_vec), Appendix (eq. f_e, eq. bound_con, Remark
matrix_scaling).
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from paper_2309_08235_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bernstein_monomial(n, j):
    """Monomial coefficients of B_{j,n}(tau) = sum_k (-1)^(k-j) C(n,k) C(k,j) tau^k."""
    c = np.zeros(n + 1)
    for k in range(j, n + 1):
        c[k] = (-1) ** (k - j) * math.comb(n, k) * math.comb(k, j)
    return c


@pytest.mark.parametrize("n,n_p,T", [(10, 100, 8.0), (10, 37, 3.0), (7, 60, 4.8), (15, 150, 12.0)])
def test_basis_against_monomial_form(oracle, n, n_p, T):
    P, Pd, Pdd = oracle.basis(n, n_p, T)
    tau = np.linspace(0.0, 1.0, n_p)
    for j in range(n + 1):
        c = bernstein_monomial(n, j)
        # the monomial form cancels heavily at high degree: tolerance from its coefficient mass
        tol = 1e-14 * np.abs(c).sum() * n * n
        np.testing.assert_allclose(P[:, j], npoly.polyval(tau, c), atol=tol)
        np.testing.assert_allclose(Pd[:, j], npoly.polyval(tau, npoly.polyder(c)) / T, atol=tol / T)
        np.testing.assert_allclose(Pdd[:, j], npoly.polyval(tau, npoly.polyder(c, 2)) / T**2,
                                   atol=tol / T**2)


def test_basis_identities(oracle):
    n, n_p, T = 10, 101, 5.0
    P, Pd, Pdd = oracle.basis(n, n_p, T)
    # partition of unity and its derivatives
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(Pd.sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose(Pdd.sum(1), 0.0, atol=1e-10)
    # endpoint interpolation
    assert P[0, 0] == 1.0 and np.all(P[0, 1:] == 0.0)
    assert P[-1, -1] == 1.0 and np.all(P[-1, :-1] == 0.0)
    # linear precision: coefficients k/n reproduce tau; velocity 1/T, acceleration 0
    k = np.arange(n + 1) / n
    np.testing.assert_allclose(P @ k, np.linspace(0, 1, n_p), atol=1e-14)
    np.testing.assert_allclose(Pd @ k, 1.0 / T, atol=1e-12)
    np.testing.assert_allclose(Pdd @ k, 0.0, atol=1e-10)


def test_basis_finite_differences(oracle):
    n, n_p, T = 10, 4001, 2.0
    P, Pd, Pdd = oracle.basis(n, n_p, T)
    h = T / (n_p - 1)
    fd1 = (P[2:] - P[:-2]) / (2 * h)
    fd2 = (Pd[2:] - Pd[:-2]) / (2 * h)
    np.testing.assert_allclose(Pd[1:-1], fd1, atol=1e-5 * np.abs(Pd).max())
    np.testing.assert_allclose(Pdd[1:-1], fd2, atol=1e-5 * np.abs(Pdd).max())


def small_problem(dims=2, n_obs=3, n_p=8, bounds=False, mask=7, horizon=3.0, seed=3):
    rng = np.random.default_rng(seed)
    c = rng.uniform(1, 4, (n_obs, dims))
    semi = np.stack([rng.uniform(0.3, 0.8, n_obs), rng.uniform(0.3, 0.8, n_obs)], 1)
    v = rng.uniform(-0.5, 0.5, (n_obs, dims))
    start = np.zeros(dims)
    goal = np.full(dims, 5.0)
    p = W.problem(dims, n_p, horizon, start, goal, c, v, semi, vmax=2.5, amax=3.0, seed=seed,
                  rho=1.3, use_bounds=bounds, smin=np.full(dims, -0.5), smax=np.full(dims, 4.5),
                  bc_final_mask=mask)
    # non-zero start velocity / acceleration so every BC row is exercised
    p["b0"][:, 1] = rng.uniform(-1, 1, dims)
    p["b0"][:, 2] = rng.uniform(-1, 1, dims)
    return p


@pytest.mark.parametrize("mask", [0, 1, 3, 5, 7])
def test_equality_rows(oracle, mask):
    p = small_problem(mask=mask)
    P, Pd, Pdd = oracle.basis(10, p["n_p"], p["horizon"])
    A, b = oracle.equality(p)
    rows = [P[0], Pd[0], Pdd[0]] + [[P[-1], Pd[-1], Pdd[-1]][q] for q in range(3) if mask >> q & 1]
    np.testing.assert_array_equal(A, np.array(rows))
    for ax in range(p["dims"]):
        want = list(p["b0"][ax]) + [p["bf"][ax][q] for q in range(3) if mask >> q & 1]
        np.testing.assert_array_equal(b[ax], want)


def dense_F(p, P, Pd, Pdd):
    """Explicit stacked F of eq. f_e (+ G of eq. bound_con): block diagonal over
    the axes, each block [F_o; Pd; Pdd] with F_o = P stacked n_obs times."""
    blk = [P] * p["n_obs"] + [Pd, Pdd]
    if p["use_bounds"]:
        blk += [-P, P]
    B = np.vstack(blk)
    dims = p["dims"]
    F = np.zeros((dims * B.shape[0], dims * B.shape[1]))
    for ax in range(dims):
        F[ax * B.shape[0]:(ax + 1) * B.shape[0], ax * B.shape[1]:(ax + 1) * B.shape[1]] = B
    return F, B


@pytest.mark.parametrize("bounds", [False, True])
@pytest.mark.parametrize("dims", [2, 3])
def test_kkt_matches_dense_F(oracle, bounds, dims):
    p = small_problem(dims=dims, bounds=bounds)
    P, Pd, Pdd = oracle.basis(10, p["n_p"], p["horizon"])
    K = oracle.kkt_matrix(p)
    A, _ = oracle.equality(p)
    F, B = dense_F(p, P, Pd, Pdd)
    nv = 11
    want = np.eye(nv) + p["rho"] * B.T @ B
    np.testing.assert_allclose(K[:nv, :nv], want, rtol=1e-13, atol=1e-12)
    np.testing.assert_array_equal(K[nv:, :nv], A)
    np.testing.assert_array_equal(K[:nv, nv:], A.T)
    assert np.all(K[nv:, nv:] == 0)
    # the full-dimension F^T F is block diagonal with the same block per axis
    FtF = F.T @ F
    for ax in range(dims):
        np.testing.assert_allclose(FtF[ax * nv:(ax + 1) * nv, ax * nv:(ax + 1) * nv], B.T @ B,
                                   rtol=1e-13)


def test_remark_matrix_scaling_dimensions(oracle):
    """Remark matrix_scaling: F is 3(n_o+2)n_p x 3n_v (3-D, no bounds)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    assert "matrix_scaling" in g["citation"]
    p = small_problem(dims=3, n_obs=4, n_p=9)
    P, Pd, Pdd = oracle.basis(10, 9, p["horizon"])
    F, _ = dense_F(p, P, Pd, Pdd)
    assert F.shape == (3 * (4 + 2) * 9, 3 * 11)


@pytest.mark.parametrize("mask", [1, 3, 7])
def test_projection_onto_equalities_closed_form(oracle, mask):
    p = small_problem(dims=3, mask=mask)
    A, b = oracle.equality(p)
    rng = np.random.default_rng(0)
    xi = rng.normal(2.0, 3.0, (5, 33))
    got = oracle.project_eq(p, xi)
    for ax in range(3):
        x = xi[:, ax * 11:(ax + 1) * 11]
        # textbook minimum-norm correction: xi - A^T (A A^T)^-1 (A xi - b)
        corr = (A.T @ np.linalg.solve(A @ A.T, (x @ A.T - b[ax]).T)).T
        np.testing.assert_allclose(got[:, ax * 11:(ax + 1) * 11], x - corr, atol=1e-10)
        np.testing.assert_allclose(got[:, ax * 11:(ax + 1) * 11] @ A.T, np.broadcast_to(b[ax], (5, len(b[ax]))),
                                   atol=1e-10)
