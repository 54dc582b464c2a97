"""GPU check of the device Cholesky factor (the sampling factor
chol(Sigma + eps I) of Alg. 1, formed in the setup and after every refit)
through the C ABI diagnostic priest_chol_selftest, against LAPACK's factor
(numpy) and against the defining identity L L^T = A.  The widths cover the
refit (256 threads), the setup (512) and a single warp; the sizes cover a
lone pivot, the 2-D and 3-D covariance sizes (2 x 11, 3 x 11) and the largest
one (3 x 16)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2309_08235_gb300 import build, priest

    build.build()
    return priest


def spd(D, seed, scale=1.0, cond=1e3):
    """A symmetric positive definite matrix with eigenvalues spread
    geometrically over [scale / cond, scale] in a random basis."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(D, D)))
    a = scale * (Q * np.geomspace(1.0, 1.0 / cond, D)) @ Q.T
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("threads", [32, 256, 512])
@pytest.mark.parametrize("D", [1, 2, 5, 22, 33, 48])
def test_cholesky_matches_lapack(P, D, threads):
    a = spd(D, seed=D)
    st, L = P.priest_chol_selftest(a, threads)
    assert st == P.PRIEST_OK
    assert np.all(np.triu(L, 1) == 0.0)
    want = np.linalg.cholesky(a)
    # forward error of a backward-stable factor: about cond(A) x eps
    assert np.abs(L - want).max() / np.abs(want).max() < 1e-12
    # backward error: |L L^T - A| <= c D eps |L| |L^T|
    assert np.abs(L @ L.T - a).max() / np.abs(a).max() < 1e-13


@pytest.mark.parametrize("scale", [1e-12, 1e-3, 1e4, 1e12])
def test_cholesky_across_magnitudes(P, scale):
    a = spd(22, seed=7, scale=scale, cond=1e6)
    st, L = P.priest_chol_selftest(a, 256)
    assert st == P.PRIEST_OK
    want = np.linalg.cholesky(a)
    assert np.abs(L - want).max() / np.abs(want).max() < 1e-9
    assert np.abs(L @ L.T - a).max() / np.abs(a).max() < 1e-13


def test_cholesky_of_the_first_sampling_covariance(P):
    """Sigma_0 = s^2 I plus chol_eps tr(Sigma_0) / D I: L is the diagonal
    sqrt(s^2 (1 + chol_eps)), exactly up to rounding."""
    D, s2, ce = 22, 0.3 ** 2, 1e-6
    a = np.eye(D) * (s2 + ce * s2)
    st, L = P.priest_chol_selftest(a, 256)
    assert st == P.PRIEST_OK
    assert np.abs(L - np.eye(D) * np.sqrt(s2 * (1 + ce))).max() < 4e-16


@pytest.mark.parametrize("bad", ["negative", "zero", "nan"])
def test_cholesky_flags_a_bad_pivot(P, bad):
    a = spd(22, seed=3)
    a[5, 5] = {"negative": -1.0, "zero": 0.0, "nan": np.nan}[bad]
    st, L = P.priest_chol_selftest(a, 256)
    assert st == P.PRIEST_ERR_NUMERIC
    # the bad pivot is taken as 1: the factor of the leading block is intact
    want = np.linalg.cholesky(a[:5, :5])
    assert np.abs(L[:5, :5] - want).max() < 1e-12
    assert np.all(np.isfinite(L))
