"""Pins of the oracle's Ogita-Aishima step (oracle/refine.py) against what
the mathematics fixes: exact eigenvectors are a fixed point (up to their own
rounding), and from a perturbed basis the step converges quadratically to
the prescribed eigenvectors and eigenvalues of A = Q diag(lambda) Q^T.  A
dropped term, a sign error or swapped indices in E breaks the quadratic
rate."""
import numpy as np

from oracle.refine import ogita_aishima_step
from paper_1811_01277_gb300 import inputs

U = 2.0 ** -53


def separated(n, seed):
    """Eigenvalues -1 + 2 (i + 1/2) / n with a small jitter: gaps near 2/n."""
    g = np.random.default_rng(seed)
    return -1.0 + 2.0 * (np.arange(n) + 0.5 + 0.2 * g.uniform(-1, 1, n)) / n


def basis_error(X, V):
    """max over columns of the distance to the matching exact eigenvector
    (signs aligned)."""
    s = np.sign(np.sum(X * V, axis=0))
    return np.abs(X - V * s).max()


def test_exact_eigenvectors_are_a_fixed_point():
    n = 120
    lam = separated(n, 1)
    A = inputs.symmetric_with_spectrum(lam, seed=2)
    w, V = np.linalg.eigh(A)
    X1, l1 = ogita_aishima_step(A, V)
    gap = np.diff(lam).min()
    assert np.abs(X1 - V).max() <= 100 * n * U / gap
    assert np.abs(l1 - lam).max() <= 100 * n * U


def test_quadratic_convergence_to_the_prescribed_eigenpairs():
    n = 150
    lam = separated(n, 3)
    A = inputs.symmetric_with_spectrum(lam, seed=4)
    _, V = np.linalg.eigh(A)                       # exact up to rounding (gaps ~ 2/n)
    g = np.random.default_rng(5)
    eps = []
    X = V + 1e-4 * g.standard_normal((n, n)) / np.sqrt(n)
    eps.append(basis_error(X, V))
    for _ in range(3):
        X, l = ogita_aishima_step(A, X)
        eps.append(basis_error(X, V))
    assert eps[0] > 1e-5
    assert eps[1] <= 50 * eps[0] ** 2 / (2.0 / n)   # quadratic, with the gap in the constant
    assert eps[2] <= max(50 * eps[1] ** 2 / (2.0 / n), 1e-12)
    assert eps[3] <= 1e-12
    assert np.abs(l - lam).max() <= 1e-13            # Rayleigh quotients of the converged basis
    assert np.abs(X.T @ X - np.eye(n)).max() <= 50 * n * U


def test_pairs_within_delta_take_half_of_r():
    """Two eigenvalues 1e-12 apart lie within delta: their E entries are
    r_ij / 2, so the step keeps the pair orthonormal instead of dividing by
    the tiny gap."""
    n = 40
    lam = separated(n, 6)
    lam[10] = lam[9] + 1e-12
    A = inputs.symmetric_with_spectrum(np.sort(lam), seed=7)
    _, V = np.linalg.eigh(A)
    g = np.random.default_rng(8)
    X = V + 1e-6 * g.standard_normal((n, n)) / np.sqrt(n)
    X1, _ = ogita_aishima_step(A, X)
    assert np.abs(X1.T @ X1 - np.eye(n)).max() <= 1e-10
