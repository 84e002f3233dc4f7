"""One Ogita-Aishima refinement step in plain numpy FP64 -- TEST
INFRASTRUCTURE ONLY (the same import rule as the rest of ``oracle``).

The step follows T. Ogita and K. Aishima, "Iterative refinement for
symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35 (2018),
Algorithm 1, in its notation: for A symmetric and X approximate
eigenvectors,

    R = I - X^T X,   S = X^T A X,   lambda_i = s_ii / (1 - r_ii),
    delta = 2 (||S - D||_2 + ||A||_2 ||R||_2),   D = diag(lambda),
    E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if |lambda_i - lambda_j| > delta,
    E_ij = r_ij / 2                                          otherwise,
    X' = X + X E.

The spectral norms are bounded here as the library bounds them (Frobenius
norms; ||A||_2 by max |lambda_i|): a larger delta only moves pairs to the
r_ij / 2 branch.  Plain numpy products; no blocking.  Pinned in
tests/test_oracle_refine.py (a fixed point at exact eigenvectors, quadratic
convergence to a prescribed spectrum and its eigenvectors)."""
import numpy as np


def ogita_aishima_step(A, X):
    """Returns (X', lambda) for one step from X; lambda are the Rayleigh
    quotients of X (the step's lambda_i)."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[1]
    R = np.eye(n) - X.T @ X
    S = X.T @ (A @ X)
    lam = np.diag(S) / (1.0 - np.diag(R))
    delta = 2.0 * (np.linalg.norm(S - np.diag(lam)) + np.abs(lam).max() * np.linalg.norm(R))
    E = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            if i != j and abs(lam[i] - lam[j]) > delta:
                E[i, j] = (S[i, j] + lam[j] * R[i, j]) / (lam[j] - lam[i])
            else:
                E[i, j] = 0.5 * R[i, j]
    return X + X @ E, lam
