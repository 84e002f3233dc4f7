"""Ogita-Aishima refinement step (gb_refine_syev_d) on matrices with a
prescribed spectrum A = Q diag(lambda) Q^T: from eigenvectors of FP32
accuracy the error falls quadratically (orthogonality and residual), the
eigenvalues converge to the prescribed ones, clustered spectra converge to
the residual/orthogonality bounds, and exact eigenvectors are a fixed point."""
import numpy as np
import pytest

from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    build.build()
    m.load()
    return m


def errors(A, X, lam):
    n = A.shape[0]
    orth = np.abs(X.T @ X - np.eye(n)).max()
    res = np.linalg.norm(A @ X - X * lam) / np.linalg.norm(A)
    return orth, res


def refine(gb, A, X0, steps):
    n = A.shape[0]
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    X = torch.from_numpy(np.ascontiguousarray(X0.T)).to(dev)       # column-major X0
    lam = torch.zeros(n, dtype=torch.float64, device=dev)
    wsb = gb.gb_refine_syev_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    out = []
    for _ in range(steps):
        gb.gb_refine_syev_d(n, A_d, n, lam, X, n, ws, wsb, torch.cuda.current_stream())
        torch.cuda.synchronize()
        out.append((lam.cpu().numpy().copy(), X.cpu().numpy().T.copy()))
    return out


def test_refine_from_fp32_eigenvectors_converges_quadratically(gb):
    n = 640
    lam0 = np.sort(np.random.default_rng(1).uniform(-1.0, 1.0, n))
    A = inputs.symmetric_with_spectrum(lam0, seed=2)
    w, V = np.linalg.eigh(A)
    X0 = V.astype(np.float32).astype(np.float64)
    X0 += 1e-6 * np.random.default_rng(3).standard_normal((n, n)) / np.sqrt(n)
    o0, r0 = errors(A, X0, w)
    steps = refine(gb, A, X0, 3)
    (l1, X1), (l2, X2), (l3, X3) = steps
    o1, r1 = errors(A, X1, l2)
    o2, r2 = errors(A, X2, l3)
    assert o0 > 1e-8 and r0 > 1e-8
    assert o1 <= 1e3 * o0 ** 2 + 50 * n * U and r1 <= 1e3 * r0 ** 2 + 50 * n * U   # quadratic
    assert o2 <= 50 * n * U and r2 <= 50 * n * U
    assert np.abs(l3 - lam0).max() / np.abs(lam0).max() <= 1e-13


def test_refine_clustered_spectrum(gb):
    """Clusters of width 1e-8 lie below the step's separation threshold, so
    the step refines each cluster's invariant subspace (the method's stated
    limit): orthogonality and the subspace residual ||A X - X (X^T A X)||
    reach the bounds, and the eigenvalues of X^T A X are the prescribed
    ones."""
    n = 512
    lam0 = inputs.clustered_spectrum(n, seed=5)
    A = inputs.symmetric_with_spectrum(lam0, seed=6)
    w, V = np.linalg.eigh(A)
    X0 = V.astype(np.float32).astype(np.float64)
    X3 = refine(gb, A, X0, 3)[-1][1]
    S = X3.T @ A @ X3
    assert np.abs(X3.T @ X3 - np.eye(n)).max() <= 50 * n * U
    assert np.linalg.norm(A @ X3 - X3 @ S) / np.linalg.norm(A) <= 50 * n * U
    assert np.abs(np.linalg.eigvalsh(S) - np.sort(lam0)).max() / np.linalg.norm(A, 2) <= 1e-12


def test_refine_exact_eigenvectors_are_a_fixed_point(gb):
    """Eigenvectors already at working accuracy move only by their own error
    (u ||A|| / gap in the directions of close neighbours) and stay within the
    residual and orthogonality bounds."""
    n = 300
    lam0 = np.sort(np.random.default_rng(7).uniform(-2.0, 2.0, n))
    A = inputs.symmetric_with_spectrum(lam0, seed=8)
    w, V = np.linalg.eigh(A)
    (lam1, X1), = refine(gb, A, V, 1)
    gap = np.diff(lam0).min()
    assert np.abs(X1 - V).max() <= 100 * U * np.abs(lam0).max() / gap
    assert np.abs(lam1 - w).max() <= 1e-13 * np.abs(w).max()
    o, r = errors(A, X1, lam1)
    assert o <= 50 * n * U and r <= 50 * n * U


def test_refine_argument_errors(gb):
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert gb.gb_refine_syev_d(0, x, 1, x, x, 1, x, 1 << 20, None, check=False) == -1
    assert gb.gb_refine_syev_d(2, x, 1, x, x, 2, x, 1 << 20, None, check=False) == -3
    wsb = gb.gb_refine_syev_workspace_bytes(2)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert gb.gb_refine_syev_d(2, x, 2, x, x, 2, ws, wsb - 1, None, check=False) == -8


@pytest.mark.parametrize("eta", [1e-7, 1e-5])
def test_refine_from_perturbed_problem_with_tight_clusters(gb, eta):
    """Start from the exact eigenvectors of A + eta P (||P||_2 ~ 1), the
    state a low-precision solve with backward error eta leaves, on a
    spectrum with runs of 8 eigenvalues 1e-6 apart: the eigenvectors of a
    run are mixed at O(eta / 1e-6) and need the Rayleigh-Ritz treatment of
    clusters.  Three steps reach the residual and orthogonality bounds and
    the prescribed eigenvalues."""
    n = 640
    lam0 = inputs.gapped_uniform_spectrum(n, seed=31)
    A = inputs.symmetric_with_spectrum(lam0, seed=32)
    g = np.random.default_rng(33)
    P = g.standard_normal((n, n))
    P = (P + P.T) / np.sqrt(8 * n)
    _, X0 = np.linalg.eigh(A + eta * P)
    o0, r0 = errors(A, X0, np.linalg.eigvalsh(A + eta * P))
    assert r0 > 1e-9
    (l1, X1), (l2, X2), (l3, X3) = refine(gb, A, X0, 3)
    o, r = errors(A, X3, np.diag(X3.T @ A @ X3))
    assert o <= 50 * n * U and r <= 50 * n * U
    assert np.abs(np.sort(l3) - lam0).max() / np.abs(lam0).max() <= 1e-13


def test_refine_step_matches_the_oracle_step(gb):
    """One step of gb_refine_syev_d against the oracle's step
    (oracle/refine.py) from the same basis, on a spectrum with gaps near 2/n
    where no pair is clustered: X' element by element and lambda.  The two
    differ only by the rounding of the residual products (u sqrt(n) / gap
    in E), five orders below the correction itself."""
    from oracle.refine import ogita_aishima_step
    n = 512
    g = np.random.default_rng(51)
    lam0 = -1.0 + 2.0 * (np.arange(n) + 0.5 + 0.2 * g.uniform(-1, 1, n)) / n
    A = inputs.symmetric_with_spectrum(lam0, seed=52)
    _, V = np.linalg.eigh(A)
    X0 = V + 1e-6 * g.standard_normal((n, n)) / np.sqrt(n)
    X_or, l_or = ogita_aishima_step(A, X0)
    (l_gpu, X_gpu), = refine(gb, A, X0, 1)
    assert np.abs(X_or - X0).max() > 1e-8                  # the correction is real
    assert np.abs(X_gpu - X_or).max() <= 1e-11
    assert np.abs(l_gpu - l_or).max() <= 1e-14
