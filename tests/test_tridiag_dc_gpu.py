"""Divide-and-conquer tridiagonal eigensolver (gb_tridiag_dc_d) through the C
ABI, against the oracle's implicit QL (eigenvalues), closed forms (Toeplitz
(2, -1)) and the eigen-relations (residual, orthogonality within 50 n u), on
the cases that exercise each of its steps: one leaf, several levels of
merges, heavy deflation (glued Wilkinson matrices, zero couplings, an
identity, tight clusters), graded entries, and the solver's all-pairs path."""
import numpy as np
import pytest

import oracle
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


def dc(gb, d, e):
    n = len(d)
    dev = torch.device("cuda")
    d_d = torch.from_numpy(np.ascontiguousarray(d, dtype=np.float64)).to(dev)
    e_d = torch.from_numpy(np.ascontiguousarray(e if n > 1 else np.zeros(1), dtype=np.float64)).to(dev)
    lam = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    Q = torch.full((n, n), np.nan, dtype=torch.float64, device=dev)   # row-major n x n = column-major Q^T
    wsb = gb.gb_tridiag_dc_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    gb.gb_tridiag_dc_d(n, d_d, e_d, lam, Q, n, ws, wsb, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(d_d.cpu().numpy(), d)            # inputs untouched
    return lam.cpu().numpy(), Q.cpu().numpy().T


def check(d, e, lam, Q, ref=None):
    n = len(d)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = max(np.linalg.norm(T, 2), np.finfo(float).tiny)
    if ref is None:
        ref = np.sort(oracle.tridiag_ql(d, e)[0])
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - ref).max() / nrm <= 1e-13
    assert np.linalg.norm(T @ Q - Q * lam) / max(np.linalg.norm(T), np.finfo(float).tiny) <= 50 * n * U
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 50 * n * U


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 100, 129, 257, 300, 640, 1000, 2048])
def test_dc_random(gb, n):
    g = np.random.default_rng(n)
    d, e = g.standard_normal(n), g.standard_normal(n - 1)
    lam, Q = dc(gb, d, e)
    check(d, e, lam, Q)


def test_dc_toeplitz_closed_form(gb):
    """(2, -1): lambda_k = 2 - 2 cos(k pi / (n + 1)), eigenvectors
    sqrt(2 / (n + 1)) sin(j k pi / (n + 1)) up to sign."""
    n = 515
    d, e = 2.0 * np.ones(n), -np.ones(n - 1)
    lam, Q = dc(gb, d, e)
    k = np.arange(1, n + 1)
    ref = 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))
    check(d, e, lam, Q, ref=ref)
    V = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(k, k) * np.pi / (n + 1))
    assert np.abs(np.abs(np.sum(V * Q, axis=0)) - 1.0).max() <= 1e-10


@pytest.mark.parametrize("glue", [1e-10, 1e-14, 0.0])
def test_dc_glued_wilkinson(gb, glue):
    """Copies of W21+ glued by tiny couplings: nearly every eigenvalue comes
    in close pairs or clusters, so most components deflate."""
    w = np.abs(np.arange(-10, 11)).astype(float)
    reps = 40
    d = np.tile(w, reps)
    e = np.ones(len(d) - 1)
    e[21 * np.arange(1, reps) - 1] = glue
    lam, Q = dc(gb, d, e)
    check(d, e, lam, Q)


def test_dc_deflation_extremes(gb):
    g = np.random.default_rng(4)
    n = 700
    cases = [
        (np.ones(n), np.zeros(n - 1)),                                            # identity: all deflate
        (g.standard_normal(n), np.where(g.random(n - 1) < 0.3, 0.0, g.standard_normal(n - 1))),
        (np.round(g.standard_normal(n) * 2) / 2, 1e-9 * g.standard_normal(n - 1)),  # tight clusters
        (np.logspace(-12, 0, n), 0.5 * np.logspace(-12, 0, n - 1)),                # graded
        (1.0 + 1e-13 * np.arange(n), 1e-14 * np.ones(n - 1)),                       # near-multiple
        (np.zeros(n), np.zeros(n - 1)),                                           # zero matrix
        (1e150 * g.standard_normal(n), 1e150 * g.standard_normal(n - 1)),           # large scale
    ]
    for d, e in cases:
        lam, Q = dc(gb, d, e)
        check(d, e, lam, Q)


def test_dc_argument_errors(gb):
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert gb.gb_tridiag_dc_d(0, x, x, x, x, 1, x, 1 << 20, None, check=False) == -1
    assert gb.gb_tridiag_dc_d(4, x, x, x, x, 3, x, 1 << 20, None, check=False) == -6
    wsb = gb.gb_tridiag_dc_workspace_bytes(4)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert gb.gb_tridiag_dc_d(4, x, x, x, x, 4, ws, wsb - 1, None, check=False) == -8


def test_solver_all_pairs_dc_against_bisection(gb):
    """The two-stage solver takes divide and conquer when 2 nev > n; with
    GB_SOLVE_TRIDIAG_BISECT it takes bisection + inverse iteration.  Both meet
    the prescribed spectrum and the residual/orthogonality bounds."""
    n, nev, nbw = 900, 900, 32
    lam0 = inputs.clustered_spectrum(n, seed=21)
    A = inputs.symmetric_with_spectrum(lam0, seed=22)
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    wsb = gb.gb_solve_workspace_bytes(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    nrm = np.linalg.norm(A, 2)
    for flags in (0, gb.GB_SOLVE_TRIDIAG_BISECT):
        ev = torch.zeros(nev, dtype=torch.float64, device=dev)
        Z = torch.zeros((nev, n), dtype=torch.float64, device=dev)
        gb.gb_solve_d(n, nev, nbw, A_d, n, ev, Z, n, ws, wsb, st, flags)
        assert gb.gb_solve_query(ws, n, nev, nbw, st) == 0
        w, Zh = ev.cpu().numpy(), Z.cpu().numpy().T
        assert np.abs(w - np.sort(lam0)).max() / nrm <= 1e-11
        assert np.linalg.norm(A @ Zh - Zh * w) / np.linalg.norm(A) <= 50 * n * U
        assert np.abs(Zh.T @ Zh - np.eye(nev)).max() <= 50 * n * U
