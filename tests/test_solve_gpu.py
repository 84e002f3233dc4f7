"""Two-stage eigensolver on the GPU (gb_solve_d / elpa_b200_solve).

Expected eigenvalues come from the oracle (its one-stage Householder
tridiagonalisation + implicit QL, up to n = 1024) or from a prescribed
spectrum (A = Q diag(lam) Q^T, closed form); LAPACK's eigvalsh is only a
secondary check.  Bounds: eigenvalues within 1e-11 ||A||_2, residual
||A Z - Z L||_F / ||A||_F and orthogonality ||Z^T Z - I||_max within 50 n u."""
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


def solve_gpu(gb, A, nev, nbw, flags=0):
    n = A.shape[0]
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    ev = torch.zeros(nev, dtype=torch.float64, device=dev)
    Z = torch.zeros((nev, n), dtype=torch.float64, device=dev)
    wsb = gb.gb_solve_workspace_bytes(n, nev, nbw)
    assert wsb > 0
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_solve_d(n, nev, nbw, A_d, n, ev, Z, n, ws, wsb, st, flags)
    assert gb.gb_solve_query(ws, n, nev, nbw, st) == 0
    return ev.cpu().numpy(), Z.cpu().numpy().T


def oracle_eigenvalues(A):
    """All eigenvalues of A, ascending, from the oracle (sytrd + QL)."""
    d, e, _, _ = oracle.sytrd(A)
    w, _ = oracle.tridiag_ql(d, e)
    return np.sort(w)


def check(A, w, Z, nev, lam):
    """lam: the expected nev lowest eigenvalues (oracle or prescribed)."""
    n = A.shape[0]
    nrm = np.linalg.norm(A, 2)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - lam[:nev]).max() / nrm <= 1e-11
    assert np.abs(w - np.linalg.eigvalsh(A)[:nev]).max() / nrm <= 1e-11   # secondary (LAPACK)
    assert np.linalg.norm(A @ Z - Z * w) / np.linalg.norm(A) <= 50 * n * U
    assert np.abs(Z.T @ Z - np.eye(nev)).max() <= 50 * n * U


@pytest.mark.parametrize("n,nev,nbw", [(2, 2, 1), (3, 1, 2), (64, 64, 8), (100, 25, 16), (257, 64, 32),
                                       (300, 300, 64), (513, 128, 64), (600, 150, 13)])
def test_solve_random_symmetric(gb, n, nev, nbw):
    A = inputs.band_symmetric(n, n, seed=n + nev)
    w, Z = solve_gpu(gb, A, nev, nbw)
    check(A, w, Z, nev, oracle_eigenvalues(A))


def test_solve_config_n1024_all_pairs(gb):
    """n = 1024, all eigenpairs, nbw = 32, A = (B + B^T)/2 with U[-1,1] entries."""
    n = 1024
    A = inputs.band_symmetric(n, n, seed=1)
    w, Z = solve_gpu(gb, A, n, 32)
    check(A, w, Z, n, oracle_eigenvalues(A))


def test_solve_clustered_spectrum(gb):
    """Prescribed spectrum with 10% of the eigenvalues in clusters of 8 of
    width 1e-8: eigenvalues to 1e-11 ||A||, residual and orthogonality."""
    n, nev = 512, 160
    lam = inputs.clustered_spectrum(n, seed=5)
    A = inputs.symmetric_with_spectrum(lam, seed=6)
    w, Z = solve_gpu(gb, A, nev, 32)
    assert np.abs(w - lam[:nev]).max() / np.abs(lam).max() <= 1e-11
    check(A, w, Z, nev, lam)


@pytest.mark.parametrize("flags", [0, 4], ids=["sliced_products", "dfma_products"])
def test_solve_large_products_both_paths(gb, flags):
    """n = 2048 (large enough that the solve's big products take the sliced
    tensor-core path by default): both product paths meet the bounds, and
    their eigenvalues agree with LAPACK to 1e-11 ||A||."""
    assert gb.GB_SOLVE_DFMA_PRODUCTS == 4
    n, nev = 2048, 512
    lam = inputs.clustered_spectrum(n, seed=21)
    A = inputs.symmetric_with_spectrum(lam, seed=22)
    w, Z = solve_gpu(gb, A, nev, 64, flags)
    assert np.abs(w - lam[:nev]).max() / np.abs(lam).max() <= 1e-11
    check(A, w, Z, nev, lam)


def test_solve_toeplitz_closed_form(gb):
    n, nev = 200, 50
    A = inputs.toeplitz_band(n, 1)
    w, Z = solve_gpu(gb, A, nev, 8)
    k = np.arange(1, n + 1)
    lam = np.sort(2 - 2 * np.cos(k * np.pi / (n + 1)))[:nev]
    assert np.abs(w - lam).max() <= 50 * n * U * 4
    check(A, w, Z, nev, lam)


def test_elpa_b200_solve_convenience(gb):
    n, nev = 300, 75
    A = inputs.band_symmetric(n, n, seed=9)
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    ev = torch.zeros(nev, dtype=torch.float64, device=dev)
    Z = torch.zeros((nev, n), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    gb.elpa_b200_solve(n, nev, A_d, n, ev, Z, n)
    check(A, ev.cpu().numpy(), Z.cpu().numpy().T, nev, oracle_eigenvalues(A))


def test_solve_argument_errors(gb):
    f = gb.gb_solve_d
    assert f(1, 1, 1, 256, 1, 256, 256, 1, 256, 1 << 30, check=False) == -1
    assert f(10, 11, 3, 256, 10, 256, 256, 10, 256, 1 << 30, check=False) == -2
    assert f(10, 5, 10, 256, 10, 256, 256, 10, 256, 1 << 30, check=False) == -3
    assert f(10, 5, 3, 256, 9, 256, 256, 10, 256, 1 << 30, check=False) == -5
    assert f(10, 5, 3, 256, 10, 256, 256, 10, 256, 16, check=False) == -10


def test_solve_release_frees_and_recreates_stream_resources(gb):
    """gb_solve_release drops the per-stream resources a solve cached (the
    look-ahead helper stream of n >= 4096, the stage events); a later solve
    on the same stream creates them again and is still correct."""
    n, nev = 4096, 256
    lam = inputs.clustered_spectrum(n, seed=41)
    A = inputs.symmetric_with_spectrum(lam, seed=42)
    st = torch.cuda.Stream()
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    wsb = gb.gb_solve_workspace_bytes(n, nev, 64)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    for rep in range(2):
        ev = torch.zeros(nev, dtype=torch.float64, device=dev)
        Z = torch.zeros((nev, n), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        gb.gb_solve_d(n, nev, 64, A_d, n, ev, Z, n, ws, wsb, st, gb.GB_SOLVE_RECORD_STAGES)
        assert gb.gb_solve_query(ws, n, nev, 64, st) == 0
        assert all(t >= 0 for t in gb.gb_solve_stage_ms(st).values())
        w = ev.cpu().numpy()
        assert np.abs(w - lam[:nev]).max() / np.abs(lam).max() <= 1e-11
        assert gb.gb_solve_release(st, 0) == gb.GB_OK
    assert gb.gb_solve_release(None, 1) == gb.GB_OK       # every stream, every device
