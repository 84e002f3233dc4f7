"""Mixed-precision solve (gb_solve_mixed_d): the two-stage solver for all
eigenpairs with FP32 products in full -> band and band -> full
(GB_SOLVE_FP32_PRODUCTS), then Ogita-Aishima refinement steps in FP64.
Checked against prescribed spectra A = Q diag(lambda) Q^T (eigenvalues known
exactly) and the residual / orthogonality bounds: the low-precision half is
measurably FP32-accurate (so the flag reaches the products), and the refined
result meets the FP64 bounds, tight clusters (runs 1e-6 apart) included."""
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


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda")


def direct(gb, A, nev, nbw, flags):
    n = A.shape[0]
    A_d = to_dev(A)
    ev = torch.zeros(nev, dtype=torch.float64, device="cuda")
    Z = torch.zeros((nev, n), dtype=torch.float64, device="cuda")
    wsb = gb.gb_solve_workspace_bytes(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    gb.gb_solve_d(n, nev, nbw, A_d, n, ev, Z, n, ws, wsb, st, flags)
    assert gb.gb_solve_query(ws, n, nev, nbw, st) == 0
    return ev.cpu().numpy(), Z.cpu().numpy().T


def mixed(gb, A, nev, nbw, steps):
    n = A.shape[0]
    A_d = to_dev(A)
    ev = torch.full((nev,), np.nan, dtype=torch.float64, device="cuda")
    Z = torch.full((nev, n), np.nan, dtype=torch.float64, device="cuda")
    wsb = gb.gb_solve_mixed_workspace_bytes(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    gb.gb_solve_mixed_d(n, nev, nbw, A_d, n, ev, Z, n, steps, ws, wsb, st)
    assert gb.gb_solve_mixed_query(ws, n, nev, nbw, st) == 0
    return ev.cpu().numpy(), Z.cpu().numpy().T


def errs(A, w, Z, lam):
    nev = len(w)
    dlam = np.abs(w - lam[:nev]).max() / np.abs(lam).max()
    res = np.linalg.norm(A @ Z - Z * w) / np.linalg.norm(A)
    orth = np.abs(Z.T @ Z - np.eye(nev)).max()
    return dlam, res, orth


def test_fp32_products_flag_gives_fp32_class_accuracy(gb):
    """n = 2048 (large enough for the sliced products): with
    GB_SOLVE_FP32_PRODUCTS the residual sits between the FP64 bound and the
    FP32 level; without it the FP64 bounds hold."""
    assert gb.GB_SOLVE_FP32_PRODUCTS == 16
    n, nev = 2048, 256
    lam = np.sort(np.random.default_rng(40).uniform(-1.0, 1.0, n))
    A = inputs.symmetric_with_spectrum(lam, seed=41)
    d64, r64, o64 = errs(A, *direct(gb, A, nev, 64, 0), lam)
    d32, r32, o32 = errs(A, *direct(gb, A, nev, 64, gb.GB_SOLVE_FP32_PRODUCTS), lam)
    assert r64 <= 50 * n * U and o64 <= 50 * n * U
    assert 1e3 * r64 < r32 <= 1e-5
    assert d32 <= 1e-5 and o32 <= 1e-5


@pytest.mark.parametrize("nev", [512, 2048])
def test_mixed_solve_refines_to_fp64(gb, nev):
    n = 2048
    lam = np.sort(np.random.default_rng(42).uniform(-1.0, 1.0, n))
    A = inputs.symmetric_with_spectrum(lam, seed=43)
    d0, r0, o0 = errs(A, *mixed(gb, A, nev, 64, 0), lam)
    assert r0 > 1e-11                                   # the low-precision half alone is not FP64
    d, r, o = errs(A, *mixed(gb, A, nev, 64, 3), lam)
    assert d <= 1e-11 and r <= 50 * n * U and o <= 50 * n * U


def test_mixed_solve_tight_clusters(gb):
    """Eigenvalues uniform in [-1, 1] with 10% in runs of 8 spaced 1e-6 (the
    mixed-precision workload's spectrum, at n = 2048)."""
    n, nev = 2048, 1024
    lam = inputs.gapped_uniform_spectrum(n, seed=44)
    A = inputs.symmetric_with_spectrum(lam, seed=45)
    d, r, o = errs(A, *mixed(gb, A, nev, 64, 3), lam)
    assert d <= 1e-11 and r <= 50 * n * U and o <= 50 * n * U


def test_mixed_solve_small_problem_takes_fp64_products(gb):
    """Below the sliced products' size threshold every product is an FP64
    DFMA product, so even zero refinement steps give FP64 results."""
    n, nev = 300, 100
    lam = np.sort(np.random.default_rng(46).uniform(-1.0, 1.0, n))
    A = inputs.symmetric_with_spectrum(lam, seed=47)
    d, r, o = errs(A, *mixed(gb, A, nev, 32, 0), lam)
    assert d <= 1e-11 and r <= 50 * n * U and o <= 50 * n * U


def test_mixed_argument_errors(gb):
    f = gb.gb_solve_mixed_d
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert f(1, 1, 1, x, 1, x, x, 1, 1, x, 1 << 30, check=False) == -1
    assert f(10, 11, 3, x, 10, x, x, 10, 1, x, 1 << 30, check=False) == -2
    assert f(10, 5, 3, x, 10, x, x, 10, gb.GB_SOLVE_MIXED_MAX_STEPS + 1, x, 1 << 30, check=False) == -9
    wsb = gb.gb_solve_mixed_workspace_bytes(10, 5, 3)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert f(10, 5, 3, x, 10, x, x, 10, 1, ws, wsb - 1, check=False) == -11
