"""Complex Hermitian two-stage solve (gb_solve_z) on matrices with a
prescribed spectrum, A = Q diag(lam) Q^H (Q Haar unitary): eigenvalues
within 1e-11 ||A||_2 of lam (LAPACK's eigvalsh only as a secondary check),
residual ||A Z - Z L||_F / ||A||_F and orthogonality ||Z^H Z - I||_max
within 50 n u."""
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


def solve_z(gb, A, nev, nbw, flags=0):
    n = A.shape[0]
    dev = torch.device("cuda")
    A_d = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
    ev = torch.zeros(nev, dtype=torch.float64, device=dev)
    Z = torch.zeros((nev, n), dtype=torch.complex128, device=dev)
    wsb = gb.gb_solve_workspace_bytes_z(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_solve_z(n, nev, nbw, A_d, n, ev, Z, n, ws, wsb, st, flags)
    assert gb.gb_solve_query_z(ws, n, nev, nbw, st) == 0
    return ev.cpu().numpy(), Z.cpu().numpy().T


def check(A, w, Z, nev, lam):
    n = A.shape[0]
    nrm = np.linalg.norm(A, 2)
    assert np.abs(w - lam[:nev]).max() / nrm <= 1e-11
    assert np.abs(w - np.linalg.eigvalsh(A)[:nev]).max() / nrm <= 1e-11   # secondary (LAPACK)
    assert np.linalg.norm(A @ Z - Z * w) / np.linalg.norm(A) <= 50 * n * U
    assert np.abs(Z.conj().T @ Z - np.eye(nev)).max() <= 50 * n * U


@pytest.mark.parametrize("n,nev,nbw", [(2, 2, 1), (5, 3, 2), (64, 64, 8), (150, 40, 16), (300, 75, 32), (400, 100, 64)])
def test_solve_hermitian_prescribed(gb, n, nev, nbw):
    """Spectrum uniform in [-1, 1] (n >= 64) or a few fixed values."""
    lam = np.sort(np.random.default_rng(n + 7).uniform(-1.0, 1.0, n)) if n >= 64 else \
        np.array([-1.0, 0.25, 0.5, 2.0, 3.0])[:n]
    A = inputs.symmetric_with_spectrum(lam, seed=n + 7, cplx=True)
    w, Z = solve_z(gb, A, nev, nbw)
    check(A, w, Z, nev, lam)


def test_solve_hermitian_clustered(gb):
    n, nev = 384, 120
    lam = inputs.clustered_spectrum(n, seed=11)
    A = inputs.symmetric_with_spectrum(lam, seed=12, cplx=True)
    w, Z = solve_z(gb, A, nev, 32)
    check(A, w, Z, nev, lam)


@pytest.mark.parametrize("flags", [0, 4], ids=["sliced_products", "dfma_products"])
def test_solve_hermitian_large_products_both_paths(gb, flags):
    """n = 1200: the complex solve's large products (ZHEMM, ZHER2K, the
    band->full products, the real Newton-Schulz step) take the sliced
    tensor-core path by default and this library's complex DFMA kernel with
    GB_SOLVE_DFMA_PRODUCTS (as do the b x b panel products on either path);
    both meet the bounds."""
    n, nev = 1200, 300
    lam = inputs.clustered_spectrum(n, seed=31)
    A = inputs.symmetric_with_spectrum(lam, seed=32, cplx=True)
    w, Z = solve_z(gb, A, nev, 64, flags)
    check(A, w, Z, nev, lam)
