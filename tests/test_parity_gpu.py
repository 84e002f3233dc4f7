"""Parity of the CUDA back-transformation with the CPU oracle, through the C ABI.

Tolerance: the two sides apply the same reflectors in the same order per
column; they differ only in rounding (the kernel fuses multiply-adds).  The
map is deterministic and acts on each column alone, so it is compared
element by element: ||Z_gpu - Z_oracle||_F / ||Z_in||_F <= 1e-12 on the whole
block and on every column (measured ~5e-15).  On eigenvector inputs the GPU
result must also satisfy ||B Z - Z L||_F/||B||_F <= 50 n u and
||Z^H Z - I||_max <= 50 n u (u = 2^-53).
"""
import numpy as np
import pytest

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
PARITY = 1e-12   # ||Z_gpu - Z_oracle||_F / ||Z_in||_F, whole block and per column


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    build.build()
    m.load()
    return m


def run_gpu(gb, n, b, hv, ht, Z, opts=None):
    """Copy to the device, call the C entry point, copy back (column-major)."""
    cplx = np.iscomplexobj(Z)
    dev = torch.device("cuda")
    ldz, nev = Z.shape
    Zt = torch.from_numpy(np.ascontiguousarray(np.asfortranarray(Z).T)).to(dev)  # (nev, ldz) row-major
    hv_d = torch.from_numpy(np.ascontiguousarray(hv)).to(dev) if hv.size else torch.zeros(1, dtype=torch.float64, device=dev)
    ht_d = torch.from_numpy(np.ascontiguousarray(ht)).to(dev) if ht.size else torch.zeros(1, dtype=torch.float64, device=dev)
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, cplx, opts)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    f = gb.gb_trans_ev_tridi_to_band_z if cplx else gb.gb_trans_ev_tridi_to_band_d
    stream = torch.cuda.current_stream()
    f(n, b, nev, hv_d, ht_d, Zt, ldz, ws, wsb, stream, opts)
    torch.cuda.synchronize()
    return np.asfortranarray(Zt.cpu().numpy().T)


def rel_err(A, B, Zin):
    return np.linalg.norm(A - B) / max(np.linalg.norm(Zin), 1e-300)


def col_err(A, B, Zin):
    """max over columns of ||A_c - B_c|| / ||Zin_c|| (zero columns must match exactly)."""
    nz = np.linalg.norm(Zin, axis=0)
    d = np.linalg.norm(A - B, axis=0)
    assert np.all(d[nz == 0] == 0)
    return float(np.max(d[nz > 0] / nz[nz > 0])) if np.any(nz > 0) else 0.0


def assert_parity(out, ref, Z):
    assert rel_err(out, ref, Z) <= PARITY
    assert col_err(out, ref, Z) <= PARITY


VARIANTS = [
    None,
    {"variant": 1, "sweeps_per_tile": 4, "cols_per_block": 32},
    {"variant": 1, "sweeps_per_tile": 8, "cols_per_block": 64},
    {"variant": 1, "sweeps_per_tile": 16, "cols_per_block": 128},
]

SMALL = [(2, 1, 3), (3, 2, 1), (17, 3, 5), (40, 8, 33), (100, 7, 70), (257, 16, 129),
         (300, 64, 77), (129, 64, 200), (64, 64, 64), (65, 63, 31), (200, 33, 45), (150, 5, 1)]


@pytest.mark.parametrize("opts", VARIANTS, ids=["default", "nb4t32", "nb8t64", "nb16t128"])
@pytest.mark.parametrize("n,b,nev", SMALL)
def test_parity_bulge_chase_reflectors(gb, n, b, nev, opts):
    B = inputs.band_symmetric(n, b, seed=n + 17 * b)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    Z = inputs.z_gaussian(n, nev, seed=n + nev)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    out = run_gpu(gb, n, b, hv, ht, Z, opts)
    assert_parity(out, ref, Z)


@pytest.mark.parametrize("opts", VARIANTS, ids=["default", "nb4t32", "nb8t64", "nb16t128"])
@pytest.mark.parametrize("n,b,nev", [(513, 32, 300), (777, 64, 129), (1000, 13, 64)])
def test_parity_synthetic_reflectors(gb, n, b, nev, opts):
    hv, ht = inputs.synthetic_reflectors(n, b, seed=n * b)
    Z = inputs.z_gaussian(n, nev, seed=11)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    out = run_gpu(gb, n, b, hv, ht, Z, opts)
    assert_parity(out, ref, Z)


def test_parity_ldz_padding(gb):
    n, b, nev = 301, 24, 50
    hv, ht = inputs.synthetic_reflectors(n, b, seed=5)
    Z = inputs.z_gaussian(n, nev, seed=6, ldz=n + 13)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    out = run_gpu(gb, n, b, hv, ht, Z)
    assert_parity(out[:n], ref[:n], Z[:n])
    assert np.array_equal(out[n:], Z[n:])  # padding rows untouched


def test_identity_cases_exact(gb):
    # b = 1 and tridiagonal input: every tau is 0, the map is the identity
    n, nev = 90, 40
    for b, B in [(1, inputs.band_symmetric(n, 1, seed=3)), (6, inputs.toeplitz_band(n, 6))]:
        d, e, hv, ht, _ = oracle.bulge_chase(B, b)
        assert np.all(ht == 0)
        Z = inputs.z_gaussian(n, nev, seed=4)
        assert np.array_equal(run_gpu(gb, n, b, hv, ht, Z), Z)


def test_noop_cases(gb):
    dev = torch.device("cuda")
    Z = torch.ones((3, 1), dtype=torch.float64, device=dev)
    assert gb.gb_trans_ev_tridi_to_band_d(1, 4, 3, None, None, Z, 1) == 0
    assert torch.all(Z == 1)
    assert gb.gb_trans_ev_tridi_to_band_d(50, 4, 0, Z, Z, None, 50) == 0


@pytest.fixture(scope="module")
def config1():
    """n = 1024, all eigenpairs, nbw = 32, A = (B + B^T)/2 with U[-1,1] band entries."""
    n, b = 1024, 32
    B = inputs.band_symmetric(n, b, seed=1)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    return n, b, B, hv, ht, w, V


@pytest.mark.parametrize("opts", VARIANTS, ids=["default", "nb4t32", "nb8t64", "nb16t128"])
def test_config1_eigenvectors(gb, config1, opts):
    n, b, B, hv, ht, w, V = config1
    ref = oracle.trans_ev(n, b, hv, ht, V)
    out = run_gpu(gb, n, b, hv, ht, V, opts)
    assert_parity(out, ref, V)
    assert np.linalg.norm(B @ out - out * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.T @ out - np.eye(n)).max() <= 50 * n * U


def test_full_size_sampled_columns(gb):
    """n = 16384, nev = 4096, nbw = 64 in the default launch configuration
    (the bench's inputs and call); 64 seeded columns checked against the
    oracle element by element (columns are independent, so a subset is an
    exact check), every column checked for norm preservation (Q2 is
    orthogonal)."""
    n, b, nev = 16384, 64, 4096
    hv, ht = inputs.synthetic_reflectors(n, b, seed=2024)
    Z = inputs.z_gaussian(n, nev, seed=2025)
    out = run_gpu(gb, n, b, hv, ht, Z)
    cols = np.sort(np.random.default_rng(7).choice(nev, 64, replace=False))
    ref = oracle.trans_ev(n, b, hv, ht, np.asfortranarray(Z[:, cols]))
    assert_parity(out[:, cols], ref, Z[:, cols])
    nin = np.linalg.norm(Z, axis=0)
    nout = np.linalg.norm(out, axis=0)
    assert np.abs(nout / nin - 1.0).max() <= 50 * n * U
