"""Complex Hermitian back-transformation (the tcgen05 pipeline on the real
2 x 2-block form -- the default for nbw in {16, 32, 64} and n >= 512 -- and
the shared-memory wavefront kernel) and real band widths above 64, against
the oracle, through the C ABI.

Parity: ||Z_gpu - Z_oracle||_F / ||Z_in||_F <= 1e-12 on the whole block and
on every column (the map is deterministic and column-wise)."""
import numpy as np
import pytest

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
PARITY = 1e-12


def assert_parity(out, ref, Z):
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= PARITY
    nz = np.linalg.norm(Z, axis=0)
    assert np.max(np.linalg.norm(out - ref, axis=0) / nz) <= PARITY


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    build.build()
    m.load()
    return m


def run(gb, n, b, hv, ht, Z, opts=None, status=0):
    dev = torch.device("cuda")
    cplx = np.iscomplexobj(Z)
    ldz, nev = Z.shape
    Zt = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    hv_d = torch.from_numpy(np.ascontiguousarray(hv)).to(dev)
    ht_d = torch.from_numpy(np.ascontiguousarray(ht)).to(dev)
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, cplx, opts)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    f = gb.gb_trans_ev_tridi_to_band_z if cplx else gb.gb_trans_ev_tridi_to_band_d
    f(n, b, nev, hv_d, ht_d, Zt, ldz, ws, wsb, st, opts)
    assert gb.gb_trans_ev_query(ws if wsb else None, wsb, st) == status
    return np.asfortranarray(Zt.cpu().numpy().T)


TC5 = {"variant": 4}


@pytest.mark.parametrize("n,b,nev", [(2, 16, 3), (3, 16, 2), (17, 16, 5), (60, 16, 33), (129, 32, 70),
                                     (200, 64, 65), (300, 64, 129), (250, 32, 257)])
def test_complex_tc5_parity_bulge_chase(gb, n, b, nev):
    """tcgen05 on the reflectors of the oracle's Hermitian bulge chase
    (length-1 reflectors with complex tau included), every column."""
    assert gb.gb_trans_ev_variant(n, b, nev, 1, TC5) == gb.GB_VARIANT_PIPELINE_TC5
    B = inputs.band_symmetric(n, b, seed=n + 3 * b, cplx=True)
    _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    Z = inputs.z_gaussian(n, nev, seed=nev + 1, cplx=True)
    out = run(gb, n, b, hv, ht, Z, TC5)
    assert_parity(out, oracle.trans_ev(n, b, hv, ht, Z), Z)


@pytest.mark.parametrize("n,b,nev", [(700, 64, 1), (1000, 16, 200), (1500, 32, 130), (2049, 64, 257)])
def test_complex_tc5_parity_synthetic(gb, n, b, nev):
    hv, ht = inputs.synthetic_reflectors(n, b, seed=n + b, cplx=True)
    Z = inputs.z_gaussian(n, nev, seed=n, cplx=True)
    assert gb.gb_trans_ev_variant(n, b, nev, 1) == gb.GB_VARIANT_PIPELINE_TC5     # the default here
    out = run(gb, n, b, hv, ht, Z)
    assert_parity(out, oracle.trans_ev(n, b, hv, ht, Z), Z)


def test_complex_tc5_eigenvectors_and_norms(gb):
    """Eigenvectors of a Hermitian band matrix (oracle chase + QL) through
    tcgen05: residual and orthogonality; columns of norms 1e-200 .. 1e200
    and a zero column keep their own relative accuracy."""
    n, b = 600, 64
    B = inputs.band_symmetric(n, b, seed=61, cplx=True)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    Z = np.asfortranarray(V[:, :150].astype(np.complex128))
    out = run(gb, n, b, hv, ht, Z)
    assert_parity(out, oracle.trans_ev(n, b, hv, ht, Z), Z)
    assert np.linalg.norm(B @ out - out * w[:150]) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.conj().T @ out - np.eye(150)).max() <= 50 * n * U
    Z2 = inputs.z_gaussian(n, 6, seed=62, cplx=True)
    Z2[:, 0] *= 1e-200
    Z2[:, 1] *= 1e200
    Z2[:, 2] = 0.0
    out2 = run(gb, n, b, hv, ht, Z2)
    ref2 = oracle.trans_ev(n, b, hv, ht, Z2)
    assert np.all(out2[:, 2] == 0)
    for c in (0, 1, 3, 4, 5):
        sc = np.abs(Z2[:, c]).max()
        assert np.linalg.norm((out2[:, c] - ref2[:, c]) / sc) / np.linalg.norm(Z2[:, c] / sc) <= PARITY


def test_complex_tc5_nonfinite_and_schedule(gb):
    """A NaN column comes back as NaN with GB_ERR_NONFINITE; the other
    columns are exact; the column batch does not change a single bit."""
    n, b, nev = 900, 32, 300
    hv, ht = inputs.synthetic_reflectors(n, b, seed=63, cplx=True)
    Z = inputs.z_gaussian(n, nev, seed=64, cplx=True)
    out0 = run(gb, n, b, hv, ht, Z)
    out1 = run(gb, n, b, hv, ht, Z, dict(TC5, column_batch=1))
    assert np.array_equal(out0, out1)
    Zb = Z.copy()
    Zb[5, 7] = np.nan + 1j
    outb = run(gb, n, b, hv, ht, Zb, status=gb.GB_ERR_NONFINITE)
    assert np.all(np.isnan(outb[:, 7]))
    keep = [c for c in range(nev) if c != 7]
    assert np.array_equal(outb[:, keep], out0[:, keep])


ZOPTS = [None, {"sweeps_per_tile": 4, "cols_per_block": 32}, {"sweeps_per_tile": 16, "cols_per_block": 64}]


@pytest.mark.parametrize("opts", ZOPTS, ids=["default", "nb4t32", "nb16t64"])
@pytest.mark.parametrize("n,b,nev", [(2, 1, 2), (3, 2, 3), (17, 3, 5), (60, 8, 33), (129, 16, 70),
                                     (200, 64, 65), (150, 37, 31)])
def test_complex_parity_bulge_chase(gb, n, b, nev, opts):
    B = inputs.band_symmetric(n, b, seed=n + b, cplx=True)
    _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    Z = inputs.z_gaussian(n, nev, seed=nev, cplx=True)
    out = run(gb, n, b, hv, ht, Z, opts)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert_parity(out, ref, Z)


def test_complex_eigenvectors_residual(gb):
    n, b = 384, 32
    B = inputs.band_symmetric(n, b, seed=77, cplx=True)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    Z = np.asfortranarray(V.astype(np.complex128))
    out = run(gb, n, b, hv, ht, Z)
    assert np.linalg.norm(B @ out - out * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.conj().T @ out - np.eye(n)).max() <= 50 * n * U


def test_complex_config_size_sampled(gb):
    """complex128 Hermitian n = 8192, nev = 2048 (25%), nbw = 64; 64 seeded
    columns against the oracle element by element, all columns for norm
    preservation."""
    n, b, nev = 8192, 64, 2048
    hv, ht = inputs.synthetic_reflectors(n, b, seed=81, cplx=True)
    Z = inputs.z_gaussian(n, nev, seed=82, cplx=True)
    out = run(gb, n, b, hv, ht, Z)
    cols = np.sort(np.random.default_rng(3).choice(nev, 64, replace=False))
    ref = oracle.trans_ev(n, b, hv, ht, np.asfortranarray(Z[:, cols]))
    assert_parity(out[:, cols], ref, Z[:, cols])
    nr = np.linalg.norm(out, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.abs(nr - 1).max() <= 50 * n * U


@pytest.mark.parametrize("n,b,nev", [(300, 65, 40), (400, 100, 33), (600, 128, 70), (520, 256, 20)])
def test_real_wide_band_parity(gb, n, b, nev):
    if n <= 400:
        B = inputs.band_symmetric(n, b, seed=n)
        _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    else:
        hv, ht = inputs.synthetic_reflectors(n, b, seed=n)
    Z = inputs.z_gaussian(n, nev, seed=5)
    out = run(gb, n, b, hv, ht, Z)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert_parity(out, ref, Z)
