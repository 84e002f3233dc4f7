"""The tensor-core pipeline (GB_VARIANT_PIPELINE_TC: tiles in compact WY form
on mma.sync bf16 by exact digit slicing, Z in per-column 64-bit fixed point)
through the C ABI, against the oracle: every supported band width, ragged
and tiny shapes, columns of wildly different norms (each column carries its
own scale), eigenvector inputs (residual and orthogonality), bit-identity
across schedules, and the bounded dependency wait."""
import numpy as np
import pytest

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
TC = {"variant": 3}


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01277_gb300 as m
    from paper_1811_01277_gb300 import build
    build.build()
    m.load()
    return m


def run(gb, n, b, hv, ht, Z, opts):
    dev = torch.device("cuda")
    ldz, nev = Z.shape
    Zt = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    hv_d = torch.from_numpy(hv).to(dev)
    ht_d = torch.from_numpy(ht).to(dev)
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, opts)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    rc = gb.gb_trans_ev_tridi_to_band_d(n, b, nev, hv_d, ht_d, Zt, ldz, ws, wsb, st, opts, check=False)
    q = gb.gb_trans_ev_query(ws if wsb else None, wsb, st)
    return rc, q, np.asfortranarray(Zt.cpu().numpy().T)


def colwise_err(out, ref, Z):
    """max over columns of ||out_c - ref_c|| / ||z_c||, each column scaled
    by its largest entry first so that norms of huge columns do not overflow."""
    s = np.abs(Z).max(axis=0)
    s[s == 0] = 1.0
    nz = np.linalg.norm(Z / s, axis=0)
    nz[nz == 0] = 1.0
    return np.max(np.linalg.norm((out - ref) / s, axis=0) / nz)


@pytest.mark.parametrize("n,b,nev", [(2, 16, 3), (17, 16, 1), (100, 16, 65), (257, 16, 129), (300, 32, 200),
                                     (129, 64, 130), (640, 64, 257), (1000, 64, 64), (65, 64, 31),
                                     (1500, 32, 100), (2049, 64, 70), (4096, 64, 96)])
def test_tc_parity(gb, n, b, nev):
    if n <= 400:
        B = inputs.band_symmetric(n, b, seed=n + b)
        _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    else:
        hv, ht = inputs.synthetic_reflectors(n, b, seed=n)
    Z = inputs.z_gaussian(n, nev, seed=nev)
    assert gb.gb_trans_ev_launch_count(n, b, nev, 0, TC) == (6 if n > 1 else 0)
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 50 * n * U
    assert colwise_err(out, ref, Z) <= 50 * n * U


def test_tc_columns_of_different_norms(gb):
    """Column scales 1e-200 .. 1e200, a zero column and a column with one
    dominant entry: each column is accurate relative to its own norm."""
    n, b, nev = 500, 64, 9
    hv, ht = inputs.synthetic_reflectors(n, b, seed=77)
    Z = inputs.z_gaussian(n, nev, seed=78)
    Z[:, 0] *= 1e-200
    Z[:, 1] *= 1e200
    Z[:, 2] = 0.0
    Z[:, 3] = 0.0
    Z[7, 3] = 3.0
    Z[:, 4] *= 2.0 ** 500
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.all(out[:, 2] == 0.0)
    assert colwise_err(out, ref, Z) <= 50 * n * U


def test_tc_columns_at_the_fixed_point_edge(gb):
    """Columns whose one entry holds the whole norm and sits just below a
    power of two (the tightest column scale), and columns of identity: each
    stays within 50 n u of the oracle and keeps its norm."""
    n, b, nev = 700, 64, 12
    hv, ht = inputs.synthetic_reflectors(n, b, seed=41)
    Z = np.zeros((n, nev), order="F")
    below = np.nextafter(1.0, 0.0)                      # 1 - 2^-53
    for c in range(nev):
        Z[(37 * c + 5) % n, c] = below * (2.0 ** (c - 6)) * (-1) ** c
    Z[:, 11] = 0.0
    Z[0, 11] = 1.0
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert colwise_err(out, ref, Z) <= 50 * n * U
    assert np.abs(np.linalg.norm(out, axis=0) / np.linalg.norm(Z, axis=0) - 1.0).max() <= 50 * n * U


def test_tc_eigenvectors_residual(gb):
    """Z_in = tridiagonal eigenvectors from the oracle's chase + QL: the
    output satisfies B Z = Z Lambda and Z^T Z = I to 50 n u."""
    n, b = 400, 32
    B = inputs.band_symmetric(n, b, seed=5)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    Z = np.asfortranarray(V[:, :200])
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    assert np.linalg.norm(B @ out - out * w[:200]) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.T @ out - np.eye(200)).max() <= 50 * n * U


@pytest.mark.parametrize("cb", [1, 3, 1024])
def test_tc_schedule_bit_identical(gb, cb):
    n, b, nev = 900, 64, 300
    hv, ht = inputs.synthetic_reflectors(n, b, seed=31)
    Z = inputs.z_gaussian(n, nev, seed=32)
    rc0, q0, out0 = run(gb, n, b, hv, ht, Z, TC)
    rc, q, out = run(gb, n, b, hv, ht, Z, dict(TC, column_batch=cb))
    assert rc0 == 0 and q0 == 0 and rc == 0 and q == 0
    assert np.array_equal(out, out0)


def test_tc_unsupported_band_width_runs_as_pipeline(gb):
    n, b, nev = 200, 8, 40
    assert gb.gb_trans_ev_launch_count(n, b, nev, 0, TC) == 1
    hv, ht = inputs.synthetic_reflectors(n, b, seed=1)
    Z = inputs.z_gaussian(n, nev, seed=2)
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    assert np.linalg.norm(out - oracle.trans_ev(n, b, hv, ht, Z)) / np.linalg.norm(Z) <= 50 * n * U


def test_tc_wait_gives_up_and_context_survives(gb):
    n, b, nev = 600, 32, 128
    hv, ht = inputs.synthetic_reflectors(n, b, seed=3)
    Z = inputs.z_gaussian(n, nev, seed=4)
    G = (n - 1 + 15) // 16
    rc, q, _ = run(gb, n, b, hv, ht, Z, dict(TC, spin_limit=20000, test_hold_group=G))
    assert rc == 0
    assert q == gb.GB_ERR_TIMEOUT
    rc, q, out = run(gb, n, b, hv, ht, Z, TC)
    assert rc == 0 and q == 0
    assert np.linalg.norm(out - oracle.trans_ev(n, b, hv, ht, Z)) / np.linalg.norm(Z) <= 50 * n * U
