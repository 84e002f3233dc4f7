"""The tensor-core pipelines through the C ABI, against the oracle:
GB_VARIANT_PIPELINE_TC5 (the default: tcgen05 MMAs with FP16 digit planes
and FP32 level sums in tensor memory, 128-column items) and
GB_VARIANT_PIPELINE_TC (warp-level mma.sync on bf16 digits, 64-column
items); both apply every tile in compact WY form by exact digit slicing with
Z in per-column 64-bit fixed point.  Covered: every supported band width, ragged
and tiny shapes, reflectors from real bulge chases at the sizes where this
kernel is the default (the oracle's chase of the n = 1024, nbw = 32 config
and the device chase at n = 2048, nbw = 64), columns of wildly different
norms (each column carries its own scale), eigenvector inputs (residual and
orthogonality), bit-identity across schedules, and the bounded dependency
wait.

Parity: the map is deterministic and column-wise, so the GPU result is held
to ||Z_gpu - Z_oracle||_F / ||Z_in||_F <= 1e-12 on the whole block and on
every column (each column relative to its own norm; measured ~5e-15)."""
import numpy as np
import pytest

import oracle
from paper_1811_01277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
PARITY = 1e-12
TC = {"variant": 3}
TC5 = {"variant": 4}
BOTH = pytest.mark.parametrize("opts", [TC5, TC], ids=["tcgen05", "mma_sync"])


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


@BOTH
@pytest.mark.parametrize("n,b,nev", [(2, 16, 3), (17, 16, 1), (100, 16, 65), (257, 16, 129), (300, 32, 200),
                                     (129, 64, 130), (640, 64, 257), (1000, 64, 64), (65, 64, 31),
                                     (1500, 32, 100), (2049, 64, 70), (4096, 64, 96), (700, 16, 300),
                                     (1200, 32, 385), (3000, 64, 513)])
def test_tc_parity(gb, n, b, nev, opts):
    if n <= 400:
        B = inputs.band_symmetric(n, b, seed=n + b)
        _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    else:
        hv, ht = inputs.synthetic_reflectors(n, b, seed=n)
    Z = inputs.z_gaussian(n, nev, seed=nev)
    assert gb.gb_trans_ev_launch_count(n, b, nev, 0, opts) == (6 if n > 1 else 0)
    assert gb.gb_trans_ev_variant(n, b, nev, 0, opts) == opts["variant"]
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= PARITY
    assert colwise_err(out, ref, Z) <= PARITY


@pytest.fixture(scope="module")
def config1():
    """n = 1024, nbw = 32, band entries U[-1,1]: the oracle's bulge chase and
    the tridiagonal's eigenvectors (oracle QL)."""
    n, b = 1024, 32
    B = inputs.band_symmetric(n, b, seed=1)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    return n, b, B, hv, ht, w, V


@pytest.mark.parametrize("opts", [None, TC], ids=["default", "mma_sync"])
def test_tc_config1_bulge_chase_reflectors(gb, config1, opts):
    """The default kernel (tcgen05) and the mma.sync one on the n = 1024
    config's own reflectors (tau = 0 runs included) and all 1024
    eigenvectors: every column against the oracle, plus residual and
    orthogonality."""
    n, b, B, hv, ht, w, V = config1
    assert gb.gb_trans_ev_variant(n, b, n, 0, None) == gb.GB_VARIANT_PIPELINE_TC5   # the library default
    assert np.any(ht == 0) and np.any(ht != 0)
    rc, q, out = run(gb, n, b, hv, ht, V, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, V)
    assert np.linalg.norm(out - ref) / np.linalg.norm(V) <= PARITY
    assert colwise_err(out, ref, V) <= PARITY
    assert np.linalg.norm(B @ out - out * w) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.T @ out - np.eye(n)).max() <= 50 * n * U


def _lower_band(B, b):
    n = B.shape[0]
    AB = np.zeros((b + 1, n), order="F")
    for d in range(b + 1):
        AB[d, :n - d] = np.diag(B, -d)
    return AB


def test_tc_device_chase_reflectors_n2048(gb):
    """n = 2048, nbw = 64: reflectors from the device bulge chase
    (gb_band_to_tridi_d), applied by the default kernel and by the oracle
    to the same Z; every column within 1e-12."""
    n, b, nev = 2048, 64, 300
    B = inputs.band_symmetric(n, b, seed=2048)
    dev = torch.device("cuda")
    AB_d = torch.from_numpy(np.ascontiguousarray(_lower_band(B, b).T)).to(dev)
    cnt = gb.gb_hh_count(n, b)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(n - 1, dtype=torch.float64, device=dev)
    hv_d = torch.zeros(cnt * b, dtype=torch.float64, device=dev)
    ht_d = torch.zeros(cnt, dtype=torch.float64, device=dev)
    wsb = gb.gb_band_to_tridi_workspace_bytes(n, b)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    gb.gb_band_to_tridi_d(n, b, AB_d, b + 1, d, e, hv_d, ht_d, ws, wsb, st)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    hv, ht = hv_d.cpu().numpy(), ht_d.cpu().numpy()
    assert np.any(ht != 0)
    Z = inputs.z_gaussian(n, nev, seed=2049)
    assert gb.gb_trans_ev_variant(n, b, nev, 0, None) == gb.GB_VARIANT_PIPELINE_TC5
    for opts in (None, TC):
        rc, q, out = run(gb, n, b, hv, ht, Z, opts)
        assert rc == 0 and q == 0
        ref = oracle.trans_ev(n, b, hv, ht, Z)
        assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= PARITY
        assert colwise_err(out, ref, Z) <= PARITY


@BOTH
def test_tc_columns_of_different_norms(gb, opts):
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
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.all(out[:, 2] == 0.0)
    assert colwise_err(out, ref, Z) <= PARITY


@BOTH
def test_tc_subnormal_columns(gb, opts):
    """A column whose largest entry is subnormal is scaled like any other
    (not flushed to zero): it matches the oracle run on the same column
    scaled by 2^600 (an exact scaling) and scaled back, to 1e-12 of its norm
    plus the output's own subnormal rounding."""
    n, b, nev = 600, 64, 6
    hv, ht = inputs.synthetic_reflectors(n, b, seed=91)
    Z = inputs.z_gaussian(n, nev, seed=92)
    Z[:, 1] *= 1e-309 / np.abs(Z[:, 1]).max()            # max 1e-309 < 2^-1022
    Z[:, 4] = 0.0
    Z[5, 4] = 5e-324                                     # the smallest subnormal, alone
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z * 2.0 ** 600) * 2.0 ** -600
    for c in range(nev):
        nz = np.linalg.norm(Z[:, c] * 2.0 ** 600) * 2.0 ** -600
        d = np.linalg.norm((out[:, c] - ref[:, c]) * 2.0 ** 600) * 2.0 ** -600
        assert d <= 1e-12 * nz + np.sqrt(n) * 2.0 ** -1074, c
    assert np.any(out[:, 1] != 0.0)        # not flushed to zero


@BOTH
def test_tc_nonfinite_columns_reported(gb, opts):
    """NaN / +Inf / -Inf entries: the call reports GB_ERR_NONFINITE, those
    columns come back all NaN, every other column is the exact result."""
    n, b, nev = 700, 64, 70
    hv, ht = inputs.synthetic_reflectors(n, b, seed=93)
    Z = inputs.z_gaussian(n, nev, seed=94)
    bad = [3, 40, 69]
    Z[17, 3] = np.nan
    Z[0, 40] = np.inf
    Z[n - 1, 69] = -np.inf
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == gb.GB_ERR_NONFINITE
    assert gb.gb_status_string(q)
    assert np.all(np.isnan(out[:, bad]))
    good = [c for c in range(nev) if c not in bad]
    ref = oracle.trans_ev(n, b, hv, ht, np.asfortranarray(Z[:, good]))
    assert colwise_err(out[:, good], ref, Z[:, good]) <= PARITY
    # the next call on the same context is clean
    Z2 = inputs.z_gaussian(n, nev, seed=95)
    rc, q, out2 = run(gb, n, b, hv, ht, Z2, opts)
    assert rc == 0 and q == 0 and np.all(np.isfinite(out2))


@BOTH
def test_tc_non_orthogonal_reflectors_reported(gb, opts):
    """tau three times the orthogonal value (I - tau v v^T then stretches by
    5 along v): the columns leave the fixed-point range, and the call
    reports GB_ERR_RANGE instead of returning wrapped values silently."""
    n, b, nev = 800, 64, 64
    hv, ht = inputs.synthetic_reflectors(n, b, seed=96)
    Z = inputs.z_gaussian(n, nev, seed=97)
    rc, q, out = run(gb, n, b, hv, 3.0 * ht, Z, opts)
    assert rc == 0 and q == gb.GB_ERR_RANGE
    assert gb.gb_status_string(q)


@BOTH
def test_tc_columns_at_the_fixed_point_edge(gb, opts):
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
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert colwise_err(out, ref, Z) <= PARITY
    assert np.abs(np.linalg.norm(out, axis=0) / np.linalg.norm(Z, axis=0) - 1.0).max() <= 50 * n * U


@BOTH
def test_tc_eigenvectors_residual(gb, opts):
    """Z_in = tridiagonal eigenvectors from the oracle's chase + QL: the
    output satisfies B Z = Z Lambda and Z^T Z = I to 50 n u."""
    n, b = 400, 32
    B = inputs.band_symmetric(n, b, seed=5)
    d, e, hv, ht, _ = oracle.bulge_chase(B, b)
    w, V = oracle.tridiag_ql(d, e)
    Z = np.asfortranarray(V[:, :200])
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    assert np.linalg.norm(B @ out - out * w[:200]) / np.linalg.norm(B) <= 50 * n * U
    assert np.abs(out.T @ out - np.eye(200)).max() <= 50 * n * U


@BOTH
@pytest.mark.parametrize("cb", [1, 3, 1024])
def test_tc_schedule_bit_identical(gb, cb, opts):
    n, b, nev = 900, 64, 300
    hv, ht = inputs.synthetic_reflectors(n, b, seed=31)
    Z = inputs.z_gaussian(n, nev, seed=32)
    rc0, q0, out0 = run(gb, n, b, hv, ht, Z, opts)
    rc, q, out = run(gb, n, b, hv, ht, Z, dict(opts, column_batch=cb))
    assert rc0 == 0 and q0 == 0 and rc == 0 and q == 0
    assert np.array_equal(out, out0)


@BOTH
def test_tc_unsupported_band_width_runs_as_pipeline(gb, opts):
    n, b, nev = 200, 8, 40
    assert gb.gb_trans_ev_launch_count(n, b, nev, 0, opts) == 1
    assert gb.gb_trans_ev_variant(n, b, nev, 0, opts) == gb.GB_VARIANT_PIPELINE
    hv, ht = inputs.synthetic_reflectors(n, b, seed=1)
    Z = inputs.z_gaussian(n, nev, seed=2)
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    assert np.linalg.norm(out - oracle.trans_ev(n, b, hv, ht, Z)) / np.linalg.norm(Z) <= PARITY


@BOTH
def test_tc_wait_gives_up_and_context_survives(gb, opts):
    n, b, nev = 600, 32, 128
    hv, ht = inputs.synthetic_reflectors(n, b, seed=3)
    Z = inputs.z_gaussian(n, nev, seed=4)
    G = (n - 1 + 15) // 16
    rc, q, _ = run(gb, n, b, hv, ht, Z, dict(opts, spin_limit=20000, test_hold_group=G))
    assert rc == 0
    assert q == gb.GB_ERR_TIMEOUT
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    assert np.linalg.norm(out - oracle.trans_ev(n, b, hv, ht, Z)) / np.linalg.norm(Z) <= PARITY


@pytest.mark.parametrize("opts", [TC5, TC, {"variant": 2}, {"variant": 1}], ids=["tcgen05", "mma_sync", "pipeline", "wavefront"])
def test_kernel_events_bracket_the_dominant_kernel(gb, opts):
    """gb_trans_ev_opts.kernel_begin_event / kernel_end_event: the library
    records the caller's events around the dominant kernel's launch(es) on the
    call's stream; the span is positive and inside the whole call's span, and
    the result is the same as without events."""
    n, b, nev = 1024, 64, 256
    hv, ht = inputs.synthetic_reflectors(n, b, seed=3)
    Z = inputs.z_gaussian(n, nev, seed=4)
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    outs = []
    for with_events in (False, True):
        Zt = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
        hv_d = torch.from_numpy(hv).to(dev)
        ht_d = torch.from_numpy(ht).to(dev)
        wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, opts)
        ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for e in ev:
            e.record(st)          # the events exist once recorded
        o = dict(opts)
        if with_events:
            o.update(kernel_begin_event=ev[1].cuda_event, kernel_end_event=ev[2].cuda_event)
        ev[0].record(st)
        gb.gb_trans_ev_tridi_to_band_d(n, b, nev, hv_d, ht_d, Zt, n, ws, wsb, st, o)
        ev[3].record(st)
        torch.cuda.synchronize()
        assert gb.gb_trans_ev_query(ws if wsb else None, wsb, st) == 0
        if with_events:
            k = ev[1].elapsed_time(ev[2])
            assert 0.0 < k <= ev[0].elapsed_time(ev[3])
            assert ev[0].elapsed_time(ev[1]) >= 0.0 and ev[2].elapsed_time(ev[3]) >= 0.0
        outs.append(Zt.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
