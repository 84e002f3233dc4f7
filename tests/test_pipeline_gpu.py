"""The pipeline variant (one launch, progress flags) through the C ABI:
parity with the oracle for every band width it supports, the documented
fallback for the others, and the bounded dependency wait: a group whose
progress is never published (test hook) must make the next group's wait give
up with GB_ERR_TIMEOUT, after which the context still works."""
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


PIPE = [{"variant": 2, "sweeps_per_tile": 8, "cols_per_block": 64},
        {"variant": 2, "sweeps_per_tile": 16, "cols_per_block": 128},
        {"variant": 2, "sweeps_per_tile": 16, "cols_per_block": 64},
        {"variant": 3}]


@pytest.mark.parametrize("opts", PIPE, ids=["nb8t64", "nb16t128", "nb16t64", "tensor_core"])
@pytest.mark.parametrize("n,b,nev", [(2, 8, 3), (9, 8, 1), (100, 8, 65), (257, 16, 129), (300, 32, 200),
                                     (129, 64, 130), (640, 64, 257), (1000, 64, 64), (65, 64, 31)])
def test_pipeline_parity(gb, n, b, nev, opts):
    if n <= 400:
        B = inputs.band_symmetric(n, b, seed=n + b)
        _, _, hv, ht, _ = oracle.bulge_chase(B, b)
    else:
        hv, ht = inputs.synthetic_reflectors(n, b, seed=n)
    Z = inputs.z_gaussian(n, nev, seed=nev)
    assert gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, opts) > (0 if n > 1 else -1)
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 1e-12


SCHED = [{"column_batch": 1, "lead_tiles": 1}, {"column_batch": 3, "lead_tiles": 1},
         {"column_batch": 3, "lead_tiles": 2}, {"column_batch": 1024, "lead_tiles": 3},
         {"column_batch": 2, "lead_tiles": 65536}]


@pytest.mark.parametrize("sched", SCHED, ids=["cb1l1", "cb3l1", "cb3l2", "cb1024l3", "cb2unbounded"])
@pytest.mark.parametrize("n,b,nev", [(300, 32, 200), (1000, 64, 300), (777, 16, 129)])
def test_pipeline_schedule_options(gb, n, b, nev, sched):
    """Column batching and the lead limit only reorder independent work:
    every column sees the same operations in the same order, so the result
    is bit-identical to the default schedule (and within tolerance of the
    oracle).  lead_tiles = 1 is the lock-step extreme of the lead limit."""
    hv, ht = inputs.synthetic_reflectors(n, b, seed=n + 7)
    Z = inputs.z_gaussian(n, nev, seed=nev + 7)
    base = {"variant": 2, "sweeps_per_tile": 16, "cols_per_block": 64}
    rc0, q0, out0 = run(gb, n, b, hv, ht, Z, base)
    rc, q, out = run(gb, n, b, hv, ht, Z, dict(base, **sched))
    assert rc0 == 0 and q0 == 0 and rc == 0 and q == 0
    assert np.array_equal(out, out0)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 1e-12


def test_pipeline_unsupported_nbw_falls_back(gb):
    n, b, nev = 200, 13, 40
    opts = {"variant": 2}
    assert gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, opts) == 0      # wavefront needs none
    assert gb.gb_trans_ev_launch_count(n, b, nev, 0, opts) > 1
    hv, ht = inputs.synthetic_reflectors(n, b, seed=1)
    Z = inputs.z_gaussian(n, nev, seed=2)
    rc, q, out = run(gb, n, b, hv, ht, Z, opts)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 1e-12


def test_pipeline_wait_gives_up_and_context_survives(gb):
    n, b, nev = 600, 32, 128
    hv, ht = inputs.synthetic_reflectors(n, b, seed=3)
    Z = inputs.z_gaussian(n, nev, seed=4)
    nb = 16
    G = (n - 1 + nb - 1) // nb
    # group G-1 (the first to run) never publishes: group G-2 must give up
    bad = {"variant": 2, "sweeps_per_tile": nb, "cols_per_block": 128, "spin_limit": 20000,
           "test_hold_group": G}
    rc, q, _ = run(gb, n, b, hv, ht, Z, bad)
    assert rc == 0
    assert q == gb.GB_ERR_TIMEOUT
    # the same workspace and context work for the next call
    good = {"variant": 2, "sweeps_per_tile": nb, "cols_per_block": 128}
    rc, q, out = run(gb, n, b, hv, ht, Z, good)
    assert rc == 0 and q == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 1e-12


def test_pipeline_host_buffer_entry_point(gb):
    n, b, nev = 700, 64, 96
    opts = {"variant": 2}
    hv, ht = inputs.synthetic_reflectors(n, b, seed=8)
    Z = inputs.z_gaussian(n, nev, seed=9)
    Zh = np.asfortranarray(Z.copy())
    nbytes = gb.gb_trans_ev_host_buffer_bytes(n, b, nev, n, 0, opts)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    rc = gb.gb_trans_ev_tridi_to_band_d_host(n, b, nev, hv, ht, Zh, n, buf, nbytes, None, opts, check=False)
    assert rc == 0
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    assert np.linalg.norm(Zh - ref) / np.linalg.norm(Z) <= 1e-12
