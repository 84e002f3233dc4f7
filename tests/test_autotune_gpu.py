"""On-the-fly autotuning of the back-transformation on the GPU: every
setting the MEDIUM walk hands out is run through the C ABI, timed with CUDA
events, checked against the oracle, and reported; the kept setting is the
fastest one measured."""
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


def test_medium_walk_on_gpu(gb):
    n, b, nev = 1500, 64, 256
    hv, ht = inputs.synthetic_reflectors(n, b, seed=15)
    Z = inputs.z_gaussian(n, nev, seed=16)
    ref = oracle.trans_ev(n, b, hv, ht, Z)
    dev = torch.device("cuda")
    hv_d, ht_d = torch.from_numpy(hv).to(dev), torch.from_numpy(ht).to(dev)
    Z0 = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)
    st = torch.cuda.current_stream()
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_MEDIUM, n, b, nev)
    times = {}
    while True:
        o = gb.gb_autotune_step(t)
        if o is None:
            break
        wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, o)
        ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
        Zt = Z0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        gb.gb_trans_ev_tridi_to_band_d(n, b, nev, hv_d, ht_d, Zt, n, ws, wsb, st, o)
        e1.record(st)
        assert gb.gb_trans_ev_query(ws if wsb else None, wsb, st) == 0
        sec = e0.elapsed_time(e1) / 1e3
        out = Zt.cpu().numpy().T
        assert np.linalg.norm(out - ref) / np.linalg.norm(Z) <= 1e-12
        times[(o.variant, o.sweeps_per_tile, o.cols_per_block, o.column_batch)] = sec
        assert gb.gb_autotune_report(t, sec) == 0
    best, s = gb.gb_autotune_best(t)
    assert len(times) == 9 + 4 + 3 + 3      # wavefront, pipeline, mma.sync and tcgen05 pipeline settings
    assert s == min(times.values())
    assert times[(best.variant, best.sweeps_per_tile, best.cols_per_block, best.column_batch)] == s
    gb.gb_autotune_destroy(t)
