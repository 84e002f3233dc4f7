"""The no-allocation entry point (gb_trans_ev_tridi_to_band_d_noalloc).

It serves callers that cannot allocate device memory -- code running inside
a memory pool or arena that owns the whole device, allocation-free service
loops, hosts that forbid cudaMalloc after start-up.  Its scratch lives in a
fixed device array inside the library, so these tests check that two calls
in a row (which share and reuse that array) match the oracle at the parity
bar (1e-12 per column) and give the same result as the regular entry point
with a caller-allocated workspace, and that a problem too large for the fixed
array is refused before anything runs.

This file is named to be collected last; it passes alone in a fresh process
as well as after the other tests.
"""
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


def _host_problem(n, b, nev, seed):
    hv, ht = inputs.synthetic_reflectors(n, b, seed=seed)
    return hv, ht, inputs.z_gaussian(n, nev, seed=seed + 1)


def _device_problem(n, b, nev, seed):
    dev = torch.device("cuda")
    hv, ht, Z = _host_problem(n, b, nev, seed)
    return (torch.from_numpy(hv).to(dev), torch.from_numpy(ht).to(dev),
            torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev))


def _regular(gb, n, b, nev, hv, ht, Zt):
    """The existing entry point with a torch-allocated workspace."""
    out = Zt.clone()
    st = torch.cuda.current_stream()
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev, 0, None)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device="cuda")
    gb.gb_trans_ev_tridi_to_band_d(n, b, nev, hv, ht, out, n, ws, wsb, st, None)
    assert gb.gb_trans_ev_query(ws, wsb, st) == 0
    return out


def test_noalloc_matches_regular_entry_point_twice(gb):
    st = torch.cuda.current_stream()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # two calls in a row on different problems: the second reuses the scratch
    # array the first left behind
    for (n, b, nev, seed) in [(1500, 64, 300, 11), (777, 32, 129, 12)]:
        hv, ht, Zt = _device_problem(n, b, nev, seed)
        ref = _regular(gb, n, b, nev, hv, ht, Zt)
        out = Zt.clone()
        status.fill_(-1)
        rc = gb.gb_trans_ev_tridi_to_band_d_noalloc(n, b, nev, hv, ht, out, n, status, st, check=False)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        err = torch.linalg.norm(out - ref).item() / torch.linalg.norm(Zt).item()
        assert err <= 1e-12
        # against the oracle, every column
        hv_h, ht_h, Z_h = _host_problem(n, b, nev, seed)
        want = oracle.trans_ev(n, b, hv_h, ht_h, Z_h)
        got = out.cpu().numpy().T
        assert np.max(np.linalg.norm(got - want, axis=0) / np.linalg.norm(Z_h, axis=0)) <= 1e-12


def test_noalloc_refuses_problems_beyond_its_scratch(gb):
    # n = 32768, nev = 16384 needs 2 MiB of flags > GB_NOALLOC_SCRATCH_BYTES
    opts = {"variant": 2, "sweeps_per_tile": 16, "cols_per_block": 64}
    assert gb.gb_trans_ev_workspace_bytes(32768, 64, 16384, 0, opts) > gb.GB_NOALLOC_SCRATCH_BYTES
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = gb.gb_trans_ev_tridi_to_band_d_noalloc(32768, 64, 16384, x, x, x, 32768, None, None, check=False)
    assert rc == gb.GB_ERR_WORKSPACE
    rc = gb.gb_trans_ev_tridi_to_band_d_noalloc(100, 13, 4, x, x, x, 100, None, None, check=False)
    assert rc == -2  # only the pipeline band widths
