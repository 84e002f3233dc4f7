"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/elpa_gb300.h declares; the layout helpers agree with the
oracle; invalid arguments are rejected before anything touches a GPU."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_1811_01277_gb300 as gb
from paper_1811_01277_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gb.load()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b((?:gb|elpa)_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "gb_trans_ev_tridi_to_band_d" in names
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(gb.EXPORTS)
    # and every export has its binding in the package namespace
    assert [nm for nm in gb.EXPORTS if not hasattr(gb, nm)] == []


@pytest.mark.parametrize("n,b", [(1, 1), (2, 1), (3, 2), (100, 7), (1024, 32), (16384, 64), (1000, 64)])
def test_layout_matches_oracle(lib, n, b):
    assert gb.gb_hh_count(n, b) == oracle.hh_count(n, b)
    for s in sorted({1, 2, n // 2, n - 2, n - 1}):
        if 1 <= s <= n - 1:
            nk = (n - s + b - 1) // b
            for k in sorted({0, nk // 2, nk - 1}):
                assert gb.gb_hh_index(n, b, s, k) == oracle.hh_index(n, b, s, k)
            assert gb.gb_hh_index(n, b, s, nk) == -1


def test_invalid_arguments_rejected_on_host(lib):
    f = gb.gb_trans_ev_tridi_to_band_d
    ok = dict(n=10, nbw=3, nev=2, hh_v=256, hh_tau=256, Z=256, ldz=10)

    def call(**kw):
        a = dict(ok, **kw)
        return f(a["n"], a["nbw"], a["nev"], a["hh_v"], a["hh_tau"], a["Z"], a["ldz"], check=False)

    assert call(n=0) == -1
    assert call(nbw=0) == -2
    assert call(nbw=gb.gb_max_nbw() + 1) == -2
    assert call(nev=-1) == -3
    assert call(hh_v=None) == -4
    assert call(hh_v=257) == -4          # misaligned
    assert call(hh_tau=None) == -5
    assert call(Z=None) == -6
    assert call(Z=260) == -6
    assert call(ldz=9) == -7
    assert f(10, 3, 2, 256, 256, 256, 10, opts={"variant": 7}, check=False) == -11
    assert f(10, 3, 2, 256, 256, 256, 10, opts={"variant": 1, "cols_per_block": 48}, check=False) == -11
    for bad in ({"column_batch": -1}, {"column_batch": 1025}, {"lead_tiles": -1}, {"lead_tiles": 65537}):
        assert f(10, 16, 2, 256, 256, 256, 10, opts=dict({"variant": 2}, **bad), check=False) == -11
        assert gb.gb_trans_ev_workspace_bytes(100, 16, 10, 0, dict({"variant": 2}, **bad)) == 0
    # no-op cases return success without touching memory or a GPU
    assert f(1, 3, 5, None, None, 256, 1, check=False) == 0
    assert f(10, 3, 0, 256, 256, None, 10, check=False) == 0
    assert gb.gb_trans_ev_tridi_to_band_z(0, 3, 2, 256, 256, 256, 10, check=False) == -1
    assert gb.gb_status_string(-3).startswith("invalid argument")
    assert gb.gb_status_string(gb.GB_ERR_TIMEOUT).startswith("a device-side")


def test_variant_resolution_is_host_only(lib):
    """AUTO resolves to the tcgen05 pipeline for real or complex nbw in
    {16, 32, 64} and n >= 512, the DFMA pipeline for the other real
    pipeline band widths, the wavefront otherwise; tensor-core requests fall
    back to the pipeline (real) or the wavefront (complex)."""
    v = gb.gb_trans_ev_variant
    assert v(16384, 64, 4096) == gb.GB_VARIANT_PIPELINE_TC5
    assert v(1024, 32, 1024) == gb.GB_VARIANT_PIPELINE_TC5
    assert v(600, 16, 10) == gb.GB_VARIANT_PIPELINE_TC5
    assert v(500, 64, 10) == gb.GB_VARIANT_PIPELINE
    assert v(4096, 8, 100) == gb.GB_VARIANT_PIPELINE
    assert v(4096, 13, 100) == gb.GB_VARIANT_WAVEFRONT
    assert v(4096, 64, 100, 1) == gb.GB_VARIANT_PIPELINE_TC5         # complex
    assert v(500, 64, 100, 1) == gb.GB_VARIANT_WAVEFRONT
    assert v(4096, 13, 100, 1) == gb.GB_VARIANT_WAVEFRONT
    assert v(4096, 64, 100, 0, {"variant": 3}) == gb.GB_VARIANT_PIPELINE_TC
    assert v(4096, 64, 100, 1, {"variant": 3}) == gb.GB_VARIANT_WAVEFRONT
    assert v(4096, 8, 100, 0, {"variant": 4}) == gb.GB_VARIANT_PIPELINE
    assert v(4096, 8, 100, 1, {"variant": 4}) == gb.GB_VARIANT_WAVEFRONT
    assert v(300, 32, 100, 1, {"variant": 4}) == gb.GB_VARIANT_PIPELINE_TC5
    assert v(4096, 64, 100, 0, {"variant": 5}) == -1
    assert gb.gb_trans_ev_launch_count(4096, 64, 100, 0, {"variant": 4}) == 6
    # the tcgen05 workspace: head, flags, scales, offsets and one 98816-byte
    # record per tile (b = 64: tiles of 32 sweeps, window 95 rows padded to 96)
    n, b, nev = 4096, 64, 300
    G = (n - 1 + 31) // 32
    tiles = sum((n - (1 + 32 * g) + b - 1) // b for g in range(G))
    wsb = gb.gb_trans_ev_workspace_bytes(n, b, nev)
    assert tiles * 98816 <= wsb <= tiles * 98816 + (1 << 20)
    # complex: tiles of 8 sweeps, the real form's record (16 reflector
    # columns, window 142 rows padded to 144): 36864 + 37504 bytes
    Gz = (n - 1 + 7) // 8
    tz = sum((n - (1 + 8 * g) + b - 1) // b for g in range(Gz))
    wz = gb.gb_trans_ev_workspace_bytes(n, b, nev, 1)
    assert tz * (36864 + 37504) <= wz <= tz * (36864 + 37504) + (1 << 20)


def test_launch_count_is_host_only(lib):
    # one launch per anti-diagonal of the tile graph
    assert gb.gb_trans_ev_launch_count(1, 4, 10) == 0
    n, b = 1024, 32
    c = gb.gb_trans_ev_launch_count(n, b, 1024, opts={"variant": 1, "sweeps_per_tile": 16})
    G = (n - 1 + 15) // 16
    assert G <= c <= G + (n + b - 1) // b


def test_device_arguments_refuse_host_memory(lib):
    """The binding refuses host tensors and arrays where the library reads
    device memory, before anything is called; raw addresses and None pass."""
    torch = pytest.importorskip("torch")
    h = torch.zeros(16, dtype=torch.float64)
    a = np.zeros(16)
    with pytest.raises(TypeError):
        gb.gb_trans_ev_tridi_to_band_d(10, 3, 2, h, h, h, 10, check=False)
    with pytest.raises(TypeError):
        gb.gb_solve_d(4, 4, 2, a, 4, a, a, 4, None, 0, None, 0, check=False)
    with pytest.raises(TypeError):
        gb.gb_dgemm_sliced("N", "N", 2, 2, 2, 1.0, h, 2, h, 2, 0.0, h, 2, None, 0, None, check=False)
    with pytest.raises(TypeError):
        gb.gb_solve_batched_d([4], [4], [h], [4], [h], [h], [4], None, 0, [0], check=False)
    # argument checks on raw addresses still reach the library
    assert gb.gb_trans_ev_tridi_to_band_d(10, 3, 2, 256, 256, 256, 9, check=False) == -7


def test_newer_entry_points_check_arguments_host_only(lib):
    """The divide-and-conquer, refinement, stage, staged-batch and graph entry
    points reject bad arguments with -i before touching a GPU, and their
    workspace queries are host arithmetic."""
    dc = gb.gb_tridiag_dc_d
    assert dc(0, 256, 256, 256, 256, 1, 256, 1 << 30, None, check=False) == -1
    assert dc(4, None, 256, 256, 256, 4, 256, 1 << 30, None, check=False) == -2
    assert dc(4, 256, None, 256, 256, 4, 256, 1 << 30, None, check=False) == -3
    assert dc(4, 256, 256, None, 256, 4, 256, 1 << 30, None, check=False) == -4
    assert dc(4, 256, 256, 256, None, 4, 256, 1 << 30, None, check=False) == -5
    assert dc(4, 256, 256, 256, 256, 3, 256, 1 << 30, None, check=False) == -6
    assert dc(4, 256, 256, 256, 256, 4, None, 1 << 30, None, check=False) == -7
    assert dc(4, 256, 256, 256, 256, 4, 256, 8, None, check=False) == -8
    assert gb.gb_tridiag_dc_workspace_bytes(0) == 0
    assert gb.gb_tridiag_dc_workspace_bytes(1000) >= 3 * 1000 * 1000 * 8
    rf = gb.gb_refine_syev_d
    assert rf(0, 256, 1, 256, 256, 1, 256, 1 << 30, None, check=False) == -1
    assert rf(4, None, 4, 256, 256, 4, 256, 1 << 30, None, check=False) == -2
    assert rf(4, 256, 3, 256, 256, 4, 256, 1 << 30, None, check=False) == -3
    assert rf(4, 256, 4, None, 256, 4, 256, 1 << 30, None, check=False) == -4
    assert rf(4, 256, 4, 256, None, 4, 256, 1 << 30, None, check=False) == -5
    assert rf(4, 256, 4, 256, 256, 3, 256, 1 << 30, None, check=False) == -6
    assert rf(4, 256, 4, 256, 256, 4, None, 1 << 30, None, check=False) == -7
    assert rf(4, 256, 4, 256, 256, 4, 256, 8, None, check=False) == -8
    assert gb.gb_refine_syev_workspace_bytes(100) >= 4 * 100 * 100 * 8
    # the mixed-precision solve
    mx = gb.gb_solve_mixed_d
    assert mx(1, 1, 1, 256, 1, 256, 256, 1, 1, 256, 1 << 30, None, check=False) == -1
    assert mx(10, 11, 3, 256, 10, 256, 256, 10, 1, 256, 1 << 30, None, check=False) == -2
    assert mx(10, 5, 10, 256, 10, 256, 256, 10, 1, 256, 1 << 30, None, check=False) == -3
    assert mx(10, 5, 3, 256, 9, 256, 256, 10, 1, 256, 1 << 30, None, check=False) == -5
    assert mx(10, 5, 3, 256, 10, 256, 256, 9, 1, 256, 1 << 30, None, check=False) == -8
    assert mx(10, 5, 3, 256, 10, 256, 256, 10, -1, 256, 1 << 30, None, check=False) == -9
    assert mx(10, 5, 3, 256, 10, 256, 256, 10, 9, 256, 1 << 30, None, check=False) == -9
    assert mx(10, 5, 3, 256, 10, 256, 256, 10, 1, None, 1 << 30, None, check=False) == -10
    assert mx(10, 5, 3, 256, 10, 256, 256, 10, 1, 256, 8, None, check=False) == -11
    assert gb.gb_solve_mixed_workspace_bytes(10, 11, 3) == 0
    assert gb.gb_solve_mixed_workspace_bytes(1000, 10, 32) >= (
        1000 * 1000 * 8 + max(gb.gb_solve_workspace_bytes(1000, 1000, 32), gb.gb_refine_syev_workspace_bytes(1000)))
    # the solve in three calls
    assert gb.gb_solve_stage_front(0, 1, 1, 1, 256, 1, 256, 1 << 30, None, check=False) == -1
    assert gb.gb_solve_stage_front(1, 100, 10, 100, 256, 100, 256, 1 << 30, None, check=False) == -3
    assert gb.gb_solve_stage_back(0, 1, 1, 1, 256, 256, 1, 256, 1 << 30, None, check=False) == -2
    assert gb.gb_solve_stage_back(0, 100, 10, 16, 256, 256, 100, None, 1 << 30, None, check=False) == -7
    assert gb.gb_solve_stage_table_bytes(0) == 0 and gb.gb_solve_stage_table_bytes(3) > 256
    ch = gb.gb_solve_stage_chase_batched
    assert ch(0, [100], [10], [16], [256], None, 1 << 20, None, check=False) == -7
    assert ch(0, [100], [10], [16], [256], 256, 16, None, check=False) == -8
    # staged batch and graph: workspace checks come first
    sizes, nevs, bws = [100, 200], [100, 50], [16, 32]
    wsb = gb.gb_solve_batched_staged_workspace_bytes(sizes, nevs, bws, 2)
    assert wsb > gb.gb_solve_batched_staged_workspace_bytes(sizes, nevs, bws, 1) > 0
    assert gb.gb_solve_batched_staged_workspace_bytes(sizes, nevs, [16, 300], 1) == 0   # nbw >= n
    args = (sizes, nevs, bws, [256, 256], sizes, [256, 256], [256, 256], sizes)
    assert gb.gb_solve_batched_staged_d(*args, None, wsb, [0, 0], check=False) == -10
    assert gb.gb_solve_batched_staged_d(*args, 256, wsb - 1, [0, 0], check=False) == -11
    with pytest.raises(gb.GbError) as e:
        gb.gb_solve_batched_graph_create(*args, None, 1 << 30, 2)
    assert e.value.status == -10
    assert gb.gb_solve_batched_graph_nodes(None) == -1
