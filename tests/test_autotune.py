"""Autotuning object (host logic, no GPU): candidate lists for the FAST and
MEDIUM levels, best-setting selection, and save/resume mid-walk."""
import os

import pytest

import paper_1811_01277_gb300 as gb
from paper_1811_01277_gb300 import build as gbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    gb.load()


def walk(t, cost):
    seen = []
    while True:
        o = gb.gb_autotune_step(t)
        if o is None:
            break
        key = (o.variant, o.sweeps_per_tile, o.cols_per_block, o.column_batch)
        seen.append(key)
        assert gb.gb_autotune_report(t, cost(key)) == 0
    return seen


def test_fast_level_tries_each_variant_once():
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_FAST, 4096, 64, 1024)
    seen = walk(t, lambda k: {1: 2.0, 2: 1.5, 3: 0.7, 4: 0.3}[k[0]])
    assert sorted(seen) == [(1, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0), (4, 0, 0, 0)]
    best, s = gb.gb_autotune_best(t)
    assert (best.variant, s) == (4, 0.3)
    gb.gb_autotune_destroy(t)
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_FAST, 4096, 13, 1024)   # no pipeline for nbw = 13
    assert walk(t, lambda k: 1.0) == [(1, 0, 0, 0)]
    gb.gb_autotune_destroy(t)


def test_medium_level_finds_minimum():
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_MEDIUM, 16384, 64, 4096)
    cost = lambda k: 1.0 + 0.01 * k[1] + (0.5 if k[0] == 1 else 0.0) + 0.001 * k[2] + 0.0001 * k[3]
    seen = walk(t, cost)
    assert len(seen) == 9 + 4 + 3 + 3 and len(set(seen)) == len(seen)
    best, s = gb.gb_autotune_best(t)
    assert (best.variant, best.sweeps_per_tile, best.cols_per_block, best.column_batch) == min(seen, key=cost)
    assert s == min(cost(k) for k in seen)
    gb.gb_autotune_destroy(t)


def test_protocol_errors_and_nothing_measured():
    assert not gb.gb_autotune_create(7, 10, 2, 2)
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_FAST, 100, 8, 10)
    assert gb.gb_autotune_best(t) == (None, None)
    gb.gb_autotune_step(t)
    with pytest.raises(gb.GbError):            # must report before the next step
        gb.gb_autotune_step(t)
    assert gb.gb_autotune_report(t, -1.0) == -2
    gb.gb_autotune_destroy(t)


def test_save_and_resume_mid_walk(tmp_path):
    path = str(tmp_path / "tune.txt")
    cost = lambda k: 3.0 - 0.1 * k[1] + 0.002 * k[2] + (0.3 if k[0] == 2 else 0.0)
    t = gb.gb_autotune_create(gb.GB_AUTOTUNE_MEDIUM, 2048, 32, 512)
    first = []
    for _ in range(5):
        o = gb.gb_autotune_step(t)
        k = (o.variant, o.sweeps_per_tile, o.cols_per_block, o.column_batch)
        first.append(k)
        gb.gb_autotune_report(t, cost(k))
    pending = gb.gb_autotune_step(t)           # handed out, not reported
    assert gb.gb_autotune_save(t, path) == 0
    gb.gb_autotune_destroy(t)
    t2 = gb.gb_autotune_load(path)
    assert t2
    assert gb.gb_autotune_progress(t2) == (5, 19)
    rest = walk(t2, cost)
    assert rest[0] == (pending.variant, pending.sweeps_per_tile, pending.cols_per_block, pending.column_batch)
    best, s = gb.gb_autotune_best(t2)
    assert (best.variant, best.sweeps_per_tile, best.cols_per_block, best.column_batch) == min(first + rest, key=cost)
    gb.gb_autotune_destroy(t2)
    with open(path, "w") as f:
        f.write("garbage\n")
    assert not gb.gb_autotune_load(path)
    assert not gb.gb_autotune_load(str(tmp_path / "missing.txt"))
