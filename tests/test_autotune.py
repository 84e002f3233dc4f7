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


def test_solve_tuner_classes_trials_and_choice(tmp_path):
    """Band-width tuning of the two-stage solve: geometric size classes, one
    trial per band width below the class's representative order, the
    fastest band width per class, the default outside the tuned range or for
    an unmeasured class, and save/resume with a trial pending."""
    t = gb.gb_solve_tuner_create(128, 2048, 4)
    assert t
    trials = []
    while True:
        tr = gb.gb_solve_tuner_step(t)
        if tr is None:
            break
        n, b = tr
        trials.append(tr)
        assert b < n and b in (16, 32, 64)
        # fake cost: 32 wins below 400, 64 above
        assert gb.gb_solve_tuner_report(t, {16: 3.0, 32: 1.0 if n < 400 else 2.0, 64: 2.0 if n < 400 else 1.0}[b]) == 0
    reps = sorted({n for n, _ in trials})
    assert len(reps) == 4 and reps[0] > 128 and reps[-1] < 2048        # geometric middles
    assert all(sum(1 for n, _ in trials if n == r) == 3 for r in reps)  # 16, 32, 64 below each
    assert gb.gb_solve_tuner_nbw(t, 130) == 32
    assert gb.gb_solve_tuner_nbw(t, 2048) == 64
    assert gb.gb_solve_tuner_nbw(t, 100) == gb.gb_solve_default_nbw(100)      # outside the range
    assert gb.gb_solve_tuner_nbw(t, 5000) == gb.gb_solve_default_nbw(5000)
    gb.gb_solve_tuner_destroy(t)
    # an unmeasured class falls back to the default; tiny orders get n - 1
    t = gb.gb_solve_tuner_create(2, 16, 1)
    assert gb.gb_solve_tuner_step(t)[1] < 16
    assert gb.gb_solve_tuner_nbw(t, 9) == gb.gb_solve_default_nbw(9)
    # save with the trial pending, load: it is handed out again
    path = tmp_path / "tuner.txt"
    assert gb.gb_solve_tuner_save(t, path) == 0
    gb.gb_solve_tuner_destroy(t)
    t2 = gb.gb_solve_tuner_load(path)
    assert t2
    n, b = gb.gb_solve_tuner_step(t2)
    assert gb.gb_solve_tuner_report(t2, 0.5) == 0
    assert gb.gb_solve_tuner_step(t2) is None
    assert gb.gb_solve_tuner_nbw(t2, 3) == min(b, 2)
    gb.gb_solve_tuner_destroy(t2)
    assert not gb.gb_solve_tuner_create(1, 10, 2) and not gb.gb_solve_tuner_create(10, 5, 2)
    assert not gb.gb_solve_tuner_create(10, 20, 0)
