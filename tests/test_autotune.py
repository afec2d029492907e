"""The autotuner's selection logic (CPU, with the timed solves replaced by
fakes): per shape class the fastest schedule that converges wins, classes
already in the table are kept, the table round-trips through JSON, and the
persistent batch's launch shape is the fastest candidate that finished."""
import json

import pytest

from paper_2012_07322_gb300 import autotune, mg


def desc(geom, n, precision="mixed"):
    return mg.grid_desc(geom, n, hi=[100.0, 3.14159], precision=precision, accel_depth=16)


def test_shape_key_and_schedule_copy():
    d = desc("sph", [64, 32])
    assert autotune.shape_key(d) == "g%d_n64x32_p%d" % (mg.GEOM["sph"], mg.MG_MIXED)
    assert autotune.shape_key(desc("sph", [64, 32], "fp64")) != autotune.shape_key(d)
    e = autotune.with_schedule(mg, d, (1, 3, 8))
    assert (e.nu1, e.nu2, e.accel_depth) == (1, 3, 8)
    assert (d.nu1, d.nu2, d.accel_depth) == (2, 2, 16)  # the original is untouched
    assert list(e.n) == list(d.n) and e.tol == d.tol and e.geom == d.geom


def test_tune_picks_the_fastest_converged_schedule(monkeypatch, tmp_path):
    # per schedule: (ms, converged, cycles); the fastest overall does not converge
    times = {(2, 2, 16): (30.0, True, 40), (2, 2, 8): (20.0, True, 50), (2, 2, 0): (5.0, False, 800),
             (1, 1, 16): (25.0, True, 60)}
    calls = []

    def fake(mg_, torch_, d, src, repeats):
        key = (d.nu1, d.nu2, d.accel_depth)
        calls.append((autotune.shape_key(d), key))
        return times[key]

    monkeypatch.setattr(autotune, "_time_solve", fake)
    path = str(tmp_path / "table.json")
    items = [(desc("sph", [64, 32]), None), (desc("sph", [64, 32]), None), (desc("cyl", [32, 64]), None)]
    table = autotune.tune(mg, None, items, path=path, candidates=list(times))
    assert set(table) == {autotune.shape_key(items[0][0]), autotune.shape_key(items[2][0])}
    for e in table.values():
        assert (e["nu1"], e["nu2"], e["accel_depth"]) == (2, 2, 8) and e["ms"] == 20.0 and e["cycles"] == 50
        assert len(e["tried"]) == len(times)
    assert len(calls) == 2 * len(times)  # one representative per shape class
    assert json.load(open(path)) == table
    # a second run keeps the classes already tuned and times nothing
    calls.clear()
    again = autotune.tune(mg, None, items, path=path, candidates=list(times))
    assert again == table and not calls
    tuned = autotune.tuned(mg, items[0][0], table)
    assert (tuned.nu1, tuned.nu2, tuned.accel_depth) == (2, 2, 8)
    other = desc("sph", [128, 64])
    assert autotune.tuned(mg, other, table) is other


class _FakeClock:
    def __init__(self):
        self.t = 0.0

    def perf_counter(self):
        return self.t


class _FakeTorch:
    class cuda:
        @staticmethod
        def synchronize():
            pass


def test_tune_launch_picks_the_fastest_shape(monkeypatch):
    clock = _FakeClock()
    ms = {(2, 16384): 0.20, (4, 16384): 0.23, (1, 0): 0.27, (8, 32768): 0.15}
    status = {(8, 32768): "noconv"}
    resets = []

    class FakeMg:
        MG_OK, MG_ERR_NOCONV, MG_ERR_STALLED = mg.MG_OK, mg.MG_ERR_NOCONV, mg.MG_ERR_STALLED

        @staticmethod
        def mg_solve_cfc_batch(problems, reports, team, team_cells, allow):
            clock.t += ms[(team, team_cells)]
            return None, {"status": status.get((team, team_cells), "ok"), "blocks": 152}

    monkeypatch.setattr(autotune.time, "perf_counter", clock.perf_counter)
    out = autotune.tune_launch(FakeMg, _FakeTorch, [], lambda: resets.append(1), candidates=list(ms), repeats=2)
    # the fastest candidate did not converge: the fastest one that did wins
    assert (out["team"], out["team_cells"]) == (2, 16384)
    assert out["ms"] == pytest.approx(200.0)
    assert len(out["tried"]) == len(ms) and len(resets) == 3 * len(ms)
    assert [t["ok"] for t in out["tried"]] == [True, True, True, False]
