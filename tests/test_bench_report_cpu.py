"""The benchmark's oracle legs on the CPU: the bounded oracle runs (one
thread and a thread pool) cover the units they report, and the error report
measures a GPU waveform against the oracle's (a float32 copy of the oracle's
own waveform is within float rounding; a planted error shows in both
figures)."""
import os
import sys

import numpy as np

from paper_2203_02479_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _tiny_workload():
    planes = [inputs.PlaneSpec(24, 400, inputs.response("bipolar"), 0),
              inputs.PlaneSpec(20, 400, inputs.response("unipolar"), 1)]
    events = [[inputs.uniform_depos(150, 24, seed=3, nticks=400), inputs.uniform_depos(120, 20, seed=4, nticks=400)],
              [inputs.uniform_depos(90, 24, seed=5, nticks=400), inputs.uniform_depos(60, 20, seed=6, nticks=400)]]
    return inputs.Workload("tiny", planes, events, True, 0.7, 11)


def test_oracle_runs_and_error_report():
    import bench
    w = _tiny_workload()
    units = bench.sample_order(w)
    assert sorted(units) == [(0, 0), (0, 1), (1, 0), (1, 1)]
    # event by event: each event's planes in a row
    assert [p for _, p in units] == [0, 1, 0, 1] and units[0][0] == units[1][0]
    seen = {}
    # a spent budget still runs the first event whole
    dp, secs, n = bench.oracle_units(w, units, 1, 0.0, lambda u, M: seen.__setitem__(u, M))
    e0 = units[0][0]
    assert n == 2 and dp == sum(d.n for d in w.events[e0]) and list(seen) == units[:2]
    seen.clear()
    dp, secs, n = bench.oracle_units(w, units, 3, 60.0, lambda u, M: seen.__setitem__(u, M))
    assert n == 4 and dp == 150 + 120 + 90 + 60 and sorted(seen) == sorted(units)
    # the unit's waveform is the oracle's simulation with its event id as Philox counter
    import oracle
    d = w.events[1][0]
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, 24, 400, w.planes[0].response, 10, fluctuate=True, p=0.7,
                          seed=11, event_id=1, plane_id=0)
    assert np.array_equal(seen[(1, 0)], ref)
    errs = {u: bench.unit_error(M.astype(np.float32), M) for u, M in seen.items()}
    rep = bench.error_summary(errs, w)
    assert rep["units"] == 4 and rep["mode"] == "binomial"
    assert rep["rel_l2_max"] <= 1e-7 and rep["max_abs_over_max"] <= 1e-7
    assert sorted(rep["by_plane"]) == ["0", "1"]
    bad = seen[(0, 1)].astype(np.float32).copy()
    peak = float(np.abs(seen[(0, 1)]).max())
    bad[5, 100] += 0.5 * peak
    errs[(0, 1)] = bench.unit_error(bad, seen[(0, 1)])
    rep = bench.error_summary(errs, w)
    assert rep["worst_unit"] == {"event": 0, "plane_id": 1}
    assert abs(rep["max_abs_over_max"] - 0.5) <= 1e-6 and rep["rel_l2_max"] > 1e-3


def test_cpu_baselines_report_cores_and_sample():
    import bench
    w = _tiny_workload()
    gpu = {(0, 0): np.zeros((24, 400), np.float32)}
    allc, errs = bench.cpu_baselines(w, 0.0, 60.0, gpu)
    assert allc["kind"] == "oracle" and allc["cores"] == (os.cpu_count() or 1) and allc["value"] > 0
    assert allc["one_thread"]["cores"] == 1 and allc["one_thread"]["value"] > 0
    assert "4 of the workload's 4" in allc["sample"]
    assert list(errs) == [(0, 0)] and errs[(0, 0)]["rel_l2"] == 1.0


def test_algorithmic_bytes_of_the_three_plane_step():
    """Per-launch minimum bytes of each stage over the event's three planes
    (800 + 800 + 960 rows of 6000 ticks, 3126 frequencies, 21 response
    wires), against the hand count: the forward reads a 4 B cell and writes
    an 8 B frequency per row, the wire convolution reads and writes the
    spectra and reads each plane's 21-row response spectrum, the inverse
    the reverse of the forward.  With every row active (the dense count):"""
    import bench
    rows, nt, nf, kw = 2560, 6000, 3126, 21
    units = [bench.UnitSpec(nw, nt, nf, 6250, kw, 100_000) for nw in (800, 800, 960)]
    tot = {k: sum(bench.algorithmic_bytes(k, u) for u in units)
           for k in ("fwd_rows", "wire_conv", "inv_rows", "memset_grid", "raster_scatter", "mark_rows")}
    assert tot["fwd_rows"] == rows * (4 * nt + 8 * nf)
    assert tot["inv_rows"] == rows * (8 * nf + 4 * nt)
    assert tot["wire_conv"] == rows * 16 * nf + 3 * 8 * nf * kw
    assert tot["memset_grid"] == rows * nt * 4
    assert tot["raster_scatter"] == 3 * 12 * 100_000 + rows * nt * 4
    assert tot["mark_rows"] == 3 * 8 * 100_000
    # the convolution's pass bytes as the benchmark line reports them
    assert tot["fwd_rows"] + tot["wire_conv"] + tot["inv_rows"] == 380_537_424


def test_algorithmic_bytes_with_active_rows():
    """With active rows each stage counts only the rows it touches: the grid
    clear and the forward's input the touched rows, the forward's output the
    rows a live row reads, the wire convolution those and the live rows, the
    inverse the live spectra in and every waveform row out."""
    import bench
    nt, nf, kw = 6000, 3126, 21
    u = bench.UnitSpec(960, nt, nf, 6250, kw, 50_000, touched=300, need=340, live=320)
    assert bench.algorithmic_bytes("memset_grid", u) == 4 * 300 * nt
    assert bench.algorithmic_bytes("fwd_rows", u) == 4 * 300 * nt + 8 * nf * 340
    assert bench.algorithmic_bytes("wire_conv", u) == 8 * nf * (340 + 320) + 8 * nf * kw
    assert bench.algorithmic_bytes("inv_rows", u) == 8 * nf * 320 + 4 * 960 * nt
    assert bench.algorithmic_bytes("raster_scatter", u) == 12 * 50_000 + 4 * 300 * nt
    dense = bench.UnitSpec(960, nt, nf, 6250, kw, 50_000)
    assert dense.touched == dense.need == dense.live == 960


def test_impact_units_in_the_work_model_and_the_oracle_leg():
    """An impact plane's unit counts I fine rows per wire in the grid, the
    first spectra and the taps, and its oracle waveform is the impact
    simulation (the fine raster and the per-position convolution)."""
    import bench
    import oracle
    I = 4
    u1 = bench.UnitSpec(100, 6000, 3126, 6250, 21, 1000, touched=60, need=80, live=70)
    uI = bench.UnitSpec(100, 6000, 3126, 6250, 21, 1000, touched=60, need=80, live=70, imp=I)
    assert bench.algorithmic_bytes("memset_grid", uI) == I * bench.algorithmic_bytes("memset_grid", u1)
    assert bench.algorithmic_bytes("raster_scatter", uI) - 12.0 * 1000 == I * 4.0 * 60 * 6000
    assert bench.algorithmic_bytes("fwd_rows", uI) == I * bench.algorithmic_bytes("fwd_rows", u1)
    assert bench.algorithmic_bytes("wire_conv", uI) == 8.0 * 3126 * (I * 80 + 70) + 8.0 * 3126 * 21 * I
    assert bench.algorithmic_bytes("inv_rows", uI) == bench.algorithmic_bytes("inv_rows", u1)
    assert bench.algorithmic_flops("wire_conv", uI) == I * bench.algorithmic_flops("wire_conv", u1)
    R = inputs.impact_response("unipolar", impacts=I, nticks=60)
    d = inputs.uniform_depos(40, 16, seed=9, nticks=300)
    w = inputs.Workload("tiny_impacts", [inputs.PlaneSpec(16, 300, R, 2)], [[d]], False, 1.0, 5)
    M = bench.oracle_unit(w, 0, 0)
    assert np.allclose(M, oracle.simulate_impacts(d.q, d.x_mm, d.t_us, 16, 300, R, 10), rtol=0, atol=1e-9)
