"""The benchmark's error-against-the-oracle report, on the CPU: the oracle
sample keeps one waveform per plane, and oracle_error_of measures a GPU
waveform against it (a float32 copy of the oracle's own waveform is within
float rounding; a planted error shows in both figures)."""
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
    events = [[inputs.uniform_depos(150, 24, seed=3, nticks=400), inputs.uniform_depos(120, 20, seed=4, nticks=400)]]
    return inputs.Workload("tiny", planes, events, True, 0.7, 11)


def test_oracle_sample_keeps_one_waveform_per_plane_and_reports_error():
    import bench
    w = _tiny_workload()
    bench._ORACLE_NEXT[0] = 0
    kept = {}
    done, secs, nplanes = bench.oracle_sample(w, 0.0, keep=kept)
    assert nplanes == 1 and done == 150 and sorted(kept) == [0]
    bench.oracle_sample(w, 0.0, keep=kept)
    bench.oracle_sample(w, 0.0, keep=kept)     # plane 0 again: the first waveform stays
    assert sorted(kept) == [0, 1]
    assert kept[0].shape == (24, 400) and kept[1].shape == (20, 400)
    gpu = [kept[0].astype(np.float32), kept[1].astype(np.float32)]
    rep = bench.oracle_error_of(gpu, kept, w)
    assert rep["mode"] == "binomial"
    assert [p["plane_id"] for p in rep["planes"]] == [0, 1]
    for p in rep["planes"]:
        assert p["rel_l2"] <= 1e-7 and p["max_abs_over_max"] <= 1e-7
    bad = [g.copy() for g in gpu]
    peak = float(np.abs(kept[1]).max())
    bad[1][5, 100] += 0.5 * peak
    rep = bench.oracle_error_of(bad, kept, w)
    assert rep["planes"][0]["rel_l2"] <= 1e-7
    assert abs(rep["planes"][1]["max_abs_over_max"] - 0.5) <= 1e-6
    assert rep["planes"][1]["rel_l2"] > 1e-3


def test_algorithmic_bytes_of_the_three_plane_step():
    """Per-launch minimum bytes of each stage over the event's three planes
    (800 + 800 + 960 rows of 6000 ticks, 3126 frequencies, 21 response
    wires), against the hand count: the forward reads a 4 B cell and writes
    an 8 B frequency per row, the wire convolution reads and writes the
    spectra and reads each plane's 21-row response spectrum, the inverse
    the reverse of the forward."""
    import bench
    rows, nt, nf, kw = 2560, 6000, 3126, 21
    tot = {k: sum(bench.algorithmic_bytes(k, nw, nt, nf, kw, 100_000) for nw in (800, 800, 960))
           for k in ("fwd_rows", "wire_conv", "inv_rows", "memset_grid", "raster_scatter")}
    assert tot["fwd_rows"] == rows * (4 * nt + 8 * nf)
    assert tot["inv_rows"] == rows * (8 * nf + 4 * nt)
    assert tot["wire_conv"] == rows * 16 * nf + 3 * 8 * nf * kw
    assert tot["memset_grid"] == rows * nt * 4
    assert tot["raster_scatter"] == 3 * 12 * 100_000 + rows * nt * 4
    # the convolution's pass bytes as the benchmark line reports them
    assert tot["fwd_rows"] + tot["wire_conv"] + tot["inv_rows"] == 380_537_424
