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
