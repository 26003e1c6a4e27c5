"""The seeded input generators against the recipe they state: determinism by
seed, ranges, the track geometry, the charge distributions, the response
shapes and the noise spectra.  Both the CUDA path and the oracle read these
inputs, so a drift in them would move both sides at once; these checks pin
them on their own."""
import math

import numpy as np
import pytest

from paper_2203_02479_gb300 import inputs


def _same(a, b):
    return all(np.array_equal(getattr(a, k), getattr(b, k)) for k in ("q", "x_mm", "t_us"))


def test_uniform_depos_recipe():
    d = inputs.uniform_depos(200_000, 960, seed=4)
    assert _same(d, inputs.uniform_depos(200_000, 960, seed=4))
    assert not _same(d, inputs.uniform_depos(200_000, 960, seed=5))
    for a in (d.q, d.x_mm, d.t_us):
        assert a.dtype == np.float32 and a.flags.c_contiguous and a.shape == (200_000,)
    assert d.x_mm.min() >= 0.0 and d.x_mm.max() < 960 * inputs.PITCH_MM
    assert d.t_us.min() > 0.0 and d.t_us.max() <= inputs.NTICKS * inputs.TICK_US
    assert d.q.min() >= 0.0
    assert abs(float(d.q.mean()) / 5000.0 - 1.0) < 0.02            # Exp(5000): s.e. 0.2%
    assert abs(float(np.median(d.q)) / (5000.0 * math.log(2.0)) - 1.0) < 0.02
    late = inputs.uniform_depos(10_000, 100, seed=1, t_min_us=1.0)
    assert late.t_us.min() > 1.0


def test_track_event_geometry_and_charge():
    n = 20_000
    ev = inputs.track_event(n, seed=8)
    ev2 = inputs.track_event(n, seed=8)
    assert all(np.array_equal(getattr(ev, k), getattr(ev2, k)) for k in ("drift_mm", "y_mm", "z_mm", "q"))
    assert ev.n == n
    drift_len = inputs.NTICKS * inputs.TICK_US * inputs.DRIFT_V_MM_US
    assert ev.drift_mm.min() >= 0.0 and ev.drift_mm.max() < drift_len
    # steps of 1 mm along straight tracks of 500 steps (reflection at the
    # drift walls keeps the step length)
    pts = np.stack([ev.drift_mm, ev.y_mm, ev.z_mm], axis=1).astype(np.float64).reshape(-1, 500, 3)
    step = np.linalg.norm(np.diff(pts, axis=1), axis=2)
    assert np.mean(np.abs(step - 1.0) < 1e-3) > 0.99
    # Moyal(6000, 600) charge clipped to [0, 60000]: mode near 6000
    assert ev.q.min() >= 0.0 and ev.q.max() <= 60000.0
    hist, edges = np.histogram(ev.q, bins=np.arange(0.0, 20000.0, 250.0))
    mode = 0.5 * (edges[np.argmax(hist)] + edges[np.argmax(hist) + 1])
    assert 5500.0 <= mode <= 6500.0


def test_plane_projection():
    """pitch = z cos a + y sin a with the box centre on the wire span's
    centre; t = drift / v."""
    ev = inputs.TrackEvent(np.array([0.0, 1600.0, 800.0], np.float32), np.array([1000.0, 0.0, 1000.0], np.float32),
                           np.array([1000.0, 0.0, 0.0], np.float32), np.array([1.0, 2.0, 3.0], np.float32))
    for g in inputs.THREE_PLANES:
        p = ev.plane(g, box_mm=2000.0)
        a = math.radians(g.angle_deg)
        half = 0.5 * g.nwires * inputs.PITCH_MM
        assert p.x_mm[0] == pytest.approx(half, abs=1e-3)          # the box centre
        assert p.x_mm[1] == pytest.approx(half - 1000.0 * (math.cos(a) + math.sin(a)), abs=1e-3)
        assert p.x_mm[2] == pytest.approx(half - 1000.0 * math.cos(a), abs=1e-3)
        assert np.allclose(p.t_us, [0.0, 1000.0, 500.0])
        assert np.array_equal(p.q, ev.q)


def test_event_depo_counts_log_uniform():
    c = inputs.event_depo_counts(4000, seed=2, lo=1000, hi=500000)
    assert c.min() >= 1000 and c.max() <= 500000
    lg = np.log(c.astype(np.float64))
    lo, hi = math.log(1000), math.log(500000)
    assert abs(lg.mean() - 0.5 * (lo + hi)) < 0.05
    assert abs(lg.std() - (hi - lo) / math.sqrt(12.0)) < 0.05


def test_response_shapes():
    for kind in ("bipolar", "unipolar"):
        R = inputs.response(kind).astype(np.float64)
        assert R.shape == (inputs.RESP_NWIRES, inputs.RESP_NTICKS)
        c = inputs.RESP_WIRE_CENTER
        assert np.allclose(R[c - 4:c], R[c + 4:c:-1])               # symmetric in wire about the centre
        assert np.argmax(np.abs(R).max(axis=1)) == c
    Ru = inputs.response("unipolar").astype(np.float64)
    assert np.argmax(Ru[10]) == 100 and (Ru >= 0).all()
    Rb = inputs.response("bipolar").astype(np.float64)
    j = np.arange(1, 90)
    assert np.allclose(Rb[10, 100 + j], -Rb[10, 100 - j], atol=1e-7)   # antisymmetric in time
    assert Rb[10, 100] == 0.0
    with pytest.raises(ValueError):
        inputs.response("tripolar")


def test_impact_response_mirror_symmetry():
    """Positions i and I - 1 - i sit symmetrically about the pitch centre, so
    their wire factors are mirror images about the centre wire."""
    I = 10
    R = inputs.impact_response("unipolar", impacts=I).astype(np.float64)
    assert R.shape == (I, inputs.RESP_NWIRES, inputs.RESP_NTICKS)
    c = inputs.RESP_WIRE_CENTER
    d = np.arange(-9, 10)
    for i in range(I):
        assert np.allclose(R[I - 1 - i][c + d], R[i][c - d], atol=1e-7)
    # a charge near the pitch's low edge induces more on the lower neighbour
    assert R[0][c - 1, 100] > R[0][c + 1, 100]
    assert R[I - 1][c + 1, 100] > R[I - 1][c - 1, 100]


def test_noise_amplitudes_shape():
    L = 6250
    a = inputs.noise_amplitudes(L).astype(np.float64)
    c = inputs.noise_amplitudes(L, "coherent").astype(np.float64)
    assert a.shape == c.shape == (L // 2 + 1,)
    peak, x0 = 2.0e5, 0.1
    k0 = int(round(x0 * L / 2))
    assert abs(np.argmax(a) - k0) <= 1 and abs(np.argmax(c) - k0) <= 1
    assert a.max() == pytest.approx(peak * 1.1, rel=1e-4)            # bump peak + white floor
    assert c.max() == pytest.approx(0.3 * peak, rel=1e-4)
    assert a[0] == pytest.approx(0.1 * peak) and c[0] == 0.0
    with pytest.raises(ValueError):
        inputs.noise_amplitudes(L, "pink")


def test_workloads():
    w = inputs.three_planes(n=3000, seed=1001)
    assert [p.nwires for p in w.planes] == [800, 800, 960]
    assert [p.plane_id for p in w.planes] == [0, 1, 2]
    assert w.fluctuate and w.p_survive == 0.7 and w.seed == 1001
    assert [d.n for d in w.events[0]] == [3000, 3000, 3000]
    # the same depos seen by the three planes: charge and time agree
    assert np.array_equal(w.events[0][0].q, w.events[0][2].q)
    assert np.array_equal(w.events[0][0].t_us, w.events[0][1].t_us)
    b = inputs.batched_events(nevents=4, seed=1002, lo=100, hi=2000)
    assert len(b.events) == 4 and all(len(ev) == 3 for ev in b.events)
    counts = inputs.event_depo_counts(4, 1002, 100, 2000)
    assert [ev[0].n for ev in b.events] == [int(n) for n in counts]
