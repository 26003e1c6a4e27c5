"""Active rows: a simulation marks the wire rows its depos may touch and the
grid clear, forward transform, wire convolution and inverse transform skip
the rest (an untouched row of S is zero through every stage).

Checked on planes whose depos fill only a band of wires (the three-plane
and batched workloads leave 25-55% of rows untouched):
  * waveforms against the FP64 oracle (expected-value mode, relative L2
    <= 1e-5) and against the same depos through ws_rasterize + ws_scatter +
    ws_convolve, which transform every row (binomial mode: the grids hold
    the same integers; relative L2 <= 1e-6, the transforms' rounding);
  * rows further than the response's reach from every touched row are
    exactly zero, and every row of the output is written (the buffer starts
    as NaN);
  * marks of an earlier call never leak into a later one: a plane that ran a
    dense event first gives bit-identical output to a fresh plane, also
    under CUDA graph replay with the depos refilled in place (the epoch
    advances on the device);
  * every wire-convolution kernel, the compensated precision path, and a
    batch mixing marked units with a noisy plane's unmarked ones.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

NW, NT = 200, 1000
KW, CENTER = 21, 10


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    wiresim.load_library()
    torch.cuda.set_device(0)
    return wiresim


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def band_depos(n, bands, seed, nt=NT):
    """n depos per band of wires [lo, hi), uniform in pitch and time."""
    qs, xs, ts = [], [], []
    for j, (lo, hi) in enumerate(bands):
        d = inputs.uniform_depos(n, hi - lo, seed + 17 * j, nticks=nt)
        qs.append(d.q); xs.append(d.x_mm + np.float32(lo * inputs.PITCH_MM)); ts.append(d.t_us)
    return inputs.PlaneDepos(np.concatenate(qs).astype(np.float32), np.concatenate(xs).astype(np.float32),
                             np.concatenate(ts).astype(np.float32))


def nan_out(nw=NW, nt=NT):
    import torch
    return torch.full((nw, nt), float("nan"), dtype=torch.float32, device="cuda")


def far_rows(bands, nw=NW, margin=KW):
    """Rows further than the response's reach (plus the one-wire widening
    and the diffusion width) from every band."""
    near = np.zeros(nw, bool)
    for lo, hi in bands:
        near[max(0, lo - margin - 3):min(nw, hi + margin + 3)] = True
    return ~near


def full_rows(ws, pl, dd, params):
    """The same depos through the unmarked path: every row transformed."""
    p = pl.rasterize(dd, params)
    g = pl.new_grid()
    pl.scatter(p, g)
    return to_np(pl.convolve(g))


BANDS = [[(80, 95)], [(0, 6)], [(194, 200)], [(20, 30), (120, 126)], [(100, 101)]]


@pytest.mark.parametrize("bands", BANDS)
def test_expected_value_band_matches_oracle(ws, bands):
    R = inputs.response("bipolar")
    pl = ws.Plane(NW, NT, R)
    d = band_depos(300, bands, seed=5)
    out = nan_out()
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(), out=out))
    assert np.isfinite(got).all()
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER)
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows(bands)] == 0).all()
    assert rel(got, full_rows(ws, pl, ws.DeviceDepos.from_plane_depos(d), ws.Params())) <= 1e-6


@pytest.mark.parametrize("bands", BANDS[:4])
def test_binomial_band_equals_every_row_transformed(ws, bands):
    pl = ws.Plane(NW, NT, inputs.response("unipolar"), plane_id=2)
    d = ws.DeviceDepos.from_plane_depos(band_depos(500, bands, seed=9))
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=321, event_id=3)
    got = to_np(pl.simulate(d, params, out=nan_out()))
    assert np.isfinite(got).all()
    assert rel(got, full_rows(ws, pl, d, params)) <= 1e-6
    assert (got[far_rows(bands)] == 0).all()


def test_no_depos_writes_zeros(ws):
    pl = ws.Plane(NW, NT, inputs.response("bipolar"))
    empty = ws.DeviceDepos(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32))
    got = to_np(pl.simulate(empty, ws.Params(fluctuate=1, p_survive=0.7), out=nan_out()))
    assert (got == 0).all()


@pytest.mark.parametrize("variant", range(10))
def test_every_wire_conv_kernel_skips_tiles_exactly(ws, variant):
    R = inputs.response("bipolar")
    pl = ws.Plane(NW, NT, R)
    pl.set_wire_conv_variant(variant)
    bands = [(40, 47), (150, 180)]
    d = band_depos(250, bands, seed=13)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(), out=nan_out()))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER)
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows(bands)] == 0).all()


def test_marks_of_an_earlier_call_do_not_leak(ws):
    R = inputs.response("bipolar")
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=77, event_id=11)
    used, fresh = ws.Plane(NW, NT, R), ws.Plane(NW, NT, R)
    for pl in (used, fresh):
        pl.set_wire_conv_variant(9)
    dense = ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(4000, NW, seed=1, nticks=NT))
    sparse = ws.DeviceDepos.from_plane_depos(band_depos(400, [(60, 70)], seed=2))
    used.simulate(dense, params)
    a = to_np(used.simulate(sparse, params, out=nan_out()))
    b = to_np(fresh.simulate(sparse, params, out=nan_out()))
    assert np.array_equal(a, b)
    # and back: a dense call after the sparse one equals a fresh dense call
    c = to_np(used.simulate(dense, params))
    fresh2 = ws.Plane(NW, NT, R)
    fresh2.set_wire_conv_variant(9)
    assert np.array_equal(c, to_np(fresh2.simulate(dense, params)))


def test_graph_replay_with_refilled_depos(ws):
    import torch
    R = inputs.response("bipolar")
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=5, event_id=2)
    pl = ws.Plane(NW, NT, R)
    pl.set_wire_conv_variant(9)
    n = 600
    da = band_depos(n, [(10, 40)], seed=3)
    db = band_depos(n, [(150, 170)], seed=4)
    dev = ws.DeviceDepos.from_plane_depos(da)
    out = torch.empty((NW, NT), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pl.simulate(dev, params, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pl.simulate(dev, params, out=out)
    ref_pl = ws.Plane(NW, NT, R)
    ref_pl.set_wire_conv_variant(9)
    for d in (db, da, db):
        for name in ("q", "x_mm", "t_us"):
            getattr(dev, name).copy_(torch.from_numpy(getattr(d, name)))
        out.fill_(float("nan"))
        g.replay()
        got = to_np(out)
        want = to_np(ref_pl.simulate(ws.DeviceDepos.from_plane_depos(d), params, out=nan_out()))
        assert np.array_equal(got, want)


def test_compensated_precision_on_a_band(ws):
    R = inputs.response("bipolar")
    pl = ws.Plane(NW, NT, R)
    bands = [(90, 110)]
    d = band_depos(800, bands, seed=21)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(precision=ws.WS_PREC_FP32_COMP),
                            out=nan_out()))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER)
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows(bands)] == 0).all()


def test_batch_mixes_marked_units_with_a_noisy_plane(ws):
    import torch
    wires = (120, 120, 144)
    planes = [ws.Plane(nw, NT, inputs.response("bipolar" if i < 2 else "unipolar"), plane_id=i)
              for i, nw in enumerate(wires)]
    L = planes[0].info.fft_len_tick
    planes[1].set_noise(inputs.noise_amplitudes(L, peak=2.0e4))
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=99, event_id=40)
    bands_of = [[(5, 20)], [(50, 60), (100, 110)], [], [(130, 144)]]
    events = []
    for e, bands in enumerate(bands_of):
        row = []
        for p, nw in enumerate(wires):
            bb = [(lo, min(hi, nw)) for lo, hi in bands if lo < nw]
            d = band_depos(200, bb, seed=70 + 10 * e + p) if bb else inputs.uniform_depos(0, nw, 0, nticks=NT)
            row.append(ws.DeviceDepos.from_plane_depos(d))
        events.append(row)
    for upw in (3, 5, 12):
        b = ws.Batch(planes, events, params, units_per_wave=upw)
        for o in b.outs:
            o.fill_(float("nan"))
        outs = [to_np(o) for o in b.run()]
        for e in range(len(events)):
            for p, pl in enumerate(planes):
                pe = ws.Params(**{**params.__dict__, "event_id": params.event_id + e})
                want = to_np(pl.simulate(events[e][p], pe))
                assert np.isfinite(outs[e * 3 + p]).all()
                assert rel(outs[e * 3 + p], want) <= 1e-6, (upw, e, p)
