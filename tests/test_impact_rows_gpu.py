"""Impact planes (the pitch axis binned at pitch / I, Sec. 2.1's per-position
field response) with active rows and in batches.

A simulation on an impact plane marks the wires its depos may touch (all I
fine rows of a marked wire are cleared and transformed together), the
impact wire convolution skips wire blocks whose outputs are all dead, and
the inverse transform writes zeros for rows no marked wire reaches.  The
results must equal the unmarked route (ws_rasterize + ws_scatter into the
fine grid + ws_convolve, which transforms every fine row) and the FP64
oracle:
  * expected-value mode: relative L2 <= 1e-5 against the oracle's impact
    simulation, with each tile shape of the TMA impact kernel;
  * binomial mode: the same integers in the fine grid, so relative L2 <=
    1e-6 against the unmarked route (the transforms' rounding);
  * rows beyond the response's reach from every band are exactly zero and
    every output row is written (outputs start as NaN);
  * marks of an earlier call never leak into a later one;
  * a response narrower than the kernels' 21-wire register window (taps
    past K_w are zero, so every row in a live output's window must hold a
    finite spectrum).
Batches of impact planes (ws_simulate_batch) equal one ws_simulate per
unit, with marked units beside a noisy plane's unmarked ones, and under
graph replay.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

NW, NT, I = 120, 1000, 10
CENTER = 10


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


def no_depos(nw):
    return inputs.uniform_depos(0, nw, 0, nticks=NT)


def nan_out(nw=NW, nt=NT):
    import torch
    return torch.full((nw, nt), float("nan"), dtype=torch.float32, device="cuda")


def far_rows(bands, nw=NW, margin=21):
    near = np.zeros(nw, bool)
    for lo, hi in bands:
        near[max(0, lo - margin - 3):min(nw, hi + margin + 3)] = True
    return ~near


def unmarked(pl, dd, params):
    """The same depos through the fine grid and ws_convolve (every fine row
    transformed)."""
    p = pl.rasterize(dd, params)
    g = pl.new_grid()
    pl.scatter(p, g)
    return to_np(pl.convolve(g))


BANDS = [[(30, 42)], [(0, 5), (110, 120)], [(60, 61)]]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("bands", BANDS)
def test_expected_value_band_matches_oracle(ws, bands, variant):
    R = inputs.impact_response("bipolar", impacts=I)
    pl = ws.Plane(NW, NT, R, plane_id=1)
    pl.set_wire_conv_variant(variant)
    d = band_depos(250, bands, seed=31)
    dd = ws.DeviceDepos.from_plane_depos(d)
    got = to_np(pl.simulate(dd, ws.Params(), out=nan_out()))
    assert np.isfinite(got).all()
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER)
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows(bands)] == 0).all()
    assert rel(got, unmarked(pl, dd, ws.Params())) <= 1e-6
    assert pl.status() == 0


@pytest.mark.parametrize("bands", BANDS[:2])
def test_binomial_band_equals_unmarked_route(ws, bands):
    pl = ws.Plane(NW, NT, inputs.impact_response("unipolar", impacts=I), plane_id=2)
    dd = ws.DeviceDepos.from_plane_depos(band_depos(400, bands, seed=8))
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=404, event_id=6)
    got = to_np(pl.simulate(dd, params, out=nan_out()))
    assert np.isfinite(got).all()
    assert rel(got, unmarked(pl, dd, params)) <= 1e-6
    assert (got[far_rows(bands)] == 0).all()


def test_no_depos_writes_zeros(ws):
    pl = ws.Plane(NW, NT, inputs.impact_response("bipolar", impacts=I))
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(no_depos(NW)), ws.Params(fluctuate=1), out=nan_out()))
    assert (got == 0).all()


def test_marks_of_an_earlier_call_do_not_leak(ws):
    R = inputs.impact_response("bipolar", impacts=I)
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=3, event_id=9)
    used, fresh = ws.Plane(NW, NT, R), ws.Plane(NW, NT, R)
    for pl in (used, fresh):
        pl.set_wire_conv_variant(1)
    dense = ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(3000, NW, seed=2, nticks=NT))
    sparse = ws.DeviceDepos.from_plane_depos(band_depos(300, [(70, 80)], seed=4))
    used.simulate(dense, params)
    a = to_np(used.simulate(sparse, params, out=nan_out()))
    b = to_np(fresh.simulate(sparse, params, out=nan_out()))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("impacts", [1, 4])
def test_narrow_response_band(ws, impacts):
    """A 7-wire response (centre 3): live outputs read 21-row windows whose
    taps past the seventh are zero."""
    kw, c = 7, 3
    if impacts == 1:
        R = inputs.response("bipolar", nwires=kw, wire_center=c)
    else:
        R = inputs.impact_response("bipolar", impacts=impacts, nwires=kw, wire_center=c)
    pl = ws.Plane(NW, NT, R, wire_center=c)
    bands = [(20, 26), (90, 100)]
    d = band_depos(300, bands, seed=77)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(), out=nan_out()))
    assert np.isfinite(got).all()
    if impacts == 1:
        ref = oracle.simulate(d.q, d.x_mm, d.t_us, NW, NT, R, c)
    else:
        ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, NW, NT, R, c)
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows(bands, margin=kw)] == 0).all()


def _impact_planes(ws, wires=(96, 96, 120)):
    kinds = ["bipolar", "bipolar", "unipolar"]
    return [ws.Plane(nw, NT, inputs.impact_response(kinds[i], impacts=I), plane_id=i) for i, nw in enumerate(wires)]


def _banded_events(ws, wires, bands_of, n=200, seed=50):
    events = []
    for e, bands in enumerate(bands_of):
        row = []
        for p, nw in enumerate(wires):
            bb = [(lo, min(hi, nw)) for lo, hi in bands if lo < nw]
            d = band_depos(n, bb, seed=seed + 10 * e + p) if bb else no_depos(nw)
            row.append(ws.DeviceDepos.from_plane_depos(d))
        events.append(row)
    return events


def test_batch_of_impact_planes_equals_per_unit_calls(ws):
    wires = (96, 96, 120)
    planes = _impact_planes(ws, wires)
    L = planes[0].info.fft_len_tick
    planes[1].set_noise(inputs.noise_amplitudes(L, peak=2.0e4))   # its units take the unmarked route
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=123, event_id=20)
    events = _banded_events(ws, wires, [[(5, 20)], [(40, 50), (80, 96)], [], [(100, 120)]])
    for upw in (1, 3, 5):
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
        assert all(pl.status() == 0 for pl in planes)


def test_batch_of_impact_planes_matches_oracle(ws):
    wires = (96, 96, 120)
    planes = _impact_planes(ws, wires)
    bands_of = [[(10, 30)], [(50, 70), (90, 96)]]
    host = [[band_depos(150, [(lo, min(hi, nw)) for lo, hi in bands if lo < nw], seed=90 + 10 * e + p)
             for p, nw in enumerate(wires)] for e, bands in enumerate(bands_of)]
    events = [[ws.DeviceDepos.from_plane_depos(d) for d in row] for row in host]
    b = ws.Batch(planes, events, ws.Params(), units_per_wave=6)
    outs = [to_np(o) for o in b.run()]
    for e, row in enumerate(host):
        for p, d in enumerate(row):
            ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, wires[p], NT, planes[p].response.cpu().numpy(), CENTER)
            assert rel(outs[e * 3 + p], ref) <= 1e-5, (e, p)


def test_batch_of_impact_planes_graph_replay(ws):
    import torch
    wires = (96, 96, 120)
    planes = _impact_planes(ws, wires)
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=9, event_id=1)
    events = _banded_events(ws, wires, [[(0, 30)], [(60, 90)]], seed=7)
    b = ws.Batch(planes, events, params)
    b.capture()
    want = [to_np(o) for o in b.run()]
    for o in b.outs:
        o.fill_(float("nan"))
    b.replay()
    torch.cuda.synchronize()
    for o, w in zip(b.outs, want):
        assert np.array_equal(to_np(o), w)


def test_batch_rejects_mixed_impact_counts(ws):
    planes = [ws.Plane(40, NT, inputs.impact_response("bipolar", impacts=I)),
              ws.Plane(40, NT, inputs.response("bipolar"))]
    events = [[ws.DeviceDepos.from_plane_depos(no_depos(40))] * 2]
    with pytest.raises(ws.WiresimError):
        ws.Batch(planes, events, ws.Params(), units_per_wave=2).run()


def test_batch_with_the_most_impact_positions_takes_one_unit_per_launch(ws):
    """32 sub-pitch positions: a launch of the impact wire convolution holds
    the tensor maps of one unit only, so a wave of three units takes three
    launches; the batch still equals per-unit calls."""
    wires, nt, I = (16, 20, 24), 1000, 32
    planes = [ws.Plane(nw, nt, inputs.impact_response("bipolar", impacts=I), plane_id=p) for p, nw in enumerate(wires)]
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=3, event_id=1)
    events = [[ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(150, nw, seed=10 * e + p, nticks=nt))
               for p, nw in enumerate(wires)] for e in range(2)]
    b = ws.Batch(planes, events, params, units_per_wave=3)
    outs = [to_np(o) for o in b.run()]
    for e in range(2):
        for p, pl in enumerate(planes):
            pe = ws.Params(**{**params.__dict__, "event_id": params.event_id + e})
            assert rel(outs[e * 3 + p], to_np(pl.simulate(events[e][p], pe))) <= 1e-6, (e, p)


@pytest.mark.parametrize("bands,circular", [([(30, 42)], False), (None, False), (None, True)])
def test_compensated_precision_on_impact_planes(ws, bands, circular):
    """FP32_COMP on an impact plane (the fine grid's low parts kept beside
    it and added by the forward transform), with active wires (a band), on
    every wire, and in circular mode (every fine row transformed), against
    the oracle and the FP32 path."""
    R = inputs.impact_response("bipolar", impacts=I)
    pl = ws.Plane(NW, NT, R, circular=circular)
    d = band_depos(300, bands, seed=17) if bands else inputs.uniform_depos(3000, NW, seed=17, nticks=NT)
    dd = ws.DeviceDepos.from_plane_depos(d)
    comp = to_np(pl.simulate(dd, ws.Params(precision=ws.WS_PREC_FP32_COMP), out=nan_out()))
    plain = to_np(pl.simulate(dd, ws.Params()))
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER, circular=circular)
    assert np.isfinite(comp).all()
    assert rel(comp, ref) <= 1e-5
    assert rel(comp, plain) <= 1e-5
    if bands:
        assert (comp[far_rows(bands)] == 0).all()


@pytest.mark.parametrize("circular,fluct", [(False, 0), (True, 0), (False, 1)])
def test_fp64_precision_on_impact_planes(ws, circular, fluct):
    """WS_PREC_FP64 on an impact plane (double fine grid, transforms and
    impact sum): the oracle's waveform up to the float output's rounding
    (binomial mode: the same counts, the oracle's random stream)."""
    nw = 60
    R = inputs.impact_response("unipolar", impacts=I)
    pl = ws.Plane(nw, NT, R, circular=circular, fp64=True, plane_id=1)
    d = inputs.uniform_depos(800, nw, seed=23, nticks=NT)
    params = ws.Params(precision=ws.WS_PREC_FP64, fluctuate=fluct, p_survive=0.7 if fluct else 1.0, seed=8,
                       event_id=2)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), params, out=nan_out(nw)))
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, nw, NT, R, CENTER, circular=circular, fluctuate=fluct,
                                  p=0.7 if fluct else 1.0, seed=8, event_id=2, plane_id=1)
    assert np.isfinite(got).all()
    assert rel(got, ref) <= 1e-7
    assert pl.status() == 0


def test_noise_on_an_impact_plane_matches_oracle(ws):
    """Eq. 1's noise term on an impact plane (every row live, so the
    unmarked route): the impact simulation plus the oracle's noise."""
    R = inputs.impact_response("bipolar", impacts=I)
    pl = ws.Plane(NW, NT, R, plane_id=3)
    L = pl.info.fft_len_tick
    amp = inputs.noise_amplitudes(L, peak=2.0e4)
    coh = inputs.noise_amplitudes(L, "coherent", peak=2.0e4)
    pl.set_noise(amp, coh, 16)
    d = band_depos(300, [(40, 60)], seed=29)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(seed=12, event_id=6), out=nan_out()))
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER) + \
        oracle.noise(NW, NT, L, amp, coh, 16, seed=12, event_id=6, plane_id=3)
    assert np.isfinite(got).all()
    assert rel(got, ref) <= 1e-5


def test_given_widths_on_an_impact_plane(ws):
    """Depos with their own widths (sigma_t, sigma_x given, no diffusion) on
    an impact plane with active wires: marks from the given pitch widths at
    pitch / I, against the oracle."""
    R = inputs.impact_response("unipolar", impacts=I)
    pl = ws.Plane(NW, NT, R)
    d = band_depos(200, [(20, 35), (90, 100)], seed=31)
    rng = np.random.Generator(np.random.PCG64(31))
    st = rng.uniform(0.2, 3.0, len(d.q)).astype(np.float32)
    sx = rng.uniform(0.05, 2.5, len(d.q)).astype(np.float32)
    dd = ws.DeviceDepos(d.q, d.x_mm, d.t_us, sigma_t_us=st, sigma_x_mm=sx)
    got = to_np(pl.simulate(dd, ws.Params(), out=nan_out()))
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, NW, NT, R, CENTER, sig_t_us=st, sig_x_mm=sx)
    assert np.isfinite(got).all()
    assert rel(got, ref) <= 1e-5
    assert (got[far_rows([(20, 35), (90, 100)])] == 0).all()
