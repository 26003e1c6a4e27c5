"""ws_simulate_batch: many events x planes per launch, against ws_simulate
unit by unit and against the FP64 oracle.

Batched and per-unit runs draw the same Philox numbers (the counter holds
the event, plane, depo and bin), so binomial grids hold the same integers;
expected-value grids differ only by the order of the float additions, so
they are compared at relative L2 <= 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _setup(ws, counts, wires=(40, 40, 48), nt=1500, seed=70, sig=False):
    planes = [ws.Plane(nw, nt, inputs.response("bipolar" if i < 2 else "unipolar"), plane_id=i)
              for i, nw in enumerate(wires)]
    events = []
    host = []
    for e, n in enumerate(counts):
        row, hrow = [], []
        for p, nw in enumerate(wires):
            d = inputs.uniform_depos(n, nw, seed + 10 * e + p, nticks=nt)
            if sig:
                rng = np.random.Generator(np.random.PCG64(seed + e))
                st = rng.choice([0.3, 40.0], n).astype(np.float32)
                sx = rng.choice([1.0, 60.0], n).astype(np.float32)
                row.append(ws.DeviceDepos(d.q, d.x_mm, d.t_us, st, sx))
                hrow.append((d, st, sx))
            else:
                row.append(ws.DeviceDepos.from_plane_depos(d))
                hrow.append((d, None, None))
        events.append(row)
        host.append(hrow)
    return planes, events, host


@pytest.mark.parametrize("fluct", [False, True])
def test_batch_equals_per_unit(ws, fluct):
    import torch
    counts = [10, 500, 2000, 0, 37]
    planes, events, _ = _setup(ws, counts)
    params = ws.Params(fluctuate=fluct, p_survive=0.7 if fluct else 0.9, seed=12345, event_id=3)
    b = ws.Batch(planes, events, params, units_per_wave=4)
    outs = b.run()
    torch.cuda.synchronize()
    for e in range(len(counts)):
        for p, pl in enumerate(planes):
            pe = ws.Params(**{**params.__dict__, "event_id": params.event_id + e})
            ref = pl.simulate(events[e][p], pe)
            torch.cuda.synchronize()
            got = outs[e * len(planes) + p].cpu().numpy()
            assert rel(got, ref.cpu().numpy()) <= 1e-6, (e, p)
    for pl in planes:
        assert pl.status() == 0


def test_batch_matches_oracle(ws):
    import torch
    counts = [300, 1200]
    planes, events, host = _setup(ws, counts, seed=80)
    b = ws.Batch(planes, events, ws.Params(), units_per_wave=6)
    outs = b.run()
    torch.cuda.synchronize()
    for e in range(len(counts)):
        for p, pl in enumerate(planes):
            d = host[e][p][0]
            ref = oracle.simulate(d.q, d.x_mm, d.t_us, pl.nwires, pl.nticks,
                                  inputs.response("bipolar" if p < 2 else "unipolar"), 10)
            assert rel(outs[e * 3 + p].cpu().numpy(), ref) <= 1e-5


def test_batch_large_patches_across_units(ws):
    """Wide given widths send patches to the warp-per-depo kernel through the
    hand-over list, whose entries carry the unit."""
    import torch
    counts = [40, 0, 25]
    planes, events, host = _setup(ws, counts, wires=(60, 60, 60), nt=800, seed=90, sig=True)
    b = ws.Batch(planes, events, ws.Params(), units_per_wave=5)
    outs = b.run()
    torch.cuda.synchronize()
    for e in range(len(counts)):
        for p, pl in enumerate(planes):
            d, st, sx = host[e][p]
            S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, pl.nwires, pl.nticks, sig_t_us=st, sig_x_mm=sx)
            ref = oracle.convolve_fft(S, inputs.response("bipolar" if p < 2 else "unipolar"), 10)
            assert rel(outs[e * 3 + p].cpu().numpy(), ref) <= 1e-5


def test_batch_graph_replay(ws):
    import torch
    counts = [100, 3000, 50]
    planes, events, _ = _setup(ws, counts, seed=100)
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=7)
    b = ws.Batch(planes, events, params, units_per_wave=3)
    first = [o.clone() for o in b.run()]
    b.capture()
    for o in b.outs:
        o.fill_(-1.0)
    b.replay()
    torch.cuda.synchronize()
    for a, o in zip(first, b.outs):
        assert torch.equal(a, o)


def test_batch_rejects_mismatched_planes(ws):
    p1 = ws.Plane(20, 1000, inputs.response())
    p2 = ws.Plane(20, 1200, inputs.response())
    d = ws.DeviceDepos([1.0], [5.0], [10.0])
    with pytest.raises(ws.WiresimError) as ei:
        ws.Batch([p1, p2], [[d, d]], ws.Params())
    assert ei.value.status == 2


def test_batch_of_no_events_and_one_wave_per_plane(ws):
    """No events: nothing is enqueued.  One plane per wave over more waves
    than streams (wave k on stream k % 3) equals one wave of everything."""
    import torch
    planes, events, _ = _setup(ws, [200, 0, 900, 50], seed=110)
    assert ws.Batch(planes, [], ws.Params()).run() == []
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=9)
    one = [o.clone() for o in ws.Batch(planes, events, params, units_per_wave=12).run()]
    many = ws.Batch(planes, events, params, units_per_wave=1).run()
    torch.cuda.synchronize()
    assert len(one) == len(many) == 12
    for a, b in zip(one, many):
        assert rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6
    for pl in planes:
        assert pl.status() == 0


def _oracle_units(w, units, fluctuate, seed_events_from=0):
    """FP64 oracle waveforms of (event, plane) units of a workload, computed
    in a thread pool (the oracle's C loops and numpy's FFT release the GIL)."""
    import concurrent.futures as cf
    import os

    def one(u):
        e, p = u
        sp, d = w.planes[p], w.events[e][p]
        S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=fluctuate,
                                  p=w.p_survive, seed=w.seed, event_id=seed_events_from + e,
                                  plane_id=sp.plane_id)
        return oracle.convolve_fft(S, sp.response, 10)

    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        return list(ex.map(one, units))


def test_batched_workload_at_full_size_against_oracle(ws):
    """The 64-event workload (log-uniform depo counts from 1k to 500k per
    event, binomial fluctuation) through ws_simulate_batch in waves of 32
    units on three streams, captured into a CUDA graph and replayed; the
    waveforms of the largest and smallest events and of eight more seeded
    events (30 units) against the FP64 oracle's, at the binomial waveform
    bound (one-electron differences move a waveform by ~1e-6)."""
    import torch
    w = inputs.batched_events()
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in w.planes]
    events = [[ws.DeviceDepos.from_plane_depos(d) for d in ev] for ev in w.events]
    params = ws.Params(fluctuate=True, p_survive=w.p_survive, seed=w.seed)
    b = ws.Batch(planes, events, params, units_per_wave=32)
    b.capture()
    for o in b.outs:
        o.fill_(float("nan"))
    b.replay()
    torch.cuda.synchronize()
    counts = np.array([ev[0].n for ev in w.events])
    rng = np.random.Generator(np.random.PCG64(1002))
    pick = [int(np.argmax(counts)), int(np.argmin(counts))]
    pick += [int(e) for e in rng.choice(np.setdiff1d(np.arange(len(counts)), pick), 8, replace=False)]
    assert counts[pick[0]] > 400_000 and counts[pick[1]] < 3_000
    units = [(e, p) for e in pick for p in range(3)]
    refs = _oracle_units(w, units, True)
    for (e, p), M in zip(units, refs):
        got = b.outs[e * 3 + p].cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all(), (e, p)
        assert rel(got, M) <= 1e-5, (e, p, rel(got, M))
        assert np.abs(got - M).max() <= 1e-4 * np.abs(M).max(), (e, p)
    for pl in planes:
        assert pl.status() == 0


def test_batched_workload_expected_value_units(ws):
    """The same 64 events in expected-value mode (no fluctuation): the
    largest event's three planes and one small event's within the
    deterministic bound 1e-5."""
    import torch
    w = inputs.batched_events(fluctuate=False, p_survive=1.0)
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in w.planes]
    events = [[ws.DeviceDepos.from_plane_depos(d) for d in ev] for ev in w.events]
    b = ws.Batch(planes, events, ws.Params(seed=w.seed), units_per_wave=32)
    outs = b.run()
    torch.cuda.synchronize()
    counts = np.array([ev[0].n for ev in w.events])
    units = [(int(np.argmax(counts)), p) for p in range(3)] + [(5, 0)]
    for (e, p), M in zip(units, _oracle_units(w, units, False)):
        assert rel(outs[e * 3 + p].cpu().numpy(), M) <= 1e-5, (e, p)


def test_large_patch_list_overflow_falls_back(ws):
    """More patches too large for the lane-per-depo kernel than the hand-over
    list holds (65,536) in one wave: the warp-per-depo kernel then walks every
    depo of the wave itself.  Expected value through the batch against the
    oracle at 1e-5; binomial through ws_simulate with exact-branch counts
    (small charges) against the oracle's integers bin by bin."""
    import torch
    nw, nt, n = 400, 6000, 40_000
    rng = np.random.Generator(np.random.PCG64(424242))
    planes = [ws.Plane(nw, nt, inputs.response("bipolar" if i < 1 else "unipolar"), plane_id=i) for i in range(2)]
    host, events = [], []
    for p in range(2):
        d = inputs.uniform_depos(n, nw, 500 + p, nticks=nt, q_mean=400.0)
        st = rng.uniform(4.5, 6.0, n).astype(np.float32)     # > 16 ticks: large
        sx = rng.uniform(0.5, 1.5, n).astype(np.float32)
        host.append((d, st, sx))
        events.append(ws.DeviceDepos(d.q, d.x_mm, d.t_us, st, sx))
    # 80k large patches in one wave of two units: past the list's capacity
    b = ws.Batch(planes, [events], ws.Params(), units_per_wave=2)
    outs = b.run()
    torch.cuda.synchronize()
    for p, (d, st, sx) in enumerate(host):
        S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, nw, nt, sig_t_us=st, sig_x_mm=sx)
        M = oracle.convolve_fft(S, planes[p].response.cpu().numpy(), 10)
        assert rel(outs[p].cpu().numpy(), M) <= 1e-5, p
    # binomial, one plane with all 40k large depos plus 40k more of the other
    d0, st0, sx0 = host[0]
    d1, st1, sx1 = host[1]
    q = np.concatenate([d0.q, d1.q]); x = np.concatenate([d0.x_mm, d1.x_mm])
    t = np.concatenate([d0.t_us, d1.t_us])
    st = np.concatenate([st0, st1]); sx = np.concatenate([sx0, sx1])
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=77, fluct_exact_max=64)
    pt = planes[0].rasterize(ws.DeviceDepos(q, x, t, st, sx), params)
    grid = planes[0].new_grid()
    planes[0].scatter(pt, grid)
    torch.cuda.synchronize()
    got = grid.cpu().numpy().astype(np.float64)
    ref = oracle.raster_scatter(q, x, t, nw, nt, sig_t_us=st, sig_x_mm=sx, fluctuate=True, p=0.7, seed=77,
                                exact_max=64)
    qw = oracle.raster_scatter(q, x, t, nw, nt, sig_t_us=st, sig_x_mm=sx)
    assert float(np.floor(qw + 0.5).max()) <= 64 * 40     # sums of exact-branch bins
    diff = np.abs(got - ref)
    assert (diff > 0).mean() < 1e-3
    assert abs(got.sum() - ref.sum()) <= 1e-4 * ref.sum()
    for pl in planes:
        assert pl.status() == 0


def test_autotuned_wave_size_is_the_fastest_and_changes_nothing(ws):
    """ws_batch_autotune on the three-plane event (100k track depos,
    binomial): the wave size it records is, within timing noise, the fastest
    of the fixed sizes (graph replays, median of 30), and a batch run with
    the recorded size (units_per_wave = 0) gives the same waveforms as every
    fixed size."""
    import torch
    w = inputs.three_planes()
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in w.planes]
    depos = [ws.DeviceDepos.from_plane_depos(d) for d in w.events[0]]
    params = ws.Params(fluctuate=True, p_survive=w.p_survive, seed=w.seed)
    auto = ws.Batch(planes, [depos], params)
    upw = auto.autotune()
    assert 1 <= upw <= 3 and planes[0].info.batch_units_per_wave == upw
    assert 0 <= planes[0].info.batch_wire_conv_variant <= 9
    ref = [o.cpu().numpy() for o in auto.run()]

    def median_ms(b):
        b.capture()
        for _ in range(3):
            b.replay()
        t = []
        for _ in range(30):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.replay()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return float(np.median(t))

    times = {}
    for fixed in (1, 2, 3):
        b = ws.Batch(planes, [depos], params, units_per_wave=fixed)
        outs = b.run()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert rel(o.cpu().numpy(), r) <= 1e-6, fixed
        times[fixed] = median_ms(b)
    assert times[upw] <= 1.15 * min(times.values()) + 0.01, (upw, times)
    for pl in planes:
        assert pl.status() == 0
