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
