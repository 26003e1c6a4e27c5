"""MultiBatch (units over several devices, Sec. 3.3) on the one GPU here:
one shard equals ws_simulate_batch over the same events, and so do two or
three shards side by side on the same device (each its own planes, stream
and workspace, the events split into contiguous cost-balanced ranges that
keep their global event ids: binomial draws are keyed by them).  In
expected-value mode every unit of a two-shard run is checked against the
FP64 oracle.

Binomial grids hold integer electron counts, so the sums are exact whatever
the order of the atomic additions; the transforms may still differ between
runs by the wire-convolution kernel each plane's autotuner picked, so the
waveforms are compared at relative L2 <= 1e-6."""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

WIRES = (40, 48, 56)
NT = 1200
COUNTS = [30, 900, 0, 2500, 120, 60, 1800]


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


def _workload():
    specs = [inputs.PlaneSpec(nw, NT, inputs.response("bipolar" if p < 2 else "unipolar"), p)
             for p, nw in enumerate(WIRES)]
    events = [[inputs.uniform_depos(n, nw, seed=900 + 7 * e + p, nticks=NT) for p, nw in enumerate(WIRES)]
              for e, n in enumerate(COUNTS)]
    return specs, events


@pytest.fixture(scope="module")
def single(ws):
    """The whole list as one ws_simulate_batch on cuda:0."""
    import torch
    specs, events = _workload()
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=4242, event_id=100)
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in specs]
    devs = [[ws.DeviceDepos.from_plane_depos(d) for d in ev] for ev in events]
    b = ws.Batch(planes, devs, params, units_per_wave=6)
    b.run()
    torch.cuda.synchronize()
    outs = [o.cpu().numpy() for o in b.outs]
    for pl in planes:
        pl.close()
    return specs, events, params, outs


@pytest.mark.parametrize("ndev", [1, 2, 3])
def test_multibatch_equals_one_batch(ws, single, ndev):
    import torch
    from paper_2203_02479_gb300 import shard
    specs, events, params, want = single
    mb = shard.MultiBatch([torch.device("cuda", 0)] * ndev, specs, events, params, units_per_wave=6)
    assert len(mb.ranges) == ndev
    assert sum(1 for e0, e1 in mb.ranges if e1 > e0) == ndev
    mb.run()
    got = mb.gather()
    assert len(got) == len(want) == len(COUNTS) * len(WIRES)
    for u, (g, w) in enumerate(zip(got, want)):
        assert g.shape == (WIRES[u % len(WIRES)], NT)
        assert rel(g, w) <= 1e-6, (u, rel(g, w))
    mb.close()


def test_multibatch_expected_value_against_oracle(ws):
    import torch
    from paper_2203_02479_gb300 import shard
    specs, events = _workload()
    mb = shard.MultiBatch([torch.device("cuda", 0)] * 2, specs, events, ws.Params(), units_per_wave=4)
    got = mb.run().gather()
    for e, ev in enumerate(events):
        for p, d in enumerate(ev):
            M = oracle.simulate(d.q, d.x_mm, d.t_us, WIRES[p], NT, specs[p].response, 10)
            assert rel(got[e * len(WIRES) + p], M) <= 1e-5, (e, p)
    mb.close()


def test_multibatch_of_impact_planes(ws):
    """Impact planes (4 sub-pitch positions) sharded over two batches on the
    one GPU equal one batch over all events."""
    import torch
    from paper_2203_02479_gb300 import shard
    specs = [inputs.PlaneSpec(nw, NT, inputs.impact_response("bipolar" if p < 2 else "unipolar", impacts=4), p)
             for p, nw in enumerate(WIRES)]
    events = [[inputs.uniform_depos(n, nw, seed=700 + 5 * e + p, nticks=NT) for p, nw in enumerate(WIRES)]
              for e, n in enumerate(COUNTS[:5])]
    params = ws.Params(fluctuate=1, p_survive=0.7, seed=77, event_id=3)
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in specs]
    devs = [[ws.DeviceDepos.from_plane_depos(d) for d in ev] for ev in events]
    b = ws.Batch(planes, devs, params, units_per_wave=3)
    b.run()
    torch.cuda.synchronize()
    want = [o.cpu().numpy() for o in b.outs]
    mb = shard.MultiBatch([torch.device("cuda", 0)] * 2, specs, events, params, units_per_wave=3)
    got = mb.run().gather()
    assert len(got) == len(want)
    for u, (g, w) in enumerate(zip(got, want)):
        assert rel(g, w) <= 1e-6, (u, rel(g, w))
    mb.close()


@pytest.mark.parametrize("fluct", [1, 2])
def test_depo_slices_with_offsets_sum_to_the_whole_plane(ws, fluct):
    """The depo split's device side: slices of one plane's depos simulated
    with their offsets (Params.depo_offset) sum to one call over the whole
    list (the random draws are keyed by the depos' indices in the list),
    and differ from it without the offsets."""
    import dataclasses
    import torch
    from paper_2203_02479_gb300 import shard
    nw, nt = 200, 6000
    d = inputs.uniform_depos(30000, nw, seed=3, nticks=nt)
    pl = ws.Plane(nw, nt, inputs.response("bipolar"))
    params = ws.Params(fluctuate=fluct, p_survive=0.7, seed=11, event_id=4)
    whole = pl.simulate(ws.DeviceDepos.from_plane_depos(d), params).clone()
    total = torch.zeros_like(whole)
    blind = torch.zeros_like(whole)
    for lo, hi in shard.depo_slices(len(d.q), 3):
        dd = ws.DeviceDepos(d.q[lo:hi], d.x_mm[lo:hi], d.t_us[lo:hi])
        total += pl.simulate(dd, dataclasses.replace(params, depo_offset=lo))
        blind += pl.simulate(dd, params)
    torch.cuda.synchronize()
    assert rel(total.cpu().numpy(), whole.cpu().numpy()) <= 1e-6
    assert rel(blind.cpu().numpy(), whole.cpu().numpy()) > 1e-4
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, inputs.response("bipolar"), 10, fluctuate=fluct, p=0.7,
                          seed=11, event_id=4, plane_id=0)
    assert rel(total.cpu().numpy(), ref) <= 1e-5
