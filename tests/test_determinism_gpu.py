"""Reproducibility on the GPU, the build's stand-in for race detection and
its resume story.

Binomial counts are integers, so their scatter-add (atomics in any order)
is exact and the transforms that follow are deterministic per row: two runs
give the same waveforms bit for bit.  The random stream is counter-based
(seed, event, plane, depo, bin), so an event simulated again on its own
from its event id is the event the first run made: "resume" is skipping
the events already done.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    wiresim.load_library()
    torch.cuda.set_device(0)
    return wiresim


def _planes(ws):
    w = inputs.three_planes()
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in w.planes]
    return w, planes


def test_binomial_runs_are_bitwise_reproducible(ws):
    import torch
    w, planes = _planes(ws)
    depos = [ws.DeviceDepos.from_plane_depos(d) for d in w.events[0]]
    for fluct in (1, 2):
        b = ws.Batch(planes, [depos], ws.Params(fluctuate=fluct, p_survive=0.7, seed=99), units_per_wave=2)
        first = [o.clone() for o in b.run()]
        second = b.run()
        torch.cuda.synchronize()
        for a, c in zip(first, second):
            assert torch.equal(a, c)


def test_resume_from_an_event_id(ws):
    """Events 0, 1, 2 in one batch against events 1 and 2 alone (event ids
    from 1): identical waveforms."""
    import torch
    _, planes = _planes(ws)
    evs = [[ws.DeviceDepos.from_plane_depos(d) for d in inputs.three_planes(n=20_000, seed=700 + e).events[0]]
           for e in range(3)]
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=5, event_id=0)
    full = [o.clone() for o in ws.Batch(planes, evs, params, units_per_wave=3).run()]
    tail = ws.Batch(planes, evs[1:], ws.Params(**{**params.__dict__, "event_id": 1}), units_per_wave=2).run()
    torch.cuda.synchronize()
    for i, o in enumerate(tail):
        assert torch.equal(o, full[3 + i]), i


def test_ws_log_reports_device_status():
    """WS_LOG set: a non-finite depo shows up on stderr when the status word
    is read (in a child process, so the environment is its own)."""
    code = (
        "import numpy as np, torch\n"
        "from paper_2203_02479_gb300 import wiresim as ws, inputs\n"
        "pl = ws.Plane(16, 300, inputs.response('bipolar'))\n"
        "d = ws.DeviceDepos(np.array([np.nan, 100.0], np.float32), np.array([10.0, 20.0], np.float32),"
        " np.array([50.0, 60.0], np.float32))\n"
        "pl.simulate(d, ws.Params())\n"
        "print('status', pl.status())\n")
    env = dict(os.environ, WS_LOG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "status 1" in r.stdout
    assert "wiresim: device status 0x1 bad-depo" in r.stderr
