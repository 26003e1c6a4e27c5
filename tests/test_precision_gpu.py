"""Precision paths of ws_simulate against the FP64 oracle.

* WS_PREC_FP64 computes widths, bin ranges, weights, binomial tails, the
  grid and both transforms in double, so it follows the oracle to the
  rounding of its float output grid: relative L2 <= 1e-7 (float rounding
  is ~3e-8 RMS) and every sample within 2 float ulps of the grid maximum.
  Binomial draws are then the same integers as the oracle's.
* WS_PREC_FP32_COMP (compensated scatter, FP64 narrow-axis weights) is held
  to the FP32 bound, relative L2 <= 1e-5.
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("circular", [False, True])
def test_fp64_expected_mode(ws, circular):
    import torch
    nw, nt = 64, 3000
    d = inputs.uniform_depos(2000, nw, 301, nticks=nt)
    R = inputs.response("bipolar")
    plane = ws.Plane(nw, nt, R, circular=circular, fp64=True)
    out = plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(precision=ws.WS_PREC_FP64, p_survive=0.9))
    torch.cuda.synchronize()
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, circular=circular, p=0.9)
    # the output grid is float: compare at the float rounding of the result
    assert rel(out.cpu().numpy(), ref) <= 1e-7
    assert np.abs(out.cpu().numpy() - ref.astype(np.float32)).max() <= 2 * np.abs(ref).max() * 2 ** -24


def test_fp64_binomial_matches_oracle_integers(ws):
    """FP64 path: the scattered counts equal the oracle's, so the simulated
    waveform is the oracle's convolution of identical integers."""
    import torch
    w = inputs.three_planes(n=20000, seed=303)
    sp, d = w.planes[2], w.events[0][2]
    plane = ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=2, fp64=True)
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=w.seed, precision=ws.WS_PREC_FP64)
    out = plane.simulate(ws.DeviceDepos.from_plane_depos(d), params)
    torch.cuda.synchronize()
    S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=True, p=0.7, seed=w.seed,
                              plane_id=2)
    ref = oracle.convolve_fft(S, sp.response, 10)
    assert rel(out.cpu().numpy(), ref) <= 1e-7


def test_compensated_mode(ws):
    import torch
    nw, nt = 96, 2000
    d = inputs.uniform_depos(5000, nw, 302, nticks=nt)
    R = inputs.response("unipolar")
    plane = ws.Plane(nw, nt, R)
    out = plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(precision=ws.WS_PREC_FP32_COMP))
    torch.cuda.synchronize()
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10)
    assert rel(out.cpu().numpy(), ref) <= 1e-5


def test_fp64_needs_fp64_workspace(ws):
    plane = ws.Plane(8, 300, inputs.response())
    d = ws.DeviceDepos([10.0], [12.0], [30.0])
    with pytest.raises(ws.WiresimError) as ei:
        plane.simulate(d, ws.Params(precision=ws.WS_PREC_FP64))
    assert ei.value.status == 6
