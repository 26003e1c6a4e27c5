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


def test_precision_study_large_planes(ws):
    """Large three-plane detector (2560 / 2560 / 3840 wires x 6000 ticks, 2M
    track depos): every precision path against the FP64 oracle, per plane,
    in binomial mode (the workload) and expected-value mode (which isolates
    arithmetic error from the rare one-electron differences of the FP32
    normal branch).  Prints the table; bounds: FP32 and FP32_COMP 1e-5,
    FP64 1e-7.  Also counts the depos whose width falls under the narrow
    threshold (sigma < bin / 8 on an axis) that FP32_COMP takes in FP64."""
    import torch
    w = inputs.large_planes(n=2_000_000)
    modes = (("fp32", ws.WS_PREC_FP32, 1e-5), ("fp32_comp", ws.WS_PREC_FP32_COMP, 1e-5),
             ("fp64", ws.WS_PREC_FP64, 1e-7))
    t = w.events[0][0].t_us.astype(np.float64)
    st = np.sqrt(2 * oracle.DL * t) / oracle.V
    sx = np.sqrt(2 * oracle.DT * t)
    narrow = (st < oracle.TICK_US / 8) | (sx < oracle.PITCH_MM / 8)
    print(f"\nnarrow depos (FP64 edges under FP32_COMP): {narrow.mean():.4%}")
    for sp, d in zip(w.planes, w.events[0]):
        plane = ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id, fp64=True)
        dd = ws.DeviceDepos.from_plane_depos(d)
        for fluct in (True, False):
            S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=fluct, p=w.p_survive,
                                      seed=w.seed, plane_id=sp.plane_id)
            ref = oracle.convolve_fft(S, sp.response, 10)
            for name, prec, bound in modes:
                params = ws.Params(fluctuate=fluct, p_survive=w.p_survive, seed=w.seed, precision=prec)
                out = plane.simulate(dd, params)
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record()
                for _ in range(3):
                    plane.simulate(dd, params, out=out)
                t1.record()
                torch.cuda.synchronize()
                got = out.cpu().numpy().astype(np.float64)
                r = rel(got, ref)
                print(f"plane {sp.plane_id} ({sp.nwires} wires) {name:9s} {'binomial' if fluct else 'expected'}: "
                      f"rel L2 {r:.2e}, max abs {np.abs(got - ref).max():.2f} of {np.abs(ref).max():.3g}, "
                      f"{t0.elapsed_time(t1) / 3:.2f} ms")
                assert r <= bound, (sp.plane_id, name, fluct, r)
        plane.close()
