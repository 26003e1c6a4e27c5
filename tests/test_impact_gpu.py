"""Sub-pitch impact positions and long responses on the GPU, against the
FP64 oracle.

An impact plane bins the pitch axis at pitch / I (fine row w*I + i) and
convolves each sub-position's rows with its own response slice,
M = sum_i R_i (*) S_i; the oracle does the same with its own raster on the
finer grid and numpy's FFT per slice.  Expected-value mode: relative L2
<= 1e-5; binomial mode: the whole waveform within 1e-4 (rare one-electron
differences, as in the plain path).
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2203_02479_gb300 import build, wiresim
    build.build()
    wiresim.load_library()
    torch.cuda.set_device(0)
    return wiresim


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nw,nt,I,circular,fluct", [
    (240, 6000, 10, False, False),     # fixed-shape transforms, 2400 fine rows
    (45, 1000, 3, True, False),        # odd wires, circular, generic transform
    (64, 2000, 6, False, True),        # binomial fluctuation on the fine bins
])
def test_impact_simulate_matches_oracle(ws, nw, nt, I, circular, fluct):
    R = inputs.impact_response("bipolar", impacts=I)
    pl = ws.Plane(nw, nt, R, circular=circular, plane_id=1)
    assert pl.impacts == I
    d = inputs.uniform_depos(4000, nw, seed=nw + I, nticks=nt)
    params = ws.Params(fluctuate=fluct, p_survive=0.7, seed=55, event_id=3)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), params))
    ref = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, nw, nt, R, 10, circular=circular, fluctuate=fluct, p=0.7,
                                  seed=55, event_id=3, plane_id=1)
    assert rel_l2(got, ref) <= (1e-4 if fluct else REL_L2)
    assert pl.status() == 0


def test_equal_slices_equal_the_plain_plane(ws):
    nw, nt, I = 96, 3000, 5
    R = inputs.response("unipolar")
    plain = ws.Plane(nw, nt, R)
    imp = ws.Plane(nw, nt, np.ascontiguousarray(np.broadcast_to(R, (I,) + R.shape)))
    d = ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(3000, nw, seed=5, nticks=nt))
    params = ws.Params(seed=1)
    assert rel_l2(to_np(imp.simulate(d, params)), to_np(plain.simulate(d, params))) <= REL_L2


def test_impact_convolve_and_patches_on_the_fine_grid(ws):
    """ws_rasterize / ws_scatter fill the fine grid and ws_convolve takes it."""
    nw, nt, I = 30, 1200, 4
    R = inputs.impact_response("unipolar", impacts=I)
    pl = ws.Plane(nw, nt, R)
    d = inputs.uniform_depos(600, nw, seed=12, nticks=nt)
    params = ws.Params(p_survive=0.9)
    patches = pl.rasterize(ws.DeviceDepos.from_plane_depos(d), params)
    fine = pl.new_grid()
    assert tuple(fine.shape) == (nw * I, nt)
    pl.scatter(patches, fine)
    S = oracle.raster_scatter_impacts(d.q, d.x_mm, d.t_us, nw, nt, I, p=0.9)
    assert rel_l2(to_np(fine), S) <= 1e-6
    M = pl.convolve(fine)
    assert rel_l2(to_np(M), oracle.convolve_impacts(S, R, 10)) <= REL_L2
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(ws.WiresimError):      # the library refuses an output on the fine input
        ws.ws_convolve(pl.handle, fine.data_ptr(), fine.data_ptr(), stream)
    with pytest.raises(ValueError):           # the binding checks the output's shape before the call
        pl.convolve(fine, out=fine)


def test_impact_planes_rejected_where_unsupported(ws):
    R = inputs.impact_response("bipolar", impacts=4)
    pl = ws.Plane(16, 500, R)
    d = ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(10, 16, seed=1, nticks=500))
    with pytest.raises(ws.WiresimError):
        pl.simulate(d, ws.Params(precision=ws.WS_PREC_FP64))
    with pytest.raises(ws.WiresimError):
        pl.set_wire_conv_variant(4)      # impact planes: four tile shapes (0 .. 3)
    import torch
    with pytest.raises(ws.WiresimError):  # the adjoint is of the expected-value path
        pl.backward(d, ws.Params(fluctuate=1), torch.zeros((16, 500), device="cuda"))


@pytest.mark.parametrize("kt", [1000, 1500])
def test_long_response(ws, kt):
    """A response of 1000+ ticks: L_t = 7200 (1000) or 7500 (1500), generic
    transform kernels, against the oracle's full linear convolution."""
    nw, nt = 128, 6000
    R = inputs.response("bipolar", nticks=kt, tick_peak=kt / 2, tick_sigma=kt / 20)
    pl = ws.Plane(nw, nt, R)
    assert pl.info.fft_len_tick == oracle.fft_len(nt + kt - 1)
    d = inputs.uniform_depos(2000, nw, seed=kt, nticks=nt)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params()))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10)
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("I", [2, 32])
def test_impact_count_limits(ws, I):
    """The smallest and largest sub-pitch position counts, depos partly off
    the grid on both sides."""
    nw, nt = 12, 900
    R = inputs.impact_response("unipolar", impacts=I)
    pl = ws.Plane(nw, nt, R)
    rng = np.random.Generator(np.random.PCG64(I))
    q = rng.exponential(5000, 300).astype(np.float32)
    x = rng.uniform(-10, nw * 5.0 + 10, 300).astype(np.float32)
    t = rng.uniform(1, nt * 0.5, 300).astype(np.float32)
    got = to_np(pl.simulate(ws.DeviceDepos(q, x, t), ws.Params()))
    ref = oracle.simulate_impacts(q, x, t, nw, nt, R, 10)
    assert rel_l2(got, ref) <= REL_L2


def test_impact_count_above_limit_rejected(ws):
    R = inputs.impact_response("unipolar", impacts=33, nwires=3, nticks=10, wire_center=1)
    with pytest.raises(ws.WiresimError):
        ws.Plane(4, 100, R, wire_center=1)
