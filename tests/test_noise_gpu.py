"""Noise term N(t, x) of Eq. 1 on the GPU against the FP64 oracle.

The GPU adds the noise spectra inside the inverse tick transform; the oracle
draws the same Philox words in C, forms the complex normals in double and
inverts with numpy.  The Box-Muller uniforms are exact on both sides (top 23
bits of a word), so the only differences are FP32 rounding of the normals
and of the transform: relative L2 <= 1e-5 as for the deterministic path,
<= 1e-7 on the FP64 path.  The transform length L given to the oracle is its
own fft_len of the plane (checked against the plane's choice).
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


def _plane(ws, nw, nt, circular=False, kind="bipolar", **kw):
    R = inputs.response(kind)
    L = oracle.fft_len(nt if circular else nt + R.shape[1] - 1)
    pl = ws.Plane(nw, nt, R, circular=circular, **kw)
    assert pl.info.fft_len_tick == L
    return pl, R, L


def _no_depos(ws):
    z = np.zeros(0, np.float32)
    return ws.DeviceDepos(z, z, z)


@pytest.mark.parametrize("nw,nt,circular,group", [
    (960, 6000, False, 32),    # L = 6250: the fixed-shape inverse kernel
    (45, 1000, False, 5),      # L = 1200 (fixed shape), odd wires, pairs straddling groups
    (33, 777, False, 1),       # L = 1000: the generic inverse kernel, group of one
    (20, 960, True, 3),        # circular, L = 960 (generic)
])
def test_noise_alone_matches_oracle(ws, nw, nt, circular, group):
    pl, R, L = _plane(ws, nw, nt, circular, plane_id=5)
    amp = inputs.noise_amplitudes(L)
    coh = inputs.noise_amplitudes(L, "coherent")
    pl.set_noise(amp, coh, group)
    params = ws.Params(seed=0x1234_5678_9ABC, event_id=77)
    got = to_np(pl.simulate(_no_depos(ws), params))
    ref = oracle.noise(nw, nt, L, amp, coh, group, seed=params.seed, event_id=77, plane_id=5)
    assert rel_l2(got, ref) <= REL_L2
    # incoherent part alone
    pl.set_noise(amp)
    got = to_np(pl.simulate(_no_depos(ws), params))
    ref = oracle.noise(nw, nt, L, amp, seed=params.seed, event_id=77, plane_id=5)
    assert rel_l2(got, ref) <= REL_L2
    assert pl.status() == 0


@pytest.mark.parametrize("fluct", [False, True])
def test_signal_plus_noise(ws, fluct):
    """The whole path with noise: raster (+ binomial), scatter, convolution
    and Eq. 1's noise term together."""
    nw, nt = 200, 6000
    pl, R, L = _plane(ws, nw, nt, plane_id=2)
    amp = inputs.noise_amplitudes(L, peak=2.0e4)
    coh = inputs.noise_amplitudes(L, "coherent", peak=2.0e4)
    pl.set_noise(amp, coh, 32)
    d = inputs.uniform_depos(3000, nw, seed=61, nticks=nt)
    params = ws.Params(fluctuate=fluct, p_survive=0.7, seed=99, event_id=4)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), params))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, fluctuate=fluct, p=0.7, seed=99, event_id=4,
                          plane_id=2, noise_amp=amp, noise_coh=coh, noise_group=32)
    # binomial mode: a few bins may differ by one electron (see the parity tests)
    assert rel_l2(got, ref) <= (REL_L2 if not fluct else 2e-5)
    if fluct:
        noise = oracle.noise(nw, nt, L, amp, coh, 32, seed=99, event_id=4, plane_id=2)
        sig = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, fluctuate=True, p=0.7, seed=99, event_id=4,
                              plane_id=2)
        assert rel_l2(got - sig, noise) <= 1e-2


def test_noise_off_restores_the_plain_path(ws):
    nw, nt = 64, 6000
    pl, R, L = _plane(ws, nw, nt)
    d = ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(500, nw, seed=3, nticks=nt))
    params = ws.Params(seed=5)
    plain = to_np(pl.simulate(d, params))
    pl.set_noise(inputs.noise_amplitudes(L))
    noisy = to_np(pl.simulate(d, params))
    assert rel_l2(noisy, plain) > 1e-3
    pl.set_noise(None)
    assert np.array_equal(to_np(pl.simulate(d, params)), plain)
    # the pure convolution never adds noise
    pl.set_noise(inputs.noise_amplitudes(L))
    import torch
    g = torch.zeros((nw, nt), dtype=torch.float32, device="cuda")
    assert not np.any(to_np(pl.convolve(g)))


def test_noise_fp64_path(ws):
    nw, nt = 30, 1000
    pl, R, L = _plane(ws, nw, nt, fp64=True, plane_id=1)
    amp = inputs.noise_amplitudes(L)
    coh = inputs.noise_amplitudes(L, "coherent")
    pl.set_noise(amp, coh, 4)
    d = inputs.uniform_depos(400, nw, seed=8, nticks=nt)
    params = ws.Params(seed=31, event_id=2, precision=ws.WS_PREC_FP64)
    got = to_np(pl.simulate(ws.DeviceDepos.from_plane_depos(d), params))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, seed=31, event_id=2, plane_id=1,
                          noise_amp=amp, noise_coh=coh, noise_group=4)
    assert rel_l2(got, ref) <= 1e-7


def test_batch_noise_equals_per_unit(ws):
    """ws_simulate_batch adds each unit's noise with its own event id."""
    import torch
    wires, nt = (40, 40, 48), 1500
    planes = [ws.Plane(nw, nt, inputs.response("bipolar" if i < 2 else "unipolar"), plane_id=i)
              for i, nw in enumerate(wires)]
    L = planes[0].info.fft_len_tick
    for i, pl in enumerate(planes):
        pl.set_noise(inputs.noise_amplitudes(L, peak=1e4 * (i + 1)), inputs.noise_amplitudes(L, "coherent"), 8)
    counts = [100, 0, 700]
    events = [[ws.DeviceDepos.from_plane_depos(inputs.uniform_depos(n, nw, 300 + 10 * e + p, nticks=nt))
               for p, nw in enumerate(wires)] for e, n in enumerate(counts)]
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=2024, event_id=9)
    b = ws.Batch(planes, events, params, units_per_wave=2)
    outs = b.run()
    torch.cuda.synchronize()
    for e in range(len(counts)):
        for p, pl in enumerate(planes):
            pe = ws.Params(**{**params.__dict__, "event_id": params.event_id + e})
            ref = to_np(pl.simulate(events[e][p], pe))
            assert rel_l2(to_np(outs[e * 3 + p]), ref) <= 1e-6, (e, p)
    # and one unit against the oracle's noise (no depos in event 1)
    ref = oracle.noise(40, nt, L, inputs.noise_amplitudes(L, peak=2e4), inputs.noise_amplitudes(L, "coherent"), 8,
                       seed=2024, event_id=10, plane_id=1)
    assert rel_l2(to_np(outs[1 * 3 + 1]), ref) <= REL_L2


def test_set_noise_argument_errors(ws):
    pl, R, L = _plane(ws, 8, 300)
    lib = ws.load_library()
    amp = inputs.noise_amplitudes(L)
    import torch
    a = torch.from_numpy(amp).cuda()
    assert lib.ws_plane_set_noise(pl.handle, a.data_ptr(), a.data_ptr(), 0, None) == 1   # coherent, no group
    assert lib.ws_plane_set_noise(pl.handle, 0, a.data_ptr(), 4, None) == 1      # coherent without incoherent
    with pytest.raises(ValueError):
        pl.set_noise(np.ones(L // 2, np.float32))


def test_noise_edge_cases(ws):
    """One wire (odd row count, a group wider than the plane), and the
    largest coherent group equal to the plane."""
    for nw, group in ((1, 48), (7, 7)):
        pl, R, L = _plane(ws, nw, 700)
        amp = inputs.noise_amplitudes(L)
        coh = inputs.noise_amplitudes(L, "coherent")
        pl.set_noise(amp, coh, group)
        got = to_np(pl.simulate(_no_depos(ws), ws.Params(seed=11)))
        ref = oracle.noise(nw, 700, L, amp, coh, group, seed=11)
        assert rel_l2(got, ref) <= REL_L2
