"""CUDA path against the FP64 oracle, element by element, on seeded inputs.

Tolerances:
  * expected-value (deterministic) mode: relative L2 <= 1e-5 of the whole
    grid, the bound the method is held to in FP32;
  * binomial mode: bins drawn on the exact branch are bit-identical except
    where FP32 and FP64 round q*w to different electron counts (those differ
    by at most one electron); normal-branch bins differ by at most one
    electron, in under 1% of bins; per-bin means and variances over seeds
    match the binomial's; simulated waveforms within relative L2 1e-5 of
    the oracle's (the one-electron differences move a waveform by ~1e-6).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
# Binomial waveforms: the FP32 transforms contribute ~5e-7 and the rare
# one-electron differences (bins where FP32 and FP64 round q*w to different
# counts, FP32 normal deviates) about as much; measured 1.0-1.4e-6 on the
# three-plane event, so 1e-5 leaves a factor of ~7 and fails a 1e-4 drift.
REL_L2_BINOMIAL = 1e-5


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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def gpu_grid_via_patches(ws, plane, d, params):
    patches = plane.rasterize(d, params)
    grid = plane.new_grid()
    plane.scatter(patches, grid)
    return patches, to_np(grid)


# ------------------------------------------------------------ convolution
@pytest.mark.parametrize("circular", [False, True])
@pytest.mark.parametrize("nw,nt,kw,kt,c", [(37, 1000, 21, 200, 10), (8, 300, 5, 17, 2),
                                           (30, 960, 21, 200, 10), (3, 125, 7, 11, 6),
                                           (131, 2048, 21, 200, 3)])
def test_convolve_matches_oracle(ws, circular, nw, nt, kw, kt, c):
    import torch
    rng = np.random.Generator(np.random.PCG64(nw * 1000 + nt + circular))
    S = rng.standard_normal((nw, nt)).astype(np.float32)
    R = rng.standard_normal((kw, kt)).astype(np.float32)
    if circular and nt not in (960, 125, 300, 1000, 2048):
        pytest.skip("circular needs a 2/3/5-smooth tick count")
    plane = ws.Plane(nw, nt, R, wire_center=c, circular=circular)
    out = plane.convolve(torch.from_numpy(S).cuda())
    ref = oracle.convolve_fft(S.astype(np.float64), R, c, circular)
    assert rel_l2(to_np(out), ref) <= REL_L2


@pytest.mark.parametrize("variant", list(range(10)))
@pytest.mark.parametrize("circular", [False, True])
def test_every_wire_conv_variant(ws, variant, circular):
    """Each wire-convolution kernel (wire blocks of 16 or 8, plain or
    Karatsuba taps, plain loads, TMA tiles or a TMA-fed chunk ring) gives
    the oracle's convolution, with a ragged wire tail; the TMA kernels are
    linear mode only."""
    import torch
    if circular and variant >= 4:
        pytest.skip("TMA tiles zero-fill outside the grid: linear mode only")
    rng = np.random.Generator(np.random.PCG64(40 + variant))
    nw, nt = 45 if variant < 4 else 311, 1000
    S = rng.standard_normal((nw, nt)).astype(np.float32)
    R = rng.standard_normal((21, 200)).astype(np.float32)
    plane = ws.Plane(nw, nt, R, circular=circular)
    plane.set_wire_conv_variant(variant)
    out = plane.convolve(torch.from_numpy(S).cuda())
    assert rel_l2(to_np(out), oracle.convolve_fft(S.astype(np.float64), R, 10, circular)) <= REL_L2


def test_convolve_in_place_and_delta_identity(ws):
    import torch
    rng = np.random.Generator(np.random.PCG64(3))
    S = rng.standard_normal((40, 777)).astype(np.float32)
    R = np.zeros((21, 200), np.float32); R[10, 0] = 1.0
    plane = ws.Plane(40, 777, R)
    g = torch.from_numpy(S).cuda()
    plane.convolve(g, out=g)            # in place
    assert rel_l2(to_np(g), S) <= 1e-6


def test_convolve_full_size_sampled_outputs(ws):
    """960 x 6000 plane: whole grid against Eq. 2 and sampled points against
    Eq. 1's direct sum."""
    import torch
    rng = np.random.Generator(np.random.PCG64(4))
    S = np.zeros((960, 6000), np.float32)
    S[:, :] = rng.exponential(1.0, S.shape) * (rng.uniform(size=S.shape) < 0.05)
    R = inputs.response("bipolar")
    plane = ws.Plane(960, 6000, R)
    out = to_np(plane.convolve(torch.from_numpy(S).cuda()))
    S64 = S.astype(np.float64)
    assert rel_l2(out, oracle.convolve_fft(S64, R, 10)) <= REL_L2
    pw = np.concatenate([[0, 959, 0, 959, 480], rng.integers(0, 960, 200)])
    pt = np.concatenate([[0, 0, 5999, 5999, 3000], rng.integers(0, 6000, 200)])
    pts = oracle.convolve_points(S64, R, 10, pw, pt)
    scale = np.abs(out).max()
    assert np.abs(out[pw, pt] - pts).max() <= 1e-5 * scale


# ------------------------------------------------------ raster + scatter
def test_rasterize_patches_match_oracle(ws):
    nw, nt = 70, 2500
    d = inputs.uniform_depos(3000, nw, seed=21, nticks=nt)
    plane = ws.Plane(nw, nt, inputs.response())
    dd = ws.DeviceDepos.from_plane_depos(d)
    params = ws.Params()
    patches, S = gpu_grid_via_patches(ws, plane, dd, params)
    ref = oracle.raster_scatter(d.q, d.x_mm, d.t_us, nw, nt)
    assert rel_l2(S, ref) <= 1e-6
    w0, nwv, t0, ntv, total = oracle.patch_extents(d.x_mm, d.t_us, nw, nt)
    g_nw = patches["nw"].cpu().numpy(); g_nt = patches["nt"].cpu().numpy()
    g_w0 = patches["w0"].cpu().numpy(); g_t0 = patches["t0"].cpu().numpy()
    same = (g_nw == nwv) & (g_nt == ntv) & ((g_w0 == w0) | (nwv == 0)) & ((g_t0 == t0) | (ntv == 0))
    # extents may differ only by a bin of zero weight where FP32 and FP64 put
    # a window edge on different sides of a bin edge
    assert same.mean() >= 0.995
    off = patches["off"].cpu().numpy()
    assert off[0] == 0 and (np.diff(off) == g_nw.astype(np.int64) * g_nt).all()
    assert abs(int(off[-1]) - total) <= 0.005 * total
    assert plane.status() == 0


def test_simulate_small_plane_expected_mode(ws):
    nw, nt = 48, 1500
    d = inputs.uniform_depos(400, nw, seed=22, nticks=nt)
    R = inputs.response("unipolar")
    plane = ws.Plane(nw, nt, R)
    out = to_np(plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params(p_survive=0.8)))
    ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, p=0.8)
    assert rel_l2(out, ref) <= REL_L2


def test_simulate_full_single_plane(ws):
    """960 wires x 6000 ticks, 1,000 uniform depos, bipolar response."""
    w = inputs.single_plane()
    sp = w.planes[0]; d = w.events[0][0]
    plane = ws.Plane(sp.nwires, sp.nticks, sp.response)
    out = to_np(plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params()))
    S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks)
    ref = oracle.convolve_fft(S, sp.response, 10)
    assert rel_l2(out, ref) <= REL_L2
    rng = np.random.Generator(np.random.PCG64(5))
    pw = rng.integers(0, sp.nwires, 300); pt = rng.integers(0, sp.nticks, 300)
    pts = oracle.convolve_points(S, sp.response, 10, pw, pt)
    assert np.abs(out[pw, pt] - pts).max() <= 1e-5 * np.abs(out).max()


def test_given_widths_and_large_patches(ws):
    """Explicit sigmas, including patches wider than one 64-bin chunk on both
    axes, point charges and depos straddling the grid edges."""
    nw, nt = 150, 900
    rng = np.random.Generator(np.random.PCG64(23))
    n = 60
    q = rng.exponential(3000, n).astype(np.float32)
    x = rng.uniform(-20, nw * 5 + 20, n).astype(np.float32)
    t = rng.uniform(-10, nt * 0.5 + 10, n).astype(np.float32)
    st = rng.choice([0.0, 0.05, 0.7, 12.0, 30.0], n).astype(np.float32)
    sx = rng.choice([0.0, 0.3, 2.0, 120.0], n).astype(np.float32)
    plane = ws.Plane(nw, nt, inputs.response())
    dd = ws.DeviceDepos(q, x, t, st, sx)
    _, S = gpu_grid_via_patches(ws, plane, dd, ws.Params())
    ref = oracle.raster_scatter(q, x, t, nw, nt, sig_t_us=st, sig_x_mm=sx)
    assert rel_l2(S, ref) <= 1e-6
    out = to_np(plane.simulate(dd, ws.Params()))
    assert rel_l2(out, oracle.convolve_fft(ref, inputs.response(), 10)) <= REL_L2


def test_edge_cases(ws):
    import torch
    nw, nt = 20, 400
    plane = ws.Plane(nw, nt, inputs.response())
    # no depos: all zeros
    empty = ws.DeviceDepos(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32))
    out = plane.simulate(empty, ws.Params())
    assert float(out.abs().max()) == 0.0
    # depos entirely off the grid: all zeros, no error
    off = ws.DeviceDepos([100.0, 100.0], [-50.0, 500.0], [10.0, 10.0])
    assert float(plane.simulate(off, ws.Params()).abs().max()) == 0.0
    assert plane.status() == 0
    # a NaN charge and a negative drift time are skipped and flagged
    bad = ws.DeviceDepos([np.nan, 100.0, 50.0], [10.0, 12.0, 20.0], [10.0, 30.0, -1.0])
    out = to_np(plane.simulate(bad, ws.Params()))
    assert plane.status() & ws.WS_DEV_BAD_DEPO
    ref = oracle.simulate([100.0], [12.0], [30.0], nw, nt, inputs.response(), 10)
    assert rel_l2(out, ref) <= REL_L2
    plane.clear_status()
    assert plane.status() == 0
    torch.cuda.synchronize()


def test_bad_given_widths_are_skipped_and_flagged(ws):
    """Given widths that are NaN, negative or infinite make the depo invalid:
    it is skipped and the status word says so; the valid depos are
    simulated as the oracle does."""
    nw, nt = 20, 400
    plane = ws.Plane(nw, nt, inputs.response())
    q = [100.0, 200.0, 300.0, 400.0, 500.0]
    x = [10.0, 30.0, 50.0, 70.0, 80.0]
    t = [20.0, 40.0, 60.0, 80.0, 100.0]
    st = [1.0, np.nan, -0.5, 1.5, 0.8]
    sx = [2.0, 1.0, 1.0, -np.inf, 3.0]
    out = to_np(plane.simulate(ws.DeviceDepos(q, x, t, st, sx), ws.Params()))
    assert plane.status() & ws.WS_DEV_BAD_DEPO
    keep = [0, 4]
    ref = oracle.simulate([q[i] for i in keep], [x[i] for i in keep], [t[i] for i in keep], nw, nt,
                          inputs.response(), 10, sig_t_us=[st[i] for i in keep], sig_x_mm=[sx[i] for i in keep])
    assert rel_l2(out, ref) <= REL_L2
    plane.clear_status()
    good = ws.DeviceDepos([q[i] for i in keep], [x[i] for i in keep], [t[i] for i in keep],
                          [st[i] for i in keep], [sx[i] for i in keep])
    assert rel_l2(to_np(plane.simulate(good, ws.Params())), out) <= 1e-6
    assert plane.status() == 0


def test_patch_capacity_overflow_is_flagged(ws):
    nw, nt = 30, 600
    d = inputs.uniform_depos(50, nw, seed=24, nticks=nt)
    plane = ws.Plane(nw, nt, inputs.response())
    dd = ws.DeviceDepos.from_plane_depos(d)
    need = plane.patch_capacity(dd, ws.Params())
    p = plane.rasterize(dd, ws.Params(), capacity=need // 2)
    assert plane.status() & 0x2
    nwv = p["nw"].cpu().numpy(); off = p["off"].cpu().numpy()
    written = nwv > 0
    assert (off[:-1][written] + nwv[written] * p["nt"].cpu().numpy()[written] <= need // 2).all()


def test_longest_transform(ws):
    """13,000 ticks: the tick transform length is 13,500 = 2^2 3^3 5^3."""
    nw, nt = 6, 13000
    d = inputs.uniform_depos(100, nw, seed=25, nticks=nt)
    R = inputs.response()
    plane = ws.Plane(nw, nt, R)
    assert plane.info.fft_len_tick == 13500
    out = to_np(plane.simulate(ws.DeviceDepos.from_plane_depos(d), ws.Params()))
    assert rel_l2(out, oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10)) <= REL_L2


# ------------------------------------------------------------ fluctuation
def _sparse_depos(n, nw, nt, seed, q_mean=400.0):
    """Depos on a lattice of 4-wire x 40-tick cells, one per cell near its
    centre, so no two patches (at most 13 ticks x 4 wires here) share a bin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cols, rows = nt // 40, nw // 4
    idx = rng.permutation(cols * rows)[:n]
    wi, ti = idx // cols, idx % cols
    x = (wi * 4 + 2) * 5.0 + rng.uniform(-2, 2, len(idx))
    t = (ti * 40 + 20) * 0.5 + rng.uniform(-3, 3, len(idx))
    q = rng.exponential(q_mean, len(idx)) + 5
    return q.astype(np.float32), x.astype(np.float32), np.maximum(t, 1.0).astype(np.float32)


def _boundary_mask(qw):
    """Bins whose expected electron count q*w lies within FP32 reach of
    n + 1/2, where FP32 and FP64 may round to different counts."""
    frac = qw - np.floor(qw)
    return np.abs(frac - 0.5) < 2e-6 * qw + 1e-5


@pytest.mark.parametrize("p", [0.7, 0.3, 0.5, 0.97])
def test_fluctuation_exact_branch_is_bit_exact(ws, p):
    """Exact branch (N <= 64 here): the CDF inversion takes the oracle's
    float decisions, so survivor counts are identical wherever FP32 and FP64
    agree on N; both sides' mirrored (p > 1/2) and direct searches."""
    nw, nt = 64, 3000
    q, x, t = _sparse_depos(300, nw, nt, 31)
    plane = ws.Plane(nw, nt, inputs.response(), plane_id=2)
    params = ws.Params(fluctuate=True, p_survive=p, seed=0xDEADBEEF12345, event_id=5, fluct_exact_max=64)
    _, S = gpu_grid_via_patches(ws, plane, ws.DeviceDepos(q, x, t), params)
    ref = oracle.raster_scatter(q, x, t, nw, nt, fluctuate=True, p=p, seed=0xDEADBEEF12345,
                                event_id=5, plane_id=2, exact_max=64)
    qw = oracle.raster_scatter(q, x, t, nw, nt)
    amb = _boundary_mask(qw)
    exact = (np.floor(qw + 0.5) <= 64) & ~amb
    assert (S[exact] == ref[exact]).all()
    assert np.abs(S - ref).max(initial=0) <= 1
    assert exact.sum() > 2000 and (S[exact] > 0).sum() > 1000


def test_fluctuation_normal_branch_within_one(ws):
    nw, nt = 64, 3000
    q, x, t = _sparse_depos(300, nw, nt, 32, q_mean=6000.0)
    plane = ws.Plane(nw, nt, inputs.response())
    params = ws.Params(fluctuate=True, p_survive=0.7, seed=99)
    _, S = gpu_grid_via_patches(ws, plane, ws.DeviceDepos(q, x, t), params)
    ref = oracle.raster_scatter(q, x, t, nw, nt, fluctuate=True, p=0.7, seed=99)
    qw = oracle.raster_scatter(q, x, t, nw, nt)
    amb = _boundary_mask(qw)
    exact = (np.floor(qw + 0.5) <= 32) & ~amb
    assert (S[exact] == ref[exact]).all()
    normal = np.floor(qw + 0.5) > 32
    diff = np.abs(S - ref)
    assert diff.max() <= 1
    assert (diff[normal] > 0).mean() < 0.01
    assert normal.sum() > 1000


def test_fluctuation_moments_over_seeds(ws):
    """Per-bin mean and variance of the survivor counts over seeds against
    p N and N p (1 - p) with N from the oracle's expected charges."""
    nw, nt = 16, 800
    q, x, t = _sparse_depos(20, nw, nt, 33, q_mean=2000.0)
    plane = ws.Plane(nw, nt, inputs.response())
    dd = ws.DeviceDepos(q, x, t)
    qw = oracle.raster_scatter(q, x, t, nw, nt)
    N = np.floor(qw + 0.5)
    m = N > 0
    K = 400
    acc = np.zeros(m.sum()); acc2 = np.zeros(m.sum())
    for s in range(K):
        _, S = gpu_grid_via_patches(ws, plane, dd, ws.Params(fluctuate=True, p_survive=0.7, seed=s))
        acc += S[m]; acc2 += S[m] ** 2
    mean = acc / K
    var = acc2 / K - mean ** 2
    p = 0.7
    z = (mean - N[m] * p) / np.sqrt(N[m] * p * (1 - p) / K)
    assert np.abs(z).max() < 5.5
    big = N[m] >= 20
    ratio = var[big] / (N[m][big] * p * (1 - p))
    assert abs(np.median(ratio) - 1) < 0.1


def test_three_planes_fluctuated_full_size(ws):
    """The three-plane workload at full size (100k track depos, binomial
    fluctuation): raster S bin by bin, and the simulated waveforms."""
    w = inputs.three_planes()
    for sp, d in zip(w.planes, w.events[0]):
        plane = ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id)
        dd = ws.DeviceDepos.from_plane_depos(d)
        params = ws.Params(fluctuate=True, p_survive=w.p_survive, seed=w.seed)
        _, S = gpu_grid_via_patches(ws, plane, dd, params)
        ref = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=True,
                                    p=w.p_survive, seed=w.seed, plane_id=sp.plane_id)
        diff = np.abs(S - ref)
        # overlapping patches: a bin sums several depos, each exact or off by one
        assert (diff > 0).mean() < 0.01
        assert diff.max() <= 4
        assert abs(S.sum() - ref.sum()) <= 1e-4 * ref.sum()
        out = to_np(plane.simulate(dd, params))
        ref_m = oracle.convolve_fft(ref, sp.response, 10)
        assert rel_l2(out, ref_m) <= REL_L2_BINOMIAL
        assert plane.status() == 0


@pytest.mark.parametrize("nw,nt,kt,circular,L,fixed", [
    (311, 6000, 200, False, 6250, 1), (7, 6000, 200, True, 6000, 1), (160, 6300, 101, False, 6400, 1),
    (305, 3000, 200, False, 3200, 1), (1, 1000, 200, False, 1200, 1), (33, 1900, 200, False, 2160, 0)])
def test_fixed_shape_row_transforms(ws, nw, nt, kt, circular, L, fixed):
    """Row kernels compiled for one radix plan (25.25.10, 25.16.15, 25.16.16,
    25.16.8, 25.16.3) and the generic kernels: odd wire counts leave a lone
    last row; more row pairs than resident CTAs."""
    import torch
    rng = np.random.Generator(np.random.PCG64(nw + nt))
    S = rng.standard_normal((nw, nt)).astype(np.float32)
    R = rng.standard_normal((21, kt)).astype(np.float32)
    plane = ws.Plane(nw, nt, R, circular=circular)
    assert plane.info.fft_len_tick == L
    assert plane.info.row_fft_fixed_shape == fixed
    out = plane.convolve(torch.from_numpy(S).cuda())
    assert rel_l2(to_np(out), oracle.convolve_fft(S.astype(np.float64), R, 10, circular)) <= REL_L2
    assert plane.status() == 0


def test_shift_equivariance_by_whole_bins(ws):
    """Depos moved by one pitch (one tick, with given widths) give the grid
    moved by one wire row (tick column).  The coordinates stay inside one
    binade ([32, 64) mm, [64, 128) us), so the moved values are exact in
    float and so are the edge offsets e - mu: only the order of the
    scatter's float additions differs."""
    import torch
    rng = np.random.Generator(np.random.PCG64(63))
    nw, nt, n = 16, 300, 2000
    q = rng.exponential(5000, n).astype(np.float32)
    x = rng.uniform(33.0, 58.0, n).astype(np.float32)
    t = rng.uniform(66.0, 127.0, n).astype(np.float32)
    st = rng.uniform(0.2, 2.0, n).astype(np.float32)
    sx = rng.uniform(0.3, 3.0, n).astype(np.float32)
    plane = ws.Plane(nw, nt, inputs.response("bipolar"))
    params = ws.Params()

    def grid(xx, tt):
        d = ws.DeviceDepos(q, xx, tt, st, sx)
        return gpu_grid_via_patches(ws, plane, d, params)[1]

    S = grid(x, t)
    Sx = grid(x + np.float32(5.0), t)
    St = grid(x, t + np.float32(0.5))
    assert rel_l2(Sx[1:], S[:-1]) <= 1e-6
    assert rel_l2(St[:, 1:], S[:, :-1]) <= 1e-6


def test_binding_checks_tensor_arguments_before_the_call(ws):
    """Tensors of the wrong shape, dtype or layout never reach the library:
    the binding raises ValueError first and the plane stays usable."""
    import torch
    R = inputs.response("bipolar")
    plane = ws.Plane(8, 300, R)
    with pytest.raises(ValueError, match="shape"):
        plane.convolve(torch.zeros((8, 299), device="cuda"))
    with pytest.raises(ValueError, match="dtype"):
        plane.convolve(torch.zeros((8, 300), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError, match="contiguous"):
        plane.convolve(torch.zeros((300, 8), device="cuda").t())
    with pytest.raises(ValueError, match="shape"):
        plane.set_response(R[:, :199])
    d = ws.DeviceDepos([3000.0], [20.0], [40.0])
    with pytest.raises(ValueError, match="shape"):
        plane.simulate(d, ws.Params(), out=torch.empty((16, 150), device="cuda"))
    with pytest.raises(ValueError, match="shape"):
        plane.backward(d, ws.Params(), torch.zeros((8, 301), device="cuda"))
    out = plane.simulate(d, ws.Params())
    assert plane.status() == 0 and float(out.abs().sum()) > 0


def test_three_planes_in_the_benchmark_launch_configuration(ws):
    """The benchmark's step at full size: the three-plane event (100k track
    depos, binomial fluctuation) through ws_simulate_batch captured into a
    CUDA graph and replayed, one plane per wave on three streams (the
    schedule the benchmark picks), and two or three planes per wave;
    waveforms against the oracle's."""
    import torch
    w = inputs.three_planes()
    planes = [ws.Plane(sp.nwires, sp.nticks, sp.response, plane_id=sp.plane_id) for sp in w.planes]
    depos = [ws.DeviceDepos.from_plane_depos(d) for d in w.events[0]]
    params = ws.Params(fluctuate=True, p_survive=w.p_survive, seed=w.seed)
    outs = {}
    for upw in (1, 2, 3):
        b = ws.Batch(planes, [depos], params, units_per_wave=upw)
        b.capture()
        for o in b.outs:
            o.fill_(float("nan"))
        b.replay()
        b.replay()
        torch.cuda.synchronize()
        outs[upw] = [o.cpu().numpy() for o in b.outs]
    for p, (sp, d) in enumerate(zip(w.planes, w.events[0])):
        S = oracle.raster_scatter(d.q, d.x_mm, d.t_us, sp.nwires, sp.nticks, fluctuate=True,
                                  p=w.p_survive, seed=w.seed, plane_id=sp.plane_id)
        M = oracle.convolve_fft(S, sp.response, 10)
        for upw in (1, 2, 3):
            assert np.isfinite(outs[upw][p]).all()
            assert rel_l2(outs[upw][p], M) <= REL_L2_BINOMIAL, (upw, p)
            assert rel_l2(outs[upw][p], outs[1][p]) <= 1e-6
    for pl in planes:
        assert pl.status() == 0
