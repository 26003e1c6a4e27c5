"""GPU adjoint (ws_simulate_backward and the autograd wrapper) against the
FP64 oracle's gradients, which tests/test_oracle_adjoint_pins.py ties to
finite differences.

Tolerance: relative L2 <= 1e-4 for each gradient vector (gq, gx, gt, gR)
and for dL/dD_L, dL/dD_T.  The GPU chain runs in FP32 (FFT adjoint with
relative error ~1e-6 of ||dS||, erfc/exp weight derivatives at ~1e-6, sums
over ~25 bins per depo), so errors of a few 1e-6 are expected; 1e-4 leaves
room for gradients that nearly cancel.

Kinks: the raster's derivative jumps by about phi(3)/sigma where a window
bound mu +- 3 sigma crosses a bin edge.  A depo whose bound lies within
FP32 reach of an edge (1e-5 sigma here) has two valid one-sided
derivatives, and FP32 and FP64 may pick different sides; such depos are
checked for finiteness only and left out of the per-depo comparison.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-4


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def kink_mask(d, nsig=3.0, reach=1e-5):
    """Depos with a window bound within `reach` sigmas of a bin edge."""
    t = d.t_us.astype(np.float64); x = d.x_mm.astype(np.float64)
    st, sx = oracle.sigmas(t)
    m = np.zeros(t.shape[0], bool)
    for mu, sg, delta in ((t, st, oracle.TICK_US), (x, sx, oracle.PITCH_MM)):
        for sign in (-1.0, 1.0):
            b = (mu + sign * nsig * sg) / delta
            m |= np.abs(b - np.round(b)) * delta < reach * np.maximum(sg, 1e-30)
    return m


def compare(got, ref, mask):
    for name, g, r in zip(("gq", "gx", "gt"), got[:3], ref[:3]):
        g = np.asarray(g, np.float64)
        assert np.isfinite(g).all(), name
        assert rel(g[~mask], r[~mask]) <= TOL, (name, rel(g[~mask], r[~mask]))
    for name, g, r in zip(("gDL", "gDT", "gR"), got[3:], ref[3:]):
        assert rel(g, r) <= TOL, (name, rel(g, r))


def _case(ws, nw, nt, n, seed, circular=False, R=None, p=1.0):
    import torch
    d = inputs.uniform_depos(n, nw, seed, nticks=nt, t_min_us=1.0)
    R = inputs.response("bipolar") if R is None else R
    T = np.random.Generator(np.random.PCG64(seed + 1)).standard_normal((nw, nt)) * 20
    M = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, circular=circular, p=p)
    G = 2 * (M - T)
    ref = oracle.simulate_backward(d.q, d.x_mm, d.t_us, nw, nt, R, 10, G, circular=circular, p=p)
    plane = ws.Plane(nw, nt, R, circular=circular)
    got = plane.backward(ws.DeviceDepos.from_plane_depos(d), ws.Params(p_survive=p),
                         torch.from_numpy(G.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return [g.cpu().numpy() if hasattr(g, "cpu") else g for g in got], ref, kink_mask(d)


@pytest.mark.parametrize("circular", [False, True])
def test_backward_matches_oracle_small(ws, circular):
    got, ref, mask = _case(ws, 40, 1200, 300, 51, circular=circular, p=0.9)
    compare(got, ref, mask)


def test_backward_full_plane_20k_depos(ws):
    """960 x 6000 plane, 20,000 depos (t >= 1 us), loss sum (M - T)^2 with a
    target simulated at shifted parameters (x + 1.5 mm, q x 1.1, D_L x 1.2,
    D_T x 0.8, R x 0.9)."""
    import torch
    nw, nt = 960, 6000
    d = inputs.uniform_depos(20000, nw, 1003, nticks=nt, t_min_us=1.0)
    R = inputs.response("bipolar")
    T = oracle.simulate(d.q * np.float32(1.1), d.x_mm + np.float32(1.5), d.t_us, nw, nt, R * np.float32(0.9), 10,
                        DL_=oracle.DL * 1.2, DT_=oracle.DT * 0.8)
    M = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10)
    G = 2 * (M - T)
    ref = oracle.simulate_backward(d.q, d.x_mm, d.t_us, nw, nt, R, 10, G)
    plane = ws.Plane(nw, nt, R)
    got = plane.backward(ws.DeviceDepos.from_plane_depos(d), ws.Params(),
                         torch.from_numpy(G.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    got = [g.cpu().numpy() if hasattr(g, "cpu") else g for g in got]
    mask = kink_mask(d)
    assert mask.mean() < 1e-3
    compare(got, ref, mask)


def test_autograd_wrapper(ws):
    """Gradients through torch.autograd equal the direct backward call, and
    the forward equals ws_simulate."""
    import torch
    from paper_2203_02479_gb300 import autograd
    nw, nt = 32, 900
    d = inputs.uniform_depos(150, nw, 61, nticks=nt, t_min_us=1.0)
    R = torch.from_numpy(inputs.response("unipolar")).cuda().requires_grad_(True)
    plane = ws.Plane(nw, nt, R.detach())
    q = torch.from_numpy(d.q).cuda().requires_grad_(True)
    x = torch.from_numpy(d.x_mm).cuda().requires_grad_(True)
    t = torch.from_numpy(d.t_us).cuda().requires_grad_(True)
    DL = torch.tensor(4e-4, dtype=torch.float64, device="cuda", requires_grad=True)
    DT = torch.tensor(8.8e-4, dtype=torch.float64, device="cuda", requires_grad=True)
    target = torch.randn(nw, nt, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3)) * 10
    M = autograd.simulate(q, x, t, DL, DT, R, plane)
    loss = ((M - target) ** 2).sum()
    loss.backward()
    G = (2 * (M.detach() - target)).contiguous()
    gq, gx, gt, gDL, gDT, gR = plane.backward(ws.DeviceDepos.from_plane_depos(d), ws.Params(), G)
    torch.cuda.synchronize()
    for a, b in ((q.grad, gq), (x.grad, gx), (t.grad, gt), (R.grad, gR)):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6
    assert rel(DL.grad.cpu().numpy(), gDL.cpu().numpy()) <= 1e-6
    assert rel(DT.grad.cpu().numpy(), gDT.cpu().numpy()) <= 1e-6
    ref_m = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, inputs.response("unipolar"), 10)
    assert rel(M.detach().cpu().numpy(), ref_m) <= 1e-5


def test_autograd_two_forwards_with_different_responses(ws):
    """Two forwards on one plane under different responses (a prediction and
    a target) before one backward through both: each forward's gradients
    are taken under its own response, against the FP64 oracle's."""
    import torch
    from paper_2203_02479_gb300 import autograd
    nw, nt = 32, 900
    d = inputs.uniform_depos(150, nw, 62, nticks=nt, t_min_us=1.0)
    R1n = inputs.response("bipolar")
    R2n = (0.7 * inputs.response("unipolar")).astype(np.float32)
    R1 = torch.from_numpy(R1n).cuda().requires_grad_(True)
    R2 = torch.from_numpy(R2n).cuda().requires_grad_(True)
    plane = ws.Plane(nw, nt, R2n)
    q = torch.from_numpy(d.q).cuda().requires_grad_(True)
    x = torch.from_numpy(d.x_mm).cuda().requires_grad_(True)
    t = torch.from_numpy(d.t_us).cuda().requires_grad_(True)
    DL = torch.tensor(4e-4, dtype=torch.float64, device="cuda", requires_grad=True)
    DT = torch.tensor(8.8e-4, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.Generator(np.random.PCG64(63))
    T1 = rng.standard_normal((nw, nt)) * 20
    T2 = rng.standard_normal((nw, nt)) * 20
    M1 = autograd.simulate(q, x, t, DL, DT, R1, plane)
    M2 = autograd.simulate(q, x, t, DL, DT, R2, plane)
    # L = <M1, T1> + <M2, T2>: dL/dM1 = T1 and dL/dM2 = T2 exactly
    loss = (M1 * torch.from_numpy(T1.astype(np.float32)).cuda()).sum() + \
        (M2 * torch.from_numpy(T2.astype(np.float32)).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    A1 = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R1n, 10)
    A2 = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R2n, 10)
    assert rel(M1.detach().cpu().numpy(), A1) <= 1e-5
    assert rel(M2.detach().cpu().numpy(), A2) <= 1e-5
    # the two backward passes add up, each under its own response
    r1 = oracle.simulate_backward(d.q, d.x_mm, d.t_us, nw, nt, R1n, 10, T1.astype(np.float32).astype(np.float64))
    r2 = oracle.simulate_backward(d.q, d.x_mm, d.t_us, nw, nt, R2n, 10, T2.astype(np.float32).astype(np.float64))
    mask = kink_mask(d)
    for got, a, b in ((q.grad, r1[0], r2[0]), (x.grad, r1[1], r2[1]), (t.grad, r1[2], r2[2])):
        g = got.cpu().numpy()
        assert rel(g[~mask], (a + b)[~mask]) <= TOL
    assert rel(R1.grad.cpu().numpy(), r1[5]) <= TOL
    assert rel(R2.grad.cpu().numpy(), r2[5]) <= TOL
    assert rel(DL.grad.cpu().numpy(), r1[3] + r2[3]) <= TOL
    assert rel(DT.grad.cpu().numpy(), r1[4] + r2[4]) <= TOL


def test_backward_rejects_fluctuation(ws):
    import torch
    plane = ws.Plane(8, 300, inputs.response())
    d = ws.DeviceDepos([10.0], [12.0], [30.0])
    with pytest.raises(ws.WiresimError):
        plane.backward(d, ws.Params(fluctuate=True, p_survive=0.7), torch.zeros(8, 300, device="cuda"))


def test_backward_wide_patches_take_the_warp_path(ws):
    """Given widths: half the depos have patches wider than the
    lane-per-depo gradient kernel takes (handed over to the warp-per-depo
    kernel through the list), half narrow; every gradient against the
    oracle's."""
    import torch
    nw, nt, n = 64, 2000, 400
    d = inputs.uniform_depos(n, nw, 71, nticks=nt, t_min_us=1.0)
    rng = np.random.Generator(np.random.PCG64(72))
    wide = rng.uniform(size=n) < 0.5
    st = np.where(wide, rng.uniform(6.0, 12.0, n), rng.uniform(0.3, 1.0, n)).astype(np.float32)
    sx = np.where(wide, rng.uniform(15.0, 40.0, n), rng.uniform(0.5, 2.0, n)).astype(np.float32)
    R = inputs.response("bipolar")
    G = np.random.Generator(np.random.PCG64(73)).standard_normal((nw, nt))
    ref = oracle.simulate_backward(d.q, d.x_mm, d.t_us, nw, nt, R, 10, G, sig_t_us=st, sig_x_mm=sx)
    plane = ws.Plane(nw, nt, R)
    got = plane.backward(ws.DeviceDepos(d.q, d.x_mm, d.t_us, st, sx), ws.Params(),
                         torch.from_numpy(G.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    got = [g.cpu().numpy() if hasattr(g, "cpu") else g for g in got]
    m = np.zeros(n, bool)
    for mu, sg, delta in ((d.t_us.astype(np.float64), st.astype(np.float64), oracle.TICK_US),
                          (d.x_mm.astype(np.float64), sx.astype(np.float64), oracle.PITCH_MM)):
        for sign in (-1.0, 1.0):
            b = (mu + sign * 3.0 * sg) / delta
            m |= np.abs(b - np.round(b)) * delta < 1e-5 * sg
    for name, g, r in zip(("gq", "gx", "gt"), got[:3], ref[:3]):
        assert np.isfinite(g).all(), name
        for sel in (wide & ~m, ~wide & ~m):
            assert rel(g[sel], r[sel]) <= TOL, (name, rel(g[sel], r[sel]))
    assert rel(got[5], ref[5]) <= TOL
    assert plane.status() == 0


def _kinks_fine(d, I, nsig=3.0, reach=1e-5):
    """kink_mask on an impact plane: the pitch axis is binned at pitch / I."""
    t = d.t_us.astype(np.float64); x = d.x_mm.astype(np.float64)
    st, sx = oracle.sigmas(t)
    m = np.zeros(t.shape[0], bool)
    for mu, sg, delta in ((t, st, oracle.TICK_US), (x, sx, oracle.PITCH_MM / I)):
        for sign in (-1.0, 1.0):
            b = (mu + sign * nsig * sg) / delta
            m |= np.abs(b - np.round(b)) * delta < reach * np.maximum(sg, 1e-30)
    return m


@pytest.mark.parametrize("nw,nt,I,n,circular", [
    (48, 1200, 4, 600, False),      # generic transforms
    (40, 900, 3, 400, True),        # circular
    (96, 6000, 10, 2000, False),    # fixed-shape transforms, patches up to ~29 fine wires
])
def test_backward_on_impact_planes_matches_oracle(ws, nw, nt, I, n, circular):
    """dL/dS_fine by each position's correlation, the depo gradients on the
    fine grid and one response gradient per slice, against the oracle's
    impact adjoint (itself pinned by finite differences)."""
    import torch
    d = inputs.uniform_depos(n, nw, nw + I, nticks=nt, t_min_us=1.0)
    R = inputs.impact_response("bipolar", impacts=I)
    T = np.random.Generator(np.random.PCG64(nw)).standard_normal((nw, nt)) * 20
    M = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, nw, nt, R, 10, circular=circular)
    G = 2 * (M - T)
    ref = oracle.simulate_backward_impacts(d.q, d.x_mm, d.t_us, nw, nt, R, 10, G, circular=circular)
    plane = ws.Plane(nw, nt, R, circular=circular)
    got = plane.backward(ws.DeviceDepos.from_plane_depos(d), ws.Params(), torch.from_numpy(G.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    got = [g.cpu().numpy() if hasattr(g, "cpu") else g for g in got]
    assert got[5].shape == (I,) + R.shape[1:]
    compare(got, ref, _kinks_fine(d, I))
    assert plane.status() == 0
