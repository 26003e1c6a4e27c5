"""Pins of the oracle's adjoint (expected-value mode) against the oracle's
own forward, which the other pins fix independently:

* the convolution adjoint and the response gradient by the dot-product
  identities <A S, G> = <S, A^T G> and <dL/dR, dR> = <G, A_dR S> (exact up
  to rounding, so a dropped term, a sign or an index shift fails);
* the per-depo and diffusion-constant gradients by central finite
  differences of the forward raster, with a Richardson check that the
  difference quotient has converged.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02479_gb300 import inputs


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("circular", [False, True])
@pytest.mark.parametrize("shape,rshape,c", [((14, 60), (5, 9), 1), ((9, 40), (7, 13), 5),
                                            ((30, 300), (21, 200), 10)])
def test_convolution_adjoint_dot_product(circular, shape, rshape, c):
    rng = _rng(sum(shape) + c)
    S = rng.standard_normal(shape)
    G = rng.standard_normal(shape)
    R = rng.standard_normal(rshape).astype(np.float32)
    lhs = np.vdot(oracle.convolve_fft(S, R, c, circular), G)
    rhs = np.vdot(S, oracle.convolve_adjoint(G, R, c, circular))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_convolution_adjoint_is_direct_correlation():
    """Tiny case: the adjoint equals its definition written as loops."""
    rng = _rng(3)
    G = rng.standard_normal((6, 11))
    R = rng.standard_normal((3, 4)).astype(np.float32)
    c = 1
    ref = np.zeros_like(G)
    for w in range(6):
        for t in range(11):
            for r in range(3):
                for j in range(4):
                    ww, tt = w + r - c, t + j
                    if 0 <= ww < 6 and tt < 11:
                        ref[w, t] += float(R[r, j]) * G[ww, tt]
    np.testing.assert_allclose(oracle.convolve_adjoint(G, R, c), ref, atol=1e-12)


@pytest.mark.parametrize("circular", [False, True])
def test_response_gradient_dot_product(circular):
    rng = _rng(5 + circular)
    S = rng.standard_normal((12, 80))
    G = rng.standard_normal((12, 80))
    kw, kt, c = 5, 17, 3
    dR = rng.standard_normal((kw, kt))
    gR = oracle.response_grad(G, S, kw, kt, c, circular)
    assert np.vdot(gR, dR) == pytest.approx(np.vdot(G, oracle.convolve_fft(S, dR, c, circular)), rel=1e-11)


def _loss_s(G, q, x, t, nw, nt, DL=oracle.DL, DT=oracle.DT, p=1.0):
    return float(np.vdot(G, oracle.raster_scatter(q, x, t, nw, nt, DL_=DL, DT_=DT, p=p)))


def _fd(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return d2, abs(d2 - d1)


def test_depo_gradients_match_finite_differences():
    nw, nt = 24, 2000
    rng = _rng(7)
    n = 6
    q = rng.uniform(1000, 8000, n)
    x = rng.uniform(20, 100, n)
    t = rng.uniform(100, 990, n)
    G = rng.standard_normal((nw, nt))
    p = 0.8
    gq, gx, gt, gDL, gDT = oracle.depo_grads(q, x, t, nw, nt, G, p=p)
    for i in range(n):
        for arr, g, h in ((q, gq, 1e-3), (x, gx, 1e-6), (t, gt, 1e-6)):
            def f(d, arr=arr):
                a = arr.copy()
                a[i] += d
                args = {"q": q, "x": x, "t": t}
                args = [a if arr is v else v for v in (q, x, t)]
                return _loss_s(G, *args, nw, nt, p=p)
            est, err = _fd(f, h)
            assert g[i] == pytest.approx(est, rel=1e-5, abs=1e-6 * max(1.0, abs(est)) + 10 * err)
    for which, g, base in (("DL", gDL, oracle.DL), ("DT", gDT, oracle.DT)):
        h = base * 1e-6

        def f(d, which=which):
            kw = {"DL": oracle.DL, "DT": oracle.DT}
            kw[which] += d
            return _loss_s(G, q, x, t, nw, nt, kw["DL"], kw["DT"], p)
        est, err = _fd(f, h)
        assert g == pytest.approx(est, rel=1e-5, abs=10 * err)


def test_full_backward_matches_finite_differences_of_the_loss():
    """L = sum (M - T)^2 through raster and convolution; gradients for q, x,
    t of two depos, D_L, D_T and two response entries."""
    nw, nt = 16, 800
    R = inputs.response("bipolar", nwires=5, nticks=40, wire_center=2, tick_peak=15.0, tick_sigma=4.0)
    R = R.astype(np.float64)
    q = np.array([3000.0, 5000.0]); x = np.array([31.0, 47.3]); t = np.array([150.2, 301.7])
    T = _rng(9).standard_normal((nw, nt)) * 50

    def loss(q=q, x=x, t=t, DL=oracle.DL, DT=oracle.DT, R=R):
        M = oracle.simulate(q, x, t, nw, nt, R, 2, DL_=DL, DT_=DT)
        return float(((M - T) ** 2).sum())

    M = oracle.simulate(q, x, t, nw, nt, R, 2)
    G = 2 * (M - T)
    gq, gx, gt, gDL, gDT, gR = oracle.simulate_backward(q, x, t, nw, nt, R, 2, G)
    for i in range(2):
        for name, g, h in (("q", gq, 1e-2), ("x", gx, 1e-6), ("t", gt, 1e-6)):
            def f(d, name=name):
                v = {"q": q.copy(), "x": x.copy(), "t": t.copy()}
                v[name][i] += d
                return loss(**v)
            est, err = _fd(f, h)
            assert g[i] == pytest.approx(est, rel=2e-5, abs=10 * err + 1e-6)
    est, err = _fd(lambda d: loss(DL=oracle.DL + d), oracle.DL * 1e-6)
    assert gDL == pytest.approx(est, rel=2e-5, abs=10 * err)
    est, err = _fd(lambda d: loss(DT=oracle.DT + d), oracle.DT * 1e-6)
    assert gDT == pytest.approx(est, rel=2e-5, abs=10 * err)
    for (r, j) in ((2, 15), (0, 3)):
        def f(d, r=r, j=j):
            R2 = R.copy()
            R2[r, j] += d
            return loss(R=R2)
        est, err = _fd(f, 1e-3)
        assert gR[r, j] == pytest.approx(est, rel=1e-6, abs=10 * err)


@pytest.mark.parametrize("circular", [False, True])
def test_impact_backward_matches_finite_differences_of_the_loss(circular):
    """An impact plane (I = 3 sub-pitch positions, slices that differ):
    L = sum (M - T)^2 through the fine raster and the per-position
    convolution; gradients for q, x, t of two depos (one near a sub-pitch
    boundary), D_L, D_T and response entries of two slices."""
    nw, nt, I, c = 12, 600, 3, 2
    R = inputs.impact_response("bipolar", impacts=I, nwires=5, nticks=40, wire_center=c, tick_peak=15.0,
                               tick_sigma=4.0).astype(np.float64)
    R[1] *= 1.3                      # slices of different size as well as shape
    q = np.array([3000.0, 5000.0]); x = np.array([23.0, 31.62]); t = np.array([150.2, 301.7])
    T = _rng(19).standard_normal((nw, nt)) * 50

    def loss(q=q, x=x, t=t, DL=oracle.DL, DT=oracle.DT, R=R):
        M = oracle.simulate_impacts(q, x, t, nw, nt, R, c, circular=circular, DL_=DL, DT_=DT)
        return float(((M - T) ** 2).sum())

    M = oracle.simulate_impacts(q, x, t, nw, nt, R, c, circular=circular)
    G = 2 * (M - T)
    gq, gx, gt, gDL, gDT, gR = oracle.simulate_backward_impacts(q, x, t, nw, nt, R, c, G, circular=circular)
    assert gR.shape == R.shape
    for i in range(2):
        for name, g, h in (("q", gq, 1e-2), ("x", gx, 1e-6), ("t", gt, 1e-6)):
            def f(d, name=name):
                v = {"q": q.copy(), "x": x.copy(), "t": t.copy()}
                v[name][i] += d
                return loss(**v)
            est, err = _fd(f, h)
            assert g[i] == pytest.approx(est, rel=2e-5, abs=10 * err + 1e-6), (name, i)
    est, err = _fd(lambda d: loss(DL=oracle.DL + d), oracle.DL * 1e-6)
    assert gDL == pytest.approx(est, rel=2e-5, abs=10 * err)
    est, err = _fd(lambda d: loss(DT=oracle.DT + d), oracle.DT * 1e-6)
    assert gDT == pytest.approx(est, rel=2e-5, abs=10 * err)
    for (s_, r, j) in ((0, 2, 15), (2, 1, 20), (1, 4, 8)):
        def f(d, s_=s_, r=r, j=j):
            R2 = R.copy()
            R2[s_, r, j] += d
            return loss(R=R2)
        est, err = _fd(f, 1e-3)
        assert gR[s_, r, j] == pytest.approx(est, rel=1e-6, abs=10 * err), (s_, r, j)


def test_impact_backward_with_equal_slices_is_the_plain_backward():
    """Equal slices make the impact plane the plain one (the fine rows of a
    wire sum to its coarse bin), so the depo and diffusion gradients agree
    with the plain adjoint and each slice's response gradient is the plain
    one's share over that position's rows (they sum to it)."""
    nw, nt, I, c = 10, 500, 4, 2
    R = inputs.response("unipolar", nwires=5, nticks=30, wire_center=c, tick_peak=10.0, tick_sigma=3.0)
    R = R.astype(np.float64)
    RI = np.broadcast_to(R, (I,) + R.shape).copy()
    rng = _rng(23)
    q = rng.uniform(1000, 6000, 5); x = rng.uniform(5, 45, 5); t = rng.uniform(50, 240, 5)
    G = rng.standard_normal((nw, nt))
    plain = oracle.simulate_backward(q, x, t, nw, nt, R, c, G)
    imp = oracle.simulate_backward_impacts(q, x, t, nw, nt, RI, c, G)
    for a, b in zip(plain[:5], imp[:5]):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-9 * np.max(np.abs(a)))
    assert np.allclose(imp[5].sum(axis=0), plain[5], rtol=1e-9, atol=1e-9 * np.max(np.abs(plain[5])))
