"""Pins of the oracle's sub-pitch impact sampling (CPU).

Reading (in the oracle): the pitch axis is binned at pitch / I, fine row
w * I + i holding the charge at sub-position i of wire w, and the response
has one slice per sub-position: M = sum_i R_i (*) S_i.  Pinned by the fine
rows summing to the coarse raster, the point charge landing in its
sub-position, equal slices reducing to the plain convolution, and the
direct sum of Eq. 1.
"""
import numpy as np

import oracle
from paper_2203_02479_gb300 import inputs


def test_fine_rows_sum_to_the_coarse_bins():
    rng = np.random.Generator(np.random.PCG64(2))
    nw, nt, I = 20, 300, 10
    q = rng.exponential(5000, 200); x = rng.uniform(-5, nw * 5 + 5, 200); t = rng.uniform(1, nt * 0.5, 200)
    fine = oracle.raster_scatter_impacts(q, x, t, nw, nt, I, p=0.8)
    coarse = oracle.raster_scatter(q, x, t, nw, nt, p=0.8)
    assert np.allclose(fine.reshape(nw, I, nt).sum(axis=1), coarse, rtol=1e-12, atol=1e-9)


def test_point_charge_lands_in_its_sub_position():
    nw, nt, I = 8, 200, 5
    for i in range(I):
        x = 3 * 5.0 + (i + 0.5) * 5.0 / I
        S = oracle.raster_scatter_impacts([1000.0], [x], [40.0], nw, nt, I, sig_t_us=[0.8], sig_x_mm=[0.0])
        rows = np.nonzero(S.sum(axis=1))[0]
        assert list(rows) == [3 * I + i]
        assert abs(S.sum() - 1000.0) < 1e-9


def test_equal_slices_reduce_to_the_plain_convolution():
    rng = np.random.Generator(np.random.PCG64(3))
    nw, nt, I = 12, 250, 4
    S_fine = rng.standard_normal((nw * I, nt))
    R = rng.standard_normal((5, 30))
    Ri = np.broadcast_to(R, (I,) + R.shape)
    got = oracle.convolve_impacts(S_fine, Ri, 2)
    ref = oracle.convolve_fft(S_fine.reshape(nw, I, nt).sum(axis=1), R, 2)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_direct_sum_per_impact():
    """Eq. 1 summed over the sub-positions, written as a direct sum (C), in
    linear and circular modes, with a non-symmetric synthetic response."""
    rng = np.random.Generator(np.random.PCG64(4))
    nw, nt, I = 9, 125, 3
    S_fine = rng.exponential(1.0, (nw * I, nt))
    R = inputs.impact_response("bipolar", impacts=I, nwires=5, nticks=17, wire_center=1, tick_peak=5.0,
                               tick_sigma=2.0)
    for circ in (False, True):
        got = oracle.convolve_impacts(S_fine, R, 1, circ)
        ref = sum(oracle.convolve_direct(S_fine[i::I], R[i], 1, circ) for i in range(I))
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_impact_response_shape_and_symmetry():
    R = inputs.impact_response("unipolar", impacts=10)
    assert R.shape == (10, 21, 200)
    # mirrored sub-positions are mirrored in the wire offset
    assert np.allclose(R[0], R[9][::-1], atol=1e-7)


def test_simulate_impacts_with_equal_slices_is_the_plain_simulation():
    """The whole impact path with every slice equal to R: the fine rows of a
    wire sum to its coarse bin, so sum_i R (*) S_i = R (*) S, the plain
    simulation, in both convolution modes (expected value, p = 0.8)."""
    nw, nt, I = 12, 300, 4
    R = inputs.response("bipolar")
    RI = np.ascontiguousarray(np.broadcast_to(R, (I,) + R.shape))
    d = inputs.uniform_depos(80, nw, seed=31, nticks=nt)
    for circular in (False, True):
        got = oracle.simulate_impacts(d.q, d.x_mm, d.t_us, nw, nt, RI, 10, circular=circular, p=0.8)
        ref = oracle.simulate(d.q, d.x_mm, d.t_us, nw, nt, R, 10, circular=circular, p=0.8)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
