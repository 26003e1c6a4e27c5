"""Pins of the oracle's noise term N(t, x) (Eq. 1) and transform length (CPU).

The paper names the noise term of Eq. 1 and leaves its model open; the
reading (amplitude spectra on the tick transform length, incoherent per wire
plus coherent per wire group, complex normals by Box-Muller from Philox
words) is stated in the oracle.  These tests check the oracle against what
that definition fixes without recomputing it: the normality and
independence of its draws, the closed-form variance, autocovariance and
group covariances of the waveforms, a direct DFT sum on small lengths, and
brute force for the transform length.
"""
import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")


def _smooth(n):
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def test_fft_len_brute_force():
    for n in range(1, 3000):
        m = oracle.fft_len(n)
        assert m >= n and _smooth(m)
        assert not any(_smooth(j) for j in range(n, m))
    # the plane sizes of the workloads (nticks + K_t - 1 = 6199; circular 960)
    assert oracle.fft_len(6000 + 200 - 1) == 6250
    assert oracle.fft_len(960) == 960


def test_draws_are_standard_normal_and_independent():
    """Interior bins carry (z1 + i z2)/sqrt 2 with z1, z2 ~ N(0, 1)
    independent; bin 0 and the Nyquist bin are real N(0, 1)."""
    L = 256
    nf = L // 2 + 1
    spec = oracle.noise_spectrum(800, L, np.ones(nf), seed=11, event_id=3, plane_id=2)
    inner = spec[:, 1:nf - 1]
    z1 = np.sqrt(2.0) * inner.real.ravel()
    z2 = np.sqrt(2.0) * inner.imag.ravel()
    n = z1.size
    for z in (z1, z2):
        assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z1, z2)[0, 1]) < 5 / np.sqrt(n)
    # neighbouring wires and neighbouring bins uncorrelated
    assert abs(np.corrcoef(inner[:-1].real.ravel(), inner[1:].real.ravel())[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(inner[:, :-1].real.ravel(), inner[:, 1:].real.ravel())[0, 1]) < 5 / np.sqrt(n)
    edge = np.concatenate([spec[:, 0], spec[:, nf - 1]])
    assert np.all(edge.imag == 0.0)
    assert scipy_stats.kstest(edge.real, "norm").pvalue > 1e-4


def test_streams_keyed_by_seed_event_plane():
    L = 64
    a = np.ones(L // 2 + 1)
    base = oracle.noise_spectrum(4, L, a, seed=1, event_id=2, plane_id=3)
    assert np.array_equal(base, oracle.noise_spectrum(4, L, a, seed=1, event_id=2, plane_id=3))
    for kw in (dict(seed=2, event_id=2, plane_id=3), dict(seed=1, event_id=3, plane_id=3),
               dict(seed=1, event_id=2, plane_id=4), dict(seed=1 << 32, event_id=2, plane_id=3)):
        other = oracle.noise_spectrum(4, L, a, **kw)
        assert not np.any(np.isclose(other, base))


@pytest.mark.parametrize("L", [12, 15, 20])
def test_waveform_is_the_inverse_dft_of_the_hermitian_extension(L):
    """n[t] = (1/L) sum_{k<L} Nhat_ext[k] e^{2 pi i k t / L}, Nhat_ext[L - k] =
    conj Nhat[k], written as a direct sum (odd and even L)."""
    rng = np.random.Generator(np.random.PCG64(L))
    nf = L // 2 + 1
    amp = rng.uniform(0.5, 2.0, nf)
    coh = rng.uniform(0.1, 1.0, nf)
    spec = oracle.noise_spectrum(5, L, amp, coh, 2, seed=9)
    got = oracle.noise(5, L - 2, L, amp, coh, 2, seed=9)
    ext = np.zeros((5, L), complex)
    ext[:, :nf] = spec
    for k in range(nf, L):
        ext[:, k] = np.conj(spec[:, L - k])
    t = np.arange(L - 2)
    k = np.arange(L)
    direct = (ext @ np.exp(2j * np.pi * np.outer(k, t) / L)) / L
    assert np.max(np.abs(direct.imag)) < 1e-12
    assert np.max(np.abs(direct.real - got)) < 1e-12


def _ext_power(A, L):
    """sum over the full spectrum k = 0 .. L-1 of A_ext[k]^2 cos(...) terms."""
    nf = L // 2 + 1
    full = np.zeros(L)
    full[:nf] = A
    for k in range(nf, L):
        full[k] = A[L - k]
    return full


def test_variance_and_autocovariance_closed_form():
    """Per-sample covariance at lag tau: (1/L^2) sum_{k<L} A_ext[k]^2
    cos(2 pi k tau / L) (stationary; tau = 0 is the variance)."""
    L = 64
    nf = L // 2 + 1
    k = np.arange(nf)
    A = 3.0 * (k / 8.0) * np.exp(-k / 8.0) + 0.5
    W = 6000
    n = oracle.noise(W, L, L, A, seed=21)
    full = _ext_power(A, L)
    kk = np.arange(L)
    for tau in (0, 1, 3, 7):
        expect = np.sum(full ** 2 * np.cos(2 * np.pi * kk * tau / L)) / L ** 2
        prod = n[:, : L - tau] * n[:, tau:]
        per_wire = prod.mean(axis=1)
        est = per_wire.mean()
        se = per_wire.std() / np.sqrt(W)
        assert abs(est - expect) < 5 * se + 1e-12, (tau, est, expect, se)
    means = n.mean(axis=1)
    assert abs(means.mean()) < 5 * means.std() / np.sqrt(W)


def test_coherent_groups():
    """Coherent part only: the wires of a group carry the same waveform;
    with both parts: within-group covariance (1/L^2) sum Ac_ext^2, none
    across groups, variance (1/L^2) sum (A_ext^2 + Ac_ext^2)."""
    L = 48
    nf = L // 2 + 1
    k = np.arange(nf)
    Ac = np.exp(-k / 6.0)
    A = 0.7 * np.ones(nf)
    only = oracle.noise(12, L, L, np.zeros(nf), Ac, 4, seed=5)
    for g in range(3):
        blk = only[4 * g: 4 * g + 4]
        assert np.array_equal(blk, np.broadcast_to(blk[0], blk.shape))
    assert not np.allclose(only[0], only[4])
    G, W = 3, 9000
    n = oracle.noise(W, L, L, A, Ac, G, seed=6)
    fa, fc = _ext_power(A, L), _ext_power(Ac, L)
    var = (np.sum(fa ** 2) + np.sum(fc ** 2)) / L ** 2
    cov_in = np.sum(fc ** 2) / L ** 2
    v = (n * n).mean(axis=1)
    c_in = (n[0::G] * n[1::G]).mean(axis=1)         # wires 3g, 3g+1: one group
    c_out = (n[2:-1:G] * n[3::G]).mean(axis=1)      # wires 3g+2, 3g+3: two groups
    for est, expect in ((v, var), (c_in, cov_in), (c_out, 0.0)):
        se = est.std() / np.sqrt(est.size)
        assert abs(est.mean() - expect) < 5 * se, (est.mean(), expect, se)


def test_simulate_adds_noise_on_the_plane_length():
    """simulate(noise) = simulate() + noise(L = fft_len(nticks + K_t - 1))."""
    rng = np.random.Generator(np.random.PCG64(8))
    nw, nt = 6, 50
    q = rng.exponential(5000, 20); x = rng.uniform(0, nw * 5.0, 20); t = rng.uniform(1, nt * 0.5, 20)
    R = rng.standard_normal((3, 7))
    L = oracle.fft_len(nt + 7 - 1)
    amp = np.ones(L // 2 + 1)
    plain = oracle.simulate(q, x, t, nw, nt, R, 1, seed=4, event_id=1, plane_id=2)
    noisy = oracle.simulate(q, x, t, nw, nt, R, 1, seed=4, event_id=1, plane_id=2, noise_amp=amp)
    assert np.allclose(noisy - plain, oracle.noise(nw, nt, L, amp, seed=4, event_id=1, plane_id=2), atol=1e-9)
