"""Pins of the FP64 oracle against things other than itself.

Each test fixes one oracle function to an independent source: a library
routine run as a black box (cuRAND's host Philox, scipy.stats.binom,
scipy.signal.convolve2d), a quadrature of the Gaussian density that never
calls erf, a closed form (patch sums, diffusion widths, delta response,
cumulants of a convolution) or brute force (Eq. 1's direct sum).  The cases
are picked so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle

# --------------------------------------------------------------- Philox


def _curand():
    for cand in (ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
                 "libcurand.so.10", "libcurand.so"):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


def _curand_host_words(lib, seed, nwords, offset=0):
    gen = ctypes.c_void_p()
    philox4_32_10 = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), philox4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(nwords)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2 ** 64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 generator, run as a library, emits block b
    of its stream as Philox(counter = (b // 65536, 0, b % 65536, 0), key =
    seed); the oracle's Philox must reproduce those words bit for bit."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    blocks = list(range(0, 24)) + [65535, 65536, 65537, 100000, 131072 + 7, 200001]
    words = _curand_host_words(lib, seed, 4 * (max(blocks) + 1)).reshape(-1, 4)
    key = oracle.seed_key(seed)
    for b in blocks:
        got = oracle.philox([b // 65536, 0, b % 65536, 0], key)
        assert (got == words[b]).all(), (seed, b, got, words[b])


@pytest.mark.parametrize("seed", [3, 0xFEDCBA9876543210])
def test_philox_second_counter_word_matches_curand(seed):
    """The same generator started 2^50 words in (block 2^48 of its stream)
    runs counters whose word 1 is not zero: block b of the stream is
    Philox(((b // 65536) mod 2^32, (b // 65536) >> 32, b % 65536, 0)).  With
    word 1 set and word 3 zero, a mix-up of the two words in the round
    function fails here (the pin above has both zero)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    key = oracle.seed_key(seed)
    for first in (2 ** 48, 2 ** 48 + 65536 * 5 + 3, 3 * 2 ** 48 + 77):
        words = _curand_host_words(lib, seed, 4 * 8, offset=4 * first).reshape(-1, 4)
        for j in range(8):
            b = first + j
            c = [(b // 65536) & 0xFFFFFFFF, (b // 65536) >> 32, b % 65536, 0]
            assert c[1] != 0
            got = oracle.philox(c, key)
            assert (got == words[j]).all(), (seed, b, got, words[j])


def test_philox_counter_words_all_matter():
    """Each counter word and each key word changes the block (no word dropped)."""
    base = oracle.philox([5, 6, 7, 8], [9, 10])
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] += 1
        assert not (oracle.philox(c, [9, 10]) == base).any()
    for i in range(2):
        k = [9, 10]
        k[i] += 1
        assert not (oracle.philox([5, 6, 7, 8], k) == base).any()


# ------------------------------------------------------------- diffusion


def test_sigmas_closed_form():
    """sigma_L = sqrt(2 D_L t)/v, sigma_T = sqrt(2 D_T t): at t = 3 ms with
    D_L = 4 cm^2/s, D_T = 8.8 cm^2/s and v = 1.6 mm/us the widths are
    sqrt(2.4)/1.6 us and sqrt(5.28) mm."""
    st, sx = oracle.sigmas([3000.0, 0.0, 750.0])
    assert st[0] == pytest.approx(math.sqrt(2.4) / 1.6, rel=1e-15)
    assert sx[0] == pytest.approx(math.sqrt(5.28), rel=1e-15)
    assert st[1] == 0.0 and sx[1] == 0.0
    assert st[2] == pytest.approx(0.5 * st[0], rel=1e-15)   # sqrt scaling
    assert sx[2] == pytest.approx(0.5 * sx[0], rel=1e-15)


# ------------------------------------------------------------ bin weights


def _gauss_mass(a, b, mu, sigma, nodes=48):
    """Mass of N(mu, sigma^2) on [a, b] by Gauss-Legendre quadrature of the
    density exp(-u^2/2)/sqrt(2 pi) (no erf anywhere)."""
    if b <= a:
        return 0.0
    x, w = np.polynomial.legendre.leggauss(nodes)
    u = 0.5 * (b - a) * x + 0.5 * (b + a)
    z = (u - mu) / sigma
    return float(0.5 * (b - a) * np.sum(w * np.exp(-0.5 * z * z)) / (sigma * math.sqrt(2 * math.pi)))


@pytest.mark.parametrize("mu,sigma,delta", [
    (10.3, 0.9, 0.5), (0.0, 0.2, 0.5), (-3.7, 1.3, 0.5), (1234.56, 2.297, 5.0),
    (17.5, 0.08, 5.0), (2.5, 3.0, 0.5), (4999.99, 0.61, 5.0), (7.25, 0.75, 0.5)])
def test_axis_weights_match_quadrature(mu, sigma, delta):
    """Weights are the Gaussian mass of each bin clipped to mu +- 3 sigma,
    normalised by the window mass: checked against quadrature of the density."""
    lo, w = oracle.axis_weights(mu, sigma, delta, 3.0)
    a, b = mu - 3 * sigma, mu + 3 * sigma
    assert lo == math.floor(a / delta)
    assert lo + len(w) - 1 == math.floor(b / delta)
    total = _gauss_mass(a, b, mu, sigma, nodes=96)
    for i, wk in enumerate(w):
        k = lo + i
        e0, e1 = max(k * delta, a), min((k + 1) * delta, b)
        assert wk == pytest.approx(_gauss_mass(e0, e1, mu, sigma) / total, abs=1e-13)
    assert w.sum() == pytest.approx(1.0, abs=1e-13)
    assert (w >= 0).all()


def test_axis_weights_point_charge():
    """sigma below 1e-6 bin widths is a point charge in bin floor(mu/delta);
    a charge exactly on an edge belongs to the upper bin."""
    assert oracle.axis_weights(7.3, 0.0, 0.5) == (14, pytest.approx(np.array([1.0])))
    lo, w = oracle.axis_weights(10.0, 1e-9, 5.0)
    assert lo == 2 and list(w) == [1.0]
    lo, w = oracle.axis_weights(-0.1, 0.0, 0.5)
    assert lo == -1


def test_axis_weights_continuous_across_window_edge():
    """A bin entering the window enters with zero weight: sliding the mean
    by eps changes every weight by O(eps)."""
    sigma, delta = 0.7, 0.5
    mu0 = 3 * sigma + 2 * delta  # lower window edge exactly on bin edge 2
    eps = 1e-9
    lo1, w1 = oracle.axis_weights(mu0 + eps, sigma, delta)
    lo2, w2 = oracle.axis_weights(mu0 - eps, sigma, delta)
    grid = {}
    for lo, w, s in ((lo1, w1, 1.0), (lo2, w2, -1.0)):
        for i, v in enumerate(w):
            grid[lo + i] = grid.get(lo + i, 0.0) + s * v
    assert max(abs(v) for v in grid.values()) < 1e-8


# -------------------------------------------------------- raster + scatter


def test_patch_is_outer_product_of_axis_weights():
    """The 2D patch is q * w_wire (rows) x w_tick (columns): a transposed or
    mis-indexed product fails."""
    q, x, t = 4321.0, 1003.7, 1234.4
    st, sx = oracle.sigmas([t])
    S = oracle.raster_scatter([q], [x], [t], 300, 3000)
    wlo, ww = oracle.axis_weights(x, sx[0], 5.0)
    tlo, wt = oracle.axis_weights(t, st[0], 0.5)
    ref = np.zeros_like(S)
    ref[wlo:wlo + len(ww), tlo:tlo + len(wt)] = q * np.outer(ww, wt)
    np.testing.assert_allclose(S, ref, rtol=0, atol=1e-12 * q)
    assert len(ww) != len(wt)


@pytest.mark.parametrize("p", [1.0, 0.7])
def test_patch_sum_equals_charge_for_interior_depos(p):
    """Normalised weights: an interior depo deposits exactly p*q."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = 200
    q = rng.exponential(5000, n)
    x = rng.uniform(50, 4750, n)
    t = rng.uniform(20, 2990, n)
    S = oracle.raster_scatter(q, x, t, 960, 6000, p=p)
    assert S.sum() == pytest.approx(p * q.sum(), rel=1e-12)


def test_point_charge_lands_in_one_bin():
    """t = 0 gives zero diffusion: all the charge sits in tick bin 0 of the
    wire holding x."""
    S = oracle.raster_scatter([100.0], [12.5], [0.0], 10, 20)
    assert S[2, 0] == 100.0 and S.sum() == 100.0


def test_scatter_is_linear():
    """The grid of many depos is the sum of single-depo grids."""
    rng = np.random.Generator(np.random.PCG64(6))
    q = rng.exponential(5000, 7); x = rng.uniform(0, 200, 7); t = rng.uniform(0, 100, 7)
    S = oracle.raster_scatter(q, x, t, 40, 200)
    parts = sum(oracle.raster_scatter(q[i:i + 1], x[i:i + 1], t[i:i + 1], 40, 200) for i in range(7))
    np.testing.assert_allclose(S, parts, rtol=1e-14, atol=1e-9)


def test_off_grid_charge_is_dropped_and_bad_depos_skipped():
    """Bins outside the grid are lost; non-finite inputs or negative drift
    times deposit nothing and are counted as skipped."""
    S, skipped = oracle.raster_scatter([100.0, 50.0, 50.0, 70.0], [-2.4, 5.0, np.nan, 5.0],
                                       [100.0, 100.0, 10.0, -5.0], 3, 400, return_skipped=True)
    assert skipped == 2
    lo, ww = oracle.axis_weights(-2.4, oracle.sigmas([100.0])[1][0], 5.0)
    inside = sum(ww[i] for i in range(len(ww)) if lo + i >= 0)
    assert S.sum() == pytest.approx(50.0 + 100.0 * inside, rel=1e-12)


# -------------------------------------------------------------- binomial


def test_survive_threshold():
    assert oracle.survive_threshold(0.7) == math.floor(0.7 * 2 ** 32)
    assert oracle.survive_threshold(0.0) == 0
    assert oracle.survive_threshold(1.0) == 2 ** 32 - 1


def test_binomial_exact_branch_matches_binomial_pmf():
    """Exact branch: the survivor counts over many independent bins follow
    Binomial(N, p) (chi-square against scipy.stats.binom)."""
    stats = pytest.importorskip("scipy.stats")
    N, p, m = 20, 0.7, 20000
    k = np.array([oracle.binomial(N, p, seed=77, wire=i // 6000, tick=i % 6000, depo=3) for i in range(m)])
    assert k.min() >= 0 and k.max() <= N
    obs = np.bincount(k, minlength=N + 1).astype(float)
    exp = stats.binom.pmf(np.arange(N + 1), N, p) * m
    keep = exp > 5
    chi2 = (((obs - exp) ** 2) / exp)[keep].sum() + 0.0
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-3
    assert k.mean() == pytest.approx(N * p, abs=4 * math.sqrt(N * p * (1 - p) / m))


_ALL_WORDS = None


def _all_words():
    """Every value of a word's top 24 bits (the inversion's uniform u)."""
    global _ALL_WORDS
    if _ALL_WORDS is None:
        _ALL_WORDS = (np.arange(1 << 24, dtype=np.uint32) << np.uint32(8))
    return _ALL_WORDS


@pytest.mark.parametrize("N,p", [(1, 0.7), (5, 0.7), (20, 0.7), (32, 0.3), (64, 0.5), (13, 0.999),
                                 (9, 0.01), (40, 0.62)])
def test_binomial_inversion_is_the_pmf_over_every_word(N, p):
    """Exact branch: over all 2^24 values of u the inversion returns k with
    frequency Binomial(N, float(p)).pmf(k), up to the float rounding of the
    running CDF (a few ulps per step) and the 2^-24 spacing of u."""
    stats = pytest.importorskip("scipy.stats")
    k = oracle.binomial_invert(N, p, _all_words())
    freq = np.bincount(k, minlength=N + 1) / float(1 << 24)
    pmf = stats.binom.pmf(np.arange(N + 1), N, float(np.float32(p)))
    assert np.abs(freq - pmf).max() <= 1e-7 * (N + 2) + 2.0 ** -24
    # u nondecreasing gives k nondecreasing (mirrored for p > 1/2)
    d = np.diff(k)
    assert (d >= 0).all() if np.float32(p) <= 0.5 else (d <= 0).all()


def test_binomial_inversion_edges():
    """u = 0 gives the smallest count, the largest u the largest reachable;
    N = 1 is a Bernoulli trial with P(k = 1) = float(p)."""
    lo, hi = np.uint32(0), np.uint32(0xFFFFFFFF)
    assert oracle.binomial_invert(10, 0.3, [lo])[0] == 0
    assert oracle.binomial_invert(10, 0.7, [lo])[0] == 10
    assert oracle.binomial_invert(10, 0.3, [hi])[0] == 10
    k = oracle.binomial_invert(1, 0.7, _all_words())
    assert abs(k.mean() - float(np.float32(0.7))) <= 2 ** -23


def test_binomial_exact_max_is_capped():
    with pytest.raises(ValueError):
        oracle.binomial(10, 0.7, 1, 0, 2, 3, exact_max=oracle.EXACT_CAP + 1)
    with pytest.raises(ValueError):
        oracle.raster_scatter([1.0], [2.0], [3.0], 4, 10, fluctuate=True, p=0.7, exact_max=100)


def test_binomial_normal_branch_moments():
    """Normal branch (N > exact_max): mean N p and variance N p (1 - p)."""
    N, p, m = 5000, 0.7, 20000
    k = np.array([oracle.binomial(N, p, seed=78, wire=i // 6000, tick=i % 6000, depo=9, event_id=2)
                  for i in range(m)],
                 dtype=float)
    var = N * p * (1 - p)
    assert k.mean() == pytest.approx(N * p, abs=4 * math.sqrt(var / m))
    assert k.var() == pytest.approx(var, rel=0.05)


def test_binomial_normal_branch_distribution():
    """Normal branch: the standardised counts follow the normal distribution
    that Box-Muller on the word's 16-bit halves draws (the CDF at seven
    points within its sampling error plus the half-count rounding), and no
    draw passes the sampler's bound |z| <= sqrt(2 ln 2^17)."""
    N, p, m = 20000, 0.3, 40000
    k = np.array([oracle.binomial(N, p, seed=79, wire=i // 4000, tick=i % 4000, depo=4, nticks=4000)
                  for i in range(m)], dtype=float)
    mean = N * oracle.survive_threshold(p) / 2 ** 32
    sd = math.sqrt(mean * (1 - oracle.survive_threshold(p) / 2 ** 32))
    z = (k - mean) / sd
    for c in (-2.5, -1.5, -0.7, 0.0, 0.7, 1.5, 2.5):
        phi = 0.5 * math.erfc(-c / math.sqrt(2))
        assert abs((z <= c).mean() - phi) <= 4 * math.sqrt(phi * (1 - phi) / m) + 0.5 / sd * 0.4
    assert np.abs(z).max() <= math.sqrt(2 * math.log(2 ** 17)) + 1.0 / sd
    assert np.abs(z).max() > 3.5


def test_binomial_bins_of_a_quad_are_independent():
    """The four bins of a quad share one Philox block, one word each: over
    many quads, the counts of two bins of the same quad are uncorrelated
    and their joint frequencies factor (chi-square test of independence),
    for two exact-branch bins and for an exact- and a normal-branch bin; a
    mix-up of the words (two bins reading one word) fails both."""
    stats = pytest.importorskip("scipy.stats")
    m = 12000
    for (na, ta), (nb, tb) in (((20, 0), (20, 1)), ((20, 2), (20, 3)), ((20, 1), (3000, 2)), ((12, 3), (12, 0))):
        a = np.array([oracle.binomial(na, 0.6, seed=80, wire=q // 1500, tick=4 * (q % 1500) + ta, depo=7)
                      for q in range(m)], dtype=float)
        b = np.array([oracle.binomial(nb, 0.6, seed=80, wire=q // 1500, tick=4 * (q % 1500) + tb, depo=7)
                      for q in range(m)], dtype=float)
        r = np.corrcoef(a, b)[0, 1]
        assert abs(r) < 4 / math.sqrt(m), (ta, tb, r)
        ca = np.digitize(a, np.quantile(a, [0.25, 0.5, 0.75]))
        cb = np.digitize(b, np.quantile(b, [0.25, 0.5, 0.75]))
        table = np.zeros((4, 4))
        np.add.at(table, (ca, cb), 1)
        table = table[table.sum(1) > 0][:, table.sum(0) > 0]
        assert stats.chi2_contingency(table)[1] > 1e-3, (ta, tb)
    # the same bin is the same draw; the quad's other words are other draws
    one = [oracle.binomial(20, 0.6, seed=81, wire=3, tick=t, depo=2) for t in range(8, 12)]
    assert one == [oracle.binomial(20, 0.6, seed=81, wire=3, tick=t, depo=2) for t in range(8, 12)]


def test_binomial_special_cases():
    assert oracle.binomial(0, 0.7, 1, 0, 2, 3) == 0
    assert oracle.binomial(40, 1.0, 1, 0, 2, 3) == 40
    assert oracle.binomial(40, 0.0, 1, 0, 2, 3) == 0
    # every draw depends on (seed, bin, depo, event/plane): different keys differ
    vals = {oracle.binomial(30, 0.5, s, 0, 2, 3) for s in range(40)}
    assert len(vals) > 5


def test_fluctuated_bins_average_to_expected_value():
    """Per-bin mean over seeds of the fluctuated grid tends to p*floor(q w + 1/2)."""
    q, x, t = [3000.0], [52.0], [2000.0]
    ref = oracle.raster_scatter(q, x, t, 30, 4200)
    mask = ref > 0
    nb = np.floor(ref[mask] + 0.5)
    p, nseeds = 0.7, 300
    acc = np.zeros(nb.shape); acc2 = np.zeros(nb.shape)
    for s in range(nseeds):
        S = oracle.raster_scatter(q, x, t, 30, 4200, fluctuate=True, p=p, seed=1000 + s)
        acc += S[mask]; acc2 += S[mask] ** 2
        assert np.all(S[~mask] == 0)
    mean = acc / nseeds
    sd = np.sqrt(nb * p * (1 - p) / nseeds) + 1e-12
    z = (mean - nb * p) / sd
    assert np.abs(z[nb > 0]).max() < 5.5


# ----------------------------------------------------------- convolution


def _rand_grid(rng, nw, nt):
    return rng.standard_normal((nw, nt))


@pytest.mark.parametrize("circular", [False, True])
@pytest.mark.parametrize("shape,rshape,c", [((12, 40), (5, 9), 2), ((9, 31), (3, 7), 0),
                                            ((16, 50), (7, 12), 5), ((6, 10), (5, 13), 1)])
def test_fft_convolution_equals_direct_sum(circular, shape, rshape, c):
    """Eq. 2 (numpy FFT) equals Eq. 1's direct sum (brute force), linear and
    circular, with an asymmetric response and an off-centre wire origin."""
    rng = np.random.Generator(np.random.PCG64(11))
    S = _rand_grid(rng, *shape)
    R = rng.standard_normal(rshape).astype(np.float32)
    M1 = oracle.convolve_fft(S, R, c, circular)
    M2 = oracle.convolve_direct(S, R, c, circular)
    np.testing.assert_allclose(M1, M2, rtol=0, atol=1e-12 * np.abs(M2).max())


def test_linear_convolution_matches_scipy_convolve2d():
    """Linear mode is scipy's full 2D convolution, windowed to the grid with
    response row wire_center at wire offset 0 and column 0 at tick offset 0."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.Generator(np.random.PCG64(12))
    S = _rand_grid(rng, 14, 60)
    R = rng.standard_normal((7, 11)).astype(np.float32)
    c = 4
    full = signal.convolve2d(S, R.astype(np.float64), mode="full")
    np.testing.assert_allclose(oracle.convolve_fft(S, R, c), full[c:c + 14, :60], atol=1e-11)
    np.testing.assert_allclose(oracle.convolve_direct(S, R, c), full[c:c + 14, :60], atol=1e-11)


def test_delta_response_is_identity():
    rng = np.random.Generator(np.random.PCG64(13))
    S = _rand_grid(rng, 20, 64)
    R = np.zeros((21, 200), np.float32)
    R[10, 0] = 1.0
    np.testing.assert_allclose(oracle.convolve_fft(S, R, 10), S, atol=1e-12)
    np.testing.assert_allclose(oracle.convolve_fft(S, R, 10, circular=True), S, atol=1e-12)
    np.testing.assert_array_equal(oracle.convolve_direct(S, R, 10), S)


def test_convolution_cumulants_add():
    """With S and R positive and nothing pushed off the grid, M's total is
    the product of totals, and its mean and variance along each axis are the
    sums of those of S and R (cumulants of a convolution add)."""
    rng = np.random.Generator(np.random.PCG64(14))
    S = np.zeros((40, 400)); S[12:20, 30:120] = rng.uniform(0.1, 1.0, (8, 90))
    R = rng.uniform(0.1, 1.0, (5, 30)).astype(np.float32)
    c = 2
    M = oracle.convolve_fft(S, R, c)
    R64 = R.astype(np.float64)
    assert M.sum() == pytest.approx(S.sum() * R64.sum(), rel=1e-12)

    def moments(A, axis, origin=0):
        m = A.sum(axis=1 - axis)
        idx = np.arange(m.shape[0]) - origin
        mean = (idx * m).sum() / m.sum()
        return mean, ((idx - mean) ** 2 * m).sum() / m.sum()

    for axis, origin in ((0, c), (1, 0)):
        ms, vs = moments(S, axis)
        mr, vr = moments(R64, axis, origin)
        mm, vm = moments(M, axis)
        assert mm == pytest.approx(ms + mr, rel=1e-11)
        assert vm == pytest.approx(vs + vr, rel=1e-10)


def test_convolve_points_matches_full_direct_sum():
    rng = np.random.Generator(np.random.PCG64(15))
    S = _rand_grid(rng, 10, 50)
    R = rng.standard_normal((5, 9)).astype(np.float32)
    M = oracle.convolve_direct(S, R, 2)
    pw = np.array([0, 3, 9, 9, 5]); pt = np.array([0, 49, 0, 48, 20])
    np.testing.assert_array_equal(oracle.convolve_points(S, R, 2, pw, pt), M[pw, pt])


def test_circular_equals_linear_when_nothing_wraps():
    rng = np.random.Generator(np.random.PCG64(16))
    S = np.zeros((24, 80)); S[6:14, 5:40] = rng.standard_normal((8, 35))
    R = rng.standard_normal((5, 9)).astype(np.float32)
    np.testing.assert_allclose(oracle.convolve_fft(S, R, 2, True), oracle.convolve_fft(S, R, 2),
                               atol=1e-12)


def test_simulate_of_one_point_charge_is_the_response():
    """A point charge q at (wire w, tick k) gives q * R placed at wire w + d,
    tick k + j: the whole path composes raster and convolution correctly."""
    R = np.random.Generator(np.random.PCG64(17)).standard_normal((5, 9)).astype(np.float32)
    M = oracle.simulate([2.0], [7 * 5.0 + 1.0], [0.0], 16, 30, R, 2)
    ref = np.zeros((16, 30))
    ref[7 - 2:7 + 3, 0:9] = 2.0 * R
    np.testing.assert_allclose(M, ref, atol=1e-12)


def test_oracle_matches_its_golden_fixtures():
    """Regression guard (not a pin): the oracle's Philox blocks and
    exact-branch counts equal the fixtures tests/golden/make_golden.py
    wrote from it."""
    import os
    gdir = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for line in open(os.path.join(gdir, "philox_blocks.txt")):
        if line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        assert list(oracle.philox(v[:4], v[4:6])) == v[6:10]
    lines = [l for l in open(os.path.join(gdir, "binomial_inversion.txt")) if not l.startswith("#")]
    words = np.array([int(x, 16) for x in lines[0].split()[1:]], dtype=np.uint32)
    for line in lines[1:]:
        head, counts = line.split(":")
        N, p = head.split()
        got = oracle.binomial_invert(int(N), float(p), words)
        assert list(got) == [int(c) for c in counts.split()], (N, p)
    for line in open(os.path.join(gdir, "binomial_bins.txt")):
        if line.startswith("#"):
            continue
        N, p, seed, w, t, d, ev, pl, nt, k = line.split()
        assert oracle.binomial(int(N), float(p), int(seed), int(w), int(t), int(d), event_id=int(ev),
                               plane_id=int(pl), nticks=int(nt)) == int(k), line


def test_convolution_parseval_against_a_direct_dft():
    """Circular mode (Eq. 2 on the grid): sum M^2 equals (1/N) sum over the
    2D spectrum of |S_hat R_hat|^2, with both spectra from an explicit DFT
    matrix (not the FFT the oracle uses)."""
    rng = np.random.Generator(np.random.PCG64(51))
    nw, nt = 6, 10
    S = rng.standard_normal((nw, nt))
    R = rng.standard_normal((3, 4))
    M = oracle.convolve_fft(S, R, 1, circular=True)
    Rc = np.zeros((nw, nt))
    for r in range(3):
        for j in range(4):
            Rc[(r - 1) % nw, j % nt] += R[r, j]
    Fw = np.exp(-2j * np.pi * np.outer(np.arange(nw), np.arange(nw)) / nw)
    Ft = np.exp(-2j * np.pi * np.outer(np.arange(nt), np.arange(nt)) / nt)
    Sh = Fw @ S @ Ft.T
    Rh = Fw @ Rc @ Ft.T
    assert abs(np.sum(M ** 2) - np.sum(np.abs(Sh * Rh) ** 2) / (nw * nt)) < 1e-9 * np.sum(M ** 2)


def test_gaussian_convolved_with_gaussian_stays_gaussian():
    """Sampled Gaussians of variances a and b (wire and tick axes) convolve
    into the sampled Gaussian of variance a + b, scaled by the product of
    the normalisations; the discrete sum differs from the continuous one by
    terms of order exp(-2 pi^2 ab/(a+b)), far below double precision here."""
    nw, nt = 64, 160
    a_w, a_t, b_w, b_t = 2.0 ** 2, 3.0 ** 2, 1.5 ** 2, 4.0 ** 2
    w = np.arange(nw)[:, None]
    t = np.arange(nt)[None, :]
    S = np.exp(-(w - 30) ** 2 / (2 * a_w) - (t - 60) ** 2 / (2 * a_t))
    kw, kt, c = 21, 81, 10               # response kept to 6.7 sigma in wires, 10 sigma in ticks
    r = np.arange(kw)[:, None] - c
    j = np.arange(kt)[None, :] - 40      # tick offset j - 40, handled by shifting the answer
    R = np.exp(-r ** 2 / (2 * b_w) - j ** 2 / (2 * b_t))
    M = oracle.convolve_fft(S, R, c)
    cw = 2 * np.pi * a_w * b_w / (a_w + b_w)
    ct = 2 * np.pi * a_t * b_t / (a_t + b_t)
    expect = np.sqrt(cw * ct) * np.exp(-(w - 30) ** 2 / (2 * (a_w + b_w)) - (t - 100) ** 2 / (2 * (a_t + b_t)))
    # away from the edges, where the response's truncation and the grid clip nothing
    sl = (slice(15, 45), slice(60, 140))
    assert np.max(np.abs(M[sl] - expect[sl])) < 1e-9 * np.max(expect)


def test_shift_equivariance_by_whole_bins():
    """Moving every depo by one pitch (or one tick, with given widths: the
    diffusion widths depend on t) moves S by one wire row (one tick column);
    the convolution (linear mode, away from the edges) follows."""
    rng = np.random.Generator(np.random.PCG64(61))
    nw, nt, n = 30, 400, 300
    q = rng.exponential(5000, n)
    x = rng.uniform(30.0, (nw - 8) * oracle.PITCH_MM, n)
    t = rng.uniform(20.0, (nt - 60) * oracle.TICK_US, n)
    st = rng.uniform(0.2, 2.0, n)
    sx = rng.uniform(0.3, 3.0, n)
    S = oracle.raster_scatter(q, x, t, nw, nt, sig_t_us=st, sig_x_mm=sx)
    Sx = oracle.raster_scatter(q, x + oracle.PITCH_MM, t, nw, nt, sig_t_us=st, sig_x_mm=sx)
    St = oracle.raster_scatter(q, x, t + oracle.TICK_US, nw, nt, sig_t_us=st, sig_x_mm=sx)
    assert np.allclose(Sx[1:], S[:-1], rtol=1e-10, atol=1e-9 * S.max())
    assert np.allclose(St[:, 1:], S[:, :-1], rtol=1e-10, atol=1e-9 * S.max())
    R = np.random.Generator(np.random.PCG64(62)).standard_normal((21, 200))
    M = oracle.convolve_fft(S, R, 10)
    Mx = oracle.convolve_fft(Sx, R, 10)
    assert np.allclose(Mx[12:-1], M[11:-2], rtol=1e-9, atol=1e-9 * np.abs(M).max())


def test_patch_extents_by_scanning_every_bin():
    """Brute force on a small grid: a bin belongs to a depo's patch when its
    interval overlaps the window mu +- 3 sigma with positive length (the
    Gaussian density is positive there, so the bin's mass is), or, for a
    point charge, when it holds mu.  Scanning every bin must give exactly the
    oracle's extents (floor-and-clamp arithmetic), for depos inside, across
    and outside the grid edges; the total is the sum of the patch sizes."""
    nw, nt, pitch, tick = 16, 60, 5.0, 0.5
    rng = np.random.Generator(np.random.PCG64(404))
    n = 400
    x = rng.uniform(-25.0, nw * pitch + 25.0, n)
    t = rng.uniform(-5.0, nt * tick + 5.0, n)
    sx = rng.uniform(0.05, 4.0, n)
    st = rng.uniform(0.02, 1.5, n)
    sx[:20] = 1e-9                     # point charges along the wire axis
    st[20:40] = 1e-9                   # and along ticks
    w0, nwp, t0, ntp, total = oracle.patch_extents(x, t, nw, nt, sig_t_us=st, sig_x_mm=sx)

    def scan(mu, sigma, delta, nbins):
        if sigma <= 1e-6 * delta:
            hit = [b for b in range(nbins) if b * delta <= mu < (b + 1) * delta]
        else:
            lo, hi = mu - 3.0 * sigma, mu + 3.0 * sigma
            hit = [b for b in range(nbins) if min((b + 1) * delta, hi) - max(b * delta, lo) > 0.0]
        return (hit[0], len(hit)) if hit else (None, 0)

    for i in range(n):
        bw, cw = scan(x[i], sx[i], pitch, nw)
        bt, ct = scan(t[i], st[i], tick, nt)
        if cw == 0 or ct == 0:
            assert nwp[i] * ntp[i] == 0, i
            continue
        assert (w0[i], nwp[i], t0[i], ntp[i]) == (bw, cw, bt, ct), i
    assert total == int(np.sum(nwp.astype(np.int64) * ntp))
    assert 0 < np.count_nonzero(nwp * ntp) < n      # some depos fall off the grid


@pytest.mark.parametrize("fluct", [0, 1, 2])
def test_slices_with_their_offsets_sum_to_the_whole_list(fluct):
    """The random counters carry each depo's index in the event's list, so
    a list rastered in slices (each with the index of its first depo)
    scatters exactly the whole list's grid, bin for bin (integer counts
    when fluctuating), while the same slices without their offsets draw
    other numbers."""
    nw, nt, n = 20, 400, 300
    rng = np.random.Generator(np.random.PCG64(41))
    q = rng.exponential(4000, n); x = rng.uniform(0, nw * 5.0, n); t = rng.uniform(1, nt * 0.5, n)
    kw = dict(fluctuate=fluct, p=0.7, seed=99, event_id=5, plane_id=1)
    whole = oracle.raster_scatter(q, x, t, nw, nt, **kw)
    cuts = [0, 70, 71, 200, 300]
    spans = list(zip(cuts[:-1], cuts[1:]))
    total = np.sum([oracle.raster_scatter(q[a:b], x[a:b], t[a:b], nw, nt, depo_offset=a, **kw) for a, b in spans],
                   axis=0)
    if fluct:
        assert np.array_equal(total, whole)
        blind = np.sum([oracle.raster_scatter(q[a:b], x[a:b], t[a:b], nw, nt, **kw) for a, b in spans], axis=0)
        assert not np.array_equal(blind, whole)
    else:
        assert np.allclose(total, whole, rtol=1e-12, atol=1e-9)
