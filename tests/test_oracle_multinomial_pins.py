"""Pins of the oracle's charge-conserving (multinomial) fluctuation (CPU).

Reading (stated in the oracle): a depo's N = floor(q + 1/2) electrons
survive as K ~ Binomial(N, p) and are spread over the patch bins
multinomially with the bin weights, by conditional binomials over the
in-grid wires, then ticks; electrons falling off the grid are lost.  These
tests hold the oracle to what that fixes: exact conservation, the
Binomial(N, p) law of the survivors, the multinomial's means, variances and
negative covariances, its full joint pmf on a tiny case (scipy), and the
expected loss at the grid edge.
"""
import numpy as np
import pytest

import oracle

stats = pytest.importorskip("scipy.stats")

NW, NT = 64, 400


def _patch(q, x, t, seed, p=1.0, exact_max=32, nw=NW, nt=NT, **kw):
    return oracle.raster_scatter([q], [x], [t], nw, nt, fluctuate=2, p=p, seed=seed,
                                 exact_max=exact_max, **kw)


def _weights(x, t, nw=NW, nt=NT):
    st, sx = oracle.sigmas([t])
    k0, wt = oracle.axis_weights(t, st[0], oracle.TICK_US)
    w0, wx = oracle.axis_weights(x, sx[0], oracle.PITCH_MM)
    W = np.zeros((nw, nt))
    W[w0:w0 + len(wx), k0:k0 + len(wt)] = np.outer(wx, wt)
    return W


def test_interior_depos_conserve_exactly():
    rng = np.random.Generator(np.random.PCG64(1))
    for i in range(300):
        q = rng.uniform(1, 60000)
        x = rng.uniform(40, NW * 5.0 - 40)
        t = rng.uniform(5, NT * 0.5 - 10)
        S = _patch(q, x, t, seed=i, exact_max=int(rng.integers(0, 65)))
        assert S.sum() == np.floor(q + 0.5)
        assert np.all(S >= 0) and np.all(S == np.round(S))


def test_survivors_are_binomial():
    x, t = 160.0, 100.0
    for N, exact_max in ((20, 32), (5000, 32)):
        K = np.array([_patch(N, x, t, seed=s, p=0.7, exact_max=exact_max).sum() for s in range(3000)])
        m, v = N * 0.7, N * 0.7 * 0.3
        assert abs(K.mean() - m) < 5 * np.sqrt(v / K.size)
        assert abs(K.var() - v) < 5 * v * np.sqrt(2.0 / K.size)
        if N <= exact_max:
            ks = np.arange(N + 1)
            f = np.bincount(K.astype(int), minlength=N + 1)
            e = stats.binom.pmf(ks, N, 0.7) * K.size
            keep = e > 5
            chi = np.sum((f[keep] - e[keep]) ** 2 / e[keep])
            assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4


@pytest.mark.parametrize("N,exact_max", [(40, 64), (3000, 32)])
def test_split_has_multinomial_moments(N, exact_max):
    """p = 1: bin counts have mean N w, variance N w (1 - w) and covariance
    -N w_a w_b (the sign independent binomials would not give)."""
    x, t = 162.0, 130.0
    W = _weights(x, t)
    idx = np.argwhere(W > 0.01)
    reps = 4000
    C = np.array([_patch(N, x, t, seed=s, exact_max=exact_max)[idx[:, 0], idx[:, 1]] for s in range(reps)])
    w = W[idx[:, 0], idx[:, 1]]
    mean_se = np.sqrt(N * w * (1 - w) / reps)
    assert np.all(np.abs(C.mean(axis=0) - N * w) < 5 * mean_se + 1e-9)
    var = N * w * (1 - w)
    assert np.all(np.abs(C.var(axis=0) - var) < 6 * var * np.sqrt(2.0 / reps) + 1e-9)
    a, b = np.argsort(w)[-2:]              # the two heaviest bins
    cov = np.mean((C[:, a] - C[:, a].mean()) * (C[:, b] - C[:, b].mean()))
    expect = -N * w[a] * w[b]
    se = np.sqrt((var[a] * var[b] + expect ** 2) / reps)
    assert abs(cov - expect) < 5 * se and expect < -5 * se


def test_joint_pmf_tiny_case():
    """N = 5 electrons over a patch of a few bins: the joint counts follow
    Multinomial(5, w) (scipy), over every outcome with enough mass."""
    x, t = 162.5, 1.0          # narrow: a handful of bins
    W = _weights(x, t)
    nz = np.argwhere(W > 0)
    w = W[nz[:, 0], nz[:, 1]]
    reps = 20000
    outcomes = {}
    for s in range(reps):
        S = _patch(5, x, t, seed=10_000 + s, exact_max=64)
        key = tuple(int(v) for v in S[nz[:, 0], nz[:, 1]])
        assert sum(key) == 5
        outcomes[key] = outcomes.get(key, 0) + 1
    chi, dof = 0.0, -1
    rest_f, rest_e = 0.0, 0.0
    for key, f in outcomes.items():
        e = stats.multinomial.pmf(key, 5, w / w.sum()) * reps
        if e > 10:
            chi += (f - e) ** 2 / e
            dof += 1
        else:
            rest_f += f
            rest_e += e
    tail_e = reps - sum(stats.multinomial.pmf(k, 5, w / w.sum()) * reps for k in outcomes
                        if stats.multinomial.pmf(k, 5, w / w.sum()) * reps > 10)
    chi += (rest_f - tail_e) ** 2 / max(tail_e, 1e-9)
    dof += 1
    assert dof >= 5
    assert stats.chi2.sf(chi, dof) > 1e-4


def test_loss_at_the_grid_edge():
    """A depo straddling wire 0 keeps K less the electrons of its off-grid
    bins: mean in-grid total = N p (in-grid weight)."""
    x, t = 1.0, 120.0
    W_all = _weights(x + 50.0, t, nw=NW + 20)          # same shape, unclipped
    st, sx = oracle.sigmas([t])
    w0, wx = oracle.axis_weights(x, sx[0], oracle.PITCH_MM)
    in_grid = wx[max(0, -w0):].sum()
    assert w0 < 0 and in_grid < 0.999
    N, p = 4000, 0.8
    tot = np.array([_patch(N, x, t, seed=s, p=p).sum() for s in range(2000)])
    expect = N * p * in_grid
    var = N * p * in_grid * (1 - p * in_grid)
    assert abs(tot.mean() - expect) < 5 * np.sqrt(var / tot.size)
    assert W_all.sum() > 0.99
