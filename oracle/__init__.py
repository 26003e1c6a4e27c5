"""FP64 oracle for the LArTPC signal-simulation hot path (arXiv 2203.02479).

TEST INFRASTRUCTURE ONLY: the tests, the package's ``smoke()`` check and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  It shares no code with the CUDA library: the per-depo loops are plain
C in ``wsoracle.c`` (compiled here with gcc on first use), the convolution of
Eq. 2 uses numpy's FFT in double precision, and Eq. 1's direct sum is in C.

Every function is pinned by ``tests/test_oracle_pins.py`` against something
other than itself; the pins are listed in each docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wsoracle.c")
_SO = os.path.join(_HERE, "_wsoracle.so")
_lock = threading.Lock()
_handle = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``wsoracle.c`` into ``_wsoracle.so`` with gcc (plain -O2, libm)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_SO)
            h.wso_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            h.wso_philox4x32_10.restype = None
            h.wso_sigmas.argtypes = [ctypes.c_int64, _f64p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _f64p, _f64p]
            h.wso_sigmas.restype = None
            h.wso_axis_weights.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int64), _f64p]
            h.wso_axis_weights.restype = ctypes.c_int
            h.wso_survive_threshold.argtypes = [ctypes.c_double]
            h.wso_survive_threshold.restype = ctypes.c_uint32
            h.wso_binomial.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int, _u32p,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            h.wso_binomial.restype = ctypes.c_int64
            h.wso_binomial_invert_many.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int64, _u32p,
                                                   np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")]
            h.wso_binomial_invert_many.restype = None
            opt_f32 = ctypes.c_void_p
            h.wso_raster_scatter.argtypes = [
                ctypes.c_int64, _f64p, _f64p, _f64p, opt_f32, opt_f32,
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _f64p]
            h.wso_raster_scatter.restype = ctypes.c_int64
            h.wso_patch_extents.argtypes = [
                ctypes.c_int64, _f64p, _f64p, opt_f32, opt_f32,
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                _i32p, _i32p, _i32p, _i32p]
            h.wso_patch_extents.restype = ctypes.c_int64
            h.wso_convolve_direct.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f32p,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _f64p]
            h.wso_convolve_direct.restype = None
            h.wso_convolve_points.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f32p,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int64, _i32p, _i32p, _f64p]
            h.wso_convolve_points.restype = None
            h.wso_depo_grads.argtypes = [
                ctypes.c_int64, _f64p, _f64p, _f64p, opt_f32, opt_f32, ctypes.c_int, ctypes.c_int,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, _f64p, _f64p, _f64p, _f64p,
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            h.wso_depo_grads.restype = ctypes.c_int64
            h.wso_noise_spectrum.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, ctypes.c_void_p, ctypes.c_int,
                                             _u32p, ctypes.c_uint32, _f64p, _f64p]
            h.wso_noise_spectrum.restype = None
            _handle = h
    return _handle


# ----------------------------------------------------------------- defaults
PITCH_MM = 5.0
TICK_US = 0.5
NSIGMA = 3.0
DL = 4.0e-4
DT = 8.8e-4
V = 1.6
EXACT_MAX = 32
EXACT_CAP = 64     # largest exact_max: keeps (1 - s)^N a normal float


def _c32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _c64(a):
    """Depo inputs in double: float32 arrays convert exactly, Python floats
    and float64 arrays are kept as they are (finite differences need that)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _opt_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------- Philox
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key (SC'11).

    Pinned against cuRAND's host Philox4_32_10 generator."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _lib().wso_philox4x32_10(c, k, out)
    return out


def seed_key(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def survive_threshold(p: float) -> int:
    return int(_lib().wso_survive_threshold(float(p)))


def binomial(N: int, p: float, seed: int, wire: int, tick: int, depo: int, event_id: int = 0,
             plane_id: int = 0, exact_max: int = EXACT_MAX, nticks: int = 6000) -> int:
    """Binomial(N, p) survivor count of bin (wire, tick) of a depo's patch on a
    grid of nticks ticks (Sec. 3.1 reading): word tick % 4 of the Philox
    block of the bin's quad (counter (0, wire*ceil(nticks/4) + tick // 4,
    depo, event << 4 | plane)); inversion of its top 24 bits for
    N <= exact_max, else Box-Muller on its two 16-bit halves.

    Pinned by the exact pmf over every value of the inversion's random word
    (exact branch), chi-square against scipy.stats.binom over many bins, the
    independence of the four bins of a quad, and the normal branch's moments
    and distribution."""
    if exact_max > EXACT_CAP:
        raise ValueError(f"exact_max above {EXACT_CAP}")
    key = seed_key(seed)
    evpl = ((event_id << 4) | (plane_id & 15)) & 0xFFFFFFFF
    quad = (wire * ((nticks + 3) // 4) + tick // 4) & 0xFFFFFFFF
    return int(_lib().wso_binomial(int(N), float(p), int(exact_max), key, quad, tick % 4,
                                   depo & 0xFFFFFFFF, evpl))


def binomial_invert(N: int, p: float, x0) -> np.ndarray:
    """Exact-branch survivor counts for Philox words x0 (the CDF inversion of
    the Sec. 3.1 reading), vectorised over x0.

    Pinned exhaustively against the Binomial pmf over all 2^24 values of
    the word's top 24 bits."""
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.uint32).ravel())
    k = np.zeros(x.shape[0], dtype=np.int64)
    _lib().wso_binomial_invert_many(int(N), float(p), x.shape[0], x, k)
    return k


# ---------------------------------------------------------------- diffusion
def sigmas(t_us, DL_: float = DL, DT_: float = DT, v: float = V):
    """sigma_L [us] = sqrt(2 D_L t)/v and sigma_T [mm] = sqrt(2 D_T t) (Sec. 2.2).

    Pinned by closed-form values."""
    t = _c64(t_us)
    st = np.zeros(t.shape[0]); sx = np.zeros(t.shape[0])
    _lib().wso_sigmas(t.shape[0], t, DL_, DT_, v, st, sx)
    return st, sx


def axis_weights(mu: float, sigma: float, delta: float, nsig: float = NSIGMA):
    """(first bin, weights) of a truncated, binned 1D Gaussian (Sec. 2.2).

    Pinned against Gauss-Legendre quadrature of the Gaussian density."""
    lo = ctypes.c_int64(0)
    cap = 1 << 16
    w = np.zeros(cap)
    n = _lib().wso_axis_weights(float(mu), float(sigma), float(delta), float(nsig), cap,
                                ctypes.byref(lo), w)
    if n < 0:
        raise ValueError("patch too large for the oracle")
    return int(lo.value), w[:n].copy()


# ------------------------------------------------------------ raster+scatter
def raster_scatter(q, x_mm, t_us, nwires: int, nticks: int, *, sig_t_us=None, sig_x_mm=None,
                   pitch_mm: float = PITCH_MM, tick_us: float = TICK_US, nsig: float = NSIGMA,
                   DL_: float = DL, DT_: float = DT, v: float = V, fluctuate: bool = False,
                   p: float = 1.0, seed: int = 0, event_id: int = 0, plane_id: int = 0,
                   exact_max: int = EXACT_MAX, depo_offset: int = 0, return_skipped: bool = False):
    """Raster every depo into its patch and scatter-add into S[wire][tick] (FP64).

    Sec. 2.2 (raster, scatter-add), Sec. 3.1 (binomial fluctuation).
    fluctuate: False/0 expected value, True/1 a binomial per bin, 2 the
    charge-conserving multinomial split of each depo's survivors.
    depo_offset: index of the first depo in the event's whole list (the
    random counters carry each depo's index in that list).  Pinned by patch
    sums (closed form), linearity and the pins of its parts; the
    multinomial by exact conservation and the multinomial's moments; slices
    with their offsets sum to the whole list."""
    q = _c64(q); x = _c64(x_mm); t = _c64(t_us)
    st = None if sig_t_us is None else _c64(sig_t_us)
    sx = None if sig_x_mm is None else _c64(sig_x_mm)
    if fluctuate and exact_max > EXACT_CAP:
        raise ValueError(f"exact_max above {EXACT_CAP}")
    S = np.zeros((nwires, nticks))
    skipped = _lib().wso_raster_scatter(
        q.shape[0], q, x, t, _opt_ptr(st), _opt_ptr(sx), nwires, nticks, pitch_mm, tick_us,
        nsig, DL_, DT_, v, int(fluctuate), float(p), int(seed) & (2 ** 64 - 1),
        event_id & 0xFFFFFFFF, plane_id & 0xFFFFFFFF, int(depo_offset) & 0xFFFFFFFF, int(exact_max), S)
    return (S, int(skipped)) if return_skipped else S


def patch_extents(x_mm, t_us, nwires: int, nticks: int, *, sig_t_us=None, sig_x_mm=None,
                  pitch_mm: float = PITCH_MM, tick_us: float = TICK_US, nsig: float = NSIGMA,
                  DL_: float = DL, DT_: float = DT, v: float = V):
    """Per-depo (w0, nw, t0, nt) of each patch clipped to the grid, and the bin total."""
    x = _c64(x_mm); t = _c64(t_us)
    n = x.shape[0]
    st = None if sig_t_us is None else _c64(sig_t_us)
    sx = None if sig_x_mm is None else _c64(sig_x_mm)
    w0 = np.zeros(n, np.int32); nw = np.zeros(n, np.int32)
    t0 = np.zeros(n, np.int32); nt = np.zeros(n, np.int32)
    total = _lib().wso_patch_extents(n, x, t, _opt_ptr(st), _opt_ptr(sx), nwires, nticks,
                                     pitch_mm, tick_us, nsig, DL_, DT_, v, w0, nw, t0, nt)
    return w0, nw, t0, nt, int(total)


# -------------------------------------------------------------- convolution
def convolve_fft(S, R, wire_center: int, circular: bool = False) -> np.ndarray:
    """Eq. 2: FT of S, multiply by the FT of R, inverse FT (numpy, FP64).

    R[r][j] is the response at wire offset r - wire_center and tick offset j.
    Linear mode transforms at the full linear-convolution size (nw + Kw - 1,
    nt + Kt - 1), so nothing wraps, and keeps the grid window; circular mode
    transforms at the grid size with the response wrapped onto it.

    Pinned against the direct sum of Eq. 1 and scipy.signal.convolve2d."""
    S = np.asarray(S, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    nw, nt = S.shape
    kw, kt = R.shape
    if circular:
        Rc = np.zeros((nw, nt))
        for r in range(kw):
            for j in range(kt):
                Rc[(r - wire_center) % nw, j % nt] += R[r, j]
        return np.fft.irfft2(np.fft.rfft2(S) * np.fft.rfft2(Rc), s=(nw, nt))
    lw, lt = nw + kw - 1, nt + kt - 1
    full = np.fft.irfft2(np.fft.rfft2(S, s=(lw, lt)) * np.fft.rfft2(R, s=(lw, lt)), s=(lw, lt))
    return np.ascontiguousarray(full[wire_center:wire_center + nw, :nt])


def convolve_direct(S, R, wire_center: int, circular: bool = False) -> np.ndarray:
    """Eq. 1 as a direct double sum (C).  Brute force for small grids."""
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
    R32 = _c32(R)
    nw, nt = S.shape
    M = np.zeros_like(S)
    _lib().wso_convolve_direct(S, nw, nt, R32, R32.shape[0], R32.shape[1], int(wire_center),
                               int(bool(circular)), M)
    return M


def convolve_points(S, R, wire_center: int, pw, pt, circular: bool = False) -> np.ndarray:
    """Eq. 1's direct sum at selected output points (w[i], t[i])."""
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
    R32 = _c32(R)
    pw = np.ascontiguousarray(np.asarray(pw, dtype=np.int32))
    pt = np.ascontiguousarray(np.asarray(pt, dtype=np.int32))
    out = np.zeros(pw.shape[0])
    _lib().wso_convolve_points(S, S.shape[0], S.shape[1], R32, R32.shape[0], R32.shape[1],
                               int(wire_center), int(bool(circular)), pw.shape[0], pw, pt, out)
    return out


def simulate(q, x_mm, t_us, nwires: int, nticks: int, R, wire_center: int = 10, *,
             circular: bool = False, noise_amp=None, noise_coh=None, noise_group: int = 1,
             fft_len_tick: int = 0, **kw) -> np.ndarray:
    """The whole hot path: raster, (fluctuate), scatter-add, convolve (Eq. 2),
    plus the noise term of Eq. 1 when noise_amp is given (on the transform
    length fft_len_tick, by default ``fft_len`` of the plane)."""
    S = raster_scatter(q, x_mm, t_us, nwires, nticks, **kw)
    M = convolve_fft(S, R, wire_center, circular)
    if noise_amp is not None:
        kt = np.asarray(R).shape[1]
        L = fft_len_tick or fft_len(nticks if circular else nticks + kt - 1)
        nk = {k: kw[k] for k in ("seed", "event_id", "plane_id") if k in kw}
        M = M + noise(nwires, nticks, L, noise_amp, noise_coh, noise_group, **nk)
    return M


def fft_len(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n: the tick axis's default transform length
    (n = nticks + K_t - 1 in linear mode, nticks in circular mode)."""
    m = max(int(n), 1)
    while True:
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            return m
        m += 1


# -------------------------------------------------------------------- noise
def noise_spectrum(nwires: int, L: int, amp, coh=None, group: int = 1, *, seed: int = 0,
                   event_id: int = 0, plane_id: int = 0) -> np.ndarray:
    """Nhat_w[k], k = 0 .. L/2, of the noise term N(t, x) of Eq. 1 (reading
    in ``wsoracle.c``): incoherent amplitudes amp[k] per wire plus coherent
    amplitudes coh[k] shared by groups of ``group`` consecutive wires, with
    complex normals from Philox words by Box-Muller.

    Pinned by the normality and independence of its draws and, through
    ``noise``, by the closed-form variance and covariances."""
    nfreq = L // 2 + 1
    a = _c64(amp)
    if a.shape != (nfreq,):
        raise ValueError("amp needs L/2 + 1 entries")
    c = None if coh is None else _c64(coh)
    if c is not None and (c.shape != (nfreq,) or group < 1):
        raise ValueError("coh needs L/2 + 1 entries and group >= 1")
    re = np.zeros((nwires, nfreq)); im = np.zeros((nwires, nfreq))
    evpl = ((event_id << 4) | (plane_id & 15)) & 0xFFFFFFFF
    _lib().wso_noise_spectrum(int(nwires), int(L), a, _opt_ptr(c), int(group), seed_key(seed), evpl, re, im)
    return re + 1j * im


def noise(nwires: int, nticks: int, L: int, amp, coh=None, group: int = 1, **kw) -> np.ndarray:
    """n_w[t] for t < nticks: the inverse real DFT (1/L normalisation, numpy)
    of ``noise_spectrum`` over the Hermitian extension.

    Pinned by the closed forms of its per-sample variance (1/L^2) sum_k A^2,
    its autocovariance and the within- and across-group covariances, and by
    a direct DFT sum on small lengths."""
    spec = noise_spectrum(nwires, L, amp, coh, group, **kw)
    return np.ascontiguousarray(np.fft.irfft(spec, n=L, axis=1)[:, :nticks])


# ------------------------------------------------------------ impact sampling
def raster_scatter_impacts(q, x_mm, t_us, nwires: int, nticks: int, impacts: int, *,
                           pitch_mm: float = PITCH_MM, **kw) -> np.ndarray:
    """The raster with the pitch axis binned at pitch/impacts: fine row
    f = w * impacts + i holds the charge of wire w at sub-pitch position i
    (the position's bin covers [(w + i/I) pitch, (w + (i+1)/I) pitch)).
    Same truncation, weights and fluctuation as ``raster_scatter`` on that
    finer grid.  Pinned by the fine rows of a wire summing to the wire's
    coarse bin (expected-value mode) and by the point charge landing in its
    sub-position's rows."""
    return raster_scatter(q, x_mm, t_us, nwires * impacts, nticks, pitch_mm=pitch_mm / impacts, **kw)


def convolve_impacts(S_fine, R, wire_center: int, circular: bool = False) -> np.ndarray:
    """Eq. 1 with a response that depends on the charge's position inside
    the pitch: M = sum_i R[i] (*) S_i with S_i[w] = S_fine[w * I + i]
    (R: impacts x K_w x K_t), each term by ``convolve_fft``.  Pinned by the
    direct sum of Eq. 1 per impact and by equal responses reducing it to
    the plain convolution of the summed grid."""
    R = np.asarray(R, dtype=np.float64)
    I = R.shape[0]
    S_fine = np.asarray(S_fine, dtype=np.float64)
    nw = S_fine.shape[0] // I
    M = np.zeros((nw, S_fine.shape[1]))
    for i in range(I):
        M += convolve_fft(S_fine[i::I], R[i], wire_center, circular)
    return M


def simulate_impacts(q, x_mm, t_us, nwires: int, nticks: int, R, wire_center: int = 10, *,
                     circular: bool = False, **kw) -> np.ndarray:
    """The hot path with sub-pitch impact positions (R: impacts x K_w x K_t)."""
    I = np.asarray(R).shape[0]
    S = raster_scatter_impacts(q, x_mm, t_us, nwires, nticks, I, **kw)
    return convolve_impacts(S, R, wire_center, circular)


# ------------------------------------------------------------------ adjoint
def convolve_adjoint(G, R, wire_center: int, circular: bool = False) -> np.ndarray:
    """Adjoint of ``convolve_fft`` applied to G = dL/dM: dL/dS[w][t] =
    sum_{r,j} R[r][j] G[w + r - c][t + j] (G zero outside the grid in linear
    mode, indices wrapping in circular mode), via numpy's FFT.

    Pinned by the dot-product identity <A S, G> = <S, A^T G>."""
    G = np.asarray(G, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    nw, nt = G.shape
    kw, kt = R.shape
    if circular:
        Rc = np.zeros((nw, nt))
        for r in range(kw):
            for j in range(kt):
                Rc[(r - wire_center) % nw, j % nt] += R[r, j]
        return np.fft.irfft2(np.fft.rfft2(G) * np.conj(np.fft.rfft2(Rc)), s=(nw, nt))
    # correlation = convolution with the response flipped on both axes
    Rf = R[::-1, ::-1]
    lw, lt = nw + kw - 1, nt + kt - 1
    full = np.fft.irfft2(np.fft.rfft2(G, s=(lw, lt)) * np.fft.rfft2(Rf, s=(lw, lt)), s=(lw, lt))
    c2 = kw - 1 - wire_center
    return np.ascontiguousarray(full[c2:c2 + nw, kt - 1:kt - 1 + nt])


def response_grad(G, S, kw: int, kt: int, wire_center: int, circular: bool = False) -> np.ndarray:
    """dL/dR[r][j] = sum_{w,t} G[w][t] S[w - (r - c)][t - j] (S zero outside
    the grid, or wrapped), the cross-correlation of G and S at the response's
    lags, via numpy's FFT.  Pinned by finite differences in R (L is linear
    in R) and by the dot-product identity."""
    G = np.asarray(G, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    nw, nt = G.shape
    out = np.zeros((kw, kt))
    if circular:
        C = np.fft.irfft2(np.fft.rfft2(G) * np.conj(np.fft.rfft2(S)), s=(nw, nt))
        for r in range(kw):
            for j in range(kt):
                out[r, j] = C[(r - wire_center) % nw, j % nt]
        return out
    lw, lt = nw + kw, nt + kt
    C = np.fft.irfft2(np.fft.rfft2(G, s=(lw, lt)) * np.conj(np.fft.rfft2(S, s=(lw, lt))), s=(lw, lt))
    for r in range(kw):
        d = r - wire_center
        out[r, :] = C[d % lw, :kt]
    return out


def depo_grads(q, x_mm, t_us, nwires: int, nticks: int, dS, *, sig_t_us=None, sig_x_mm=None,
               pitch_mm: float = PITCH_MM, tick_us: float = TICK_US, nsig: float = NSIGMA,
               DL_: float = DL, DT_: float = DT, v: float = V, p: float = 1.0):
    """(gq, gx, gt, gDL, gDT): gradients of L through the expected-value
    raster given dS = dL/dS (closed form in C).  Pinned by central finite
    differences of ``raster_scatter``."""
    q = _c64(q); x = _c64(x_mm); t = _c64(t_us)
    n = q.shape[0]
    st = None if sig_t_us is None else _c64(sig_t_us)
    sx = None if sig_x_mm is None else _c64(sig_x_mm)
    dS = np.ascontiguousarray(np.asarray(dS, dtype=np.float64))
    gq = np.zeros(n); gx = np.zeros(n); gt = np.zeros(n)
    gDL = ctypes.c_double(0.0); gDT = ctypes.c_double(0.0)
    _lib().wso_depo_grads(n, q, x, t, _opt_ptr(st), _opt_ptr(sx), nwires, nticks, pitch_mm, tick_us, nsig,
                          DL_, DT_, v, float(p), dS, gq, gx, gt, ctypes.byref(gDL), ctypes.byref(gDT))
    return gq, gx, gt, float(gDL.value), float(gDT.value)


def simulate_backward(q, x_mm, t_us, nwires: int, nticks: int, R, wire_center: int, G, *,
                      circular: bool = False, **kw):
    """All gradients of L given G = dL/dM: (gq, gx, gt, gDL, gDT, gR)."""
    dS = convolve_adjoint(G, R, wire_center, circular)
    rkw = {k: v for k, v in kw.items() if k in ("sig_t_us", "sig_x_mm", "pitch_mm", "tick_us", "nsig",
                                                 "DL_", "DT_", "v", "p")}
    gq, gx, gt, gDL, gDT = depo_grads(q, x_mm, t_us, nwires, nticks, dS, **rkw)
    S = raster_scatter(q, x_mm, t_us, nwires, nticks, **rkw)
    gR = response_grad(G, S, np.asarray(R).shape[0], np.asarray(R).shape[1], wire_center, circular)
    return gq, gx, gt, gDL, gDT, gR


def simulate_backward_impacts(q, x_mm, t_us, nwires: int, nticks: int, R, wire_center: int, G, *,
                              circular: bool = False, **kw):
    """All gradients of L given G = dL/dM on a plane with sub-pitch impact
    positions (R: impacts x K_w x K_t; the forward is ``simulate_impacts``,
    M = sum_i R_i (*) S_i with S_i[w] = S_fine[w * I + i]):
    dL/dS_fine[w * I + i] = (R_i's convolution adjoint of G)[w]; the depo
    gradients of the raster on the fine grid (nwires * I bins at pitch / I,
    the forward's own binning); dL/dR_i = the response gradient of G against
    S_i.  Returns (gq, gx, gt, gDL, gDT, gR) with gR shaped like R.  Pinned
    by central finite differences of the impact simulation's loss."""
    R = np.asarray(R, dtype=np.float64)
    I, kw_, kt_ = R.shape
    rkw = {k: v for k, v in kw.items() if k in ("sig_t_us", "sig_x_mm", "pitch_mm", "tick_us", "nsig",
                                                 "DL_", "DT_", "v", "p")}
    pitch = rkw.pop("pitch_mm", PITCH_MM)
    dS = np.zeros((nwires * I, nticks))
    for i in range(I):
        dS[i::I] = convolve_adjoint(G, R[i], wire_center, circular)
    gq, gx, gt, gDL, gDT = depo_grads(q, x_mm, t_us, nwires * I, nticks, dS, pitch_mm=pitch / I, **rkw)
    S = raster_scatter_impacts(q, x_mm, t_us, nwires, nticks, I, pitch_mm=pitch, **rkw)
    gR = np.stack([response_grad(G, S[i::I], kw_, kt_, wire_center, circular) for i in range(I)])
    return gq, gx, gt, gDL, gDT, gR
