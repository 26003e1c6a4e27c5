/*
 * FP64 oracle for the LArTPC signal-simulation hot path (arXiv 2203.02479).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Plain single-threaded loops in double precision, following the method in
 * the order the paper gives it:
 *   - diffusion of each depo into a 2D distribution (Sec. 2.2),
 *   - raster: binning that distribution into a patch (Sec. 2.2, "Raster"),
 *   - optional binomial charge fluctuation (Sec. 3.1),
 *   - scatter-add of patches into a dense wire x tick grid (Sec. 2.2,
 *     "Scatter-add"; Sec. 2.3 dense matrix),
 *   - the convolution of Eq. 1 written out as a direct sum (the FFT form of
 *     Eq. 2 lives in the Python layer, on numpy's FFT).
 * Where the paper is silent (bin edges, truncation, normalisation, the
 * fluctuation sampler and its random stream) the readings are stated next to
 * the code that takes them.
 *
 * Every function below is pinned by tests against something other than
 * itself: Gauss-Legendre quadrature of the Gaussian (bin weights), closed
 * forms (patch sums, delta response), cuRAND's host Philox generator (the
 * random stream), the exact binomial pmf (the sampler, over every value of
 * its random word), binomial moments, and scipy's convolve2d
 * (the convolution).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, as defined by Salmon, Moraes, Dror
 * and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten
 * rounds of two 32x32->64 multiplies by fixed odd constants, the high halves
 * XORed with the other two counter words and the key, the key bumped by the
 * golden-ratio and sqrt(3)-1 Weyl constants between rounds. */
#define WSO_PHILOX_M0 0xD2511F53u
#define WSO_PHILOX_M1 0xCD9E8D57u
#define WSO_PHILOX_W0 0x9E3779B9u
#define WSO_PHILOX_W1 0xBB67AE85u

void wso_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += WSO_PHILOX_W0; k1 += WSO_PHILOX_W1; }
        uint64_t p0 = (uint64_t)WSO_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)WSO_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Diffusion along the drift (Sec. 2.2): longitudinal width in time
 * sigma_L = sqrt(2 D_L t) / v, transverse width in pitch sigma_T =
 * sqrt(2 D_T t).  Units: mm, microseconds. */
void wso_sigmas(int64_t n, const double* t_us, double DL, double DT, double v,
                double* sig_t_us, double* sig_x_mm)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = t_us[i];
        sig_t_us[i] = sqrt(2.0 * DL * t) / v;
        sig_x_mm[i] = sqrt(2.0 * DT * t);
    }
}

/* ------------------------------------------------------------------------ */
/* Raster along one axis (Sec. 2.2, "Raster").
 *
 * Readings (the paper only says each distribution is "binned"):
 *   - bin k covers [k*delta, (k+1)*delta);
 *   - the Gaussian is truncated to [mu - nsig*sigma, mu + nsig*sigma] and
 *     the bins overlapping that window form the patch;
 *   - each bin's weight is the Gaussian mass on the bin clipped to the
 *     window, Phi(b) - Phi(a) = (erf(b') - erf(a'))/2, divided by the
 *     window's total mass erf(nsig/sqrt 2), so the weights sum to one;
 *   - sigma <= 1e-6*delta is a point charge: weight 1 in floor(mu/delta).
 * Returns the number of bins n and writes lo (first bin) and w[0..n);
 * w must hold at least maxn values; returns -1 if n > maxn. */
int wso_axis_weights(double mu, double sigma, double delta, double nsig,
                     int maxn, int64_t* lo, double* w)
{
    if (!(sigma > 1e-6 * delta)) {
        *lo = (int64_t)floor(mu / delta);
        if (maxn < 1) return -1;
        w[0] = 1.0;
        return 1;
    }
    double a = mu - nsig * sigma, b = mu + nsig * sigma;
    int64_t klo = (int64_t)floor(a / delta), khi = (int64_t)floor(b / delta);
    int64_t n = khi - klo + 1;
    if (n > maxn) return -1;
    double norm = erf(nsig / sqrt(2.0));
    double s2 = sqrt(2.0) * sigma;
    for (int64_t k = klo; k <= khi; ++k) {
        double e0 = fmax((double)k * delta, a);
        double e1 = fmin((double)(k + 1) * delta, b);
        w[k - klo] = 0.5 * (erf((e1 - mu) / s2) - erf((e0 - mu) / s2)) / norm;
    }
    *lo = klo;
    return (int)n;
}

/* ------------------------------------------------------------------------ */
/* Binomial charge fluctuation (Sec. 3.1: the CPU reference draws binomial
 * numbers; the sampler itself is not given).  Reading: each bin holds
 * N = floor(q*w + 1/2) electrons, each surviving independently with
 * probability p; the bins draw independently.  Random stream: Philox4x32-10
 * keyed by the seed; one block serves a quad, the four consecutive ticks
 * 4g .. 4g+3 of one wire w of one depo, with the counter
 * (0, w*ceil(nticks/4) + g, depo index, event << 4 | plane), and bin (w, k)
 * takes word k % 4 of its quad's block.  That one word decides the bin:
 *   - N <= exact_max (at most WSO_EXACT_CAP): inversion of the Binomial CDF
 *     in single precision from the word's top 24 bits (see
 *     wso_binomial_invert).
 *   - N > exact_max: normal approximation, Box-Muller on the word's two
 *     16-bit halves, u1 = (x >> 16 + 1/2)/2^16, u2 = (x & 0xFFFF + 1/2)/2^16,
 *     z = sqrt(-2 ln u1) cos(2 pi u2) (so |z| <= sqrt(2 ln 2^17) = 4.86),
 *     k = clamp(floor(N p + z sqrt(N p (1 - p)) + 1/2), 0, N), p = T/2^32
 *     with T = floor(p * 2^32).
 *   - p >= 1 keeps every electron, p <= 0 none.
 * The four words of a block are independent, so are the bins of a quad. */
#define WSO_EXACT_CAP 64

uint32_t wso_survive_threshold(double p)
{
    if (!(p > 0.0)) return 0u;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return (uint32_t)floor(p * 4294967296.0);
}

/* Sequential-search inversion of the Binomial(N, p) CDF, every step a
 * single-precision operation in a fixed order (so that any IEEE-754 machine
 * takes the same decisions):
 *   pf = (float)p; the search runs on s = min(pf, 1 - pf) and the count is
 *   mirrored (N - k) when pf > 1/2;
 *   f_0 = (1 - s)^N by binary powering over the bits of N, low bit first;
 *   r = s / (1 - s);  f_{k+1} = ((f_k r) (N - k)) (1/(k+1)), where 1/(k+1) is
 *   the float reciprocal;  F_k = F_{k-1} + f_k;
 *   u = (x0 >> 8) 2^-24;  k = the first k with u < F_k, else N.
 * The probability of each k is F_k - F_{k-1} over the 2^24 values of u,
 * Binomial(N, s) up to float rounding.  N <= WSO_EXACT_CAP keeps f_0 above
 * 2^-64, a normal float. */
int64_t wso_binomial_invert(int64_t N, double p, uint32_t x0)
{
    const float pf = (float)p;
    const int flip = pf > 0.5f;
    const float s = flip ? 1.0f - pf : pf;
    const float r = s / (1.0f - s);
    float base = 1.0f - s, f = 1.0f;
    for (int64_t n = N; n > 0; n >>= 1) {
        if (n & 1) f = f * base;
        base = base * base;
    }
    const float u = (float)(x0 >> 8) * 5.9604644775390625e-8f;
    float F = f;
    int64_t k = 0;
    while (!(u < F) && k < N) {
        const float inv = 1.0f / (float)(k + 1);
        f = f * r;
        f = f * (float)(N - k);
        f = f * inv;
        F = F + f;
        ++k;
    }
    return flip ? N - k : k;
}

/* wso_binomial_invert over an array of words (for the exhaustive pin). */
void wso_binomial_invert_many(int64_t N, double p, int64_t n, const uint32_t* x0, int64_t* k)
{
    for (int64_t i = 0; i < n; ++i) k[i] = wso_binomial_invert(N, p, x0[i]);
}

/* Quad index and word of bin (w, k) on a grid of nticks ticks. */
static uint32_t wso_quad(int64_t w, int64_t k, int nticks) { return (uint32_t)(w * ((nticks + 3) / 4) + k / 4); }

int64_t wso_binomial(int64_t N, double p, int exact_max, const uint32_t key[2],
                     uint32_t quad, uint32_t word, uint32_t depo, uint32_t evpl)
{
    if (N <= 0) return 0;
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return N;
    if (exact_max > WSO_EXACT_CAP || word > 3u) return -1;
    uint32_t T = wso_survive_threshold(p);
    uint32_t ctr[4], x[4];
    ctr[0] = 0; ctr[1] = quad; ctr[2] = depo; ctr[3] = evpl;
    wso_philox4x32_10(ctr, key, x);
    const uint32_t xw = x[word];
    if (N <= exact_max) return wso_binomial_invert(N, p, xw);
    double u1 = ((double)(xw >> 16) + 0.5) / 65536.0;
    double u2 = ((double)(xw & 0xFFFFu) + 0.5) / 65536.0;
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    double pe = (double)T / 4294967296.0;
    double mean = (double)N * pe;
    double k = floor(mean + z * sqrt(mean * (1.0 - pe)) + 0.5);
    if (k < 0.0) k = 0.0;
    if (k > (double)N) k = (double)N;
    return (int64_t)k;
}

/* ------------------------------------------------------------------------ */
/* Charge-conserving fluctuation (alternative sampler; the paper's CPU
 * reference draws binomials, Sec. 3.1, without saying how the bins share a
 * depo's electrons).  Reading: the depo carries N = floor(q + 1/2)
 * electrons; K ~ Binomial(N, p) survive (block (5, 0, depo, evpl), the
 * sampler of wso_binomial); the K are spread over the patch multinomially
 * with the bin weights w_x[j] w_t[i]: over the in-grid wires in order by
 * conditional binomials n_j ~ Binomial(rem, w_x[j] / W) (W the wire mass
 * not yet visited, W = 1 at the start, both in float; block
 * (4, wire, depo, evpl)), then within wire j over its in-grid ticks the
 * same way (block (3, wire * nticks + tick, depo, evpl)).  Electrons still
 * unassigned after the last in-grid bin belong to bins off the grid and are
 * lost; when every bin of an axis's window is on the grid, that axis's
 * last bin takes all that remain, so an interior depo keeps exactly K.
 * A conditional draw Binomial(n, pr), pr a float: pr <= 0 gives 0, pr >= 1
 * gives n; n <= exact_max: the float inversion of wso_binomial_invert; else
 * the normal approximation from words 0, 1 of the block (Box-Muller as in
 * wso_binomial), k = clamp(floor(n pr + z sqrt(n pr (1 - pr)) + 1/2), 0, n). */
static int64_t wso_binom_var(int64_t n, float pr, int exact_max, const uint32_t key[2],
                             uint32_t c0, uint32_t c1, uint32_t depo, uint32_t evpl)
{
    if (n <= 0 || !(pr > 0.0f)) return 0;
    if (pr >= 1.0f) return n;
    uint32_t ctr[4] = {c0, c1, depo, evpl}, x[4];
    wso_philox4x32_10(ctr, key, x);
    if (n <= exact_max) return wso_binomial_invert(n, (double)pr, x[0]);
    double u1 = ((double)x[0] + 0.5) / 4294967296.0;
    double u2 = ((double)x[1] + 0.5) / 4294967296.0;
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    double mean = (double)n * (double)pr;
    double k = floor(mean + z * sqrt(mean * (1.0 - (double)pr)) + 0.5);
    if (k < 0.0) k = 0.0;
    if (k > (double)n) k = (double)n;
    return (int64_t)k;
}

/* Survivors of the depo, then its multinomial split, added into S. */
static void wso_multinomial_depo(double q, int64_t wlo, int nw, const double* wx, int64_t klo, int nt,
                                 const double* wt, int nwires, int nticks, double p, int exact_max,
                                 const uint32_t key[2], uint32_t depo, uint32_t evpl, double* S)
{
    int64_t N = (int64_t)floor(q + 0.5);
    if (N <= 0 || !(p > 0.0)) return;
    int64_t K = N;
    if (p < 1.0) {
        uint32_t ctr[4] = {5u, 0u, depo, evpl}, x[4];
        wso_philox4x32_10(ctr, key, x);
        if (N <= exact_max) {
            K = wso_binomial_invert(N, p, x[0]);
        } else {
            const uint32_t T = wso_survive_threshold(p);
            double u1 = ((double)x[0] + 0.5) / 4294967296.0;
            double u2 = ((double)x[1] + 0.5) / 4294967296.0;
            double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            double pe = (double)T / 4294967296.0;
            double mean = (double)N * pe;
            double k = floor(mean + z * sqrt(mean * (1.0 - pe)) + 0.5);
            K = (int64_t)(k < 0.0 ? 0.0 : (k > (double)N ? (double)N : k));
        }
    }
    int64_t rem = K;
    float Wx = 1.0f;
    const int64_t wlast = wlo + nw - 1, klast = klo + nt - 1;
    /* the last bin takes all that remain only if no bin of the axis is off the grid */
    const int wfull = wlo >= 0 && wlast < nwires, kfull = klo >= 0 && klast < nticks;
    for (int a = 0; a < nw && rem > 0; ++a) {
        const int64_t w = wlo + a;
        if (w < 0 || w >= nwires) continue;
        const float wf = (float)wx[a];
        const float pr = (wfull && w == wlast) ? 1.0f : wf / Wx;
        const int64_t nj = wso_binom_var(rem, pr, exact_max, key, 4u, (uint32_t)w, depo, evpl);
        rem -= nj;
        Wx = Wx - wf;
        int64_t rem2 = nj;
        float Wt = 1.0f;
        for (int b = 0; b < nt && rem2 > 0; ++b) {
            const int64_t k = klo + b;
            if (k < 0 || k >= nticks) continue;
            const float tf = (float)wt[b];
            const float pt = (kfull && k == klast) ? 1.0f : tf / Wt;
            const int64_t m = wso_binom_var(rem2, pt, exact_max, key, 3u, (uint32_t)(w * (int64_t)nticks + k),
                                            depo, evpl);
            rem2 -= m;
            Wt = Wt - tf;
            S[w * (int64_t)nticks + k] += (double)m;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One plane's raster + fluctuation + scatter-add (Sec. 2.2).  Depos are
 * processed one by one; each patch bin inside the nwires x nticks grid is
 * added into S (row-major [wire][tick], double).  Bins outside the grid are
 * dropped: charge leaving the readout is lost.  A depo with a non-finite
 * input or negative drift time contributes nothing and is counted in the
 * return value.
 *
 * sig_t_us / sig_x_mm may be NULL, in which case they come from diffusion.
 * If fluctuate == 0 a bin receives the expected value p*q*w_t*w_x; if 1 a
 * binomial count (see wso_binomial); if 2 the depo's surviving electrons are
 * spread multinomially (see wso_multinomial_depo).  depo0 is the index of
 * depo 0 in the event's whole depo list: the random counters carry the
 * depo's index in that list (depo0 + i), so a list rastered in slices
 * draws exactly as in one call. */
#define WSO_MAXBINS 65536

int64_t wso_raster_scatter(int64_t n, const double* q, const double* x_mm, const double* t_us,
                           const double* sig_t_us, const double* sig_x_mm,
                           int nwires, int nticks, double pitch_mm, double tick_us,
                           double nsig, double DL, double DT, double v,
                           int fluctuate, double p, uint64_t seed, uint32_t event_id,
                           uint32_t plane_id, uint32_t depo0, int exact_max, double* S)
{
    if (fluctuate && exact_max > WSO_EXACT_CAP) return -1;
    double* wt = (double*)malloc(sizeof(double) * WSO_MAXBINS);
    double* wx = (double*)malloc(sizeof(double) * WSO_MAXBINS);
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t evpl = (event_id << 4) | (plane_id & 15u);
    int64_t skipped = 0;
    for (int64_t i = 0; i < n; ++i) {
        double qi = q[i], xi = x_mm[i], ti = t_us[i];
        double st, sx;
        if (sig_t_us) { st = sig_t_us[i]; sx = sig_x_mm[i]; }
        else { st = sqrt(2.0 * DL * ti) / v; sx = sqrt(2.0 * DT * ti); }
        if (!isfinite(qi) || !isfinite(xi) || !isfinite(ti) || !isfinite(st) || !isfinite(sx) ||
            st < 0.0 || sx < 0.0) { ++skipped; continue; }
        int64_t klo, wlo;
        int nt = wso_axis_weights(ti, st, tick_us, nsig, WSO_MAXBINS, &klo, wt);
        int nw = wso_axis_weights(xi, sx, pitch_mm, nsig, WSO_MAXBINS, &wlo, wx);
        if (nt < 0 || nw < 0) { ++skipped; continue; }
        if (fluctuate == 2) {
            wso_multinomial_depo(qi, wlo, nw, wx, klo, nt, wt, nwires, nticks, p, exact_max, key,
                                 depo0 + (uint32_t)i, evpl, S);
            continue;
        }
        for (int a = 0; a < nw; ++a) {
            int64_t w = wlo + a;
            if (w < 0 || w >= nwires) continue;
            for (int b = 0; b < nt; ++b) {
                int64_t k = klo + b;
                if (k < 0 || k >= nticks) continue;
                double val;
                if (fluctuate) {
                    int64_t N = (int64_t)floor(qi * wt[b] * wx[a] + 0.5);
                    val = (double)wso_binomial(N, p, exact_max, key, wso_quad(w, k, nticks), (uint32_t)(k % 4),
                                               depo0 + (uint32_t)i, evpl);
                } else {
                    val = p * qi * wt[b] * wx[a];
                }
                S[w * (int64_t)nticks + k] += val;
            }
        }
    }
    free(wt); free(wx);
    return skipped;
}

/* Per-depo patch extents, clipped to the grid (for comparing patch lists).
 * Writes w0, nw, t0, nt per depo (nw = nt = 0 for an empty or skipped
 * patch).  Returns the total number of in-grid bins. */
int64_t wso_patch_extents(int64_t n, const double* x_mm, const double* t_us,
                          const double* sig_t_us, const double* sig_x_mm,
                          int nwires, int nticks, double pitch_mm, double tick_us,
                          double nsig, double DL, double DT, double v,
                          int32_t* w0, int32_t* nw, int32_t* t0, int32_t* nt)
{
    double* tmp = (double*)malloc(sizeof(double) * WSO_MAXBINS);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        double xi = x_mm[i], ti = t_us[i];
        double st, sx;
        if (sig_t_us) { st = sig_t_us[i]; sx = sig_x_mm[i]; }
        else { st = sqrt(2.0 * DL * ti) / v; sx = sqrt(2.0 * DT * ti); }
        w0[i] = nw[i] = t0[i] = nt[i] = 0;
        if (!isfinite(xi) || !isfinite(ti) || !isfinite(st) || !isfinite(sx) || st < 0 || sx < 0)
            continue;
        int64_t klo, wlo;
        int ntt = wso_axis_weights(ti, st, tick_us, nsig, WSO_MAXBINS, &klo, tmp);
        int nww = wso_axis_weights(xi, sx, pitch_mm, nsig, WSO_MAXBINS, &wlo, tmp);
        if (ntt < 0 || nww < 0) continue;
        int64_t a0 = wlo < 0 ? 0 : wlo, a1 = wlo + nww > nwires ? nwires : wlo + nww;
        int64_t b0 = klo < 0 ? 0 : klo, b1 = klo + ntt > nticks ? nticks : klo + ntt;
        if (a1 <= a0 || b1 <= b0) continue;
        w0[i] = (int32_t)a0; nw[i] = (int32_t)(a1 - a0);
        t0[i] = (int32_t)b0; nt[i] = (int32_t)(b1 - b0);
        total += (a1 - a0) * (b1 - b0);
    }
    free(tmp);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 written out: M(t, x) = sum over t', x' of R(t - t', x - x') S(t', x')
 * on the discrete grid.  R is resp_nw x resp_nt (row-major [wire][tick]);
 * response row r holds wire offset d = r - wire_center, column j holds tick
 * offset j (causal).  circular == 0: S is zero outside the grid and M is
 * kept on the grid; circular != 0: indices wrap modulo the grid (the
 * literal discrete form of Eq. 2). */
void wso_convolve_direct(const double* S, int nwires, int nticks,
                         const float* R, int resp_nw, int resp_nt, int wire_center,
                         int circular, double* M)
{
    for (int64_t w = 0; w < nwires; ++w) {
        for (int64_t t = 0; t < nticks; ++t) {
            double acc = 0.0;
            for (int r = 0; r < resp_nw; ++r) {
                int64_t ws = w - (r - wire_center);
                if (circular) { ws %= nwires; if (ws < 0) ws += nwires; }
                else if (ws < 0 || ws >= nwires) continue;
                for (int j = 0; j < resp_nt; ++j) {
                    int64_t ts = t - j;
                    if (circular) { ts %= nticks; if (ts < 0) ts += nticks; }
                    else if (ts < 0) break;
                    acc += (double)R[r * resp_nt + j] * S[ws * nticks + ts];
                }
            }
            M[w * nticks + t] = acc;
        }
    }
}

/* The same sum at selected output points only (w[i], t[i]). */
void wso_convolve_points(const double* S, int nwires, int nticks,
                         const float* R, int resp_nw, int resp_nt, int wire_center,
                         int circular, int64_t npts, const int32_t* pw, const int32_t* pt,
                         double* out)
{
    for (int64_t i = 0; i < npts; ++i) {
        int64_t w = pw[i], t = pt[i];
        double acc = 0.0;
        for (int r = 0; r < resp_nw; ++r) {
            int64_t ws = w - (r - wire_center);
            if (circular) { ws %= nwires; if (ws < 0) ws += nwires; }
            else if (ws < 0 || ws >= nwires) continue;
            for (int j = 0; j < resp_nt; ++j) {
                int64_t ts = t - j;
                if (circular) { ts %= nticks; if (ts < 0) ts += nticks; }
                else if (ts < 0) break;
                acc += (double)R[r * resp_nt + j] * S[ws * nticks + ts];
            }
        }
        out[i] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the expected-value raster (Sec. 2.2) for dL/dS given.
 *
 * With standardized clamped edges u_e = clamp((e - mu)/sigma, -n, n), a bin's
 * weight is w = [Phi(u1) - Phi(u0)] / erf(n/sqrt 2).  An edge that sits on the
 * window bound moves with mu and sigma, so its Phi stays at Phi(+-n) and it
 * contributes nothing; an interior edge contributes
 *   dPhi(u)/dmu = -phi(u)/sigma,  dPhi(u)/dsigma = -u phi(u)/sigma.
 * The patch is p q w_t w_x, so per depo
 *   dL/dq = p sum dS w_t w_x,  dL/dmu_t = p q sum dS w_x dw_t/dmu_t, ...
 * and through diffusion sigma_L = sqrt(2 D_L t)/v, sigma_T = sqrt(2 D_T t):
 *   dL/dt += dL/dsigma_t sigma_t/(2t) + dL/dsigma_x sigma_x/(2t),
 *   dL/dD_L = sum dL/dsigma_t sigma_t/(2 D_L), dL/dD_T likewise.
 * With given widths the sigma terms stay out of dL/dt and dL/dD are zero.
 * A point-charge axis (sigma <= 1e-6 delta) has zero mu and sigma
 * derivatives. */
static int axis_weights_grad(double mu, double sigma, double delta, double nsig, int maxn, int64_t* lo,
                             double* w, double* dmu, double* dsig)
{
    if (!(sigma > 1e-6 * delta)) {
        *lo = (int64_t)floor(mu / delta);
        w[0] = 1.0; dmu[0] = 0.0; dsig[0] = 0.0;
        return 1;
    }
    double a = mu - nsig * sigma, b = mu + nsig * sigma;
    int64_t klo = (int64_t)floor(a / delta), khi = (int64_t)floor(b / delta);
    int64_t n = khi - klo + 1;
    if (n > maxn) return -1;
    double norm = erf(nsig / sqrt(2.0));
    double inv_s2pi = 1.0 / sqrt(2.0 * M_PI);
    for (int64_t k = klo; k <= khi; ++k) {
        double e0 = (double)k * delta, e1 = (double)(k + 1) * delta;
        int c0 = e0 <= a, c1 = e1 >= b;          /* edge clamped to the window bound */
        double u0 = c0 ? -nsig : (e0 - mu) / sigma;
        double u1 = c1 ? nsig : (e1 - mu) / sigma;
        double p0 = c0 ? 0.0 : exp(-0.5 * u0 * u0) * inv_s2pi;
        double p1 = c1 ? 0.0 : exp(-0.5 * u1 * u1) * inv_s2pi;
        int64_t i = k - klo;
        w[i] = 0.5 * (erf(u1 / sqrt(2.0)) - erf(u0 / sqrt(2.0))) / norm;
        dmu[i] = -(p1 - p0) / (sigma * norm);
        dsig[i] = -(u1 * p1 - u0 * p0) / (sigma * norm);
    }
    *lo = klo;
    return (int)n;
}

int64_t wso_depo_grads(int64_t n, const double* q, const double* x_mm, const double* t_us,
                       const double* sig_t_us, const double* sig_x_mm,
                       int nwires, int nticks, double pitch_mm, double tick_us,
                       double nsig, double DL, double DT, double v, double p,
                       const double* dS, double* gq, double* gx, double* gt, double* gDL, double* gDT)
{
    double *wt = malloc(sizeof(double) * WSO_MAXBINS), *mt = malloc(sizeof(double) * WSO_MAXBINS),
           *st_ = malloc(sizeof(double) * WSO_MAXBINS);
    double *wx = malloc(sizeof(double) * WSO_MAXBINS), *mx = malloc(sizeof(double) * WSO_MAXBINS),
           *sx_ = malloc(sizeof(double) * WSO_MAXBINS);
    int64_t skipped = 0;
    double sDL = 0.0, sDT = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double qi = q[i], xi = x_mm[i], ti = t_us[i];
        double st, sx;
        int given = sig_t_us != NULL;
        if (given) { st = sig_t_us[i]; sx = sig_x_mm[i]; }
        else { st = sqrt(2.0 * DL * ti) / v; sx = sqrt(2.0 * DT * ti); }
        gq[i] = gx[i] = gt[i] = 0.0;
        if (!isfinite(qi) || !isfinite(xi) || !isfinite(ti) || !isfinite(st) || !isfinite(sx) ||
            st < 0.0 || sx < 0.0) { ++skipped; continue; }
        int64_t klo, wlo;
        int nt = axis_weights_grad(ti, st, tick_us, nsig, WSO_MAXBINS, &klo, wt, mt, st_);
        int nw = axis_weights_grad(xi, sx, pitch_mm, nsig, WSO_MAXBINS, &wlo, wx, mx, sx_);
        if (nt < 0 || nw < 0) { ++skipped; continue; }
        double Sq = 0, Smt = 0, Sst = 0, Smx = 0, Ssx = 0;
        for (int a = 0; a < nw; ++a) {
            int64_t w = wlo + a;
            if (w < 0 || w >= nwires) continue;
            for (int b = 0; b < nt; ++b) {
                int64_t k = klo + b;
                if (k < 0 || k >= nticks) continue;
                double g = dS[w * (int64_t)nticks + k];
                Sq += g * wt[b] * wx[a];
                Smt += g * mt[b] * wx[a];
                Sst += g * st_[b] * wx[a];
                Smx += g * wt[b] * mx[a];
                Ssx += g * wt[b] * sx_[a];
            }
        }
        double dq = p * Sq, dmt = p * qi * Smt, dst = p * qi * Sst, dmx = p * qi * Smx, dsx = p * qi * Ssx;
        gq[i] = dq;
        gx[i] = dmx;
        gt[i] = dmt;
        if (!given && ti > 0.0) {
            gt[i] += dst * st / (2.0 * ti) + dsx * sx / (2.0 * ti);
            if (DL > 0.0) sDL += dst * st / (2.0 * DL);
            if (DT > 0.0) sDT += dsx * sx / (2.0 * DT);
        }
    }
    *gDL = sDL;
    *gDT = sDT;
    free(wt); free(mt); free(st_); free(wx); free(mx); free(sx_);
    return skipped;
}

/* ------------------------------------------------------------------------ */
/* Noise term N(t, x) of Eq. 1 (Sec. 2.1).  The paper names the term and
 * leaves it out of the ported signal path; its model is not given.  Reading
 * taken here: per wire, a stationary Gaussian process given by amplitude
 * spectra on the tick axis's transform length L, an incoherent part
 * independent per wire and a coherent part shared by the wires of a group of
 * G consecutive wires:
 *   Nhat_w[k] = A[k] xi_w[k] + Ac[k] xi'_{floor(w / G)}[k],  k = 0 .. L/2,
 * with xi = (z1 + i z2) / sqrt 2 for 0 < k < L/2 and xi = z1 at k = 0 and
 * k = L/2 (L even), and the noise waveform n_w[t] = (1/L) sum over the
 * Hermitian extension of Nhat_w[k] e^{2 pi i k t / L} (the Python layer does
 * that sum with numpy's inverse real FFT).
 * The normals: z1 = sqrt(-2 ln u1) cos(2 pi u2), z2 = sqrt(-2 ln u1)
 * sin(2 pi u2) (Box and Muller, 1958), u = (m + 1/2) / 2^23 with m the top 23
 * bits of a Philox word.  Incoherent wire w, bin k: Philox block with counter
 * (1, k, floor(w / 2), event << 4 | plane), words 2 (w mod 2) and
 * 2 (w mod 2) + 1; coherent group g: counter (2, k, floor(g / 2), same),
 * words 2 (g mod 2), 2 (g mod 2) + 1.  (The fluctuation's counters start
 * with 0, so the streams are disjoint.)
 * re, im: nwires x nfreq outputs (nfreq = L/2 + 1).  coh may be NULL. */
static void wso_normal_pair(uint32_t a, uint32_t b, double* z1, double* z2)
{
    const double u1 = ((double)(a >> 9) + 0.5) / 8388608.0;
    const double u2 = ((double)(b >> 9) + 0.5) / 8388608.0;
    const double rad = sqrt(-2.0 * log(u1));
    *z1 = rad * cos(2.0 * M_PI * u2);
    *z2 = rad * sin(2.0 * M_PI * u2);
}

static void wso_xi(int k, int L, uint32_t domain, int64_t idx, const uint32_t key[2], uint32_t evpl,
                   double* re, double* im)
{
    const uint32_t ctr[4] = {domain, (uint32_t)k, (uint32_t)(idx / 2), evpl};
    uint32_t x[4];
    wso_philox4x32_10(ctr, key, x);
    const int h = (int)(idx % 2);
    double z1, z2;
    wso_normal_pair(x[2 * h], x[2 * h + 1], &z1, &z2);
    if (k == 0 || 2 * k == L) {
        *re = z1;
        *im = 0.0;
    } else {
        *re = z1 / sqrt(2.0);
        *im = z2 / sqrt(2.0);
    }
}

void wso_noise_spectrum(int nwires, int L, const double* amp, const double* coh, int group,
                        const uint32_t key[2], uint32_t evpl, double* re, double* im)
{
    const int nfreq = L / 2 + 1;
    for (int w = 0; w < nwires; ++w) {
        for (int k = 0; k < nfreq; ++k) {
            double xr, xi;
            wso_xi(k, L, 1u, w, key, evpl, &xr, &xi);
            double sr = amp[k] * xr, si = amp[k] * xi;
            if (coh) {
                wso_xi(k, L, 2u, w / group, key, evpl, &xr, &xi);
                sr += coh[k] * xr;
                si += coh[k] * xi;
            }
            re[(int64_t)w * nfreq + k] = sr;
            im[(int64_t)w * nfreq + k] = si;
        }
    }
}
