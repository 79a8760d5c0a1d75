/*
 * EPIC imaging oracle: plain, slow, FP64 CPU implementation of the E-field
 * Parallel Imaging Correlator's data-parallel path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the library never does, and this file shares no code,
 * tables or headers with it.
 *
 * Two formulations, written from the paper:
 *
 *   O1 (epic_direct)  Eq. 4 and the block chain of Sec. 2.2: calibrate each
 *       antenna voltage, grid it through the illumination kernel W, take the
 *       unnormalised inverse 2-D Fourier transform, form the polarisation
 *       products F_p F_q^*, sum them over the integration and subtract the
 *       autocorrelation term.
 *
 *   O2 (epic_fx)      Eq. 1-3: the FX-correlator route.  Exact integer
 *       visibilities V_ab = sum_t e_a e_b^*, calibrated, gridded with the
 *       baseline kernel B = W (x) W^* (the correlation of the antenna kernel
 *       with itself) for every pair a != b, then one inverse transform.
 *       Eq. 3 states that this equals O1 once the a = b (auto) terms are
 *       dropped.
 *
 * Readings of points the paper leaves open (each is also in the design notes):
 *   - ci4 byte: real part = high nibble, imaginary = low nibble, two's
 *     complement, values -8..7 (Sec. 2.1 "4+4 complex integers").
 *   - transform: F(l) = sum_k G(k) exp(+2 pi i k.l / N), unnormalised (Eq. 4
 *     writes FT^-1; Eq. 1 fixes the exp(-2 pi i ...) visibility sign).
 *   - integration is a sum over time; flag MEAN divides by T.
 *   - products XX = F_X F_X^*, YY = F_Y F_Y^*, XY = F_X F_Y^*, YX = F_Y F_X^*
 *     (Sec. 3.2 lists V_Y V_Y^* twice; the fourth product is read as YX).
 *   - gains multiply: e~ = g e, per (channel, antenna, polarisation).
 *   - the grid is circular (indices mod N); the image is fft-shifted: output
 *     pixel (i, j) holds l = (j - N/2, i - N/2).
 *   - kernel W is stored [K][K] with index [dy + h][dx + h], h = (K-1)/2;
 *     antenna a's footprint covers cells k_a + (dx, dy).
 *   - the autocorrelation term is exactly the a = b part of F_p F_q^*:
 *     A_pq |W^(l)|^2 with A_pq = sum_a g_ap g_aq^* sum_t e_ap e_aq^* and
 *     W^(l) = sum_d W(d) exp(+2 pi i d.l / N).
 *   - antenna -> cell map (Sec. 3.1, nearest neighbour on a grid of spacing
 *     du wavelengths): k = llround(((x - x_c) f) / (c0 du)) + N/2 per axis,
 *     x_c the centroid of the layout.
 *   - geometric-delay correction (Sec. 2.2, the delay-correction block ahead
 *     of gridding): with delays != NULL ([T][A] seconds, and the channel
 *     frequencies f_c), e~_ap(t) = g_ap exp(+2 pi i f_c tau_a(t)) e_ap(t);
 *     tau_a(t) > 0 means the wavefront reaches antenna a later than the phase
 *     centre.  The factor has unit modulus and is shared by both
 *     polarisations, so the autocorrelation term does not change.
 *   - per-antenna kernels (Eq. 3 writes W_a; Sec. 3.1 A-projection): with
 *     kernels_per_antenna != 0 the kernel array is [A][K][K] and antenna a
 *     grids through W_a; the auto term becomes sum_a A_a,pq |W^_a(l)|^2 and
 *     the FX route grids pair (a, b) with B_ab(rho) = sum_d W_a(d) W_b^*(d - rho).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define ORACLE_C0 299792458.0
#define ORACLE_MEAN 1u
#define ORACLE_NO_AUTOSUB 2u

/* ------------------------------------------------------------ ci4 (a1) */

void oracle_ci4_unpack(uint8_t b, int *re, int *im)
{
    int hi = (b >> 4) & 0xF;
    int lo = b & 0xF;
    *re = hi >= 8 ? hi - 16 : hi;
    *im = lo >= 8 ? lo - 16 : lo;
}

static inline cplx ci4_value(uint8_t b)
{
    int re, im;
    oracle_ci4_unpack(b, &re, &im);
    return (double)re + I * (double)im;
}

/* ------------------------------------------------------------ cell map */

int oracle_cell_map(const double *ant_xy, int A, const double *freq_hz, int C,
                    const int *grid_n, double du, int *cells /* [C][A][2] */)
{
    if (A <= 0 || C <= 0 || du <= 0) return -1;
    double sx = 0, sy = 0;
    for (int a = 0; a < A; a++) { sx += ant_xy[2 * a]; sy += ant_xy[2 * a + 1]; }
    double cx = sx / A, cy = sy / A;
    for (int c = 0; c < C; c++) {
        int half = grid_n[c] / 2;
        for (int a = 0; a < A; a++) {
            double x = ant_xy[2 * a] - cx, y = ant_xy[2 * a + 1] - cy;
            cells[(c * A + a) * 2 + 0] = (int)llround((x * freq_hz[c]) / (ORACLE_C0 * du)) + half;
            cells[(c * A + a) * 2 + 1] = (int)llround((y * freq_hz[c]) / (ORACLE_C0 * du)) + half;
        }
    }
    return 0;
}

/* ------------------------------------------------------------ own FFT */

/* Unnormalised DFT X[k] = sum_n x[n] w^{n k}, w = exp(sign 2 pi i / n), computed
 * recursively by splitting on the smallest prime factor (decimation in time).
 * tw[e] = exp(sign 2 pi i e / ntop) for the top-level length; a sub-length n
 * that divides ntop uses tw[e * (ntop / n)]. */
typedef struct { int ntop; const cplx *tw; } fft_ctx;

static int smallest_factor(int n)
{
    for (int r = 2; r * r <= n; r++)
        if (n % r == 0) return r;
    return n;
}

static void fft_rec(const fft_ctx *ctx, const cplx *x, int n, int stride, cplx *out, cplx *scratch)
{
    if (n == 1) { out[0] = x[0]; return; }
    int r = smallest_factor(n);
    int m = n / r;
    int step = ctx->ntop / n;
    /* transform the r decimated subsequences x[j + r q] into out[j m .. j m + m) */
    for (int j = 0; j < r; j++)
        fft_rec(ctx, x + (size_t)j * stride, m, stride * r, out + (size_t)j * m, scratch + n);
    /* combine: X[k + s m] = sum_j w_n^{j (k + s m)} Y_j[k] */
    for (int k = 0; k < m; k++) {
        for (int s = 0; s < r; s++) {
            int kk = k + s * m;
            cplx acc = 0;
            for (int j = 0; j < r; j++) {
                long e = ((long)j * kk) % n;
                acc += out[(size_t)j * m + k] * ctx->tw[e * step];
            }
            scratch[kk] = acc;
        }
    }
    memcpy(out, scratch, sizeof(cplx) * (size_t)n);
}

static cplx *make_twiddles(int n, int sign)
{
    cplx *tw = malloc(sizeof(cplx) * (size_t)n);
    for (int k = 0; k < n; k++) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        tw[k] = cos(ang) + I * sin(ang);
    }
    return tw;
}

/* in-place 1-D transform of n = ctx->ntop complex values with the given stride */
static void fft_strided(const fft_ctx *ctx, cplx *x, int stride, cplx *buf /* >= 4n */)
{
    int n = ctx->ntop;
    cplx *in = buf, *out = buf + n, *scr = buf + 2 * n;
    for (int i = 0; i < n; i++) in[i] = x[(size_t)i * stride];
    fft_rec(ctx, in, n, 1, out, scr);
    for (int i = 0; i < n; i++) x[(size_t)i * stride] = out[i];
}

/* exported for the FFT pin: interleaved complex, in place, sign = +1 or -1 */
void oracle_fft1d(double *x_interleaved, int n, int sign)
{
    cplx *tw = make_twiddles(n, sign);
    fft_ctx ctx = {n, tw};
    cplx *buf = malloc(sizeof(cplx) * (size_t)(6 * n + 64));
    fft_strided(&ctx, (cplx *)x_interleaved, 1, buf);
    free(buf);
    free(tw);
}

/* 2-D inverse (+i) unnormalised transform of an N x N row-major grid [ky][kx] */
static void ifft2(const fft_ctx *ctx, cplx *g, cplx *buf)
{
    int N = ctx->ntop;
    for (int y = 0; y < N; y++) fft_strided(ctx, g + (size_t)y * N, 1, buf);
    for (int x = 0; x < N; x++) fft_strided(ctx, g + x, N, buf);
}

void oracle_ifft2(double *g_interleaved, int N)
{
    cplx *tw = make_twiddles(N, +1);
    fft_ctx ctx = {N, tw};
    cplx *buf = malloc(sizeof(cplx) * (size_t)(6 * N + 64));
    ifft2(&ctx, (cplx *)g_interleaved, buf);
    free(buf);
    free(tw);
}

/* ------------------------------------------------------------ kernel power */

/* |W^(l)|^2 with W^(l) = sum_d W(d) exp(+2 pi i d.l / N), by direct sum, on the
 * fft-shifted pixel layout out[i][j], l = (j - N/2, i - N/2). */
void oracle_kernel_power(const double *W_il, int K, int N, double *out)
{
    const cplx *W = (const cplx *)W_il;
    int h = (K - 1) / 2;
    for (int i = 0; i < N; i++) {
        int ly = i - N / 2;
        for (int j = 0; j < N; j++) {
            int lx = j - N / 2;
            cplx s = 0;
            for (int dy = -h; dy <= h; dy++)
                for (int dx = -h; dx <= h; dx++) {
                    double ang = 2.0 * M_PI * (double)(dx * lx + dy * ly) / (double)N;
                    s += W[(dy + h) * K + (dx + h)] * (cos(ang) + I * sin(ang));
                }
            out[(size_t)i * N + j] = creal(s) * creal(s) + cimag(s) * cimag(s);
        }
    }
}

/* ------------------------------------------------------------ shared checks */

static int check_args(int T, int C, int A, int P, int K, const int *grid_n)
{
    if (T < 0 || C <= 0 || A <= 0 || (P != 1 && P != 2) || K <= 0 || (K % 2) == 0) return -1;
    for (int c = 0; c < C; c++)
        if (grid_n[c] < 2 || (grid_n[c] % 2) != 0) return -1;
    return 0;
}

static inline int wrap(int k, int N) { int r = k % N; return r < 0 ? r + N : r; }

static size_t channel_offset(const int *grid_n, int c, int NP)
{
    size_t off = 0;
    for (int i = 0; i < c; i++) off += (size_t)NP * grid_n[i] * grid_n[i];
    return off;
}

/* A_pq(c) = sum_a g_ap g_aq^* sum_t e_ap e_aq^*, the inner sum exact in int64 */
static void auto_power(const uint8_t *v, const cplx *g, int T, int C, int A, int P, int c,
                       cplx *Apq /* [P][P] */)
{
    for (int p = 0; p < P; p++)
        for (int q = 0; q < P; q++) Apq[p * P + q] = 0;
    for (int a = 0; a < A; a++) {
        long long sre[4] = {0, 0, 0, 0}, sim[4] = {0, 0, 0, 0};
        for (int t = 0; t < T; t++) {
            for (int p = 0; p < P; p++)
                for (int q = 0; q < P; q++) {
                    int rp, ip, rq, iq;
                    oracle_ci4_unpack(v[(((size_t)t * C + c) * A + a) * P + p], &rp, &ip);
                    oracle_ci4_unpack(v[(((size_t)t * C + c) * A + a) * P + q], &rq, &iq);
                    sre[p * P + q] += (long long)rp * rq + (long long)ip * iq;
                    sim[p * P + q] += (long long)ip * rq - (long long)rp * iq;
                }
        }
        for (int p = 0; p < P; p++)
            for (int q = 0; q < P; q++) {
                cplx gp = g ? g[((size_t)c * A + a) * P + p] : 1.0;
                cplx gq = g ? g[((size_t)c * A + a) * P + q] : 1.0;
                Apq[p * P + q] += gp * conj(gq) * ((double)sre[p * P + q] + I * (double)sim[p * P + q]);
            }
    }
}

/* kernel tap of antenna a at offset (dy, dx) */
static inline cplx wtap(const cplx *W, int K, int per_antenna, int a, int dy, int dx)
{
    int h = (K - 1) / 2;
    return W[((size_t)(per_antenna ? a : 0) * K + (dy + h)) * K + (dx + h)];
}

/* per-antenna auto sums A_a,pq = g_ap g_aq^* sum_t e_ap e_aq^* (inner sum exact in int64) */
static void auto_power_antenna(const uint8_t *v, const cplx *g, int T, int C, int A, int P, int c, int a,
                               cplx *Apq /* [P][P] */)
{
    for (int p = 0; p < P; p++)
        for (int q = 0; q < P; q++) {
            long long sre = 0, sim = 0;
            for (int t = 0; t < T; t++) {
                int rp, ip, rq, iq;
                oracle_ci4_unpack(v[(((size_t)t * C + c) * A + a) * P + p], &rp, &ip);
                oracle_ci4_unpack(v[(((size_t)t * C + c) * A + a) * P + q], &rq, &iq);
                sre += (long long)rp * rq + (long long)ip * iq;
                sim += (long long)ip * rq - (long long)rp * iq;
            }
            cplx gp = g ? g[((size_t)c * A + a) * P + p] : 1.0;
            cplx gq = g ? g[((size_t)c * A + a) * P + q] : 1.0;
            Apq[p * P + q] = gp * conj(gq) * ((double)sre + I * (double)sim);
        }
}

/* auto image sum_a A_a,pq |W^_a(l)|^2 on the shifted layout, per product */
static void auto_image(const uint8_t *v, const cplx *g, int T, int C, int A, int P, int c,
                       const double *W_il, int K, int per_antenna, int N, int NP, cplx *out /* [NP][N][N] */)
{
    static const int PQP[4] = {0, 1, 0, 1}, PQQ[4] = {0, 1, 1, 0};
    size_t NN = (size_t)N * N;
    double *Wp = malloc(sizeof(double) * NN);
    for (size_t i = 0; i < (size_t)NP * NN; i++) out[i] = 0;
    for (int a = 0; a < (per_antenna ? A : 1); a++) {
        cplx Apq[4];
        if (per_antenna) auto_power_antenna(v, g, T, C, A, P, c, a, Apq);
        else auto_power(v, g, T, C, A, P, c, Apq);
        oracle_kernel_power(W_il + (size_t)(per_antenna ? a : 0) * K * K * 2, K, N, Wp);
        for (int pq = 0; pq < NP; pq++)
            for (size_t i = 0; i < NN; i++) out[(size_t)pq * NN + i] += Apq[PQP[pq] * P + PQQ[pq]] * Wp[i];
    }
    free(Wp);
}

/* exp(+2 pi i f tau), the delay correction of one antenna, straight from the definition */
static inline cplx delay_factor(const double *freq_hz, const double *delays, int A, int t, int c, int a)
{
    double ang = 2.0 * M_PI * freq_hz[c] * delays[(size_t)t * A + a];
    return cos(ang) + I * sin(ang);
}

/* product index -> (p, q): XX, YY, XY, YX */
static const int PQ_P[4] = {0, 1, 0, 1};
static const int PQ_Q[4] = {0, 1, 1, 0};

/* ------------------------------------------------------------ O1: EPIC direct */

int oracle_epic_direct(const uint8_t *v, const double *gains_il, int T, int C, int A, int P,
                       const int *cells, const int *grid_n, const double *W_il, int K,
                       int per_antenna, const double *freq_hz, const double *delays,
                       unsigned flags, double *out_il)
{
    if (check_args(T, C, A, P, K, grid_n)) return -1;
    if (delays && !freq_hz) return -1;
    const cplx *g = (const cplx *)gains_il;
    const cplx *W = (const cplx *)W_il;
    cplx *out = (cplx *)out_il;
    int NP = P == 2 ? 4 : 1;
    int h = (K - 1) / 2;

#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; c++) {
        int N = grid_n[c];
        size_t NN = (size_t)N * N;
        cplx *G = calloc((size_t)P * NN, sizeof(cplx));
        cplx *S = calloc((size_t)NP * NN, sizeof(cplx));
        cplx *buf = malloc(sizeof(cplx) * (size_t)(6 * N + 64));
        double *Wp = malloc(sizeof(double) * NN);
        cplx *tw = make_twiddles(N, +1);
        fft_ctx ctx = {N, tw};
        for (int t = 0; t < T; t++) {
            /* a1-a3: unpack, calibrate, grid (circular) */
            memset(G, 0, sizeof(cplx) * (size_t)P * NN);
            for (int p = 0; p < P; p++) {
                cplx *Gp = G + (size_t)p * NN;
                for (int a = 0; a < A; a++) {
                    cplx e = ci4_value(v[(((size_t)t * C + c) * A + a) * P + p]);
                    if (g) e *= g[((size_t)c * A + a) * P + p];
                    if (delays) e *= delay_factor(freq_hz, delays, A, t, c, a);
                    int kx = cells[((size_t)c * A + a) * 2 + 0];
                    int ky = cells[((size_t)c * A + a) * 2 + 1];
                    for (int dy = -h; dy <= h; dy++)
                        for (int dx = -h; dx <= h; dx++)
                            Gp[(size_t)wrap(ky + dy, N) * N + wrap(kx + dx, N)] += wtap(W, K, per_antenna, a, dy, dx) * e;
                }
                /* a4: inverse transform to the sky */
                ifft2(&ctx, Gp, buf);
            }
            /* a5-a6: polarisation products, summed over time */
            for (int pq = 0; pq < NP; pq++) {
                const cplx *Fp = G + (size_t)PQ_P[pq] * NN;
                const cplx *Fq = G + (size_t)PQ_Q[pq] * NN;
                cplx *Sp = S + (size_t)pq * NN;
                for (size_t i = 0; i < NN; i++) Sp[i] += Fp[i] * conj(Fq[i]);
            }
        }
        /* a7-a8: autocorrelation term and shifted output */
        cplx *autos = malloc(sizeof(cplx) * (size_t)NP * NN);
        auto_image(v, g, T, C, A, P, c, W_il, K, per_antenna, N, NP, autos);
        cplx *oc = out + channel_offset(grid_n, c, NP);
        double scale = ((flags & ORACLE_MEAN) && T > 0) ? 1.0 / T : 1.0;
        for (int pq = 0; pq < NP; pq++) {
            for (int i = 0; i < N; i++)
                for (int j = 0; j < N; j++) {
                    int fy = wrap(i - N / 2, N), fx = wrap(j - N / 2, N);
                    cplx val = S[(size_t)pq * NN + (size_t)fy * N + fx];
                    if (!(flags & ORACLE_NO_AUTOSUB)) val -= autos[(size_t)pq * NN + (size_t)i * N + j];
                    oc[(size_t)pq * NN + (size_t)i * N + j] = val * scale;
                }
        }
        free(autos);
        free(G); free(S); free(buf); free(Wp); free(tw);
    }
    return 0;
}

/* ------------------------------------------------------------ O1 E-field images */

/* The electric-field images themselves (the abstract and Sec. 1: EPIC makes
 * "electric field or intensity images"): O1's steps a1-a4 only -- calibrate,
 * grid, inverse transform -- written per sample, channel and polarisation on
 * the fft-shifted layout, with no products, no time sum and no autocorrelation
 * term.  out: complex [T][sum_c P N_c^2], per sample the channels packed in
 * order, each [P][N_c][N_c]. */
int oracle_epic_efield(const uint8_t *v, const double *gains_il, int T, int C, int A, int P,
                       const int *cells, const int *grid_n, const double *W_il, int K,
                       int per_antenna, const double *freq_hz, const double *delays, double *out_il)
{
    if (check_args(T, C, A, P, K, grid_n)) return -1;
    if (delays && !freq_hz) return -1;
    const cplx *g = (const cplx *)gains_il;
    const cplx *W = (const cplx *)W_il;
    cplx *out = (cplx *)out_il;
    int h = (K - 1) / 2;
    size_t per_sample = channel_offset(grid_n, C, P);

#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; c++) {
        int N = grid_n[c];
        size_t NN = (size_t)N * N;
        cplx *G = malloc(sizeof(cplx) * NN);
        cplx *buf = malloc(sizeof(cplx) * (size_t)(6 * N + 64));
        cplx *tw = make_twiddles(N, +1);
        fft_ctx ctx = {N, tw};
        for (int t = 0; t < T; t++) {
            cplx *ot = out + (size_t)t * per_sample + channel_offset(grid_n, c, P);
            for (int p = 0; p < P; p++) {
                memset(G, 0, sizeof(cplx) * NN);
                for (int a = 0; a < A; a++) {
                    cplx e = ci4_value(v[(((size_t)t * C + c) * A + a) * P + p]);
                    if (g) e *= g[((size_t)c * A + a) * P + p];
                    if (delays) e *= delay_factor(freq_hz, delays, A, t, c, a);
                    int kx = cells[((size_t)c * A + a) * 2 + 0];
                    int ky = cells[((size_t)c * A + a) * 2 + 1];
                    for (int dy = -h; dy <= h; dy++)
                        for (int dx = -h; dx <= h; dx++)
                            G[(size_t)wrap(ky + dy, N) * N + wrap(kx + dx, N)] += wtap(W, K, per_antenna, a, dy, dx) * e;
                }
                ifft2(&ctx, G, buf);
                for (int i = 0; i < N; i++)
                    for (int j = 0; j < N; j++)
                        ot[(size_t)p * NN + (size_t)i * N + j] = G[(size_t)wrap(i - N / 2, N) * N + wrap(j - N / 2, N)];
            }
        }
        free(G); free(buf); free(tw);
    }
    return 0;
}

/* Per-(c, p) grid energy sum_t sum_k |G_p(k, t)|^2 with the O1 gridding, for
 * the Parseval pin. */
int oracle_grid_energy(const uint8_t *v, const double *gains_il, int T, int C, int A, int P,
                       const int *cells, const int *grid_n, const double *W_il, int K,
                       int per_antenna, double *energy /* [C][P] */)
{
    if (check_args(T, C, A, P, K, grid_n)) return -1;
    const cplx *g = (const cplx *)gains_il;
    const cplx *W = (const cplx *)W_il;
    int h = (K - 1) / 2;
    for (int c = 0; c < C; c++) {
        int N = grid_n[c];
        size_t NN = (size_t)N * N;
        cplx *G = malloc(sizeof(cplx) * NN);
        for (int p = 0; p < P; p++) {
            double e_sum = 0;
            for (int t = 0; t < T; t++) {
                memset(G, 0, sizeof(cplx) * NN);
                for (int a = 0; a < A; a++) {
                    cplx e = ci4_value(v[(((size_t)t * C + c) * A + a) * P + p]);
                    if (g) e *= g[((size_t)c * A + a) * P + p];
                    int kx = cells[((size_t)c * A + a) * 2 + 0];
                    int ky = cells[((size_t)c * A + a) * 2 + 1];
                    for (int dy = -h; dy <= h; dy++)
                        for (int dx = -h; dx <= h; dx++)
                            G[(size_t)wrap(ky + dy, N) * N + wrap(kx + dx, N)] += wtap(W, K, per_antenna, a, dy, dx) * e;
                }
                for (size_t i = 0; i < NN; i++) e_sum += creal(G[i]) * creal(G[i]) + cimag(G[i]) * cimag(G[i]);
            }
            energy[c * P + p] = e_sum;
        }
        free(G);
    }
    return 0;
}

/* ------------------------------------------------------------ O2: FX route */

int oracle_epic_fx(const uint8_t *v, const double *gains_il, int T, int C, int A, int P,
                   const int *cells, const int *grid_n, const double *W_il, int K,
                   int per_antenna, const double *freq_hz, const double *delays,
                   unsigned flags, double *out_il)
{
    if (check_args(T, C, A, P, K, grid_n)) return -1;
    if (delays && !freq_hz) return -1;
    const cplx *g = (const cplx *)gains_il;
    const cplx *W = (const cplx *)W_il;
    cplx *out = (cplx *)out_il;
    int NP = P == 2 ? 4 : 1;
    int h = (K - 1) / 2;
    int R = 2 * K - 1;              /* baseline kernel support, rho in [-(K-1), K-1]^2 */

    /* baseline kernel B_ab(rho) = sum_d W_a(d) W_b^*(d - rho); one kernel for all pairs unless per antenna */
    int nk = per_antenna ? A : 1;
    cplx *B = calloc((size_t)nk * nk * R * R, sizeof(cplx));
    for (int ka = 0; ka < nk; ka++)
        for (int kb = 0; kb < nk; kb++)
            for (int ry = -(K - 1); ry <= K - 1; ry++)
                for (int rx = -(K - 1); rx <= K - 1; rx++) {
                    cplx s = 0;
                    for (int dy = -h; dy <= h; dy++)
                        for (int dx = -h; dx <= h; dx++) {
                            int ey = dy - ry, ex = dx - rx;
                            if (ey < -h || ey > h || ex < -h || ex > h) continue;
                            s += wtap(W, K, 1, ka, dy, dx) * conj(wtap(W, K, 1, kb, ey, ex));
                        }
                    B[(((size_t)ka * nk + kb) * R + (ry + K - 1)) * R + (rx + K - 1)] = s;
                }

#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < C; c++) {
        int N = grid_n[c];
        size_t NN = (size_t)N * N;
        /* Eq. 1: exact integer visibilities V[a][b][p][q] = sum_t e_ap e_bq^*; with
         * delay corrections the per-sample phases d_a(t) d_b(t)^* enter the sum, which
         * is then taken in complex FP64 (Vd) */
        long long *Vre = calloc((size_t)A * A * P * P, sizeof(long long));
        long long *Vim = calloc((size_t)A * A * P * P, sizeof(long long));
        cplx *Vd = delays ? calloc((size_t)A * A * P * P, sizeof(cplx)) : NULL;
        cplx *dph = delays ? malloc(sizeof(cplx) * (size_t)A) : NULL;
        int *er = malloc(sizeof(int) * (size_t)A * P), *ei = malloc(sizeof(int) * (size_t)A * P);
        for (int t = 0; t < T; t++) {
            for (int a = 0; a < A; a++)
                for (int p = 0; p < P; p++)
                    oracle_ci4_unpack(v[(((size_t)t * C + c) * A + a) * P + p], &er[a * P + p], &ei[a * P + p]);
            if (delays)
                for (int a = 0; a < A; a++) dph[a] = delay_factor(freq_hz, delays, A, t, c, a);
            for (int a = 0; a < A; a++)
                for (int b = 0; b < A; b++)
                    for (int p = 0; p < P; p++)
                        for (int q = 0; q < P; q++) {
                            size_t ix = (((size_t)a * A + b) * P + p) * P + q;
                            int ra = er[a * P + p], ia = ei[a * P + p];
                            int rb = er[b * P + q], ib = ei[b * P + q];
                            long long vr = (long long)ra * rb + (long long)ia * ib;
                            long long vi = (long long)ia * rb - (long long)ra * ib;
                            if (delays) Vd[ix] += dph[a] * conj(dph[b]) * ((double)vr + I * (double)vi);
                            else {
                                Vre[ix] += vr;
                                Vim[ix] += vi;
                            }
                        }
        }
        /* Eq. 2-3: grid calibrated cross visibilities with B at offset k_a - k_b */
        cplx *Vg = calloc((size_t)NP * NN, sizeof(cplx));
        for (int a = 0; a < A; a++)
            for (int b = 0; b < A; b++) {
                if (a == b) continue;     /* autocorrelations removed */
                int dx0 = cells[((size_t)c * A + a) * 2 + 0] - cells[((size_t)c * A + b) * 2 + 0];
                int dy0 = cells[((size_t)c * A + a) * 2 + 1] - cells[((size_t)c * A + b) * 2 + 1];
                for (int pq = 0; pq < NP; pq++) {
                    int p = PQ_P[pq], q = PQ_Q[pq];
                    size_t ix = (((size_t)a * A + b) * P + p) * P + q;
                    cplx Vab = delays ? Vd[ix] : (double)Vre[ix] + I * (double)Vim[ix];
                    cplx ga = g ? g[((size_t)c * A + a) * P + p] : 1.0;
                    cplx gb = g ? g[((size_t)c * A + b) * P + q] : 1.0;
                    cplx Vc = ga * conj(gb) * Vab;
                    cplx *Vp = Vg + (size_t)pq * NN;
                    const cplx *Bab = B + ((size_t)(per_antenna ? a : 0) * nk + (per_antenna ? b : 0)) * R * R;
                    for (int ry = -(K - 1); ry <= K - 1; ry++)
                        for (int rx = -(K - 1); rx <= K - 1; rx++)
                            Vp[(size_t)wrap(dy0 + ry, N) * N + wrap(dx0 + rx, N)] +=
                                Vc * Bab[(ry + K - 1) * R + (rx + K - 1)];
                }
            }
        /* inverse transform by direct separable DFT with an exact-index twiddle table */
        cplx *tw = malloc(sizeof(cplx) * (size_t)N);
        for (int k = 0; k < N; k++) {
            double ang = 2.0 * M_PI * (double)k / (double)N;
            tw[k] = cos(ang) + I * sin(ang);
        }
        cplx *tmp = malloc(sizeof(cplx) * NN);
        cplx *oc = out + channel_offset(grid_n, c, NP);
        double scale = ((flags & ORACLE_MEAN) && T > 0) ? 1.0 / T : 1.0;
        cplx *autos = NULL;
        if (flags & ORACLE_NO_AUTOSUB) {
            /* put the autos back (the direct form keeps them without subtraction) */
            autos = malloc(sizeof(cplx) * (size_t)NP * NN);
            auto_image(v, g, T, C, A, P, c, W_il, K, per_antenna, N, NP, autos);
        }
        for (int pq = 0; pq < NP; pq++) {
            const cplx *Vp = Vg + (size_t)pq * NN;
            /* along x: tmp[ky][lx] = sum_kx Vp[ky][kx] w^{kx lx} */
            for (int ky = 0; ky < N; ky++)
                for (int lx = 0; lx < N; lx++) {
                    cplx s = 0;
                    for (int kx = 0; kx < N; kx++) s += Vp[(size_t)ky * N + kx] * tw[((long)kx * lx) % N];
                    tmp[(size_t)ky * N + lx] = s;
                }
            /* along y, then write shifted */
            for (int i = 0; i < N; i++) {
                int ly = wrap(i - N / 2, N);
                for (int j = 0; j < N; j++) {
                    int lx = wrap(j - N / 2, N);
                    cplx s = 0;
                    for (int ky = 0; ky < N; ky++) s += tmp[(size_t)ky * N + lx] * tw[((long)ky * ly) % N];
                    if (autos) s += autos[(size_t)pq * NN + (size_t)i * N + j];
                    oc[(size_t)pq * NN + (size_t)i * N + j] = s * scale;
                }
            }
        }
        free(autos);
        free(Vre); free(Vim); free(Vd); free(dph); free(er); free(ei); free(Vg); free(tw); free(tmp);
    }
    free(B);
    return 0;
}

/* number of OpenMP threads the oracle will use (reported by the CPU baseline) */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
#else
int oracle_threads(void) { return 1; }
#endif
