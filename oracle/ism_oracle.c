/*
 * ism_oracle.c -- plain, slow, FP64 CPU oracle for the image-source method
 * (Diaz-Guerra, Miguel, Beltran: "gpuRIR: A Python Library for Room Impulse
 * Response Simulation with GPU Acceleration").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
 * call this file: it exists so that tests/, the smoke check and the CPU
 * baseline leg of bench.py can compare the CUDA library against the plain
 * definition of the method.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function follows one passage of the paper and evaluates it literally,
 * image by image and sample by sample, in double precision.  Where the paper is
 * silent or garbled the reading taken is stated beside the code:
 *   - eq. (2) prints ||p_r - p_s||; the text says the distance is to the image
 *     p_n, which is what is used.
 *   - the wall exponents of eq. (4) are not spelled out; they follow from the
 *     mirror geometry of eq. (1) (see image_exponents()).
 *   - eq. (8) prints exp(log10(T60/20)(t - t0)), which is not a 60 dB decay in
 *     T60; the envelope used is the Sabine one it is meant to express:
 *     power falls by 60 dB in T60 seconds.
 *   - the envelope amplitude A, fitted to the image-source part (Section 2.2), is the
 *     detrended power of the last 20 ms of the image-source part.
 *   - the noise is logistic with unit variance driven by Philox4x32-10.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math: the
 * FP32 noise transform must round every operation exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Section 2.1: the image grid.  ceil(-N/2) <= n < ceil(N/2) on every axis.   */
/* ------------------------------------------------------------------------- */
static int ceil_div2_neg(int N) { return -(N / 2); }          /* ceil(-N/2) for N >= 0 */
static int ceil_div2(int N) { return (N + 1) / 2; }            /* ceil(N/2)  for N >= 0 */

void oracle_grid_bounds(int N, int* n_lo, int* n_hi_excl)
{
    *n_lo = ceil_div2_neg(N);
    *n_hi_excl = ceil_div2(N);
}

/* Eq. (1): coordinate of image n along one axis of length L for a source at xs. */
double oracle_image_coord(int n, double L, double xs)
{
    if (n % 2 == 0) return (double)n * L + xs;
    return (double)(n + 1) * L - xs;
}

/* Eq. (4), "product of the reflection coefficients of each wall crossed":
 * the path from image n to the receiver crosses the planes x = kL for every k
 * strictly between the image cell and the room.  Planes with k even are images
 * of the wall at x = 0 (beta_x0), planes with k odd images of the wall at x = L
 * (beta_x1).  Counting them gives, for n even, |n|/2 crossings of each wall;
 * for n odd, |n-1|/2 of the near wall and |n+1|/2 of the far wall.  n = -1 is
 * the mirror across x = 0 (one hit of beta_x0), n = +1 across x = L. */
void oracle_image_exponents(int n, int* e0, int* e1)
{
    if (n % 2 == 0) {
        *e0 = abs(n) / 2;
        *e1 = abs(n) / 2;
    } else {
        *e0 = abs(n - 1) / 2;
        *e1 = abs(n + 1) / 2;
    }
}

static double ipow(double b, int e)
{
    double r = 1.0;                 /* 0^0 = 1: the direct path keeps weight 1 */
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* sin(pi x) with the argument reduced exactly, so that it is exactly zero at
 * integers (eq. (6) with f_c = f_s/2 has its zeros on the sampling grid). */
static double sinpi_exact(double x)
{
    double k = nearbyint(x);
    double r = x - k;               /* exact for |x| < 2^52 */
    double s = sin(ORACLE_PI * r);
    long long ki = (long long)k;
    return (ki & 1LL) ? -s : s;
}

/* Eq. (6): Peterson's windowed sinc, with the cut-off at Nyquist (f_c = f_s/2).
 * x is the time offset t - tau expressed in samples (x = f_s (t - tau)); Tw is
 * the window length in seconds.  Returns 0 outside |t| < Tw/2. */
double oracle_delta_prime(double x, double fs, double Tw)
{
    double t = x / fs;
    if (!(fabs(t) < 0.5 * Tw)) return 0.0;
    double w = 0.5 * (1.0 + cos(2.0 * ORACLE_PI * t / Tw));
    /* sinc(2 pi f_c t) with f_c = f_s/2: argument pi x */
    double sc = (x == 0.0) ? 1.0 : sinpi_exact(x) / (ORACLE_PI * x);
    return w * sc;
}

/* Enumerate the images of one source-receiver pair (eq. (1)-(4)).
 * For each image writes n[3], position[3], exponents e[6] (x0,x1,y0,y1,z0,z1),
 * distance d, delay tau and amplitude A.  Returns the number of images, which
 * is N[0]*N[1]*N[2] by construction.  Any output pointer may be NULL. */
long oracle_enumerate_images(const double L[3], const double beta[6], double c,
                             const double ps[3], const double pr[3], const int N[3],
                             int* n_out, double* pos_out, int* e_out,
                             double* d_out, double* tau_out, double* amp_out)
{
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) oracle_grid_bounds(N[a], &lo[a], &hi[a]);
    long idx = 0;
    for (int nx = lo[0]; nx < hi[0]; ++nx)
        for (int ny = lo[1]; ny < hi[1]; ++ny)
            for (int nz = lo[2]; nz < hi[2]; ++nz) {
                int n[3] = {nx, ny, nz};
                double p[3];
                int e[6];
                double bn = 1.0, d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    p[a] = oracle_image_coord(n[a], L[a], ps[a]);                 /* eq. (1) */
                    oracle_image_exponents(n[a], &e[2 * a], &e[2 * a + 1]);
                    bn *= ipow(beta[2 * a], e[2 * a]) * ipow(beta[2 * a + 1], e[2 * a + 1]);
                    double dd = pr[a] - p[a];
                    d2 += dd * dd;
                }
                double d = sqrt(d2);                                             /* eq. (2) */
                double tau = d / c;                                              /* eq. (3) */
                double A = bn / (4.0 * ORACLE_PI * d);                           /* eq. (4) */
                if (n_out) { n_out[3 * idx] = nx; n_out[3 * idx + 1] = ny; n_out[3 * idx + 2] = nz; }
                if (pos_out) for (int a = 0; a < 3; ++a) pos_out[3 * idx + a] = p[a];
                if (e_out) for (int w = 0; w < 6; ++w) e_out[6 * idx + w] = e[w];
                if (d_out) d_out[idx] = d;
                if (tau_out) tau_out[idx] = tau;
                if (amp_out) amp_out[idx] = A;
                ++idx;
            }
    return idx;
}

/* Receiver polar pattern (Section 4 names polar patterns and orientation of
 * the receivers without a formula).  Reading: the first-order family
 * g(theta) = alpha + (1 - alpha) cos(theta), theta the angle between the
 * receiver's orientation o and the direction from the receiver to the image
 * source; alpha = 1 omnidirectional, 3/4 subcardioid, 1/2 cardioid, 1/4
 * hypercardioid, 0 bidirectional.  The gain multiplies the image's amplitude
 * A of eq. (4).  o need not be of unit length. */
double oracle_pattern_gain(double alpha, const double o[3], const double pr[3], const double p_img[3])
{
    double dot = 0.0, oo = 0.0, dd = 0.0;
    for (int a = 0; a < 3; ++a) {
        double v = p_img[a] - pr[a];
        dot += o[a] * v;
        oo += o[a] * o[a];
        dd += v * v;
    }
    return alpha + (1.0 - alpha) * dot / (sqrt(oo) * sqrt(dd));
}

/* Eq. (5) with eq. (6): h[k] = sum_n g_n A_n delta'(k/f_s - tau_n) for the
 * samples 0 <= k < n_ism of one pair (g_n = 1 without a polar pattern, i.e.
 * orient == NULL).  Image-major, every image of the grid, every sample inside
 * its window; no binning, no tiling. */
static void rir_one(const double L[3], const double beta[6], double c, double fs, double Tw,
                    const double ps[3], const double pr[3], const int N[3], int n_ism, double* h,
                    const double* orient, double alpha)
{
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) oracle_grid_bounds(N[a], &lo[a], &hi[a]);
    for (int k = 0; k < n_ism; ++k) h[k] = 0.0;
    for (int nx = lo[0]; nx < hi[0]; ++nx)
        for (int ny = lo[1]; ny < hi[1]; ++ny)
            for (int nz = lo[2]; nz < hi[2]; ++nz) {
                int n[3] = {nx, ny, nz};
                double bn = 1.0, d2 = 0.0, p[3];
                for (int a = 0; a < 3; ++a) {
                    p[a] = oracle_image_coord(n[a], L[a], ps[a]);
                    int e0, e1;
                    oracle_image_exponents(n[a], &e0, &e1);
                    bn *= ipow(beta[2 * a], e0) * ipow(beta[2 * a + 1], e1);
                    double dd = pr[a] - p[a];
                    d2 += dd * dd;
                }
                double d = sqrt(d2);
                double tau = d / c;
                double A = bn / (4.0 * ORACLE_PI * d);
                if (orient) A *= oracle_pattern_gain(alpha, orient, pr, p);
                double s = fs * d / c;                       /* tau in samples */
                /* samples with |k/f_s - tau| < Tw/2 */
                double half = 0.5 * Tw * fs;
                long k0 = (long)floor(s - half);
                long k1 = (long)ceil(s + half);
                if (k0 < 0) k0 = 0;
                if (k1 > n_ism - 1) k1 = n_ism - 1;
                for (long k = k0; k <= k1; ++k) {
                    double x = (double)k - s;
                    h[k] += A * oracle_delta_prime(x, fs, Tw);
                }
                (void)tau;
            }
}

/* Batch driver: n_pairs independent pairs given by their positions
 * (ps[i], pr[i]); out is [n_pairs][n_ism].  OpenMP over pairs. */
void oracle_rir_list(const double L[3], const double beta[6], double c, double fs, double Tw,
                     const double* ps, const double* pr, int n_pairs, const int N[3], int n_ism,
                     double* out, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < n_pairs; ++i)
        rir_one(L, beta, c, fs, Tw, ps + 3 * i, pr + 3 * i, N, n_ism, out + (long)i * n_ism, NULL, 1.0);
    (void)n_threads;
}

/* As oracle_rir_list, with a receiver polar pattern: orient is [n_pairs][3],
 * the orientation of each pair's receiver. */
void oracle_rir_list_pattern(const double L[3], const double beta[6], double c, double fs, double Tw,
                             const double* ps, const double* pr, const double* orient, double alpha,
                             int n_pairs, const int N[3], int n_ism, double* out, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < n_pairs; ++i)
        rir_one(L, beta, c, fs, Tw, ps + 3 * i, pr + 3 * i, N, n_ism, out + (long)i * n_ism, orient + 3 * i, alpha);
    (void)n_threads;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Eq. (7): Sabine.  T60 = 0.161 V / sum_i S_i alpha_i, alpha_i = 1 - beta_i^2 */
/* ------------------------------------------------------------------------- */
static void wall_areas(const double L[3], double S[6])
{
    S[0] = S[1] = L[1] * L[2];
    S[2] = S[3] = L[0] * L[2];
    S[4] = S[5] = L[0] * L[1];
}

double oracle_t60_sabine(const double L[3], const double beta[6])
{
    double S[6], den = 0.0;
    wall_areas(L, S);
    for (int i = 0; i < 6; ++i) den += S[i] * (1.0 - beta[i] * beta[i]);
    return 0.161 * L[0] * L[1] * L[2] / den;
}

/* Inverse of eq. (7) for the library helper of Section 4: the reflection
 * coefficients that give a wanted T60.  alpha_i = w_i alpha_0 with one common
 * alpha_0; beta_i = +sqrt(1 - alpha_i) (or the negative root, Section 2.2).
 * Returns 0 on success, 1 if some alpha_i >= 1 or the weights are degenerate. */
int oracle_beta_sabine(const double L[3], double T60, const double w[6], int negative,
                       double beta_out[6])
{
    double S[6], sw = 0.0;
    wall_areas(L, S);
    for (int i = 0; i < 6; ++i) sw += S[i] * w[i];
    if (!(sw > 0.0) || !(T60 > 0.0)) return 1;
    double a0 = 0.161 * L[0] * L[1] * L[2] / (T60 * sw);
    for (int i = 0; i < 6; ++i) {
        double a = w[i] * a0;
        if (a >= 1.0 || a < 0.0) return 1;
        double b = sqrt(1.0 - a);
        beta_out[i] = negative ? -b : b;
    }
    return 0;
}

/* Section 4 helper: time at which the Sabine decay reaches att_dB. */
double oracle_att2t_sabine(double att_dB, double T60) { return att_dB / 60.0 * T60; }

/* Section 4 helper: images per axis so that no reflection arriving before T is
 * lost.  An image of index n is at least (|n|-1) L from the receiver (eq. (1)
 * with both points inside the room), so every image within c (T + Tw/2) has
 * |n| <= M = ceil(c (T + Tw/2) / L) + 1; the grid n in [-M, M] is N = 2M + 1. */
void oracle_nb_img_from_t(double T, const double L[3], double c, double Tw, int N_out[3])
{
    double R = c * (T + 0.5 * Tw);
    for (int a = 0; a < 3; ++a) {
        int M = (int)ceil(R / L[a]) + 1;
        N_out[a] = 2 * M + 1;
    }
}

/* ------------------------------------------------------------------------- */
/* Section 2.2 "Diffuse reverberation" and Section 3.3: logistic noise with   */
/* an exponential power envelope.  The random numbers are Philox4x32-10       */
/* (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies */
/* on a 4-word counter, keyed by 2 words bumped by the Weyl constants.        */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 32-bit word that drives sample k of RIR `rir`: counter (k/4, rir, 0, 0),
 * key (seed low, seed high), word k mod 4. */
uint32_t oracle_noise_word(uint64_t seed, uint32_t rir, uint32_t k)
{
    uint32_t ctr[4] = {k >> 2, rir, 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox4x32_10(ctr, key, o);
    return o[k & 3u];
}

/* Uniform in (0,1), exactly representable in FP32: (2m+1) 2^-24, m = x >> 9. */
float oracle_uniform_f32(uint32_t x)
{
    float m = (float)(x >> 9);
    return (m + 0.5f) * 0x1p-23f;
}

/* Natural logarithm in FP32 from correctly rounded operations only, in a fixed
 * order (the written specification both the oracle and the kernel follow):
 *   x = m 2^e with m in (sqrt(1/2), sqrt(2)];
 *   ln m = 2 atanh(t), t = (m-1)/(m+1), atanh(t) = t + t^3/3 + t^5/5 + ... ;
 *   ln x = e ln2 + ln m, ln2 split in a short head and a tail.
 * Valid for positive normal x (the noise transform only feeds it u/(1-u)
 * with u in [2^-24, 1-2^-24]). */
float oracle_ln_f32(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    uint32_t mb = (bits & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mb, 4);
    if (m > 1.41421353816986083984375f) {          /* largest float below sqrt(2) */
        m = m * 0.5f;
        e = e + 1;
    }
    float t = (m - 1.0f) / (m + 1.0f);
    float t2 = t * t;
    float p = fmaf(t2, 2.0f / 11.0f, 2.0f / 9.0f);
    p = fmaf(t2, p, 2.0f / 7.0f);
    p = fmaf(t2, p, 2.0f / 5.0f);
    p = fmaf(t2, p, 2.0f / 3.0f);
    float t3 = t * t2;
    float lnm = fmaf(t3, p, 2.0f * t);
    float ef = (float)e;
    const float ln2_hi = 0.693145751953125f;            /* 12 low mantissa bits zero */
    const float ln2_lo = 1.428606765330187e-06f;         /* FP32(ln2 - ln2_hi) */
    return fmaf(ef, ln2_hi, fmaf(ef, ln2_lo, lnm));
}

void oracle_ln_f32_array(const float* x, float* y, long n)
{
    for (long i = 0; i < n; ++i) y[i] = oracle_ln_f32(x[i]);
}

/* Unit-variance logistic variate from u: z = (sqrt(3)/pi) ln(u / (1-u)). */
float oracle_logistic_f32(float u)
{
    const float k = 0.5513288974761963f;                /* sqrt(3)/pi rounded to FP32 */
    float r = u / (1.0f - u);
    return k * oracle_ln_f32(r);
}

/* z for samples k0 .. k0+n-1 of RIR `rir` (bit-exact reference for the kernel). */
void oracle_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z)
{
    for (int i = 0; i < n; ++i)
        z[i] = oracle_logistic_f32(oracle_uniform_f32(oracle_noise_word(seed, rir, k0 + (uint32_t)i)));
}

/* Envelope amplitude at t0 = n_ism/f_s, fitted to the image-source part
 * (Section 2.2): mean of h[k]^2 10^(-6 (t0 - t_k)/T60) over the last
 * W = ceil(0.02 f_s) image-source samples, i.e. the ISM power brought forward
 * to t0 along the 60 dB/T60 decay of eq. (8) (earlier samples carry more
 * power, so they are scaled down to the level they would have at t0). */
double oracle_envelope_amp(const double* h, int n_ism, double fs, double T60)
{
    int W = (int)ceil(0.02 * fs);
    if (W > n_ism) W = n_ism;
    if (W <= 0) return 0.0;
    double acc = 0.0;
    for (int k = n_ism - W; k < n_ism; ++k) {
        double dt = (double)(n_ism - k) / fs;
        acc += h[k] * h[k] * pow(10.0, -6.0 * dt / T60);
    }
    return acc / (double)W;
}

/* Eq. (8), read as a 60 dB decay over T60: sqrt(P(t)) for t = k/f_s >= t0. */
double oracle_envelope_sqrt(double A, int k, int n_ism, double fs, double T60)
{
    double dt = (double)(k - n_ism) / fs;
    return sqrt(A * pow(10.0, -6.0 * dt / T60));
}

/* The diffuse tail of one RIR: h[k] = z_k sqrt(P(t_k)) for n_ism <= k < n_s,
 * with A supplied by the caller (so that it can be compared given the same A). */
void oracle_tail(uint64_t seed, uint32_t rir, double A, int n_ism, int n_s, double fs, double T60,
                 double* h)
{
    for (int k = n_ism; k < n_s; ++k) {
        float z = oracle_logistic_f32(oracle_uniform_f32(oracle_noise_word(seed, rir, (uint32_t)k)));
        h[k] = (double)z * oracle_envelope_sqrt(A, k, n_ism, fs, T60);
    }
}

/* ------------------------------------------------------------------------- */
/* Energy-decay envelope after Lehmann and Johansson, which Section 2.2 cites */
/* as the more faithful (and costlier) alternative to the Sabine exponential. */
/* The paper gives no formula; the reading taken (parity pinned by closed     */
/* forms and by the energy decay of the images themselves, see the tests):    */
/* the images of a shoebox room fill space with density 1/V; an image at     */
/* distance r in direction u is reached through about r |u_a| / L_a          */
/* reflections on the two walls of axis a, half on each, so it carries the   */
/* energy prod_a rho_a^(r |u_a| / L_a) / (4 pi r)^2 with rho_a =             */
/* |beta_a0 beta_a1| (eq. (4) squared).  The r^2 growth of a shell cancels    */
/* the spreading, and the energy arriving at time t = r / c is proportional   */
/* to the average over directions                                             */
/*   E(t) = (1 / 4 pi) oint prod_a rho_a^(c t |u_a| / L_a) dOmega.            */
/* |u_a| is the same in all eight octants, so the average is taken over one:  */
/* theta, phi in [0, pi/2], u = (sin t cos p, sin t sin p, cos t), dOmega =   */
/* sin t dt dp, weight 8 / (4 pi) = 2 / pi, with the product quadrature rule  */
/* whose n nodes x[i] and weights w[i] on [-1, 1] the caller supplies.        */
/* ------------------------------------------------------------------------- */
double oracle_lj_energy(const double L[3], const double beta[6], double c, double t, const double* x,
                        const double* w, int n)
{
    double rho[3];
    for (int a = 0; a < 3; ++a) rho[a] = fabs(beta[2 * a] * beta[2 * a + 1]);
    const double h = 0.25 * ORACLE_PI;   /* [-1, 1] -> [0, pi/2]: angle = (x + 1) pi / 4 */
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        const double th = (x[i] + 1.0) * h;
        for (int j = 0; j < n; ++j) {
            const double ph = (x[j] + 1.0) * h;
            const double u[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
            double f = 1.0;
            for (int a = 0; a < 3; ++a) f *= pow(rho[a], c * t * u[a] / L[a]);
            acc += w[i] * h * w[j] * h * sin(th) * f;
        }
    }
    return acc * 2.0 / ORACLE_PI;
}

/* E(t) at several times (t[m], m < n_t). */
void oracle_lj_energy_many(const double L[3], const double beta[6], double c, const double* t, int n_t,
                           const double* x, const double* w, int n, double* out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int m = 0; m < n_t; ++m) out[m] = oracle_lj_energy(L, beta, c, t[m], x, w, n);
}

/* ------------------------------------------------------------------------- */
/* Gradient of a loss through eq. (1)-(6).  g[k] = dLoss/dh[k], k < n_ism.    */
/* Writes dLoss/dbeta[6], dLoss/dps[3], dLoss/dpr[3] for one pair.            */
/* ------------------------------------------------------------------------- */
/* D(x) = w(x) sinc(x) in the sample variable; dD/dx. */
static double dprime_dx(double x, double Nw)
{
    if (!(fabs(x) < 0.5 * Nw)) return 0.0;
    double a = 2.0 * ORACLE_PI * x / Nw;
    double w = 0.5 * (1.0 + cos(a));
    double dw = -0.5 * sin(a) * 2.0 * ORACLE_PI / Nw;
    double sc, dsc;
    if (x == 0.0) {
        sc = 1.0;
        dsc = 0.0;
    } else {
        sc = sinpi_exact(x) / (ORACLE_PI * x);
        double cp = cos(ORACLE_PI * (x - nearbyint(x))) * ((((long long)nearbyint(x)) & 1LL) ? -1.0 : 1.0);
        dsc = (cp - sc) / x;
    }
    return dw * sc + w * dsc;
}

void oracle_rir_grad(const double L[3], const double beta[6], double c, double fs, double Tw,
                     const double ps[3], const double pr[3], const int N[3], int n_ism,
                     const double* g, double dbeta[6], double dps[3], double dpr[3])
{
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) oracle_grid_bounds(N[a], &lo[a], &hi[a]);
    for (int i = 0; i < 6; ++i) dbeta[i] = 0.0;
    for (int a = 0; a < 3; ++a) { dps[a] = 0.0; dpr[a] = 0.0; }
    double Nw = Tw * fs;
    for (int nx = lo[0]; nx < hi[0]; ++nx)
        for (int ny = lo[1]; ny < hi[1]; ++ny)
            for (int nz = lo[2]; nz < hi[2]; ++nz) {
                int n[3] = {nx, ny, nz};
                int e[6];
                double p[3], diff[3], d2 = 0.0, sgn[3];
                for (int a = 0; a < 3; ++a) {
                    p[a] = oracle_image_coord(n[a], L[a], ps[a]);
                    sgn[a] = (n[a] % 2 == 0) ? 1.0 : -1.0;     /* d p_n / d p_s */
                    oracle_image_exponents(n[a], &e[2 * a], &e[2 * a + 1]);
                    diff[a] = pr[a] - p[a];
                    d2 += diff[a] * diff[a];
                }
                double bn = 1.0;
                for (int w = 0; w < 6; ++w) bn *= ipow(beta[w], e[w]);
                double d = sqrt(d2);
                double A = bn / (4.0 * ORACLE_PI * d);
                double s = fs * d / c;
                double half = 0.5 * Nw;
                long k0 = (long)floor(s - half), k1 = (long)ceil(s + half);
                if (k0 < 0) k0 = 0;
                if (k1 > n_ism - 1) k1 = n_ism - 1;
                double gA = 0.0, gs = 0.0;
                for (long k = k0; k <= k1; ++k) {
                    double x = (double)k - s;
                    gA += g[k] * oracle_delta_prime(x, fs, Tw);
                    gs += g[k] * (-A) * dprime_dx(x, Nw);        /* d h_k / d s */
                }
                if (gA == 0.0 && gs == 0.0) continue;
                /* d/d beta_w of A = beta_n / (4 pi d): product rule, valid at beta = 0 */
                for (int w = 0; w < 6; ++w) {
                    if (e[w] == 0) continue;
                    double part = (double)e[w] * ipow(beta[w], e[w] - 1);
                    for (int v = 0; v < 6; ++v)
                        if (v != w) part *= ipow(beta[v], e[v]);
                    dbeta[w] += gA * part / (4.0 * ORACLE_PI * d);
                }
                double gd = gA * (-A / d) + gs * (fs / c);
                for (int a = 0; a < 3; ++a) {
                    double dd = diff[a] / d;                   /* d d / d p_r */
                    dpr[a] += gd * dd;
                    dps[a] += gd * (-dd) * sgn[a];
                }
            }
}
