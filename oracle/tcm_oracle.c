/*
 * tcm_oracle.c -- CPU oracle for the Triggered Cells Method (Naeh, arXiv:1702.00216).
 *
 * TEST INFRASTRUCTURE ONLY (see tcm_oracle.h).  Plain, slow, obviously correct
 * C.  Built with -O2 -ffp-contract=off and without -ffast-math, so every + - *
 * is one IEEE round-to-nearest operation and subnormals are kept.
 *
 * The type-generic parts (dense FDTD and TCM) live in tcm_oracle_impl.inc,
 * included once with REAL = float and once with REAL = double.
 */
#define _GNU_SOURCE
#include "tcm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) n = 1;
    omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Media rules at one node (Media section: media given by rules).  Later rules
 * override earlier ones: background, then layers, then spheres. */
static float media_rule_c(int64_t i, int64_t j, int64_t l, float c_background,
                          int n_layers, const double *layer_z, const float *layer_c,
                          int n_spheres, const double *sph, const float *sphere_c)
{
    float c = c_background;
    for (int m = 0; m < n_layers; ++m)
        if ((double)l >= layer_z[m]) c = layer_c[m];
    for (int s = 0; s < n_spheres; ++s) {
        double dx = (double)i - sph[4 * s + 0];
        double dy = (double)j - sph[4 * s + 1];
        double dz = (double)l - sph[4 * s + 2];
        double r = sph[4 * s + 3];
        if (dx * dx + dy * dy + dz * dz <= r * r) c = sphere_c[s];
    }
    return c;
}

void orc_rules_c(int64_t nx, int64_t ny, int64_t nz, float c_background,
                 int n_layers, const double *layer_z, const float *layer_c,
                 int n_spheres, const double *sphere_xyzr, const float *sphere_c,
                 float *c_out)
{
    for (int64_t l = 0; l < nz; ++l)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                c_out[(l * ny + j) * nx + i] =
                    media_rule_c(i, j, l, c_background, n_layers, layer_z, layer_c,
                                 n_spheres, sphere_xyzr, sphere_c);
}

/* Eq. 3 coefficient (c*dt/dx)^2, formed in FP64. */
static double k_of_c(float c, double dt, double dx)
{
    double r = (double)c * dt / dx;
    return r * r;
}

void orc_k_from_c_f32(const float *c, int64_t n, double dt, double dx, float *k_out)
{
    for (int64_t i = 0; i < n; ++i) k_out[i] = (float)k_of_c(c[i], dt, dx);
}

void orc_k_from_c_f64(const float *c, int64_t n, double dt, double dx, double *k_out)
{
    for (int64_t i = 0; i < n; ++i) k_out[i] = k_of_c(c[i], dt, dx);
}

/* ---- energy ------------------------------------------------------------- */
/* Leapfrog energy (see header).  Plain double loops; the FP32 entry widens
 * each value first. */
#define ENERGY_BODY(KT, FT)                                                              \
    double e = 0.0;                                                                      \
    for (int64_t l = 0; l < nz; ++l)                                                     \
        for (int64_t j = 0; j < ny; ++j)                                                 \
            for (int64_t i = 0; i < nx; ++i) {                                           \
                int64_t id = (l * ny + j) * nx + i;                                      \
                double bi = (double)b[id];                                               \
                double nb = 0.0;                                                         \
                if (i > 0) nb += (double)b[id - 1];                                      \
                if (i < nx - 1) nb += (double)b[id + 1];                                 \
                if (j > 0) nb += (double)b[id - nx];                                     \
                if (j < ny - 1) nb += (double)b[id + nx];                                \
                if (l > 0) nb += (double)b[id - nx * ny];                                \
                if (l < nz - 1) nb += (double)b[id + nx * ny];                           \
                double kb = 6.0 * bi - nb;                                               \
                double d = (double)a[id] - bi;                                           \
                e += d * d / (double)k[id] + (double)a[id] * kb;                         \
            }                                                                            \
    return e;

double orc_energy_f64(int64_t nx, int64_t ny, int64_t nz, const double *k,
                      const double *a, const double *b)
{
    ENERGY_BODY(double, double)
}

double orc_energy_f32(int64_t nx, int64_t ny, int64_t nz, const float *k,
                      const float *a, const float *b)
{
    ENERGY_BODY(float, float)
}

/* ---- 16-bit storage formats ------------------------------------------------ */
/* Round v to nearest-even with `bits` significant bits, the quantum never
 * below 2^min_exp (gradual underflow), overflowing to inf at 2^max_exp.
 * In binary64 every step is exact: v has 24 bits, v / quantum is an integer
 * plus a fraction of at most 24 bits, and rint() rounds ties to even. */
static float round_to_format(float v, int bits, int min_exp, int max_exp)
{
    if (v == 0.0f || isnan(v) || isinf(v)) return v;
    int e;
    frexp((double)v, &e);   /* |v| in [2^(e-1), 2^e) */
    int qe = (e - 1) - (bits - 1);
    if (qe < min_exp) qe = min_exp;
    const double quantum = ldexp(1.0, qe);
    const double r = rint((double)v / quantum) * quantum;
    if (fabs(r) >= ldexp(1.0, max_exp)) return v < 0 ? -INFINITY : INFINITY;
    return (float)r;
}

/* bfloat16: 1+7 bits significand, exponent field as binary32 (bias 127):
 * smallest subnormal 2^-126 * 2^-7 = 2^-133, finite values below 2^128. */
float orc_round_bf16(float v) { return round_to_format(v, 8, -133, 128); }

/* binary16: 1+10 bits significand, bias 15: smallest subnormal 2^-24, largest
 * finite (2 - 2^-10) * 2^15 = 65504, everything rounding to 2^16 overflows. */
float orc_round_f16(float v) { return round_to_format(v, 11, -24, 16); }

/* ---- Fourier transform for the frequency-domain shut-down (Eq. 7) -------- */
/* In-place complex DFT of length n (a power of two) by the radix-2
 * Cooley-Tukey algorithm: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n), no
 * scaling.  Input permuted to bit-reversed order, then log2(n) butterfly
 * passes. */
void orc_fft(double *re, double *im, int n, int sign)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / len;
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                const double wr = cos(ang * k), wi = sin(ang * k);
                const int a = i + k, b = i + k + len / 2;
                const double xr = re[b] * wr - im[b] * wi, xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr;
                im[b] = im[a] - xi;
                re[a] += xr;
                im[a] += xi;
            }
    }
}

/* Low-pass response at DFT index kappa of length M: nu = min(kappa, M -
 * kappa) / (M/2) in [0, 1] (1 = Nyquist); 1 up to `pass`, 0 from `stop`, a
 * raised cosine between. */
double orc_lpf_response(int kappa, int M, double pass, double stop)
{
    const int kk = kappa < M - kappa ? kappa : M - kappa;
    const double nu = (double)kk / (M / 2.0);
    if (nu <= pass) return 1.0;
    if (nu >= stop) return 0.0;
    return 0.5 * (1.0 + cos(M_PI * (nu - pass) / (stop - pass)));
}

/* Eq. 7 on one region: v (L*L*L doubles, x fastest) is zero-padded to
 * M*M*M, transformed (3D DFT = 1D transforms along x, y, z), multiplied by
 * H(kx) H(ky) H(kz), transformed back and scaled by 1/M^3; the real part of
 * the first L*L*L samples replaces v. */
void orc_lpf_region(double *v, int L, int M, double pass, double stop)
{
    const size_t n3 = (size_t)M * M * M;
    double *re = (double *)calloc(n3, sizeof(double));
    double *im = (double *)calloc(n3, sizeof(double));
    double *lr = (double *)malloc((size_t)M * sizeof(double));
    double *li = (double *)malloc((size_t)M * sizeof(double));
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) re[((size_t)z * M + y) * M + x] = v[((size_t)z * L + y) * L + x];
    for (int pass_dir = 0; pass_dir < 2; ++pass_dir) {
        const int sign = pass_dir == 0 ? -1 : 1;
        for (int axis = 0; axis < 3; ++axis) {
            const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)M : (size_t)M * M);
            for (int a = 0; a < M; ++a)
                for (int b = 0; b < M; ++b) {
                    size_t base;
                    if (axis == 0) base = ((size_t)a * M + b) * M;
                    else if (axis == 1) base = (size_t)a * M * M + b;
                    else base = (size_t)a * M + b;
                    for (int k = 0; k < M; ++k) {
                        lr[k] = re[base + k * stride];
                        li[k] = im[base + k * stride];
                    }
                    orc_fft(lr, li, M, sign);
                    for (int k = 0; k < M; ++k) {
                        re[base + k * stride] = lr[k];
                        im[base + k * stride] = li[k];
                    }
                }
        }
        if (pass_dir == 0)
            for (int kz = 0; kz < M; ++kz)
                for (int ky = 0; ky < M; ++ky)
                    for (int kx = 0; kx < M; ++kx) {
                        const double h = orc_lpf_response(kx, M, pass, stop) * orc_lpf_response(ky, M, pass, stop) *
                                         orc_lpf_response(kz, M, pass, stop);
                        const size_t i = ((size_t)kz * M + ky) * M + kx;
                        re[i] *= h;
                        im[i] *= h;
                    }
    }
    const double inv = 1.0 / (double)n3;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) v[((size_t)z * L + y) * L + x] = re[((size_t)z * M + y) * M + x] * inv;
    free(re); free(im); free(lr); free(li);
}

/* ---- type-generic programs ---------------------------------------------- */
#define REAL float
#define SFX(name) name##_f32
#define ORC_TCM_STRUCT orc_tcm_f32_s
#include "tcm_oracle_impl.inc"
#undef REAL
#undef SFX
#undef ORC_TCM_STRUCT

#define REAL double
#define SFX(name) name##_f64
#define ORC_TCM_STRUCT orc_tcm_f64_s
#include "tcm_oracle_impl.inc"
#undef REAL
#undef SFX
#undef ORC_TCM_STRUCT
