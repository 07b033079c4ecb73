/*
 * ac_oracle.c -- plain, slow FP64 CPU oracle for Monte-Carlo snakuscule evolution
 * (Lotfollahi et al., "Three-Dimensional GPU-Accelerated Active Contours for
 * Automated Localization of Cells in Large Images", arXiv:1804.06304).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path.  Every quantity is computed in double precision, one
 * sample at a time, in the order the paper states the method:
 *
 *   state    identifier points p, q with p_y = q_y, p_z = q_z      (Eq. 6)
 *   energy   E = (q_x - p_x)^-d * sum_k S(r) I(k)                   (Eqs. 5-6)
 *   sum_k    Monte-Carlo estimate over uniform samples in the ball of radius
 *            R + dR/2 ("Monte-Carlo Integration" section), each sample weighted by
 *            V/N with V the ball volume
 *   partials dE/dp, dE/dq                                           (Eqs. 7-11)
 *   update   p <- p - eps dE/dp, q <- q - eps dE/dq, eps = eps0/sqrt(n) (Eqs. 12-15)
 *   localize drop E > E0, overlap competition ||c'-c''|| < rho max(R',R'')
 *            with the lower energy surviving ("Results and Discussion")
 *   grid     the same sums over the voxel centres inside R + dR/2, each weighted
 *            by one voxel volume: Eq. 5 taken literally (the paper's integration
 *            before it moved to sampling)
 *   stopping optional rules for the paper's future work (convergence freeze, energy
 *            culling): see or_params and or_evolve
 *
 * Readings where the paper is silent:
 *   - the image between voxel centres is the trilinear (2D: bilinear) interpolant,
 *     clamp-to-edge outside the volume;
 *   - S(r;R) = -1 + 2 ramp((r - rho R)/dr) - ramp((r - R)/dR), ramp(t) =
 *     clamp(t + 1/2, 0, 1): -1 in the inner ball, +1 in the annulus, linear bands
 *     of the fixed widths dr = dR / 2^(1/d) and dR (Eq. 5 and the relation below
 *     it), zero beyond R + dR/2; this is the only piecewise-linear shape for which
 *     the integral of S r^(d-1) vanishes for every R;
 *   - d = 3 in 3D (alpha = 3, Eq. 4) and d = 2 in 2D (the same symmetric-slope
 *     argument gives alpha = 2 for disks);
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
 *     (block, iteration, contour, stream) and key (seed_lo, seed_hi); the words of
 *     one iteration and contour form the stream block 0, block 1, ... (four words
 *     each) and sample j takes words 2 j and 2 j + 1 (one block per two samples);
 *     2D: two 24-bit uniforms u = (w >> 8) * 2^-24, one per word, and the paper's
 *     disk point (sqrt(u0) cos th, sqrt(u0) sin th), th = 2 pi u1; 3D: three 21-bit
 *     uniforms from the 64 bits, u0 = the top 21 bits of w0, u1 = the low 21 bits of
 *     w1, u2 = the low 11 bits of w0 followed by the top 10 bits of w1, each times
 *     2^-21, and the ball point cbrt(u0) (sin phi cos th, sin phi sin th, cos phi)
 *     with cos phi = 1 - 2 u1, th = 2 pi u2;
 *   - clamps that the paper does not state: |dc| <= max_step, |dR| <= max_step,
 *     R in [Rmin, Rmax], c inside the box of voxel centres;
 *   - T iterations = T evaluations; the update follows evaluations 1..T-1, so the
 *     reported energy belongs to the reported state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, written from the round function and key schedule published */
/* by Salmon, Moraes, Dror and Shaw (SC'11).                                 */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A 32-bit word to a uniform in [0, 1): its top 24 bits times 2^-24. */
double or_uniform24(uint32_t w)
{
    return (double)(w >> 8) * (1.0 / 16777216.0);
}

/* The three 21-bit uniforms of a 3D sample from its two words: the 64 bits give
 * u0 = w0 bits 31..11, u1 = w1 bits 20..0, u2 = w0 bits 10..0 then w1 bits 31..22,
 * each an integer below 2^21 times 2^-21 (w1 bit 21 is unused). */
void or_uniforms21(uint32_t w0, uint32_t w1, double u[3])
{
    const uint32_t a = w0 >> 11;
    const uint32_t b = w1 & 0x1FFFFFu;
    const uint32_t c = ((w0 & 0x7FFu) << 10) | (w1 >> 22);
    u[0] = (double)a / 2097152.0;
    u[1] = (double)b / 2097152.0;
    u[2] = (double)c / 2097152.0;
}

/* The unit-ball (disk) point of one sample from its two random words. */
void or_unit_sample(int ndim, const uint32_t w[2], double u[3])
{
    if (ndim == 3) {
        double v[3];
        or_uniforms21(w[0], w[1], v);
        double rad = cbrt(v[0]);
        double cphi = 1.0 - 2.0 * v[1];
        double sphi = sqrt(fmax(0.0, 1.0 - cphi * cphi));
        double th = 2.0 * OR_PI * v[2];
        u[0] = rad * sphi * cos(th);
        u[1] = rad * sphi * sin(th);
        u[2] = rad * cphi;
    } else {
        double r = or_uniform24(w[0]);
        double th = 2.0 * OR_PI * or_uniform24(w[1]);
        u[0] = sqrt(r) * cos(th);
        u[1] = sqrt(r) * sin(th);
        u[2] = 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Image model                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    const void *data;  /* voxel values, x fastest                          */
    int32_t dtype;     /* 0 uint8, 1 uint16, 2 binary16 bits, 3 float32     */
    int32_t ndim;      /* 2 or 3                                           */
    int64_t n[3];      /* voxels along x, y, z (z = 1 in 2D)               */
    int64_t pitch[3];  /* element strides along x, y, z                    */
    double spacing[3]; /* physical size of a voxel along x, y, z           */
    double scale;      /* intensity = scale * stored value                 */
    int32_t analytic;  /* 1: ignore the voxels, use the analytic blob below */
    int32_t pad_;
    double blob_c[3];  /* analytic image: offset + grad.x + amp [|x-c| < r] */
    double blob_r, blob_amp, offset;
    double grad[3];
} or_image;

/* IEEE binary16 bits to a double, from the format's definition. */
double or_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1, ex = (h >> 10) & 31, man = h & 1023;
    double v;
    if (ex == 0)
        v = ldexp((double)man, -24);              /* subnormal: man * 2^-14 / 2^10 */
    else if (ex == 31)
        v = man ? NAN : INFINITY;
    else
        v = ldexp(1.0 + man / 1024.0, ex - 15);
    return sign ? -v : v;
}

static double voxel(const or_image *img, int64_t i, int64_t j, int64_t k)
{
    int64_t off = i * img->pitch[0] + j * img->pitch[1] + k * img->pitch[2];
    switch (img->dtype) {
    case 0: return (double)((const uint8_t *)img->data)[off];
    case 1: return (double)((const uint16_t *)img->data)[off];
    case 2: return or_half_to_double(((const uint16_t *)img->data)[off]);
    default: return (double)((const float *)img->data)[off];
    }
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* I(x) at a physical position: the multilinear interpolant of the voxel values,
 * voxel centres at integer indices (index = position / spacing), each tap index
 * clamped to the volume (clamp-to-edge). */
double or_image_value(const or_image *img, const double x[3])
{
    if (img->analytic) {
        double d2 = 0.0, lin = 0.0;
        for (int a = 0; a < img->ndim; ++a) {
            double t = x[a] - img->blob_c[a];
            d2 += t * t;
            lin += img->grad[a] * x[a];
        }
        return img->offset + lin + (sqrt(d2) < img->blob_r ? img->blob_amp : 0.0);
    }
    int64_t base[3] = {0, 0, 0};
    double frac[3] = {0, 0, 0};
    for (int a = 0; a < img->ndim; ++a) {
        double xi = x[a] / img->spacing[a];
        double f = floor(xi);
        base[a] = (int64_t)f;
        frac[a] = xi - f;
    }
    double acc = 0.0;
    int corners = img->ndim == 3 ? 8 : 4;
    for (int m = 0; m < corners; ++m) {
        int ox = m & 1, oy = (m >> 1) & 1, oz = (m >> 2) & 1;
        double wgt = (ox ? frac[0] : 1.0 - frac[0]) * (oy ? frac[1] : 1.0 - frac[1]);
        if (img->ndim == 3) wgt *= (oz ? frac[2] : 1.0 - frac[2]);
        int64_t i = clampi(base[0] + ox, 0, img->n[0] - 1);
        int64_t j = clampi(base[1] + oy, 0, img->n[1] - 1);
        int64_t k = img->ndim == 3 ? clampi(base[2] + oz, 0, img->n[2] - 1) : 0;
        acc += wgt * voxel(img, i, j, k);
    }
    return img->scale * acc;
}

/* ------------------------------------------------------------------------- */
/* Weight function S(r;R) and its partials (Eq. 5, Fig. 4d reading)         */
/* ------------------------------------------------------------------------- */
static double ramp(double t) { t += 0.5; return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }
/* band membership: t in [-1/2, 1/2) */
static int inband(double t) { return t >= -0.5 && t < 0.5; }

double or_rho(int ndim) { return ndim == 3 ? pow(2.0, -1.0 / 3.0) : pow(2.0, -0.5); }

/* out[0] = S, out[1] = dS/dR (r fixed), out[2] = dS/dr (R fixed) */
void or_weight(int ndim, double r, double R, double dR, double out[3])
{
    double rho = or_rho(ndim);
    double dr = dR * rho;              /* dr = dR / 2^(1/d): 3D relation below Eq. 5 */
    double t1 = (r - rho * R) / dr;    /* inner band, centred on rho R */
    double t2 = (r - R) / dR;          /* outer band, centred on R     */
    out[0] = -1.0 + 2.0 * ramp(t1) - ramp(t2);
    out[1] = (inband(t1) ? -2.0 * rho / dr : 0.0) + (inband(t2) ? 1.0 / dR : 0.0);
    out[2] = (inband(t1) ? 2.0 / dr : 0.0) - (inband(t2) ? 1.0 / dR : 0.0);
}

/* ------------------------------------------------------------------------- */
/* Energy and partials at (p, q): Eqs. 5-11 with the Monte-Carlo measure     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t ndim;
    int32_t N;          /* samples per contour and iteration */
    int32_t T;          /* iterations                        */
    int32_t pad_;
    double eps0;        /* learning-rate constant of eps = eps0/sqrt(n) */
    double dR;          /* fixed outer band width                        */
    double Rmin, Rmax;  /* radius clamp                                  */
    double max_step;    /* per-iteration step clamp                      */
    double edge_tol;    /* band-edge proximity that flags a sample       */
    uint32_t key[2];    /* Philox key (seed low, seed high)              */
    uint32_t stream_id; /* fourth counter word                           */
    int32_t integration;/* 0: Monte-Carlo samples; 1: the voxel grid K of Eq. 5 */
    /* stopping rules (0 disables each): a contour stops when its proposed step
     * (largest coordinate change of c and R) is below freeze_tol for freeze_iters
     * consecutive updates (that last step is not applied), or when its energy at
     * iteration cull_iter is above cull_E (no update after it) */
    double freeze_tol;
    int32_t freeze_iters;
    int32_t cull_iter;
    double cull_E;
} or_params;

/* Result layout of or_eval_pq (doubles). */
enum {
    OR_E = 0,
    OR_DEDP = 1,      /* 3: dE/dp_x, dE/dp_y, dE/dp_z (Eqs. 7, 9, 10) */
    OR_DEDQ = 4,      /* 3: dE/dq_x, dE/dq_y, dE/dq_z (Eqs. 8, 9, 10) */
    OR_DEDR = 7,      /* dE/dR = dE/dq_x - dE/dp_x                   */
    OR_DEDC = 8,      /* 3: dE/dc = dE/dp + dE/dq                     */
    OR_MAG_E = 11,    /* magnitude sums for tolerances                */
    OR_MAG_R = 12,
    OR_MAG_C = 13,    /* 3 */
    OR_FLAGS = 16,    /* samples within edge_tol of a band edge       */
    OR_SUM_SI = 17,   /* the raw sum over K of S I (MC measure)       */
    OR_VAR_E = 18,    /* variance of the MC estimate of E             */
    OR_VAR_R = 19,    /* ... of dE/dR                                 */
    OR_VAR_C = 20,    /* 3: ... of dE/dc                              */
    OR_MAG_G = 23,    /* gamma V/N sum |S'(r)| I: direction-free magnitude of dE/dc */
    OR_MAG_I = 24,    /* gamma V/N sum |I|: intensity mass of the footprint       */
    OR_RES_LEN = 25
};

static void sample_block(const or_params *P, int64_t blk, int64_t iter, int64_t k, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)iter, (uint32_t)k, P->stream_id};
    or_philox4x32_10(ctr, P->key, w);
}

/* Reader of the word stream of one (iteration, contour): word m is word m % 4 of
 * block m / 4; the last block drawn is kept. */
typedef struct {
    int64_t blk;
    uint32_t w[4];
} word_stream;

static void sample_words(const or_params *P, word_stream *S, int64_t j, int64_t iter, int64_t k, uint32_t out[2])
{
    for (int t = 0; t < 2; ++t) {
        const int64_t m = 2 * j + t;
        if (m / 4 != S->blk) {
            S->blk = m / 4;
            sample_block(P, S->blk, iter, k, S->w);
        }
        out[t] = S->w[m % 4];
    }
}

/* Running sums over the points of K for one evaluation: the weighted sums of S I
 * and of the partials of S with respect to p and q times I (Eqs. 5, 7-10), the
 * magnitude sums that scale the parity tolerances, and raw moments of the
 * per-point terms (for the Monte-Carlo variance). */
typedef struct {
    double sSI, sdpx, sdqx, sdpy, sdpz;
    double mSI, mdSdR, mc[3], mg, mi;
    double m1[5], m2[5];
    int64_t flags, count;
} or_sums;

/* One point x of K with image value I and measure w, for the contour of centre c
 * and radius R. */
static void add_point(or_sums *A, const or_params *P, const double c[3], double R, const double edges[4],
                      const double x[3], double I, double w)
{
    const int d = P->ndim;
    double r2 = 0, dir[3] = {0, 0, 0}, Sw[3];
    for (int a = 0; a < d; ++a) r2 += (x[a] - c[a]) * (x[a] - c[a]);
    const double r = sqrt(r2);
    if (r > 0)
        for (int a = 0; a < d; ++a) dir[a] = (x[a] - c[a]) / r;
    or_weight(d, r, R, P->dR, Sw);
    const double S = Sw[0], dSdR = Sw[1], dSdr = Sw[2];
    /* chain rule through r = |k - c|, c = (p + q)/2, R = (q_x - p_x)/2 */
    const double dSdpx = dSdr * (-0.5 * dir[0]) + dSdR * (-0.5);
    const double dSdqx = dSdr * (-0.5 * dir[0]) + dSdR * (+0.5);
    const double dSdpy = dSdr * (-0.5 * dir[1]);
    const double dSdpz = dSdr * (-0.5 * dir[2]);
    A->sSI += w * S * I;
    A->sdpx += w * dSdpx * I;
    A->sdqx += w * dSdqx * I;
    A->sdpy += w * dSdpy * I;
    A->sdpz += w * dSdpz * I;
    A->mSI += w * fabs(S * I);
    A->mdSdR += w * fabs(dSdR * I);
    for (int a = 0; a < d; ++a) A->mc[a] += w * fabs(dSdr * dir[a] * I);
    A->mg += w * fabs(dSdr * I);
    A->mi += w * fabs(I);
    const double terms[5] = {S * I, (-(double)d / R * S + dSdR) * I, -dSdr * dir[0] * I, -dSdr * dir[1] * I,
                             -dSdr * dir[2] * I};
    for (int m = 0; m < 5; ++m) {
        A->m1[m] += terms[m];
        A->m2[m] += terms[m] * terms[m];
    }
    for (int e = 0; e < 4; ++e)
        if (fabs(r - edges[e]) < P->edge_tol) {
            ++A->flags;
            break;
        }
    ++A->count;
}

/* Sums to E and its partials (Eqs. 6-11); mc_V > 0: Monte-Carlo with ball volume
 * mc_V, which also gives the variance of each estimate. */
static void finish_pq(const or_sums *A, const or_params *P, const double p[3], const double q[3], double mc_V,
                      double *res)
{
    const int d = P->ndim;
    const double R = 0.5 * (q[0] - p[0]);
    const double L = q[0] - p[0];
    const double gamma = 1.0 / pow(L, d);          /* Eq. 11 with exponent d */
    memset(res, 0, sizeof(double) * OR_RES_LEN);
    res[OR_E] = gamma * A->sSI;                                      /* Eq. 6 */
    res[OR_DEDP + 0] = gamma * ((double)d / L * A->sSI + A->sdpx);  /* Eq. 7 */
    res[OR_DEDQ + 0] = gamma * (-(double)d / L * A->sSI + A->sdqx); /* Eq. 8 */
    res[OR_DEDP + 1] = res[OR_DEDQ + 1] = gamma * A->sdpy;           /* Eq. 9 */
    res[OR_DEDP + 2] = res[OR_DEDQ + 2] = d == 3 ? gamma * A->sdpz : 0.0; /* Eq. 10 */
    res[OR_DEDR] = res[OR_DEDQ + 0] - res[OR_DEDP + 0];
    for (int a = 0; a < 3; ++a) res[OR_DEDC + a] = res[OR_DEDP + a] + res[OR_DEDQ + a];
    res[OR_MAG_E] = gamma * A->mSI;
    res[OR_MAG_R] = gamma * ((double)d / R * A->mSI + A->mdSdR);
    for (int a = 0; a < 3; ++a) res[OR_MAG_C + a] = gamma * A->mc[a];
    res[OR_FLAGS] = (double)A->flags;
    res[OR_SUM_SI] = A->sSI;
    res[OR_MAG_G] = gamma * A->mg;
    res[OR_MAG_I] = gamma * A->mi;
    if (mc_V > 0 && A->count > 0)
        for (int m = 0; m < 5; ++m) {
            /* each sample's term times gamma V is an unbiased one-sample estimate */
            double mean = A->m1[m] / A->count, var = A->m2[m] / A->count - mean * mean;
            double sc = gamma * mc_V;
            res[OR_VAR_E + m] = (var > 0 ? var : 0) * sc * sc / A->count;
        }
}

static void band_edges(const or_params *P, double R, double edges[4])
{
    const double rho = or_rho(P->ndim), dr = P->dR * rho;
    edges[0] = rho * R - 0.5 * dr;
    edges[1] = rho * R + 0.5 * dr;
    edges[2] = R - 0.5 * P->dR;
    edges[3] = R + 0.5 * P->dR;
}

/* Monte-Carlo form ("Monte-Carlo Integration" section): K is N uniform samples of
 * the ball of radius R + dR/2, each of measure V/N. */
void or_eval_pq(const or_image *img, const or_params *P, const double p[3], const double q[3],
                int64_t iter, int64_t k, double *res)
{
    const int d = P->ndim;
    const double R = 0.5 * (q[0] - p[0]);          /* R = ||p - q|| / 2, Eq. 6 */
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = 0.5 * (p[a] + q[a]);
    const double Ro = R + 0.5 * P->dR;             /* radius of K (Eq. 5) */
    const double V = d == 3 ? 4.0 / 3.0 * OR_PI * Ro * Ro * Ro : OR_PI * Ro * Ro;
    const double wmc = V / P->N;                   /* measure of one MC sample */
    double edges[4];
    band_edges(P, R, edges);
    or_sums A;
    memset(&A, 0, sizeof(A));
    word_stream S = {-1, {0, 0, 0, 0}};
    uint32_t w[2];
    for (int64_t j = 0; j < P->N; ++j) {
        double u[3], x[3];
        sample_words(P, &S, j, iter, k, w);
        or_unit_sample(d, w, u);
        for (int a = 0; a < 3; ++a) x[a] = c[a] + Ro * u[a];
        if (d == 2) x[2] = c[2];
        add_point(&A, P, c, R, edges, x, or_image_value(img, x), wmc);
    }
    finish_pq(&A, P, p, q, V, res);
}

/* Grid form, Eq. 5 taken literally (the paper's integration before Monte Carlo):
 * K is every voxel centre k (index times spacing) with |k - c| <= R + dR/2, each of
 * measure one voxel volume, the image extended beyond the volume by clamp-to-edge
 * as for the samples. */
void or_eval_grid_pq(const or_image *img, const or_params *P, const double p[3], const double q[3], double *res)
{
    const int d = P->ndim;
    const double R = 0.5 * (q[0] - p[0]);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = 0.5 * (p[a] + q[a]);
    const double Ro = R + 0.5 * P->dR;
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double vox = 1.0;
    for (int a = 0; a < d; ++a) {
        lo[a] = (int64_t)ceil((c[a] - Ro) / img->spacing[a]);
        hi[a] = (int64_t)floor((c[a] + Ro) / img->spacing[a]);
        vox *= img->spacing[a];
    }
    double edges[4];
    band_edges(P, R, edges);
    or_sums A;
    memset(&A, 0, sizeof(A));
    for (int64_t kk = lo[2]; kk <= hi[2]; ++kk)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                double x[3] = {i * img->spacing[0], j * img->spacing[1], d == 3 ? kk * img->spacing[2] : c[2]};
                double r2 = 0;
                for (int a = 0; a < d; ++a) r2 += (x[a] - c[a]) * (x[a] - c[a]);
                if (r2 > Ro * Ro) continue;
                add_point(&A, P, c, R, edges, x, or_image_value(img, x), vox);
            }
    finish_pq(&A, P, p, q, 0.0, res);
}

static void eval_any(const or_image *img, const or_params *P, const double p[3], const double q[3], int64_t iter,
                     int64_t k, double *res)
{
    if (P->integration == 1) or_eval_grid_pq(img, P, p, q, res);
    else or_eval_pq(img, P, p, q, iter, k, res);
}

/* Same evaluation from the centre/radius form of the state. */
void or_eval_cr(const or_image *img, const or_params *P, const double c[3], double R,
                int64_t iter, int64_t k, double *res)
{
    double p[3] = {c[0] - R, c[1], c[2]}, q[3] = {c[0] + R, c[1], c[2]};
    eval_any(img, P, p, q, iter, k, res);
}

/* Eq. 5 taken literally: the sum over the voxel grid K inside R + dR/2, times the
 * voxel volume, normalised by (2R)^d.  Used for the grid-versus-MC comparison. */
double or_energy_grid(const or_image *img, int ndim, const double c[3], double R, double dR)
{
    const double Ro = R + 0.5 * dR;
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double vox = 1.0;
    for (int a = 0; a < ndim; ++a) {
        lo[a] = (int64_t)ceil((c[a] - Ro) / img->spacing[a]);
        hi[a] = (int64_t)floor((c[a] + Ro) / img->spacing[a]);
        vox *= img->spacing[a];
    }
    double s = 0.0;
    for (int64_t k = lo[2]; k <= hi[2]; ++k)
        for (int64_t j = lo[1]; j <= hi[1]; ++j)
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                double x[3] = {i * img->spacing[0], j * img->spacing[1], ndim == 3 ? k * img->spacing[2] : c[2]};
                double r2 = 0;
                for (int a = 0; a < ndim; ++a) r2 += (x[a] - c[a]) * (x[a] - c[a]);
                double r = sqrt(r2);
                if (r > Ro) continue;
                double Sw[3];
                or_weight(ndim, r, R, dR, Sw);
                s += Sw[0] * or_image_value(img, x) * vox;
            }
    return s / pow(2.0 * R, ndim);
}

/* ------------------------------------------------------------------------- */
/* Update (Eqs. 12-15) and the clamps the paper leaves open                  */
/* ------------------------------------------------------------------------- */
void or_update_pq(const or_image *img, const or_params *P, int64_t iter, const double *res,
                  double p[3], double q[3])
{
    const int d = P->ndim;
    const double eps = P->eps0 / sqrt((double)iter);  /* eps = eps0 / sqrt(n) */
    double pn[3], qn[3];
    for (int a = 0; a < 3; ++a) {
        pn[a] = p[a] - eps * res[OR_DEDP + a];          /* p + eps dp/dt, Eqs. 12, 14 */
        qn[a] = q[a] - eps * res[OR_DEDQ + a];          /* q + eps dq/dt, Eqs. 13, 15 */
    }
    /* clamps, applied to the centre/radius the identifier points define */
    double c0[3], c1[3], dc[3], nrm2 = 0;
    for (int a = 0; a < 3; ++a) {
        c0[a] = 0.5 * (p[a] + q[a]);
        c1[a] = 0.5 * (pn[a] + qn[a]);
        dc[a] = a < d ? c1[a] - c0[a] : 0.0;
        nrm2 += dc[a] * dc[a];
    }
    const double R0 = 0.5 * (q[0] - p[0]);
    double dRr = 0.5 * (qn[0] - pn[0]) - R0;
    const double nrm = sqrt(nrm2);
    if (nrm > P->max_step)
        for (int a = 0; a < 3; ++a) dc[a] *= P->max_step / nrm;
    if (dRr > P->max_step) dRr = P->max_step;
    if (dRr < -P->max_step) dRr = -P->max_step;
    double R = R0 + dRr;
    if (R < P->Rmin) R = P->Rmin;
    if (R > P->Rmax) R = P->Rmax;
    double c[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = c0[a] + dc[a];
        if (a < d) {
            double top = (double)(img->n[a] - 1) * img->spacing[a];
            if (c[a] < 0.0) c[a] = 0.0;
            if (c[a] > top) c[a] = top;
        }
    }
    p[0] = c[0] - R; q[0] = c[0] + R;
    p[1] = q[1] = c[1];
    p[2] = q[2] = c[2];
}

/* Trace record per (iteration, contour): cx, cy, cz, R, E, dE/dR, dE/dcx, dE/dcy, dE/dcz */
enum { OR_TRACE_LEN = 9 };

/* Evolve C contours for T iterations.  cR holds (cx, cy, cz, R) per contour (in and
 * out); ids[i] is the contour index that enters the Philox counter; E_out receives
 * the energy of the final state; trace (T x C x 9, optional) records every
 * evaluation.  Contours are independent (the "Parallelizing the process" section),
 * so they are spread over `nthreads` OpenMP threads. */
/* T iterations per contour: evaluate, then update (Eqs. 12-15), with the
 * stopping rules of or_params.  `stops` (optional): 0 ran all T iterations, 1
 * stopped by the step rule, 2 stopped by the energy rule; `n_eval` (optional):
 * evaluations made.  A stopped contour keeps the state and energy of its last
 * evaluation; trace rows after it are left untouched. */
void or_evolve(const or_image *img, const or_params *P, int64_t C, const int64_t *ids,
               double *cR, double *E_out, double *trace, int32_t *stops, int32_t *n_eval, int nthreads)
{
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
    for (int64_t i = 0; i < C; ++i) {
        double p[3] = {cR[4 * i] - cR[4 * i + 3], cR[4 * i + 1], cR[4 * i + 2]};
        double q[3] = {cR[4 * i] + cR[4 * i + 3], cR[4 * i + 1], cR[4 * i + 2]};
        double res[OR_RES_LEN];
        int32_t stop = 0, evals = 0, small = 0;
        for (int64_t n = 1; n <= P->T; ++n) {
            eval_any(img, P, p, q, n, ids[i], res);
            evals = (int32_t)n;
            if (trace) {
                double *t = trace + ((n - 1) * C + i) * OR_TRACE_LEN;
                t[0] = 0.5 * (p[0] + q[0]); t[1] = p[1]; t[2] = p[2];
                t[3] = 0.5 * (q[0] - p[0]);
                t[4] = res[OR_E]; t[5] = res[OR_DEDR];
                t[6] = res[OR_DEDC]; t[7] = res[OR_DEDC + 1]; t[8] = res[OR_DEDC + 2];
            }
            if (P->cull_iter > 0 && n == P->cull_iter && res[OR_E] > P->cull_E) {
                stop = 2;
                break;
            }
            if (n == P->T) break;
            double pn[3] = {p[0], p[1], p[2]}, qn[3] = {q[0], q[1], q[2]};
            or_update_pq(img, P, n, res, pn, qn);
            if (P->freeze_iters > 0) {
                double step = fabs(0.5 * (qn[0] - pn[0]) - 0.5 * (q[0] - p[0]));   /* |dR| */
                for (int a = 0; a < P->ndim; ++a) {
                    double ca = 0.5 * (p[a] + q[a]), cn = 0.5 * (pn[a] + qn[a]);
                    if (fabs(cn - ca) > step) step = fabs(cn - ca);
                }
                small = step < P->freeze_tol ? small + 1 : 0;
                if (small >= P->freeze_iters) {
                    stop = 1;
                    break;
                }
            }
            memcpy(p, pn, sizeof(p));
            memcpy(q, qn, sizeof(q));
        }
        cR[4 * i] = 0.5 * (p[0] + q[0]);
        cR[4 * i + 1] = p[1];
        cR[4 * i + 2] = p[2];
        cR[4 * i + 3] = 0.5 * (q[0] - p[0]);
        E_out[i] = res[OR_E];
        if (stops) stops[i] = stop;
        if (n_eval) n_eval[i] = evals;
    }
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Initial lattice (Fig. 1b, Fig. 4b): neighbours sqrt(1.5) R0 apart          */
/* ------------------------------------------------------------------------- */
/* Seeds sit at the centres of cubic cells of side `stride` that tile the volume
 * box [-s/2, n s - s/2] per axis (the leftover split evenly at both ends);
 * R0 = stride / sqrt(1.5).  Writes (cx, cy, cz, R) rows, x fastest, and returns the
 * count; `out` may be NULL to query the count. */
int64_t or_seed_lattice(int ndim, const int64_t n[3], const double spacing[3], double stride,
                        double *out)
{
    int64_t L[3] = {1, 1, 1};
    double first[3] = {0, 0, 0};
    for (int a = 0; a < ndim; ++a) {
        double ext = (double)n[a] * spacing[a];
        L[a] = (int64_t)floor(ext / stride);
        if (L[a] < 1) L[a] = 1;
        first[a] = -0.5 * spacing[a] + 0.5 * (ext - (double)L[a] * stride) + 0.5 * stride;
    }
    int64_t count = L[0] * L[1] * L[2];
    if (!out) return count;
    double R0 = stride / sqrt(1.5);
    int64_t m = 0;
    for (int64_t k = 0; k < L[2]; ++k)
        for (int64_t j = 0; j < L[1]; ++j)
            for (int64_t i = 0; i < L[0]; ++i, ++m) {
                out[4 * m + 0] = first[0] + i * stride;
                out[4 * m + 1] = first[1] + j * stride;
                out[4 * m + 2] = ndim == 3 ? first[2] + k * stride : 0.0;
                out[4 * m + 3] = R0;
            }
    return count;
}

/* ------------------------------------------------------------------------- */
/* Localization: energy cull and overlap competition ("Results and Discussion") */
/* ------------------------------------------------------------------------- */
typedef struct { double E; int64_t id; } or_key;

static int cmp_key(const void *a, const void *b)
{
    const or_key *x = (const or_key *)a, *y = (const or_key *)b;
    if (x->E < y->E) return -1;
    if (x->E > y->E) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Drops contours with E > E0 or non-finite E, then visits the rest from the lowest
 * energy up (ties by lower index) and keeps each one that overlaps no contour kept
 * before it, overlap meaning |c' - c''| < rho max(R', R'').  cR rows are
 * (cx, cy, cz, R) indexed by contour id 0..C-1.  Writes the kept ids in acceptance
 * order and returns their count. */
int64_t or_localize(int ndim, int64_t C, const double *cR, const double *E, double E0,
                    int64_t *out_ids)
{
    const double rho = or_rho(ndim);
    or_key *keys = (or_key *)malloc(sizeof(or_key) * (size_t)(C > 0 ? C : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < C; ++i)
        if (isfinite(E[i]) && !(E[i] > E0)) { keys[m].E = E[i]; keys[m].id = i; ++m; }
    qsort(keys, (size_t)m, sizeof(or_key), cmp_key);
    int64_t kept = 0;
    for (int64_t a = 0; a < m; ++a) {
        const double *ca = cR + 4 * keys[a].id;
        int overlap = 0;
        for (int64_t b = 0; b < kept && !overlap; ++b) {
            const double *cb = cR + 4 * out_ids[b];
            double d2 = 0;
            for (int x = 0; x < ndim; ++x) d2 += (ca[x] - cb[x]) * (ca[x] - cb[x]);
            double lim = rho * (ca[3] > cb[3] ? ca[3] : cb[3]);
            if (sqrt(d2) < lim) overlap = 1;
        }
        if (!overlap) out_ids[kept++] = keys[a].id;
    }
    free(keys);
    return kept;
}

/* ------------------------------------------------------------------------- */
/* Batch helpers for the tests (plain loops over the functions above)       */
/* ------------------------------------------------------------------------- */
void or_philox_batch(int64_t n, const uint32_t *ctrs, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) or_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

void or_weight_batch(int ndim, int64_t n, const double *r, double R, double dR, double *out)
{
    for (int64_t i = 0; i < n; ++i) or_weight(ndim, r[i], R, dR, out + 3 * i);
}

void or_image_values(const or_image *img, int64_t n, const double *x, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_image_value(img, x + 3 * i);
}

/* The first N unit-ball (or disk) sample points of contour k at iteration `iter`,
 * drawn exactly as or_eval_pq draws them. */
void or_unit_samples(const or_params *P, int64_t iter, int64_t k, double *out)
{
    word_stream S = {-1, {0, 0, 0, 0}};
    uint32_t w[2];
    for (int64_t j = 0; j < P->N; ++j) {
        sample_words(P, &S, j, iter, k, w);
        or_unit_sample(P->ndim, w, out + 3 * j);
    }
}

/* Teacher-forced evaluation of many (state, iteration, contour) triples: rows of
 * `cR` are (cx, cy, cz, R), `iters` and `ks` give n and k; writes OR_RES_LEN doubles
 * per row.  Independent rows are spread over `nthreads` OpenMP threads. */
void or_eval_many(const or_image *img, const or_params *P, int64_t m, const double *cR, const int64_t *iters,
                  const int64_t *ks, double *res, int nthreads)
{
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (int64_t i = 0; i < m; ++i)
        or_eval_cr(img, P, cR + 4 * i, cR[4 * i + 3], iters[i], ks[i], res + (int64_t)OR_RES_LEN * i);
}
