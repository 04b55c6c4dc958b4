/*
 * das_oracle.c -- plain FP64 CPU oracle for plane-wave delay-and-sum (DAS)
 * beamforming of baseband IQ data, coherent compounding and ensemble Power Doppler.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference the CUDA library
 * is compared against.  Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It shares
 * no header, helper, table or constant with the CUDA library.
 *
 * What it computes (paper Sec. 2.1, the three DAS steps; Eq. 1 counts the points):
 *   for every voxel v and frame f
 *     y[v][f] = sum_t sum_c  a(v,c) * exp(+j 2 pi fc (t0 + s/fs)) * lerp(iq[t][c][.][f], s)
 *     s       = s_tx(t,v) + s_rx(v,c)                         (delay in samples)
 *     s_tx    = ((u_t . p_v)/c - t0) * fs                      (plane-wave arrival)
 *     s_rx    = |p_v - e_c| * fs / c                           (receive path)
 *     lerp(x, s) = (1-w) x[i0] + w x[i0+1],  i0 = floor(s), w = s - i0,
 *                  and 0 unless 0 <= i0 <= S-2                  (Sec. 4.1: linear interp.)
 *     a(v,c)  = F-number aperture window (Sec. 4.1, "f-number")
 *   Power Doppler (Sec. 5):  P[v] = sum_f |y[v][f]|^2.
 * Hybrid delays (Sec. 4.3: transmit arrival precomputed per voxel, receive delay per
 * element) change nothing in the result; the oracle simply evaluates the sum.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R2 plane-wave time zero: the wavefront passes the array origin at t = 0; sample n
 *      is at t0 + n/fs.  u = (sin az cos el, sin el, cos az cos el).
 *   R4 baseband rotation: IQ = LPF{RF e^{-j 2 pi fc t}}, so the beamformer rotates by
 *      e^{+j 2 pi fc (t0 + s/fs)}.
 *   R5 out of range: a tap pair contributes only if 0 <= i0 and i0 + 1 <= S - 1.
 *   R6 aperture: rho = lateral distance (|dx| in 2D, sqrt(dx^2+dy^2) in 3D); the element
 *      contributes iff dz > 0 and rho * 2 F# <= dz (apod "none": always).  Windows of
 *      t = rho F# / dz in [0, 1/2]: boxcar 1, Hann cos^2(pi t), Gaussian exp(-8 t^2).
 *      No normalisation.
 *   R7 no spreading loss, no element directivity.
 *   R1 two delay modes:
 *      exact    -- every step in FP64 (the physics definition);
 *      contract -- the delay/index steps in the float32 precision of the paper's
 *                  arrays (Table 3: float32 coordinates and arrival times), with this
 *                  fixed sequence: coordinates scaled by fs/c in FP64 then rounded to
 *                  float; s_tx = RN_float(fma(ux,px, fma(uy,py, uz*pz)) * fs/c - t0 fs)
 *                  in FP64; rx = sqrtf(fmaf(dx,dx, fmaf(dy,dy, dz*dz))); s = s_tx + rx;
 *                  i0 = floorf(s); w = s - i0; aperture test in float, squared:
 *                  fmaf(dx,dx, dy*dy) * RN_float(4 F#^2) <= dz*dz (and dz > 0).  Everything
 *                  after the index (window value, phase, interpolation, sums) is FP64.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared  (no fast-math: the float
 * steps of the contract mode must round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_APOD_NONE 0
#define OR_APOD_BOXCAR 1
#define OR_APOD_HANN 2
#define OR_APOD_GAUSS 3

typedef struct {
    int32_t ndim, n_elem, n_tx, n_samples, n_frames, apod, mode, pad_;
    int64_t n_vox;
    const float *elem_pos;      /* [n_elem][3] metres                              */
    const float *vox_pos;       /* [n_vox][3] metres, or NULL: regular grid below   */
    int32_t grid_dims[3], pad2_;
    double grid_origin[3], grid_step[3];
    const double *tx_angles;    /* [n_tx][2] (azimuth, elevation) radians           */
    const float *tx_arrival;    /* [n_tx][n_vox] arrival times in s, or NULL        */
    double fs, fc, c, t0, f_number;
} oracle_desc;

/* one (voxel, element, transmit) term, before the frame loop */
typedef struct {
    int valid;      /* R5 range test and R6 aperture test both passed */
    int in_aperture;
    int64_t i0;
    double s;       /* delay in samples (float value widened, in contract mode) */
    double w;       /* interpolation weight s - i0 */
    double a;       /* aperture window value */
    double re, im;  /* a * exp(+j 2 pi fc (t0 + s/fs)) */
} term_t;

/* ---- geometry ---------------------------------------------------------- */

/* voxel centre in metres: explicit list, or origin + index * step (x fastest) */
static void voxel_position(const oracle_desc *d, int64_t v, double p[3])
{
    if (d->vox_pos) {
        for (int k = 0; k < 3; ++k) p[k] = (double)d->vox_pos[3 * v + k];
        return;
    }
    int64_t nx = d->grid_dims[0], ny = d->grid_dims[1];
    int64_t ix = v % nx, iy = (v / nx) % ny, iz = v / (nx * ny);
    p[0] = d->grid_origin[0] + (double)ix * d->grid_step[0];
    p[1] = d->grid_origin[1] + (double)iy * d->grid_step[1];
    p[2] = d->grid_origin[2] + (double)iz * d->grid_step[2];
}

/* plane-wave propagation direction for transmit t (reading R2) */
static void tx_direction(const oracle_desc *d, int t, double u[3])
{
    double az = d->tx_angles[2 * t], el = d->tx_angles[2 * t + 1];
    u[0] = sin(az) * cos(el);
    u[1] = sin(el);
    u[2] = cos(az) * cos(el);
}

/* ---- transmit delay (Sec. 4.3: the precomputed per-voxel arrival time) ---- */

static double tx_samples_exact(const oracle_desc *d, int t, int64_t v, const double p[3])
{
    if (d->tx_arrival)
        return ((double)d->tx_arrival[(int64_t)t * d->n_vox + v] - d->t0) * d->fs;
    double u[3];
    tx_direction(d, t, u);
    return ((u[0] * p[0] + u[1] * p[1] + u[2] * p[2]) / d->c - d->t0) * d->fs;
}

static float tx_samples_contract(const oracle_desc *d, int t, int64_t v, const double p[3])
{
    double t0fs = d->t0 * d->fs;
    if (d->tx_arrival)
        return (float)fma((double)d->tx_arrival[(int64_t)t * d->n_vox + v], d->fs, -t0fs);
    double u[3];
    tx_direction(d, t, u);
    double k = d->fs / d->c;
    double dot = fma(u[0], p[0], fma(u[1], p[1], u[2] * p[2]));
    return (float)fma(dot, k, -t0fs);
}

/* ---- aperture window (reading R6), t = rho * F# / dz in [0, 1/2] ---------- */

static double window_value(int apod, double t)
{
    switch (apod) {
    case OR_APOD_HANN: { double cp = cos(M_PI * t); return cp * cp; }
    case OR_APOD_GAUSS: return exp(-8.0 * t * t);
    default: return 1.0;
    }
}

/* ---- one term (v, c, t) ------------------------------------------------ */

static void make_term(const oracle_desc *d, int64_t v, int c, int t, const double p[3], term_t *o)
{
    const float *e = d->elem_pos + 3 * (int64_t)c;
    double s, rho, dz;
    int in_ap;
    if (d->mode == 0) {                         /* exact: all FP64 */
        double dx = p[0] - (double)e[0], dy = p[1] - (double)e[1];
        dz = p[2] - (double)e[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        s = tx_samples_exact(d, t, v, p) + r * d->fs / d->c;
        rho = sqrt(dx * dx + dy * dy);
        in_ap = (d->apod == OR_APOD_NONE) || (dz > 0.0 && rho * 2.0 * d->f_number <= dz);
    } else {                                    /* contract: float32 delay sequence */
        double k = d->fs / d->c;
        float vx = (float)(p[0] * k), vy = (float)(p[1] * k), vz = (float)(p[2] * k);
        float ex = (float)((double)e[0] * k), ey = (float)((double)e[1] * k),
              ez = (float)((double)e[2] * k);
        float fdx = vx - ex, fdy = vy - ey, fdz = vz - ez;
        float rx = sqrtf(fmaf(fdx, fdx, fmaf(fdy, fdy, fdz * fdz)));
        float fs_ = tx_samples_contract(d, t, v, p) + rx;
        /* aperture test squared (rho*2F# <= dz  <=>  rho^2 * 4F#^2 <= dz^2 for dz > 0) */
        float frho2 = fmaf(fdx, fdx, fdy * fdy);
        float four_f2 = (float)(4.0 * d->f_number * d->f_number);
        in_ap = (d->apod == OR_APOD_NONE) || (fdz > 0.0f && frho2 * four_f2 <= fdz * fdz);
        s = (double)fs_;
        rho = sqrt((double)frho2);
        dz = (double)fdz;
    }
    o->s = s;
    o->in_aperture = in_ap;
    double fl = floor(s);
    /* R5: 0 <= i0 <= S-2  <=>  0 <= s < S-1 */
    int in_range = (s >= 0.0) && (s < (double)(d->n_samples - 1));
    o->valid = in_ap && in_range;
    o->i0 = in_range ? (int64_t)fl : -1;
    o->w = s - fl;
    o->a = 0.0;
    o->re = o->im = 0.0;
    if (!o->valid) return;
    double tt = (d->apod == OR_APOD_NONE || dz <= 0.0) ? 0.0 : rho * d->f_number / dz;
    o->a = window_value(d->apod, tt);
    double phase = 2.0 * M_PI * (d->fc * d->t0 + s * d->fc / d->fs);   /* R4 */
    o->re = o->a * cos(phase);
    o->im = o->a * sin(phase);
}

/* ---- public entry points ----------------------------------------------- */

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * y[n][F] (complex, interleaved re/im, FP64) and pd[n] for the voxels vox_idx[0..n-1].
 * iq: complex64 [T][C][S][F] interleaved.  Either output may be NULL.
 */
int oracle_das(const oracle_desc *d, const float *iq, const int64_t *vox_idx, int64_t n,
               double *y, double *pd, int nthreads)
{
    if (!d || !iq || !vox_idx || n < 0) return 1;
    set_threads(nthreads);
    const int T = d->n_tx, C = d->n_elem, F = d->n_frames;
    const int64_t S = d->n_samples;
    int64_t j;
#pragma omp parallel for schedule(dynamic, 16)
    for (j = 0; j < n; ++j) {
        int64_t v = vox_idx[j];
        double p[3];
        voxel_position(d, v, p);
        double *acc = (double *)calloc((size_t)2 * F, sizeof(double));
        for (int t = 0; t < T; ++t) {
            for (int c = 0; c < C; ++c) {
                term_t tm;
                make_term(d, v, c, t, p, &tm);
                if (!tm.valid) continue;
                const float *x0 = iq + (((int64_t)t * C + c) * S + tm.i0) * F * 2;
                const float *x1 = x0 + (int64_t)F * 2;
                for (int f = 0; f < F; ++f) {
                    double lr = (1.0 - tm.w) * (double)x0[2 * f] + tm.w * (double)x1[2 * f];
                    double li = (1.0 - tm.w) * (double)x0[2 * f + 1] + tm.w * (double)x1[2 * f + 1];
                    acc[2 * f] += tm.re * lr - tm.im * li;
                    acc[2 * f + 1] += tm.re * li + tm.im * lr;
                }
            }
        }
        double pw = 0.0;
        for (int f = 0; f < F; ++f) pw += acc[2 * f] * acc[2 * f] + acc[2 * f + 1] * acc[2 * f + 1];
        if (y) memcpy(y + (size_t)j * 2 * F, acc, sizeof(double) * 2 * F);
        if (pd) pd[j] = pw;
        free(acc);
    }
    return 0;
}

/*
 * Per-term records for the voxels vox_idx[0..n-1], layout [n][C][T]:
 * i0 (-1 when out of range), valid (R5 and R6), w, s, window value, complex weight.
 * Any output may be NULL.
 */
int oracle_terms(const oracle_desc *d, const int64_t *vox_idx, int64_t n, int64_t *i0,
                 uint8_t *valid, double *w, double *s, double *a, double *cw, int nthreads)
{
    if (!d || !vox_idx || n < 0) return 1;
    set_threads(nthreads);
    const int T = d->n_tx, C = d->n_elem;
    int64_t j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < n; ++j) {
        double p[3];
        voxel_position(d, vox_idx[j], p);
        for (int c = 0; c < C; ++c)
            for (int t = 0; t < T; ++t) {
                term_t tm;
                make_term(d, vox_idx[j], c, t, p, &tm);
                int64_t o = (j * C + c) * T + t;
                if (i0) i0[o] = tm.i0;
                if (valid) valid[o] = (uint8_t)tm.valid;
                if (w) w[o] = tm.w;
                if (s) s[o] = tm.s;
                if (a) a[o] = tm.a;
                if (cw) { cw[2 * o] = tm.re; cw[2 * o + 1] = tm.im; }
            }
    }
    return 0;
}

/* Contract-mode transmit table, float [T][V] in samples (Sec. 4.3 precompute). */
int oracle_tx_table(const oracle_desc *d, float *out)
{
    if (!d || !out) return 1;
    int64_t V = d->n_vox;
    int64_t v;
#pragma omp parallel for schedule(static)
    for (v = 0; v < V; ++v) {
        double p[3];
        voxel_position(d, v, p);
        for (int t = 0; t < d->n_tx; ++t) out[(int64_t)t * V + v] = tx_samples_contract(d, t, v, p);
    }
    return 0;
}

/* Exact-mode transmit delay in samples, double [T][n] for the listed voxels. */
int oracle_tx_exact(const oracle_desc *d, const int64_t *vox_idx, int64_t n, double *out)
{
    if (!d || !vox_idx || !out) return 1;
    for (int64_t j = 0; j < n; ++j) {
        double p[3];
        voxel_position(d, vox_idx[j], p);
        for (int t = 0; t < d->n_tx; ++t) out[(int64_t)t * n + j] = tx_samples_exact(d, t, vox_idx[j], p);
    }
    return 0;
}
