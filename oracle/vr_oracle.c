/*
 * vr_oracle.c -- plain FP64 CPU ray caster: the definition the CUDA path is
 * checked against.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark may load this library.  It shares no code, header,
 * table or constant with the CUDA library; it is deliberately slow and written
 * for a reader to check against the paper by eye.
 *
 * What it computes (Hassan et al. 2012, Section 3.3 "Transfer functions",
 * 3.3.2 "Generic transfer function volume rendering", 3.4 "The frame
 * composition processes", and the constant-step trilinear sampling of
 * Section 4.4 "3D spectrum tool"): one ray per output pixel is clipped to the
 * volume box and sampled at a constant step; each sample is the trilinear
 * interpolation of the grid, mapped through a discrete RGBA transfer function
 * (colour plus an opacity in [0,1] per data level), and the samples are merged
 * front to back with the "over" operator (emission-absorption model of
 * Levoy 1988, which the paper cites).  Early ray termination is not in the
 * paper; it is a stated extension: stop after the sample at which the
 * accumulated opacity reaches the threshold.
 *
 * Readings where the paper is silent (all of them documented with the build):
 *   - camera: f = normalize(forward), r = normalize(f x up), u = r x f; pixel
 *     centres at +1/2; row 0 is the top (+u); aspect = W/H.  Orthographic rays
 *     start on the image plane and are not clipped at t = 0; perspective rays
 *     start at the eye and keep t >= 0.
 *   - grid: voxel centres at integer indices, box = closed [0, n-1] per axis.
 *   - samples: t_k = t_in + (k + 1/2) * step while t_k <= t_out, i.e.
 *     n = floor((t_out - t_in)/step + 1/2); positions are o + t_k d, never
 *     accumulated.  The step is in world units along the unit direction.
 *   - trilinear: cell origin i0 = clamp(floor(x), 0, n-2), weight x - i0.
 *   - transfer function: u = clamp((v - vmin)/(vmax - vmin), 0, 1) * (K-1),
 *     i0 = min(floor(u), K-2), w = u - i0, linear blend of entries i0, i0+1;
 *     entries are straight (not premultiplied) RGBA; no opacity correction.
 *   - composite: C += T a c; T *= (1 - a); stop after the sample once
 *     1 - T >= thr (thr > 1 disables); output (C + T bg.rgb, 1 - T + T bg.a).
 *
 * The backward pass is plain reverse-mode differentiation of that forward
 * definition: every sample of a ray is stored, then the ray is walked back to
 * front with suffix accumulators (no division by transmittance), followed by
 * the chain rule through the transfer-function blend and the trilinear
 * weights.
 *
 * The same ray also serves the paper's other tools (end of this file): the
 * 3D spectrum tool of Section 4.4 (the values along one pixel's line of
 * sight), maximum intensity projection (Section 3.3.1) and the
 * sigma-clipping transfer function of Section 4.5 (sample values scaled by
 * the statistics of a mini-map of region means and standard deviations), and
 * the global statistics of Sections 4.1-4.3 (histogram, mean and standard
 * deviation, Torben's median as the appendix gives it).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Types (this file's own; nothing is shared with the CUDA library)          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;                 /* 0 orthographic, 1 perspective */
    double eye[3];
    double forward[3];
    double up[3];
    double fov_y_deg;         /* perspective: full vertical field of view */
    double ortho_height;      /* orthographic: world height of the image */
    int width, height;
} orc_camera;

typedef struct {
    const void *data;         /* dense, x fastest then y then z */
    int dtype;                /* 0 float32, 1 float64, 2 binary16 bits, 3 bfloat16 bits */
    int64_t n[3];             /* nx, ny, nz (each >= 2) */
    double origin[3];         /* world position of voxel (0,0,0) */
    double spacing[3];        /* world size of one voxel step per axis */
} orc_volume;

typedef struct {
    const double *tf;         /* K x 4 straight RGBA */
    int K;
    double vmin, vmax;
    double step;              /* world units, > 0 */
    double ert;               /* early-termination opacity; > 1 disables */
    double bg[4];             /* background RGBA */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Voxel access (exact widening of the stored value)                         */
/* ------------------------------------------------------------------------ */

static double half_bits_to_double(uint16_t h)
{
    /* IEEE 754 binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits. */
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double mag;
    if (e == 0)
        mag = ldexp((double)m, -24);                  /* subnormal: m * 2^-24 */
    else if (e == 31)
        mag = m ? NAN : INFINITY;
    else
        mag = ldexp((double)(1024 + m), e - 25);      /* (1 + m/1024) * 2^(e-15) */
    return s ? -mag : mag;
}

static double bf16_bits_to_double(uint16_t b)
{
    /* bfloat16 is the upper half of an IEEE binary32. */
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

static double voxel_at(const orc_volume *v, int64_t x, int64_t y, int64_t z)
{
    int64_t i = (z * v->n[1] + y) * v->n[0] + x;
    switch (v->dtype) {
    case 0: return (double)((const float *)v->data)[i];
    case 1: return ((const double *)v->data)[i];
    case 2: return half_bits_to_double(((const uint16_t *)v->data)[i]);
    default: return bf16_bits_to_double(((const uint16_t *)v->data)[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Camera (per pixel ray in world space)                                     */
/* ------------------------------------------------------------------------ */

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void normalize3(double a[3])
{
    double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

typedef struct { double f[3], r[3], u[3]; } basis;

static basis camera_basis(const orc_camera *c)
{
    basis b;
    memcpy(b.f, c->forward, sizeof b.f);
    normalize3(b.f);
    cross3(b.f, c->up, b.r);
    normalize3(b.r);
    cross3(b.r, b.f, b.u);
    return b;
}

/* Ray through the centre of pixel (i, j): origin o and unit direction d. */
static void pixel_ray(const orc_camera *c, const basis *b, int i, int j, double o[3], double d[3])
{
    double sx = ((i + 0.5) / c->width) * 2.0 - 1.0;
    double sy = 1.0 - ((j + 0.5) / c->height) * 2.0;
    double aspect = (double)c->width / (double)c->height;
    if (c->kind == 0) {
        double hh = 0.5 * c->ortho_height;
        for (int a = 0; a < 3; ++a) {
            o[a] = c->eye[a] + sx * hh * aspect * b->r[a] + sy * hh * b->u[a];
            d[a] = b->f[a];
        }
    } else {
        double th = tan(c->fov_y_deg * M_PI / 360.0);   /* tan(fov/2) */
        for (int a = 0; a < 3; ++a) {
            o[a] = c->eye[a];
            d[a] = b->f[a] + sx * th * aspect * b->r[a] + sy * th * b->u[a];
        }
        normalize3(d);
    }
}

/* ------------------------------------------------------------------------ */
/* Box clipping (slab method) in voxel coordinates                           */
/* ------------------------------------------------------------------------ */

/* p_vox(t) = ov + t * dv, t in world units along the unit world direction.
 * Returns 1 and [t_in, t_out] when the ray meets the closed box [0, n-1]^3
 * over an interval of positive length, else 0. */
static int clip_box(const orc_volume *v, int perspective, const double ov[3], const double dv[3],
                    double *t_in, double *t_out)
{
    double tin = perspective ? 0.0 : -INFINITY, tout = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = 0.0, hi = (double)(v->n[a] - 1);
        if (dv[a] == 0.0) {
            if (ov[a] < lo || ov[a] > hi) return 0;   /* parallel and outside */
            continue;                                   /* parallel and inside */
        }
        double t0 = (lo - ov[a]) / dv[a], t1 = (hi - ov[a]) / dv[a];
        if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
        if (t0 > tin) tin = t0;
        if (t1 < tout) tout = t1;
    }
    *t_in = tin;
    *t_out = tout;
    return tin < tout;
}

/* ------------------------------------------------------------------------ */
/* Trilinear interpolation and transfer function                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t idx[8];           /* dense voxel indices of the 8 corners */
    double wt[8];             /* their trilinear weights */
} corners;

static double trilinear(const orc_volume *v, const double p[3], corners *cs)
{
    int64_t c0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        int64_t i0 = (int64_t)fl;
        if (i0 < 0) i0 = 0;
        if (i0 > v->n[a] - 2) i0 = v->n[a] - 2;
        c0[a] = i0;
        fr[a] = p[a] - (double)i0;
    }
    double val = 0.0;
    int k = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx, ++k) {
                double w = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1]) *
                           (dz ? fr[2] : 1.0 - fr[2]);
                int64_t x = c0[0] + dx, y = c0[1] + dy, z = c0[2] + dz;
                if (cs) {
                    cs->idx[k] = (z * v->n[1] + y) * v->n[0] + x;
                    cs->wt[k] = w;
                }
                val += w * voxel_at(v, x, y, z);
            }
    return val;
}

typedef struct {
    int i0;                   /* lower table entry */
    double w;                 /* blend weight of entry i0+1 */
    int interior;             /* vmin < v < vmax: the lookup has a slope in v */
} tf_pos;

static void tf_lookup(const orc_params *P, double v, double rgba[4], tf_pos *pos)
{
    double s = (v - P->vmin) / (P->vmax - P->vmin);
    int interior = (s > 0.0 && s < 1.0);
    if (!(s > 0.0)) s = 0.0;                 /* also maps NaN to the low end */
    if (s > 1.0) s = 1.0;
    double u = s * (P->K - 1);
    int i0 = (int)floor(u);
    if (i0 > P->K - 2) i0 = P->K - 2;
    double w = u - i0;
    for (int ch = 0; ch < 4; ++ch)
        rgba[ch] = (1.0 - w) * P->tf[4 * i0 + ch] + w * P->tf[4 * (i0 + 1) + ch];
    if (pos) { pos->i0 = i0; pos->w = w; pos->interior = interior; }
}

/* ------------------------------------------------------------------------ */
/* Per-ray forward                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double ov[3], dv[3];      /* ray in voxel coordinates */
    double t_in;
    int64_t n;                /* samples on the clipped ray (before early termination) */
    double margin_n;          /* distance of (t_out-t_in)/step + 1/2 to the nearest integer */
} ray_setup;

static void setup_ray(const orc_volume *v, const orc_camera *c, const basis *b, const orc_params *P,
                      int i, int j, ray_setup *rs)
{
    double o[3], d[3];
    pixel_ray(c, b, i, j, o, d);
    for (int a = 0; a < 3; ++a) {
        rs->ov[a] = (o[a] - v->origin[a]) / v->spacing[a];
        rs->dv[a] = d[a] / v->spacing[a];
    }
    double tin, tout;
    if (!clip_box(v, c->kind == 1, rs->ov, rs->dv, &tin, &tout)) {
        rs->n = 0;
        rs->t_in = 0.0;
        rs->margin_n = INFINITY;
        return;
    }
    double q = (tout - tin) / P->step + 0.5;
    rs->n = (int64_t)floor(q);
    rs->margin_n = fabs(q - floor(q + 0.5));
    rs->t_in = tin;
}

static void sample_pos(const ray_setup *rs, const orc_params *P, int64_t k, double p[3])
{
    double t = rs->t_in + ((double)k + 0.5) * P->step;
    for (int a = 0; a < 3; ++a) p[a] = rs->ov[a] + t * rs->dv[a];
}

/* Renders pixel (i, j); writes RGBA, the number of composited samples and the
 * two decision margins (sample count, early termination). */
static void render_pixel(const orc_volume *v, const orc_camera *c, const basis *b, const orc_params *P,
                         int i, int j, double out[4], int32_t *n_used, double *m_n, double *m_ert)
{
    ray_setup rs;
    setup_ray(v, c, b, P, i, j, &rs);
    double C[3] = {0.0, 0.0, 0.0}, T = 1.0, mert = INFINITY;
    int64_t used = 0;
    for (int64_t k = 0; k < rs.n; ++k) {
        double p[3], rgba[4];
        sample_pos(&rs, P, k, p);
        double val = trilinear(v, p, NULL);
        tf_lookup(P, val, rgba, NULL);
        double a = rgba[3];
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * rgba[ch];
        T *= (1.0 - a);
        used = k + 1;
        double opacity = 1.0 - T;
        if (P->ert <= 1.0) {
            double m = fabs(opacity - P->ert);
            if (m < mert) mert = m;
        }
        if (opacity >= P->ert) break;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * P->bg[ch];
    out[3] = 1.0 - T + T * P->bg[3];
    if (n_used) *n_used = (int32_t)used;
    if (m_n) *m_n = rs.margin_n;
    if (m_ert) *m_ert = mert;
}

/* ------------------------------------------------------------------------ */
/* Threaded driver over image rows                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_volume *v;
    const orc_camera *c;
    const orc_params *P;
    basis b;
    int row0, row1, stride, first;
    double *rgba;             /* H*W*4 */
    int32_t *n_used;          /* H*W or NULL */
    double *margin_n;         /* H*W or NULL */
    double *margin_ert;       /* H*W or NULL */
    /* backward */
    const double *grad_rgba;
    double *grad_tf;          /* private K*4 */
    double *grad_vox;         /* private nx*ny*nz or NULL */
    double *kink_vox;         /* private nx*ny*nz or NULL: see orc_render_backward_kinks */
    double *mag_vox;          /* private nx*ny*nz or NULL: see orc_render_backward_kinks */
    double kink_eps;          /* table-coordinate distance that counts as "at a kink" */
} job;

/* Pixels of rows [row0, row1) are dealt to the threads round-robin. */
static void *fwd_worker(void *arg)
{
    job *J = (job *)arg;
    int W = J->c->width;
    int64_t first = (int64_t)J->row0 * W, last = (int64_t)J->row1 * W;
    for (int64_t px = first + J->first; px < last; px += J->stride) {
        int j = (int)(px / W), i = (int)(px % W);
        render_pixel(J->v, J->c, &J->b, J->P, i, j, J->rgba + 4 * px,
                     J->n_used ? J->n_used + px : NULL, J->margin_n ? J->margin_n + px : NULL,
                     J->margin_ert ? J->margin_ert + px : NULL);
    }
    return NULL;
}

static int run_threads(job *jobs, int nthreads, void *(*fn)(void *))
{
    if (nthreads <= 1) {
        fn(&jobs[0]);
        return 0;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -3;
    int started = 0, rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) { rc = -3; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    for (int t = started; t < nthreads && rc == 0; ++t) fn(&jobs[t]);
    free(th);
    return rc;
}

static int check_args(const orc_volume *v, const orc_camera *c, const orc_params *P)
{
    if (!v || !c || !P || !v->data || !P->tf) return -1;
    for (int a = 0; a < 3; ++a)
        if (v->n[a] < 2 || !(v->spacing[a] > 0.0)) return -1;
    if (c->width <= 0 || c->height <= 0 || P->K < 2 || !(P->step > 0.0) || !(P->vmax > P->vmin)) return -1;
    if (c->kind != 0 && c->kind != 1) return -1;
    return 0;
}

/* Forward render of rows [row0, row1) of the image.  Outputs are indexed by
 * the full image (row j, column i at j*W + i); rows outside the range are not
 * touched.  Returns 0, or -1 on invalid arguments. */
int orc_render(const orc_volume *v, const orc_camera *c, const orc_params *P, int row0, int row1,
               double *rgba, int32_t *n_used, double *margin_n, double *margin_ert, int nthreads)
{
    if (check_args(v, c, P) || !rgba) return -1;
    if (row0 < 0) row0 = 0;
    if (row1 > c->height) row1 = c->height;
    if (nthreads < 1) nthreads = 1;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    if (!jobs) return -3;
    basis b = camera_basis(c);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].v = v; jobs[t].c = c; jobs[t].P = P; jobs[t].b = b;
        jobs[t].row0 = row0; jobs[t].row1 = row1; jobs[t].stride = nthreads; jobs[t].first = t;
        jobs[t].rgba = rgba; jobs[t].n_used = n_used;
        jobs[t].margin_n = margin_n; jobs[t].margin_ert = margin_ert;
    }
    int rc = run_threads(jobs, nthreads, fwd_worker);
    free(jobs);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Backward: store-all reverse mode, back to front                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    double val;               /* interpolated sample value */
    double rgba[4];
    double T;                 /* transmittance in front of the sample */
    tf_pos pos;
    corners cs;
} stored_sample;

static void backward_pixel(job *J, int i, int j, stored_sample **buf, int64_t *cap)
{
    const orc_volume *v = J->v;
    const orc_params *P = J->P;
    ray_setup rs;
    setup_ray(v, J->c, &J->b, P, i, j, &rs);
    if (rs.n <= 0) return;
    if (rs.n > *cap) {
        free(*buf);
        *cap = rs.n;
        *buf = (stored_sample *)malloc(sizeof(stored_sample) * (size_t)rs.n);
    }
    stored_sample *S = *buf;

    /* Forward, storing every composited sample. */
    double T = 1.0;
    int64_t used = 0;
    for (int64_t k = 0; k < rs.n; ++k) {
        double p[3];
        sample_pos(&rs, P, k, p);
        double val = trilinear(v, p, &S[k].cs);
        tf_lookup(P, val, S[k].rgba, &S[k].pos);
        S[k].val = val;
        S[k].T = T;
        T *= (1.0 - S[k].rgba[3]);
        used = k + 1;
        if (1.0 - T >= P->ert) break;
    }

    /* Output I = (C + T_n bg.rgb, 1 - T_n (1 - bg.a)).  With g = dL/dI.rgb and
     * gA = dL/dI.a the loss reacts to C through g and to T_n through gT. */
    const double *gI = J->grad_rgba + 4 * ((int64_t)j * J->c->width + i);
    double g[3] = {gI[0], gI[1], gI[2]};
    double gT = g[0] * P->bg[0] + g[1] * P->bg[1] + g[2] * P->bg[2] - gI[3] * (1.0 - P->bg[3]);

    /* Suffix accumulators normalised to the transmittance behind sample k:
     * Ssuf = sum_{j>k} (T_j / T_{k+1}) a_j (c_j . g),  Psuf = T_n / T_{k+1}. */
    double Ssuf = 0.0, Psuf = 1.0;
    double scale = (double)(P->K - 1) / (P->vmax - P->vmin);
    for (int64_t k = used - 1; k >= 0; --k) {
        const stored_sample *s = &S[k];
        double a = s->rgba[3];
        double cg = s->rgba[0] * g[0] + s->rgba[1] * g[1] + s->rgba[2] * g[2];
        double dr[4];
        for (int ch = 0; ch < 3; ++ch) dr[ch] = s->T * a * g[ch];     /* dL/dc_k */
        dr[3] = s->T * (cg - Ssuf - gT * Psuf);                        /* dL/da_k */
        const double Ssuf_k = Ssuf, Psuf_k = Psuf;                      /* behind sample k */
        Ssuf = a * cg + (1.0 - a) * Ssuf;
        Psuf = (1.0 - a) * Psuf;

        int i0 = s->pos.i0;
        double w = s->pos.w;
        double dv = 0.0;
        for (int ch = 0; ch < 4; ++ch) {
            J->grad_tf[4 * i0 + ch] += (1.0 - w) * dr[ch];
            J->grad_tf[4 * (i0 + 1) + ch] += w * dr[ch];
            dv += dr[ch] * (P->tf[4 * (i0 + 1) + ch] - P->tf[4 * i0 + ch]);
        }
        if (J->grad_vox && s->pos.interior) {
            dv *= scale;
            for (int q = 0; q < 8; ++q) J->grad_vox[s->cs.idx[q]] += s->cs.wt[q] * dv;
        }
        if (J->mag_vox && s->pos.interior) {
            /* the magnitudes that make up this sample's voxel term before any
             * cancellation: |dL/dc| |dc/dv| per colour channel and, for the
             * opacity, T (|c.g| + |suffix colour| + |suffix transmittance term|) |da/dv| */
            double mag = 0.0;
            for (int ch = 0; ch < 3; ++ch)
                mag += fabs(dr[ch]) * fabs(P->tf[4 * (i0 + 1) + ch] - P->tf[4 * i0 + ch]);
            mag += s->T * (fabs(cg) + fabs(Ssuf_k) + fabs(gT * Psuf_k)) * fabs(P->tf[4 * (i0 + 1) + 3] - P->tf[4 * i0 + 3]);
            mag *= scale;
            for (int q = 0; q < 8; ++q) J->mag_vox[s->cs.idx[q]] += s->cs.wt[q] * mag;
        }
        if (J->kink_vox) {
            /* The voxel gradient uses the slope of the table interval that holds
             * u = (v - vmin)/(vmax - vmin) (K-1).  Within kink_eps of an interval
             * end the interval is decided by rounding: the other side's slope
             * (or no slope past vmin / vmax) is an equally valid one-sided
             * derivative.  The largest change of this sample's voxel term that
             * such a choice makes is added to its eight corners' bound. */
            double u = (s->val - P->vmin) / (P->vmax - P->vmin) * (P->K - 1);   /* unclamped */
            double alt = -1.0;            /* |dv| change, or < 0 when not at a kink */
            double m = floor(u + 0.5);    /* nearest interval end */
            if (fabs(u - m) < J->kink_eps && m >= 0.0 && m <= (double)(P->K - 1)) {
                int mi = (int)m;
                int ci = s->pos.interior ? i0 : -1;   /* interval of the chosen slope; -1: none */
                int oi;                               /* interval on the other side of end m */
                if (!s->pos.interior) oi = mi == 0 ? 0 : P->K - 2;
                else if (mi == i0) oi = mi - 1;       /* u at or just above m */
                else oi = mi;                         /* u just below m */
                if (oi > P->K - 2) oi = -1;           /* past vmax: no slope */
                double cur = 0.0, oth = 0.0;
                for (int ch = 0; ch < 4; ++ch) {
                    if (ci >= 0) cur += dr[ch] * (P->tf[4 * (ci + 1) + ch] - P->tf[4 * ci + ch]);
                    if (oi >= 0) oth += dr[ch] * (P->tf[4 * (oi + 1) + ch] - P->tf[4 * oi + ch]);
                }
                alt = fabs(oth - cur) * scale;
            }
            if (alt > 0.0)
                for (int q = 0; q < 8; ++q) J->kink_vox[s->cs.idx[q]] += s->cs.wt[q] * alt;
        }
    }
}

static void *bwd_worker(void *arg)
{
    job *J = (job *)arg;
    stored_sample *buf = NULL;
    int64_t cap = 0;
    int W = J->c->width;
    int64_t first = (int64_t)J->row0 * W, last = (int64_t)J->row1 * W;
    for (int64_t px = first + J->first; px < last; px += J->stride)
        backward_pixel(J, (int)(px % W), (int)(px / W), &buf, &cap);
    free(buf);
    return NULL;
}

/* Gradients of L with respect to the K x 4 table and (optionally) the dense
 * voxels, given dL/dI (H*W*4), over the pixels of rows [row0, row1).  Both outputs are overwritten.  Per-thread
 * partial sums are added in thread order, so the result is deterministic for
 * a given thread count. */
int orc_render_backward_kinks(const orc_volume *v, const orc_camera *c, const orc_params *P, int row0, int row1,
                              const double *grad_rgba, double *grad_tf, double *grad_vox, double *kink_vox,
                              double *mag_vox, double kink_eps, int nthreads);

int orc_render_backward(const orc_volume *v, const orc_camera *c, const orc_params *P, int row0, int row1,
                        const double *grad_rgba, double *grad_tf, double *grad_vox, int nthreads)
{
    return orc_render_backward_kinks(v, c, P, row0, row1, grad_rgba, grad_tf, grad_vox, NULL, NULL, 0.0,
                                     nthreads);
}

/* The same, also writing (when kink_vox is not NULL) a per-voxel bound on
 * how far the voxel gradient may move when the table interval of samples
 * within kink_eps (in table entries) of an interval end -- including vmin
 * and vmax -- is decided the other way, as a lower-precision evaluation of
 * the same samples may do: the sum over such samples of the change of their
 * voxel term, weighted like the term itself.  The voxel gradient of a
 * piecewise-linear table is discontinuous at those ends; the bound says how
 * much of a result is decided there rather than by the method.  mag_vox
 * (when not NULL) receives per voxel the sum of the magnitudes that make up
 * its gradient terms before any cancellation (the scale of the rounding
 * error an evaluation in lower precision can make). */
int orc_render_backward_kinks(const orc_volume *v, const orc_camera *c, const orc_params *P, int row0, int row1,
                              const double *grad_rgba, double *grad_tf, double *grad_vox, double *kink_vox,
                              double *mag_vox, double kink_eps, int nthreads)
{
    if (check_args(v, c, P) || !grad_rgba || !grad_tf) return -1;
    if (nthreads < 1) nthreads = 1;
    int64_t nvox = v->n[0] * v->n[1] * v->n[2];
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    if (!jobs) return -3;
    basis b = camera_basis(c);
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].v = v; jobs[t].c = c; jobs[t].P = P; jobs[t].b = b;
        jobs[t].row0 = row0 < 0 ? 0 : row0;
        jobs[t].row1 = row1 > c->height ? c->height : row1;
        jobs[t].stride = nthreads; jobs[t].first = t;
        jobs[t].grad_rgba = grad_rgba;
        jobs[t].grad_tf = (double *)calloc((size_t)P->K * 4, sizeof(double));
        jobs[t].grad_vox = grad_vox ? (double *)calloc((size_t)nvox, sizeof(double)) : NULL;
        jobs[t].kink_vox = kink_vox ? (double *)calloc((size_t)nvox, sizeof(double)) : NULL;
        jobs[t].mag_vox = mag_vox ? (double *)calloc((size_t)nvox, sizeof(double)) : NULL;
        jobs[t].kink_eps = kink_eps;
        if (!jobs[t].grad_tf || (grad_vox && !jobs[t].grad_vox) || (kink_vox && !jobs[t].kink_vox) ||
            (mag_vox && !jobs[t].mag_vox))
            rc = -3;
    }
    if (rc == 0) rc = run_threads(jobs, nthreads, bwd_worker);
    if (rc == 0) {
        memset(grad_tf, 0, sizeof(double) * (size_t)P->K * 4);
        if (grad_vox) memset(grad_vox, 0, sizeof(double) * (size_t)nvox);
        if (kink_vox) memset(kink_vox, 0, sizeof(double) * (size_t)nvox);
        if (mag_vox) memset(mag_vox, 0, sizeof(double) * (size_t)nvox);
        for (int t = 0; t < nthreads; ++t) {
            for (int q = 0; q < P->K * 4; ++q) grad_tf[q] += jobs[t].grad_tf[q];
            if (grad_vox)
                for (int64_t q = 0; q < nvox; ++q) grad_vox[q] += jobs[t].grad_vox[q];
            if (kink_vox)
                for (int64_t q = 0; q < nvox; ++q) kink_vox[q] += jobs[t].kink_vox[q];
            if (mag_vox)
                for (int64_t q = 0; q < nvox; ++q) mag_vox[q] += jobs[t].mag_vox[q];
        }
    }
    for (int t = 0; t < nthreads; ++t) {
        free(jobs[t].grad_tf); free(jobs[t].grad_vox); free(jobs[t].kink_vox); free(jobs[t].mag_vox);
    }
    free(jobs);
    return rc;
}

/* Single-sample probes used by the tests: the trilinear value at a voxel
 * position, and the table lookup of a value. */
double orc_trilinear(const orc_volume *v, const double p[3])
{
    return trilinear(v, p, NULL);
}

void orc_tf_lookup(const orc_params *P, double val, double rgba[4])
{
    tf_lookup(P, val, rgba, NULL);
}

/* Ray setup probe: voxel-space origin/direction, t_in and the sample count of
 * pixel (i, j).  Returns the sample count (0 on a miss). */
int64_t orc_ray(const orc_volume *v, const orc_camera *c, const orc_params *P, int i, int j,
                double ov[3], double dv[3], double *t_in)
{
    basis b = camera_basis(c);
    ray_setup rs;
    setup_ray(v, c, &b, P, i, j, &rs);
    for (int a = 0; a < 3; ++a) { ov[a] = rs.ov[a]; dv[a] = rs.dv[a]; }
    *t_in = rs.t_in;
    return rs.n;
}

/* ======================================================================== */
/* Further uses of the same ray (Sections 3.3.1, 4.4 and 4.5)                */
/* ======================================================================== */

/* ------------------------------------------------------------------------ */
/* 3D spectrum tool (Section 4.4): the data profile along one pixel's line   */
/* of sight, sampled at the renderer's positions with trilinear values.      */
/* ------------------------------------------------------------------------ */

/* Values of the first `max` samples of pixel (i, j)'s clipped ray (no table,
 * no early termination).  Returns the ray's sample count (0 on a miss). */
int64_t orc_profile(const orc_volume *v, const orc_camera *c, const orc_params *P, int i, int j, double *values,
                    int64_t max)
{
    if (check_args(v, c, P)) return -1;
    basis b = camera_basis(c);
    ray_setup rs;
    setup_ray(v, c, &b, P, i, j, &rs);
    for (int64_t k = 0; k < rs.n && k < max; ++k) {
        double p[3];
        sample_pos(&rs, P, k, p);
        values[k] = trilinear(v, p, NULL);
    }
    return rs.n;
}

/* ------------------------------------------------------------------------ */
/* Maximum intensity projection (Section 3.3.1): only the largest value on   */
/* each ray is shown, through the colour map.                                */
/* ------------------------------------------------------------------------ */

/* Reading: the pixel is the table entry of the ray's largest sample value,
 * composited once over the background, (a c + (1 - a) bg.rgb, a + (1 - a)
 * bg.a) -- a one-sample front-to-back composite; a ray that misses the box
 * shows the background.  Every sample of the ray is visited (no early
 * termination). */
static void mip_pixel(const orc_volume *v, const orc_camera *c, const basis *b, const orc_params *P, int i, int j,
                      double out[4], int32_t *n_used, double *vmax)
{
    ray_setup rs;
    setup_ray(v, c, b, P, i, j, &rs);
    double m = -INFINITY;
    for (int64_t k = 0; k < rs.n; ++k) {
        double p[3];
        sample_pos(&rs, P, k, p);
        double val = trilinear(v, p, NULL);
        if (val > m) m = val;
    }
    if (rs.n > 0) {
        double rgba[4];
        tf_lookup(P, m, rgba, NULL);
        double a = rgba[3];
        for (int ch = 0; ch < 3; ++ch) out[ch] = a * rgba[ch] + (1.0 - a) * P->bg[ch];
        out[3] = a + (1.0 - a) * P->bg[3];
    } else {
        for (int ch = 0; ch < 4; ++ch) out[ch] = P->bg[ch];
    }
    if (n_used) *n_used = (int32_t)rs.n;
    if (vmax) *vmax = rs.n > 0 ? m : NAN;
}

/* ------------------------------------------------------------------------ */
/* Sigma-clipping transfer function (Section 4.5): a statistical mini-map    */
/* summarises regions of the cube; each sample value is scaled by its        */
/* region statistics (trilinear on the mini-map) before the table lookup.    */
/* ------------------------------------------------------------------------ */

/* Mini-map: the cube is split into regions of region[a] voxels per axis (the
 * last region of an axis keeps the remainder); point q = (k*mj + j)*mi + i
 * holds the mean (stats[2q]) and the population standard deviation
 * (stats[2q+1]) of region (i, j, k)'s voxels.  m[] receives the point counts
 * per axis.  Returns 0, or -1 on invalid arguments. */
int orc_minimap(const orc_volume *v, const int region[3], double *stats, int64_t m[3])
{
    if (!v || !v->data || !stats) return -1;
    for (int a = 0; a < 3; ++a) {
        if (region[a] < 1) return -1;
        m[a] = (v->n[a] + region[a] - 1) / region[a];
    }
    for (int64_t k = 0; k < m[2]; ++k)
        for (int64_t j = 0; j < m[1]; ++j)
            for (int64_t i = 0; i < m[0]; ++i) {
                int64_t lo[3] = {i * region[0], j * region[1], k * region[2]}, hi[3];
                for (int a = 0; a < 3; ++a) {
                    hi[a] = lo[a] + region[a];
                    if (hi[a] > v->n[a]) hi[a] = v->n[a];
                }
                double sum = 0.0, cnt = 0.0;
                for (int64_t z = lo[2]; z < hi[2]; ++z)
                    for (int64_t y = lo[1]; y < hi[1]; ++y)
                        for (int64_t x = lo[0]; x < hi[0]; ++x) {
                            sum += voxel_at(v, x, y, z);
                            cnt += 1.0;
                        }
                double mean = sum / cnt, ss = 0.0;
                for (int64_t z = lo[2]; z < hi[2]; ++z)
                    for (int64_t y = lo[1]; y < hi[1]; ++y)
                        for (int64_t x = lo[0]; x < hi[0]; ++x) {
                            double d = voxel_at(v, x, y, z) - mean;
                            ss += d * d;
                        }
                int64_t q = (k * m[1] + j) * m[0] + i;
                stats[2 * q] = mean;
                stats[2 * q + 1] = sqrt(ss / cnt);
            }
    return 0;
}

typedef struct {
    const double *stats;
    int64_t m[3];
    int region[3];
} minimap;

/* Statistics at voxel position p: trilinear over the points, point i of axis
 * a sitting at (i + 1/2) region[a] - 1/2 (the centre of a full region);
 * beyond the first and last points the nearest point's value (the weight is
 * clamped to [0, 1]); an axis with one point is constant. */
static void minimap_sample(const minimap *mm, const double p[3], double *mean, double *sd)
{
    int64_t i0[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        if (mm->m[a] < 2) {
            i0[a] = 0;
            w[a] = 0.0;
            continue;
        }
        double g = (p[a] + 0.5) / mm->region[a] - 0.5;
        int64_t f = (int64_t)floor(g);
        if (f < 0) f = 0;
        if (f > mm->m[a] - 2) f = mm->m[a] - 2;
        double t = g - (double)f;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        i0[a] = f;
        w[a] = t;
    }
    double acc[2] = {0.0, 0.0};
    for (int q = 0; q < 8; ++q) {
        int64_t ix = i0[0] + (q & 1), iy = i0[1] + ((q >> 1) & 1), iz = i0[2] + ((q >> 2) & 1);
        double wt = ((q & 1) ? w[0] : 1.0 - w[0]) * (((q >> 1) & 1) ? w[1] : 1.0 - w[1]) *
                    (((q >> 2) & 1) ? w[2] : 1.0 - w[2]);
        if (wt == 0.0) continue;
        int64_t idx = (iz * mm->m[1] + iy) * mm->m[0] + ix;
        acc[0] += wt * mm->stats[2 * idx];
        acc[1] += wt * mm->stats[2 * idx + 1];
    }
    *mean = acc[0];
    *sd = acc[1];
}

/* Probe of the mini-map interpolation (tests). */
void orc_minimap_sample(const double *stats, const int64_t m[3], const int region[3], const double p[3],
                        double out[2])
{
    minimap mm;
    mm.stats = stats;
    for (int a = 0; a < 3; ++a) { mm.m[a] = m[a]; mm.region[a] = region[a]; }
    minimap_sample(&mm, p, &out[0], &out[1]);
}

/* The sample value in units of the local standard deviation above the local
 * mean; a standard deviation below 1e-30 counts as 1e-30. */
static double sigma_value(const minimap *mm, const double p[3], double val)
{
    double mean, sd;
    minimap_sample(mm, p, &mean, &sd);
    if (!(sd > 1e-30)) sd = 1e-30;
    return (val - mean) / sd;
}

/* The composite render of render_pixel with every sample value replaced by
 * sigma_value before the table lookup ([vmin, vmax] are in units of sigma). */
static void sigma_pixel(const orc_volume *v, const orc_camera *c, const basis *b, const orc_params *P,
                        const minimap *mm, int i, int j, double out[4], int32_t *n_used)
{
    ray_setup rs;
    setup_ray(v, c, b, P, i, j, &rs);
    double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
    int64_t used = 0;
    for (int64_t k = 0; k < rs.n; ++k) {
        double p[3], rgba[4];
        sample_pos(&rs, P, k, p);
        double val = sigma_value(mm, p, trilinear(v, p, NULL));
        tf_lookup(P, val, rgba, NULL);
        double a = rgba[3];
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * rgba[ch];
        T *= (1.0 - a);
        used = k + 1;
        if (1.0 - T >= P->ert) break;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * P->bg[ch];
    out[3] = 1.0 - T + T * P->bg[3];
    if (n_used) *n_used = (int32_t)used;
}

typedef struct {
    job base;
    int mode;                 /* 1 MIP, 2 sigma clipping */
    const minimap *mm;
    double *vmax;             /* MIP: H*W or NULL */
} mode_job;

static void *mode_worker(void *arg)
{
    mode_job *M = (mode_job *)arg;
    job *J = &M->base;
    int W = J->c->width;
    int64_t first = (int64_t)J->row0 * W, last = (int64_t)J->row1 * W;
    for (int64_t px = first + J->first; px < last; px += J->stride) {
        int j = (int)(px / W), i = (int)(px % W);
        int32_t *nu = J->n_used ? J->n_used + px : NULL;
        if (M->mode == 1)
            mip_pixel(J->v, J->c, &J->b, J->P, i, j, J->rgba + 4 * px, nu, M->vmax ? M->vmax + px : NULL);
        else
            sigma_pixel(J->v, J->c, &J->b, J->P, M->mm, i, j, J->rgba + 4 * px, nu);
    }
    return NULL;
}

static int run_mode(const orc_volume *v, const orc_camera *c, const orc_params *P, int mode, const minimap *mm,
                    int row0, int row1, double *rgba, int32_t *n_used, double *vmax, int nthreads)
{
    if (check_args(v, c, P) || !rgba) return -1;
    if (row0 < 0) row0 = 0;
    if (row1 > c->height) row1 = c->height;
    if (nthreads < 1) nthreads = 1;
    mode_job *jobs = (mode_job *)calloc((size_t)nthreads, sizeof(mode_job));
    if (!jobs) return -3;
    basis b = camera_basis(c);
    for (int t = 0; t < nthreads; ++t) {
        job *J = &jobs[t].base;
        J->v = v; J->c = c; J->P = P; J->b = b;
        J->row0 = row0; J->row1 = row1; J->stride = nthreads; J->first = t;
        J->rgba = rgba; J->n_used = n_used;
        jobs[t].mode = mode; jobs[t].mm = mm; jobs[t].vmax = vmax;
    }
    int rc = 0;
    if (nthreads <= 1) {
        mode_worker(&jobs[0]);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        int started = 0;
        if (!th) rc = -3;
        for (int t = 0; t < nthreads && th; ++t) {
            if (pthread_create(&th[t], NULL, mode_worker, &jobs[t]) != 0) break;
            ++started;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        for (int t = started; t < nthreads && th; ++t) mode_worker(&jobs[t]);
        free(th);
    }
    free(jobs);
    return rc;
}

/* Maximum intensity projection of rows [row0, row1); vmax (H*W, may be NULL)
 * receives each ray's largest value (NaN on a miss). */
int orc_render_mip(const orc_volume *v, const orc_camera *c, const orc_params *P, int row0, int row1, double *rgba,
                   int32_t *n_used, double *vmax, int nthreads)
{
    return run_mode(v, c, P, 1, NULL, row0, row1, rgba, n_used, vmax, nthreads);
}

/* Sigma-clipping render of rows [row0, row1) with the mini-map `stats` of
 * orc_minimap (m[] points per axis, regions of region[] voxels). */
int orc_render_sigma(const orc_volume *v, const orc_camera *c, const orc_params *P, const double *stats,
                     const int64_t m[3], const int region[3], int row0, int row1, double *rgba, int32_t *n_used,
                     int nthreads)
{
    if (!stats) return -1;
    minimap mm;
    mm.stats = stats;
    for (int a = 0; a < 3; ++a) {
        if (region[a] < 1 || m[a] < 1) return -1;
        mm.m[a] = m[a];
        mm.region[a] = region[a];
    }
    return run_mode(v, c, P, 2, &mm, row0, row1, rgba, n_used, NULL, nthreads);
}

/* ======================================================================== */
/* Global statistics of the cube (Sections 4.1-4.3)                          */
/* ======================================================================== */

/* NULL (undefined, NaN) voxels are left out of every statistic (Section 4
 * asks for their special handling).  The stored values are widened exactly. */

/* Count, mean, population standard deviation, minimum and maximum of the
 * non-NaN voxels (two passes in FP64).  out = {count, mean, sd, min, max}. */
int orc_moments(const orc_volume *v, double out[5])
{
    if (!v || !v->data) return -1;
    double n = 0.0, sum = 0.0, mn = INFINITY, mx = -INFINITY;
    for (int64_t z = 0; z < v->n[2]; ++z)
        for (int64_t y = 0; y < v->n[1]; ++y)
            for (int64_t x = 0; x < v->n[0]; ++x) {
                double a = voxel_at(v, x, y, z);
                if (isnan(a)) continue;
                n += 1.0;
                sum += a;
                if (a < mn) mn = a;
                if (a > mx) mx = a;
            }
    double mean = n > 0 ? sum / n : NAN, ss = 0.0;
    for (int64_t z = 0; z < v->n[2]; ++z)
        for (int64_t y = 0; y < v->n[1]; ++y)
            for (int64_t x = 0; x < v->n[0]; ++x) {
                double a = voxel_at(v, x, y, z);
                if (isnan(a)) continue;
                ss += (a - mean) * (a - mean);
            }
    out[0] = n;
    out[1] = mean;
    out[2] = n > 0 ? sqrt(ss / n) : NAN;
    out[3] = mn;
    out[4] = mx;
    return 0;
}

/* Histogram of the non-NaN voxels over [lo, hi] in nbins equal bins (Section
 * 4.1): value a goes to bin floor((a - lo) / (hi - lo) * nbins), the value hi
 * to the last bin; values outside [lo, hi] are not counted. */
int orc_histogram(const orc_volume *v, double lo, double hi, int nbins, uint64_t *counts)
{
    if (!v || !v->data || !counts || nbins < 1 || !(hi > lo)) return -1;
    for (int b = 0; b < nbins; ++b) counts[b] = 0;
    for (int64_t z = 0; z < v->n[2]; ++z)
        for (int64_t y = 0; y < v->n[1]; ++y)
            for (int64_t x = 0; x < v->n[0]; ++x) {
                double a = voxel_at(v, x, y, z);
                if (!(a >= lo && a <= hi)) continue;          /* also drops NaN */
                int64_t b = (int64_t)floor((a - lo) / (hi - lo) * nbins);
                if (b >= nbins) b = nbins - 1;
                counts[b] += 1;
            }
    return 0;
}

/* Median of the non-NaN voxels by Torben Mogensen's method as the paper's
 * appendix states it: repeated passes that count the values below, above and
 * equal to a guess halfway between the current bounds, and note the largest
 * value below and the smallest above it, until neither side holds more than
 * half of the values.  The result is the value of rank (n + 1) / 2 (integer
 * division, 1-based): the median for odd n, the lower median for even n.
 * *passes receives the number of passes.  Returns 0, -1 without values. */
int orc_median(const orc_volume *v, double *median, int *passes)
{
    double m5[5];
    if (orc_moments(v, m5) || !(m5[0] > 0)) return -1;
    const int64_t n = (int64_t)m5[0], half = (n + 1) / 2;
    double lo = m5[3], hi = m5[4];
    int it = 0;
    int64_t less, greater, equal;
    double guess, max_lt, min_gt;
    for (;;) {
        ++it;
        guess = 0.5 * (lo + hi);
        less = greater = equal = 0;
        max_lt = lo;
        min_gt = hi;
        for (int64_t z = 0; z < v->n[2]; ++z)
            for (int64_t y = 0; y < v->n[1]; ++y)
                for (int64_t x = 0; x < v->n[0]; ++x) {
                    double a = voxel_at(v, x, y, z);
                    if (isnan(a)) continue;
                    if (a < guess) {
                        ++less;
                        if (a > max_lt) max_lt = a;
                    } else if (a > guess) {
                        ++greater;
                        if (a < min_gt) min_gt = a;
                    } else {
                        ++equal;
                    }
                }
        if (less <= half && greater <= half) break;
        if (less > greater) hi = max_lt;
        else lo = min_gt;
    }
    if (less >= half) *median = max_lt;
    else if (less + equal >= half) *median = guess;
    else *median = min_gt;
    if (passes) *passes = it;
    return 0;
}

/* ======================================================================== */
/* Sort-last rendering of sub-boxes (Sections 3.2 and 3.4)                   */
/* ======================================================================== */

/* The paper splits the cube into sub-cubes, renders each on its own GPU and
 * merges the sub-images in visibility order with the over operator.  Here a
 * sub-box is a range of cells [lo, hi) per axis; a sample belongs to the
 * sub-box holding its cell (the cell origin of the trilinear interpolation,
 * clamp(floor(p), 0, n-2)), so every sample of a ray belongs to exactly one
 * sub-box of a partition.  Samples sit at the positions of the whole volume's
 * ray (the same t_in), so the sub-images composite to the whole render.
 *
 * Per pixel: the premultiplied partial colour C and transmittance T of the
 * sub-box's samples (front to back, no early termination, no background),
 * the ray parameter of its first sample (depth; +inf if none) and the count. */
static void subbox_pixel(const orc_volume *v, const orc_camera *c, const basis *b, const orc_params *P,
                         const int64_t lo[3], const int64_t hi[3], int i, int j, double out[4], double *depth,
                         int32_t *count)
{
    ray_setup rs;
    setup_ray(v, c, b, P, i, j, &rs);
    double C[3] = {0.0, 0.0, 0.0}, T = 1.0, first = INFINITY;
    int32_t used = 0;
    for (int64_t k = 0; k < rs.n; ++k) {
        double p[3];
        sample_pos(&rs, P, k, p);
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            int64_t x0 = (int64_t)floor(p[a]);
            if (x0 < 0) x0 = 0;
            if (x0 > v->n[a] - 2) x0 = v->n[a] - 2;
            if (x0 < lo[a] || x0 >= hi[a]) inside = 0;
        }
        if (!inside) continue;
        double rgba[4];
        tf_lookup(P, trilinear(v, p, NULL), rgba, NULL);
        double a = rgba[3];
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * rgba[ch];
        T *= (1.0 - a);
        if (used == 0) first = rs.t_in + ((double)k + 0.5) * P->step;
        ++used;
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = T;
    if (depth) *depth = first;
    if (count) *count = used;
}

/* Sub-box render of rows [row0, row1) (single thread; test sizes). */
int orc_render_subbox(const orc_volume *v, const orc_camera *c, const orc_params *P, const int64_t lo[3],
                      const int64_t hi[3], int row0, int row1, double *partial, double *depth, int32_t *count)
{
    if (check_args(v, c, P) || !partial) return -1;
    basis b = camera_basis(c);
    int W = c->width;
    if (row0 < 0) row0 = 0;
    if (row1 > c->height) row1 = c->height;
    for (int j = row0; j < row1; ++j)
        for (int i = 0; i < W; ++i) {
            int64_t px = (int64_t)j * W + i;
            subbox_pixel(v, c, &b, P, lo, hi, i, j, partial + 4 * px, depth ? depth + px : NULL,
                         count ? count + px : NULL);
        }
    return 0;
}

/* Over-composite of k partial images per pixel in order of their depth
 * (front first): C = C1 + T1 C2 + T1 T2 C3 + ..., T = T1 T2 ...; the pixel is
 * (C + T bg.rgb, 1 - T + T bg.a).  partials[q] / depths[q] index pixel px at
 * 4 px / px. */
void orc_composite(int k, const double *const *partials, const double *const *depths, int64_t npx,
                   const double bg[4], double *rgba)
{
    int *ord = (int *)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
    for (int64_t px = 0; px < npx; ++px) {
        for (int q = 0; q < k; ++q) ord[q] = q;
        for (int q = 1; q < k; ++q)                 /* insertion sort by depth */
            for (int r = q; r > 0 && depths[ord[r]][px] < depths[ord[r - 1]][px]; --r) {
                int t = ord[r]; ord[r] = ord[r - 1]; ord[r - 1] = t;
            }
        double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
        for (int q = 0; q < k; ++q) {
            const double *s = partials[ord[q]] + 4 * px;
            for (int ch = 0; ch < 3; ++ch) C[ch] += T * s[ch];
            T *= s[3];
        }
        for (int ch = 0; ch < 3; ++ch) rgba[4 * px + ch] = C[ch] + T * bg[ch];
        rgba[4 * px + 3] = 1.0 - T + T * bg[3];
    }
    free(ord);
}
