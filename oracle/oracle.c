/*
 * oracle.c -- FP64 reference implementation of the GSRF per-receiver render.
 *
 * TEST INFRASTRUCTURE ONLY (see gsrf_oracle.h for the readings it fixes).
 * Slow and plain on purpose: every quantity is computed from its definition in
 * the paper, one ray and one Gaussian at a time.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "gsrf_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Fourier-Legendre basis (Sec. 4.2, Eq. 9)                                   */
/* ------------------------------------------------------------------------- */

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* P_l^m for m >= 0 by the standard three-term recurrence in l, starting from
 * P_m^m = (2m-1)!! (1-x^2)^{m/2} and P_{m+1}^m = (2m+1) x P_m^m.  No
 * Condon-Shortley factor (-1)^m. */
static double legendre_pos(int l, int m, double x)
{
    double pmm = 1.0;
    double sx = sqrt((1.0 - x) * (1.0 + x));
    for (int i = 1; i <= m; ++i) pmm *= (double)(2 * i - 1) * sx;
    if (l == m) return pmm;
    double pm1 = x * (double)(2 * m + 1) * pmm;
    if (l == m + 1) return pm1;
    double p2 = pmm, p1 = pm1, p = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        p = ((double)(2 * ll - 1) * x * p1 - (double)(ll + m - 1) * p2) / (double)(ll - m);
        p2 = p1;
        p1 = p;
    }
    return p;
}

double or_legendre(int l, int m, double x)
{
    if (l < 0 || m > l || m < -l) return 0.0;
    if (m >= 0) return legendre_pos(l, m, x);
    int am = -m;
    double sign = (am & 1) ? -1.0 : 1.0;
    return sign * factorial(l - am) / factorial(l + am) * legendre_pos(l, am, x);
}

void or_basis_l(double alpha, double x, int32_t L, double *Y)
{
    for (int l = 0; l <= L; ++l)
        for (int m = -l; m <= l; ++m) {
            int n = l * l + l + m;
            double p = or_legendre(l, m, x);
            Y[2 * n + 0] = cos((double)m * alpha) * p;
            Y[2 * n + 1] = sin((double)m * alpha) * p;
        }
}

void or_basis(double alpha, double x, double *Y) { or_basis_l(alpha, x, 3, Y); }

static int32_t degree_of(const or_grid *g) { return g->fle_degree > 0 ? g->fle_degree : 3; }

/* ------------------------------------------------------------------------- */
/* Gaussian primitive (Sec. 4.2): Sigma = R S S^T R^T                          */
/* ------------------------------------------------------------------------- */

void or_gaussian(const or_scene *s, int64_t k, double *Sigma, double *Sinv, double *opacity)
{
    const float *q4 = s->quats + 4 * k;
    double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    double qn = sqrt(w * w + x * x + y * y + z * z);
    if (qn > 0.0) { w /= qn; x /= qn; y /= qn; z /= qn; }
    else { w = 1.0; x = y = z = 0.0; }
    double R[9] = {
        1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z),       2.0 * (x * z + w * y),
        2.0 * (x * y + w * z),       1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
        2.0 * (x * z - w * y),       2.0 * (y * z + w * x),       1.0 - 2.0 * (x * x + y * y)};
    double sc[3];
    for (int i = 0; i < 3; ++i) sc[i] = exp((double)s->log_scales[3 * k + i]);
    double M[9]; /* M = R S */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * sc[j];
    double Sg[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int l = 0; l < 3; ++l) a += M[3 * i + l] * M[3 * j + l];
            Sg[3 * i + j] = a;
        }
    if (Sigma) memcpy(Sigma, Sg, sizeof Sg);
    if (Sinv) { /* adjugate / determinant */
        double a = Sg[0], b = Sg[1], c = Sg[2], d = Sg[3], e = Sg[4], f = Sg[5],
               g = Sg[6], h = Sg[7], i = Sg[8];
        double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
        double det = a * A + b * B + c * C;
        Sinv[0] = A / det;
        Sinv[1] = -(b * i - c * h) / det;
        Sinv[2] = (b * f - c * e) / det;
        Sinv[3] = B / det;
        Sinv[4] = (a * i - c * g) / det;
        Sinv[5] = -(a * f - c * d) / det;
        Sinv[6] = C / det;
        Sinv[7] = -(a * h - b * g) / det;
        Sinv[8] = (a * e - b * d) / det;
    }
    if (opacity) *opacity = 1.0 / (1.0 + exp(-(double)s->opacity_logit[k]));
}

/* ------------------------------------------------------------------------- */
/* Ray-ellipsoid intersection (App. D.3, App. A.2)                              */
/* ------------------------------------------------------------------------- */

static double quad(const double *Q, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += a[i] * Q[3 * i + j] * b[j];
    return s;
}

int or_intersect(const double *Sinv, const double *mu, const double *r, const double *v,
                 double r_rx, double *out)
{
    double w[3] = {r[0] - mu[0], r[1] - mu[1], r[2] - mu[2]};
    /* A d^2 + 2 B d + (C - 9) = 0 */
    double A = quad(Sinv, v, v);
    double B = quad(Sinv, v, w);
    double C = quad(Sinv, w, w);
    double m2 = C - B * B / A; /* Mahalanobis^2 at the closest approach */
    double disc = B * B - A * (C - 9.0);
    for (int i = 0; i < 8; ++i) out[i] = 0.0;
    out[5] = m2;
    out[8] = A;
    out[9] = C;
    if (!(disc > 0.0)) return 0;
    double sq = sqrt(disc);
    double t_out = (-B + sq) / A, t_in = (-B - sq) / A;
    out[0] = t_in;
    out[1] = t_out;
    if (t_out < r_rx) return 0;
    /* only the part of the chord beyond the ray-emitting sphere is traversed */
    double t_a = t_in > r_rx ? t_in : r_rx;
    double t_rep = 0.5 * (t_a + t_out);
    double e[3];
    for (int i = 0; i < 3; ++i) e[i] = r[i] + t_rep * v[i] - mu[i];
    double m2r = quad(Sinv, e, e);
    out[2] = t_a;
    out[3] = t_out - t_a;
    out[4] = t_rep;
    out[6] = m2r;
    out[7] = exp(-0.5 * m2r);
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Splatting + 64-bit key sort (Alg. 1, App. E)                              */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t id; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static int32_t n_tiles_u(const or_grid *g) { return (g->n_az + g->tile_w - 1) / g->tile_w; }
static int32_t n_tiles_v(const or_grid *g) { return (g->n_el + g->tile_h - 1) / g->tile_h; }

int64_t or_bin(const or_scene *s, const float *rx, const or_grid *g,
               uint64_t *keys, uint32_t *ids, int64_t cap, int64_t *tile_start)
{
    const int32_t ntu = n_tiles_u(g), ntv = n_tiles_v(g), nt = ntu * ntv;
    int64_t total = 0;
    for (int64_t k = 0; k < s->n; ++k) {
        uint64_t mask; int32_t lo, hi;
        total += or_cover_f32(s->means + 3 * k, s->log_scales + 3 * k, rx, g, &mask, &lo, &hi);
    }
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(total > 0 ? total : 1));
    int64_t p = 0;
    for (int64_t k = 0; k < s->n; ++k) {
        uint64_t mask; int32_t lo, hi;
        int32_t c = or_cover_f32(s->means + 3 * k, s->log_scales + 3 * k, rx, g, &mask, &lo, &hi);
        if (!c) continue;
        uint32_t dk = or_depth_key_f32(s->means + 3 * k, rx);
        for (int32_t tv = lo; tv <= hi; ++tv)
            for (int32_t tu = 0; tu < ntu; ++tu)
                if ((mask >> tu) & 1ull) {
                    kv[p].key = ((uint64_t)(uint32_t)(tv * ntu + tu) << 32) | (uint64_t)dk;
                    kv[p].id = (uint32_t)k;
                    ++p;
                }
    }
    qsort(kv, (size_t)total, sizeof(kv_t), kv_cmp);
    if (tile_start) {
        int64_t j = 0;
        for (int32_t t = 0; t <= nt; ++t) {
            while (j < total && (int64_t)(kv[j].key >> 32) < t) ++j;
            tile_start[t] = j;
        }
    }
    if (total <= cap) {
        for (int64_t j = 0; j < total; ++j) {
            if (keys) keys[j] = kv[j].key;
            if (ids) ids[j] = kv[j].id;
        }
    }
    free(kv);
    return total <= cap ? total : -total;
}

void or_path_phase(const or_scene *s, const float *rx, const float *tx, double f, double *phi)
{
    for (int64_t k = 0; k < s->n; ++k) {
        double dt = 0.0, dr = 0.0;
        for (int i = 0; i < 3; ++i) {
            double m = s->means[3 * k + i];
            dt += ((double)tx[i] - m) * ((double)tx[i] - m);
            dr += (m - (double)rx[i]) * (m - (double)rx[i]);
        }
        double cyc = f * (sqrt(dt) + sqrt(dr)) / OR_C_LIGHT;
        phi[k] = 2.0 * M_PI * (cyc - floor(cyc));
    }
}

/* ------------------------------------------------------------------------- */
/* The render (blend loop of Alg. 1; Eq. 14; App. A.3)                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    const or_scene *s;
    const or_grid *g;
    double rx[3], tx[3];
    double f0, df;
    int32_t n_f, mode;
    /* per Gaussian, FP64 */
    double *Sinv, *mu, *op, *dpath, *b;
    double *psig;           /* variant 1: psi_k at the direction of mu_k, [n][2] */
    float *circ;            /* variant 4: splatting circle (u_k, v_k, r_k^2), [n][3] */
    /* candidate lists */
    const int64_t *tile_start;
    const uint32_t *ids;    /* mode 0 */
    const uint32_t *order;  /* mode 1: every Gaussian, depth order */
    const int32_t *ray_idx;
    int64_t n_rays;
    int32_t n_threads;
    const or_bands *bands;
    /* forward outputs */
    double *S, *T, *Ta, *Sabs, *Scond;
    int32_t *nhit, *ntest;
    uint32_t *flags;
    /* gradient: upstream G and per-thread accumulators */
    const double *G;
    double *gacc; /* [n_threads][n][GR_STRIDE] */
} rctx;

typedef struct { rctx *c; int32_t tid; } rarg;

static void ray_geometry(const or_grid *g, int32_t ray, double *alpha, double *x, double *v)
{
    int32_t u = ray % g->n_az, vv = ray / g->n_az;
    double a = ((double)g->az0_deg + ((double)u + 0.5) * (double)g->daz_deg) * M_PI / 180.0;
    double e = ((double)g->el0_deg + ((double)vv + 0.5) * (double)g->del_deg) * M_PI / 180.0;
    v[0] = cos(e) * cos(a);
    v[1] = cos(e) * sin(a);
    v[2] = sin(e);
    *alpha = a;
    *x = sin(e);
}

static void ray_list(const rctx *c, int32_t ray, const uint32_t **list, int64_t *len)
{
    if (c->mode == 1) {
        *list = c->order;
        *len = c->s->n;
        return;
    }
    const or_grid *g = c->g;
    int32_t ntu = n_tiles_u(g);
    int32_t u = ray % g->n_az, v = ray / g->n_az;
    int32_t t = (v / g->tile_h) * ntu + (u / g->tile_w);
    *list = c->ids + c->tile_start[t];
    *len = c->tile_start[t + 1] - c->tile_start[t];
}

/* The other outcome of a hit decision that fell inside a band and missed: a ray that
 * passes just outside the 3-sigma boundary (in_m2) grazes it at its closest approach;
 * one whose exit lies just short of r_rx enters at r_rx.  Both with dt = 0. */
static int flipped_hit(const double *Sinv, const double *mu, const double *r, const double *v,
                       double r_rx, int in_m2, double *out)
{
    double w[3] = {r[0] - mu[0], r[1] - mu[1], r[2] - mu[2]};
    double t;
    if (in_m2) {
        t = -quad(Sinv, v, w) / quad(Sinv, v, v);
        if (t < r_rx) return 0;
    } else {
        t = r_rx;
    }
    double e[3];
    for (int i = 0; i < 3; ++i) e[i] = r[i] + t * v[i] - mu[i];
    double m2r = quad(Sinv, e, e);
    out[0] = out[1] = out[2] = out[4] = t;
    out[3] = 0.0;
    out[6] = m2r;
    out[7] = exp(-0.5 * m2r);
    return 1;
}

/* The intersection record out[] of or_intersect with the closest approach moved from m2
 * to m2 + e: half chord sqrt((9 - m2)/A) about t_mid = (t_in + t_out) / 2, clipped at r_rx,
 * midpoint of the clipped chord and the weight there (App. D.3, App. A.2).  Used only by
 * the perturbation study of the rounding model (or_bands.m2_shift). */
static void shift_m2(double *out, double e, double r_rx)
{
    const double A = out[8], tm = 0.5 * (out[0] + out[1]);
    const double m2 = out[5] + e;
    const double hh = sqrt(fmax(9.0 - m2, 0.0) / A);
    const double t_out = tm + hh, t_a = fmax(tm - hh, r_rx);
    const double dt = fmax(t_out - t_a, 0.0);
    const double t_rep = t_a + 0.5 * dt;
    out[0] = tm - hh;
    out[1] = t_out;
    out[2] = t_a;
    out[3] = dt;
    out[4] = t_rep;
    out[5] = m2;
    out[6] = m2 + A * (t_rep - tm) * (t_rep - tm);
    out[7] = exp(-0.5 * out[6]);
}

/* A hit of the variant that orders a ray's hits by t_mid (closest approach). */
typedef struct {
    double tm, h[10], delta;
    int64_t pos;
    uint32_t k;
    int flipped;
} tmid_hit;

static int tmid_cmp(const void *a, const void *b)
{
    const tmid_hit *x = (const tmid_hit *)a, *y = (const tmid_hit *)b;
    if (x->tm != y->tm) return x->tm < y->tm ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

static void render_one(rctx *c, int64_t i)
{
    const or_grid *g = c->g;
    const int32_t ray = c->ray_idx ? c->ray_idx[i] : (int32_t)i;
    const int32_t nf = c->n_f;
    const int32_t Ldeg = degree_of(g), nb = (Ldeg + 1) * (Ldeg + 1);
    double alpha, x, v[3], Y[2 * OR_NB_MAX];
    ray_geometry(g, ray, &alpha, &x, v);
    or_basis_l(alpha, x, Ldeg, Y);

    const uint32_t *list;
    int64_t len;
    ray_list(c, ray, &list, &len);
    const int32_t ray_u = ray % g->n_az, ray_v = ray / g->n_az;

    double S[2 * 256], T[2 * 256];
    for (int f = 0; f < nf; ++f) { S[2 * f] = S[2 * f + 1] = 0.0; T[2 * f] = 1.0; T[2 * f + 1] = 0.0; }
    double Ta = 1.0, sabs = 0.0, scond = 0.0, gsum = 0.0, lnta_err = 0.0;
    int32_t nh = 0, nt = 0, namb = 0;
    uint32_t fl = 0;
    double t_stop = INFINITY;  /* variant 16: t_mid of the terminating hit */
    const or_bands *bd = c->bands;
    /* variant 16: take every hit decision first, then composite the hits in ascending
     * t_mid (ties by list position); two hits closer in t_mid than FP32 resolves on the
     * GPU (4e-6 |t| + 1e-6) are an ambiguous order, swapped in flip mode */
    const int by_tmid = (g->variant & 16) != 0;
    tmid_hit *hits = NULL;
    int64_t n_hits = 0;
    /* variant 16 takes every decision before compositing, but like the default's walk only
     * the ones at or before the termination point (along t_mid) can change the ray: their
     * t_mid is kept here and counted once that point is known */
    double *amb_tm = NULL;
    int64_t n_amb = 0;
    for (int64_t j = 0; j < (by_tmid ? len : 0); ++j) {
        uint32_t k = list[j];
        tmid_hit hr;
        ++nt;
        if ((g->variant & 4) && !or_circle_in(c->circ + 3 * k, ray_u, ray_v)) continue;
        int hit = or_intersect(c->Sinv + 9 * k, c->mu + 3 * k, c->rx, v, g->r_rx, hr.h);
        hr.delta = bd ? bd->m2_err * sqrt(hr.h[9]) + bd->m2_abs : 0.0;
        hr.flipped = 0;
        if (bd) {
            int in_m2 = fabs(hr.h[5] - 9.0) < bd->m2_mult * hr.delta;
            int in_t = hr.h[5] < 9.0 && fabs(hr.h[1] - (double)g->r_rx) < bd->t_band;
            if (in_m2) fl |= OR_FLAG_M2;
            if (in_t) fl |= OR_FLAG_TOUT;
            if (in_m2 || in_t) {
                if (!amb_tm) amb_tm = (double *)malloc(sizeof(double) * (size_t)(2 * len + 1));
                amb_tm[n_amb++] = 0.5 * (hr.h[0] + hr.h[1]);
                if (bd->flip) {
                    hit = hit ? 0 : flipped_hit(c->Sinv + 9 * k, c->mu + 3 * k, c->rx, v, (double)g->r_rx, in_m2,
                                                hr.h);
                    hr.flipped = 1;
                }
            }
        }
        if (!hit) continue;
        if (!hits) hits = (tmid_hit *)malloc(sizeof(tmid_hit) * (size_t)len);
        hr.tm = hr.flipped ? hr.h[4] : 0.5 * (hr.h[0] + hr.h[1]);
        hr.pos = j;
        hr.k = k;
        hits[n_hits++] = hr;
    }
    if (n_hits > 1) {
        qsort(hits, (size_t)n_hits, sizeof(tmid_hit), tmid_cmp);
        for (int64_t a = 0; a + 1 < n_hits; ++a) {
            const double tb = 4e-6 * fmax(fabs(hits[a].tm), 1.0) + 1e-6;
            if (fabs(hits[a + 1].tm - hits[a].tm) < tb) {
                fl |= OR_FLAG_ORDER;
                if (!amb_tm) amb_tm = (double *)malloc(sizeof(double) * (size_t)(2 * len + 1));
                amb_tm[n_amb++] = fmin(hits[a].tm, hits[a + 1].tm);
                if (bd && bd->flip) {
                    tmid_hit t = hits[a];
                    hits[a] = hits[a + 1];
                    hits[a + 1] = t;
                    ++a;
                }
            }
        }
    }
    for (int64_t j = 0; j < (by_tmid ? n_hits : len); ++j) {
        uint32_t k;
        double h[10];
        double delta;
        int hit, flipped = 0;
        if (by_tmid) {
            k = hits[j].k;
            memcpy(h, hits[j].h, sizeof h);
            delta = hits[j].delta;
            flipped = hits[j].flipped;
            hit = 1;
            goto composite;
        }
        k = list[j];
        ++nt;
        if ((g->variant & 4) && !or_circle_in(c->circ + 3 * k, ray_u, ray_v)) continue;
        hit = or_intersect(c->Sinv + 9 * k, c->mu + 3 * k, c->rx, v, g->r_rx, h);
        delta = bd ? bd->m2_err * sqrt(h[9]) + bd->m2_abs : 0.0;
        if (bd) {
            int in_m2 = fabs(h[5] - 9.0) < bd->m2_mult * delta;
            int in_t = h[5] < 9.0 && fabs(h[1] - (double)g->r_rx) < bd->t_band;
            if (in_m2) fl |= OR_FLAG_M2;
            if (in_t) fl |= OR_FLAG_TOUT;
            if (in_m2 || in_t) {
                ++namb;
                if (bd->flip) {
                    hit = hit ? 0 : flipped_hit(c->Sinv + 9 * k, c->mu + 3 * k, c->rx, v,
                                                (double)g->r_rx, in_m2, h);
                    flipped = 1;
                }
            }
        }
        if (!hit) continue;
    composite:;
        if (bd && bd->m2_shift && nh < bd->shift_stride) {
            const double sh = bd->m2_shift[(size_t)i * (size_t)bd->shift_stride + (size_t)nh];
            if (sh != 0.0) shift_m2(h, sh * delta, (double)g->r_rx);
        }
        double a = c->op[k] * h[7];
        if (a > (double)g->alpha_max) a = (double)g->alpha_max;
        const float *cf = c->s->coeffs + (size_t)k * 2 * nb;
        double pr = 0.0, pi = 0.0; /* psi_k(ray) = sum_n c_n Y_n */
        if (g->variant & 1) {
            pr = c->psig[2 * k];
            pi = c->psig[2 * k + 1];
        } else {
            for (int n = 0; n < nb; ++n) {
                double cr = cf[2 * n], ci = cf[2 * n + 1];
                pr += cr * Y[2 * n] - ci * Y[2 * n + 1];
                pi += cr * Y[2 * n + 1] + ci * Y[2 * n];
            }
        }
        const double zabs = a * sqrt(pr * pr + pi * pi) * Ta; /* |z_k|, every frequency */
        sabs += zabs;
        if (bd) {
            /* first-order error of S from delta on this pair: its own weight
             * (dg/dm2 = -g/2), then every later term through 1 - alpha and through the
             * transmittance phase omega b dt; d(dt)/dm2 = -1/(A h) with h the half chord,
             * capped by the chord a grazing pair can have at all, 2 sqrt(2 delta / A) */
            const double hh = 0.5 * h[3] > 0.0 ? sqrt(fmax((9.0 - h[5]) / h[8], 0.0)) : 0.0;
            const double cap = 2.0 * sqrt(2.0 * delta / h[8]);
            double ddt = hh > 0.0 ? delta / (h[8] * hh) : cap;
            if (ddt > cap || flipped) ddt = cap;
            const double fmax_hz = c->f0 + (double)(nf - 1) * c->df;
            const double om = 2.0 * M_PI * fmax_hz / OR_C_LIGHT;
            scond += zabs * (gsum + 0.5 * delta);
            gsum += fabs(om * c->b[k]) * ddt + (a < (double)g->alpha_max ? a * 0.5 * delta / (1.0 - a) : 0.0);
            lnta_err += (a < (double)g->alpha_max ? a * 0.5 * delta / (1.0 - a) : 0.0) + 1e-7;
        }
        double dk = c->dpath[k]; /* Tx -> mu_k -> Rx */
        if (g->variant & 8) {    /* Tx -> x_rep -> Rx along this ray */
            double a2 = 0.0, b2 = 0.0;
            for (int i = 0; i < 3; ++i) {
                const double xr = c->rx[i] + h[4] * v[i];
                a2 += (c->tx[i] - xr) * (c->tx[i] - xr);
                b2 += (xr - c->rx[i]) * (xr - c->rx[i]);
            }
            dk = sqrt(a2) + sqrt(b2);
        }
        for (int f = 0; f < nf; ++f) {
            double fr = c->f0 + (double)f * c->df;
            double ph = 2.0 * M_PI * fr * dk / OR_C_LIGHT;
            double er = cos(ph), ei = -sin(ph);             /* e^{-j phi} */
            double zr = a * (pr * er - pi * ei), zi = a * (pr * ei + pi * er);
            S[2 * f] += zr * T[2 * f] - zi * T[2 * f + 1];
            S[2 * f + 1] += zr * T[2 * f + 1] + zi * T[2 * f];
            double th = 2.0 * M_PI * fr * c->b[k] * h[3] / OR_C_LIGHT;
            double rr = (1.0 - a) * cos(th), ri = -(1.0 - a) * sin(th); /* rho_k */
            double tr = T[2 * f] * rr - T[2 * f + 1] * ri;
            double ti = T[2 * f] * ri + T[2 * f + 1] * rr;
            T[2 * f] = tr;
            T[2 * f + 1] = ti;
        }
        Ta *= (1.0 - a);
        ++nh;
        if (g->eps_T > 0.0f) {
            int stop = Ta < (double)g->eps_T;
            if (bd && fabs(log(Ta / (double)g->eps_T)) < bd->term_mult * lnta_err + bd->term_abs) {
                fl |= OR_FLAG_TERM;
                ++namb;
                if (bd->flip) stop = !stop;
            }
            if (stop) {
                if (by_tmid) t_stop = hits[j].tm;
                break;
            }
        }
    }
    if (by_tmid) {
        const double tb = 4e-6 * fmax(fabs(t_stop), 1.0) + 1e-6;
        for (int64_t a = 0; a < n_amb; ++a) namb += amb_tm[a] <= t_stop + tb;
        free(amb_tm);
    }
    free(hits);
    fl |= (uint32_t)(namb > 255 ? 255 : namb) << 8;
    for (int f = 0; f < nf; ++f) {
        if (c->S) { c->S[2 * ((size_t)f * c->n_rays + i)] = S[2 * f]; c->S[2 * ((size_t)f * c->n_rays + i) + 1] = S[2 * f + 1]; }
        if (c->T) { c->T[2 * ((size_t)f * c->n_rays + i)] = T[2 * f]; c->T[2 * ((size_t)f * c->n_rays + i) + 1] = T[2 * f + 1]; }
    }
    if (c->Ta) c->Ta[i] = Ta;
    if (c->Sabs) c->Sabs[i] = sabs;
    if (c->Scond) c->Scond[i] = scond;
    if (c->nhit) c->nhit[i] = nh;
    if (c->ntest) c->ntest[i] = nt;
    if (c->flags) c->flags[i] = fl;
}

static void *render_worker(void *p)
{
    rarg *a = (rarg *)p;
    for (int64_t i = a->tid; i < a->c->n_rays; i += a->c->n_threads) render_one(a->c, i);
    return NULL;
}

static int prepare(rctx *c, const or_scene *s, const float *rx, const float *tx, const or_grid *g)
{
    int64_t n = s->n;
    size_t nn = (size_t)(n > 0 ? n : 1);
    c->Sinv = (double *)malloc(sizeof(double) * 9 * nn);
    c->mu = (double *)malloc(sizeof(double) * 3 * nn);
    c->op = (double *)malloc(sizeof(double) * nn);
    c->dpath = (double *)malloc(sizeof(double) * nn);
    c->b = (double *)malloc(sizeof(double) * nn);
    c->psig = (double *)malloc(sizeof(double) * 2 * nn);
    c->circ = (float *)malloc(sizeof(float) * 3 * nn);
    for (int i = 0; i < 3; ++i) {
        c->rx[i] = rx[i];
        c->tx[i] = tx[i];
    }
    for (int64_t k = 0; k < n; ++k) {
        or_gaussian(s, k, NULL, c->Sinv + 9 * k, c->op + k);
        double dt = 0.0, dr = 0.0;
        for (int i = 0; i < 3; ++i) {
            c->mu[3 * k + i] = s->means[3 * k + i];
            double a = (double)tx[i] - c->mu[3 * k + i], b = c->mu[3 * k + i] - (double)rx[i];
            dt += a * a;
            dr += b * b;
        }
        c->dpath[k] = sqrt(dt) + sqrt(dr); /* Tx -> mu_k -> Rx */
        c->b[k] = s->phase_b ? (double)s->phase_b[k] : 0.0;
        if (g->variant & 4)
            or_circle_f32(s->means + 3 * k, s->log_scales + 3 * k, s->quats + 4 * k, rx, g, c->circ + 3 * k);
        if (g->variant & 2) { /* normalised density: 1 / ((2 pi)^1.5 |Sigma|^0.5), |Sigma|^0.5 = s0 s1 s2 */
            double ls = (double)s->log_scales[3 * k] + s->log_scales[3 * k + 1] + s->log_scales[3 * k + 2];
            c->op[k] *= exp(-ls) / pow(2.0 * M_PI, 1.5);
        }
        if (g->variant & 1) { /* psi_k at the direction of mu_k (alpha = 0 on the vertical) */
            double v[3] = {c->mu[3 * k] - rx[0], c->mu[3 * k + 1] - rx[1], c->mu[3 * k + 2] - rx[2]};
            double D = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), rho = hypot(v[0], v[1]);
            double al = rho > 0.0 ? atan2(v[1], v[0]) : 0.0, x = D > 0.0 ? v[2] / D : 0.0;
            const int32_t Lg = degree_of(g), nbg = (Lg + 1) * (Lg + 1);
            double Yg[2 * OR_NB_MAX], pr = 0.0, pi = 0.0;
            or_basis_l(al, x, Lg, Yg);
            const float *cf = s->coeffs + (size_t)k * 2 * nbg;
            for (int n2 = 0; n2 < nbg; ++n2) {
                pr += cf[2 * n2] * Yg[2 * n2] - cf[2 * n2 + 1] * Yg[2 * n2 + 1];
                pi += cf[2 * n2] * Yg[2 * n2 + 1] + cf[2 * n2 + 1] * Yg[2 * n2];
            }
            c->psig[2 * k] = pr;
            c->psig[2 * k + 1] = pi;
        }
    }
    /* candidate lists */
    int32_t nt = n_tiles_u(g) * n_tiles_v(g);
    c->tile_start = NULL;
    c->ids = NULL;
    c->order = NULL;
    if (c->mode == 0) {
        int64_t *ts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt + 1));
        int64_t tot = -or_bin(s, rx, g, NULL, NULL, -1, ts);
        uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(tot > 0 ? tot : 1));
        or_bin(s, rx, g, NULL, ids, tot, ts);
        c->tile_start = ts;
        c->ids = ids;
    } else {
        kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * nn);
        for (int64_t k = 0; k < n; ++k) {
            kv[k].key = or_depth_key_f32(s->means + 3 * k, rx);
            kv[k].id = (uint32_t)k;
        }
        qsort(kv, (size_t)n, sizeof(kv_t), kv_cmp);
        uint32_t *ord = (uint32_t *)malloc(sizeof(uint32_t) * nn);
        for (int64_t k = 0; k < n; ++k) ord[k] = kv[k].id;
        free(kv);
        c->order = ord;
    }
    return 0;
}

static void release(rctx *c)
{
    free(c->Sinv); free(c->mu); free(c->op); free(c->dpath); free(c->b); free(c->psig); free(c->circ);
    free((void *)c->tile_start); free((void *)c->ids); free((void *)c->order);
}

static int check_args(const or_scene *s, const or_grid *g, int32_t n_f, int32_t mode)
{
    if (!s || !g || s->n < 0 || n_f < 1 || n_f > 256 || (mode != 0 && mode != 1)) return -1;
    if (g->n_az < 1 || g->n_el < 1 || g->tile_w < 1 || g->tile_h < 1) return -1;
    if ((g->n_az + g->tile_w - 1) / g->tile_w > 64) return -1;
    if (!(g->daz_deg > 0.0f) || !(g->del_deg > 0.0f)) return -1;
    if (g->variant < 0 || g->variant > 31) return -1;
    if (g->fle_degree < 0 || g->fle_degree > OR_L_MAX) return -1;
    return 0;
}

static void run_threads(rctx *c, void *(*fn)(void *))
{
    int32_t nt = c->n_threads;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    rarg *args = (rarg *)malloc(sizeof(rarg) * (size_t)nt);
    for (int32_t t = 0; t < nt; ++t) {
        args[t].c = c;
        args[t].tid = t;
        pthread_create(&th[t], NULL, fn, &args[t]);
    }
    for (int32_t t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
}

int or_render(const or_scene *s, const float *rx, const float *tx, double f0, double df,
              int32_t n_f, const or_grid *g, int32_t mode, const int32_t *ray_idx,
              int64_t n_rays, int32_t n_threads, const or_bands *bands,
              double *S, double *T, double *Ta, double *Sabs, double *Scond, int32_t *nhit,
              int32_t *ntest, uint32_t *flags)
{
    if (check_args(s, g, n_f, mode)) return -1;
    rctx c;
    memset(&c, 0, sizeof c);
    c.s = s; c.g = g; c.f0 = f0; c.df = df; c.n_f = n_f; c.mode = mode;
    c.ray_idx = ray_idx;
    c.n_rays = ray_idx ? n_rays : (int64_t)g->n_az * g->n_el;
    c.n_threads = n_threads < 1 ? 1 : n_threads;
    c.bands = bands;
    c.S = S; c.T = T; c.Ta = Ta; c.Sabs = Sabs; c.Scond = Scond; c.nhit = nhit; c.ntest = ntest; c.flags = flags;
    prepare(&c, s, rx, tx, g);
    run_threads(&c, render_worker);
    release(&c);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradients (App. D), written in oracle_grad.c                                 */
/* ------------------------------------------------------------------------- */
#include "oracle_grad.inc"
