/*
 * oracle_f32.c -- the integer decisions of the splatting step, taken in FP32.
 *
 * TEST INFRASTRUCTURE ONLY (see gsrf_oracle.h).
 *
 * The depth sort key (App. E: the low 32 bits of each splat key hold the distance
 * to the receiver) and the set of tiles a Gaussian is splatted to (Sec. 4.3) are
 * integers decided by floating point.  The kernels take these decisions in FP32, so
 * the oracle takes them in FP32 too, with the same sequence of correctly rounded
 * operations (+ - * / sqrt, no fused multiply-add: this file is compiled with
 * -ffp-contract=off), which makes keys and lists comparable bit for bit.
 *
 * Coverage rule (a conservative reading of the paper's splatting, written out in the
 * design notes): the 3-sigma ellipsoid lies inside the sphere of radius
 * 3 * max(scale) about mu; the sphere radius is inflated by 1% (Rc = 3.03 max s).  A
 * ray starts on the emitting sphere |x - r| = r_rx (App. A.2), so only directions
 * whose ray meets that sphere of radius Rc beyond r_rx matter.  They form a cone about
 * c = mu - r (D = |c|) whose half-angle theta has D sin(theta) = Rs:
 *   Rs = Rc            when r_e^2 <= D^2 - Rc^2 (the tangent points lie beyond r_e);
 *   cos(theta) = (D^2 + r_e^2 - Rc^2) / (2 D r_e) otherwise (the rim of the part of
 *                      the sphere beyond r_e, by the law of cosines), and every
 *                      direction when that numerator is <= 0;
 * with r_e = 0.999 r_rx (a margin for the FP32 exit distance of the hit test).  A tile
 * is covered when the centre of at least one of its ray bins lies inside the angular
 * bounding box of that cone:
 *   elevation  el_c +- asin(Rs / D),        el_c = asin(cz / D)
 *   azimuth    az_c +- asin(Rs / rho),      az_c = atan2(cy, cx), rho = |(cx, cy)|
 * with every azimuth when rho <= Rs (the cone holds the vertical), every tile when
 * the cone is a hemisphere or wider, and no tile when D + Rc < r_rx (the sphere lies
 * inside the ray-emitting sphere).  exp, atan2 and asin are evaluated by the short
 * formulas below (a textbook series for exp after exact argument reduction; fitted
 * polynomials for atan and asin after exact identities), not by libm, so that both
 * sides round identically.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include "gsrf_oracle.h"

#define RAD2DEG_F 57.2957795f

/* exp(x) = 2^n * e^(f ln 2) with n = floor(x log2 e); Taylor series of e^t to t^9. */
static float det_exp(float x)
{
    float y = x * 1.44269504f;
    float n = floorf(y);
    float f = y - n;
    float t = f * 0.693147182f;
    float p = 2.75573192e-6f;
    p = p * t + 2.48015873e-5f;
    p = p * t + 1.98412698e-4f;
    p = p * t + 1.38888889e-3f;
    p = p * t + 8.33333333e-3f;
    p = p * t + 4.16666667e-2f;
    p = p * t + 1.66666667e-1f;
    p = p * t + 0.5f;
    p = p * t + 1.0f;
    p = p * t + 1.0f;
    return ldexpf(p, (int)n);
}

/* atan(t), t in [0, 1]: above tan(pi/8) the identity atan(t) = pi/4 + atan((t - 1) /
 * (t + 1)) maps the argument into [-tan(pi/8), 0]; there atan(u) = u + u z Q(z), z = u^2,
 * Q of degree 4, a least-squares fit of (atan(u) - u) / (u z) on z in [0, tan^2(pi/8)]
 * (FP32 coefficients; the FP32 evaluation stays within 6.3e-8 relative of atan). */
static float det_atan_poly(float u)
{
    float z = u * u;
    float q = -0.0607130416f;
    q = q * z + 0.105907731f;
    q = q * z + -0.142430648f;
    q = q * z + 0.199984416f;
    q = q * z + -0.333333135f;
    return u + (u * z) * q;
}

static float det_atan_unit(float t)
{
    if (t <= 0.414213568f) return det_atan_poly(t);
    return 0.785398163f + det_atan_poly((t - 1.0f) / (t + 1.0f));
}

static float det_atan2(float y, float x)
{
    float ax = fabsf(x), ay = fabsf(y), a;
    if (ax == 0.0f && ay == 0.0f) return 0.0f;
    if (ay <= ax) a = det_atan_unit(ay / ax);
    else a = 1.57079633f - det_atan_unit(ax / ay);
    if (x < 0.0f) a = 3.14159265f - a;
    if (y < 0.0f) a = -a;
    return a;
}

/* asin(x), x in [0, 1/2]: x + x z P(z) with z = x^2 and P of degree 4, a least-squares
 * fit of (asin(x) - x) / (x z) on z in [0, 1/4] (FP32 coefficients; the FP32 evaluation
 * stays within 6.6e-8 relative of asin).  For |s| > 1/2 the half-angle identity
 * asin(a) = pi/2 - 2 asin(sqrt((1 - a) / 2)) maps the argument below 1/2. */
static float det_asin_poly(float z)
{
    float p = 0.0421473645f;
    p = p * z + 0.0241886489f;
    p = p * z + 0.0454691872f;
    p = p * z + 0.0749529824f;
    return p * z + 0.166667536f;
}

static float det_asin(float s)
{
    if (s > 1.0f) s = 1.0f;
    if (s < -1.0f) s = -1.0f;
    float a = fabsf(s), r;
    if (a <= 0.5f) {
        float z = a * a;
        r = a + (a * z) * det_asin_poly(z);
    } else {
        float z = (1.0f - a) * 0.5f;
        float w = sqrtf(z);
        r = 1.57079633f - 2.0f * (w + (w * z) * det_asin_poly(z));
    }
    return s < 0.0f ? -r : r;
}

/* exported for the pins: the same three functions, callable one value at a time */
float or_det_exp(float x) { return det_exp(x); }
float or_det_atan2(float y, float x) { return det_atan2(y, x); }
float or_det_asin(float s) { return det_asin(s); }

uint32_t or_depth_key_f32(const float *mu, const float *r)
{
    float cx = mu[0] - r[0], cy = mu[1] - r[1], cz = mu[2] - r[2];
    float d2 = cx * cx;
    d2 = d2 + cy * cy;
    d2 = d2 + cz * cz;
    float D = sqrtf(d2);
    uint32_t bits;
    memcpy(&bits, &D, sizeof bits);
    return bits;
}

static int32_t ceil_div_i(int32_t a, int32_t b) { return (a + b - 1) / b; }

int32_t or_cover_f32(const float *mu, const float *log_scale, const float *r, const or_grid *g,
                     uint64_t *mask_out, int32_t *tv_lo_out, int32_t *tv_hi_out)
{
    const int32_t ntu = ceil_div_i(g->n_az, g->tile_w);
    const int32_t ntv = ceil_div_i(g->n_el, g->tile_h);
    const uint64_t all_u = (ntu >= 64) ? ~0ull : ((1ull << ntu) - 1ull);

    float cx = mu[0] - r[0], cy = mu[1] - r[1], cz = mu[2] - r[2];
    float rho2 = cx * cx;
    rho2 = rho2 + cy * cy;
    float d2 = rho2 + cz * cz;
    float D = sqrtf(d2);
    float lsm = log_scale[0];
    if (log_scale[1] > lsm) lsm = log_scale[1];
    if (log_scale[2] > lsm) lsm = log_scale[2];
    float Rc = 3.03f * det_exp(lsm);

    *mask_out = 0;
    *tv_lo_out = 1;
    *tv_hi_out = 0;
    if (D + Rc < g->r_rx) return 0;
    /* the cone of directions that meet the sphere beyond r_e */
    float Rs = Rc;
    int all = D <= Rc;
    float re = g->r_rx * 0.999f;
    if (re > 0.0f) {
        float re2 = re * re;
        float a = d2 - Rc * Rc;
        if (re2 > a) {
            float num = a + re2;
            if (num > 0.0f) {
                float cm = num / ((2.0f * D) * re);
                if (cm > 1.0f) cm = 1.0f;
                Rs = D * sqrtf((1.0f - cm) * (1.0f + cm));
                all = 0;
            }
        }
    }
    if (all) {
        *mask_out = all_u;
        *tv_lo_out = 0;
        *tv_hi_out = ntv - 1;
        return ntu * ntv;
    }

    /* elevation bins whose centre lies in [el_c - d, el_c + d] */
    float elc = det_asin(cz / D) * RAD2DEG_F;
    float eld = det_asin(Rs / D) * RAD2DEG_F;
    float vlo = ceilf((elc - eld - g->el0_deg) / g->del_deg - 0.5f);
    float vhi = floorf((elc + eld - g->el0_deg) / g->del_deg - 0.5f);
    if (vlo < 0.0f) vlo = 0.0f;
    if (vhi > (float)(g->n_el - 1)) vhi = (float)(g->n_el - 1);
    if (vlo > vhi) return 0;
    int32_t tv_lo = (int32_t)vlo / g->tile_h, tv_hi = (int32_t)vhi / g->tile_h;

    uint64_t mask = 0;
    float rho = sqrtf(rho2);
    if (rho <= Rs) {
        mask = all_u;
    } else {
        float azc = det_atan2(cy, cx) * RAD2DEG_F;
        float azd = det_asin(Rs / rho) * RAD2DEG_F;
        float rel = azc - g->az0_deg;
        if (rel < 0.0f) rel = rel + 360.0f;
        if (rel < 0.0f) rel = rel + 360.0f;
        if (rel >= 360.0f) rel = rel - 360.0f;
        float lo = rel - azd, hi = rel + azd;
        for (int w = -1; w <= 1; ++w) {
            float off = 360.0f * (float)w;
            float ulo = ceilf((lo + off) / g->daz_deg - 0.5f);
            float uhi = floorf((hi + off) / g->daz_deg - 0.5f);
            if (ulo < 0.0f) ulo = 0.0f;
            if (uhi > (float)(g->n_az - 1)) uhi = (float)(g->n_az - 1);
            if (ulo > uhi) continue;
            int32_t t0 = (int32_t)ulo / g->tile_w, t1 = (int32_t)uhi / g->tile_w;
            for (int32_t t = t0; t <= t1; ++t) mask |= 1ull << t;
        }
    }
    if (!mask) return 0;
    *mask_out = mask;
    *tv_lo_out = tv_lo;
    *tv_hi_out = tv_hi;
    return (int32_t)__builtin_popcountll(mask) * (tv_hi - tv_lo + 1);
}

/* The paper's splatting circle (Sec. 4.3, "Splatting Process"), the culling of plan
 * variant 4.  The projected centre is the bin of the receiving plane that holds the
 * direction of c = mu - r: the spherical coordinates of Sec. 4.3 (azimuth atan2(cy, cx),
 * elevation asin(cz / D)) discretised by floor with the grid's own origin and step (the
 * paper's one-degree grid has az0 = 0, el0 = -90).  The spread is the largest
 * eigenvalue of Sigma2D = J Sigma J^T, J = d(u, v)/d mu at mu in bins per metre:
 *   du/dmu = (180 / pi / daz) (-cy, cx, 0) / rho^2
 *   dv/dmu = (180 / pi / del) (-cx cz, -cy cz, rho^2) / (rho D^2)
 * (rho = |(cx, cy)|), with Sigma = R diag(s)^2 R^T; J Sigma J^T has entries
 * (diag(s) R^T J_a) . (diag(s) R^T J_b).  r_k^2 = 9 lambda_max.  On the vertical
 * (rho = 0) J does not exist and every ray passes (r_k^2 = +inf), as it does when the
 * arithmetic overflows. */
void or_circle_f32(const float *mu, const float *log_scale, const float *quat, const float *r,
                   const or_grid *g, float *out)
{
    float cx = mu[0] - r[0], cy = mu[1] - r[1], cz = mu[2] - r[2];
    float rho2 = cx * cx;
    rho2 = rho2 + cy * cy;
    float d2 = rho2 + cz * cz;
    float D = sqrtf(d2);
    float az = det_atan2(cy, cx) * RAD2DEG_F;
    float rel = az - g->az0_deg;
    if (rel < 0.0f) rel = rel + 360.0f;
    if (rel < 0.0f) rel = rel + 360.0f;
    if (rel >= 360.0f) rel = rel - 360.0f;
    out[0] = floorf(rel / g->daz_deg);
    float el = D > 0.0f ? det_asin(cz / D) * RAD2DEG_F : 0.0f;
    out[1] = floorf((el - g->el0_deg) / g->del_deg);
    out[2] = INFINITY;
    if (!(rho2 > 0.0f)) return;
    float rho = sqrtf(rho2);
    float ku = RAD2DEG_F / (g->daz_deg * rho2);
    float kv = RAD2DEG_F / (g->del_deg * (rho * d2));
    float ju[3] = {-cy * ku, cx * ku, 0.0f};
    float jv[3] = {(-cx * cz) * kv, (-cy * cz) * kv, rho2 * kv};
    /* rotation of the normalised quaternion (w, x, y, z), scales exp(log s) */
    float qw = quat[0], qx = quat[1], qy = quat[2], qz = quat[3];
    float n2 = qw * qw;
    n2 = n2 + qx * qx;
    n2 = n2 + qy * qy;
    n2 = n2 + qz * qz;
    if (n2 > 0.0f) {
        float qn = sqrtf(n2);
        qw = qw / qn; qx = qx / qn; qy = qy / qn; qz = qz / qn;
    } else {
        qw = 1.0f; qx = 0.0f; qy = 0.0f; qz = 0.0f;
    }
    float R[9];
    R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    R[1] = 2.0f * (qx * qy - qw * qz);
    R[2] = 2.0f * (qx * qz + qw * qy);
    R[3] = 2.0f * (qx * qy + qw * qz);
    R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
    R[5] = 2.0f * (qy * qz - qw * qx);
    R[6] = 2.0f * (qx * qz - qw * qy);
    R[7] = 2.0f * (qy * qz + qw * qx);
    R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
    float A = 0.0f, B = 0.0f, C = 0.0f;
    for (int i = 0; i < 3; ++i) {
        float si = det_exp(log_scale[i]);
        float tu = R[i] * ju[0] + R[3 + i] * ju[1];
        tu = tu + R[6 + i] * ju[2];
        float tv = R[i] * jv[0] + R[3 + i] * jv[1];
        tv = tv + R[6 + i] * jv[2];
        float au = si * tu, av = si * tv;
        A = A + au * au;
        B = B + au * av;
        C = C + av * av;
    }
    float h = (A - C) * 0.5f;
    float lam = (A + C) * 0.5f + sqrtf(h * h + B * B);
    float r2 = 9.0f * lam;
    out[2] = r2 < INFINITY ? r2 : INFINITY; /* NaN from overflow: every ray */
}

int or_circle_in(const float *circle, int32_t u, int32_t v)
{
    float du = (float)u - circle[0], dv = (float)v - circle[1];
    float d2 = du * du + dv * dv;
    return d2 <= circle[2];
}
