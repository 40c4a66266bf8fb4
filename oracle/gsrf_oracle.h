/*
 * gsrf_oracle.h -- plain FP64 CPU oracle for the GSRF per-receiver render
 * (complex-valued 3D Gaussians, arXiv 2502.01826).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it is
 * loaded by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark, and by nothing else.  It shares no source with the CUDA path.
 *
 * What it computes, in the paper's order (Alg. 1, App. C):
 *   1. per Gaussian: Sigma = R S S^T R^T (Sec. 4.2), its inverse, opacity,
 *      distance to the receiver and the Tx -> Gaussian -> Rx path phase;
 *   2. splatting: which 16x16 ray tiles each Gaussian may touch (Sec. 4.3) and
 *      the per-tile lists sorted by (tile | depth) keys (App. E);
 *   3. per ray: the ray-ellipsoid quadratic (App. D.3), the midpoint
 *      representative point (App. A.2) and the complex front-to-back sum of
 *      Eq. 14 / App. A.3;
 *   4. gradients of a real loss through the same sum (App. D), analytically.
 * Floating point is FP64 throughout, except two routines that take integer
 * decisions (depth sort keys and tile coverage) in FP32, the precision of the
 * kernel that takes the same decisions.
 *
 * Readings of the paper that the oracle fixes (every one is also listed in the
 * repository's design notes):
 *   - alpha_k = min(o_k * g_k, alpha_max) with o_k = sigmoid(opacity logit) and the
 *     unnormalised weight g_k = exp(-m2_rep / 2); the complex transmittance of a
 *     Gaussian is rho_k = (1 - alpha_k) exp(-j 2 pi f b_k dt_k / c)   (App. A.2);
 *   - each Gaussian re-radiates with the path phase exp(-j 2 pi f d_k / c),
 *     d_k = |t - mu_k| + |mu_k - r|  (Sec. 2, multipath phase; Huygens source);
 *   - the 3-sigma ellipsoid is Mahalanobis^2 = 9 (App. D.3);
 *   - the Fourier-Legendre basis is evaluated per ray at the ray's azimuth alpha and
 *     x = sin(elevation); P_l^m carries no Condon-Shortley phase and
 *     P_l^{-m} = (-1)^m (l-m)!/(l+m)! P_l^m; coefficient n = l*l + l + m (Eq. 9);
 *   - depth order is ascending |mu_k - r| (FP32 bits), ties by Gaussian index;
 *   - hit iff m2 < 9 and t_out >= r_rx; t_in is clipped to r_rx (Eq. 10);
 *   - c = 3e8 m/s exactly (the worked example of Sec. 2).
 */
#ifndef GSRF_ORACLE_H
#define GSRF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NB 16            /* Fourier-Legendre coefficients at the default degree L = 3 */
#define OR_L_MAX 5
#define OR_NB_MAX 36        /* (OR_L_MAX + 1)^2 */
#define OR_C_LIGHT 3.0e8    /* propagation speed, m/s */

typedef struct {
    int32_t n_az, n_el;          /* rays per row / column of the receiving plane */
    float az0_deg, daz_deg;      /* azimuth of the grid origin and bin width */
    float el0_deg, del_deg;      /* elevation of the grid origin and bin height */
    float r_rx;                  /* radius of the ray-emitting sphere, m */
    float eps_T;                 /* early-termination threshold on prod(1-alpha); 0 = off */
    float alpha_max;             /* clamp on alpha */
    int32_t tile_w, tile_h;      /* rays per tile along azimuth / elevation */
    int32_t variant;             /* readings other than the default (bit mask), forward only:
                                  *   1  the Fourier-Legendre radiance of Gaussian k is taken at
                                  *      the direction of mu_k seen from the receiver (Sec. 4.3's
                                  *      v_k) for every ray, instead of at each ray's direction;
                                  *   2  the weight is the normalised Gaussian density at the
                                  *      representative point (App. A.3), g / ((2 pi)^1.5 |Sigma|^0.5)
                                  *   4  a ray (u, v) meets Gaussian k only inside its splatting
                                  *      circle on the receiving plane (Sec. 4.3, the paper's own
                                  *      culling: or_circle_f32), on top of the exact test
                                  *   8  the path of each (ray, Gaussian) pair runs through its
                                  *      representative point: d = |t - x_rep| + |x_rep - r|
                                  *      (Sec. 4.4's x_rep) instead of through mu_k
                                  *  16  a ray composites its hits in ascending t_mid (the
                                  *      closest approach along the ray, Sec. 4.4's "distance
                                  *      along the ray path"; ties by list position) instead of
                                  *      in the list's order of |mu_k - r| (App. E) */
    int32_t fle_degree;          /* Fourier-Legendre degree L of the radiance, 1..5 (0 = 3): the
                                  * scene carries (L + 1)^2 complex coefficients per Gaussian,
                                  * index l*l + l + m (Sec. 4.2) */
} or_grid;

typedef struct {
    int64_t n;
    const float *means;          /* [n,3] */
    const float *log_scales;     /* [n,3] */
    const float *quats;          /* [n,4]  w,x,y,z (not necessarily unit) */
    const float *opacity_logit;  /* [n] */
    const float *coeffs;         /* [n,16,2] */
    const float *phase_b;        /* [n] or NULL (= 0) */
} or_scene;

/* Per-ray ambiguity flags written by or_render. */
#define OR_FLAG_M2     1u   /* a tested pair has |m2 - 9| below the m2 band */
#define OR_FLAG_TOUT   2u   /* a tested pair has |t_out - r_rx| below the t band */
#define OR_FLAG_TERM   4u   /* prod(1-alpha) came within the termination band of eps_T */
#define OR_FLAG_ORDER  8u   /* variant 16: two hits' t_mid within the order band */

/* Rounding model of an FP32 evaluation of the same render, used to say where FP32
 * and FP64 may legitimately differ.  The closest approach m2 of pair k carries an
 * error of about delta_k = m2_err * sqrt(C_k) + m2_abs (C_k the Mahalanobis^2 distance of the
 * receiver: the whitened offset is ~sqrt(C_k) long and every FP32 operation on it
 * rounds at ~1e-7 relative).  A decision is "in band" when it lies within
 * m2_mult * delta_k of 9 (hit or miss), within t_band of r_rx (exit point), or when
 * |ln(Ta / eps_T)| is within term_mult times the propagated error of ln Ta plus
 * term_abs.  Sconst (below) is the first-order error of S that the same deltas cause. */
typedef struct {
    double m2_err;      /* error model of m2 per unit of sqrt(C) */
    double m2_abs;      /* plus this absolute error */
    double m2_mult;     /* band half-width on m2 in units of delta_k */
    double t_band;      /* absolute band (m) on t_out around r_rx */
    double term_mult;   /* band on |ln(Ta/eps_T)| in units of its propagated error */
    double term_abs;    /* plus this absolute band */
    int32_t flip;       /* nonzero: take every decision inside a band the other way */
    /* Perturbation study of this rounding model (tests of Scond), NULL = none: the m2 of
     * the j-th composited pair of selected ray i (j < shift_stride) is moved by
     * m2_shift[i * shift_stride + j] * delta_k, and the pair's clipped chord, midpoint and
     * weight are derived again from the moved m2 (the hit decision is kept; a chord that
     * no longer reaches r_rx has length 0 at r_rx). */
    const double *m2_shift;
    int32_t shift_stride;
} or_bands;

/* ---- building blocks (exported so the tests can pin them one by one) ---- */

/* Associated Legendre function P_l^m(x), -l <= m <= l, no Condon-Shortley phase. */
double or_legendre(int l, int m, double x);

/* The 16 complex basis values Y_n = e^{i m alpha} P_l^m(x), n = l*l + l + m (L = 3). */
void or_basis(double alpha_rad, double x, double *Y /* [16][2] */);
/* The same up to degree L (1..5): (L + 1)^2 values. */
void or_basis_l(double alpha_rad, double x, int32_t L, double *Y /* [(L+1)^2][2] */);

/* Gaussian k: Sigma (row-major 3x3), Sigma^-1, opacity in (0,1). */
void or_gaussian(const or_scene *s, int64_t k, double *Sigma, double *Sinv, double *opacity);

/* Ray r + t v (|v| = 1) against the 3-sigma ellipsoid of (mu, Sinv).
 * Returns 1 on a hit (m2 < 9 and t_out >= r_rx).  out[0..9] =
 * {t_in, t_out, t_a, dt, t_rep, m2, m2_rep, g, A, C}. */
int or_intersect(const double *Sinv, const double *mu, const double *r, const double *v,
                 double r_rx, double *out);

/* ---- FP32 decision routines (identical arithmetic to the kernels) ---- */

/* The deterministic FP32 exp / atan2 / asin used by the coverage rule. */
float or_det_exp(float x);
float or_det_atan2(float y, float x);
float or_det_asin(float s);

/* FP32 bits of |mu - r| computed as sqrt((dx*dx + dy*dy) + dz*dz), no contraction. */
uint32_t or_depth_key_f32(const float *mu, const float *r);

/* Tile coverage of Gaussian (mu, log_scale) seen from r: azimuth-tile bit mask
 * (bit tu), elevation tile range [tv_lo, tv_hi] (empty if tv_lo > tv_hi).
 * Returns the number of tiles covered. */
int32_t or_cover_f32(const float *mu, const float *log_scale, const float *r, const or_grid *g,
                     uint64_t *mask, int32_t *tv_lo, int32_t *tv_hi);

/* The paper's splatting circle of Gaussian (mu, log_scale, quat) seen from r (Sec. 4.3,
 * "Splatting Process"): out = (u_k, v_k, r_k^2) with (u_k, v_k) the grid bin holding
 * the direction of mu - r and r_k = 3 sqrt(lambda_max(J Sigma J^T)), J the Jacobian of
 * the (u, v) bin coordinates with respect to mu, in bins; r_k^2 = +inf where J is
 * undefined (mu - r vertical).  Ray (u, v) is inside when (u - u_k)^2 + (v - v_k)^2
 * <= r_k^2, both sums in FP32 as here.  The decision is taken in FP32 with the kernels'
 * sequence of correctly rounded operations. */
void or_circle_f32(const float *mu, const float *log_scale, const float *quat, const float *r,
                   const or_grid *g, float *out);
int or_circle_in(const float *circle, int32_t u, int32_t v);

/* Splatting + sort for one receiver: all (tile, Gaussian) instances ordered by
 * the 64-bit key (tile << 32 | depth bits), ties by Gaussian index.
 * tile_start[n_tiles + 1] gives each tile's range.  Returns the number of pairs, or
 * -(pairs) if it exceeds cap (nothing written then beyond tile_start). */
int64_t or_bin(const or_scene *s, const float *rx, const or_grid *g,
               uint64_t *keys, uint32_t *ids, int64_t cap, int64_t *tile_start);

/* Path phase of every Gaussian at frequency f (Sec. 2 multipath model, reading R8):
 * phi_k = 2 pi f (|t - mu_k| + |mu_k - r|) / c reduced to [0, 2 pi), FP64. */
void or_path_phase(const or_scene *s, const float *rx, const float *tx, double f, double *phi);

/* ---- the render ---- */

/* Render receiver rx for transmitter tx at frequencies f0 + i*df, i < n_f.
 * mode 0: candidates from the tile lists (Alg. 1); mode 1: brute force, every
 * Gaussian for every ray (same order).  ray_idx selects rays (v*n_az + u); NULL =
 * all rays in row-major order.  Outputs (any may be NULL):
 *   S     [n_f][n_rays][2]  received complex signal per ray
 *   T     [n_f][n_rays][2]  transmittance after the last processed Gaussian
 *   Ta    [n_rays]          prod(1 - alpha) after the last processed Gaussian
 *   Sabs  [n_rays]          sum over composited Gaussians of |z_k| = alpha_k |psi_k| |T_k|
 *                           (the scale of the sum, identical at every frequency)
 *   Scond [n_rays]          first-order error of |S| when every composited pair's m2 is
 *                           off by its delta_k (bands->m2_err; 0 if bands is NULL):
 *                           through its weight, through 1 - alpha of the pairs behind
 *                           it, and through the transmittance phase 2 pi f b dt / c,
 *                           whose chord dt = 2 sqrt((9 - m2)/A) is steep near grazing
 *   nhit  [n_rays]          Gaussians composited
 *   ntest [n_rays]          candidates tested
 *   flags [n_rays]          OR_FLAG_* ambiguity bits in bits 0-7 and, in bits 8-15, how
 *                           many decisions of the ray fell inside a band (bands may be
 *                           NULL = none).  With bands->flip set, those decisions are
 *                           taken the other way: a pair inside the m2 band that missed
 *                           grazes at its closest approach (dt = 0, weight exp(-m2/2)),
 *                           one inside the t band that missed is entered at r_rx with
 *                           dt = 0; a hit inside a band is dropped; a stop inside the
 *                           termination band continues and vice versa.
 * Returns 0, or a negative value on bad arguments. */
int or_render(const or_scene *s, const float *rx, const float *tx, double f0, double df,
              int32_t n_f, const or_grid *g, int32_t mode, const int32_t *ray_idx,
              int64_t n_rays, int32_t n_threads, const or_bands *bands,
              double *S, double *T, double *Ta, double *Sabs, double *Scond, int32_t *nhit,
              int32_t *ntest, uint32_t *flags);

/* Gradient of L = sum_rays sum_f Re(conj(G) S) for the given dL/dRe S, dL/dIm S
 * (G [n_f][n_rays][2]), with respect to the raw parameters, at the grid's degree L.
 * Gradient buffers are overwritten ([n,3],[n,3],[n,4],[n],[n,(L+1)^2,2],[n]); any may be
 * NULL.  Same ray selection, mode and termination rule as or_render; the default reading
 * and variants 2 (normalised weight) and 4 (the paper's splatting-circle culling) only. */
int or_render_grad(const or_scene *s, const float *rx, const float *tx, double f0, double df,
                   int32_t n_f, const or_grid *g, int32_t mode, const int32_t *ray_idx,
                   int64_t n_rays, int32_t n_threads, const double *G,
                   double *g_means, double *g_log_scales, double *g_quats,
                   double *g_opacity_logit, double *g_coeffs, double *g_phase_b);

#ifdef __cplusplus
}
#endif
#endif
