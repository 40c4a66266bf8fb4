// k_project.cu -- Alg. 1's splatting step: per-Gaussian shape records and
// per-(receiver, Gaussian) view records, depth keys and tile coverage.
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

// Clear the status word; first_bad holds INT_MAX until a non-finite Gaussian is seen.
__global__ void k_status_init(DevStatus* st) {
    if (threadIdx.x == 0) {
        st->code = GSRF_OK;
        st->first_bad = 0x7fffffff;
        st->required_pairs = 0;
        for (int i = 0; i < 4; ++i) st->stats[i] = 0ull;
    }
}

constexpr int kPrepThreads = 64;
constexpr int kCoefMax = 2 * (kMaxDegree + 1) * (kMaxDegree + 1);  // floats of c at the largest degree
static_assert(fle_floats(kMaxDegree) <= kCoefMax, "folded coefficients fit the staging rows");
constexpr int kShapeFloats = (int)(sizeof(GShape) / sizeof(float));

// The per-Gaussian part of k_prepare: c = its coefficients, and its shape record and
// folded coefficients q written to the block's staging rows.
__device__ __forceinline__ void prepare_one(const gsrf_gaussians& g, const float* __restrict__ tx, int64_t k,
                                            const float* c, float* sgo, float* q, double* __restrict__ dpath_t,
                                            DevStatus* st, int variant, int L) {
    const float mx = g.means[3 * k], my = g.means[3 * k + 1], mz = g.means[3 * k + 2];
    const float l0 = g.log_scales[3 * k], l1 = g.log_scales[3 * k + 1], l2 = g.log_scales[3 * k + 2];
    float qw = g.quats[4 * k], qx = g.quats[4 * k + 1], qy = g.quats[4 * k + 2], qz = g.quats[4 * k + 3];
    const float ol = g.opacity_logit[k];
    const float b = g.phase_b ? g.phase_b[k] : 0.0f;
    bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(l0) && isfinite(l1) &&
                  isfinite(l2) && isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) &&
                  !isnan(ol) && isfinite(b);
    const int nb = (L + 1) * (L + 1);  // coefficients of degree L (Sec. 4.2)
    for (int i = 0; i < 2 * nb; ++i) finite = finite && isfinite(c[i]);
    if (!finite) {
        atomicCAS(&st->code, (int)GSRF_OK, (int)GSRF_ERR_NONFINITE);
        atomicMin(&st->first_bad, (int)k);
    }
    const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (n2 > 0.0f) {
        const float inv = 1.0f / sqrtf(n2);
        qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    } else {
        qw = 1.0f; qx = qy = qz = 0.0f;
    }
    const float R[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy),
                        2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx),
                        2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)};
    const float is[3] = {expf(-l0), expf(-l1), expf(-l2)};
    GShape out;
    const float sc[3] = {expf(l0), expf(l1), expf(l2)};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            out.W[3 * i + j] = R[3 * j + i] * is[i];
            out.M[3 * i + j] = R[3 * j + i] * sc[i];
        }
    out.pad2[0] = out.pad2[1] = out.pad2[2] = 0.0f;
    out.o = 1.0f / (1.0f + expf(-ol));
    // normalised density (a variant reading): 1 / ((2 pi)^1.5 s0 s1 s2) folded into o
    if (variant & GSRF_VARIANT_NORMALISED_WEIGHT) out.o *= expf(-(l0 + l1 + l2)) * 0.0634936359f;
    out.b = b;
    out.pad = 0.0f;
    const float* of = reinterpret_cast<const float*>(&out);
    for (int i = 0; i < kShapeFloats; ++i) sgo[i] = of[i];
    const double dx = (double)tx[0] - mx, dy = (double)tx[1] - my, dz = (double)tx[2] - mz;
    dpath_t[k] = sqrt(dx * dx + dy * dy + dz * dz);
    // folded Fourier-Legendre coefficients (see fle_floats): the m = 0 pairs, then per
    // (l, m > 0) in m-major order the four reals that fold c_{l,m} Y_{l,m} + c_{l,-m}
    // Y_{l,-m} with Y_{l,-m} = kappa conj(Y_{l,m}), kappa = (-1)^m (l-m)!/(l+m)!
    const int m0 = fle_m0_floats(L);
    for (int l = 0; l <= L; ++l) {
        q[2 * l] = c[2 * (l * l + l)];
        q[2 * l + 1] = c[2 * (l * l + l) + 1];
    }
    for (int i = 2 * (L + 1); i < m0; ++i) q[i] = 0.0f;
    int t = 0;
    for (int m = 1; m <= L; ++m) {
        for (int l = m; l <= L; ++l, ++t) {
            float prod = 1.0f;  // (l+m)!/(l-m)!, exact in FP32 up to L = 5 (10! < 2^24)
            for (int i = l - m + 1; i <= l + m; ++i) prod *= (float)i;
            const float kap = ((m & 1) ? -1.0f : 1.0f) / prod;
            const int np = l * l + l + m, nm = l * l + l - m;
            const float cr = c[2 * np], ci = c[2 * np + 1];
            const float dr = kap * c[2 * nm], di = kap * c[2 * nm + 1];
            q[m0 + 4 * t] = cr + dr;
            q[m0 + 4 * t + 1] = di - ci;
            q[m0 + 4 * t + 2] = ci + di;
            q[m0 + 4 * t + 3] = cr - dr;
        }
    }
}

// One thread per Gaussian: W = diag(1/s) R^T with R the rotation of the normalised
// quaternion (Sec. 4.2, Sigma = R S S^T R^T, so Sigma^-1 = W^T W), opacity = sigmoid,
// and |t - mu| in FP64 for the path phase.  A block's coefficients come in, and its
// folded coefficients and shape records go out, through shared memory (rows padded to an
// odd stride), so that global memory is read and written in consecutive words rather
// than one 128-byte record per thread.

__global__ void __launch_bounds__(kPrepThreads) k_prepare(gsrf_gaussians g, const float* __restrict__ tx,
                                                          GShape* __restrict__ shape, double* __restrict__ dpath_t,
                                                          float* __restrict__ fle, DevStatus* st, int variant, int L) {
    __shared__ float sc[kPrepThreads * (kCoefMax + 1)];
    __shared__ float sq[kPrepThreads * (kCoefMax + 1)];
    __shared__ float sg[kPrepThreads * (kShapeFloats + 1)];
    const int64_t k0 = (int64_t)blockIdx.x * kPrepThreads, k = k0 + threadIdx.x;
    const int mb = (int)min((int64_t)kPrepThreads, g.n - k0);  // Gaussians of this block
    const int nb = (L + 1) * (L + 1);                          // coefficients of degree L (Sec. 4.2)
    const int nc = 2 * nb, nq = fle_floats(L);
    for (int i = threadIdx.x; i < mb * nc; i += kPrepThreads) {
        const int gi = i / nc;
        sc[gi * (nc + 1) + (i - gi * nc)] = g.coeffs[k0 * nc + i];
    }
    __syncthreads();
    if (k < g.n) prepare_one(g, tx, k, sc + threadIdx.x * (nc + 1), sg + threadIdx.x * (kShapeFloats + 1),
                             sq + threadIdx.x * (nq + 1), dpath_t, st, variant, L);
    __syncthreads();
    for (int i = threadIdx.x; i < mb * nq; i += kPrepThreads) {
        const int gi = i / nq;
        fle[k0 * nq + i] = sq[gi * (nq + 1) + (i - gi * nq)];
    }
    float* shape_f = reinterpret_cast<float*>(shape);
    for (int i = threadIdx.x; i < mb * kShapeFloats; i += kPrepThreads) {
        const int gi = i / kShapeFloats;
        shape_f[k0 * kShapeFloats + i] = sg[gi * (kShapeFloats + 1) + (i - gi * kShapeFloats)];
    }
}



// Per-ray table of the receiving grid, in FP64 and rounded once to FP32: the ray direction
// (cos el cos az, cos el sin az, sin el) at the bin centre and the basis values the
// folded Fourier-Legendre sum of degree L needs (see raytab_floats): P_l^m without the
// Condon-Shortley phase at x = sin el, by the recurrences P_m^m = (2m-1)!! (1-x^2)^{m/2},
// P_{m+1}^m = (2m+1) x P_m^m, (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m.
// The table is separable: a ray's direction and basis are products of factors of its
// azimuth bin u (cos, sin of m az, m = 0..L) and of its elevation bin v (sin and cos of el,
// P_l^m).  k_raytab_factors computes them once per column and once per row (FP64), and
// k_raytab forms each ray's products in FP64 and rounds them once to FP32.
constexpr int kRayU = 2 * kMaxDegree;                                 // (cos, sin)(m az), m = 1..L
constexpr int kRayV = 2 + (kMaxDegree + 1) * (kMaxDegree + 2) / 2;  // sin el, cos el, P_l^m (m <= l)

// One item (a column or a row) per 32-thread block, lane 0 computing: FP64 runs at about
// 1.7 operations per clock per SM on this part, so the few hundred items are spread over
// every SM rather than packed into a handful of blocks.
__global__ void __launch_bounds__(32) k_raytab_factors(gsrf_grid gr, int L, double* __restrict__ fu,
                                                       double* __restrict__ fv) {
    if (threadIdx.x != 0) return;
    const int i = blockIdx.x;
    const double deg = 0.017453292519943295;
    if (i < gr.n_az) {
        const double az = ((double)gr.az0_deg + ((double)i + 0.5) * (double)gr.daz_deg) * deg;
        double* f = fu + (size_t)i * kRayU;
        for (int m = 1; m <= L; ++m) sincos((double)m * az, &f[2 * m - 1], &f[2 * m - 2]);
    } else if (i < gr.n_az + gr.n_el) {
        const int v = i - gr.n_az;
        const double el = ((double)gr.el0_deg + ((double)v + 0.5) * (double)gr.del_deg) * deg;
        double se, ce;
        sincos(el, &se, &ce);
        const double x = se, sx = ce;
        double P[kMaxDegree + 1][kMaxDegree + 1];
        for (int m = 0; m <= L; ++m) {
            double pmm = 1.0;
            for (int j = 1; j <= m; ++j) pmm *= (double)(2 * j - 1) * sx;
            P[m][m] = pmm;
            if (m + 1 <= L) P[m + 1][m] = (double)(2 * m + 1) * x * pmm;
            for (int l = m + 2; l <= L; ++l)
                P[l][m] = ((double)(2 * l - 1) * x * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
        }
        double* f = fv + (size_t)v * kRayV;
        f[0] = se;
        f[1] = ce;
        for (int l = 0; l <= L; ++l)
            for (int m = 0; m <= l; ++m) f[2 + l * (l + 1) / 2 + m] = P[l][m];
    }
}

__global__ void __launch_bounds__(256) k_raytab(gsrf_grid gr, int L, const double* __restrict__ fu,
                                                const double* __restrict__ fv, float* __restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gr.n_az * gr.n_el) return;
    const int u = i % gr.n_az, v = i / gr.n_az;
    const double* a = fu + (size_t)u * kRayU;
    const double* e = fv + (size_t)v * kRayV;
    const double c1 = a[0], s1 = a[1], se = e[0], ce = e[1];
    const int nf = raytab_floats(L);
    float* t = tab + (size_t)i * nf;
    t[0] = (float)(ce * c1);
    t[1] = (float)(ce * s1);
    t[2] = (float)se;
    int o = 3;
    for (int l = 1; l <= L; ++l) t[o++] = (float)e[2 + l * (l + 1) / 2];
    for (int m = 1; m <= L; ++m) {
        const double cm = a[2 * m - 2], sm = a[2 * m - 1];
        for (int l = m; l <= L; ++l) {
            const double plm = e[2 + l * (l + 1) / 2 + m];
            t[o++] = (float)(cm * plm);
            t[o++] = (float)(sm * plm);
        }
    }
    while (o < nf) t[o++] = 0.0f;
}

// Tile coverage: the bins of the receiving plane whose centre lies in the angular
// bounding box of the cone of directions along which a ray, after leaving the emitting
// sphere |x - r| = r_rx (App. A.2), can still meet the sphere of radius
// Rc = 3.03 max(s) about mu (it holds the 3-sigma ellipsoid with a 1% margin).  The cone
// has axis c = mu - r and half-angle theta with Rs = D sin(theta) (D = |c|):
//   Rs = Rc when the tangent points of the sphere lie beyond the emitting sphere
//        (r_e^2 <= D^2 - Rc^2), the usual cone of a sphere;
//   else the sphere's exit point must lie beyond r_e, and the rim of that cap is the
//        circle where both spheres meet: cos(theta) = (D^2 + r_e^2 - Rc^2) / (2 D r_e)
//        (law of cosines), every direction when that is <= 0;
// with r_e = 0.999 r_rx, a margin for the FP32 exit distance of the hit test.  Nothing
// is covered when D + Rc < r_rx.  Deterministic FP32 throughout: the oracle takes the
// same sequence of correctly rounded operations.  Rs_out returns D sin(theta) and wide
// whether theta reaches 90 degrees (every tile), for the render's direction pre-test.
__device__ __forceinline__ Cover cover_of(float cx, float cy, float cz, float lsm, const gsrf_grid& gr,
                                          int ntu, int ntv, float& D_out, float& Rs_out, bool& wide) {
    const unsigned long long all_u = ntu >= 64 ? ~0ull : ((1ull << ntu) - 1ull);
    Cover cv;
    cv.mask = 0ull;
    cv.tv = 1u;  // lo = 1 > hi = 0: empty
    cv.count = 0u;
    const float rho2 = dadd(dmul(cx, cx), dmul(cy, cy));
    const float d2 = dadd(rho2, dmul(cz, cz));
    const float D = dsqrt(d2);
    const float Rc = dmul(3.03f, det_exp(lsm));
    D_out = D;
    Rs_out = 0.0f;
    wide = false;
    if (dadd(D, Rc) < gr.r_rx) return cv;
    float Rs = Rc;
    bool all = D <= Rc;
    const float re = dmul(gr.r_rx, 0.999f);
    if (re > 0.0f) {
        const float re2 = dmul(re, re);
        const float a = dsub(d2, dmul(Rc, Rc));
        if (re2 > a) {
            const float num = dadd(a, re2);
            if (num > 0.0f) {
                const float cm = fminf(ddiv(num, dmul(dmul(2.0f, D), re)), 1.0f);
                Rs = dmul(D, dsqrt(dmul(dsub(1.0f, cm), dadd(1.0f, cm))));
                all = false;
            }
        }
    }
    Rs_out = Rs;
    if (all) {
        wide = true;
        cv.mask = all_u;
        cv.tv = (uint32_t)(ntv - 1) << 16;
        cv.count = (uint32_t)(ntu * ntv);
        return cv;
    }
    const float rad2deg = 57.2957795f;
    const float elc = dmul(det_asin(ddiv(cz, D)), rad2deg);
    const float eld = dmul(det_asin(ddiv(Rs, D)), rad2deg);
    float vlo = ceilf(dsub(ddiv(dsub(dsub(elc, eld), gr.el0_deg), gr.del_deg), 0.5f));
    float vhi = floorf(dsub(ddiv(dsub(dadd(elc, eld), gr.el0_deg), gr.del_deg), 0.5f));
    vlo = fmaxf(vlo, 0.0f);
    vhi = fminf(vhi, (float)(gr.n_el - 1));
    if (vlo > vhi) return cv;
    const int tv_lo = (int)vlo / gr.tile_h, tv_hi = (int)vhi / gr.tile_h;
    unsigned long long mask = 0ull;
    const float rho = dsqrt(rho2);
    if (rho <= Rs) {
        mask = all_u;
    } else {
        const float azc = dmul(det_atan2(cy, cx), rad2deg);
        const float azd = dmul(det_asin(ddiv(Rs, rho)), rad2deg);
        float rel = dsub(azc, gr.az0_deg);
        if (rel < 0.0f) rel = dadd(rel, 360.0f);
        if (rel < 0.0f) rel = dadd(rel, 360.0f);
        if (rel >= 360.0f) rel = dsub(rel, 360.0f);
        const float lo = dsub(rel, azd), hi = dadd(rel, azd);
        // a window whose bins all fall outside the grid is skipped without its divides,
        // with the result the full computation gives: xhi < 0 makes its last bin negative,
        // and xlo >= daz (n_az + 2) (one bin of margin for the rounding of that product)
        // puts its first bin beyond n_az.  Most Gaussians skip both wrapped windows.
        const float past = dmul(gr.daz_deg, (float)(gr.n_az + 2));
#pragma unroll
        for (int w = -1; w <= 1; ++w) {
            const float off = dmul(360.0f, (float)w);
            const float xlo = dadd(lo, off), xhi = dadd(hi, off);
            if (xhi < 0.0f || xlo >= past) continue;
            float ulo = ceilf(dsub(ddiv(xlo, gr.daz_deg), 0.5f));
            float uhi = floorf(dsub(ddiv(xhi, gr.daz_deg), 0.5f));
            ulo = fmaxf(ulo, 0.0f);
            uhi = fminf(uhi, (float)(gr.n_az - 1));
            if (ulo > uhi) continue;
            const int t0 = (int)ulo / gr.tile_w, t1 = (int)uhi / gr.tile_w;
            const unsigned long long hi_bits = t1 >= 63 ? ~0ull : ((2ull << t1) - 1ull);
            mask |= hi_bits & ~((1ull << t0) - 1ull);
        }
    }
    if (!mask) return cv;
    cv.mask = mask;
    cv.tv = (uint32_t)tv_lo | ((uint32_t)tv_hi << 16);
    cv.count = (uint32_t)(__popcll(mask) * (tv_hi - tv_lo + 1));
    return cv;
}

// Error-free FP32 transformations (Knuth's two-sum, the FMA two-product) and |a - b| of
// two FP32 points to about 47 bits, returned in FP64.  Every step is an explicit
// round-to-nearest operation, so the compiler cannot contract or reorder it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void pair_add(float& h, float& l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(l, bl));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}
__device__ __forceinline__ double pair_dist(float ax, float ay, float az, float bx, float by, float bz) {
    float ch[3], cl[3];
    two_sum(ax, -bx, ch[0], cl[0]);
    two_sum(ay, -by, ch[1], cl[1]);
    two_sum(az, -bz, ch[2], cl[2]);
    float h = 0.0f, l = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float p = __fmul_rn(ch[i], ch[i]);
        const float pe = __fmaf_rn(ch[i], ch[i], -p);              // ch^2 = p + pe exactly
        const float q = __fmaf_rn(__fmul_rn(2.0f, ch[i]), cl[i], pe);  // + 2 ch cl (cl^2 < 2^-48 ch^2)
        pair_add(h, l, p, q);
    }
    if (!(h > 0.0f)) return 0.0;
    const float sq = __fsqrt_rn(h);
    const float res = __fadd_rn(__fmaf_rn(-sq, sq, h), l);            // (h + l) - sq^2
    const float corr = __fdiv_rn(res, __fmul_rn(2.0f, sq));
    return (double)sq + (double)corr;
}

// Radiance (Eq. 9) of one Gaussian, from its folded coefficients q (see kFle), in the
// direction (cx, cy, cz) (a variant reading: the direction of mu from the receiver); the
// same basis as the ray table, x = sin(elevation), azimuth 0 on the vertical.
__device__ __forceinline__ void radiance_at(const float* __restrict__ q, float cx, float cy, float cz, float& pr,
                                            float& pi) {
    const float rho = sqrtf(cx * cx + cy * cy), D = sqrtf(rho * rho + cz * cz);
    const float x = D > 0.0f ? cz / D : 0.0f, sx = D > 0.0f ? rho / D : 1.0f;
    const float c1 = rho > 0.0f ? cx / rho : 1.0f, s1 = rho > 0.0f ? cy / rho : 0.0f;
    const float c2 = c1 * c1 - s1 * s1, s2 = 2.0f * s1 * c1;
    const float c3 = c1 * c2 - s1 * s2, s3 = s1 * c2 + c1 * s2;
    const float x2 = x * x, sx2 = sx * sx;
    const float P[3] = {x, 1.5f * x2 - 0.5f, x * (2.5f * x2 - 1.5f)};
    const float P11 = sx, P21 = 3.0f * x * sx, P31 = (7.5f * x2 - 1.5f) * sx;
    const float P22 = 3.0f * sx2, P32 = 15.0f * x * sx2, P33 = 15.0f * sx2 * sx;
    const float Y[12] = {c1 * P11, s1 * P11, c1 * P21, s1 * P21, c1 * P31, s1 * P31,
                         c2 * P22, s2 * P22, c2 * P32, s2 * P32, c3 * P33, s3 * P33};
    pr = q[0] + q[2] * P[0] + q[4] * P[1] + q[6] * P[2];
    pi = q[1] + q[3] * P[0] + q[5] * P[1] + q[7] * P[2];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const float* e = q + 8 + 4 * t;
        pr += e[0] * Y[2 * t] + e[1] * Y[2 * t + 1];
        pi += e[2] * Y[2 * t] + e[3] * Y[2 * t + 1];
    }
}

// One thread per (receiver, Gaussian): depth key and coverage; then, for a Gaussian that
// covers some tile, whitened offset, cone term and path phase (a Gaussian in no tile's
// list keeps only c and a NaN cone term: nothing reads the rest).
__global__ void __launch_bounds__(256) k_view(gsrf_gaussians g, const float* __restrict__ rxp,
                                              const GShape* __restrict__ shape,
                                              const double* __restrict__ dpath_t, gsrf_grid gr,
                                              int ntu, int ntv, double f0_over_c, float two_pi_df_over_c,
                                              View* __restrict__ view, Cover* __restrict__ cover,
                                              uint32_t* __restrict__ dkey, float* __restrict__ rx_keep,
                                              const float* __restrict__ txp, float* __restrict__ tx_keep,
                                              const float* __restrict__ fle, int variant,
                                              float4* __restrict__ circle) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (k == 0) {  // the render and its backward read the positions from the workspace
        rx_keep[3 * r] = rxp[3 * r];
        rx_keep[3 * r + 1] = rxp[3 * r + 1];
        rx_keep[3 * r + 2] = rxp[3 * r + 2];
        if (r == 0) {
            tx_keep[0] = txp[0];
            tx_keep[1] = txp[1];
            tx_keep[2] = txp[2];
        }
    }
    if (k >= g.n) return;
    const size_t o = (size_t)r * g.n + k;
    const float rx = rxp[3 * r], ry = rxp[3 * r + 1], rz = rxp[3 * r + 2];
    const float mx = g.means[3 * k], my = g.means[3 * k + 1], mz = g.means[3 * k + 2];
    const float ux = rx - mx, uy = ry - my, uz = rz - mz;
    View v;
    v.c[0] = -ux;
    v.c[1] = -uy;
    v.c[2] = -uz;
    // depth key and coverage: deterministic FP32 on c = mu - r
    const float cx = dsub(mx, rx), cy = dsub(my, ry), cz = dsub(mz, rz);
    const float D = depth_of(cx, cy, cz);
    const float lsm = fmaxf(fmaxf(g.log_scales[3 * k], g.log_scales[3 * k + 1]), g.log_scales[3 * k + 2]);
    float D_c, Rs;
    bool wide;
    const Cover cv = cover_of(cx, cy, cz, lsm, gr, ntu, ntv, D_c, Rs, wide);
    cover[o] = cv;
    dkey[o] = cv.count ? __float_as_uint(D) : kAbsentKey;  // no tile: left out of the depth sort
    if (!cv.count) {
        // in no tile's list, so nothing reads the rest of the record: c and a NaN mark only
        reinterpret_cast<float4*>(view + o)[0] = make_float4(-ux, -uy, -uz, __int_as_float(0x7fc00000));
        return;
    }
    // whitened receiver offset (FP32, contraction allowed: not a decision)
    const GShape sh = shape[k];
    v.w[0] = sh.W[0] * ux + sh.W[1] * uy + sh.W[2] * uz;
    v.w[1] = sh.W[3] * ux + sh.W[4] * uy + sh.W[5] * uz;
    v.w[2] = sh.W[6] * ux + sh.W[7] * uy + sh.W[8] * uz;
    if (variant & GSRF_VARIANT_PAPER_CULLING)
        circle[o] = circle_of(cx, cy, cz, g.log_scales + 3 * k, g.quats + 4 * k, gr);
    // direction pre-test of the render: D cos(theta) of the cover's cone less a rounding
    // margin; below -D (every direction passes) when the cone is a hemisphere or wider
    v.ccos = wide ? -1.0f - D_c : sqrtf(fmaxf(D_c * D_c - Rs * Rs, 0.0f)) - 2e-6f * D_c;
    // path phase: d = |t - mu| + |mu - r| and d f0 / c reduced to [0, 1) in FP64.  |mu - r|
    // comes as an exact FP32 pair computation (FP64 square roots are slow on this part):
    // mu - r by two-sum, the squares by FMA two-products, their sum by pair additions and
    // the square root by one Newton correction, about 47 significant bits in all.
    const double d = dpath_t[k] + pair_dist(mx, my, mz, rx, ry, rz);
    const double cyc = d * f0_over_c;
    const float fr = (float)(cyc - floor(cyc));
    float s, c;
    sincospif(2.0f * fr, &s, &c);
    v.er = c;
    v.ei = -s;
    v.omd = two_pi_df_over_c * (float)d;
    v.pad0 = v.pad1 = 0.0f;
    if (variant & GSRF_VARIANT_RADIANCE_AT_MEAN) radiance_at(fle + (size_t)k * kFle, -ux, -uy, -uz, v.pad0, v.pad1);
    view[o] = v;
}

static void launch_raytab(const gsrf_plan* p, const Layout& L, void* ws, cudaStream_t st) {
    const int n_rays = p->grid.n_az * p->grid.n_el, n_fac = p->grid.n_az + p->grid.n_el;
    double* fu = at<double>(ws, L.rayfac);
    double* fv = fu + (size_t)p->grid.n_az * kRayU;
    k_raytab_factors<<<n_fac, 32, 0, st>>>(p->grid, plan_degree(p), fu, fv);
    k_raytab<<<(n_rays + 255) / 256, 256, 0, st>>>(p->grid, plan_degree(p), fu, fv, at<float>(ws, L.raytab));
}

cudaError_t launch_project(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, const float* rx,
                           const float* tx, void* ws, cudaStream_t st) {
    DevStatus* status = at<DevStatus>(ws, L.status);
    k_status_init<<<1, 32, 0, st>>>(status);
    if (L.n == 0) {
        launch_raytab(p, L, ws, st);
        cudaError_t e = cudaMemcpyAsync(at<float>(ws, L.rxpos), rx, sizeof(float) * 3 * L.n_rx,
                                        cudaMemcpyDeviceToDevice, st);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    launch_raytab(p, L, ws, st);
    const unsigned nb = (unsigned)((L.n + 255) / 256);
    k_prepare<<<(unsigned)((L.n + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0, st>>>(
        *g, tx, at<GShape>(ws, L.gshape), at<double>(ws, L.dpath),
                                  at<float>(ws, L.fle), status, p->variant, plan_degree(p));
    k_view<<<dim3(nb, L.n_rx), 256, 0, st>>>(*g, rx, at<GShape>(ws, L.gshape), at<double>(ws, L.dpath),
                                              p->grid, L.ntu, L.ntv, p->f0_hz / kC,
                                              (float)(2.0 * 3.14159265358979323846 * p->df_hz / kC),
                                              at<View>(ws, L.view), at<Cover>(ws, L.cover),
                                              at<uint32_t>(ws, L.dkey), at<float>(ws, L.rxpos), tx,
                                              at<float>(ws, L.txpos), at<float>(ws, L.fle), p->variant,
                                              at<float4>(ws, L.circle));
    return cudaGetLastError();
}

}  // namespace gsrf
