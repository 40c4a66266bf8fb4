// gsrf_internal.cuh -- device structures, workspace layout and shared device helpers
// of the GB300 GSRF render (arXiv 2502.01826).  Internal to libgsrf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsrf.h"

namespace gsrf {

constexpr int kNB = 16;               // Fourier-Legendre coefficients, L = 3 (Sec. 4.2)
constexpr double kC = 3.0e8;          // propagation speed (Sec. 2 worked example)
constexpr int kTile = 16;             // rays per tile side (App. E)
constexpr int kRenderThreads = kTile * kTile;
constexpr int kChunk = 4096;          // items per block in the sort passes
constexpr int kSmallChunk = 1024;     // items per block in the one-segment small-key sort (item orders)
constexpr int kDChunk = 2048;         // items per block in the depth passes
constexpr int kEChunk = 1024;         // depth-sorted Gaussians per block in the emission
constexpr int kESlice = 512;          // pairs per emission work item
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kMaxTiles = 1024;       // bins of the tile counting sort
// The depth key of a (receiver, Gaussian) that covers no tile: an FP32 NaN pattern, which
// no distance has, so the depth sort can leave such Gaussians out.
constexpr uint32_t kAbsentKey = 0xffffffffu;
constexpr int kMaxNf = 64;

// Per-Gaussian shape record: whitening matrix W = diag(1/s) R^T (so that
// (x-mu)^T Sigma^-1 (x-mu) = |W (x-mu)|^2), opacity and excess-phase coefficient; then
// M = diag(s) R^T = W^-T, with n^T Sigma n = |M n|^2, so that the 3-sigma ellipsoid
// reaches 3 |M n| along a unit normal n (its support function).  The render stages the
// first 48 bytes per candidate; M feeds its warp-level plane test.
struct __align__(16) GShape {
    float W[9];
    float o;
    float b;
    float pad;
    float M[9];
    float pad2[3];
};

// Per-(receiver, Gaussian) view record: offset c = mu - r and D cos(theta) of the cone
// of directions that can meet the Gaussian's bounding sphere beyond the emitting sphere
// (the render's pre-test; negative when every direction can), whitened receiver offset
// w = W (r - mu), path phasor e^{-j 2 pi f0 d / c} and the per-subcarrier phase step
// 2 pi df d / c.
struct __align__(16) View {
    float c[3];
    float ccos;
    float w[3];
    float er;
    float ei;
    float omd;
    float pad0, pad1;
};

// Fourier-Legendre coefficients folded for the per-ray basis of m >= 0 only
// (Y_{l,-m} = kappa_{lm} conj(Y_{l,m}), kappa_{lm} = (-1)^m (l-m)!/(l+m)!):
//   m = 0 terms (l = 0..3): c_{l,0} as (re, im)                       -> q[0..7]
//   m > 0 terms, (l,m) = (1,1),(2,1),(3,1),(2,2),(3,2),(3,3): with c = c_{l,m},
//   d = kappa c_{l,-m}: (c.re + d.re, d.im - c.im, c.im + d.im, c.re - d.re) -> q[8..31]
// so that psi = sum_m0 c P + sum_m>0 (e1 yr + e2 yi) + j (e3 yr + e4 yi).
constexpr int kFle = 32;

// Per-ray table of the receiving grid (independent of the receiver): direction,
// P_1^0, P_2^0, P_3^0 at x = sin(elevation) and Y_{l,m} for the six m > 0 terms.
constexpr int kRayTab = 20;  // floats: dx dy dz P10 | P20 P30 y11 | y21 y31 | y22 y32 | y33 - -

// Per-degree sizes (Sec. 4.2's study of L = 1..5).  Folded coefficients: the m = 0
// pairs (c_l0 re, im) for l = 0..L padded to whole float4, then one float4 per (l, m > 0)
// in m-major order ((1,1) (2,1) .. (L,1) (2,2) .. (L,L)).  Ray table: direction, P_l0 for
// l = 1..L, then (Re, Im) of Y_{l,m>0} in the same order, padded to whole float4.
__host__ __device__ constexpr int fle_floats(int L) { return 4 * ((L + 2) / 2) + 2 * L * (L + 1); }
__host__ __device__ constexpr int fle_m0_floats(int L) { return 4 * ((L + 2) / 2); }
__host__ __device__ constexpr int raytab_floats(int L) { return 4 * ((L * (L + 2) + 6) / 4); }
static_assert(fle_floats(3) == kFle && raytab_floats(3) == kRayTab, "the L = 3 layouts");
constexpr int kMaxDegree = 5;  // the largest Fourier-Legendre degree a plan may ask for
inline int plan_degree(const gsrf_plan* p) { return p->fle_degree > 0 ? p->fle_degree : 3; }
// Backward accumulators per Gaussian: W 9, mu 3, opacity, b, then the coefficient
// gradients in chunks of 16 basis values x (dL/d psi_re, dL/d psi_im), rounded to float4.
__host__ __device__ constexpr int grad_chunks(int L) { return ((L + 1) * (L + 1) + 15) / 16; }
__host__ __device__ constexpr int grad_floats(int L) { return 4 * ((14 + 32 * grad_chunks(L) + 3) / 4); }
static_assert(grad_floats(3) == 48, "the L = 3 accumulator");

// Tile coverage of a Gaussian seen from a receiver: azimuth-tile bit mask,
// elevation tile range packed lo | hi << 16, number of tiles.
struct __align__(16) Cover {
    unsigned long long mask;
    uint32_t tv;
    uint32_t count;
};

struct __align__(16) DevStatus {
    int32_t code;
    int32_t first_bad;
    long long required_pairs;
    unsigned long long stats[4];
};

// Per-ray state the backward replays from: list position (inside the tile's list) of
// the last composited Gaussian (-1 = none), prod(1 - alpha) and the complex
// transmittance at f0 after it, and (several frequencies) Gamma = sum of b dt over the
// composited pairs, which gives the transmittance at f0 + s df as T(f0) e^{-j s 2 pi df
// Gamma / c}.
struct __align__(16) RayState {
    int32_t last;
    float Ta;
    float Tr, Ti;
    float Gam;
    float pad[3];
};

struct Layout {
    // byte offsets
    size_t status, rxpos, txpos, gacc, raytab, fle, gshape, dpath, view, cover, rayfac, dkey, dkey2, dval, dval2, dhist, dvis, dchunk_sum, egroup, eslice,
        rx_base, rx_total, pchunk_base, pkeys, pkeys2, pids, pids2, tile_start, thist, qkeys, qkeys2, qorder, qhist,
        qcounter, circle, tbuf, total;
    int32_t ntu, ntv, n_tiles;
    int32_t n_rx;
    int64_t n;
    int64_t cap;
    int32_t dchunks;      // depth-sort chunks per receiver
    int32_t echunks;      // emission chunks per receiver
    int64_t pchunks_max;  // upper bound on pair chunks over all receivers
};

bool make_layout(const gsrf_plan* p, Layout* L);

template <typename T>
__host__ __device__ inline T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// ---------------------------------------------------------------------------
// Deterministic FP32 arithmetic for the two integer decisions of the splatting
// step (depth keys, tile coverage).  Only correctly rounded operations, written
// with _rn intrinsics so that no multiply-add is fused: the result is the same
// bit pattern on any IEEE-754 machine that evaluates the same sequence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float dsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ddiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float dsqrt(float a) { return __fsqrt_rn(a); }

// |c| in deterministic FP32 (the depth sort key's value, App. E: the low 32 bits of a splat
// key), c = mu - r.
__device__ __forceinline__ float depth_of(float cx, float cy, float cz) {
    return dsqrt(dadd(dadd(dmul(cx, cx), dmul(cy, cy)), dmul(cz, cz)));
}

// exp(x) for the culling radius: 2^n * e^t with n = floor(x log2 e), t = frac * ln 2,
// e^t by its Taylor series to t^9 (error ~1e-7, far inside the 1% radius margin).
__device__ __forceinline__ float det_exp(float x) {
    float y = dmul(x, 1.44269504f);
    float n = floorf(y);
    float t = dmul(dsub(y, n), 0.693147182f);
    float p = 2.75573192e-6f;
    p = dadd(dmul(p, t), 2.48015873e-5f);
    p = dadd(dmul(p, t), 1.98412698e-4f);
    p = dadd(dmul(p, t), 1.38888889e-3f);
    p = dadd(dmul(p, t), 8.33333333e-3f);
    p = dadd(dmul(p, t), 4.16666667e-2f);
    p = dadd(dmul(p, t), 1.66666667e-1f);
    p = dadd(dmul(p, t), 0.5f);
    p = dadd(dmul(p, t), 1.0f);
    p = dadd(dmul(p, t), 1.0f);
    return ldexpf(p, (int)n);
}

// atan on [0, 1]: above tan(pi/8), atan(t) = pi/4 + atan((t - 1) / (t + 1)) brings the
// argument into [-tan(pi/8), 0]; there atan(u) = u + u z Q(z), z = u^2, with Q a degree-4
// least-squares fit of (atan(u) - u) / (u z) on z in [0, tan^2(pi/8)] (coefficients
// rounded to FP32; the FP32 evaluation is within 6.3e-8 relative of atan).
__device__ __forceinline__ float det_atan_poly(float u) {
    const float z = dmul(u, u);
    float q = -0.0607130416f;
    q = dadd(dmul(q, z), 0.105907731f);
    q = dadd(dmul(q, z), -0.142430648f);
    q = dadd(dmul(q, z), 0.199984416f);
    q = dadd(dmul(q, z), -0.333333135f);
    return dadd(u, dmul(dmul(u, z), q));
}

__device__ __forceinline__ float det_atan_unit(float t) {
    if (t <= 0.414213568f) return det_atan_poly(t);
    return dadd(0.785398163f, det_atan_poly(ddiv(dsub(t, 1.0f), dadd(t, 1.0f))));
}

__device__ __forceinline__ float det_atan2(float y, float x) {
    float ax = fabsf(x), ay = fabsf(y), a;
    if (ax == 0.0f && ay == 0.0f) return 0.0f;
    if (ay <= ax) a = det_atan_unit(ddiv(ay, ax));
    else a = dsub(1.57079633f, det_atan_unit(ddiv(ax, ay)));
    if (x < 0.0f) a = dsub(3.14159265f, a);
    if (y < 0.0f) a = -a;
    return a;
}

// asin on [0, 1/2]: x + x z P(z), z = x^2, with P a degree-4 least-squares fit of
// (asin(x) - x) / (x z) on z in [0, 1/4] (coefficients rounded to FP32; the FP32 evaluation
// is within 6.6e-8 relative of asin there).  Above 1/2 the half-angle identity
// asin(a) = pi/2 - 2 asin(sqrt((1 - a) / 2)) brings the argument back below 1/2.
__device__ __forceinline__ float det_asin_poly(float z) {
    float p = 0.0421473645f;
    p = dadd(dmul(p, z), 0.0241886489f);
    p = dadd(dmul(p, z), 0.0454691872f);
    p = dadd(dmul(p, z), 0.0749529824f);
    return dadd(dmul(p, z), 0.166667536f);
}

__device__ __forceinline__ float det_asin(float s) {
    s = fminf(fmaxf(s, -1.0f), 1.0f);
    const float a = fabsf(s);
    float r;
    if (a <= 0.5f) {
        const float z = dmul(a, a);
        r = dadd(a, dmul(dmul(a, z), det_asin_poly(z)));
    } else {
        const float z = dmul(dsub(1.0f, a), 0.5f);
        const float w = dsqrt(z);
        r = dsub(1.57079633f, dmul(2.0f, dadd(w, dmul(dmul(w, z), det_asin_poly(z)))));
    }
    return s < 0.0f ? -r : r;
}

// The paper's splatting circle (Sec. 4.3, "Splatting Process"; plan variant
// GSRF_VARIANT_PAPER_CULLING).  Centre: the bin of the receiving plane that holds the
// direction of c = mu - r (azimuth atan2(cy, cx), elevation asin(cz / D), floored with the
// grid's origin and step).  Spread: lambda_max of Sigma2D = J Sigma J^T with J = d(u, v)/d mu
// in bins per metre,
//   du/dmu = (180 / pi / daz) (-cy, cx, 0) / rho^2,
//   dv/dmu = (180 / pi / del) (-cx cz, -cy cz, rho^2) / (rho D^2),
// Sigma = R diag(s)^2 R^T, so Sigma2D_ab = (diag(s) R^T J_a) . (diag(s) R^T J_b); r^2 = 9
// lambda_max.  Returns (u_k, v_k, r^2, 0); r^2 = +inf (every ray) where J does not exist
// (rho = 0) or the arithmetic overflows.  Deterministic FP32 (R and s rebuilt from the raw
// parameters with correctly rounded operations), so the oracle decides identically.
__device__ __forceinline__ float4 circle_of(float cx, float cy, float cz, const float* ls, const float* q,
                                            const gsrf_grid& gr) {
    const float rad2deg = 57.2957795f;
    const float rho2 = dadd(dmul(cx, cx), dmul(cy, cy));
    const float d2 = dadd(rho2, dmul(cz, cz));
    const float D = dsqrt(d2);
    float rel = dsub(dmul(det_atan2(cy, cx), rad2deg), gr.az0_deg);
    if (rel < 0.0f) rel = dadd(rel, 360.0f);
    if (rel < 0.0f) rel = dadd(rel, 360.0f);
    if (rel >= 360.0f) rel = dsub(rel, 360.0f);
    float4 out;
    out.x = floorf(ddiv(rel, gr.daz_deg));
    const float el = D > 0.0f ? dmul(det_asin(ddiv(cz, D)), rad2deg) : 0.0f;
    out.y = floorf(ddiv(dsub(el, gr.el0_deg), gr.del_deg));
    out.z = __int_as_float(0x7f800000);  // +inf
    out.w = 0.0f;
    if (!(rho2 > 0.0f)) return out;
    const float rho = dsqrt(rho2);
    const float ku = ddiv(rad2deg, dmul(gr.daz_deg, rho2));
    const float kv = ddiv(rad2deg, dmul(gr.del_deg, dmul(rho, d2)));
    const float ju0 = dmul(-cy, ku), ju1 = dmul(cx, ku), ju2 = 0.0f;
    const float jv0 = dmul(dmul(-cx, cz), kv), jv1 = dmul(dmul(-cy, cz), kv), jv2 = dmul(rho2, kv);
    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float n2 = dadd(dadd(dadd(dmul(qw, qw), dmul(qx, qx)), dmul(qy, qy)), dmul(qz, qz));
    if (n2 > 0.0f) {
        const float qn = dsqrt(n2);
        qw = ddiv(qw, qn);
        qx = ddiv(qx, qn);
        qy = ddiv(qy, qn);
        qz = ddiv(qz, qn);
    } else {
        qw = 1.0f;
        qx = qy = qz = 0.0f;
    }
    float R[9];
    R[0] = dsub(1.0f, dmul(2.0f, dadd(dmul(qy, qy), dmul(qz, qz))));
    R[1] = dmul(2.0f, dsub(dmul(qx, qy), dmul(qw, qz)));
    R[2] = dmul(2.0f, dadd(dmul(qx, qz), dmul(qw, qy)));
    R[3] = dmul(2.0f, dadd(dmul(qx, qy), dmul(qw, qz)));
    R[4] = dsub(1.0f, dmul(2.0f, dadd(dmul(qx, qx), dmul(qz, qz))));
    R[5] = dmul(2.0f, dsub(dmul(qy, qz), dmul(qw, qx)));
    R[6] = dmul(2.0f, dsub(dmul(qx, qz), dmul(qw, qy)));
    R[7] = dmul(2.0f, dadd(dmul(qy, qz), dmul(qw, qx)));
    R[8] = dsub(1.0f, dmul(2.0f, dadd(dmul(qx, qx), dmul(qy, qy))));
    float A = 0.0f, B = 0.0f, C = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float si = det_exp(ls[i]);
        const float tu = dadd(dadd(dmul(R[i], ju0), dmul(R[3 + i], ju1)), dmul(R[6 + i], ju2));
        const float tv = dadd(dadd(dmul(R[i], jv0), dmul(R[3 + i], jv1)), dmul(R[6 + i], jv2));
        const float au = dmul(si, tu), av = dmul(si, tv);
        A = dadd(A, dmul(au, au));
        B = dadd(B, dmul(au, av));
        C = dadd(C, dmul(av, av));
    }
    const float h = dmul(dsub(A, C), 0.5f);
    const float lam = dadd(dmul(dadd(A, C), 0.5f), dsqrt(dadd(dmul(h, h), dmul(B, B))));
    const float r2 = dmul(9.0f, lam);
    if (r2 < __int_as_float(0x7f800000)) out.z = r2;  // NaN or inf: every ray
    return out;
}

// Ray (u, v) inside a splatting circle (circle_of): (u - u_k)^2 + (v - v_k)^2 <= r^2.
__device__ __forceinline__ bool circle_in(const float4& cc, int u, int v) {
    const float du = dsub((float)u, cc.x), dv = dsub((float)v, cc.y);
    return dadd(dmul(du, du), dmul(dv, dv)) <= cc.z;
}

// ---------------------------------------------------------------------------
// launchers (one translation unit each)
// ---------------------------------------------------------------------------
cudaError_t launch_project(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g,
                           const float* rx, const float* tx, void* ws, cudaStream_t st);
cudaError_t launch_bin(const gsrf_plan* p, const Layout& L, void* ws, cudaStream_t st);
cudaError_t launch_pair_keys(const Layout& L, void* ws, cudaStream_t st);
// Depth sort of every receiver's n keys in one thread-block cluster per receiver
// (k_dsort.cu): applies when n keys fit in the largest cluster that runs on the device.
bool depth_sort_cluster_applies(long long n);
cudaError_t launch_depth_sort_cluster(const uint32_t* dkey, long long n, int n_rx, uint32_t* dval, uint32_t* nvis,
                                      cudaStream_t st);
cudaError_t launch_render_fwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g,
                              void* ws, float* out, void* ray_state, cudaStream_t st);
cudaError_t launch_signal(const float* rays, int n_rx, int n_f, int n_el, int n_az, int mode,
                          float* out, cudaStream_t st);
cudaError_t launch_sort_small_keys(const uint32_t* keys, uint32_t* keys_out, uint32_t* vals_out, long long n,
                                   int nbins, uint32_t* hist, cudaStream_t st);
cudaError_t launch_sort_small_keys_segmented(const uint32_t* keys, uint32_t* keys_out, uint32_t* vals_out, int n_seg,
                                             const long long* seg_base, const uint32_t* chunk_base, long long chunks,
                                             int nbins, uint32_t* hist, cudaStream_t st);
// Work items of a render launch: item id = ((r * n_tiles + tile) * per_tile + k), k < per_tile
// (ray block and subcarrier chunk).  Writes the heaviest-first order of the n_rx * n_tiles *
// per_tile items into the workspace's queue buffers and zeroes the queue counter.
cudaError_t launch_item_order(const Layout& L, void* ws, int per_tile, uint32_t** order,
                              unsigned long long** counter, cudaStream_t st);
// Geometry of the warps' ray blocks: width bw (a power of two, 4..32), height 32 / bw.
int plan_block_w(const gsrf_plan* p);
int plan_stage(const gsrf_plan* p);
// Persistent batched render of n_jobs projected and binned problems (n_f == 1 each).
size_t batch_workspace_bytes(int n_jobs, const gsrf_plan* plans);
long long batch_items(int n_jobs, const gsrf_plan* plans);
cudaError_t launch_render_batch(int n_jobs, const gsrf_plan* plans, void* const* workspaces, float* const* outs,
                                void* batch_ws, unsigned long long* job_done, bool job_order, cudaStream_t st);
cudaError_t launch_render_bwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, void* ws,
                              const void* ray_state, const float* grad_rays, float* g_means, float* g_log_scales,
                              float* g_quats, float* g_opacity_logit, float* g_coeffs, float* g_phase_b,
                              cudaStream_t st);

}  // namespace gsrf

namespace gsrf {

// ---------------------------------------------------------------------------
// Geometry of one (ray, candidate) pair, shared by the forward and the backward
// render so that both take exactly the same hit decisions: every operation that
// feeds a decision is an explicit round-to-nearest intrinsic, so the compiler cannot
// contract it differently in the two kernels.
//
// Records (6 float4): v0 = (c = mu - r, D cos theta), v1 = (w = W (r - mu), er),
// v2 = (ei, omd, -, -), s0 = W0..W3, s1 = W4..W7, s2 = (W8, o, b, -).
// Per ray, in order: the 3-sigma ellipsoid in whitened coordinates,
// m2 A = |w x v'|^2 < 9 A (v' = W v, Lagrange's identity, App. D.3 quadratic with
// A = |v'|^2, B = w.v', C = |w|^2); the chord's exit t_out = t_mid + h >= r_rx with
// t_mid = -B/A, h = sqrt((9 - m2)/A).  The direction cone (c, D cos theta: the
// directions that meet the bounding sphere beyond the emitting sphere) is tested once
// per warp (bundle_meets), never per ray: it only ever rejects pairs these two tests
// reject too.
// ---------------------------------------------------------------------------
// Single hardware instructions (no compiler choice of sequence), so that the forward and
// the backward take the same value.
__device__ __forceinline__ float rcp_hw(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_hw(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Cone of a warp's rays: unit axis b and cos / sin of the half-angle beta that holds
// all of them (with a small angular margin).
struct Bundle {
    float bx, by, bz, cb, sb;
};

__device__ __forceinline__ Bundle warp_bundle(bool valid, float dx, float dy, float dz) {
    float sx = valid ? dx : 0.0f, sy = valid ? dy : 0.0f, sz = valid ? dz : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    const float in = rsqrtf(fmaxf(sx * sx + sy * sy + sz * sz, 1e-30f));
    Bundle b;
    b.bx = sx * in;
    b.by = sy * in;
    b.bz = sz * in;
    float c = valid ? dx * b.bx + dy * b.by + dz * b.bz : 1.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c = fminf(c, __shfl_xor_sync(0xffffffffu, c, o));
    c = fmaxf(fminf(c, 1.0f), -1.0f) - 2e-5f;  // margin for rounding of the axis and rays
    b.cb = c;
    b.sb = sqrtf(fmaxf(1.0f - c * c, 0.0f));
    return b;
}

// Can a ray of the bundle lie in the record's direction cone (axis c = mu - r, half-angle
// theta, c.w = D cos(theta))?  Only if angle(b, c) <= beta + theta, i.e.
// c.b >= D cos(beta + theta) = cos(beta) D cos(theta) - sin(beta) D sin(theta).  Every
// ray may when either cone is a hemisphere or wider.
__device__ __forceinline__ bool bundle_meets(const Bundle& b, float4 c) {
    if (c.w < 0.0f || b.cb <= 0.0f) return true;
    const float D2 = c.x * c.x + c.y * c.y + c.z * c.z;
    const float dsn = sqrtf(fmaxf(D2 - c.w * c.w, 0.0f));  // D sin(theta)
    const float cd = c.x * b.bx + c.y * b.by + c.z * b.bz;
    return cd >= b.cb * c.w - b.sb * dsn - 1e-4f * (c.w + dsn);
}

// Five half-spaces n.x >= n.w that hold every point of the warp's bw x bh block of rays
// beyond the emitting sphere (x = t d, t >= r_rx).  Four pass through the receiver
// (n.w = 0): the vertical planes at the block's first and last azimuth, and planes
// tilted to its lowest and highest elevation; each is moved along the warp axis b until
// it clears all of the warp's rays (a margin of 1e-6 in n.d).  The fifth is the depth
// plane b.x >= r_rx cb - 1e-4: b.d >= cb on every ray (cb holds a margin), so a ray
// point at t >= r_rx lies beyond it; it drops candidates whose ellipsoid ends inside the
// emitting sphere in the warp's directions, which are most of the near misses in a
// dense scene.  An ellipsoid that lies wholly outside one half-space meets no ray of
// the warp beyond r_rx.  Every lane computes the same planes; lane j < kPlanes writes
// plane j to the warp's shared slots.
constexpr int kOrderCap = 512;  // hits per ray kept by the t_mid-order variant
constexpr int kPlanes = 5;
constexpr int kPlaneSlots = kPlanes + 1;  // + the warp bundle's cos / sin (bundle_at)

__device__ __forceinline__ void warp_planes(const gsrf_grid& gr, int u_lo, int v_lo, int bw, int bh, const Bundle& b,
                                            bool valid, float dx, float dy, float dz, float4* spl) {
    const int u_hi = min(u_lo + bw - 1, gr.n_az - 1), v_hi = min(v_lo + bh - 1, gr.n_el - 1);
    const float kDeg = 0.0174532925f;
    const float a0 = (gr.az0_deg + ((float)u_lo + 0.5f) * gr.daz_deg) * kDeg;
    const float a1 = (gr.az0_deg + ((float)u_hi + 0.5f) * gr.daz_deg) * kDeg;
    const float e0 = (gr.el0_deg + ((float)v_lo + 0.5f) * gr.del_deg) * kDeg;
    const float e1 = (gr.el0_deg + ((float)v_hi + 0.5f) * gr.del_deg) * kDeg;
    float sa0, ca0, sa1, ca1, se0, ce0, se1, ce1, sam, cam;
    sincosf(a0, &sa0, &ca0);
    sincosf(a1, &sa1, &ca1);
    sincosf(e0, &se0, &ce0);
    sincosf(e1, &se1, &ce1);
    sincosf(0.5f * (a0 + a1), &sam, &cam);
    float n[4][3] = {{-sa0, ca0, 0.0f}, {sa1, -ca1, 0.0f}, {-se0 * cam, -se0 * sam, ce0}, {se1 * cam, se1 * sam, -ce1}};
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float m = valid ? n[j][0] * dx + n[j][1] * dy + n[j][2] * dz : 1e30f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        m -= 1e-6f;
        if (m < 0.0f) {
            // b.d >= b.cb > 0 on every ray, so n + (-m / b.cb) b clears them all
            const float lam = b.cb > 0.0f ? -m / b.cb : 0.0f;
            const float keep = b.cb > 0.0f ? 1.0f : 0.0f;  // no plane when the warp spans a hemisphere
            n[j][0] = keep * (n[j][0] + lam * b.bx);
            n[j][1] = keep * (n[j][1] + lam * b.by);
            n[j][2] = keep * (n[j][2] + lam * b.bz);
        }
        if (lane == j) spl[j] = make_float4(n[j][0], n[j][1], n[j][2], 0.0f);
    }
    if (lane == 4)
        spl[4] = b.cb > 0.0f ? make_float4(b.bx, b.by, b.bz, gr.r_rx * b.cb - 1e-4f) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (lane == 5) spl[5] = make_float4(b.cb, b.sb, 0.0f, 0.0f);
    __syncwarp();
}

// The warp bundle back from the slots warp_planes wrote (so that a kernel need not hold
// it in registers across its loop).  The axis is only stored when cb > 0; otherwise the
// bundle spans a hemisphere and bundle_meets accepts every candidate without it.
__device__ __forceinline__ Bundle bundle_at(const float4* spl) {
    const float4 ax = spl[4], cs = spl[5];
    Bundle b;
    b.bx = ax.x;
    b.by = ax.y;
    b.bz = ax.z;
    b.cb = cs.x;
    b.sb = cs.y;
    return b;
}

// Can the 3-sigma ellipsoid about mu (c = mu - r; M from the shape record) reach the
// inner side of all five half-spaces?  Its support along n is n.c + 3 |M n|, so it does
// iff n.c - n.w + 3 |M n| >= 0; a 1% margin (3.03) covers rounding (at least 3e-4 m for
// the smallest scales, far above the FP32 error of the per-ray exit point).  A zero
// plane never rejects.
__device__ __forceinline__ bool planes_meet(const float4* spl, const float4& c, const GShape* sh) {
    const float4* mm = reinterpret_cast<const float4*>(sh) + 3;
    const float4 m0 = __ldg(mm), m1 = __ldg(mm + 1), m2 = __ldg(mm + 2);
    bool meet = true;
#pragma unroll
    for (int j = 0; j < kPlanes; ++j) {
        const float4 n = spl[j];
        const float s0 = m0.x * n.x + m0.y * n.y + m0.z * n.z;
        const float s1 = m0.w * n.x + m1.x * n.y + m1.y * n.z;
        const float s2 = m1.z * n.x + m1.w * n.y + m2.x * n.z;
        const float nc = n.x * c.x + n.y * c.y + n.z * c.z - n.w;
        meet = meet && (nc >= 0.0f || nc * nc <= 9.1809f * (s0 * s0 + s1 * s1 + s2 * s2));
    }
    return meet;
}

struct PairGeo {
    float vx, vy, vz;  // v' = W v
    float A, iA, m2, tm, h, t_out, t_a, dt, dl, m2r;
};

__device__ __forceinline__ bool pair_hits(const float4& v1, const float4& s0, const float4& s1, const float4& s2,
                                          float dx, float dy, float dz, float r_rx, PairGeo& g) {
    g.vx = __fmaf_rn(s0.z, dz, __fmaf_rn(s0.y, dy, __fmul_rn(s0.x, dx)));
    g.vy = __fmaf_rn(s1.y, dz, __fmaf_rn(s1.x, dy, __fmul_rn(s0.w, dx)));
    g.vz = __fmaf_rn(s2.x, dz, __fmaf_rn(s1.w, dy, __fmul_rn(s1.z, dx)));
    g.A = __fmaf_rn(g.vz, g.vz, __fmaf_rn(g.vy, g.vy, __fmul_rn(g.vx, g.vx)));
    const float cx = __fsub_rn(__fmul_rn(v1.y, g.vz), __fmul_rn(v1.z, g.vy));
    const float cy = __fsub_rn(__fmul_rn(v1.z, g.vx), __fmul_rn(v1.x, g.vz));
    const float cz = __fsub_rn(__fmul_rn(v1.x, g.vy), __fmul_rn(v1.y, g.vx));
    const float m2A = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmul_rn(cx, cx)));
    if (m2A >= __fmul_rn(9.0f, g.A)) return false;
    g.iA = rcp_hw(g.A);
    g.m2 = __fmul_rn(m2A, g.iA);
    const float B = __fmaf_rn(v1.z, g.vz, __fmaf_rn(v1.y, g.vy, __fmul_rn(v1.x, g.vx)));
    g.tm = -__fmul_rn(B, g.iA);
    g.h = sqrt_hw(fmaxf(__fmul_rn(__fsub_rn(9.0f, g.m2), g.iA), 0.0f));
    g.t_out = __fadd_rn(g.tm, g.h);
    if (g.t_out < r_rx) return false;
    g.t_a = fmaxf(__fsub_rn(g.tm, g.h), r_rx);
    g.dt = __fsub_rn(g.t_out, g.t_a);
    g.dl = __fsub_rn(__fmul_rn(0.5f, __fadd_rn(g.t_a, g.t_out)), g.tm);
    g.m2r = __fmaf_rn(__fmul_rn(g.A, g.dl), g.dl, g.m2);
    return true;
}

// Radiance psi of one Gaussian along one ray (Eq. 9) from its folded coefficients q
// (see fle_floats) and the ray's basis values: P = (P_10 .. P_L0), Y = the complex
// Y_{l,m>0} in m-major order.  One fused multiply-add per product, accumulated in order.
template <int L, bool SHARED = false>
__device__ __forceinline__ void fle_psi(const float4* __restrict__ q4, const float* P, const float* Y,
                                        float& pr, float& pi) {
    // SHARED: the coefficients were staged in shared memory (plain loads)
    auto ld = [&](int i) -> float4 { if constexpr (SHARED) return q4[i]; else return __ldg(q4 + i); };
    constexpr int kQ0 = fle_m0_floats(L) / 4;
    float m0[4 * kQ0];
#pragma unroll
    for (int i = 0; i < kQ0; ++i) {
        const float4 a = ld(i);
        m0[4 * i] = a.x;
        m0[4 * i + 1] = a.y;
        m0[4 * i + 2] = a.z;
        m0[4 * i + 3] = a.w;
    }
    pr = m0[0];
    pi = m0[1];
#pragma unroll
    for (int l = 1; l <= L; ++l) {
        pr = fmaf(m0[2 * l], P[l - 1], pr);
        pi = fmaf(m0[2 * l + 1], P[l - 1], pi);
    }
#pragma unroll
    for (int t = 0; t < L * (L + 1) / 2; ++t) {
        const float4 e = ld(kQ0 + t);
        pr = fmaf(e.y, Y[2 * t + 1], fmaf(e.x, Y[2 * t], pr));
        pi = fmaf(e.w, Y[2 * t + 1], fmaf(e.z, Y[2 * t], pi));
    }
}

// The ray's direction and basis values from the per-grid ray table (see raytab_floats).
template <int L>
__device__ __forceinline__ void load_ray(const float* raytab, size_t ray, float& dx, float& dy, float& dz,
                                         float* P, float* Y) {
    constexpr int kN = raytab_floats(L);
    const float4* t4 = reinterpret_cast<const float4*>(raytab + ray * kN);
    float t[kN];
#pragma unroll
    for (int i = 0; i < kN / 4; ++i) {
        const float4 a = t4[i];
        t[4 * i] = a.x;
        t[4 * i + 1] = a.y;
        t[4 * i + 2] = a.z;
        t[4 * i + 3] = a.w;
    }
    dx = t[0];
    dy = t[1];
    dz = t[2];
#pragma unroll
    for (int l = 0; l < L; ++l) P[l] = t[3 + l];
#pragma unroll
    for (int n = 0; n < L * (L + 1); ++n) Y[n] = t[3 + L + n];
}

// Opacity-weighted Gaussian at the midpoint and its clamp (R1, R2): alpha = min(o g, amax).
__device__ __forceinline__ float pair_alpha(float o, float m2r, float amax, float& gw) {
    gw = __expf(-0.5f * m2r);
    return fminf(o * gw, amax);
}

// Transmittance phase rotation e^{-j theta}, theta = pi x, x = 2 f b dt / c, with x
// reduced exactly to [-1, 1] before the hardware sine / cosine.
__device__ __forceinline__ void phase_rot(float x, float& sn, float& cs) {
    const float xr = x - 2.0f * rintf(0.5f * x);
    __sincosf(3.14159265f * xr, &sn, &cs);
}

}  // namespace gsrf
