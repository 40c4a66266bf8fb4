// k_render.cu -- Alg. 1 lines 6-12 ("Blend"), Eq. 14 / App. A.3: per-ray complex
// front-to-back accumulation over the tile's depth-sorted Gaussians.
//
// One CTA per (receiver, 16x16 ray tile), one thread per ray.  The tile's candidates
// are staged kBatch at a time into shared memory (whitening matrix, whitened receiver
// offset, opacity, path phasor, excess-phase coefficient, 16 complex coefficients);
// every ray then tests them in list order.  A ray stops once prod(1 - alpha) drops
// below eps_T; the CTA stops when all its rays have (__syncthreads_count).
//
// Intersection in whitened coordinates: with W = diag(1/s) R^T, the ray point
// r + t v maps to w + t v' (w = W (r - mu), v' = W v), so the paper's quadratic
// A t^2 + 2 B t + (C - 9) = 0 (App. D.3) has A = |v'|^2, B = w.v', C = |w|^2 and the
// closest approach m2 = C - B^2/A = |w + t_mid v'|^2 at t_mid = -B/A.  Forming m2 as a
// squared norm avoids the cancellation of C - B^2/A in FP32 (C reaches 1e5 for small
// far Gaussians); the roots are t_mid +- sqrt((9 - m2)/A).
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

constexpr int kBatch = 128;

struct RenderArgs {
    const GShape* shape;
    const View* view;
    const float* coeffs;
    const uint32_t* pids;
    const long long* rx_base;
    const uint32_t* tile_start;
    float* out;
    RayState* rs;
    DevStatus* st;
    gsrf_grid gr;
    int ntu, n_tiles, n_rx;
    long long n;
    float omega0;  // 2 pi f0 / c
};

// Fourier-Legendre basis of one ray (Eq. 9): Y_n = e^{i m az} P_l^m(x), x = sin(el),
// n = l*l + l + m, P without the Condon-Shortley phase and
// P_l^{-m} = (-1)^m (l-m)!/(l+m)! P_l^m.
__device__ __forceinline__ void ray_basis(float az, float x, float sx, float* Yr, float* Yi) {
    float c1, s1, c2, s2, c3, s3;
    sincosf(az, &s1, &c1);
    sincosf(2.0f * az, &s2, &c2);
    sincosf(3.0f * az, &s3, &c3);
    const float x2 = x * x, sx2 = sx * sx;
    const float P00 = 1.0f;
    const float P10 = x, P11 = sx;
    const float P20 = 1.5f * x2 - 0.5f, P21 = 3.0f * x * sx, P22 = 3.0f * sx2;
    const float P30 = x * (2.5f * x2 - 1.5f), P31 = (7.5f * x2 - 1.5f) * sx, P32 = 15.0f * x * sx2,
                P33 = 15.0f * sx2 * sx;
    // m = 0
    Yr[0] = P00; Yi[0] = 0.0f;
    Yr[2] = P10; Yi[2] = 0.0f;
    Yr[6] = P20; Yi[6] = 0.0f;
    Yr[12] = P30; Yi[12] = 0.0f;
    // m = +-1: factor for -1 is -(l-1)!/(l+1)!
    Yr[3] = c1 * P11;  Yi[3] = s1 * P11;
    Yr[1] = -0.5f * c1 * P11; Yi[1] = 0.5f * s1 * P11;
    Yr[7] = c1 * P21;  Yi[7] = s1 * P21;
    Yr[5] = -(1.0f / 6.0f) * c1 * P21; Yi[5] = (1.0f / 6.0f) * s1 * P21;
    Yr[13] = c1 * P31; Yi[13] = s1 * P31;
    Yr[11] = -(1.0f / 12.0f) * c1 * P31; Yi[11] = (1.0f / 12.0f) * s1 * P31;
    // m = +-2: factor (l-2)!/(l+2)!
    Yr[8] = c2 * P22;  Yi[8] = s2 * P22;
    Yr[4] = (1.0f / 24.0f) * c2 * P22; Yi[4] = -(1.0f / 24.0f) * s2 * P22;
    Yr[14] = c2 * P32; Yi[14] = s2 * P32;
    Yr[10] = (1.0f / 120.0f) * c2 * P32; Yi[10] = -(1.0f / 120.0f) * s2 * P32;
    // m = +-3: factor -(l-3)!/(l+3)!
    Yr[15] = c3 * P33; Yi[15] = s3 * P33;
    Yr[9] = -(1.0f / 720.0f) * c3 * P33; Yi[9] = (1.0f / 720.0f) * s3 * P33;
}

__global__ void __launch_bounds__(kRenderThreads) k_render_fwd(RenderArgs a) {
    __shared__ float4 s_geo[kBatch][4];  // W0..W3 | W4..W7 | W8 w0 w1 w2 | o er ei b
    __shared__ float4 s_cf[kBatch][8];   // 16 complex coefficients
    __shared__ unsigned long long s_stats[2];

    const int tile = blockIdx.x, r = blockIdx.y;
    const int tu = tile % a.ntu, tv = tile / a.ntu;
    const int u = tu * kTile + (threadIdx.x & (kTile - 1));
    const int v = tv * kTile + (threadIdx.x / kTile);
    const gsrf_grid& gr = a.gr;
    const bool valid = u < gr.n_az && v < gr.n_el;
    if (threadIdx.x < 2) s_stats[threadIdx.x] = 0ull;

    const float deg = 0.0174532925199432958f;
    const float az = (gr.az0_deg + ((float)u + 0.5f) * gr.daz_deg) * deg;
    const float el = (gr.el0_deg + ((float)v + 0.5f) * gr.del_deg) * deg;
    float se, ce, sa, ca;
    sincosf(el, &se, &ce);
    sincosf(az, &sa, &ca);
    const float dx = ce * ca, dy = ce * sa, dz = se;
    float Yr[kNB], Yi[kNB];
    ray_basis(az, se, ce, Yr, Yi);

    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const long long base0 = a.rx_base[r];
    const long long lo = base0 + a.tile_start[ts], hi = base0 + a.tile_start[ts + 1];
    const float r_rx = gr.r_rx, eps_T = gr.eps_T, amax = gr.alpha_max;

    float Sr = 0.0f, Si = 0.0f, Tr = 1.0f, Ti = 0.0f, Ta = 1.0f;
    int last = -1;
    bool done = !valid;
    unsigned tests = 0, hits = 0;

    for (long long b0 = lo; b0 < hi; b0 += kBatch) {
        const int cnt = (int)min((long long)kBatch, hi - b0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const uint32_t id = a.pids[b0 + threadIdx.x];
            const float4* sh = reinterpret_cast<const float4*>(a.shape + id);
            const float4* vw = reinterpret_cast<const float4*>(a.view + (size_t)r * a.n + id);
            const float4 g0 = sh[0], g1 = sh[1], g2 = sh[2];  // W0-3, W4-7, W8 o b pad
            const float4 v0 = vw[0], v1 = vw[1];              // w0 w1 w2 er, ei omd - -
            s_geo[threadIdx.x][0] = g0;
            s_geo[threadIdx.x][1] = g1;
            s_geo[threadIdx.x][2] = make_float4(g2.x, v0.x, v0.y, v0.z);
            s_geo[threadIdx.x][3] = make_float4(g2.y, v0.w, v1.x, g2.z);
            const float4* cf = reinterpret_cast<const float4*>(a.coeffs + (size_t)id * 2 * kNB);
#pragma unroll
            for (int q = 0; q < 8; ++q) s_cf[threadIdx.x][q] = cf[q];
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 g0 = s_geo[j][0], g1 = s_geo[j][1], g2 = s_geo[j][2];
                const float vx = g0.x * dx + g0.y * dy + g0.z * dz;
                const float vy = g0.w * dx + g1.x * dy + g1.y * dz;
                const float vz = g1.z * dx + g1.w * dy + g2.x * dz;
                const float A = vx * vx + vy * vy + vz * vz;
                const float B = g2.y * vx + g2.z * vy + g2.w * vz;
                const float iA = 1.0f / A;
                const float tm = -B * iA;
                const float px = g2.y + tm * vx, py = g2.z + tm * vy, pz = g2.w + tm * vz;
                const float m2 = px * px + py * py + pz * pz;
                ++tests;
                if (m2 >= 9.0f) continue;
                const float h = sqrtf((9.0f - m2) * iA);
                const float t_out = tm + h;
                if (t_out < r_rx) continue;
                // hit: chord beyond the emitting sphere, midpoint weight (App. A.2)
                const float t_a = fmaxf(tm - h, r_rx);
                const float dt = t_out - t_a;
                const float dl = 0.5f * (t_a + t_out) - tm;
                const float m2r = m2 + A * dl * dl;
                const float4 g3 = s_geo[j][3];
                const float alpha = fminf(g3.x * expf(-0.5f * m2r), amax);
                float pr = 0.0f, pi = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 c = s_cf[j][q];
                    pr += c.x * Yr[2 * q] - c.y * Yi[2 * q] + c.z * Yr[2 * q + 1] - c.w * Yi[2 * q + 1];
                    pi += c.x * Yi[2 * q] + c.y * Yr[2 * q] + c.z * Yi[2 * q + 1] + c.w * Yr[2 * q + 1];
                }
                // E_k T
                const float etr = g3.y * Tr - g3.z * Ti, eti = g3.y * Ti + g3.z * Tr;
                Sr += alpha * (pr * etr - pi * eti);
                Si += alpha * (pr * eti + pi * etr);
                float sn, cs;
                sincosf(a.omega0 * g3.w * dt, &sn, &cs);
                const float om = 1.0f - alpha;
                const float nTr = om * (Tr * cs + Ti * sn);
                Ti = om * (Ti * cs - Tr * sn);
                Tr = nTr;
                Ta *= om;
                ++hits;
                last = (int)(b0 - base0) + j;
                if (Ta < eps_T) {
                    done = true;
                    break;
                }
            }
        }
        if (__syncthreads_count(!done) == 0) break;
    }

    if (valid) {
        const size_t ray = ((size_t)r * gr.n_el + v) * gr.n_az + u;  // n_f == 1
        reinterpret_cast<float2*>(a.out)[ray] = make_float2(Sr, Si);
        if (a.rs) {
            RayState s;
            s.last = last;
            s.Ta = Ta;
            s.Tr = Tr;
            s.Ti = Ti;
            a.rs[ray] = s;
        }
    }
    // statistics: candidate tests and composited pairs
    unsigned long long t64 = tests, h64 = hits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t64 += __shfl_down_sync(0xffffffffu, t64, o);
        h64 += __shfl_down_sync(0xffffffffu, h64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_stats[0], t64);
        atomicAdd(&s_stats[1], h64);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.st->stats[0], s_stats[0]);
        atomicAdd(&a.st->stats[1], s_stats[1]);
    }
}

cudaError_t launch_render_fwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, void* ws,
                              float* out, void* ray_state, cudaStream_t st) {
    RenderArgs a;
    a.shape = at<GShape>(ws, L.gshape);
    a.view = at<View>(ws, L.view);
    a.coeffs = g->coeffs;
    a.pids = at<uint32_t>(ws, L.pids);
    a.rx_base = at<long long>(ws, L.rx_base);
    a.tile_start = at<uint32_t>(ws, L.tile_start);
    a.out = out;
    a.rs = static_cast<RayState*>(ray_state);
    a.st = at<DevStatus>(ws, L.status);
    a.gr = p->grid;
    a.ntu = L.ntu;
    a.n_tiles = L.n_tiles;
    a.n_rx = L.n_rx;
    a.n = L.n;
    a.omega0 = (float)(2.0 * 3.14159265358979323846 * p->f0_hz / kC);
    cudaError_t e = cudaMemsetAsync(&a.st->stats[0], 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_render_fwd<<<dim3(L.n_tiles, L.n_rx), kRenderThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gsrf
