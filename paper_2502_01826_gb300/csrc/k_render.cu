// k_render.cu -- Alg. 1 lines 6-12 ("Blend"), Eq. 14 / App. A.3: per-ray complex
// front-to-back accumulation over the tile's depth-sorted Gaussians.
//
// Layout of the work: a CTA of 4 warps covers half of a 16x16 ray tile (16 x 8 rays),
// each warp an 8 x 4 block of rays, one ray per thread.  Every warp walks its tile's
// candidate list on its own, 32 candidates per batch: lane i takes candidate b0 + i,
// tests its direction cone against the cone of the warp's 32 rays and its ellipsoid
// against four planes that bound those rays and, if it may be hit, copies its
// records into the warp's half of a double buffer with cp.async while
// the warp works on the current batch; the rays then visit only the candidates of the
// ballot mask, in list order.  Warps never wait for one another and a warp leaves as
// soon as its 32 rays have terminated (prod(1 - alpha) < eps_T).
//
// Per candidate and ray (pair_cone / pair_hits, shared with the backward):
//   (1) direction cone: v lies in the cone of directions that meet the bounding sphere
//       of the 3-sigma ellipsoid beyond the emitting sphere, c.v >= D cos(theta);
//   (2) 3-sigma ellipsoid in whitened coordinates: with W = diag(1/s) R^T the ray
//       r + t v maps to w + t v' (w = W (r - mu), v' = W v), so the paper's quadratic
//       A t^2 + 2 B t + (C - 9) = 0 (App. D.3) has A = |v'|^2, B = w.v', C = |w|^2;
//       the closest approach is m2 = C - B^2/A = |w x v'|^2 / A (Lagrange's identity),
//       free of the cancellation of C - B^2/A in FP32 (C reaches 1e5);
//   (3) the chord t_mid +- sqrt((9 - m2)/A) must reach r_rx; it is clipped there and
//       the Gaussian is weighted at the midpoint of the clipped chord (App. A.2).
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

constexpr int kWarps = 4;        // warps per CTA: half a 16 x 16 tile (16 x 8 rays)
constexpr int kThreads = 32 * kWarps;
constexpr int kWB = 32;          // candidates per warp batch, one per lane
constexpr int kRec = 6;          // float4 per staged candidate: 3 of View, 3 of GShape

struct RenderArgs {
    const GShape* shape;
    const View* view;
    const float* fle;
    const float* raytab;
    const uint32_t* pids;
    const long long* rx_base;
    const uint32_t* tile_start;
    float* out;
    RayState* rs;
    DevStatus* st;
    gsrf_grid gr;
    int ntu, n_tiles, n_rx;
    long long n;
    float om_pi;  // 2 f0 / c: sincospi argument per unit of b dt
    int n_f;      // frequencies f0 + s df
    float dlt;    // 2 pi df / c: subcarrier phase step per metre of excess path
};

constexpr int kMaxJobs = 96;

// Up to kMaxJobs render problems (one receiver group of one scene each) passed by value
// to the persistent kernel; item_base[j] is the first work item of job j.
struct BatchArgs {
    int n_jobs;
    unsigned long long item_base[kMaxJobs + 1];
    RenderArgs jobs[kMaxJobs];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Ray of thread t: CTA half h of the 16 x 16 tile holds rows 8h .. 8h+7; each warp an
// 8 x 4 block of rays so that its lanes see nearly the same candidates.
__device__ __forceinline__ void cta_ray(int t, int half, int& lx, int& ly) {
    const int lane = t & 31, w = t >> 5;
    lx = ((w & 1) << 3) | (lane & 7);
    ly = (half << 3) | ((w >> 1) << 2) | (lane >> 3);
}

// Radiance psi of one Gaussian along one ray (Eq. 9) from the folded coefficients q
// (see kFle) and the ray's basis values: P = (P10, P20, P30), Y = six complex Y_{l,m>0}.
__device__ __forceinline__ void fle_psi(const float4* __restrict__ q4, const float* P, const float* Y,
                                        float& pr, float& pi) {
    const float4 a0 = __ldg(q4), a1 = __ldg(q4 + 1);
    pr = a0.x + a0.z * P[0] + a1.x * P[1] + a1.z * P[2];
    pi = a0.y + a0.w * P[0] + a1.y * P[1] + a1.w * P[2];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const float4 e = __ldg(q4 + 2 + t);
        pr += e.x * Y[2 * t] + e.y * Y[2 * t + 1];
        pi += e.z * Y[2 * t] + e.w * Y[2 * t + 1];
    }
}

// The ray's direction and basis values from the per-grid ray table.
__device__ __forceinline__ void load_ray(const float* raytab, size_t ray, float& dx, float& dy, float& dz,
                                         float* P, float* Y) {
    const float4* t4 = reinterpret_cast<const float4*>(raytab + ray * kRayTab);
    const float4 t0 = t4[0], t1 = t4[1], t2 = t4[2], t3 = t4[3], t5 = t4[4];
    dx = t0.x; dy = t0.y; dz = t0.z; P[0] = t0.w;
    P[1] = t1.x; P[2] = t1.y; Y[0] = t1.z; Y[1] = t1.w;
    Y[2] = t2.x; Y[3] = t2.y; Y[4] = t2.z; Y[5] = t2.w;
    Y[6] = t3.x; Y[7] = t3.y; Y[8] = t3.z; Y[9] = t3.w;
    Y[10] = t5.x; Y[11] = t5.y;
}

// One warp renders the 8 x 4 block wq (0..7) of rays of tile `tile` for receiver r: it
// walks the tile's list in batches of 32 candidates staged into its own buffers
// (sbuf, sid), without waiting for any other warp.
//
// NFC = 1: one frequency.  NFC > 1: the lanes handle subcarriers s0 .. s0 + NFC - 1
// (s0 = chunk * NFC); the contribution of a pair at f0 + s df is z0 r^s with
// r = e^{-j (2 pi df d / c + 2 pi df Gamma / c)}, Gamma = sum over earlier pairs of b dt,
// because T(f0 + s df) = T(f0) e^{-j s 2 pi df Gamma / c} and E(f0 + s df) =
// E(f0) e^{-j s 2 pi df d / c}; the powers of r come from one sincos and a recurrence.
template <int NFC>
__device__ __forceinline__ void render_block(const RenderArgs& a, int r, int tile, int wq, int chunk,
                                             float4 (*sbuf)[kWB][kRec], uint32_t (*sid)[kWB], float4* spl) {
    const int lane = threadIdx.x & 31;
    const int tu = tile % a.ntu, tv = tile / a.ntu;
    const int lx = ((wq & 1) << 3) | (lane & 7);
    const int ly = ((wq >> 1) << 2) | (lane >> 3);
    const int u = tu * kTile + lx, v = tv * kTile + ly;
    const gsrf_grid& gr = a.gr;
    const bool valid = u < gr.n_az && v < gr.n_el;

    float dx = 0.0f, dy = 0.0f, dz = 1.0f, P[3] = {0.0f, 0.0f, 0.0f}, Y[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) Y[i] = 0.0f;
    if (valid) load_ray(a.raytab, (size_t)v * gr.n_az + u, dx, dy, dz, P, Y);
    const Bundle bun = warp_bundle(valid, dx, dy, dz);
    warp_planes(gr, tu * kTile + ((wq & 1) << 3), tv * kTile + ((wq >> 1) << 2), bun, valid, dx, dy, dz, spl);

    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const long long base0 = a.rx_base[r];
    const long long lo = base0 + a.tile_start[ts], hi = base0 + a.tile_start[ts + 1];
    const float r_rx = gr.r_rx, eps_T = gr.eps_T, amax = gr.alpha_max;
    const View* __restrict__ view = a.view + (size_t)r * a.n;

    float Sr = 0.0f, Si = 0.0f, Tr = 1.0f, Ti = 0.0f, Ta = 1.0f;
    float Sf[2 * NFC];
#pragma unroll
    for (int i = 0; i < 2 * NFC; ++i) Sf[i] = 0.0f;
    float Gam = 0.0f;
    const int s0 = chunk * NFC;
    int last = -1;
    bool done = !valid;
    unsigned tests = 0, hits = 0;

    // Stage the batch starting at b0 into buffer bf: lane i takes candidate b0 + i,
    // tests its bounding sphere against the warp's cone and, if it may be hit, copies
    // its records; returns the mask of candidates that may be hit.
    auto stage = [&](int bf, long long b0) -> uint32_t {
        bool keep = false;
        if (b0 + lane < hi) {
            const uint32_t id = a.pids[b0 + lane];
            const float4* vw = reinterpret_cast<const float4*>(view + id);
            const float4 c = __ldg(vw);
            keep = bundle_meets(bun, c) && planes_meet(spl, c, a.shape + id);
            if (keep) {
                sid[bf][lane] = id;
                const float4* sh = reinterpret_cast<const float4*>(a.shape + id);
                float4* dst = sbuf[bf][lane];
                dst[0] = c;
                cp_async16(dst + 1, vw + 1);
                cp_async16(dst + 2, vw + 2);
                cp_async16(dst + 3, sh + 0);
                cp_async16(dst + 4, sh + 1);
                cp_async16(dst + 5, sh + 2);
                asm volatile("prefetch.global.L1 [%0];\n" ::"l"(a.fle + (size_t)id * kFle));
            }
        }
        cp_async_commit();
        return __ballot_sync(0xffffffffu, keep);
    };

    if (!__all_sync(0xffffffffu, done)) {
        int bf = 0;
        uint32_t mask = stage(0, lo);
        for (long long b0 = lo; b0 < hi; b0 += kWB, bf ^= 1) {
            const uint32_t next = stage(bf ^ 1, b0 + kWB);  // empty past the end of the list
            cp_async_wait_prev();
            __syncwarp();
            const int cnt = (int)min((long long)kWB, hi - b0);
            if (!done) {
                int stop = cnt;
                for (uint32_t m = mask; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    const float4* rec = sbuf[bf][j];
                    if (!pair_cone(rec[0], dx, dy, dz)) continue;
                    const float4 v1 = rec[1], s2 = rec[5];
                    PairGeo pg;
                    if (!pair_hits(v1, rec[3], rec[4], s2, dx, dy, dz, r_rx, pg)) continue;
                    float gw;
                    const float alpha = pair_alpha(s2.y, pg.m2r, amax, gw);
                    float pr, pi;
                    fle_psi(reinterpret_cast<const float4*>(a.fle + (size_t)sid[bf][j] * kFle), P, Y, pr, pi);
                    // S += alpha psi E T, E = e^{-j phi} = (er, ei)
                    const float er = v1.w, ei = rec[2].x;
                    const float etr = er * Tr - ei * Ti, eti = er * Ti + ei * Tr;
                    if constexpr (NFC == 1) {
                        Sr += alpha * (pr * etr - pi * eti);
                        Si += alpha * (pr * eti + pi * etr);
                    } else {
                        // z at the chunk's first subcarrier, then one rotation per step
                        const float ws = rec[2].y + a.dlt * Gam;
                        float rs, rc, ss, sc;
                        sincosf(ws, &rs, &rc);
                        sincosf((float)s0 * ws, &ss, &sc);
                        const float z0r = alpha * (pr * etr - pi * eti), z0i = alpha * (pr * eti + pi * etr);
                        float zr = z0r * sc + z0i * ss, zi = z0i * sc - z0r * ss;
#pragma unroll
                        for (int q = 0; q < NFC; ++q) {
                            Sf[2 * q] += zr;
                            Sf[2 * q + 1] += zi;
                            const float nzr = zr * rc + zi * rs;
                            zi = zi * rc - zr * rs;
                            zr = nzr;
                        }
                        Gam += s2.z * pg.dt;
                    }
                    // T *= (1 - alpha) e^{-j theta}, theta = 2 pi f0 b dt / c
                    float sn, cs;
                    phase_rot(a.om_pi * s2.z * pg.dt, sn, cs);
                    const float om = 1.0f - alpha;
                    const float nTr = om * (Tr * cs + Ti * sn);
                    Ti = om * (Ti * cs - Tr * sn);
                    Tr = nTr;
                    Ta *= om;
                    ++hits;
                    last = (int)(b0 - lo) + j;  // position inside the tile's list
                    if (Ta < eps_T) {
                        done = true;
                        stop = j + 1;
                        break;
                    }
                }
                tests += (unsigned)stop;
            }
            mask = next;
            __syncwarp();
            if (__all_sync(0xffffffffu, done)) break;
        }
        cp_async_wait_all();
    }

    if (valid) {
        const size_t plane = (size_t)gr.n_el * gr.n_az, pix = (size_t)v * gr.n_az + u;
        const size_t ray = (size_t)r * plane + pix;
        if constexpr (NFC == 1) {
            reinterpret_cast<float2*>(a.out)[ray] = make_float2(Sr, Si);
        } else {
            float2* o2 = reinterpret_cast<float2*>(a.out) + ((size_t)r * a.n_f + s0) * plane + pix;
#pragma unroll
            for (int q = 0; q < NFC; ++q)
                if (s0 + q < a.n_f) o2[(size_t)q * plane] = make_float2(Sf[2 * q], Sf[2 * q + 1]);
        }
        if (a.rs && chunk == 0) {
            RayState s;
            s.last = last;
            s.Ta = Ta;
            s.Tr = Tr;
            s.Ti = Ti;
            s.Gam = Gam;
            s.pad[0] = s.pad[1] = s.pad[2] = 0.0f;
            a.rs[ray] = s;
        }
    }
    // statistics: list positions tested and composited pairs, one atomic per warp
    unsigned long long t64 = tests, h64 = hits;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t64 += __shfl_down_sync(0xffffffffu, t64, o);
        h64 += __shfl_down_sync(0xffffffffu, h64, o);
    }
    if (lane == 0 && chunk == 0) {
        atomicAdd(&a.st->stats[0], t64);
        atomicAdd(&a.st->stats[1], h64);
    }
}

// Plain launch: CTA = (half tile, receiver, subcarrier chunk), 4 warps = 4 ray blocks.
template <int NFC>
__global__ void __launch_bounds__(kThreads, NFC == 1 ? 8 : 4) k_render_fwd(RenderArgs a) {
    __shared__ float4 sbuf[kWarps][2][kWB][kRec];
    __shared__ uint32_t sid[kWarps][2][kWB];
    __shared__ float4 spl[kWarps][4];
    const int warp = threadIdx.x >> 5;
    render_block<NFC>(a, blockIdx.y, blockIdx.x >> 1, (blockIdx.x & 1) * kWarps + warp, blockIdx.z, sbuf[warp],
                      sid[warp], spl[warp]);
}

// Persistent batched launch: every warp takes work items -- (job, receiver, tile, ray
// block) -- from one counter, in the heaviest-first order the item sort produced, until
// none is left.  No warp waits for another.
__global__ void __launch_bounds__(kThreads, 8) k_render_batch(BatchArgs b, const uint32_t* __restrict__ order,
                                                              unsigned long long* __restrict__ counter) {
    __shared__ float4 sbuf[kWarps][2][kWB][kRec];
    __shared__ uint32_t sid[kWarps][2][kWB];
    __shared__ float4 spl[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long total = b.item_base[b.n_jobs];
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        const unsigned long long id = order[it];
        int j = 0;
        while (j + 1 < b.n_jobs && b.item_base[j + 1] <= id) ++j;
        const RenderArgs& a = b.jobs[j];
        const unsigned long long local = id - b.item_base[j];
        const int per_rx = a.n_tiles * 8;
        const int r = (int)(local / per_rx), rem = (int)(local % per_rx);
        render_block<1>(a, r, rem >> 3, rem & 7, 0, sbuf[warp], sid[warp], spl[warp]);
    }
}

// Persistent launch of one problem (n_f = 1): like k_render_batch, every warp takes work
// items (receiver, tile, ray block) from one counter, in the heaviest-first order of
// k_queue_keys, until none is left; a warp that finishes early takes the next item
// instead of idling until the other warps of its CTA are done.
__global__ void __launch_bounds__(kThreads, 8) k_render_queue(RenderArgs a, const uint32_t* __restrict__ order,
                                                              unsigned long long* __restrict__ counter,
                                                              unsigned long long total) {
    __shared__ float4 sbuf[kWarps][2][kWB][kRec];
    __shared__ uint32_t sid[kWarps][2][kWB];
    __shared__ float4 spl[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_rx = a.n_tiles * 8;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        const uint32_t id = order[it];
        const int r = (int)(id / (uint32_t)per_rx), rem = (int)(id % (uint32_t)per_rx);
        render_block<1>(a, r, rem >> 3, rem & 7, 0, sbuf[warp], sid[warp], spl[warp]);
    }
}

__global__ void k_queue_keys(RenderArgs a, unsigned long long total, uint32_t* __restrict__ keys) {
    const unsigned long long id = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total) return;
    const int per_rx = a.n_tiles * 8;
    const int r = (int)(id / per_rx), tile = (int)(id % per_rx) >> 3;
    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const uint32_t len = a.tile_start[ts + 1] - a.tile_start[ts];
    keys[id] = (uint32_t)__clz((int)(len + 1u));  // 31 - floor(log2(len + 1))
}

// Cost key of every work item: its tile's list length, heaviest first (bucket
// 31 - floor(log2(len + 1)), so that an ascending stable sort puts long lists first).
__global__ void k_batch_keys(BatchArgs b, uint32_t* __restrict__ keys) {
    const unsigned long long id = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= b.item_base[b.n_jobs]) return;
    int j = 0;
    while (j + 1 < b.n_jobs && b.item_base[j + 1] <= id) ++j;
    const RenderArgs& a = b.jobs[j];
    const unsigned long long local = id - b.item_base[j];
    const int per_rx = a.n_tiles * 8;
    const int r = (int)(local / per_rx), tile = (int)(local % per_rx) >> 3;
    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const uint32_t len = a.tile_start[ts + 1] - a.tile_start[ts];
    keys[id] = 31u - (31u - (uint32_t)__clz((int)(len + 1u)));
}

static RenderArgs render_args(const gsrf_plan* p, const Layout& L, void* ws, float* out, void* ray_state) {
    RenderArgs a;
    a.shape = at<GShape>(ws, L.gshape);
    a.view = at<View>(ws, L.view);
    a.fle = at<float>(ws, L.fle);
    a.raytab = at<float>(ws, L.raytab);
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
    a.om_pi = (float)(2.0 * p->f0_hz / kC);
    a.n_f = p->n_f;
    a.dlt = (float)(2.0 * 3.14159265358979323846 * p->df_hz / kC);
    return a;
}

cudaError_t launch_render_fwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, void* ws,
                              float* out, void* ray_state, cudaStream_t st) {
    RenderArgs a = render_args(p, L, ws, out, ray_state);
    (void)g;
    cudaError_t e = cudaMemsetAsync(&a.st->stats[0], 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (p->n_f == 1) {
        // persistent: heaviest-first work queue over (receiver, tile, ray block) items
        const long long n = (long long)L.n_rx * L.n_tiles * 8;
        uint32_t* keys = at<uint32_t>(ws, L.qkeys);
        uint32_t* keys2 = at<uint32_t>(ws, L.qkeys2);
        uint32_t* order = at<uint32_t>(ws, L.qorder);
        uint32_t* hist = at<uint32_t>(ws, L.qhist);
        unsigned long long* counter = at<unsigned long long>(ws, L.qcounter);
        k_queue_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, (unsigned long long)n, keys);
        if ((e = launch_sort_small_keys(keys, keys2, order, n, 32, hist, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_queue, kThreads, 0)) != cudaSuccess)
            return e;
        const long long ctas_needed = (n + kWarps - 1) / kWarps;
        const int grid = (int)min((long long)sms * max(per_sm, 1), ctas_needed);
        k_render_queue<<<grid, kThreads, 0, st>>>(a, order, counter, (unsigned long long)n);
    } else if (p->n_f <= 8) {
        k_render_fwd<8><<<dim3(2 * L.n_tiles, L.n_rx, 1), kThreads, 0, st>>>(a);
    } else {
        k_render_fwd<16><<<dim3(2 * L.n_tiles, L.n_rx, (p->n_f + 15) / 16), kThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace gsrf

namespace gsrf {

static long long batch_items(int n_jobs, const gsrf_plan* plans) {
    long long t = 0;
    for (int j = 0; j < n_jobs; ++j) {
        Layout L;
        make_layout(&plans[j], &L);
        t += (long long)L.n_rx * L.n_tiles * 8;
    }
    return t;
}

// batch workspace: keys, sorted keys, order, histogram, counter
size_t batch_workspace_bytes(int n_jobs, const gsrf_plan* plans) {
    const long long n = batch_items(n_jobs, plans);
    const long long chunks = (n + kChunk - 1) / kChunk;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(n * 4) * 3 + al(chunks * 32 * 4) + al(8);
}

cudaError_t launch_render_batch(int n_jobs, const gsrf_plan* plans, void* const* workspaces, float* const* outs,
                                void* batch_ws, cudaStream_t st) {
    BatchArgs b;
    b.n_jobs = n_jobs;
    unsigned long long base = 0;
    for (int j = 0; j < n_jobs; ++j) {
        Layout L;
        make_layout(&plans[j], &L);
        b.jobs[j] = render_args(&plans[j], L, workspaces[j], outs[j], nullptr);
        b.item_base[j] = base;
        base += (unsigned long long)L.n_rx * L.n_tiles * 8;
        cudaError_t e = cudaMemsetAsync(&b.jobs[j].st->stats[0], 0, 2 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    b.item_base[n_jobs] = base;
    const long long n = (long long)base;
    const long long chunks = (n + kChunk - 1) / kChunk;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* w = static_cast<char*>(batch_ws);
    uint32_t* keys = reinterpret_cast<uint32_t*>(w);
    uint32_t* keys2 = reinterpret_cast<uint32_t*>(w + al(n * 4));
    uint32_t* order = reinterpret_cast<uint32_t*>(w + 2 * al(n * 4));
    uint32_t* hist = reinterpret_cast<uint32_t*>(w + 3 * al(n * 4));
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(w + 3 * al(n * 4) + al(chunks * 32 * 4));
    if (n == 0) return cudaSuccess;
    k_batch_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b, keys);
    cudaError_t e = launch_sort_small_keys(keys, keys2, order, n, 32, hist, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    // one resident wave: every SM holds as many CTAs as it can run at once
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_batch, kThreads, 0)) != cudaSuccess)
        return e;
    const long long ctas_needed = (n + kWarps - 1) / kWarps;
    const int grid = (int)min((long long)sms * max(per_sm, 1), ctas_needed);
    k_render_batch<<<grid, kThreads, 0, st>>>(b, order, counter);
    return cudaGetLastError();
}

}  // namespace gsrf
