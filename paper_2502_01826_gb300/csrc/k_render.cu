// k_render.cu -- Alg. 1's blend loop, Eq. 14 / App. A.3: per-ray complex
// front-to-back accumulation over the tile's depth-sorted Gaussians.
//
// Layout of the work: a work item is one warp's block of bw x bh = 32 rays (one ray per
// lane) inside one tile of one receiver, for one chunk of subcarriers.  The tile shape
// comes from the grid (tile_w x tile_h), the block width from the plan (bw in 4..32,
// default 8 x 4), so a tile holds (tile_w / bw) (tile_h / bh) blocks.  A persistent wave
// of CTAs takes items from one counter in heaviest-first order (tile list length), so a
// warp that finishes early takes the next item.
//
// Each warp walks its tile's candidate list on its own, WB (16 or 32, from the plan)
// candidates per batch: lane i < WB takes candidate p0 + i, tests its direction cone
// against the cone of the warp's rays and its ellipsoid against five half-spaces that
// hold those rays beyond the emitting sphere (warp_planes) and, if it may be hit,
// copies its records into the warp's half of a double buffer with cp.async while the
// warp works on the current batch (the cone test's input, and the list ids, are fetched
// one and two batches earlier still); the rays then visit only the candidates of the
// ballot mask, in list order.  A warp's item ends as soon as its 32 rays have
// terminated (prod(1 - alpha) < eps_T).  After the warp-level tests, nine in ten rays
// would pass a per-ray direction-cone test, so the forward goes straight to the exact
// test.
//
// Per candidate and ray (pair_hits, shared with the backward):
//   (1) 3-sigma ellipsoid in whitened coordinates: with W = diag(1/s) R^T the ray
//       r + t v maps to w + t v' (w = W (r - mu), v' = W v), so the paper's quadratic
//       A t^2 + 2 B t + (C - 9) = 0 (App. D.3) has A = |v'|^2, B = w.v', C = |w|^2;
//       the closest approach is m2 = C - B^2/A = |w x v'|^2 / A (Lagrange's identity),
//       free of the cancellation of C - B^2/A in FP32 (C reaches 1e5);
//   (2) the chord t_mid +- sqrt((9 - m2)/A) must reach r_rx; it is clipped there and
//       the Gaussian is weighted at the midpoint of the clipped chord (App. A.2).
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

constexpr int kWarps = 4;        // warps per CTA, each on its own work items
constexpr int kThreads = 32 * kWarps;
// float4 per staged candidate: View floats 4..11 (w, er | ei, omd, psi at the mean) and
// the first 48 bytes of GShape (W, o, b); the forward needs no c or D cos(theta) per ray
constexpr int kRec = 5;
// Per batch, the Fourier-Legendre coefficients (L = 3: 128 bytes) of the first kCoefSlots
// candidates of the ballot mask are staged with their records, in mask order, so that
// their radiance reads shared memory instead of a cold global line; later candidates of
// the batch read global memory.  Seven slots (7 KB per CTA) keep 7 CTAs per SM.
constexpr int kCoefSlots = 7;

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
    int bw_log;   // log2 of the ray-block width bw (block height 32 / bw)
    int nbx;      // ray blocks per tile along azimuth (tile_w / bw)
    int per_tile; // work items per tile: ray blocks x subcarrier chunks
    int nchunk;   // subcarrier chunks
    float4* ck;   // transmittance checkpoints [slot][ray] (Tr, Ti, Gamma, Ta), or null
    int ck_every; // list positions between checkpoints (a multiple of 32)
    int ck_slots;
    int variant;  // GSRF_VARIANT_* bits
    const float4* circle;  // the paper's splatting circles [receiver][Gaussian] (that variant only)
    const float* rxpos;    // receiver and transmitter positions (the path-through-x_rep variant)
    const float* txpos;
    unsigned long long* tbuf;  // per-ray hit keys of the t_mid-order variant [ray][kOrderCap]
};

// Path of a composited pair through its representative point (plan variant
// GSRF_VARIANT_PATH_AT_REP): delta = (|t - x_rep| + |x_rep - r|) - (|t - mu| + |mu - r|)
// with x_rep = r + t_rep v.  Written without cancellation: e = x_rep - mu is the closest
// approach's offset from mu, W^-1 (w + t_mid v') = M^T (v' x (w x v')) / A (Lagrange's
// identity on the whitened quantities of the hit test), plus (t_rep - t_mid) v; then
// |c + e| - |c| = (2 c.e + e.e) / (|c + e| + |c|) for c = mu - r (|c + e| = t_rep) and for
// c = mu - t.  FP32 gives delta to about 1e-8 m, far below a wavelength.
__device__ __forceinline__ float path_delta(const float4& cv, const GShape* sh, const float4& w, const PairGeo& g,
                                            float dx, float dy, float dz, float tx, float ty, float tz) {
    const float4* m4 = reinterpret_cast<const float4*>(sh) + 3;
    const float4 m0 = __ldg(m4), m1 = __ldg(m4 + 1), m2 = __ldg(m4 + 2);
    const float M[9] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x};
    const float cx = w.y * g.vz - w.z * g.vy, cy = w.z * g.vx - w.x * g.vz, cz = w.x * g.vy - w.y * g.vx;
    const float px = (g.vy * cz - g.vz * cy) * g.iA, py = (g.vz * cx - g.vx * cz) * g.iA,
                pz = (g.vx * cy - g.vy * cx) * g.iA;
    const float ex = M[0] * px + M[3] * py + M[6] * pz + g.dl * dx;
    const float ey = M[1] * px + M[4] * py + M[7] * pz + g.dl * dy;
    const float ez = M[2] * px + M[5] * py + M[8] * pz + g.dl * dz;
    const float ee = ex * ex + ey * ey + ez * ez;
    const float D = sqrtf(cv.x * cv.x + cv.y * cv.y + cv.z * cv.z);
    const float t_rep = g.tm + g.dl;
    const float dr = (2.0f * (cv.x * ex + cv.y * ey + cv.z * ez) + ee) / (t_rep + D);
    const float qx = cv.x - tx, qy = cv.y - ty, qz = cv.z - tz;  // mu - t
    const float Q = sqrtf(qx * qx + qy * qy + qz * qz);
    const float Qe = sqrtf((qx + ex) * (qx + ex) + (qy + ey) * (qy + ey) + (qz + ez) * (qz + ez));
    const float dt = (2.0f * (qx * ex + qy * ey + qz * ez) + ee) / (Qe + Q);
    return dr + dt;
}

// Jobs of a batched launch are described by a table of RenderArgs in device memory (the
// batch workspace), written by k_put_jobs from chunks of kJobsPerPut passed by value.
constexpr int kJobsPerPut = 48;

struct JobChunk {
    int first, count, n_bases;  // n_bases = count, + 1 in the last chunk (the item total)
    unsigned long long item_base[kJobsPerPut + 1];
    uint32_t chunk_base[kJobsPerPut + 1];  // prefix of ceil(items / kChunk) (the job-order sort)
    RenderArgs jobs[kJobsPerPut];
};
static_assert(sizeof(JobChunk) <= 32000, "kernel parameters are limited to 32764 bytes");

// The SM's global nanosecond timer (the same clock on every SM).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Job of work item id: the last j with item_base[j] <= id (item_base ascending, n_jobs + 1
// entries, item_base[0] = 0).
__device__ __forceinline__ int job_of(const unsigned long long* __restrict__ item_base, int n_jobs,
                                      unsigned long long id) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_base[mid] <= id) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One warp renders work item k (ray block k / nchunk, subcarrier chunk k % nchunk) of
// tile `tile` for receiver r: it walks the tile's list in batches of WB candidates staged
// into its own buffers (sbuf, sid), without waiting for any other warp.
//
// NFC = 1: one frequency.  NFC > 1: the lanes handle subcarriers s0 .. s0 + NFC - 1
// (s0 = chunk * NFC); the contribution of a pair at f0 + s df is z0 r^s with
// r = e^{-j (2 pi df d / c + 2 pi df Gamma / c)}, Gamma = sum over earlier pairs of b dt,
// because T(f0 + s df) = T(f0) e^{-j s 2 pi df Gamma / c} and E(f0 + s df) =
// E(f0) e^{-j s 2 pi df d / c}; the powers of r come from one sincos and a recurrence.
template <int NFC, int WB, int L, bool PATH = false, bool ORDER = false>
__device__ __forceinline__ void render_block(const RenderArgs& a, int r, int tile, int k,
                                             float4 (*sbuf)[WB][kRec], uint32_t (*sid)[WB], float4* spl,
                                             float4 (*stin)[1], float4 (*scoef)[kCoefSlots][8]) {
    const int lane = threadIdx.x & 31;
    const gsrf_grid& gr = a.gr;
    const int chunk = k % a.nchunk, blk = k / a.nchunk;
    const int bw = 1 << a.bw_log, bh = 32 >> a.bw_log;
    const int tu = tile % a.ntu, tv = tile / a.ntu;
    const int u_lo = tu * gr.tile_w + (blk % a.nbx) * bw, v_lo = tv * gr.tile_h + (blk / a.nbx) * bh;
    const int u = u_lo + (lane & (bw - 1)), v = v_lo + (lane >> a.bw_log);
    const bool valid = u < gr.n_az && v < gr.n_el;

    float dx = 0.0f, dy = 0.0f, dz = 1.0f, P[L], Y[L * (L + 1)];
#pragma unroll
    for (int i = 0; i < L; ++i) P[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < L * (L + 1); ++i) Y[i] = 0.0f;
    if (valid) load_ray<L>(a.raytab, (size_t)v * gr.n_az + u, dx, dy, dz, P, Y);
    const Bundle bun = warp_bundle(valid, dx, dy, dz);
    warp_planes(gr, u_lo, v_lo, bw, bh, bun, valid, dx, dy, dz, spl);

    // the tile's list: ids[0 .. len) (a list holds each Gaussian at most once, so its
    // positions fit in 32 bits: n_gauss < 2^31)
    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const uint32_t* __restrict__ ids = a.pids + a.rx_base[r] + a.tile_start[ts];
    const int len = (int)(a.tile_start[ts + 1] - a.tile_start[ts]);
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
    unsigned hits = 0;
    // the t_mid-order variant: this ray's sorted hit keys (in the workspace) and their count
    int nord = 0;
    bool overflow = false;
    unsigned long long* tb = nullptr;
    if constexpr (ORDER)
        tb = a.tbuf + ((size_t)r * gr.n_el * gr.n_az + (size_t)(valid ? v : 0) * gr.n_az + (valid ? u : 0)) * kOrderCap;

    // The staging runs one batch ahead of the test: the first 16 bytes of each list
    // position's view record (c, D cos(theta): the cone test's input) are copied into the
    // warp's stin slot with cp.async while the warp composites the batch before, and the
    // list ids two batches ahead are loaded into registers, so that a batch's test waits
    // on one dependent load (the M block, only where the cone test passes) instead of
    // three (id, c, M).
    auto issue_tin = [&](int p0, uint32_t id) {
        if (lane < WB && p0 + lane < len) cp_async16(stin[lane] + 0, reinterpret_cast<const float4*>(view + id));
        cp_async_commit();
    };
    // Test the batch at p0 against the warp's cone (c from its arrived stin slot) and
    // half-spaces, and copy the records of the candidates that may be hit into buffer bf,
    // with the coefficients of the first kCoefSlots of them (slot = rank in the mask);
    // returns the mask of candidates that may be hit.
    auto test_stage = [&](int bf, int p0, uint32_t id) -> uint32_t {
        bool keep = false;
        if (lane < WB && p0 + lane < len) {
            const float4 c = stin[lane][0];
            keep = bundle_meets(bundle_at(spl), c) && planes_meet(spl, c, a.shape + id);
        }
        const uint32_t kmask = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            sid[bf][lane] = id;
            const float4* vw = reinterpret_cast<const float4*>(view + id);
            const float4* sh = reinterpret_cast<const float4*>(a.shape + id);
            float4* dst = sbuf[bf][lane];
            cp_async16(dst + 0, vw + 1);
            cp_async16(dst + 1, vw + 2);
            cp_async16(dst + 2, sh + 0);
            cp_async16(dst + 3, sh + 1);
            cp_async16(dst + 4, sh + 2);
            const int slot = __popc(kmask & ((1u << lane) - 1u));
            if (L == 3 && !ORDER && slot < kCoefSlots) {  // the t_mid pass composites later, from global memory
                const float4* qf = reinterpret_cast<const float4*>(a.fle + (size_t)id * kFle);
                float4* qd = scoef[bf][slot];
#pragma unroll
                for (int i = 0; i < 8; ++i) cp_async16(qd + i, qf + i);
            }
        }
        cp_async_commit();
        return kmask;
    };
    auto list_id = [&](int p) -> uint32_t { return (lane < WB && p + lane < len) ? ids[p + lane] : 0u; };

    if (!__all_sync(0xffffffffu, done)) {
        int bf = 0;
        const uint32_t id0 = list_id(0);
        issue_tin(0, id0);
        uint32_t id_t = list_id(WB);
        cp_async_wait_all();
        __syncwarp();
        uint32_t mask = test_stage(0, 0, id0);
        issue_tin(WB, id_t);
        uint32_t id_n = list_id(2 * WB);
        for (int p0 = 0; p0 < len; p0 += WB, bf ^= 1) {
            if (!ORDER && a.ck && chunk == 0) {
                // transmittance in front of list position K, 2K, ... (a batch start)
                const int p = p0;
                if (p > 0 && p % a.ck_every == 0 && p / a.ck_every <= a.ck_slots && valid) {
                    const size_t rays = (size_t)a.n_rx * gr.n_el * gr.n_az;
                    const size_t ray = ((size_t)r * gr.n_el + v) * gr.n_az + u;
                    a.ck[(size_t)(p / a.ck_every - 1) * rays + ray] = make_float4(Tr, Ti, Gam, Ta);
                }
            }
            cp_async_wait_all();  // this batch's records and the next batch's test inputs
            __syncwarp();
            const uint32_t next = test_stage(bf ^ 1, p0 + WB, id_t);  // empty past the end of the list
            issue_tin(p0 + 2 * WB, id_n);
            id_t = id_n;
            id_n = list_id(p0 + 3 * WB);
            if (!done) {
                int slot = -1;
                for (uint32_t m = mask; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    ++slot;
                    const float4* rec = sbuf[bf][j];
                    if ((a.variant & GSRF_VARIANT_PAPER_CULLING) &&
                        !circle_in(__ldg(a.circle + (size_t)r * a.n + sid[bf][j]), u, v))
                        continue;  // outside the Gaussian's splatting circle (Sec. 4.3)
                    const float4 v1 = rec[0], s2 = rec[4];
                    PairGeo pg;
                    if (!pair_hits(v1, rec[2], rec[3], s2, dx, dy, dz, r_rx, pg)) continue;
                    if constexpr (ORDER) {
                        // GSRF_VARIANT_ORDER_T_MID, first pass: keep the kOrderCap smallest
                        // (t_mid, list position) keys, sorted by insertion (the list's |mu - r|
                        // order is close to t_mid order, so few keys move); a full buffer
                        // drops its largest key
                        uint32_t ku = __float_as_uint(pg.tm);
                        ku = (ku & 0x80000000u) ? ~ku : (ku | 0x80000000u);
                        const unsigned long long key = ((unsigned long long)ku << 32) | (uint32_t)(p0 + j);
                        if (nord == kOrderCap) {
                            overflow = true;
                            if (key > tb[kOrderCap - 1]) continue;
                            --nord;
                        }
                        int q = nord;
                        while (q > 0 && tb[q - 1] > key) {
                            tb[q] = tb[q - 1];
                            --q;
                        }
                        tb[q] = key;
                        ++nord;
                        continue;
                    }
                    float gw;
                    const float alpha = pair_alpha(s2.y, pg.m2r, amax, gw);
                    float pr, pi;
                    if (a.variant & GSRF_VARIANT_RADIANCE_AT_MEAN) {  // one radiance per Gaussian
                        pr = rec[1].z;
                        pi = rec[1].w;
                    } else {
                        if (L == 3 && slot < kCoefSlots)
                            fle_psi<L, true>(scoef[bf][slot], P, Y, pr, pi);
                        else
                            fle_psi<L>(reinterpret_cast<const float4*>(a.fle + (size_t)sid[bf][j] * fle_floats(L)), P,
                                       Y, pr, pi);
                    }
                    // S += alpha psi E T, E = e^{-j phi} = (er, ei)
                    float er = v1.w, ei = rec[1].x;
                    if constexpr (PATH) {  // GSRF_VARIANT_PATH_AT_REP: the path through x_rep
                        const uint32_t id = sid[bf][j];
                        const float4 cv = __ldg(reinterpret_cast<const float4*>(view + id));
                        const float dl = path_delta(cv, a.shape + id, v1, pg, dx, dy, dz,
                                                    a.txpos[0] - a.rxpos[3 * r], a.txpos[1] - a.rxpos[3 * r + 1],
                                                    a.txpos[2] - a.rxpos[3 * r + 2]);
                        float sn, cs;
                        phase_rot(a.om_pi * dl, sn, cs);  // e^{-j 2 pi f0 delta / c}
                        const float nr = er * cs + ei * sn;
                        ei = ei * cs - er * sn;
                        er = nr;
                    }
                    const float etr = er * Tr - ei * Ti, eti = er * Ti + ei * Tr;
                    if constexpr (NFC == 1) {
                        Sr += alpha * (pr * etr - pi * eti);
                        Si += alpha * (pr * eti + pi * etr);
                    } else {
                        // z at the chunk's first subcarrier, then one rotation per step
                        const float ws = rec[1].y + a.dlt * Gam;
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
                    last = p0 + j;  // position inside the tile's list
                    if (Ta < eps_T) {
                        done = true;
                        break;
                    }
                }
            }
            mask = next;
            __syncwarp();
            if (__all_sync(0xffffffffu, done)) break;
        }
        cp_async_wait_all();
    }
    if constexpr (ORDER) {
        // second pass: the kept hits in ascending t_mid, each re-tested (the same FP32
        // decision) and composited, until prod(1 - alpha) < eps_T; a ray that dropped hits
        // and did not terminate on the kept ones needed more than kOrderCap
        bool ended = false;
        for (int q = 0; q < nord; ++q) {
            const uint32_t pos = (uint32_t)tb[q];
            const uint32_t id = ids[pos];
            const float4* vw = reinterpret_cast<const float4*>(view + id);
            const float4* sh = reinterpret_cast<const float4*>(a.shape + id);
            const float4 v1 = __ldg(vw + 1), r1 = __ldg(vw + 2), s2 = __ldg(sh + 2);
            PairGeo pg;
            if (!pair_hits(v1, __ldg(sh), __ldg(sh + 1), s2, dx, dy, dz, r_rx, pg)) continue;
            float gw;
            const float alpha = pair_alpha(s2.y, pg.m2r, amax, gw);
            float pr, pi;
            if (a.variant & GSRF_VARIANT_RADIANCE_AT_MEAN) {
                pr = r1.z;
                pi = r1.w;
            } else {
                fle_psi<L>(reinterpret_cast<const float4*>(a.fle + (size_t)id * fle_floats(L)), P, Y, pr, pi);
            }
            const float er = v1.w, ei = r1.x;
            const float etr = er * Tr - ei * Ti, eti = er * Ti + ei * Tr;
            Sr += alpha * (pr * etr - pi * eti);
            Si += alpha * (pr * eti + pi * etr);
            float sn, cs;
            phase_rot(a.om_pi * s2.z * pg.dt, sn, cs);
            const float om = 1.0f - alpha;
            const float nTr = om * (Tr * cs + Ti * sn);
            Ti = om * (Ti * cs - Tr * sn);
            Tr = nTr;
            Ta *= om;
            ++hits;
            if (Ta < eps_T) {
                ended = true;
                break;
            }
        }
        if (overflow && !ended) atomicCAS(&a.st->code, (int)GSRF_OK, (int)GSRF_ERR_UNSUPPORTED);
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
        if (!ORDER && a.rs && chunk == 0) {
            // RayState {last, Ta, Tr, Ti | Gam, pad[3]} as two 16-byte stores
            float4* rs4 = reinterpret_cast<float4*>(a.rs + ray);
            rs4[0] = make_float4(__int_as_float(last), Ta, Tr, Ti);
            rs4[1] = make_float4(Gam, 0.0f, 0.0f, 0.0f);
        }
    }
    // statistics: list positions tested and composited pairs, one atomic per warp
    // list positions this ray tested: up to its terminating pair, else the whole list
    unsigned long long t64 = !valid ? 0ull
                             : ((done && !ORDER) ? (unsigned long long)(last + 1) : (unsigned long long)len),
                       h64 = hits;
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

// Persistent launch of one problem: every warp takes work items (receiver, tile, ray
// block, subcarrier chunk) from one counter, in heaviest-first order, until none is
// left; a warp that finishes early takes the next item instead of idling until the
// other warps of its CTA are done.
// One frequency: 7 CTAs per SM up to L = 3 (72 registers), fewer for the larger bases of
// L = 4 and 5.  Several frequencies (L = 3 only) take one chunk of 8, 16, 32 or 64
// subcarriers per walk, the smallest that holds n_f (so at most 64 subcarriers need one
// walk; more per lane costs registers, not walks): 4 CTAs per SM for chunks of 8 and 16,
// 3 for 32 (168 registers), 2 for 64 (242, no spills).  PATH: the path-through-x_rep
// variant, a separate instance so that its arithmetic costs the others no registers.
template <int NFC, int WB, int L, bool PATH = false, bool ORDER = false>
__global__ void __launch_bounds__(kThreads, NFC == 1 ? ((PATH || ORDER) ? 6 : (L <= 3 ? 7 : (L == 4 ? 6 : 5))) : (NFC <= 16 ? 4 : (NFC == 32 ? 3 : 2)))
    k_render_queue(RenderArgs a,
                                                                            const uint32_t* __restrict__ order,
                                                                            unsigned long long* __restrict__ counter,
                                                                            unsigned long long total) {
    __shared__ float4 sbuf[kWarps][2][WB][kRec];
    __shared__ uint32_t sid[kWarps][2][WB];
    __shared__ float4 spl[kWarps][kPlaneSlots];
    __shared__ float4 stin[kWarps][WB][1];
    __shared__ float4 scoef[kWarps][2][kCoefSlots][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned per_rx = (unsigned)a.n_tiles * (unsigned)a.per_tile;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        const uint32_t id = order[it];
        const unsigned rem = id % per_rx;
        render_block<NFC, WB, L, PATH, ORDER>(a, (int)(id / per_rx), (int)(rem / (unsigned)a.per_tile),
                                 (int)(rem % (unsigned)a.per_tile), sbuf[warp], sid[warp], spl[warp], stin[warp], scoef[warp]);
    }
}

// Persistent batched launch over several problems (n_f = 1 each): work items (job,
// receiver, tile, ray block), same queue discipline.  The warp copies its item's job
// description from the device table into shared memory.  With job_done set, the warp
// that finishes an item of job j raises job_done[j] to the global timer (the job's
// completion time) and every warp lowers job_done[n_jobs] to its start time.  6 CTAs
// per SM: at 7 (72 registers) the job bookkeeping spills; at 6 it takes 79, no spills.
// job_order: the order holds, for queue position `it`, an item's index inside the job
// whose range of positions holds `it` (jobs taken in their given order, heaviest first
// inside each); otherwise the item's global id (heaviest first over all jobs).
template <int WB>
__global__ void __launch_bounds__(kThreads, 6)
    k_render_batch(const RenderArgs* __restrict__ jobs, const unsigned long long* __restrict__ item_base, int n_jobs,
                   const uint32_t* __restrict__ order, unsigned long long* __restrict__ counter,
                   unsigned long long* __restrict__ job_done, int job_order) {
    __shared__ float4 sbuf[kWarps][2][WB][kRec];
    __shared__ uint32_t sid[kWarps][2][WB];
    __shared__ float4 spl[kWarps][kPlaneSlots];
    __shared__ float4 stin[kWarps][WB][1];
    __shared__ float4 scoef[kWarps][2][kCoefSlots][8];
    __shared__ RenderArgs sjob[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long total = item_base[n_jobs];
    if (job_done && lane == 0) atomicMin(job_done + n_jobs, global_ns());
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        int j;
        unsigned long long id;
        if (job_order) {
            j = job_of(item_base, n_jobs, it);
            id = item_base[j] + order[it];
        } else {
            id = order[it];
            j = job_of(item_base, n_jobs, id);
        }
        {  // the job's description, one 32-bit word per lane and step
            constexpr int kWords = (int)(sizeof(RenderArgs) / 4);
            __syncwarp();
            const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs + j);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sjob[warp]);
            for (int w = lane; w < kWords; w += 32) dst[w] = src[w];
            __syncwarp();
        }
        const RenderArgs& a = sjob[warp];
        const unsigned long long local = id - item_base[j];
        const unsigned long long per_rx = (unsigned long long)a.n_tiles * a.per_tile;
        const unsigned rem = (unsigned)(local % per_rx);
        render_block<1, WB, 3>(a, (int)(local / per_rx), (int)(rem / (unsigned)a.per_tile),
                               (int)(rem % (unsigned)a.per_tile), sbuf[warp], sid[warp], spl[warp], stin[warp], scoef[warp]);
        if (job_done && lane == 0) atomicMax(job_done + j, global_ns());
    }
}

// Copies a chunk of job descriptions and item bases into the device table and clears
// each job's statistics (candidate tests, composited pairs).
__global__ void k_put_jobs(JobChunk c, RenderArgs* __restrict__ jobs, unsigned long long* __restrict__ item_base,
                           uint32_t* __restrict__ chunk_base) {
    constexpr int kWords = (int)(sizeof(RenderArgs) / 4);
    for (int i = threadIdx.x; i < c.count * kWords; i += blockDim.x) {
        const int j = i / kWords, w = i % kWords;
        reinterpret_cast<uint32_t*>(jobs + c.first + j)[w] = reinterpret_cast<const uint32_t*>(&c.jobs[j])[w];
    }
    for (int j = threadIdx.x; j < c.n_bases; j += blockDim.x) {
        item_base[c.first + j] = c.item_base[j];
        chunk_base[c.first + j] = c.chunk_base[j];
    }
    for (int j = threadIdx.x; j < c.count; j += blockDim.x) {
        c.jobs[j].st->stats[0] = 0ull;
        c.jobs[j].st->stats[1] = 0ull;
    }
}

// Cost key of every work item: its tile's list length, heaviest first (bucket
// 31 - floor(log2(len + 1)), so that an ascending stable sort puts long lists first).
__global__ void k_item_keys(const uint32_t* __restrict__ tile_start, int n_tiles, int per_tile,
                            unsigned long long total, uint32_t* __restrict__ keys) {
    const unsigned long long id = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total) return;
    const unsigned long long t = id / (unsigned)per_tile;  // r * n_tiles + tile
    const size_t ts = (size_t)(t / (unsigned)n_tiles) * (n_tiles + 1) + (size_t)(t % (unsigned)n_tiles);
    const uint32_t len = tile_start[ts + 1] - tile_start[ts];
    keys[id] = (uint32_t)__clz((int)(len + 1u));
}

__global__ void k_batch_keys(const RenderArgs* __restrict__ jobs, const unsigned long long* __restrict__ item_base,
                             int n_jobs, uint32_t* __restrict__ keys) {
    const unsigned long long id = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= item_base[n_jobs]) return;
    const int j = job_of(item_base, n_jobs, id);
    const RenderArgs& a = jobs[j];
    const unsigned long long t = (id - item_base[j]) / (unsigned)a.per_tile;
    const size_t ts = (size_t)(t / (unsigned)a.n_tiles) * (a.n_tiles + 1) + (size_t)(t % (unsigned)a.n_tiles);
    const uint32_t len = a.tile_start[ts + 1] - a.tile_start[ts];
    keys[id] = (uint32_t)__clz((int)(len + 1u));
}

int plan_block_w(const gsrf_plan* p) { return p->ray_block_w == 0 ? 8 : p->ray_block_w; }
int plan_stage(const gsrf_plan* p) { return p->stage == 0 ? 32 : p->stage; }

cudaError_t launch_item_order(const Layout& L, void* ws, int per_tile, uint32_t** order,
                              unsigned long long** counter, cudaStream_t st) {
    const long long n = (long long)L.n_rx * L.n_tiles * per_tile;
    uint32_t* keys = at<uint32_t>(ws, L.qkeys);
    uint32_t* keys2 = at<uint32_t>(ws, L.qkeys2);
    *order = at<uint32_t>(ws, L.qorder);
    *counter = at<unsigned long long>(ws, L.qcounter);
    k_item_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(at<uint32_t>(ws, L.tile_start), L.n_tiles, per_tile,
                                                             (unsigned long long)n, keys);
    cudaError_t e = launch_sort_small_keys(keys, keys2, *order, n, 32, at<uint32_t>(ws, L.qhist), st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(*counter, 0, sizeof(unsigned long long), st);
}

// One resident wave of CTAs for a persistent kernel: every SM holds as many as it can
// run at once, and no more than the items need.
template <typename K>
static cudaError_t resident_grid(K kernel, long long items, int* grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0)) != cudaSuccess) return e;
    const long long ctas_needed = (items + kWarps - 1) / kWarps;
    *grid = (int)max(1ll, min((long long)sms * max(per_sm, 1), ctas_needed));
    return cudaSuccess;
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
    const int bw = plan_block_w(p);
    a.bw_log = __builtin_ctz((unsigned)bw);
    a.nbx = p->grid.tile_w / bw;
    const int nfc = p->n_f == 1 ? 1 : (p->n_f <= 8 ? 8 : (p->n_f <= 16 ? 16 : (p->n_f <= 32 ? 32 : 64)));
    a.nchunk = (p->n_f + nfc - 1) / nfc;
    a.per_tile = (p->grid.tile_w * p->grid.tile_h / 32) * a.nchunk;
    const size_t rays = (size_t)p->n_rx * p->grid.n_az * p->grid.n_el;
    a.ck = (ray_state && p->ckpt_every > 0)
               ? reinterpret_cast<float4*>(static_cast<char*>(ray_state) + rays * sizeof(RayState))
               : nullptr;
    a.ck_every = p->ckpt_every > 0 ? p->ckpt_every : 1;
    a.ck_slots = p->ckpt_slots;
    a.variant = p->variant;
    a.circle = (p->variant & GSRF_VARIANT_PAPER_CULLING) ? at<float4>(ws, L.circle) : nullptr;
    a.rxpos = at<float>(ws, L.rxpos);
    a.txpos = at<float>(ws, L.txpos);
    a.tbuf = (p->variant & GSRF_VARIANT_ORDER_T_MID) ? at<unsigned long long>(ws, L.tbuf) : nullptr;
    return a;
}

template <int NFC, int WB, int L = 3, bool PATH = false, bool ORDER = false>
static cudaError_t launch_queue(const RenderArgs& a, const uint32_t* order, unsigned long long* counter, long long n,
                                cudaStream_t st) {
    int grid = 0;
    cudaError_t e = resident_grid(k_render_queue<NFC, WB, L, PATH, ORDER>, n, &grid);
    if (e != cudaSuccess) return e;
    k_render_queue<NFC, WB, L, PATH, ORDER><<<grid, kThreads, 0, st>>>(a, order, counter, (unsigned long long)n);
    return cudaGetLastError();
}

// One frequency at Fourier-Legendre degree L (1..5), stage of 16 or 32 candidates.
template <int WB>
static cudaError_t launch_queue_degree(int L, const RenderArgs& a, const uint32_t* order, unsigned long long* counter,
                                       long long n, cudaStream_t st) {
    switch (L) {
        case 1: return launch_queue<1, WB, 1>(a, order, counter, n, st);
        case 2: return launch_queue<1, WB, 2>(a, order, counter, n, st);
        case 4: return launch_queue<1, WB, 4>(a, order, counter, n, st);
        case 5: return launch_queue<1, WB, 5>(a, order, counter, n, st);
        default: return launch_queue<1, WB, 3>(a, order, counter, n, st);
    }
}

cudaError_t launch_render_fwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, void* ws,
                              float* out, void* ray_state, cudaStream_t st) {
    RenderArgs a = render_args(p, L, ws, out, ray_state);
    (void)g;
    cudaError_t e = cudaMemsetAsync(&a.st->stats[0], 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    uint32_t* order = nullptr;
    unsigned long long* counter = nullptr;
    if ((e = launch_item_order(L, ws, a.per_tile, &order, &counter, st)) != cudaSuccess) return e;
    const long long n = (long long)L.n_rx * L.n_tiles * a.per_tile;
    const bool wb16 = plan_stage(p) == 16;
    if (p->variant & GSRF_VARIANT_ORDER_T_MID)  // one frequency, L = 3 (checked with the plan)
        return wb16 ? launch_queue<1, 16, 3, false, true>(a, order, counter, n, st)
                    : launch_queue<1, 32, 3, false, true>(a, order, counter, n, st);
    if (p->variant & GSRF_VARIANT_PATH_AT_REP)  // one frequency, L = 3 (checked with the plan)
        return wb16 ? launch_queue<1, 16, 3, true>(a, order, counter, n, st)
                    : launch_queue<1, 32, 3, true>(a, order, counter, n, st);
    if (p->n_f == 1)
        return wb16 ? launch_queue_degree<16>(plan_degree(p), a, order, counter, n, st)
                    : launch_queue_degree<32>(plan_degree(p), a, order, counter, n, st);
    if (p->n_f <= 8) return wb16 ? launch_queue<8, 16>(a, order, counter, n, st) : launch_queue<8, 32>(a, order, counter, n, st);
    if (p->n_f <= 16) return wb16 ? launch_queue<16, 16>(a, order, counter, n, st) : launch_queue<16, 32>(a, order, counter, n, st);
    if (p->n_f <= 32) return wb16 ? launch_queue<32, 16>(a, order, counter, n, st) : launch_queue<32, 32>(a, order, counter, n, st);
    return wb16 ? launch_queue<64, 16>(a, order, counter, n, st) : launch_queue<64, 32>(a, order, counter, n, st);
}

long long batch_items(int n_jobs, const gsrf_plan* plans) {
    long long n = 0;
    for (int j = 0; j < n_jobs; ++j) {
        Layout L;
        make_layout(&plans[j], &L);
        n += (long long)L.n_rx * L.n_tiles * (plans[j].grid.tile_w * plans[j].grid.tile_h / 32);
    }
    return n;
}

// Batch workspace: item keys (two buffers), their order, the counting-sort histogram (per
// job chunks in job order), the queue counter, the job table, the item bases and the
// jobs' first sort chunks.
struct BatchLayout {
    size_t keys, keys2, order, hist, counter, jobs, base, cbase, total;
};

static BatchLayout batch_layout(int n_jobs, long long n) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const long long chunks = (n + kSmallChunk - 1) / kSmallChunk + n_jobs;  // either sort's chunks
    BatchLayout b;
    b.keys = 0;
    b.keys2 = b.keys + al(n * 4);
    b.order = b.keys2 + al(n * 4);
    b.hist = b.order + al(n * 4);
    b.counter = b.hist + al(chunks * 32 * 4);
    b.jobs = b.counter + al(8);
    b.base = b.jobs + al((size_t)n_jobs * sizeof(RenderArgs));
    b.cbase = b.base + al((size_t)(n_jobs + 1) * 8);
    b.total = b.cbase + al((size_t)(n_jobs + 1) * 4);
    return b;
}

size_t batch_workspace_bytes(int n_jobs, const gsrf_plan* plans) {
    return batch_layout(n_jobs, batch_items(n_jobs, plans)).total;
}

cudaError_t launch_render_batch(int n_jobs, const gsrf_plan* plans, void* const* workspaces, float* const* outs,
                                void* batch_ws, unsigned long long* job_done, bool job_order, cudaStream_t st) {
    const long long n = batch_items(n_jobs, plans);
    const BatchLayout bl = batch_layout(n_jobs, n);
    char* w = static_cast<char*>(batch_ws);
    RenderArgs* jobs = reinterpret_cast<RenderArgs*>(w + bl.jobs);
    unsigned long long* base = reinterpret_cast<unsigned long long*>(w + bl.base);
    uint32_t* cbase = reinterpret_cast<uint32_t*>(w + bl.cbase);
    cudaError_t e = cudaSuccess;
    if (job_done) {
        // completion times 0, the launch's start time "infinitely late" until a warp lowers it
        if ((e = cudaMemsetAsync(job_done, 0, (size_t)n_jobs * 8, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(job_done + n_jobs, 0xff, 8, st)) != cudaSuccess) return e;
    }
    // the job table, kJobsPerPut descriptions per copy launch (passed by value)
    unsigned long long acc = 0;
    uint32_t cacc = 0;
    for (int first = 0; first < n_jobs; first += kJobsPerPut) {
        JobChunk c;
        c.first = first;
        c.count = min(kJobsPerPut, n_jobs - first);
        for (int i = 0; i < c.count; ++i) {
            const int j = first + i;
            Layout L;
            make_layout(&plans[j], &L);
            c.jobs[i] = render_args(&plans[j], L, workspaces[j], outs[j], nullptr);
            c.item_base[i] = acc;
            c.chunk_base[i] = cacc;
            const unsigned long long items = (unsigned long long)L.n_rx * L.n_tiles * c.jobs[i].per_tile;
            acc += items;
            cacc += (uint32_t)((items + kChunk - 1) / kChunk);
        }
        c.n_bases = c.count;
        if (first + c.count == n_jobs) {
            c.item_base[c.n_bases] = acc;
            c.chunk_base[c.n_bases++] = cacc;
        }
        k_put_jobs<<<1, 256, 0, st>>>(c, jobs, base, cbase);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    uint32_t* keys = reinterpret_cast<uint32_t*>(w + bl.keys);
    uint32_t* keys2 = reinterpret_cast<uint32_t*>(w + bl.keys2);
    uint32_t* order = reinterpret_cast<uint32_t*>(w + bl.order);
    uint32_t* hist = reinterpret_cast<uint32_t*>(w + bl.hist);
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(w + bl.counter);
    k_batch_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(jobs, base, n_jobs, keys);
    e = job_order ? launch_sort_small_keys_segmented(keys, keys2, order, n_jobs, reinterpret_cast<const long long*>(base),
                                                     cbase, cacc, 32, hist, st)
                  : launch_sort_small_keys(keys, keys2, order, n, 32, hist, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    int grid = 0;
    if (plan_stage(&plans[0]) == 16) {
        if ((e = resident_grid(k_render_batch<16>, n, &grid)) != cudaSuccess) return e;
        k_render_batch<16><<<grid, kThreads, 0, st>>>(jobs, base, n_jobs, order, counter, job_done, job_order ? 1 : 0);
    } else {
        if ((e = resident_grid(k_render_batch<32>, n, &grid)) != cudaSuccess) return e;
        k_render_batch<32><<<grid, kThreads, 0, st>>>(jobs, base, n_jobs, order, counter, job_done, job_order ? 1 : 0);
    }
    return cudaGetLastError();
}

}  // namespace gsrf
