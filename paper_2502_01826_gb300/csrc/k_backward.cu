// k_backward.cu -- the adjoint of the render (App. D): gradients of a real loss L with
// respect to every Gaussian parameter, given G = dL/dRe S + j dL/dIm S per ray.
//
// k_render_bwd walks each ray's list back to front from its last composited pair, with
// the same work items (receiver, tile, ray block, subcarrier chunk), warp cone and
// planes, and the same hit decisions (pair_hits) as the forward.  Transmittance is recomputed, not stored: T_k = T_{k+1} e^{+j theta_k} /
// (1 - alpha_k), starting from the T the forward left in the ray state.  With
// z_k = alpha_k psi_k E_k T_k and the suffix R_k = sum_{j>k} z_j (App. D.1, D.2):
//     dS/dalpha_k = psi_k E_k T_k - R_k / (1 - alpha_k),   dS/dtheta_k = -j R_k,
//     dS/dphi_k = -j z_k,                                  dS/dpsi_k = alpha_k E_k T_k,
// and dL/dp = Re(conj(G) dS/dp).  App. D.3 then carries dL/dalpha through the midpoint
// weight and the quadratic A t^2 + 2 B t + (C - 9) = 0 (here A = |v'|^2, B = w.v',
// C = |w|^2 in whitened coordinates) to the whitening matrix W and the mean; the path
// phase phi = 2 pi f d / c adds its own term to the mean.  Per candidate, the 46
// gradient values of the warp's 32 rays are summed by butterfly reduce-scatters (47
// shuffles; lane L ends with totals L and L/2; the 32 coefficient values in a lane-
// permuted order that needs no selects) and added to the Gaussian's accumulator with one
// atomic per value.
//
// k_grad_params chains the accumulators to the raw parameters: W = diag(1/s) R^T to the
// log-scales and to the (unnormalised) quaternion, the opacity through its sigmoid, the
// folded Fourier-Legendre coefficients back to the 16 complex coefficients.
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

constexpr int kBW = 4;           // warps per CTA
constexpr int kBThreads = 32 * kBW;
constexpr int kBB = 32;          // candidates per warp batch
// Per batch, the Fourier-Legendre coefficients (L = 3) of the kBCoefSlots candidates of the
// mask that the reverse walk meets first (the highest list positions) are staged in shared
// memory with their records, so that their radiance reads shared memory; the others read
// global memory.  10 slots (10 KB per CTA) keep 5 CTAs per SM.
constexpr int kBCoefSlots = 10;
// Accumulator floats per Gaussian: W 9, mu 3, o, b, then the coefficient gradients in
// chunks of 32 (dL/d psi_re and dL/d psi_im times 16 basis values each) -- grad_floats(L)
// in the internal header; 48 at L <= 3.

struct BwdArgs {
    const GShape* shape;
    const View* view;
    const float* fle;
    const float* raytab;
    const uint32_t* pids;
    const long long* rx_base;
    const uint32_t* tile_start;
    const float* rxpos;
    const float* txpos;
    const RayState* rs;
    const float* grad_rays;
    float* acc;
    gsrf_grid gr;
    int ntu, n_tiles;
    long long n;
    float om_pi;  // 2 f0 / c
    int n_f;      // frequencies f0 + s df
    float dlt;    // 2 pi df / c
    int bw_log;   // log2 of the ray-block width (block height 32 / width)
    int nbx;      // ray blocks per tile along azimuth
    int per_tile; // work items per tile: ray blocks
    int g_pairs;  // several frequencies: subcarrier pairs of the upstream gradient, ceil(n_f / 2)
    int g_stride4;  // float4s per lane row of it in shared memory (g_pairs, made odd)
    int n_rx;
    const float4* ck;  // the forward's transmittance checkpoints [slot][ray], or null
    int variant;       // 0, or GSRF_VARIANT_NORMALISED_WEIGHT / GSRF_VARIANT_PAPER_CULLING bits
    const float4* circle;  // the paper's splatting circles [receiver][Gaussian] (culling variant)
    int ck_every, ck_slots;
};

__device__ __forceinline__ void cp_async16b(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Butterfly reduce-scatter of 16 values over a warp: afterwards lanes 2L and 2L + 1 hold
// the sum of value L over all lanes.
__device__ __forceinline__ float reduce_scatter16(float* v, int lane) {
#pragma unroll
    for (int off = 16, n = 16; off >= 2; off >>= 1, n >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < n / 2) {
                const float send = up ? v[i] : v[i + n / 2];
                const float keep = up ? v[i + n / 2] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// One warp's work item: ray block k of tile `tile` for receiver r.  MF = false: one
// frequency.  MF = true: all n_f subcarriers f0 + s df in one walk.  There the pair's
// contribution at subcarrier s is z_k r_k^s, r_k = e^{-j (2 pi df d_k / c + 2 pi df
// Gamma_k / c)} (Gamma_k = sum of b dt in front of k), exactly as the forward builds it.
// With c_s = conj(G_s), every sum over s that the gradient needs is one of
//     H_k = sum_s c_s r_k^s,   H'_k = sum_s omega_s c_s r_k^s,
// and the suffix sums Q_k = sum_{j>k} alpha_j psi_j w_j H_j (and Q' with H'), which
// replace the n_f suffixes R_s: sum_s c_s R_{k,s} = Q_k.  Per pair the lane evaluates H
// and H' by Horner's rule over the ray's n_f upstream values (held in shared memory):
// with omega_s = omega_0 + s 2 pi df / c, H' = omega_0 H + (2 pi df / c) r dH/dr, and
// Horner's rule gives dH/dr in the same pass.
template <bool MF, int L>
__device__ __forceinline__ void bwd_block(const BwdArgs& a, int r, int tile, int k, float4 (*sbuf)[kBB][6],
                                          uint32_t (*sid)[kBB], float4* spl, float (*sbp)[32],
                                          float4 (*scoef)[kBCoefSlots][8], float4* sg) {
    constexpr int NB = (L + 1) * (L + 1), NCH = grad_chunks(L);
    const int lane = threadIdx.x & 31;
    const gsrf_grid& gr = a.gr;
    const int blk = k;
    const int bw = 1 << a.bw_log, bh = 32 >> a.bw_log;
    const int tu = tile % a.ntu, tv = tile / a.ntu;
    const int u_lo = tu * gr.tile_w + (blk % a.nbx) * bw, v_lo = tv * gr.tile_h + (blk / a.nbx) * bh;
    const int u = u_lo + (lane & (bw - 1)), v = v_lo + (lane >> a.bw_log);
    const bool valid = u < gr.n_az && v < gr.n_el;

    // ray: direction, basis, cone of the warp, state and upstream gradient
    float dx = 0.0f, dy = 0.0f, dz = 1.0f, P[L], Y[L * (L + 1)];
#pragma unroll
    for (int i = 0; i < L; ++i) P[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < L * (L + 1); ++i) Y[i] = 0.0f;
    int last = -1;
    float Tr = 0.0f, Ti = 0.0f, Gam = 0.0f;
    float Gr = 0.0f, Gi = 0.0f, Rr = 0.0f, Ri = 0.0f;  // one frequency: upstream G and suffix R
    float Qr = 0.0f, Qi = 0.0f, Q2r = 0.0f, Q2i = 0.0f;  // several: the suffix sums Q and Q'
    const size_t plane = (size_t)gr.n_el * gr.n_az, pix = valid ? (size_t)v * gr.n_az + u : 0;
    if (valid) {
        load_ray<L>(a.raytab, pix, dx, dy, dz, P, Y);
        const RayState s = a.rs[(size_t)r * plane + pix];
        last = s.last;
        Tr = s.Tr;
        Ti = s.Ti;
        Gam = s.Gam;
        if constexpr (!MF) {
            const float2 g = reinterpret_cast<const float2*>(a.grad_rays)[(size_t)r * plane + pix];
            Gr = g.x;
            Gi = g.y;
        }
    }
    if constexpr (MF) {  // this lane's row: G_0 .. G_{n_f - 1}, zero-padded to 2 g_pairs
        float2* row = reinterpret_cast<float2*>(sg + lane * a.g_stride4);
        const float2* g2 = reinterpret_cast<const float2*>(a.grad_rays) + (size_t)r * a.n_f * plane + pix;
        for (int s = 0; s < 2 * a.g_pairs; ++s)
            row[s] = (valid && s < a.n_f) ? g2[(size_t)s * plane] : make_float2(0.0f, 0.0f);
    }
    // The ray's basis in the order of the coefficient accumulators -- 1, P_10 .. P_L0,
    // then (Re, Im) of the Y_{l,m>0} in m-major order, zero-padded to chunks of 16 --
    // stored per lane with slot 16 c + i holding basis value 16 c + (i ^ (lane & 15)),
    // the order the select-free reduce-scatter below needs.
    {
        float b[16 * NCH];
        b[0] = 1.0f;
#pragma unroll
        for (int l = 0; l < L; ++l) b[1 + l] = P[l];
#pragma unroll
        for (int n = 0; n < L * (L + 1); ++n) b[1 + L + n] = Y[n];
#pragma unroll
        for (int i = NB; i < 16 * NCH; ++i) b[i] = 0.0f;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int i = 0; i < 16; ++i) sbp[16 * c + i][lane] = b[16 * c + (i ^ (lane & 15))];
        __syncwarp();
    }
    const Bundle bun = warp_bundle(valid, dx, dy, dz);  // the forward's warp cone and planes
    warp_planes(gr, u_lo, v_lo, bw, bh, bun, valid, dx, dy, dz, spl);

    // positions are inside the tile's list; a state that points past it (another plan's,
    // or garbage) is clamped so that no read leaves the list
    const size_t ts = (size_t)r * (a.n_tiles + 1) + tile;
    const uint32_t* __restrict__ ids = a.pids + a.rx_base[r] + a.tile_start[ts];  // the tile's list
    const int len = (int)(a.tile_start[ts + 1] - a.tile_start[ts]);
    last = min(last, len - 1);
    int wlast = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    if (wlast < 0) return;  // no ray of this warp composited anything
    const float r_rx = gr.r_rx, amax = gr.alpha_max;
    const View* __restrict__ view = a.view + (size_t)r * a.n;
    const float rx = a.rxpos[3 * r], ry = a.rxpos[3 * r + 1], rz = a.rxpos[3 * r + 2];
    const float omega = 3.14159265f * a.om_pi;  // 2 pi f0 / c

    auto stage = [&](int bf, int p0, int pend) -> uint32_t {
        bool keep = false;
        if (p0 + lane < pend) {
            const uint32_t id = ids[p0 + lane];
            const float4* vw = reinterpret_cast<const float4*>(view + id);
            const float4 c = __ldg(vw);
            keep = bundle_meets(bundle_at(spl), c) && planes_meet(spl, c, a.shape + id);
        }
        const uint32_t kmask = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t id = ids[p0 + lane];
            const float4* vw = reinterpret_cast<const float4*>(view + id);
            sid[bf][lane] = id;
            const float4* sh = reinterpret_cast<const float4*>(a.shape + id);
            float4* dst = sbuf[bf][lane];
            dst[0] = __ldg(vw);
            cp_async16b(dst + 1, vw + 1);
            cp_async16b(dst + 2, vw + 2);
            cp_async16b(dst + 3, sh + 0);
            cp_async16b(dst + 4, sh + 1);
            cp_async16b(dst + 5, sh + 2);
            // slot = rank from the top of the mask (the walk goes from high positions down)
            const int slot = __popc(kmask >> lane) - 1;
            if (L == 3 && slot < kBCoefSlots) {
                const float4* qf = reinterpret_cast<const float4*>(a.fle + (size_t)id * kFle);
#pragma unroll
                for (int i = 0; i < 8; ++i) cp_async16b(scoef[bf][slot] + i, qf + i);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        return kmask;
    };

    // batches that hold list positions 0 .. wlast, from the last one down
    const int end = wlast + 1;
    int b0 = (wlast / kBB) * kBB;
    int bf = 0;
    uint32_t mask = stage(0, b0, end);
    for (; b0 >= 0; b0 -= kBB, bf ^= 1) {
        const uint32_t next = b0 - kBB >= 0 ? stage(bf ^ 1, b0 - kBB, end) : (stage(bf ^ 1, end, end), 0u);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();
        int slot = -1;
        for (uint32_t m = mask; m;) {
            const int j = 31 - __clz(m);
            m &= ~(1u << j);
            ++slot;
            const int pos = b0 + j;
            const float4* rec = sbuf[bf][j];
            const float4 v1 = rec[1], s0 = rec[3], s1 = rec[4], s2 = rec[5];
            const float4 v0 = rec[0];  // c = mu - r, used by the hit path
            PairGeo pg;
            // the forward's hit decision: inside the splatting circle (culling variant), then
            // the exact test
            bool hit = pos <= last &&
                       (!(a.variant & GSRF_VARIANT_PAPER_CULLING) ||
                        circle_in(__ldg(a.circle + (size_t)r * a.n + sid[bf][j]), u, v)) &&
                       pair_hits(v1, s0, s1, s2, dx, dy, dz, r_rx, pg);
            if (!__any_sync(0xffffffffu, hit)) continue;
            float go[16];
            float g_pr = 0.0f, g_pi = 0.0f;  // dL/d psi (real, imaginary) of this pair on this ray
#pragma unroll
            for (int i = 0; i < 16; ++i) go[i] = 0.0f;
            if (hit) {
                float gw;
                const float o = s2.y;
                const float alpha = pair_alpha(o, pg.m2r, amax, gw);
                const bool clamped = o * gw >= amax;
                float pr, pi;
                if (L == 3 && slot < kBCoefSlots)
                    fle_psi<L, true>(scoef[bf][slot], P, Y, pr, pi);
                else
                    fle_psi<L>(reinterpret_cast<const float4*>(a.fle + (size_t)sid[bf][j] * fle_floats(L)), P, Y, pr,
                               pi);
                // T before this pair: undo (1 - alpha) e^{-j theta}
                float sn, cs;
                phase_rot(a.om_pi * s2.z * pg.dt, sn, cs);
                const float iom = 1.0f / (1.0f - alpha);
                const float nTr = (Tr * cs - Ti * sn) * iom;
                Ti = (Ti * cs + Tr * sn) * iom;
                Tr = nTr;
                // w = E T at f0; Theta = sum_s omega_s Re(conj(G_s) dS_s/dtheta_s),
                // Phi = sum_s omega_s Re(conj(G_s) dS_s/dphi_s) (App. D.1, D.2)
                const float er = v1.w, ei = rec[2].x;
                const float wr = er * Tr - ei * Ti, wi = er * Ti + ei * Tr;
                float g_alpha, Theta, Phi;
                if constexpr (!MF) {
                    const float zr = alpha * (pr * wr - pi * wi), zi = alpha * (pr * wi + pi * wr);
                    const float Xr = pr * wr - pi * wi - Rr * iom, Xi = pr * wi + pi * wr - Ri * iom;
                    g_alpha = Gr * Xr + Gi * Xi;
                    Theta = (Gr * Ri - Gi * Rr) * omega;
                    Phi = (Gr * zi - Gi * zr) * omega;
                    const float ur = alpha * wr, ui = alpha * wi;
                    g_pr = Gr * ur + Gi * ui;
                    g_pi = Gi * ur - Gr * ui;
                    Rr += zr;
                    Ri += zi;
                } else {
                    Gam -= s2.z * pg.dt;  // Gamma in front of this pair
                    const float ws = rec[2].y + a.dlt * Gam;
                    float rs, rc;
                    sincosf(ws, &rs, &rc);  // r = e^{-j ws} = rc - j rs
                    // Horner in x = r^2 on the even and odd coefficients, two independent
                    // chains: H = E(x) + r O(x) with E = sum_k conj(G_2k) x^k, O = sum_k
                    // conj(G_2k+1) x^k, and D = r dH/dr = 2 x E'(x) + r (O(x) + 2 x O'(x));
                    // each chain carries its derivative (E' <- E' x + E, E <- E x + c)
                    const float4* row = sg + lane * a.g_stride4;
                    const float c2 = rc * rc - rs * rs, s2x = 2.0f * rs * rc;  // x = c2 - j s2x
                    float er = 0.0f, ei = 0.0f, edr = 0.0f, edi = 0.0f;  // E, E'
                    float orr = 0.0f, oi = 0.0f, odr = 0.0f, odi = 0.0f;  // O, O'
                    for (int i = a.g_pairs - 1; i >= 0; --i) {
                        const float4 c = row[i];  // G_{2i} (x, y), G_{2i+1} (z, w)
                        float t = edr * c2 + edi * s2x + er;
                        edi = edi * c2 - edr * s2x + ei;
                        edr = t;
                        t = er * c2 + ei * s2x + c.x;
                        ei = ei * c2 - er * s2x - c.y;
                        er = t;
                        t = odr * c2 + odi * s2x + orr;
                        odi = odi * c2 - odr * s2x + oi;
                        odr = t;
                        t = orr * c2 + oi * s2x + c.z;
                        oi = oi * c2 - orr * s2x - c.w;
                        orr = t;
                    }
                    const float hr = er + (orr * rc + oi * rs), hi = ei + (oi * rc - orr * rs);
                    const float xer = edr * c2 + edi * s2x, xei = edi * c2 - edr * s2x;  // x E'
                    const float ur = orr + 2.0f * (odr * c2 + odi * s2x), ui = oi + 2.0f * (odi * c2 - odr * s2x);
                    const float dr = 2.0f * xer + (ur * rc + ui * rs), di = 2.0f * xei + (ui * rc - ur * rs);
                    // H' = omega_0 H + dlt D
                    const float h2r = omega * hr + a.dlt * dr;
                    const float h2i = omega * hi + a.dlt * di;
                    const float pwr = pr * wr - pi * wi, pwi = pr * wi + pi * wr;  // psi w at f0
                    const float xr = pwr * hr - pwi * hi, xi = pwr * hi + pwi * hr;  // psi w H
                    const float yr = pwr * h2r - pwi * h2i, yi = pwr * h2i + pwi * h2r;  // psi w H'
                    g_alpha = xr - Qr * iom;
                    Theta = Q2i;
                    Phi = alpha * yi;
                    g_pr = alpha * (wr * hr - wi * hi);
                    g_pi = -alpha * (wr * hi + wi * hr);
                    Qr += alpha * xr;
                    Qi += alpha * xi;
                    Q2r += alpha * yr;
                    Q2i += alpha * yi;
                }
                // transmittance phase theta_s = omega_s b dt
                const float g_b = Theta * pg.dt;
                const float g_dt = Theta * s2.z;
                // alpha = o g, g = exp(-m2r / 2)
                float g_o = 0.0f, g_m2r = 0.0f;
                if (!clamped) {
                    g_o = g_alpha * gw;
                    g_m2r = -0.5f * g_alpha * o * gw;
                }
                // (m2r, dt) <- (A, B, C); t_mid = -B/A, h = sqrt((9 - m2)/A), B = -A t_mid.
                // d dt / d m2 = -1 / (A h) is unbounded as the ray grazes the 3-sigma
                // boundary, but m2 itself is only known to about 1e-6 |w| in FP32 (C = |w|^2
                // reaches 1e5): below the chord such an error allows, h_f = sqrt(2e-6 |w| / A),
                // the chord is rounding noise, so its derivatives are taken at h_f there
                const float A = pg.A, tm = pg.tm;
                const float wn = sqrtf(v1.x * v1.x + v1.y * v1.y + v1.z * v1.z);
                const float h = fmaxf(pg.h, sqrtf(2e-6f * wn * pg.iA));
                const float iAh = 1.0f / (A * h);
                float gA, gB, gC;
                if (tm - pg.h >= r_rx) {  // the chord is not clipped at the emitting sphere
                    gA = g_m2r * tm * tm - g_dt * (tm * tm + h * h) * iAh;
                    gB = g_m2r * 2.0f * tm - g_dt * 2.0f * tm * iAh;
                    gC = g_m2r - g_dt * iAh;
                } else {
                    const float t_out = pg.t_out, t_rep = 0.5f * (r_rx + t_out);
                    const float doA = -t_out * pg.iA - 0.5f * (tm * tm - h * h) * iAh;
                    const float doB = (-1.0f - tm / h) * pg.iA;
                    const float doC = -0.5f * iAh;
                    const float lin = A * pg.dl;  // half of d m2r / d t_rep
                    gA = g_m2r * (t_rep * t_rep + lin * doA) + g_dt * doA;
                    gB = g_m2r * (2.0f * t_rep + lin * doB) + g_dt * doB;
                    gC = g_m2r * (1.0f + lin * doC) + g_dt * doC;
                }
                // A = |v'|^2, B = w.v', C = |w|^2
                const float w0 = v1.x, w1 = v1.y, w2 = v1.z;
                const float gv0 = 2.0f * gA * pg.vx + gB * w0, gv1 = 2.0f * gA * pg.vy + gB * w1,
                            gv2 = 2.0f * gA * pg.vz + gB * w2;
                const float gw0 = gB * pg.vx + 2.0f * gC * w0, gw1 = gB * pg.vy + 2.0f * gC * w1,
                            gw2 = gB * pg.vz + 2.0f * gC * w2;
                // v' = W v, w = W (r - mu) with r - mu = -c
                const float ux = -v0.x, uy = -v0.y, uz = -v0.z;
                go[0] = gv0 * dx + gw0 * ux; go[1] = gv0 * dy + gw0 * uy; go[2] = gv0 * dz + gw0 * uz;
                go[3] = gv1 * dx + gw1 * ux; go[4] = gv1 * dy + gw1 * uy; go[5] = gv1 * dz + gw1 * uz;
                go[6] = gv2 * dx + gw2 * ux; go[7] = gv2 * dy + gw2 * uy; go[8] = gv2 * dz + gw2 * uz;
                // dL/dmu = -W^T g_w + (path) g_phi omega (unit(mu - t) + unit(mu - r))
                float gmx = -(s0.x * gw0 + s0.w * gw1 + s1.z * gw2);
                float gmy = -(s0.y * gw0 + s1.x * gw1 + s1.w * gw2);
                float gmz = -(s0.z * gw0 + s1.y * gw1 + s2.x * gw2);
                const float mx = v0.x + rx, my = v0.y + ry, mz = v0.z + rz;
                const float tx = mx - a.txpos[0], ty = my - a.txpos[1], tz = mz - a.txpos[2];
                const float it = rsqrtf(fmaxf(tx * tx + ty * ty + tz * tz, 1e-30f));
                const float ir = rsqrtf(fmaxf(v0.x * v0.x + v0.y * v0.y + v0.z * v0.z, 1e-30f));
                const float gd = Phi;
                gmx += gd * (tx * it + v0.x * ir);
                gmy += gd * (ty * it + v0.y * ir);
                gmz += gd * (tz * it + v0.z * ir);
                go[9] = gmx; go[10] = gmy; go[11] = gmz;
                go[12] = g_o;
                go[13] = g_b;
            }
            float* acc = a.acc + (size_t)sid[bf][j] * grad_floats(L);
            // coefficient gradients, per chunk c of 16 basis values: value v (0..31) is
            // g_pr b[16 c + v] for v < 16 and g_pi b[16 c + v - 16] after, summed over the
            // warp's rays.  Stored in slot v ^ lane, every lane keeps the lower half and
            // sends the upper half in every butterfly round, with no selects; lane L ends
            // with value L, added to accumulator 14 + 32 c + L.
            {
                const bool sw = (lane & 16) != 0;
                const float ga = sw ? g_pi : g_pr, gb = sw ? g_pr : g_pi;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    float q[32];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float bi = sbp[16 * c + i][lane];
                        q[i] = ga * bi;
                        q[16 + i] = gb * bi;
                    }
#pragma unroll
                    for (int off = 16, n = 32; off >= 1; off >>= 1, n >>= 1) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (i < n / 2) q[i] += __shfl_xor_sync(0xffffffffu, q[i + n / 2], off);
                    }
                    atomicAdd(acc + 14 + 32 * c + lane, q[0]);
                }
            }
            const float so = reduce_scatter16(go, lane);
            if ((lane & 1) == 0 && (lane >> 1) < 14) atomicAdd(acc + (lane >> 1), so);
        }
        mask = next;
        if (a.ck) {
            // in front of list position b0: take the forward's own transmittance where it
            // kept one, so that division by (1 - alpha) runs over at most K positions
            const int p = b0;
            if (p > 0 && p % a.ck_every == 0 && p / a.ck_every <= a.ck_slots && valid) {
                const size_t rays = (size_t)a.n_rx * gr.n_el * gr.n_az;
                const size_t ray = ((size_t)r * gr.n_el + v) * gr.n_az + u;
                const float4 c = a.ck[(size_t)(p / a.ck_every - 1) * rays + ray];
                Tr = c.x;
                Ti = c.y;
                Gam = c.z;
            }
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Persistent launch: every warp takes work items (receiver, tile, ray block) from one
// counter, heaviest first, until none is left.  One frequency: 5 CTAs per SM up to L = 3
// (at most 102 registers, no spills), 4 at L = 4, 3 at L = 5 (the larger basis).  Several
// frequencies: 2, with each warp's upstream rows in dynamic shared memory (66 KB per CTA
// at 64 subcarriers).
template <bool MF, int L>
__global__ void __launch_bounds__(kBThreads, MF ? 2 : (L <= 3 ? 5 : (L == 4 ? 4 : 3)))
    k_render_bwd(BwdArgs a, const uint32_t* __restrict__ order, unsigned long long* __restrict__ counter,
                 unsigned long long total) {
    __shared__ float4 sbuf[kBW][2][kBB][6];
    __shared__ uint32_t sid[kBW][2][kBB];
    __shared__ float4 spl[kBW][kPlaneSlots];
    __shared__ float sbp[kBW][16 * grad_chunks(L)][32];
    __shared__ float4 scoef[kBW][2][kBCoefSlots][8];
    extern __shared__ float4 sgrad[];  // several frequencies: [warp][lane][g_stride4]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned per_rx = (unsigned)a.n_tiles * (unsigned)a.per_tile;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total) break;
        const uint32_t id = order[it];
        const unsigned rem = id % per_rx;
        bwd_block<MF, L>(a, (int)(id / per_rx), (int)(rem / (unsigned)a.per_tile), (int)(rem % (unsigned)a.per_tile),
                         sbuf[warp], sid[warp], spl[warp], sbp[warp], scoef[warp],
                         MF ? sgrad + (size_t)warp * 32 * a.g_stride4 : nullptr);
        __syncwarp();
    }
}

// Raw-parameter gradients from the accumulators (one thread per Gaussian, += into the
// caller's buffers; any may be null).
template <int L>
__global__ void __launch_bounds__(256) k_grad_params(gsrf_gaussians g, const GShape* __restrict__ shape,
                                                     const float* __restrict__ acc, float* g_means,
                                                     float* g_log_scales, float* g_quats, float* g_opacity_logit,
                                                     float* g_coeffs, float* g_phase_b, int variant) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const float* A = acc + (size_t)k * grad_floats(L);
    // the normalised-weight variant: the opacity in alpha is o N, N = e^{-(l0 + l1 + l2)} /
    // (2 pi)^1.5 (folded into the shape record the same way), so dL/dlogit carries N and
    // every log-scale also gets -o N dL/d(o N)
    const float o = 1.0f / (1.0f + expf(-g.opacity_logit[k]));
    const float N = (variant & GSRF_VARIANT_NORMALISED_WEIGHT)
                        ? expf(-(g.log_scales[3 * k] + g.log_scales[3 * k + 1] + g.log_scales[3 * k + 2])) *
                              0.0634936359f
                        : 1.0f;
    const float gN = (variant & GSRF_VARIANT_NORMALISED_WEIGHT) ? -A[12] * o * N : 0.0f;
    // W = diag(1/s) R^T: W_ij = R_ji / s_i
    float qw = g.quats[4 * k], qx = g.quats[4 * k + 1], qy = g.quats[4 * k + 2], qz = g.quats[4 * k + 3];
    const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    const bool degenerate = !(n2 > 0.0f);
    const float qn = degenerate ? 1.0f : sqrtf(n2);
    if (degenerate) { qw = 1.0f; qx = qy = qz = 0.0f; }
    else { qw /= qn; qx /= qn; qy /= qn; qz /= qn; }
    const float R[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy),
                        2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx),
                        2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)};
    float GR[9];
    for (int i = 0; i < 3; ++i) {
        const float is = expf(-g.log_scales[3 * k + i]);
        float gis = 0.0f;
        for (int j = 0; j < 3; ++j) {
            GR[3 * j + i] = A[3 * i + j] * is;  // dL/dR_ji
            gis += A[3 * i + j] * R[3 * j + i];
        }
        if (g_log_scales) g_log_scales[3 * k + i] += -gis * is + gN;  // d(1/s)/dls = -1/s
    }
    if (g_quats) {
        const float dw[9] = {0, -2 * qz, 2 * qy, 2 * qz, 0, -2 * qx, -2 * qy, 2 * qx, 0};
        const float ddx[9] = {0, 2 * qy, 2 * qz, 2 * qy, -4 * qx, -2 * qw, 2 * qz, 2 * qw, -4 * qx};
        const float ddy[9] = {-4 * qy, 2 * qx, 2 * qw, 2 * qx, 0, 2 * qz, -2 * qw, 2 * qz, -4 * qy};
        const float ddz[9] = {-4 * qz, -2 * qw, 2 * qx, 2 * qw, -4 * qz, 2 * qy, 2 * qx, 2 * qy, 0};
        float gq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int i = 0; i < 9; ++i) {
            gq[0] += GR[i] * dw[i];
            gq[1] += GR[i] * ddx[i];
            gq[2] += GR[i] * ddy[i];
            gq[3] += GR[i] * ddz[i];
        }
        if (!degenerate) {
            const float qh[4] = {qw, qx, qy, qz};
            const float dot = gq[0] * qh[0] + gq[1] * qh[1] + gq[2] * qh[2] + gq[3] * qh[3];
            for (int i = 0; i < 4; ++i) g_quats[4 * k + i] += (gq[i] - qh[i] * dot) / qn;
        }
    }
    if (g_means)
        for (int i = 0; i < 3; ++i) g_means[3 * k + i] += A[9 + i];
    if (g_opacity_logit) {
        g_opacity_logit[k] += A[12] * N * o * (1.0f - o);  // through the sigmoid (and N)
    }
    if (g_phase_b) g_phase_b[k] += A[13];
    if (g_coeffs) {
        // accumulator 14 + 32 c + v: dL/d psi_re (v < 16) or dL/d psi_im (v >= 16) times
        // basis value 16 c + v % 16 of (1, P_10 .. P_L0, Re Y, Im Y of the Y_{l,m>0});
        // restored to the folded coefficients (see fle_floats), then unfolded
        constexpr int NB = (L + 1) * (L + 1);
        auto gre = [&](int i) { return A[14 + 32 * (i / 16) + i % 16]; };
        auto gim = [&](int i) { return A[14 + 32 * (i / 16) + 16 + i % 16]; };
        float* gc = g_coeffs + (size_t)k * 2 * NB;
        for (int l = 0; l <= L; ++l) {  // m = 0: c_{l,0} multiplies P_l0 (P_00 = 1)
            gc[2 * (l * l + l)] += gre(l);
            gc[2 * (l * l + l) + 1] += gim(l);
        }
        // m > 0, m-major: e1 = cr + dr, e2 = di - ci, e3 = ci + di, e4 = cr - dr with
        // d = kappa c_{l,-m}, kappa = (-1)^m (l-m)!/(l+m)!; e1, e2 multiply Re, Im Y in psi_re,
        // e3, e4 in psi_im
        int t = 0;
        for (int m = 1; m <= L; ++m) {
            for (int l = m; l <= L; ++l, ++t) {
                float prod = 1.0f;
                for (int i = l - m + 1; i <= l + m; ++i) prod *= (float)i;
                const float kap = ((m & 1) ? -1.0f : 1.0f) / prod;
                const int yb = 1 + L + 2 * t;
                const float e1 = gre(yb), e2 = gre(yb + 1), e3 = gim(yb), e4 = gim(yb + 1);
                const int np = l * l + l + m, nm = l * l + l - m;
                gc[2 * np] += e1 + e4;
                gc[2 * np + 1] += e3 - e2;
                gc[2 * nm] += kap * (e1 - e4);
                gc[2 * nm + 1] += kap * (e2 + e3);
            }
        }
    }
}

cudaError_t launch_render_bwd(const gsrf_plan* p, const Layout& L, const gsrf_gaussians* g, void* ws,
                              const void* ray_state, const float* grad_rays, float* g_means, float* g_log_scales,
                              float* g_quats, float* g_opacity_logit, float* g_coeffs, float* g_phase_b,
                              cudaStream_t st) {
    if (L.n == 0) return cudaSuccess;
    float* acc = at<float>(ws, L.gacc);
    const int deg = plan_degree(p);
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)L.n * grad_floats(deg) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    BwdArgs a;
    a.shape = at<GShape>(ws, L.gshape);
    a.view = at<View>(ws, L.view);
    a.fle = at<float>(ws, L.fle);
    a.raytab = at<float>(ws, L.raytab);
    a.pids = at<uint32_t>(ws, L.pids);
    a.rx_base = at<long long>(ws, L.rx_base);
    a.tile_start = at<uint32_t>(ws, L.tile_start);
    a.rxpos = at<float>(ws, L.rxpos);
    a.txpos = at<float>(ws, L.txpos);
    a.rs = static_cast<const RayState*>(ray_state);
    a.grad_rays = grad_rays;
    a.acc = acc;
    a.gr = p->grid;
    a.ntu = L.ntu;
    a.n_tiles = L.n_tiles;
    a.n = L.n;
    a.om_pi = (float)(2.0 * p->f0_hz / kC);
    a.n_f = p->n_f;
    a.dlt = (float)(2.0 * 3.14159265358979323846 * p->df_hz / kC);
    const int bw = plan_block_w(p);
    a.bw_log = __builtin_ctz((unsigned)bw);
    a.nbx = p->grid.tile_w / bw;
    a.per_tile = p->grid.tile_w * p->grid.tile_h / 32;
    a.g_pairs = (p->n_f + 1) / 2;
    a.g_stride4 = a.g_pairs | 1;  // an odd stride keeps the lanes' 16-byte reads conflict-free
    const size_t dyn = p->n_f > 1 ? (size_t)kBW * 32 * a.g_stride4 * sizeof(float4) : 0;
    a.n_rx = L.n_rx;
    const size_t rays = (size_t)p->n_rx * p->grid.n_az * p->grid.n_el;
    a.ck = p->ckpt_every > 0
               ? reinterpret_cast<const float4*>(static_cast<const char*>(ray_state) + rays * sizeof(RayState))
               : nullptr;
    a.ck_every = p->ckpt_every > 0 ? p->ckpt_every : 1;
    a.ck_slots = p->ckpt_slots;
    a.variant = p->variant;
    a.circle = (p->variant & GSRF_VARIANT_PAPER_CULLING) ? at<float4>(ws, L.circle) : nullptr;
    uint32_t* order = nullptr;
    unsigned long long* counter = nullptr;
    if ((e = launch_item_order(L, ws, a.per_tile, &order, &counter, st)) != cudaSuccess) return e;
    const long long n = (long long)L.n_rx * L.n_tiles * a.per_tile;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    auto run = [&](auto kernel) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (r != cudaSuccess) return r;
        int per_sm = 0;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBThreads, dyn);
        if (r != cudaSuccess) return r;
        const int grid = (int)max(1ll, min((long long)sms * max(per_sm, 1), (n + kBW - 1) / kBW));
        kernel<<<grid, kBThreads, dyn, st>>>(a, order, counter, (unsigned long long)n);
        return cudaGetLastError();
    };
    if (p->n_f == 1) {
        switch (deg) {  // several frequencies: L = 3 only (checked with the plan)
            case 1: e = run(k_render_bwd<false, 1>); break;
            case 2: e = run(k_render_bwd<false, 2>); break;
            case 4: e = run(k_render_bwd<false, 4>); break;
            case 5: e = run(k_render_bwd<false, 5>); break;
            default: e = run(k_render_bwd<false, 3>); break;
        }
    } else {
        e = run(k_render_bwd<true, 3>);
    }
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((L.n + 255) / 256);
    const GShape* sh = at<GShape>(ws, L.gshape);
    switch (deg) {
        case 1: k_grad_params<1><<<nb, 256, 0, st>>>(*g, sh, acc, g_means, g_log_scales, g_quats, g_opacity_logit, g_coeffs, g_phase_b, p->variant); break;
        case 2: k_grad_params<2><<<nb, 256, 0, st>>>(*g, sh, acc, g_means, g_log_scales, g_quats, g_opacity_logit, g_coeffs, g_phase_b, p->variant); break;
        case 4: k_grad_params<4><<<nb, 256, 0, st>>>(*g, sh, acc, g_means, g_log_scales, g_quats, g_opacity_logit, g_coeffs, g_phase_b, p->variant); break;
        case 5: k_grad_params<5><<<nb, 256, 0, st>>>(*g, sh, acc, g_means, g_log_scales, g_quats, g_opacity_logit, g_coeffs, g_phase_b, p->variant); break;
        default: k_grad_params<3><<<nb, 256, 0, st>>>(*g, sh, acc, g_means, g_log_scales, g_quats, g_opacity_logit, g_coeffs, g_phase_b, p->variant); break;
    }
    return cudaGetLastError();
}

}  // namespace gsrf
