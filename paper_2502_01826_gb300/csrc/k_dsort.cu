// k_dsort.cu -- the depth sort of the key sort (Alg. 1, App. E) for one receiver inside
// one thread-block cluster.  The per-receiver sort is a stable LSD radix sort like the
// one in k_bin.cu (the first pass dropping the Gaussians that cover no tile, ties in input
// order, so ties by Gaussian index), but over key - min of the receiver's visible keys:
// the FP32 depth bits of one room span about 26 bits, so 9-bit digits need three passes
// instead of four 8-bit ones (as many 9-bit passes as the span needs up to 27 bits, else
// four 8-bit passes).  Subtracting the minimum keeps the order of the keys, so the
// permutation is the same.  The keys stay on chip between the passes: the cluster's CTAs
// hold the receiver's (key, id) items in shared memory, each pass ranks them with warp
// peer groups and stores every item straight into the shared memory of the CTA that holds
// its new position (distributed shared memory).  The keys are read from HBM once and the
// sorted ids written once, in one launch instead of twelve.
//
// Layout: CTA c of the cluster holds positions [c * sl, (c + 1) * sl) of the current
// order, sl = ceil(m / C) for the m items of the pass; warp w of a CTA takes a
// contiguous run of ceil(sl / threads) * 32 of them, 32 per round, so the order
// (CTA, warp, round, lane) is the position order and the ranks keep it.
#include "gsrf_internal.cuh"
#include <atomic>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace gsrf {

constexpr int kCsThreads = 1024;
constexpr int kCsWarps = kCsThreads / 32;
constexpr int kCsIpt = 16;                   // items a thread holds at most
constexpr int kCsCap = kCsThreads * kCsIpt;  // items a CTA holds at most
constexpr int kCsMaxCluster = 8;             // larger clusters measured slower than the global passes
constexpr int kCsStride = kCsWarps + 1;      // padded digit row of the per-warp counts
constexpr int kCsRankShift = 20;             // id in the low 20 bits, rank above
constexpr uint32_t kCsNone = 0xffffffffu;    // an empty register slot

static_assert((long long)kCsCap * kCsMaxCluster <= (1ll << kCsRankShift), "ids must fit below the rank");
static_assert(kCsIpt * 32 <= (1 << (32 - kCsRankShift - 1)), "ranks must fit above the id");

constexpr int kCsDigits = 512;  // 9-bit digits at most
struct CsShared {
    uint2 item[kCsCap];                    // (key - min, Gaussian id) at the CTA's positions
    uint32_t wcnt[kCsDigits * kCsStride];  // per (digit, warp): count, then exclusive prefix
    uint32_t ctot[kCsDigits];              // the CTA's count per digit (read by the cluster)
    uint32_t base[kCsDigits];              // the digit's first position for this CTA's items
    uint32_t wsum[kCsDigits / 32];
    uint32_t total;
    uint32_t kmin, kmax;                   // the CTA's visible keys (read by the cluster)
    uint32_t gmin, gmax;                   // the receiver's, over the cluster
    unsigned long long inv;  // ceil(2^40 / slice): dest / slice as one multiply and shift
};

// Rank the registers' items of one pass: per warp and digit, the running count in
// wcnt gives each item its place among the warp's items of the same digit.
__device__ __forceinline__ void cs_rank(const uint32_t (&key)[kCsIpt], uint32_t (&val)[kCsIpt], int ipt, int shift,
                                        int width, uint32_t* wcnt, int warp, uint32_t lt) {
    const uint32_t dmask = (1u << width) - 1u;
#pragma unroll
    for (int j = 0; j < kCsIpt; ++j) {
        if (j < ipt) {  // warp-uniform
            const bool valid = val[j] != kCsNone;
            const uint32_t dg = valid ? (key[j] >> shift) & dmask : kCsNone;
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                if (b < width) {  // uniform
                    const uint32_t bb = __ballot_sync(0xffffffffu, (dg >> b) & 1u);
                    peers &= ((dg >> b) & 1u) ? bb : ~bb;
                }
            }
            const uint32_t r = (uint32_t)__popc(peers & lt);
            uint32_t old = 0;
            if (valid) old = wcnt[dg * kCsStride + warp];
            __syncwarp();
            if (valid && r == 0) wcnt[dg * kCsStride + warp] = old + (uint32_t)__popc(peers);
            __syncwarp();
            if (valid) val[j] |= (old + r) << kCsRankShift;
        }
    }
}

// One cluster of C CTAs per receiver (grid n_rx * C).  dkey: the receivers' n depth keys
// each (kAbsentKey: covers no tile); dval: gets each receiver's ids (0 .. n - 1) of the
// Gaussians that cover a tile, in (depth, id) order, at the receiver's offset r * n;
// nvis: their number per receiver.
__global__ void __launch_bounds__(kCsThreads, 1)
    k_depth_sort_cluster(const uint32_t* __restrict__ dkey, long long n, uint32_t* __restrict__ dval,
                         uint32_t* __restrict__ nvis) {
    extern __shared__ __align__(16) unsigned char cs_raw[];
    CsShared& S = *reinterpret_cast<CsShared*>(cs_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    const long long rx = blockIdx.x / C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t* keys = dkey + rx * n;

    for (int i = threadIdx.x; i < kCsDigits * kCsStride; i += kCsThreads) S.wcnt[i] = 0;
    if (threadIdx.x == 0) {
        S.kmin = 0xffffffffu;
        S.kmax = 0u;
    }

    uint32_t key[kCsIpt], val[kCsIpt];
    // pass 0 reads CTA c's slice of the n keys from global memory
    // (positions fit in 32 bits: n <= kCsCap * kCsMaxCluster)
    int sl = (int)((n + C - 1) / C);
    int lo = min(c * sl, (int)n);
    int m = min(sl, (int)n - lo);
    int ipt = (m + kCsThreads - 1) / kCsThreads;
    int wbeg = warp * ipt * 32;
#pragma unroll
    for (int j = 0; j < kCsIpt; ++j) {
        key[j] = 0;
        val[j] = kCsNone;
        const int p = wbeg + j * 32 + lane;
        if (j < ipt && p < m) {
            key[j] = keys[lo + p];
            if (key[j] != kAbsentKey) val[j] = (uint32_t)(lo + p);
        }
    }
    __syncthreads();  // wcnt, kmin and kmax cleared
    // the span of the receiver's visible keys, so that the sort runs over key - min and
    // over as few digits as that needs
    {
        uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
        for (int j = 0; j < kCsIpt; ++j)
            if (val[j] != kCsNone) {
                mn = min(mn, key[j]);
                mx = max(mx, key[j]);
            }
        mn = __reduce_min_sync(0xffffffffu, mn);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) {
            atomicMin(&S.kmin, mn);
            atomicMax(&S.kmax, mx);
        }
    }
    cl.sync();
    if (warp == 0) {
        uint32_t mn = 0xffffffffu, mx = 0u;
        if (lane < C) {
            mn = *cl.map_shared_rank(&S.kmin, lane);
            mx = *cl.map_shared_rank(&S.kmax, lane);
        }
        mn = __reduce_min_sync(0xffffffffu, mn);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) {
            S.gmin = mn;
            S.gmax = mx;
        }
    }
    __syncthreads();
    const uint32_t gmin = S.gmin;
    const uint32_t span = S.gmax >= gmin ? S.gmax - gmin : 0u;
    const int bits = 32 - __clz((int)span);
    const int width = bits <= 27 ? 9 : 8;
    const int npass = bits <= 27 ? max(1, (bits + 8) / 9) : 4;
#pragma unroll
    for (int j = 0; j < kCsIpt; ++j)
        if (val[j] != kCsNone) key[j] -= gmin;
    const int nb = 1 << width;

    for (int pass = 0; pass < npass; ++pass) {
        const int shift = width * pass;
        const bool last = pass == npass - 1;
        if (pass > 0) {
#pragma unroll
            for (int j = 0; j < kCsIpt; ++j) {
                key[j] = 0;
                val[j] = kCsNone;
                const int p = wbeg + j * 32 + lane;
                if (j < ipt && p < m) {
                    const uint2 it = S.item[p];
                    key[j] = it.x;
                    val[j] = it.y;
                }
            }
        }
        cs_rank(key, val, ipt, shift, width, S.wcnt, warp, lt);
        __syncthreads();
        // per digit, the exclusive prefix over the warps and the CTA's count
        for (int d = warp; d < nb; d += kCsWarps) {
            const uint32_t v = S.wcnt[d * kCsStride + lane];
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            S.wcnt[d * kCsStride + lane] = x - v;
            if (lane == 31) S.ctot[d] = x;
        }
        cl.sync();  // every CTA's counts are complete, and every item is in registers
        uint32_t tot = 0, before = 0, incl = 0;
        if (threadIdx.x < nb) {
            const int d = threadIdx.x;
            for (int q = 0; q < C; ++q) {
                const uint32_t x = cl.map_shared_rank(S.ctot, q)[d];
                if (q < c) before += x;
                tot += x;
            }
            incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) S.wsum[warp] = incl;
        }
        __syncthreads();
        if (threadIdx.x < nb) {
            uint32_t wb = 0, all = 0;
#pragma unroll
            for (int w = 0; w < kCsDigits / 32; ++w) {
                if (w < nb / 32) {
                    if (w < warp) wb += S.wsum[w];
                    all += S.wsum[w];
                }
            }
            S.base[threadIdx.x] = wb + incl - tot + before;
            if (threadIdx.x == 0) {
                S.total = all;
                // dest < 2^20 and slice <= 2^14, so (dest * ceil(2^40 / slice)) >> 40 is the
                // exact quotient (Granlund and Montgomery, 1994: the error term dest * e /
                // 2^40 with e < slice stays below 1 / slice)
                const unsigned long long sl_n = ((unsigned long long)all + C - 1) / C;
                S.inv = sl_n ? ((1ull << 40) + sl_n - 1) / sl_n : 0ull;
            }
        }
        __syncthreads();
        const uint32_t m_next = S.total;  // items in the cluster after this pass
        if (pass == 0 && c == 0 && threadIdx.x == 0) nvis[rx] = m_next;
        const uint32_t sl_next = (m_next + (uint32_t)C - 1u) / (uint32_t)C;
        const unsigned long long inv = S.inv;
#pragma unroll
        for (int j = 0; j < kCsIpt; ++j) {
            if (j < ipt && val[j] != kCsNone) {
                const uint32_t d = (key[j] >> shift) & (uint32_t)(nb - 1);
                const uint32_t id = val[j] & ((1u << kCsRankShift) - 1u);
                const uint32_t dest = S.base[d] + S.wcnt[d * kCsStride + warp] + (val[j] >> kCsRankShift);
                if (last) {
                    dval[rx * n + dest] = id;
                } else {
                    const uint32_t q = (uint32_t)(((unsigned long long)dest * inv) >> 40);
                    cl.map_shared_rank(S.item, (int)q)[dest - q * sl_next] = make_uint2(key[j], id);
                }
            }
        }
        cl.sync();  // every item is in place and every count read
        for (int i = threadIdx.x; i < nb * kCsStride; i += kCsThreads) S.wcnt[i] = 0;
        sl = (int)sl_next;
        lo = min(c * sl, (int)m_next);
        m = min(sl, (int)m_next - lo);
        ipt = (m + kCsThreads - 1) / kCsThreads;
        wbeg = warp * ipt * 32;
        __syncthreads();
    }
}

// Cluster size for n keys per receiver, 0 when the cluster sort does not apply (more keys
// than kCsMaxCluster CTAs hold, or no cluster of that size fits on the device).  Above 8
// CTAs (13 for 200k Gaussians) only one cluster fits per GPC and the global passes are
// faster.  Whether a cluster size fits is a property of the device, cached per device; the
// kernel's shared-memory attribute is set again before every launch (a device reset clears
// it).
constexpr int kCsMaxDevices = 64;
static int cluster_for(long long n) {
    if (n <= 0) return 0;
    const long long C = (n + kCsCap - 1) / kCsCap;
    if (C > kCsMaxCluster) return 0;
    int dev = 0;
    if (cudaPeekAtLastError() != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess || dev < 0 ||
        dev >= kCsMaxDevices)
        return 0;  // leave a pending error to its caller
    // 0 unknown, 1 fits, -1 does not
    static std::atomic<int> fits[kCsMaxDevices][kCsMaxCluster + 1] = {};
    if (fits[dev][C].load(std::memory_order_relaxed) == 0) {
        int ok = -1;
        const int smem = (int)sizeof(CsShared);
        if (cudaFuncSetAttribute(k_depth_sort_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)C);
            cfg.blockDim = dim3(kCsThreads);
            cfg.dynamicSmemBytes = (size_t)smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k_depth_sort_cluster, &cfg) == cudaSuccess && clusters > 0)
                ok = 1;
        }
        (void)cudaGetLastError();  // a refused attribute is an answer, not an error of the call
        fits[dev][C].store(ok, std::memory_order_relaxed);  // racing threads store the same answer
    }
    return fits[dev][C].load(std::memory_order_relaxed) > 0 ? (int)C : 0;
}

bool depth_sort_cluster_applies(long long n) { return cluster_for(n) > 0; }

cudaError_t launch_depth_sort_cluster(const uint32_t* dkey, long long n, int n_rx, uint32_t* dval, uint32_t* nvis,
                                      cudaStream_t st) {
    const int C = cluster_for(n);
    if (C == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_depth_sort_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(CsShared));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(n_rx * C));
    cfg.blockDim = dim3(kCsThreads);
    cfg.dynamicSmemBytes = sizeof(CsShared);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_depth_sort_cluster, dkey, n, dval, nvis);
}

}  // namespace gsrf
