// k_bin.cu -- the key sort of Alg. 1 and App. E: splat keys (tile << 32 | depth), one
// sort, tile ranges.  The 64-bit sort is done as
//   (1) a stable LSD radix sort of each receiver's n FP32 depth keys (4 x 8-bit digits);
//   (2) emission of the (tile, Gaussian) pairs in that depth order;
//   (3) a stable counting sort of each receiver's pairs by tile (the high 32 bits),
// which leaves every tile's Gaussians in (depth, index) order: the same permutation as
// one stable sort of the full 64-bit keys, with 4 passes over n keys and one pass over
// the pairs instead of 8 passes over the pairs.
//
// Every pass is a (histogram, scan, scatter) triple over blocks of kChunk items.
// Ranks inside a block come from warp peer groups (one ballot per digit bit), so equal
// digits keep their input order: the sort is stable and its output deterministic.  Passes
// with at most 256 bins scatter four keys per thread per round (k_scatter4).
#include "gsrf_internal.cuh"

namespace gsrf {

// Which items a block owns.  Segments are receivers; either one every eq_len items (of
// length eq_len, or len[s] <= eq_len when len is given: the blocks past a segment's end
// own nothing) or given by base[] with chunk_base[] = prefix of ceil(len / kChunk).
// drop: keys equal to kAbsentKey are left out (counted by no histogram, written by no
// scatter), so a pass that drops them compacts each segment.
struct Segs {
    int n_seg;
    long long eq_len;  // >= 0: segments at multiples of eq_len, in blocks of eq_chunk items
    int eq_chunks;     // blocks per segment (ceil(eq_len / eq_chunk))
    int eq_chunk;
    const long long* base;
    const uint32_t* chunk_base;
    const uint32_t* len;  // equal-stride segments: their lengths (null: eq_len each)
    int drop;
};

__device__ __forceinline__ bool block_items(const Segs& S, long long b, long long& lo, long long& hi,
                                            long long& seg_lo, int& seg) {
    if (S.eq_len >= 0) {
        seg = (int)(b / S.eq_chunks);
        const long long c = b % S.eq_chunks;
        if (seg >= S.n_seg) return false;
        seg_lo = (long long)seg * S.eq_len;
        lo = seg_lo + c * S.eq_chunk;
        hi = min(lo + (long long)S.eq_chunk, seg_lo + (S.len ? (long long)S.len[seg] : S.eq_len));
        return lo < hi;
    }
    if (b >= (long long)S.chunk_base[S.n_seg]) return false;
    int a = 0, z = S.n_seg - 1;
    while (a < z) {
        const int m = (a + z + 1) >> 1;
        if ((long long)S.chunk_base[m] <= b) a = m;
        else z = m - 1;
    }
    seg = a;
    seg_lo = S.base[a];
    lo = seg_lo + (b - (long long)S.chunk_base[a]) * kChunk;
    hi = min(lo + (long long)kChunk, S.base[a + 1]);
    return lo < hi;
}

__device__ __forceinline__ void chunk_range(const Segs& S, int seg, long long& c0, long long& c1) {
    if (S.eq_len >= 0) {
        c0 = (long long)seg * S.eq_chunks;
        c1 = c0 + (S.len ? (long long)((S.len[seg] + S.eq_chunk - 1) / S.eq_chunk) : S.eq_chunks);
    } else {
        c0 = S.chunk_base[seg];
        c1 = S.chunk_base[seg + 1];
    }
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
    return (uint32_t)(key >> shift) & mask;
}

__device__ __forceinline__ bool capacity_failed(const DevStatus* st) {
    return st != nullptr && *(volatile const int32_t*)&st->code == (int32_t)GSRF_ERR_CAPACITY;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_hist(const K* __restrict__ keys, Segs S, int shift,
                                                       uint32_t mask, int nbins, uint32_t* __restrict__ H,
                                                       const DevStatus* st) {
    if (capacity_failed(st)) return;
    __shared__ uint32_t h[kMaxTiles];
    long long lo, hi, seg_lo;
    int seg;
    if (!block_items(S, blockIdx.x, lo, hi, seg_lo, seg)) return;
    for (int i = threadIdx.x; i < nbins; i += kSortThreads) h[i] = 0;
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += kSortThreads) {
        const K key = keys[i];
        if (!(S.drop && key == (K)kAbsentKey)) atomicAdd(&h[digit_of(key, shift, mask)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += kSortThreads) H[(size_t)blockIdx.x * nbins + i] = h[i];
}

// Block-wide exclusive scan of one value per thread (kSortThreads threads).
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total, T* sh /* [kSortWarps] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    T wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        if (w < warp) wbase += sh[w];
        tot += sh[w];
    }
    __syncthreads();
    if (total) *total = tot;
    return wbase + x - v;
}

// One block per segment: turn per-block digit counts H[block][digit] into absolute
// destinations inside the segment; optionally record each digit's [start, end) and the
// segment's item count.  With fewer digits than threads, each digit's chunks are split
// over G = threads / nbins groups of threads (one pass that sums the groups' spans, one
// that writes the destinations), so that the whole block walks the counts.
__global__ void __launch_bounds__(kSortThreads) k_scan(Segs S, int nbins, uint32_t* __restrict__ H,
                                                       uint32_t* __restrict__ bin_start,
                                                       const DevStatus* st, uint32_t* __restrict__ seg_total = nullptr) {
    if (capacity_failed(st)) return;
    __shared__ uint32_t tot[kMaxTiles];
    __shared__ uint32_t sstart[kMaxTiles];
    __shared__ uint32_t part[kSortThreads];  // per (group, digit): the sum of the groups before
    __shared__ uint32_t sh[kSortWarps];
    const int seg = blockIdx.x;
    long long c0, c1;
    chunk_range(S, seg, c0, c1);
    const int G = nbins < kSortThreads ? kSortThreads / nbins : 1;
    const long long span = (c1 - c0 + G - 1) / G;
    for (int t = threadIdx.x; t < G * nbins; t += kSortThreads) {
        const int d = t % nbins, g = t / nbins;
        const long long a = c0 + g * span, b = min(a + span, c1);
        uint32_t run = 0;
        for (long long cb = a; cb < b; cb += 8) {  // 8 independent loads in flight
#pragma unroll
            for (int j = 0; j < 8; ++j) run += cb + j < b ? H[(size_t)(cb + j) * nbins + d] : 0u;
        }
        if (G > 1) part[t] = run;
        else tot[d] = run;
    }
    __syncthreads();
    if (G > 1) {
        for (int d = threadIdx.x; d < nbins; d += kSortThreads) {
            uint32_t p = 0;
            for (int g = 0; g < G; ++g) {
                const uint32_t x = part[g * nbins + d];
                part[g * nbins + d] = p;
                p += x;
            }
            tot[d] = p;
        }
        __syncthreads();
    }
    // exclusive scan over digits, kSortThreads at a time
    uint32_t carry = 0;
    for (int d0 = 0; d0 < nbins; d0 += kSortThreads) {
        const int d = d0 + threadIdx.x;
        const uint32_t v = d < nbins ? tot[d] : 0u;
        uint32_t t;
        const uint32_t ex = block_excl_scan<uint32_t>(v, &t, sh);
        if (d < nbins) {
            sstart[d] = carry + ex;
            if (bin_start) bin_start[(size_t)seg * (nbins + 1) + d] = carry + ex;
        }
        carry += t;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < G * nbins; t += kSortThreads) {
        const int d = t % nbins, g = t / nbins;
        const long long a = c0 + g * span, b = min(a + span, c1);
        uint32_t run = sstart[d] + (G > 1 ? part[t] : 0u);
        for (long long cb = a; cb < b; cb += 8) {
            uint32_t v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = cb + j < b ? H[(size_t)(cb + j) * nbins + d] : 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (cb + j < b) H[(size_t)(cb + j) * nbins + d] = run;
                run += v[j];
            }
        }
    }
    if (bin_start && threadIdx.x == 0) bin_start[(size_t)seg * (nbins + 1) + nbins] = carry;
    if (seg_total && threadIdx.x == 0) seg_total[seg] = carry;
}

// Stable scatter.  vin == nullptr: the value is the item's index inside its segment;
// kout == nullptr: only the values are written.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                          K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                          Segs S, int shift, uint32_t mask, int nbins,
                                                          const uint32_t* __restrict__ H, const DevStatus* st) {
    if (capacity_failed(st)) return;
    __shared__ uint32_t base[kMaxTiles];
    __shared__ uint8_t cnt[kSortWarps][kMaxTiles];
    long long lo, hi, seg_lo;
    int seg;
    if (!block_items(S, blockIdx.x, lo, hi, seg_lo, seg)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < nbins; d += kSortThreads) {
        base[d] = H[(size_t)blockIdx.x * nbins + d];
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) cnt[w][d] = 0;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (long long r0 = lo; r0 < hi; r0 += kSortThreads) {
        const long long i = r0 + threadIdx.x;
        bool valid = i < hi;
        K key = 0;
        uint32_t val = 0, d = 0xffffffffu;
        if (valid) {
            key = kin[i];
            valid = !(S.drop && key == (K)kAbsentKey);
        }
        if (valid) {
            val = vin ? vin[i] : (uint32_t)(i - seg_lo);
            d = digit_of(key, shift, mask);
        }
        // lanes with the same digit: one ballot per digit bit (every digit is below
        // nbins), and the same validity
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
        if (!valid) peers = ~peers;
        for (uint32_t bit = 1; bit < (uint32_t)nbins; bit <<= 1) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d & bit) != 0);
            peers &= (d & bit) ? bb : ~bb;
        }
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) cnt[warp][d] = (uint8_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = base[d] + rank;
            for (int w = 0; w < warp; ++w) off += cnt[w][d];
            if (kout) kout[seg_lo + off] = key;
            vout[seg_lo + off] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < nbins; dd += kSortThreads) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                t += cnt[w][dd];
                cnt[w][dd] = 0;
            }
            base[dd] += t;
        }
        __syncthreads();
    }
}

// Stable scatter for at most 256 bins, four keys per thread per round: key s of thread t
// is item r0 + 256 s + t, so the (sub-round, warp, lane) order of a round of 1024 keys is
// the input order.  Ranks inside a warp come from ballots; a per-digit exclusive prefix
// over the 32 (sub-round, warp) slots, in that order, places each warp's group.  The
// round's keys are first gathered in shared memory in (digit, input) order and then
// written out by consecutive threads, so that each digit's run of the round goes to
// consecutive addresses instead of one scattered store per key.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_scatter4(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           Segs S, int shift, uint32_t mask, int nbins,
                                                           const uint32_t* __restrict__ H, const DevStatus* st) {
    if (capacity_failed(st)) return;
    constexpr int R = 4;
    __shared__ uint32_t base[256];
    __shared__ uint32_t tot[256];
    __shared__ uint32_t lstart[256];  // the digit's first place in the round's reordered keys
    __shared__ uint16_t cnt[R][kSortWarps][256];
    __shared__ K skey[R * kSortThreads];
    __shared__ uint32_t sval[R * kSortThreads];
    __shared__ uint32_t sh[kSortWarps];
    long long lo, hi, seg_lo;
    int seg;
    if (!block_items(S, blockIdx.x, lo, hi, seg_lo, seg)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        base[d] = d < nbins ? H[(size_t)blockIdx.x * nbins + d] : 0u;
#pragma unroll
        for (int s = 0; s < R; ++s)
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) cnt[s][w][d] = 0;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (long long r0 = lo; r0 < hi; r0 += R * kSortThreads) {
        K key[R];
        uint32_t val[R], dg[R];
        int rank[R];
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const long long i = r0 + (long long)s * kSortThreads + threadIdx.x;
            bool valid = i < hi;
            key[s] = 0;
            val[s] = 0;
            dg[s] = 0xffffffffu;
            if (valid) {
                key[s] = kin[i];
                valid = !(S.drop && key[s] == (K)kAbsentKey);
            }
            if (valid) {
                val[s] = vin ? vin[i] : (uint32_t)(i - seg_lo);
                dg[s] = digit_of(key[s], shift, mask);
            }
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
            for (uint32_t bit = 1; bit < (uint32_t)nbins; bit <<= 1) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (dg[s] & bit) != 0);
                peers &= (dg[s] & bit) ? bb : ~bb;
            }
            rank[s] = __popc(peers & lt);
            if (valid && rank[s] == 0) cnt[s][warp][dg[s]] = (uint16_t)__popc(peers);
        }
        __syncthreads();
        // per digit (one per thread), the exclusive prefix over the slots in (sub-round,
        // warp) order, the round's count, and the digit's start in the reordered round
        const int d = threadIdx.x;
        uint32_t run = 0;
        if (d < nbins) {
            uint32_t c[R][kSortWarps];  // all loads first: one latency instead of a chain of 32
#pragma unroll
            for (int s = 0; s < R; ++s)
#pragma unroll
                for (int w = 0; w < kSortWarps; ++w) c[s][w] = cnt[s][w][d];
#pragma unroll
            for (int s = 0; s < R; ++s)
#pragma unroll
                for (int w = 0; w < kSortWarps; ++w) {
                    cnt[s][w][d] = (uint16_t)run;
                    run += c[s][w];
                }
            tot[d] = run;
        }
        uint32_t n_round;
        const uint32_t ls = block_excl_scan<uint32_t>(run, &n_round, sh);
        if (d < nbins) lstart[d] = ls;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < R; ++s) {
            if (dg[s] != 0xffffffffu) {
                const uint32_t lp = lstart[dg[s]] + cnt[s][warp][dg[s]] + (uint32_t)rank[s];
                skey[lp] = key[s];
                sval[lp] = val[s];
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < n_round; j += kSortThreads) {
            const K k = skey[j];
            const uint32_t dj = digit_of(k, shift, mask);
            const uint32_t off = base[dj] + (j - lstart[dj]);
            if (kout) kout[seg_lo + off] = k;
            vout[seg_lo + off] = sval[j];
        }
        __syncthreads();
        if (d < nbins) {
            base[d] += tot[d];
#pragma unroll
            for (int s = 0; s < R; ++s)
#pragma unroll
                for (int w = 0; w < kSortWarps; ++w) cnt[s][w][d] = 0;
        }
        __syncthreads();
    }
}

// The four-keys scatter where every digit is below 256, else one key per thread.
template <typename K>
static void launch_scatter(unsigned blocks, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, Segs S,
                           int shift, uint32_t mask, int nbins, const uint32_t* H, const DevStatus* st_dev,
                           cudaStream_t st) {
    if (nbins <= 256)
        k_scatter4<K><<<blocks, kSortThreads, 0, st>>>(kin, vin, kout, vout, S, shift, mask, nbins, H, st_dev);
    else
        k_scatter<K><<<blocks, kSortThreads, 0, st>>>(kin, vin, kout, vout, S, shift, mask, nbins, H, st_dev);
}

// ---- emission -------------------------------------------------------------

// Position of the k-th (from 0) set bit of x; k < popc(x).
__device__ __forceinline__ int select_bit(uint32_t x, uint32_t k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const uint32_t c = (uint32_t)__popc(x & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Per (receiver, emission chunk of kEChunk depth-sorted Gaussians): number of pairs,
// and for each group of 32 consecutive Gaussians of the chunk (the emission's work item)
// its first pair relative to the chunk's.  A receiver's sorted Gaussians are the
// nvis[r] that cover some tile.
__global__ void __launch_bounds__(kSortThreads) k_count_chunks(const uint32_t* __restrict__ dval,
                                                               const Cover* __restrict__ cover, long long n,
                                                               const uint32_t* __restrict__ nvis, int dchunks,
                                                               uint32_t* __restrict__ chunk_sum,
                                                               uint32_t* __restrict__ group_off) {
    constexpr int G = kEChunk / 32;  // groups per chunk
    __shared__ uint32_t gs[G];
    const int r = blockIdx.y, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long lo = (long long)c * kEChunk, hi = min(lo + (long long)kEChunk, (long long)nvis[r]);
    // group g = items 32 g .. 32 g + 31 of the chunk: round g / kSortWarps, warp g % kSortWarps
    for (int k = 0; k < kEChunk / kSortThreads; ++k) {
        const long long i = lo + (long long)k * kSortThreads + threadIdx.x;
        uint32_t v = i < hi ? cover[(size_t)r * n + dval[(size_t)r * n + i]].count : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) gs[k * kSortWarps + warp] = v;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan over the chunk's groups (G = 32: one per lane)
        const uint32_t v = gs[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        group_off[((size_t)r * dchunks + c) * G + lane] = x - v;
        if (lane == 31) chunk_sum[(size_t)r * dchunks + c] = x;
    }
}

// One block: chunk offsets per receiver, receiver bases, capacity check, the chunk
// table of the tile sort and the slice table of the emission.  A warp scans one
// receiver's chunk sums 32 at a time (shuffles); the receivers' bases are block scans,
// kSortThreads receivers at a time.
__global__ void __launch_bounds__(kSortThreads) k_scan_pairs(uint32_t* __restrict__ chunk_sum, int n_rx, int dchunks,
                                                             long long cap, long long* __restrict__ rx_base,
                                                             uint32_t* __restrict__ rx_total,
                                                             uint32_t* __restrict__ pchunk_base, DevStatus* st,
                                                             uint32_t* __restrict__ eslice_base) {
    __shared__ long long shl[kSortWarps];
    __shared__ uint32_t shu[kSortWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < n_rx; r += kSortWarps) {
        uint32_t* cs = chunk_sum + (size_t)r * dchunks;
        uint32_t carry = 0;
        for (int c0 = 0; c0 < dchunks; c0 += 32) {
            const int c = c0 + lane;
            const uint32_t v = c < dchunks ? cs[c] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (c < dchunks) cs[c] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) rx_total[r] = carry;
    }
    __syncthreads();
    long long b = 0;
    uint32_t cb = 0, es = 0;
    for (int r0 = 0; r0 < n_rx; r0 += kSortThreads) {
        const int r = r0 + threadIdx.x;
        const uint32_t t = r < n_rx ? rx_total[r] : 0u;
        long long tb;
        uint32_t tc, te;
        const long long xb = block_excl_scan<long long>((long long)t, &tb, shl);
        const uint32_t xc = block_excl_scan<uint32_t>((t + kChunk - 1) / kChunk, &tc, shu);
        const uint32_t xe = block_excl_scan<uint32_t>((t + kESlice - 1) / kESlice, &te, shu);
        if (r < n_rx) {
            rx_base[r] = b + xb;
            pchunk_base[r] = cb + xc;
            eslice_base[r] = es + xe;
        }
        b += tb;
        cb += tc;
        es += te;
    }
    if (threadIdx.x == 0) {
        rx_base[n_rx] = b;
        pchunk_base[n_rx] = cb;
        eslice_base[n_rx] = es;
        st->required_pairs = b;
    }
    if (b > cap) {  // uniform: every thread holds the same totals
        if (threadIdx.x == 0) atomicCAS(&st->code, (int)GSRF_OK, (int)GSRF_ERR_CAPACITY);
        __syncthreads();
        // a failed bin leaves no pairs: downstream kernels see empty lists
        for (int r = threadIdx.x; r <= n_rx; r += kSortThreads) {
            rx_base[r] = 0;
            pchunk_base[r] = 0;
            eslice_base[r] = 0;
        }
    }
}

// Expand the depth-sorted Gaussians into their (tile, Gaussian) pairs, written
// contiguously in depth order as (tile index, Gaussian id).  The work is split into
// slices of kESlice consecutive pairs of a receiver (eslice_base), one per warp at a time,
// so that the nearest Gaussians, whose covers are the widest, spread over many warps
// instead of one.  A slice finds the group of 32 sorted Gaussians that holds its first
// pair by a binary search over the groups' first pairs (chunk_off + group_off), loads that
// group and writes the slice's part of the group's run 32 slots at a time (coalesced):
// each slot finds its Gaussian by a search over the warp's inclusive counts and its tile
// from its index inside that Gaussian's cover (elevation rows of the set azimuth tiles,
// in order); then it goes on with the next group until the slice is done.  The group
// loads are pipelined: the sorted ids two groups ahead and the covers one group ahead are
// in flight while a group is written.
__global__ void __launch_bounds__(kSortThreads) k_emit(const uint32_t* __restrict__ dval,
                                                       const Cover* __restrict__ cover, long long n,
                                                       const uint32_t* __restrict__ nvis, int dchunks,
                                                       const uint32_t* __restrict__ chunk_off,
                                                       const uint32_t* __restrict__ group_off,
                                                       const long long* __restrict__ rx_base,
                                                       const uint32_t* __restrict__ rx_total,
                                                       const uint32_t* __restrict__ eslice_base, int n_rx, int ntu,
                                                       const uint32_t* __restrict__ pchunk_base, int n_tiles,
                                                       uint32_t* __restrict__ thist,
                                                       uint32_t* __restrict__ ptile, uint32_t* __restrict__ pids,
                                                       const DevStatus* st) {
    if (capacity_failed(st)) return;
    constexpr int G = kEChunk / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t slices = eslice_base[n_rx];
    const uint32_t warps = gridDim.x * kSortWarps;
    for (uint32_t w = blockIdx.x * kSortWarps + (threadIdx.x >> 5); w < slices; w += warps) {
        // receiver: the last r with eslice_base[r] <= w
        int r = 0;
        for (int z = n_rx; r < z;) {
            const int mid = (r + z + 1) >> 1;
            if (eslice_base[mid] <= w) r = mid;
            else z = mid - 1;
        }
        const uint32_t total_r = rx_total[r];
        uint32_t P0 = (w - eslice_base[r]) * (uint32_t)kESlice;
        const uint32_t P1 = min(P0 + (uint32_t)kESlice, total_r);
        const long long nv = nvis[r];
        const int ng = (int)((nv + 31) / 32);
        const uint32_t* co = chunk_off + (size_t)r * dchunks;
        const uint32_t* go = group_off + (size_t)r * dchunks * G;
        // the group that holds pair P0: the last g with first pair <= P0
        int g = 0;
        for (int z = ng - 1; g < z;) {
            const int mid = (g + z + 1) >> 1;
            if (co[mid / G] + go[mid] <= P0) g = mid;
            else z = mid - 1;
        }
        uint32_t* kout = ptile + rx_base[r];
        uint32_t* iout = pids + rx_base[r];
        // loads pipelined across groups: the ids two groups ahead, the covers one ahead
        const uint32_t* dv = dval + (size_t)r * n;
        const Cover* cov = cover + (size_t)r * n;
        auto id_of = [&](int gg) -> uint32_t {
            const long long i = (long long)gg * 32 + lane;
            return (gg < ng && i < nv) ? dv[i] : 0xffffffffu;
        };
        uint32_t id_c = id_of(g), id_n = id_of(g + 1);
        Cover cv_c = {0ull, 0u, 0u};
        if (id_c != 0xffffffffu) cv_c = cov[id_c];
        while (P0 < P1 && g < ng) {  // uniform over the warp
            Cover cv_n = {0ull, 0u, 0u};
            if (id_n != 0xffffffffu) cv_n = cov[id_n];
            const uint32_t id_nn = id_of(g + 2);
            const uint32_t gid = id_c != 0xffffffffu ? id_c : 0u;
            const uint32_t cnt = cv_c.count, tvw = cv_c.tv;
            const uint32_t mlo = (uint32_t)cv_c.mask, mhi = (uint32_t)(cv_c.mask >> 32);
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t base = co[g / G] + go[g];  // the group's first pair
            const uint32_t q1 = min(P1 - base, total);
            for (uint32_t s0 = P0 - base; s0 < q1; s0 += 32) {
                const uint32_t q = s0 + lane;
                int j = 0;  // lanes whose inclusive count is <= q: the owner of slot q
#pragma unroll
                for (int b = 16; b; b >>= 1) {
                    const uint32_t t = __shfl_sync(0xffffffffu, incl, j + b - 1);
                    if (t <= q) j += b;
                }
                const uint32_t oi = __shfl_sync(0xffffffffu, incl, j), oc = __shfl_sync(0xffffffffu, cnt, j);
                const uint32_t ogid = __shfl_sync(0xffffffffu, gid, j);
                const uint32_t otv = __shfl_sync(0xffffffffu, tvw, j);
                const uint32_t olo = __shfl_sync(0xffffffffu, mlo, j), ohi = __shfl_sync(0xffffffffu, mhi, j);
                if (q < q1) {
                    const uint32_t p = q - (oi - oc);  // pair index inside the owner's cover
                    const uint32_t nlo = __popc(olo), nb = nlo + __popc(ohi);
                    const uint32_t row = p / nb, col = p - row * nb;
                    const int tu = col < nlo ? select_bit(olo, col) : 32 + select_bit(ohi, col - nlo);
                    const int tv = (int)(otv & 0xffffu) + (int)row;
                    const uint32_t tile = (uint32_t)(tv * ntu + tu);
                    kout[base + q] = tile;
                    // the tile pass's histogram: pairs per (pair chunk of kChunk, tile)
                    atomicAdd(thist + (size_t)(pchunk_base[r] + (base + q) / (uint32_t)kChunk) * n_tiles + tile, 1u);
                    iout[base + q] = ogid;
                }
            }
            P0 = base + total;
            ++g;
            id_c = id_n;
            cv_c = cv_n;
            id_n = id_nn;
        }
    }
}

// The bin's zeroed state in one launch: tile ranges, the emission's tile histogram and
// the receivers' first pairs (all zero: no pairs, should the bin stop early).
__global__ void k_zero_bin(uint32_t* ts, size_t nts, uint32_t* th, size_t nth, long long* rxb, int nrxb) {
    const size_t step = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t i = t0; i < nts; i += step) ts[i] = 0;
    for (size_t i = t0; i < nth; i += step) th[i] = 0;
    for (size_t i = t0; i < (size_t)nrxb; i += step) rxb[i] = 0;
}

// One stable counting pass over n 32-bit keys (digit = key & (nbins - 1), nbins <= 256):
// vals_out gets the item indices in key order.  hist needs ceil(n / kSmallChunk) * nbins
// words.  Blocks of kSmallChunk keys (one round of k_scatter4) spread the few tens of
// thousands of work items over many SMs.
cudaError_t launch_sort_small_keys(const uint32_t* keys, uint32_t* keys_out, uint32_t* vals_out, long long n,
                                   int nbins, uint32_t* hist, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int chunks = (int)((n + kSmallChunk - 1) / kSmallChunk);
    Segs sg{1, n, chunks, kSmallChunk, nullptr, nullptr, nullptr, 0};
    k_hist<uint32_t><<<chunks, kSortThreads, 0, st>>>(keys, sg, 0, (uint32_t)(nbins - 1), nbins, hist, nullptr);
    k_scan<<<1, kSortThreads, 0, st>>>(sg, nbins, hist, nullptr, nullptr);
    launch_scatter<uint32_t>(chunks, keys, nullptr, keys_out, vals_out, sg, 0, (uint32_t)(nbins - 1), nbins, hist,
                             nullptr, st);
    return cudaGetLastError();
}

// The same per segment: n_seg segments of items [seg_base[s], seg_base[s + 1]) (device),
// chunk_base = the prefix of their ceil(length / kChunk) (device, n_seg + 1 entries),
// chunks = chunk_base[n_seg].  vals_out gets each item's index inside its segment, in
// key order within the segment.  hist needs chunks * nbins words.
cudaError_t launch_sort_small_keys_segmented(const uint32_t* keys, uint32_t* keys_out, uint32_t* vals_out, int n_seg,
                                             const long long* seg_base, const uint32_t* chunk_base, long long chunks,
                                             int nbins, uint32_t* hist, cudaStream_t st) {
    if (chunks == 0) return cudaSuccess;
    Segs sg{n_seg, -1, 0, kChunk, seg_base, chunk_base, nullptr, 0};
    k_hist<uint32_t><<<(unsigned)chunks, kSortThreads, 0, st>>>(keys, sg, 0, (uint32_t)(nbins - 1), nbins, hist,
                                                                nullptr);
    k_scan<<<n_seg, kSortThreads, 0, st>>>(sg, nbins, hist, nullptr, nullptr);
    launch_scatter<uint32_t>((unsigned)chunks, keys, nullptr, keys_out, vals_out, sg, 0, (uint32_t)(nbins - 1), nbins,
                             hist, nullptr, st);
    return cudaGetLastError();
}

cudaError_t launch_bin(const gsrf_plan* p, const Layout& L, void* ws, cudaStream_t st) {
    const bool on_chip = depth_sort_cluster_applies(L.n);  // before any launch of this call
    DevStatus* status = at<DevStatus>(ws, L.status);
    const size_t nts = (size_t)L.n_rx * (L.n_tiles + 1);
    const size_t nth = (size_t)L.pchunks_max * L.n_tiles;
    const size_t nz = max(nts, nth);
    k_zero_bin<<<(unsigned)min((nz + 255) / 256, (size_t)4096), 256, 0, st>>>(
        at<uint32_t>(ws, L.tile_start), nts, at<uint32_t>(ws, L.thist), nth, at<long long>(ws, L.rx_base), L.n_rx + 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (L.n == 0) return cudaSuccess;

    // (1) depth sort, per receiver: keys dkey -> dkey2 -> dkey ..., values likewise.  The
    // first pass drops the Gaussians that cover no tile (key kAbsentKey) and records how
    // many are left per receiver; the other passes sort only those.  Receivers whose keys
    // fit in one cluster's shared memory are sorted on chip (k_dsort.cu), the same
    // permutation in one launch.
    uint32_t* nvis = at<uint32_t>(ws, L.dvis);
    const Segs ds_all{L.n_rx, L.n, L.dchunks, kDChunk, nullptr, nullptr, nullptr, 1};
    const Segs ds_vis{L.n_rx, L.n, L.dchunks, kDChunk, nullptr, nullptr, nvis, 0};
    const unsigned dblocks = (unsigned)(L.n_rx * L.dchunks);
    uint32_t* k_in = at<uint32_t>(ws, L.dkey);
    uint32_t* k_out = at<uint32_t>(ws, L.dkey2);
    uint32_t* v_in = nullptr;
    uint32_t* v_out = at<uint32_t>(ws, L.dval);
    uint32_t* v_alt = at<uint32_t>(ws, L.dval2);
    uint32_t* H = at<uint32_t>(ws, L.dhist);
    const int passes = on_chip ? 0 : 4;
    if (passes == 0) {  // all four passes on chip, one cluster per receiver
        if ((e = launch_depth_sort_cluster(k_in, L.n, L.n_rx, v_out, nvis, st)) != cudaSuccess) return e;
        v_in = v_out;
    }
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        const Segs& ds = pass == 0 ? ds_all : ds_vis;
        k_hist<uint32_t><<<dblocks, kSortThreads, 0, st>>>(k_in, ds, shift, 0xffu, 256, H, nullptr);
        k_scan<<<L.n_rx, kSortThreads, 0, st>>>(ds, 256, H, nullptr, nullptr, pass == 0 ? nvis : nullptr);
        // the last pass writes the sorted ids only: nothing reads the sorted keys
        launch_scatter<uint32_t>(dblocks, k_in, v_in, pass == 3 ? nullptr : k_out, v_out, ds, shift, 0xffu, 256, H,
                                 nullptr, st);
        uint32_t* t = k_in; k_in = k_out; k_out = t;
        v_in = v_out;
        v_out = (v_out == at<uint32_t>(ws, L.dval)) ? v_alt : at<uint32_t>(ws, L.dval);
    }
    const uint32_t* dval_sorted = v_in;  // each receiver's ids in (depth, id) order

    // (2) emission in depth order
    uint32_t* chunk_sum = at<uint32_t>(ws, L.dchunk_sum);
    uint32_t* group_off = at<uint32_t>(ws, L.egroup);
    uint32_t* eslice_base = at<uint32_t>(ws, L.eslice);
    k_count_chunks<<<dim3(L.echunks, L.n_rx), kSortThreads, 0, st>>>(dval_sorted, at<Cover>(ws, L.cover), L.n,
                                                                       nvis, L.echunks, chunk_sum, group_off);
    k_scan_pairs<<<1, kSortThreads, 0, st>>>(chunk_sum, L.n_rx, L.echunks, L.cap, at<long long>(ws, L.rx_base),
                                             at<uint32_t>(ws, L.rx_total), at<uint32_t>(ws, L.pchunk_base), status,
                                             eslice_base);
    // one resident wave of warps striding over the slices
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_emit, kSortThreads, 0)) != cudaSuccess) return e;
    const long long max_slices = ((long long)L.cap + kESlice - 1) / kESlice + L.n_rx;
    const unsigned emit_grid =
        (unsigned)max(1ll, min((long long)sms * max(per_sm, 1), (max_slices + kSortWarps - 1) / kSortWarps));
    uint32_t* ptile = at<uint32_t>(ws, L.pkeys2);  // the pairs' tile indices, in depth order
    uint32_t* TH = at<uint32_t>(ws, L.thist);       // zeroed by k_zero_bin, filled by the emission
    k_emit<<<emit_grid, kSortThreads, 0, st>>>(dval_sorted, at<Cover>(ws, L.cover), L.n, nvis, L.echunks, chunk_sum,
                                               group_off, at<long long>(ws, L.rx_base), at<uint32_t>(ws, L.rx_total),
                                               eslice_base, L.n_rx, L.ntu, at<uint32_t>(ws, L.pchunk_base), L.n_tiles,
                                               TH, ptile, at<uint32_t>(ws, L.pids2), status);

    // (3) stable counting sort of each receiver's pairs by tile index: ids pids2 -> pids (the
    // 64-bit splat keys are formed only on request, by launch_pair_keys)
    Segs ps{L.n_rx, -1, 0, kChunk, at<long long>(ws, L.rx_base), at<uint32_t>(ws, L.pchunk_base), nullptr, 0};
    const unsigned pblocks = (unsigned)L.pchunks_max;
    k_scan<<<L.n_rx, kSortThreads, 0, st>>>(ps, L.n_tiles, TH, at<uint32_t>(ws, L.tile_start), status);
    launch_scatter<uint32_t>(pblocks, ptile, at<uint32_t>(ws, L.pids2), nullptr, at<uint32_t>(ws, L.pids), ps, 0,
                             0xffffffffu, L.n_tiles, TH, status, st);
    (void)p;
    return cudaGetLastError();
}

// The sorted 64-bit splat keys (tile << 32 | FP32 depth bits) of the last bin, for
// inspection: the render needs only the ids and the tile ranges.  One block per (tile,
// receiver); the depth bits are recomputed from the view record's c = mu - r by the same
// deterministic operations as the projection's depth key.
__global__ void __launch_bounds__(kSortThreads) k_pair_keys(const View* __restrict__ view,
                                                            const uint32_t* __restrict__ pids,
                                                            const long long* __restrict__ rx_base,
                                                            const uint32_t* __restrict__ tile_start, int n_tiles,
                                                            long long n, unsigned long long* __restrict__ keys) {
    const int t = blockIdx.x, r = blockIdx.y;
    const size_t ts = (size_t)r * (n_tiles + 1) + t;
    const uint32_t b = tile_start[ts], e = tile_start[ts + 1];
    for (uint32_t i = b + threadIdx.x; i < e; i += kSortThreads) {
        const long long p = rx_base[r] + i;
        const View& v = view[(size_t)r * n + pids[p]];
        keys[p] = ((unsigned long long)(uint32_t)t << 32) | __float_as_uint(depth_of(v.c[0], v.c[1], v.c[2]));
    }
}

cudaError_t launch_pair_keys(const Layout& L, void* ws, cudaStream_t st) {
    if (L.n == 0 || L.n_tiles == 0) return cudaSuccess;
    k_pair_keys<<<dim3(L.n_tiles, L.n_rx), kSortThreads, 0, st>>>(
        at<View>(ws, L.view), at<uint32_t>(ws, L.pids), at<long long>(ws, L.rx_base), at<uint32_t>(ws, L.tile_start),
        L.n_tiles, L.n, at<unsigned long long>(ws, L.pkeys));
    return cudaGetLastError();
}

}  // namespace gsrf
