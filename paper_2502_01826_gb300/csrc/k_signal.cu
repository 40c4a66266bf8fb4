// k_signal.cu -- received signal from the per-ray signals (Sec. 4.4, loss paragraph):
// the single-antenna complex sum over rays, its power in dB, the incoherent power sum,
// and the spatial-spectrum magnitude.  Accumulation in a fixed order: each thread sums its
// rays in compensated FP32 (Knuth's two-sum, an error-free transformation of each
// addition, so the pair (sum, error) carries the exact running sum up to the error
// term's own rounding), then the threads' partials are added in FP64.
#include <cooperative_groups.h>
#include <math.h>

#include "gsrf_internal.cuh"

namespace cg = cooperative_groups;

namespace gsrf {

constexpr int kSigThreads = 256;

constexpr int kSigCluster = 8;  // CTAs per (receiver, frequency) sum

// s + c += x: Knuth's two-sum of s and x (the rounded sum t and its exact error), the
// error added to the compensation c.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// One thread-block cluster of kSigCluster CTAs per (receiver, frequency): CTA c, thread t
// sums rays c * 256 + t + k * 256 * kSigCluster (k = 0, 1, ...) in compensated FP32 (the
// power sum, of positive terms, in plain FP32) and converts its partial to FP64 once; a
// fixed FP64 tree in shared memory gives each CTA's partial, and CTA 0 adds the partials
// of CTAs 0 .. kSigCluster - 1, in that order, through distributed shared memory.  The
// order never depends on timing, and all SMs share the work.
__global__ void __cluster_dims__(kSigCluster, 1, 1) __launch_bounds__(kSigThreads)
    k_signal_sum(const float2* __restrict__ rays, int n_rays, int mode, float* __restrict__ out) {
    __shared__ double sr[kSigThreads], si[kSigThreads], sp[kSigThreads];
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int rf = blockIdx.x / kSigCluster;
    const float2* S = rays + (size_t)rf * n_rays;
    float fr = 0.0f, cr = 0.0f, fi = 0.0f, ci = 0.0f, fp = 0.0f;
    const bool power = mode == GSRF_SIG_POWER_SUM;
    for (int i = c * kSigThreads + threadIdx.x; i < n_rays; i += kSigThreads * kSigCluster) {
        const float2 s = S[i];
        two_sum_acc(fr, cr, s.x);
        two_sum_acc(fi, ci, s.y);
        if (power) fp += s.x * s.x + s.y * s.y;
    }
    sr[threadIdx.x] = (double)fr + (double)cr;
    si[threadIdx.x] = (double)fi + (double)ci;
    sp[threadIdx.x] = (double)fp;
    __syncthreads();
    for (int w = kSigThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
            sp[threadIdx.x] += sp[threadIdx.x + w];
        }
        __syncthreads();
    }
    cl.sync();  // every CTA's partial is in its shared memory
    if (c == 0 && threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0, tp = 0.0;
        for (int k = 0; k < kSigCluster; ++k) {
            tr += *cl.map_shared_rank(&sr[0], k);
            ti += *cl.map_shared_rank(&si[0], k);
            tp += *cl.map_shared_rank(&sp[0], k);
        }
        if (mode == GSRF_SIG_COMPLEX_SUM) {
            out[2 * rf] = (float)tr;
            out[2 * rf + 1] = (float)ti;
        } else if (mode == GSRF_SIG_RSSI_DB) {
            out[rf] = (float)(10.0 * log10(tr * tr + ti * ti));
        } else {
            out[rf] = (float)tp;
        }
    }
    cl.sync();  // CTA 0 has read the others' shared memory
}

__global__ void k_spectrum_mag(const float2* __restrict__ rays, size_t n, float* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 s = rays[i];
        out[i] = sqrtf(s.x * s.x + s.y * s.y);
    }
}

cudaError_t launch_signal(const float* rays, int n_rx, int n_f, int n_el, int n_az, int mode, float* out,
                          cudaStream_t st) {
    const float2* R = reinterpret_cast<const float2*>(rays);
    if (mode == GSRF_SIG_SPECTRUM_MAG) {
        const size_t n = (size_t)n_rx * n_f * n_el * n_az;
        const unsigned blocks = (unsigned)min((size_t)152 * 16, (n + 255) / 256);
        k_spectrum_mag<<<blocks, 256, 0, st>>>(R, n, out);
    } else {
        k_signal_sum<<<n_rx * n_f * kSigCluster, kSigThreads, 0, st>>>(R, n_el * n_az, mode, out);
    }
    return cudaGetLastError();
}

}  // namespace gsrf
