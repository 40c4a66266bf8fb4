// k_signal.cu -- received signal from the per-ray signals (Sec. 4.4, loss paragraph):
// the single-antenna complex sum over rays, its power in dB, the incoherent power sum,
// and the spatial-spectrum magnitude.  FP64 accumulation in a fixed order.
#include <math.h>

#include "gsrf_internal.cuh"

namespace gsrf {

constexpr int kSigThreads = 256;

// One block per (receiver, frequency): thread t sums rays t, t + 256, ...; then a
// fixed tree in shared memory.  The order never depends on timing.
__global__ void __launch_bounds__(kSigThreads) k_signal_sum(const float2* __restrict__ rays, int n_rays, int mode,
                                                            float* __restrict__ out) {
    __shared__ double sr[kSigThreads], si[kSigThreads], sp[kSigThreads];
    const float2* S = rays + (size_t)blockIdx.x * n_rays;
    double ar = 0.0, ai = 0.0, ap = 0.0;
    for (int i = threadIdx.x; i < n_rays; i += kSigThreads) {
        const float2 s = S[i];
        ar += (double)s.x;
        ai += (double)s.y;
        ap += (double)s.x * s.x + (double)s.y * s.y;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    sp[threadIdx.x] = ap;
    __syncthreads();
    for (int w = kSigThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
            sp[threadIdx.x] += sp[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (mode == GSRF_SIG_COMPLEX_SUM) {
            out[2 * blockIdx.x] = (float)sr[0];
            out[2 * blockIdx.x + 1] = (float)si[0];
        } else if (mode == GSRF_SIG_RSSI_DB) {
            out[blockIdx.x] = (float)(10.0 * log10(sr[0] * sr[0] + si[0] * si[0]));
        } else {
            out[blockIdx.x] = (float)sp[0];
        }
    }
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
        k_signal_sum<<<n_rx * n_f, kSigThreads, 0, st>>>(R, n_el * n_az, mode, out);
    }
    return cudaGetLastError();
}

}  // namespace gsrf
