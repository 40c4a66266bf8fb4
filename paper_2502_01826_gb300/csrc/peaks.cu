// peaks.cu -- throughput microbenchmarks of the GB300 pipes that bound the render:
// FP32 fused multiply-add (scalar and the packed pair form fma.rn.f32x2), the
// special-function unit (ex2, rcp, rsqrt, sqrt, sin, cos), FP64 fused multiply-add and
// TF32 matrix multiply-accumulate (the warp-level mma.sync form).  They give the denominators of the render's roofline; they are measurement
// tools of this library, not part of the render (libgsrf_peaks.so, separate from
// libgsrf.so).
//
// Each kernel runs `iters` rounds of 16 dependent steps on each of 8 independent chains
// per thread (per warp for the matrix form), so the pipe, not latency, is the limit once
// the grid fills the SMs.  A chain's value is written only if it equals a value it
// cannot take, which keeps the compiler from dropping the work.  The ex2 chain runs into
// +inf and stays there; the unit's rate does not depend on the operand's value.  A
// special-function step also carries one FP32 add (see step).
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsrf_peaks {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

enum Kind {
    FMA32 = 0, EX2 = 1, RCP = 2, RSQRT = 3, SQRT = 4, SIN = 5, COS = 6, FMA64 = 7, MMA_TF32 = 8, FMA32X2 = 9,
    N_KINDS = 10
};

// One dependent step of a chain.  The special-function kinds take f(x + b): the add (on
// the FP32 pipe, eight times wider than the special-function unit) keeps the assembler
// from folding a chain such as rcp(rcp(x)) back to x.
template <int K>
__device__ __forceinline__ float step(float x, float a, float b) {
    float y;
    if constexpr (K == FMA32) asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(x), "f"(a), "f"(b));
    if constexpr (K == EX2)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; ex2.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    if constexpr (K == RCP)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; rcp.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    if constexpr (K == RSQRT)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; rsqrt.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    if constexpr (K == SQRT)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; sqrt.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    if constexpr (K == SIN)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; sin.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    if constexpr (K == COS)
        asm volatile("{ .reg .f32 t; add.f32 t, %1, %2; cos.approx.ftz.f32 %0, t; }" : "=f"(y) : "f"(x), "f"(b));
    return y;
}

template <int K>
__global__ void __launch_bounds__(256) k_scalar(int iters, float* out) {
    const float a = 0.999f + 1e-9f * threadIdx.x, b = 1e-3f;
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 0.01f * c + 1e-6f * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = step<K>(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma64(int iters, float* out) {
    const double a = 0.999 + 1e-12 * threadIdx.x, b = 1e-3;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 0.01 * c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5) out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// Packed FP32 pairs: one fma.rn.f32x2 instruction is two fused multiply-adds.
__global__ void __launch_bounds__(256) k_fma32x2(int iters, float* out) {
    unsigned long long x[kChains], a, b;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(0.999f + 1e-9f * threadIdx.x), "f"(0.998f));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(1e-3f), "f"(2e-3f));
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(0.5f + 0.01f * c), "f"(0.25f));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a), "l"(b));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == -1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + D for a 16 x 8 x 8 TF32 tile per warp instruction (2048 FLOP), eight
// independent accumulators per warp.
__global__ void __launch_bounds__(256) k_mma_tf32(int iters, float* out) {
    uint32_t a0 = 0x3f800000u ^ threadIdx.x, a1 = 0x3f000000u, a2 = 0x3e800000u, a3 = 0x3e000000u;
    uint32_t b0 = 0x3f800000u, b1 = 0x3f000000u ^ threadIdx.x;
    float d[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0.0f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};"
                    : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == -1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gsrf_peaks

using namespace gsrf_peaks;

extern "C" {

// Operations one launch performs: per thread (scalar kinds; the packed kind counts its
// two multiply-adds) or per warp (the matrix kind, in FLOP: 2 x 16 x 8 x 8 per
// instruction).
double gsrf_peak_ops(int kind, int blocks, int iters) {
    const double per = (double)iters * kUnroll * kChains;
    if (kind == MMA_TF32) return per * blocks * (256 / 32) * 2.0 * 16 * 8 * 8;
    if (kind == FMA32X2) return per * blocks * 256.0 * 2.0;
    return per * blocks * 256.0;
}

// Launch microbenchmark `kind` (0 FP32 FMA, 1 ex2, 2 rcp, 3 rsqrt, 4 sqrt, 5 sin, 6 cos,
// 7 FP64 FMA, 8 TF32 mma.sync, 9 packed FP32x2 FMA) on `blocks` CTAs of 256 threads, `iters` rounds each, on
// `stream`.  out [dev] holds blocks x 256 floats (written only in a case that cannot
// occur).  Returns 0, or the CUDA error of the launch; 1 for an unknown kind or a size
// out of range.
int gsrf_peak_launch(int kind, int blocks, int iters, float* out, void* stream) {
    if (kind < 0 || kind >= N_KINDS || blocks < 1 || blocks > (1 << 20) || iters < 1 || !out) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case FMA32: k_scalar<FMA32><<<blocks, 256, 0, st>>>(iters, out); break;
        case EX2: k_scalar<EX2><<<blocks, 256, 0, st>>>(iters, out); break;
        case RCP: k_scalar<RCP><<<blocks, 256, 0, st>>>(iters, out); break;
        case RSQRT: k_scalar<RSQRT><<<blocks, 256, 0, st>>>(iters, out); break;
        case SQRT: k_scalar<SQRT><<<blocks, 256, 0, st>>>(iters, out); break;
        case SIN: k_scalar<SIN><<<blocks, 256, 0, st>>>(iters, out); break;
        case COS: k_scalar<COS><<<blocks, 256, 0, st>>>(iters, out); break;
        case FMA64: k_fma64<<<blocks, 256, 0, st>>>(iters, out); break;
        case FMA32X2: k_fma32x2<<<blocks, 256, 0, st>>>(iters, out); break;
        default: k_mma_tf32<<<blocks, 256, 0, st>>>(iters, out); break;
    }
    return (int)cudaGetLastError();
}

}  // extern "C"
