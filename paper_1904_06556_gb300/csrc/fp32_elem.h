// FP32 element arithmetic shared by the single-pass fine-level operators (fused.cu, strip.cu): the
// factored element matrix of pbm_internal.h applied with displacement components x and y paired in
// one float2 (the packed FP32 instructions do two operations in one), component z alone, and the CTA
// sum of the per-thread partials in FP64.
#pragma once

#include <cuda_runtime.h>

namespace pbm {

// The element arithmetic keeps displacement components x and y of a coefficient as one float2 and
// runs it with the paired FP32 instructions (one instruction for two operations), component z alone.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Khat of pbm_internal.h with the diagonal of components x, y as pairs
struct KeHat2 {
    float2 dg01[8];
    float dg2[8];
    float lam4[2];
    float mu4[2];
};

// Y = Khat X on (x, y) pairs and z: the diagonal in pairs, the couplings per component
__device__ __forceinline__ void khat_apply2(const KeHat2& K, const float2 (&X01)[8], const float (&X2)[8],
                                            float2 (&Y01)[8], float (&Y2)[8]) {
    auto get = [&](int d, int i) -> float { return d == 0 ? X01[i].x : (d == 1 ? X01[i].y : X2[i]); };
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        Y01[q] = mul2(K.dg01[q], X01[q]);
        Y2[q] = K.dg2[q] * X2[q];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = c == 0 ? Y01[q].x : (c == 1 ? Y01[q].y : Y2[q]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d == c) continue;
                const int r = 3 - c - d;
                const int br = (q >> r) & 1;
                const int qc = (q >> c) & 1, qd = (q >> d) & 1;
                if (qc == 1 && qd == 0) acc = fmaf(K.lam4[br], get(d, (q & ~(1 << c)) | (1 << d)), acc);
                if (qd == 1 && qc == 0) acc = fmaf(K.mu4[br], get(d, (q & ~(1 << d)) | (1 << c)), acc);
            }
            if (c == 0) Y01[q].x = acc;
            else if (c == 1) Y01[q].y = acc;
            else Y2[q] = acc;
        }
    }
    Y01[0] = make_float2(0.0f, 0.0f);
    Y2[0] = 0.0f;
}

template <int NT>
__device__ __forceinline__ double fused_cta_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

}  // namespace pbm
