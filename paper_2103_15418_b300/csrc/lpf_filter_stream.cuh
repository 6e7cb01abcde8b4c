// Building blocks of the streaming box filters (lpf_residual.cuh):
// cancellation-free horizontal window sums ("two stacks"), cp.async copies and
// clipped window counts.
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

constexpr int kStreamTX = 128;      // output columns per strip

// out[c] = sum_{q=0..2R} in(c + q) for c in [c0, c0 + len), len <= RR <= 2R + 1,
// as SUF + PRE around the pivot c0 + 2R: every output is the sum of two sums of
// consecutive inputs, never a difference, so no FP32 cancellation residue.
template <int R, int RR, typename Ld, typename St>
__device__ __forceinline__ void two_stack_run(int c0, int len, Ld&& ld, St&& st) {
    float suf[RR < 2 * R ? RR : 2 * R];
    float acc = 0.f;
#pragma unroll
    for (int i = 2 * R - 1; i >= 0; --i) {
        acc += ld(c0 + i);
        if (i < RR) suf[i] = acc;
    }
    float pre = 0.f;
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        if (i < len) {
            pre += ld(c0 + 2 * R + i);
            float v = pre;
            if (i < 2 * R) v += suf[i];
            st(c0 + i, v);
        }
    }
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}
// 16-byte copy; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

// (n_y, 1/n_y) of an image row's clipped vertical window; n_y = 0 outside the image.
template <int R>
__device__ __forceinline__ float2 row_count(int y, int H) {
    if (y < 0 || y >= H) return make_float2(0.f, 0.f);
    int c = min(y + R, H - 1) - max(y - R, 0) + 1;
    return make_float2((float)c, 1.0f / (float)c);
}

}  // namespace lpf
