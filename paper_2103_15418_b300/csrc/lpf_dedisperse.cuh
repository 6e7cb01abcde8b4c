// Shift-sum kernels of the dispersed-transient search (sm_103a).
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

// ------------------------------------------------------------------ a3: shift-sum
// D[r][p] = sum_{f=0..F-1} ring[(Tmod - lag[r][f]) mod depth][f][p] for the
// distinct delay rows r, lag[r][f] = max_f delay - delay[r][f] (frames back
// from the newest frame).  Each thread owns consecutive pixels (4 for FP32
// storage, 8 for 16-bit storage, so every load is 16 bytes) and walks the rows
// of one segment (blockIdx.y) in order: the current plane value of each subband
// stays in registers and is reloaded only when the row's lag of that subband
// differs from the previous row's (bit f of chg[r]; every subband at the first
// row of a segment).  The sum itself is formed afresh for every row in the
// order f = 0, 1, ..., F-1 (FP32), so its rounding is that of a plain F-term sum.
template <int FMAX>
__global__ void __launch_bounds__(256) k_dedisperse(
    const float* __restrict__ ring, float* __restrict__ D, const int16_t* __restrict__ lag,
    const uint32_t* __restrict__ chg, int F, int depth, int Tmod, int n_rows, int seg_rows, int64_t P) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (q >= P) return;
    const int r0 = blockIdx.y * seg_rows, r1 = min(n_rows, r0 + seg_rows);
    float4 cur[FMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f) cur[f] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = r0; r < r1; ++r) {
        const uint32_t m = (r == r0) ? 0xffffffffu : __ldg(chg + r);
        const int16_t* lr = lag + (int64_t)r * F;
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
            if (f < F && ((m >> f) & 1u)) {
                int slot = Tmod - (int)__ldg(lr + f);
                if (slot < 0) slot += depth;
                cur[f] = ld4(ring + ((int64_t)slot * F + f) * P + q);
            }
        }
        float4 acc = cur[0];
#pragma unroll
        for (int f = 1; f < FMAX; ++f) {
            if (f < F) { acc.x += cur[f].x; acc.y += cur[f].y; acc.z += cur[f].z; acc.w += cur[f].w; }
        }
        st4(D + (int64_t)r * P + q, acc);
    }
}

__device__ __forceinline__ float2 to_float2(unsigned u, const __half*) {
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}
__device__ __forceinline__ float2 to_float2(unsigned u, const __nv_bfloat16*) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}

// 16-bit storage: 8 pixels per thread, plane values kept packed and widened to
// FP32 when summed (same order, same FP32 arithmetic as above).
template <int FMAX, typename TS>
__global__ void __launch_bounds__(256) k_dedisperse16(
    const TS* __restrict__ ring, float* __restrict__ D, const int16_t* __restrict__ lag,
    const uint32_t* __restrict__ chg, int F, int depth, int Tmod, int n_rows, int seg_rows, int64_t P) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (q >= P) return;
    const int r0 = blockIdx.y * seg_rows, r1 = min(n_rows, r0 + seg_rows);
    uint4 cur[FMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f) cur[f] = make_uint4(0u, 0u, 0u, 0u);
    for (int r = r0; r < r1; ++r) {
        const uint32_t m = (r == r0) ? 0xffffffffu : __ldg(chg + r);
        const int16_t* lr = lag + (int64_t)r * F;
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
            if (f < F && ((m >> f) & 1u)) {
                int slot = Tmod - (int)__ldg(lr + f);
                if (slot < 0) slot += depth;
                cur[f] = __ldg(reinterpret_cast<const uint4*>(ring + ((int64_t)slot * F + f) * P + q));
            }
        }
        float a[8];
        {
            const unsigned* u = reinterpret_cast<const unsigned*>(&cur[0]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 v = to_float2(u[k], static_cast<const TS*>(nullptr));
                a[2 * k] = v.x;
                a[2 * k + 1] = v.y;
            }
        }
#pragma unroll
        for (int f = 1; f < FMAX; ++f) {
            if (f < F) {
                const unsigned* u = reinterpret_cast<const unsigned*>(&cur[f]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 v = to_float2(u[k], static_cast<const TS*>(nullptr));
                    a[2 * k] += v.x;
                    a[2 * k + 1] += v.y;
                }
            }
        }
        float4* o = reinterpret_cast<float4*>(D + (int64_t)r * P + q);
        o[0] = make_float4(a[0], a[1], a[2], a[3]);
        o[1] = make_float4(a[4], a[5], a[6], a[7]);
    }
}

}  // namespace lpf
