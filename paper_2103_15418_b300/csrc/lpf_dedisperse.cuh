// Shift-sum kernels of the dispersed-transient search (sm_103a).
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

// ------------------------------------------------------------------ a3: shift-sum
// D[r][p] = sum_{f=0..F-1} ring[(Tmod - lag[r][f]) mod depth][f][p] for the
// distinct delay rows r, lag[r][f] = max_f delay - delay[r][f] (frames back
// from the newest frame).  A block owns a run of consecutive pixels and walks
// the rows of one segment (blockIdx.y) in order.  Each thread holds 16 bytes of
// every subband's current plane in registers (4 pixels of FP32 storage, 8 of
// 16-bit storage) and reloads a subband only when the row's lag of it differs
// from the previous row's (bit f of chg[r]; every subband at the first row of
// a segment).  The plane index slot * F + f of every (row, subband) of the
// segment is computed once per block into shared memory.  The sum is formed
// afresh for every row in the order f = 0, 1, ..., F-1 in FP32, so its rounding
// is that of a plain F-term sum (packed pair adds round each lane like scalar
// adds).  FULL: F == FMAX at compile time.

// shared-memory bytes of the plane table of a segment of seg_rows rows
__host__ __device__ constexpr size_t dedisperse_smem_bytes(int seg_rows, int F) {
    return (size_t)seg_rows * (F + 1) * sizeof(uint32_t);
}

__device__ __forceinline__ void plane_table(uint32_t* tab, uint32_t* msk, const int16_t* __restrict__ lag,
                                            const uint32_t* __restrict__ chg, int F, int depth, int Tmod,
                                            int r0, int nr) {
    for (int i = threadIdx.x; i < nr * F; i += blockDim.x) {
        const int r = r0 + i / F, f = i - (i / F) * F;
        int slot = Tmod - (int)__ldg(lag + (int64_t)r * F + f);
        if (slot < 0) slot += depth;
        tab[i] = (uint32_t)(slot * F + f);
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) msk[i] = i == 0 ? 0xffffffffu : __ldg(chg + r0 + i);
    __syncthreads();
}

template <int FMAX, bool FULL>
__global__ void __launch_bounds__(256) k_dedisperse(
    const float* __restrict__ ring, float* __restrict__ D, const int16_t* __restrict__ lag,
    const uint32_t* __restrict__ chg, int F, int depth, int Tmod, int n_rows, int seg_rows, int64_t P) {
    extern __shared__ uint32_t dd_tab[];
    if (FULL) F = FMAX;
    const int r0 = blockIdx.y * seg_rows, nr = min(n_rows, r0 + seg_rows) - r0;
    uint32_t* msk = dd_tab + seg_rows * F;
    plane_table(dd_tab, msk, lag, chg, F, depth, Tmod, r0, nr);
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (q >= P) return;
    const char* base = reinterpret_cast<const char*>(ring + q);
    const uint64_t PB = (uint64_t)P * sizeof(float);
    float* dst = D + (int64_t)r0 * P + q;
    float4 cur[FMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f) cur[f] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < nr; ++i) {
        const uint32_t m = msk[i];
        const uint32_t* tr = dd_tab + i * F;
#pragma unroll
        for (int f = 0; f < FMAX; ++f)
            if ((FULL || f < F) && (m & (1u << f)))
                cur[f] = __ldg(reinterpret_cast<const float4*>(base + tr[f] * PB));
        float2 a0 = make_float2(cur[0].x, cur[0].y), a1 = make_float2(cur[0].z, cur[0].w);
#pragma unroll
        for (int f = 1; f < FMAX; ++f)
            if (FULL || f < F) {
                a0 = __fadd2_rn(a0, make_float2(cur[f].x, cur[f].y));
                a1 = __fadd2_rn(a1, make_float2(cur[f].z, cur[f].w));
            }
        // streaming stores: the 0.84 GB of R images should not push ring planes that
        // later rows reload out of L2
        __stcs(reinterpret_cast<float4*>(dst), make_float4(a0.x, a0.y, a1.x, a1.y));
        dst += P;
    }
}

__device__ __forceinline__ float2 to_float2(unsigned u, const __half*) {
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
}
__device__ __forceinline__ float2 to_float2(unsigned u, const __nv_bfloat16*) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}

// x += the two 16-bit values of u (low half into x, high half into y) by the
// mixed-precision add: the 16-bit operand is widened exactly, so each result is
// the FP32 sum rounded once, as a widening followed by an FP32 add
__device__ __forceinline__ void add_pair(unsigned u, float& x, float& y, const __half*) {
    asm("{\n.reg .b16 lo, hi;\nmov.b32 {lo, hi}, %2;\nadd.rn.f32.f16 %0, lo, %0;\nadd.rn.f32.f16 %1, hi, %1;\n}"
        : "+f"(x), "+f"(y) : "r"(u));
}
__device__ __forceinline__ void add_pair(unsigned u, float& x, float& y, const __nv_bfloat16*) {
    asm("{\n.reg .b16 lo, hi;\nmov.b32 {lo, hi}, %2;\nadd.rn.f32.bf16 %0, lo, %0;\nadd.rn.f32.bf16 %1, hi, %1;\n}"
        : "+f"(x), "+f"(y) : "r"(u));
}

// 16-bit storage: 8 pixels per thread, plane values kept packed; the first
// subband is widened and every further one added by mixed-precision adds (same
// order, same FP32 rounding as above).
template <int FMAX, bool FULL, typename TS>
__global__ void __launch_bounds__(256) k_dedisperse16(
    const TS* __restrict__ ring, float* __restrict__ D, const int16_t* __restrict__ lag,
    const uint32_t* __restrict__ chg, int F, int depth, int Tmod, int n_rows, int seg_rows, int64_t P) {
    extern __shared__ uint32_t dd_tab[];
    if (FULL) F = FMAX;
    const int r0 = blockIdx.y * seg_rows, nr = min(n_rows, r0 + seg_rows) - r0;
    uint32_t* msk = dd_tab + seg_rows * F;
    plane_table(dd_tab, msk, lag, chg, F, depth, Tmod, r0, nr);
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (q >= P) return;
    const char* base = reinterpret_cast<const char*>(ring + q);
    const uint64_t PB = (uint64_t)P * sizeof(TS);
    float* dst = D + (int64_t)r0 * P + q;
    uint4 cur[FMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f) cur[f] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = 0; i < nr; ++i) {
        const uint32_t m = msk[i];
        const uint32_t* tr = dd_tab + i * F;
#pragma unroll
        for (int f = 0; f < FMAX; ++f)
            if ((FULL || f < F) && (m & (1u << f)))
                cur[f] = __ldg(reinterpret_cast<const uint4*>(base + tr[f] * PB));
        float2 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = to_float2((&cur[0].x)[k], static_cast<const TS*>(nullptr));
#pragma unroll
        for (int f = 1; f < FMAX; ++f)
            if (FULL || f < F) {
#pragma unroll
                for (int k = 0; k < 4; ++k) add_pair((&cur[f].x)[k], a[k].x, a[k].y, static_cast<const TS*>(nullptr));
            }
        float4* o = reinterpret_cast<float4*>(dst);
        __stcs(o, make_float4(a[0].x, a[0].y, a[1].x, a[1].y));          // streaming, as above
        __stcs(o + 1, make_float4(a[2].x, a[2].y, a[3].x, a[3].y));
        dst += P;
    }
}

}  // namespace lpf
