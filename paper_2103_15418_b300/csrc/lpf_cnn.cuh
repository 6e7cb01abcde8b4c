// Parameter-inference network on the dynamic-spectrum batch (Sec. 2.3):
// convolutions with Leaky ReLU hidden states, a final linear layer, and a head
// giving the mean mu and the Cholesky factor L (positive diagonal) of a Gaussian
// over the parameters theta.  The paper gives the form, not the layers; the
// network here (fixed weights supplied by the caller) is
//   conv1 3x3 1 -> 16, Leaky ReLU, 2x2 mean    (CUDA cores, FP32)   -> BF16
//   conv2 3x3 16 -> 32, Leaky ReLU, 2x2 mean   (tensor cores)       -> BF16
//   conv3 3x3 32 -> 64, Leaky ReLU, mean over the pixels (tensor cores) -> FP32
//   head 64 -> 5: mu = (z0, z1), L = [[exp z2, 0], [z3, exp z4]]
// with zero padding 1 and alpha = 0.01.  Activations between layers are
// stored channel-last ([n][y][x][c]) in BF16, the tensor cores' operand type;
// every sum is FP32.
//
// conv2 and conv3 are implicit GEMMs on the tcgen05 tensor cores (lpf_tc.cuh):
// one CTA of 128 threads takes 128 output pixels (rows of A), gathers their 3x3
// neighbourhoods (K = 9 Cin, column k = tap Cin + c) from the BF16 input into
// shared memory, stages the weights [Cout][K] beside them, and one thread issues
// K / 16 MMAs of 128 x Cout x 16 into tensor memory (FP32).  Thread t then reads
// row t back (tcgen05.ld), adds the bias, applies the Leaky ReLU and pools:
//   conv2: rows are ordered (2x2 window, position in it), so the four pixels
//          of a window are four consecutive lanes of one warp (shuffles);
//   conv3: rows are ordered (spectrum, pixel) and a spectrum's pixels are a
//          whole number of rows per tile; their mean goes through shared
//          memory, and the head follows in the same CTA.
#pragma once
#include "lpf_tc.cuh"

#include <cuda_bf16.h>
#include <stdint.h>

namespace lpf {
namespace cnn {

constexpr float kAlpha = 0.01f;
constexpr int kC1 = 16, kC2 = 32, kC3 = 64, kOut = 5;
constexpr int kRows = 128;                 // output pixels per CTA of a tensor-core layer
constexpr uint64_t kWaitNs = 200000000ull; // MMA completion wait limit (0.2 s)

__device__ __forceinline__ float leaky(float h) { return h >= 0.f ? h : kAlpha * h; }

// ---------------------------------------------------------------------------
// conv1 (one input channel): one thread per 2x2 output window of one spectrum;
// the 4x4 input patch around it (zero outside), 16 channels x 4 pixels x 9 taps,
// bias, Leaky ReLU, mean of the window, BF16 out [n][H/2][W/2][16].
__global__ void __launch_bounds__(256) k_cnn_conv1(const float* __restrict__ x, int n, int H, int W,
                                                   const float* __restrict__ w, const float* __restrict__ b,
                                                   __nv_bfloat16* __restrict__ out) {
    __shared__ float sw[kC1 * 9], sb[kC1];
    for (int i = threadIdx.x; i < kC1 * 9; i += blockDim.x) sw[i] = w[i];
    for (int i = threadIdx.x; i < kC1; i += blockDim.x) sb[i] = b[i];
    __syncthreads();
    const int Hp = H / 2, Wp = W / 2;
    const int64_t total = (int64_t)n * Hp * Wp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / (Hp * Wp));
        const int rem = (int)(i - (int64_t)s * Hp * Wp);
        const int py = rem / Wp, px = rem - py * Wp;
        const float* xs = x + (int64_t)s * H * W;
        float p[4][4];
#pragma unroll
        for (int dy = 0; dy < 4; ++dy)
#pragma unroll
            for (int dx = 0; dx < 4; ++dx) {
                const int yy = 2 * py - 1 + dy, xx = 2 * px - 1 + dx;
                p[dy][dx] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(xs + yy * W + xx) : 0.f;
            }
        uint32_t packed[kC1 / 2];
#pragma unroll
        for (int c = 0; c < kC1; ++c) {
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int oy = q >> 1, ox = q & 1;
                float acc = sb[c];
#pragma unroll
                for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) acc = fmaf(sw[c * 9 + ky * 3 + kx], p[oy + ky][ox + kx], acc);
                v[q] = leaky(acc);
            }
            const float m = ((v[0] + v[1]) + (v[2] + v[3])) * 0.25f;
            const __nv_bfloat16 h = __float2bfloat16_rn(m);
            const uint16_t u = *reinterpret_cast<const uint16_t*>(&h);
            if (c & 1) packed[c >> 1] |= (uint32_t)u << 16;
            else packed[c >> 1] = u;
        }
        uint4* o = reinterpret_cast<uint4*>(out + i * kC1);
        o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    }
}

// ---------------------------------------------------------------------------
// conv2 / conv3 on the tensor cores.  in: BF16 [n][H][W][CIN]; wk: BF16
// [COUT][9 CIN] (k = (ky 3 + kx) CIN + c); bias FP32 [COUT].
//   GPOOL false: out BF16 [n][H/2][W/2][COUT], 2x2 means;
//   GPOOL true:  the mean over the H W pixels of each spectrum, then the head
//                (hw [5][COUT], hb [5]) -> res FP32 [n][5]; H W divides 128.
// err: bit 0 set when an MMA completion wait ran out (the CTA then writes
// nothing and releases its tensor memory).
template <int CIN, int COUT, bool GPOOL>
__global__ void __launch_bounds__(kRows) k_cnn_conv_tc(const __nv_bfloat16* __restrict__ in, int n, int H, int W,
                                                       const __nv_bfloat16* __restrict__ wk,
                                                       const float* __restrict__ bias,
                                                       __nv_bfloat16* __restrict__ out,
                                                       const float* __restrict__ hw, const float* __restrict__ hb,
                                                       float* __restrict__ res, unsigned* __restrict__ err) {
    constexpr int K = 9 * CIN, KC = K / 8;
    constexpr uint32_t NCOLS = COUT < 32 ? 32 : COUT;
    static_assert(CIN % 8 == 0 && K % 16 == 0 && COUT % 32 == 0 && COUT >= 32 && COUT <= 256, "shapes");
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sA = smem;                         // 128 x K, K-major core matrices
    uint8_t* sB = smem + kRows * K * 2;         // COUT x K
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int P = H * W;                        // pixels per spectrum at this layer
    const int64_t M = (int64_t)n * P;           // output pixels (rows)
    const int64_t m = (int64_t)blockIdx.x * kRows + t;
    if (warp == 0) tc::tmem_alloc(&tslot, NCOLS);
    if (t == 0) tc::mbar_init(&mbar, 1);
    // weights
    for (int i = t; i < COUT * KC; i += kRows) {
        const int r = i / KC, j = i - r * KC;
        *reinterpret_cast<uint4*>(sB + tc::kmajor_offset(r, 8 * j, KC)) =
            __ldg(reinterpret_cast<const uint4*>(wk + (int64_t)r * K + 8 * j));
    }
    // this thread's row: its output pixel and 3x3 neighbourhood
    const bool live = m < M;
    int s = 0, y = 0, x = 0;
    if (live) {
        if (GPOOL) {
            s = (int)(m / P);
            const int pix = (int)(m - (int64_t)s * P);
            y = pix / W;
            x = pix - y * W;
        } else {
            // rows ordered (2x2 window, position in the window)
            const int Wp = W / 2, Pp = (H / 2) * Wp;
            const int64_t win = m >> 2;
            const int q = (int)(m & 3);
            s = (int)(win / Pp);
            const int rem = (int)(win - (int64_t)s * Pp);
            const int py = rem / Wp, px = rem - py * Wp;
            y = 2 * py + (q >> 1);
            x = 2 * px + (q & 1);
        }
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        const bool ok = live && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const __nv_bfloat16* src = in + (((int64_t)s * H + (ok ? yy : 0)) * W + (ok ? xx : 0)) * CIN;
#pragma unroll
        for (int c8 = 0; c8 < CIN / 8; ++c8) {
            const uint4 v = ok ? __ldg(reinterpret_cast<const uint4*>(src + 8 * c8)) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(t, tap * CIN + 8 * c8, KC)) = v;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    if (t == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, COUT);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll 1
        for (int ks = 0; ks < K / 16; ++ks)
            tc::mma_bf16(taddr, tc::smem_desc(a0 + 256 * ks, 128, KC * 128), tc::smem_desc(b0 + 256 * ks, 128, KC * 128),
                         idesc, ks > 0 ? 1u : 0u);
        tc::mma_commit(&mbar);
    }
    const bool done = tc::mbar_wait(&mbar, 0, kWaitNs);
    tc::fence_after_sync();
    if (!done && t == 0) atomicOr(err, 1u);
    const bool all_done = __syncthreads_and(done);
    if (all_done) {
        if constexpr (!GPOOL) {
            // bias, Leaky ReLU, mean of the 2x2 window over lanes 4p .. 4p + 3
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 32) {
                float v[32];
                tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + c0, v);
                uint32_t packed[16];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    float h = leaky(v[c] + __ldg(bias + c0 + c));
                    h += __shfl_xor_sync(0xffffffffu, h, 1);
                    h += __shfl_xor_sync(0xffffffffu, h, 2);
                    const __nv_bfloat16 bh = __float2bfloat16_rn(h * 0.25f);
                    const uint16_t u = *reinterpret_cast<const uint16_t*>(&bh);
                    if (c & 1) packed[c >> 1] |= (uint32_t)u << 16;
                    else packed[c >> 1] = u;
                }
                if (live && (lane & 3) == 0) {
                    uint4* o = reinterpret_cast<uint4*>(out + (m >> 2) * COUT + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        o[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                }
            }
        } else {
            // rows -> shared memory (A is free now), then per spectrum and channel
            // the mean over its pixels, then the head
            float* red = reinterpret_cast<float*>(sA);            // [128][COUT + 1]
#pragma unroll
            for (int c0 = 0; c0 < COUT; c0 += 32) {
                float v[32];
                tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
                for (int c = 0; c < 32; ++c) red[t * (COUT + 1) + c0 + c] = leaky(v[c] + __ldg(bias + c0 + c));
            }
            __syncthreads();
            const int spt = kRows / P;                            // spectra per tile
            float* feat = red + kRows * (COUT + 1);               // [spt][COUT], spt <= 128
            static_assert(kRows * (COUT + 1) * 4 + kRows * COUT * 4 <= kRows * K * 2, "features fit in the A tile");
            for (int i = t; i < spt * COUT; i += kRows) {
                const int sp = i / COUT, c = i - sp * COUT;
                float acc = 0.f;
                for (int r = 0; r < P; ++r) acc += red[(sp * P + r) * (COUT + 1) + c];
                feat[sp * COUT + c] = acc / (float)P;
            }
            __syncthreads();
            const int64_t s0 = (int64_t)blockIdx.x * spt;
            for (int i = t; i < spt * kOut; i += kRows) {
                const int sp = i / kOut, o = i - sp * kOut;
                if (s0 + sp >= n) continue;
                float z = __ldg(hb + o);
                for (int c = 0; c < COUT; ++c) z = fmaf(__ldg(hw + o * COUT + c), feat[sp * COUT + c], z);
                res[(s0 + sp) * kOut + o] = (o == 2 || o == 4) ? expf(z) : z;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, NCOLS);
}

// A and B tiles (the conv3 epilogue reuses A for its rows and features)
template <int CIN, int COUT>
constexpr size_t conv_tc_smem_bytes() {
    return (size_t)kRows * 9 * CIN * 2 + (size_t)COUT * 9 * CIN * 2;
}

}  // namespace cnn
}  // namespace lpf
