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
// For 32 x 64 spectra the whole network runs instead as one persistent kernel
// with the activations in shared memory (k_cnn_fused_32x64, at the end).
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


// ---------------------------------------------------------------------------
// The whole network for 32 x 64 spectra in one persistent kernel: a CTA of 128
// threads takes one spectrum at a time and keeps every activation in shared
// memory, so a spectrum costs one 8 KB read and a 20-byte write of HBM.  The
// next spectrum's input is copied in (cp.async) while the tensor cores work on
// the current one.
//   conv1 (CUDA cores, FP32): thread t computes the 2x2-pooled pixels
//         (4 j + t / 32, t % 32), j = 0..3; the two horizontally adjacent
//         outputs of a window share every weight, so they are one packed FP32x2
//         FMA chain (each lane rounds like the scalar chain of k_cnn_conv1).
//   conv2 (tcgen05): act1 is stored with a zero border as [c / 8][18][34][c % 8]
//         (16 x 32 pixels + 1 on each side), so the 8 pixels of one image row
//         and 8 channels are one core matrix.  An output tile of 16 rows x 8
//         columns (M = 128, row m = 8 y + i) then needs no gathered copy: for
//         tap (ky, kx) the A operand is the same storage seen from pixel
//         (ky, 8 q + kx), with 34 pixels between 8-row groups (stride offset)
//         and the next 8 channels one plane further (leading offset).  Nine
//         MMAs of 128 x 32 x 16 per tile, four tiles per spectrum.
//   conv2 epilogue: bias, Leaky ReLU, 2x2 mean over lanes m ^ 1 and m ^ 8, BF16
//         into act2 stored likewise as [c / 8][18][18][c % 8] (8 x 16 pixels,
//         a zero border, and 8 more zero rows).
//   conv3 (tcgen05): an 8 x 16 spectrum is two column halves of 8; each half is
//         an M = 128 MMA whose first 64 rows are its 8 x 8 pixels and whose
//         other 64 rows read the zero rows below and are not used (twice the
//         MMA work of conv3 in exchange for no gather).  2 x 9 taps x 2 K-steps
//         of 128 x 64 x 16.
//   conv3 epilogue: warps 0 and 1 hold the 64 + 64 pixels: bias, Leaky ReLU, the
//         two halves added per thread, the 64 rows summed per channel through
//         shared memory (over act1, whose border is zeroed again afterwards),
//         the mean, then the head (threads 0..4).
// Tensor memory: 256 columns per CTA (conv2: 4 x 32, conv3: 2 x 64); two CTAs
// per SM use all 512.
namespace fused {
constexpr int H0 = 32, W0 = 64, H1 = 16, W1 = 32, H2 = 8, W2 = 16;
constexpr int Y1 = H1 + 2, X1 = W1 + 2;          // act1 with its border
constexpr int Y2 = 18, X2 = W2 + 2;              // act2: border + 8 zero rows
constexpr int K2 = 9 * kC1, K3 = 9 * kC2;        // 144, 288
constexpr uint32_t OFF_W2 = 0;
constexpr uint32_t OFF_W3 = OFF_W2 + kC2 * K2 * 2;             // 9216
constexpr uint32_t OFF_A1 = OFF_W3 + kC3 * K3 * 2;             // + 36864
constexpr uint32_t OFF_A2 = OFF_A1 + 2 * Y1 * X1 * 16;         // + 19584
constexpr uint32_t OFF_X = OFF_A2 + 4 * Y2 * X2 * 16;          // + 20736
constexpr uint32_t SMEM = OFF_X + H0 * W0 * 4;                 // + 8192
constexpr int RP = kC3 + 1;                                    // row pitch of the channel sums (in act1)
constexpr uint32_t TCOLS = 256;
static_assert(OFF_A1 % 128 == 0 && OFF_A2 % 128 == 0 && OFF_X % 16 == 0, "alignment");
static_assert(64 * RP * 4 <= 2 * Y1 * X1 * 16, "channel sums fit in act1");
}  // namespace fused

// the input spectrum s (8 KB) into shared memory, 16 bytes per copy
__device__ __forceinline__ void cnn_fetch_spectrum(uint8_t* dst, const float* x, int s) {
    const char* src = reinterpret_cast<const char*>(x + (int64_t)s * fused::H0 * fused::W0);
    for (int i = threadIdx.x; i < fused::H0 * fused::W0 / 4; i += kRows) {
        const uint32_t d = tc::smem_u32(dst + 16 * i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 16 * i));
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

__global__ void __launch_bounds__(kRows, 2) k_cnn_fused_32x64(
    const float* __restrict__ x, int n, const float* __restrict__ w1, const float* __restrict__ b1,
    const __nv_bfloat16* __restrict__ wk2, const float* __restrict__ b2, const __nv_bfloat16* __restrict__ wk3,
    const float* __restrict__ b3, const float* __restrict__ hw, const float* __restrict__ hb,
    float* __restrict__ res, unsigned* __restrict__ err) {
    using namespace fused;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ float2 sw1[kC1 * 9];                  // conv1 weights, each twice (packed FMA operand)
    __shared__ float sb1[kC1], sb2[kC2], sb3[kC3], shw[kOut * kC3], shb[kOut], sfeat[kC3];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if ((int)blockIdx.x < n) cnn_fetch_spectrum(smem + OFF_X, x, blockIdx.x);
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (t == 0) tc::mbar_init(&mbar, 1);
    for (int i = t; i < kC1 * 9; i += kRows) sw1[i] = make_float2(w1[i], w1[i]);
    for (int i = t; i < kOut * kC3; i += kRows) shw[i] = hw[i];
    if (t < kC1) sb1[t] = b1[t];
    if (t < kC2) sb2[t] = b2[t];
    if (t < kC3) sb3[t] = b3[t];
    if (t < kOut) shb[t] = hb[t];
    // weights in the K-major core-matrix layout
    for (int i = t; i < kC2 * (K2 / 8); i += kRows) {
        const int r = i / (K2 / 8), j = i - r * (K2 / 8);
        *reinterpret_cast<uint4*>(smem + OFF_W2 + tc::kmajor_offset(r, 8 * j, K2 / 8)) =
            __ldg(reinterpret_cast<const uint4*>(wk2 + r * K2 + 8 * j));
    }
    for (int i = t; i < kC3 * (K3 / 8); i += kRows) {
        const int r = i / (K3 / 8), j = i - r * (K3 / 8);
        *reinterpret_cast<uint4*>(smem + OFF_W3 + tc::kmajor_offset(r, 8 * j, K3 / 8)) =
            __ldg(reinterpret_cast<const uint4*>(wk3 + r * K3 + 8 * j));
    }
    // act1 and act2 start zero: borders and spare rows stay zero
    for (uint32_t o = OFF_A1 + 16 * t; o < OFF_X; o += 16 * kRows)
        *reinterpret_cast<uint4*>(smem + o) = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t sbase = tc::smem_u32(smem);
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const float* sx = reinterpret_cast<const float*>(smem + OFF_X);
    float* rows = reinterpret_cast<float*>(smem + OFF_A1);
    bool ok = true;
    for (int s = blockIdx.x; s < n && ok; s += gridDim.x) {
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();
        // ---- conv1 -> act1 (interior), from the spectrum in shared memory
#pragma unroll 1
        for (int jj = 0; jj < 4; ++jj) {
            const int py = 4 * jj + warp, px = lane;
            // P[r][k] = (p[r][k], p[r][k + 1]): the inputs of the left and right output
            float2 P[4][3];
#pragma unroll
            for (int dy = 0; dy < 4; ++dy) {
                const int yy = 2 * py - 1 + dy;
                float p[4];
#pragma unroll
                for (int dx = 0; dx < 4; ++dx) {
                    const int xx = 2 * px - 1 + dx;
                    p[dx] = (yy >= 0 && yy < H0 && xx >= 0 && xx < W0) ? sx[yy * W0 + xx] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) P[dy][k] = make_float2(p[k], p[k + 1]);
            }
            uint32_t packed[kC1 / 2];
#pragma unroll
            for (int c = 0; c < kC1; ++c) {
                float2 a[2];
#pragma unroll
                for (int oy = 0; oy < 2; ++oy) {
                    a[oy] = make_float2(sb1[c], sb1[c]);
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) a[oy] = __ffma2_rn(sw1[c * 9 + ky * 3 + kx], P[oy + ky][kx], a[oy]);
                }
                const float m = ((leaky(a[0].x) + leaky(a[0].y)) + (leaky(a[1].x) + leaky(a[1].y))) * 0.25f;
                const __nv_bfloat16 h = __float2bfloat16_rn(m);
                const uint16_t u = *reinterpret_cast<const uint16_t*>(&h);
                if (c & 1) packed[c >> 1] |= (uint32_t)u << 16;
                else packed[c >> 1] = u;
            }
#pragma unroll
            for (int cg = 0; cg < 2; ++cg)
                *reinterpret_cast<uint4*>(smem + OFF_A1 + ((cg * Y1 + py + 1) * X1 + px + 1) * 16) =
                    make_uint4(packed[4 * cg], packed[4 * cg + 1], packed[4 * cg + 2], packed[4 * cg + 3]);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // the next spectrum's input, behind the tensor-core work on this one
        if (s + (int)gridDim.x < n) cnn_fetch_spectrum(smem + OFF_X, x, s + gridDim.x);
        // ---- conv2: 4 tiles x 9 taps, A read in place from act1
        if (t == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, kC2);
#pragma unroll 1
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const uint64_t ad = tc::smem_desc(sbase + OFF_A1 + (ky * X1 + 8 * q + kx) * 16, Y1 * X1 * 16, X1 * 16);
                    const uint64_t bd = tc::smem_desc(sbase + OFF_W2 + 256 * tap, 128, (K2 / 8) * 128);
                    tc::mma_bf16(taddr + 32 * q, ad, bd, idesc, tap > 0 ? 1u : 0u);
                }
            tc::mma_commit(&mbar);
        }
        bool done = tc::mbar_wait(&mbar, 0, kWaitNs);
        tc::fence_after_sync();
        if (!__syncthreads_and(done)) {
            if (t == 0) atomicOr(err, 1u);
            tc::mbar_wait(&mbar, 0, kWaitNs);     // the MMAs still in flight, bounded
            ok = false;
            break;
        }
        // ---- conv2 epilogue: row m = 32 warp + lane = 8 y + i of tile q
        {
            const int m = 32 * warp + lane, y = m >> 3, i = m & 7;
            const bool keep = ((y | i) & 1) == 0;
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                float v[32];
                tc::tmem_ld32(taddr + lane_off + 32 * q, v);
                uint32_t packed[16];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    float h = leaky(v[c] + sb2[c]);
                    h += __shfl_xor_sync(0xffffffffu, h, 1);
                    h += __shfl_xor_sync(0xffffffffu, h, 8);
                    const __nv_bfloat16 bh = __float2bfloat16_rn(h * 0.25f);
                    const uint16_t u = *reinterpret_cast<const uint16_t*>(&bh);
                    if (c & 1) packed[c >> 1] |= (uint32_t)u << 16;
                    else packed[c >> 1] = u;
                }
                if (keep) {
                    const int pr = y >> 1, pc = 4 * q + (i >> 1);
#pragma unroll
                    for (int cg = 0; cg < 4; ++cg)
                        *reinterpret_cast<uint4*>(smem + OFF_A2 + ((cg * Y2 + pr + 1) * X2 + pc + 1) * 16) =
                            make_uint4(packed[4 * cg], packed[4 * cg + 1], packed[4 * cg + 2], packed[4 * cg + 3]);
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // ---- conv3: two column halves x 9 taps x 2 K-steps
        if (t == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, kC3);
#pragma unroll 1
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ad = tc::smem_desc(
                            sbase + OFF_A2 + ((2 * ks * Y2 + ky) * X2 + 8 * h + kx) * 16, Y2 * X2 * 16, X2 * 16);
                        const uint64_t bd =
                            tc::smem_desc(sbase + OFF_W3 + (4 * tap + 2 * ks) * 128, 128, (K3 / 8) * 128);
                        tc::mma_bf16(taddr + 128 + 64 * h, ad, bd, idesc, (tap | ks) ? 1u : 0u);
                    }
                }
            tc::mma_commit(&mbar);
        }
        done = tc::mbar_wait(&mbar, 1, kWaitNs);
        tc::fence_after_sync();
        if (!__syncthreads_and(done)) {
            if (t == 0) atomicOr(err, 1u);
            tc::mbar_wait(&mbar, 1, kWaitNs);     // the MMAs still in flight, bounded
            ok = false;
            break;
        }
        // ---- conv3 epilogue: warps 0 and 1 (rows 0..63 = pixel (m / 8, 8 h + m % 8));
        // act1 is free (the conv2 MMAs have completed) and takes the channel sums
        if (warp < 2) {
            const int m = 32 * warp + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < kC3; c0 += 32) {
                float vl[32], vr[32];
                tc::tmem_ld32(taddr + lane_off + 128 + c0, vl);
                tc::tmem_ld32(taddr + lane_off + 192 + c0, vr);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float bc = sb3[c0 + c];
                    rows[m * RP + c0 + c] = leaky(vl[c] + bc) + leaky(vr[c] + bc);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (t < kC3) {
            float acc = 0.f;
            for (int m = 0; m < 64; ++m) acc += rows[m * RP + t];
            sfeat[t] = acc * (1.0f / (H2 * W2));
        }
        __syncthreads();
        if (t < kOut) {
            float z = shb[t];
            for (int c = 0; c < kC3; ++c) z = fmaf(shw[t * kC3 + c], sfeat[c], z);
            res[(int64_t)s * kOut + t] = (t == 2 || t == 4) ? expf(z) : z;
        }
        // act1 again: zero its border (the next conv1 writes the interior)
        for (int i = t; i < 2 * Y1 * X1; i += kRows) {
            const int cg = i / (Y1 * X1), r = i - cg * (Y1 * X1), yy = r / X1, xx = r - yy * X1;
            if (yy == 0 || yy == Y1 - 1 || xx == 0 || xx == X1 - 1)
                *reinterpret_cast<uint4*>(smem + OFF_A1 + i * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, TCOLS);
}

}  // namespace cnn
}  // namespace lpf
