// Streaming box filter + detection for a compile-time box radius R <= 15.
//
// One CTA owns a strip of TX = 128 output columns of one dedispersed image and
// walks down it in blocks of 32 rows, so rows are never recomputed (only the
// 2R-column halo of the strip is).  Per block:
//   1. D rows of the next block (strip + 2R halo each side) are prefetched with
//      cp.async into the other half of a double buffer while this block runs
//   2. horizontal window sums of D ("two stacks", cancellation free)   -> hX
//   3. per column: vertical sliding sum of hX -> C = sum / n, residual D - C
//      stored in a shared ring of 64 rows
//   4. horizontal window sums of E = (D - C)^2                          -> hX
//   5. per column: vertical compensated (Neumaier) sliding sum of hX -> S,
//      snr = (D - C)/sqrt(S), threshold, 3x3 local maximum, stats, emission
// The vertical pass of C runs R rows behind the input and that of S 2R rows
// behind; the column thread that computes C for a column is the one that later
// computes S for it, and the residual ring carries D - C across that lag.  The
// lagged reads of D itself (D at row yc for the residual, the 3x3 neighbours of
// a candidate) go to global memory, where those rows are still L2-resident.
// Out-of-image rows and columns contribute zeros, and C and S divide by the
// in-image window count, which clips every window to the image (Sec. 2.1.1).
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

constexpr int kStreamTX = 128;
constexpr int kStreamThreads = 192;

template <int R>
struct StreamGeom {
    static constexpr int TX = kStreamTX;
    static constexpr int WC = TX + 2 * R;        // columns carrying C and the residual
    static constexpr int WD = TX + 4 * R;        // columns carrying D
    static constexpr int SD = WD | 1;            // odd strides: conflict-free column walks
    static constexpr int SX = WC | 1;
    static constexpr int L = 2 * R + 1;
    static constexpr int NR1 = (WC + L - 1) / L;         // runs per row, horizontal pass 1
    static constexpr int RR1 = (WC + NR1 - 1) / NR1;
    static constexpr int NR2 = (TX + L - 1) / L;         // runs per row, horizontal pass 2
    static constexpr int RR2 = (TX + NR2 - 1) / NR2;
    static constexpr size_t smem_floats = (size_t)64 * SD + (size_t)32 * SX + (size_t)64 * SX;
    static constexpr int NLOAD = (32 * WD + kStreamThreads - 1) / kStreamThreads;
};

// out[c] = sum_{q=0..2R} in(c + q) for c in [c0, c0 + len), len <= RR <= 2R + 1,
// as SUF + PRE around the pivot c0 + 2R (sums of consecutive inputs only).
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

// Neumaier-compensated accumulation s + c += x.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    float t = s + x;
    float e = (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    c += e;
    s = t;
}

template <int R>
__device__ __forceinline__ float inv_count(int y, int n) {
    int c = min(y + R, n - 1) - max(y - R, 0) + 1;
    return c == 2 * R + 1 ? 1.0f / (float)(2 * R + 1) : 1.0f / (float)c;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Issue the copies of D rows [ybase, ybase + 32) x cols [x0 - 2R, x0 + TX + 2R) into dst
// (zero-filled outside the image).
template <int R>
__device__ __forceinline__ void load_block_async(float* dst, const float* Dimg, int ybase, int x0,
                                                 int H, int W, int t) {
    using G = StreamGeom<R>;
#pragma unroll 4
    for (int q = 0; q < G::NLOAD; ++q) {
        int idx = t + q * kStreamThreads;
        if (idx < 32 * G::WD) {
            int j = idx / G::WD, c = idx - j * G::WD;
            int y = ybase + j, x = x0 - 2 * R + c;
            bool in = y < H && x >= 0 && x < W;
            cp_async4(dst + j * G::SD + c, in ? Dimg + (int64_t)y * W + x : Dimg, in);
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kStreamThreads, 2) k_filter_stream(FilterArgs a) {
    using G = StreamGeom<R>;
    constexpr int TX = G::TX, WC = G::WC, WD = G::WD, SD = G::SD, SX = G::SX;
    constexpr int NT = kStreamThreads;
    extern __shared__ float sm[];
    float* Dring = sm;                  // [2][32][SD] D rows of a block, double buffer; col = x - (x0 - 2R)
    float* hX = Dring + 64 * SD;        // [32][SX]  horizontal sums of the block
    float* Rring = hX + 32 * SX;        // [64][SX]  residual D - C; col = x - (x0 - R)

    const int strip = blockIdx.x, row = blockIdx.y;
    const int x0 = strip * TX;
    const int H = a.H, W = a.W;
    const float* Dimg = a.D + (int64_t)row * a.P;
    const int t = threadIdx.x;
    const int lane = t & 31;

    const int xc = x0 - R + t;                       // this thread's column
    const bool col_c = t < WC;
    const bool xc_in = col_c && xc >= 0 && xc < W;
    const bool col_s = t >= R && t < R + TX && xc < W;
    const float inv_nx = xc_in ? inv_count<R>(xc, W) : 0.f;
    const int nxc = xc_in ? min(xc + R, W - 1) - max(xc - R, 0) + 1 : 1;

    float histD[32], histE[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { histD[j] = 0.f; histE[j] = 0.f; }
    float vD = 0.f, vEs = 0.f, vEc = 0.f;
    double d1 = 0.0, d2 = 0.0, dc = 0.0;
    const int m0 = a.member_start[row], nm = a.member_start[row + 1] - m0;

    const int nblk = (H + 2 * R + 31) / 32;
    load_block_async<R>(Dring, Dimg, 0, x0, H, W, t);
    cp_async_commit();
    for (int k = 0; k < nblk; ++k) {
        const int ybase = k * 32;
        // ---- 1. prefetch block k + 1 into the other half, wait for block k
        if (k + 1 < nblk)
            load_block_async<R>(Dring + ((k + 1) & 1) * 32 * SD, Dimg, ybase + 32, x0, H, W, t);
        cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
        // ---- 2. hX[j][c] = sum of D over columns c .. c + 2R (ring cols) of row ybase + j
        for (int it = t; it < 32 * G::NR1; it += NT) {
            int j = it & 31, run = it >> 5;
            int c0 = run * G::RR1;
            int len = min(G::RR1, WC - c0);
            const float* in = Dring + ((k & 1) * 32 + j) * SD;
            float* out = hX + j * SX;
            two_stack_run<R, G::RR1>(c0, len, [&](int c) { return in[c]; },
                                     [&](int c, float v) { out[c] = v; });
        }
        __syncthreads();
        // ---- 3. vertical sliding sum -> C for row yc = ybase + j - R, residual D - C
        if (col_c) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float in = hX[j * SX + t];
                float out = histD[(j + 31 - 2 * R) & 31];
                histD[j] = in;
                vD += in - out;
                const int yc = ybase + j - R;
                float res = 0.f;
                if (xc_in && yc >= 0 && yc < H) {
                    // correctly rounded division: C is exact when the window is constant
                    int ny = min(yc + R, H - 1) - max(yc - R, 0) + 1;
                    float C = __fdiv_rn(vD, (float)(ny * nxc));
                    res = __ldg(Dimg + (int64_t)yc * W + xc) - C;
                }
                Rring[(yc & 63) * SX + t] = res;
            }
        }
        __syncthreads();
        // ---- 4. hX[j][cs] = sum of E = res^2 over ring cols cs .. cs + 2R of row yc
        for (int it = t; it < 32 * G::NR2; it += NT) {
            int j = it & 31, run = it >> 5;
            int c0 = run * G::RR2;
            int len = min(G::RR2, TX - c0);
            const float* in = Rring + ((ybase + j - R) & 63) * SX;
            float* out = hX + j * SX;
            two_stack_run<R, G::RR2>(c0, len, [&](int c) { float r = in[c]; return r * r; },
                                     [&](int c, float v) { out[c] = v; });
        }
        __syncthreads();
        // ---- 5. vertical compensated sum -> S for row ys = ybase + j - 2R; detect
        {
            float s1 = 0.f, s2 = 0.f;
            int cnt = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float in = col_s ? hX[j * SX + (t - R)] : 0.f;
                float out = histE[(j + 31 - 2 * R) & 31];
                histE[j] = in;
                comp_add(vEs, vEc, in);
                comp_add(vEs, vEc, -out);
                const int ys = ybase + j - 2 * R;
                bool cand = false;
                float snr = 0.f;
                if (col_s && ys >= 0 && ys < H) {
                    float S = (vEs + vEc) * (inv_count<R>(ys, H) * inv_nx);
                    if (S > 0.f) {
                        float res = Rring[(ys & 63) * SX + t];
                        snr = res * rsqrtf(S);
                        s1 += snr;
                        s2 += snr * snr;
                        cnt += 1;
                        if (snr > a.kappa) {
                            const float* p = Dimg + (int64_t)ys * W + xc;
                            const float dv = __ldg(p);
                            bool mx = true;
#pragma unroll
                            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    if (dy == 0 && dx == 0) continue;
                                    int yy = ys + dy, xx = xc + dx;
                                    if (yy >= 0 && yy < H && xx >= 0 && xx < W &&
                                        __ldg(p + (int64_t)dy * W + dx) > dv)
                                        mx = false;
                                }
                            cand = mx;
                        }
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, cand);
                if (bal) {
                    int leader = __ffs(bal) - 1;
                    unsigned base = 0;
                    if (lane == leader) base = atomicAdd(a.counter, (unsigned)(__popc(bal) * nm));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (cand) {
                        unsigned rank = __popc(bal & ((1u << lane) - 1u));
                        uint64_t pix = ((uint64_t)ys << a.bx) | (uint64_t)xc;
                        for (int m = 0; m < nm; ++m) {
                            unsigned idx = base + rank * nm + m;
                            if (idx < (unsigned)a.cap) {
                                a.keys[idx] = ((uint64_t)a.member_ord[m0 + m] << (a.bx + a.by)) | pix;
                                a.vals[idx] = snr;
                            }
                        }
                    }
                }
            }
            d1 += s1;
            d2 += s2;
            dc += cnt;
        }
        __syncthreads();
    }

    // per-CTA stats partials in FP64, fixed reduction order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        dc += __shfl_down_sync(0xffffffffu, dc, o);
    }
    __shared__ double red[NT / 32][3];
    if (lane == 0) { red[t >> 5][0] = d1; red[t >> 5][1] = d2; red[t >> 5][2] = dc; }
    __syncthreads();
    if (t == 0) {
        double q1 = 0, q2 = 0, qc = 0;
        for (int w = 0; w < NT / 32; ++w) { q1 += red[w][0]; q2 += red[w][1]; qc += red[w][2]; }
        double* p = a.partials + ((int64_t)row * gridDim.x + strip) * 3;
        p[0] = q1; p[1] = q2; p[2] = qc;
    }
}

}  // namespace lpf
