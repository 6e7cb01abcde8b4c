// Streaming box filter + detection for a compile-time box radius R <= 15.
//
// One CTA owns a strip of TX = 128 output columns of one dedispersed image and
// walks down it in blocks of B = NP (2R + 1) <= 32 rows, so rows are never
// recomputed (only the 2R-column halo of the strip is).  Per block:
//   1. D rows of the block (strip + 2R halo each side) are in one half of a
//      double buffer (cp.async prefetch issued during the previous block)
//   2. horizontal window sums of D ("two stacks", cancellation free)   -> hX
//   3. per column: vertical sliding sum of hX -> C, residual D - C into a
//      shared ring of 64 rows; then the prefetch of the next block is issued
//   4. horizontal window sums of E = (D - C)^2                          -> hX
//   5. per column: vertical window sum of hX as the suffix of the previous
//      (2R + 1)-row segment plus the prefix of the current one (exact: sums of
//      consecutive terms only) -> S, snr = (D - C)/sqrt(S), threshold, 3x3
//      local maximum, stats, emission
// The vertical pass of C runs R rows behind the input and that of S 2R rows
// behind; the column thread that computes C for a column is the one that later
// computes S for it, and the residual ring carries D - C across that lag.
// Out-of-image rows and columns contribute zeros, and C and S divide by the
// in-image window count, which clips every window to the image (Sec. 2.1.1).
// C = sum / n is formed as sum * (1/n) refined by one Newton step against the
// exact count n, so a constant window gives C equal to that constant and S = 0.
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

constexpr int kStreamTX = 128;
constexpr int kStreamThreads = 192;

template <int R>
struct StreamGeom {
    static constexpr int TX = kStreamTX;
    static constexpr int L = 2 * R + 1;           // vertical segment length
    static constexpr int NP = 32 / L;             // segments per block
    static constexpr int B = NP * L;              // rows per block
    static constexpr int WC = TX + 2 * R;         // columns carrying C and the residual
    static constexpr int WD = TX + 4 * R;         // columns carrying D
    static constexpr int SD = WD | 1;             // odd strides: conflict-free column walks
    static constexpr int SX = WC | 1;
    static constexpr int NR1 = (WC + L - 1) / L;          // runs per row, horizontal pass 1
    static constexpr int RR1 = (WC + NR1 - 1) / NR1;
    static constexpr int NR2 = (TX + L - 1) / L;          // runs per row, horizontal pass 2
    static constexpr int RR2 = (TX + NR2 - 1) / NR2;
    static constexpr size_t smem_floats = (size_t)2 * B * SD + (size_t)B * SX + (size_t)64 * SX;
    static_assert(WD <= kStreamThreads && WC <= kStreamThreads, "one thread per column");
    static_assert(B + R <= 64, "residual ring too short");
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

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Copies of D rows [ybase, ybase + B) x cols [x0 - 2R, x0 + TX + 2R) into dst,
// one column per thread, zero-filled outside the image.
template <int R>
__device__ __forceinline__ void load_block_async(float* dst, const float* Dimg, int ybase, int x0,
                                                 int H, int W, int t) {
    using G = StreamGeom<R>;
    if (t >= G::WD) return;
    const int x = x0 - 2 * R + t;
    const bool colok = x >= 0 && x < W;
    const float* src = Dimg + (int64_t)ybase * W + x;
#pragma unroll
    for (int j = 0; j < G::B; ++j) {
        bool in = colok && (ybase + j) < H;
        cp_async4(dst + j * G::SD + t, in ? src : Dimg, in);
        src += W;
    }
}

// (n_y, 1/n_y) of an image row's clipped vertical window; n_y = 0 outside the image.
template <int R>
__device__ __forceinline__ float2 row_count(int y, int H) {
    if (y < 0 || y >= H) return make_float2(0.f, 0.f);
    int c = min(y + R, H - 1) - max(y - R, 0) + 1;
    return make_float2((float)c, 1.0f / (float)c);
}

// Candidates of one image row of a warp (rare): 3x3 local maximum of D clipped
// to the image (ties count as maxima), then one warp-aggregated reservation and
// one record per DM trial sharing this delay row.  Kept out of line so the
// unrolled row loops stay small.  Every lane of the warp calls it.
__device__ __noinline__ void emit_candidates(const FilterArgs& a, const float* Dimg, int ys, int xc,
                                             float snr, bool cand, int m0, int nm) {
    const int H = a.H, W = a.W;
    const int lane = threadIdx.x & 31;
    if (cand) {
        const float* p = Dimg + (int64_t)ys * W + xc;
        const float dv = __ldg(p);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dy == 0 && dx == 0) continue;
                int yy = ys + dy, xx = xc + dx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W && __ldg(p + (int64_t)dy * W + dx) > dv)
                    cand = false;
            }
    }
    unsigned bal = __ballot_sync(0xffffffffu, cand);
    if (!bal) return;
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

template <int R>
__global__ void __launch_bounds__(kStreamThreads, 2) k_filter_stream(FilterArgs a) {
    using G = StreamGeom<R>;
    constexpr int TX = G::TX, WC = G::WC, SD = G::SD, SX = G::SX, B = G::B, L = G::L;
    constexpr int NT = kStreamThreads;
    extern __shared__ float sm[];
    float* Dbuf = sm;                   // [2][B][SD] D rows of a block, double buffer; col = x - (x0 - 2R)
    float* hX = Dbuf + 2 * B * SD;      // [B][SX]  horizontal sums of the block
    float* Rring = hX + B * SX;         // [64][SX] residual D - C by row & 63; col = x - (x0 - R)
    __shared__ float2 rowC[B], rowS[B]; // clipped row counts for the C rows and the S rows

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
    const int nxc = xc_in ? min(xc + R, W - 1) - max(xc - R, 0) + 1 : 0;
    const float nxf = (float)nxc;
    const float inv_nx = xc_in ? 1.0f / nxf : 0.f;

    float histD[L];                      // hX of the last L rows (sliding sum of C)
    float raw[L], suf[L];                // two-stack of the S sums: current segment, previous suffix
#pragma unroll
    for (int i = 0; i < L; ++i) { histD[i] = 0.f; raw[i] = 0.f; suf[i] = 0.f; }
    float vD = 0.f, pre = 0.f;
    double d1 = 0.0, d2 = 0.0, dc = 0.0;
    const int m0 = a.member_start[row], nm = a.member_start[row + 1] - m0;

    const int nblk = (H + 2 * R + B - 1) / B;
    load_block_async<R>(Dbuf, Dimg, 0, x0, H, W, t);
    cp_async_commit();
    for (int k = 0; k < nblk; ++k) {
        const int ybase = k * B;
        const float* Dcur = Dbuf + (k & 1) * B * SD;
        const float* Dprev = Dbuf + ((k + 1) & 1) * B * SD;
        if (t < B) rowC[t] = row_count<R>(ybase + t - R, H);
        else if (t < 2 * B) rowS[t - B] = row_count<R>(ybase + (t - B) - 2 * R, H);
        cp_async_wait_all();
        __syncthreads();
        // ---- 2. hX[j][c] = sum of D over columns c .. c + 2R (buffer cols) of row ybase + j
        for (int it = t; it < B * G::NR1; it += NT) {
            int j = it % B, run = it / B;
            int c0 = run * G::RR1;
            int len = min(G::RR1, WC - c0);
            const float* in = Dcur + j * SD;
            float* out = hX + j * SX;
            two_stack_run<R, G::RR1>(c0, len, [&](int c) { return in[c]; },
                                     [&](int c, float v) { out[c] = v; });
        }
        __syncthreads();
        // ---- 3. vertical sliding sum -> C for row yc = ybase + j - R, residual D - C
        if (col_c) {
#pragma unroll
            for (int j = 0; j < B; ++j) {
                float in = hX[j * SX + t];
                float out = histD[j % L];
                histD[j % L] = in;
                vD += in - out;
                const int yc = ybase + j - R;
                const float2 cy = rowC[j];
                const float dv = (j >= R) ? Dcur[(j - R) * SD + t + R] : Dprev[(B + j - R) * SD + t + R];
                const float n = cy.x * nxf, inv = cy.y * inv_nx;
                const float c0 = vD * inv;
                const float C = fmaf(fmaf(-c0, n, vD), inv, c0);
                Rring[(yc & 63) * SX + t] = (n > 0.f) ? dv - C : 0.f;
            }
        }
        __syncthreads();
        // the previous block's rows are no longer needed: prefetch the next block
        if (k + 1 < nblk) load_block_async<R>(Dbuf + ((k + 1) & 1) * B * SD, Dimg, ybase + B, x0, H, W, t);
        cp_async_commit();
        // ---- 4. hX[j][cs] = sum of E = res^2 over ring cols cs .. cs + 2R of row yc
        for (int it = t; it < B * G::NR2; it += NT) {
            int j = it % B, run = it / B;
            int c0 = run * G::RR2;
            int len = min(G::RR2, TX - c0);
            const float* in = Rring + ((ybase + j - R) & 63) * SX;
            float* out = hX + j * SX;
            two_stack_run<R, G::RR2>(c0, len, [&](int c) { float r = in[c]; return r * r; },
                                     [&](int c, float v) { out[c] = v; });
        }
        __syncthreads();
        // ---- 5. vertical segment sums -> S for row ys = ybase + j - 2R; detect
        {
            float s1 = 0.f, s2 = 0.f, cnt = 0.f;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const int o = j % L;
                const float in = col_s ? hX[j * SX + (t - R)] : 0.f;
                raw[o] = in;
                pre = (o == 0) ? in : pre + in;
                const float Ssum = (o + 1 < L) ? suf[o + 1] + pre : pre;
                if (o == L - 1) {
                    // suffix sums of the finished segment for the next one
                    float acc = 0.f;
#pragma unroll
                    for (int i = L - 1; i >= 1; --i) { acc += raw[i]; suf[i] = acc; }
                }
                const int ys = ybase + j - 2 * R;
                const float2 sy = rowS[j];
                const float S = Ssum * (sy.y * inv_nx);
                const bool valid = col_s && sy.x > 0.f && S > 0.f;
                float snr = 0.f;
                if (valid) {
                    snr = Rring[(ys & 63) * SX + t] * rsqrtf(S);
                    s1 += snr;
                    s2 = fmaf(snr, snr, s2);
                    cnt += 1.f;
                }
                const bool cand = valid && snr > a.kappa;
                if (__any_sync(0xffffffffu, cand))
                    emit_candidates(a, Dimg, ys, xc, snr, cand, m0, nm);
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
