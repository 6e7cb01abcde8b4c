// The streaming filter of the residual path (Sec. 2.1.1 spread, threshold and
// the per-trial statistics): k_filter_res reads the R_d = D_d - C_d images of
// the shift-sum, forms S_d = box mean of R_d^2, snr = R_d / sqrt(S_d), the
// statistics partials, and appends every threshold crossing to the list that
// k_lmax_res (lpf_residual.cuh) resolves.
#pragma once
#include "lpf_residual.cuh"

namespace lpf {

// ---------------------------------------------------------------------------
// Geometry of k_filter_res: R rows in shared memory start on 16-byte
// boundaries (column 0 is image column x0 - A, A = r rounded up to a multiple
// of 4), so they are copied 16 bytes at a time and read as float4.  The pitch
// SD = 4 (mod 32) words makes the float4 reads of 32 lanes on 32 rows
// conflict-free (8 lanes per wavefront, each on its own 16-byte bank group).
template <int R>
struct FiltGeom {
    static constexpr int TX = 128;
    static constexpr int L = 2 * R + 1;
    static constexpr int NP = 32 / L;
    static constexpr int B = NP * L;                         // rows per block
    static constexpr int A = (R + 3) & ~3;                   // left margin
    static constexpr int WL = (TX + A + R + 3) & ~3;         // loaded columns
    static constexpr int NC = WL / 4;                        // 16-byte chunks per row
    static constexpr int SD = ((WL + 27) & ~31) + 4;         // pitch, = 4 (mod 32)
    static constexpr int SX = TX | 1;
    static constexpr int RR = (2 * R + 1) & ~3;              // run length (multiple of 4, <= 2r+1)
    static constexpr int NR = (TX + RR - 1) / RR;
    static constexpr int LAST = TX - (NR - 1) * RR;
    static constexpr int NT = 160;
    static_assert(SD >= WL && SD % 32 == 4 && NC >= 32 && NC <= 64, "copy by one warp, two chunks a lane");
    static_assert(B <= 32 && LAST > 0 && LAST <= RR, "lane = row; ragged last run");
};

// Horizontal window sums of R^2 for the outputs c0 .. c0 + LEN - 1 (relative to
// x0) of one shared-memory row: the inputs v[i] = R(x0 + c0 - r + i), i in
// [0, 2r + LEN), lie at row columns c0 + (A - r) + i.  Two stacks around the
// pivot i = 2r (SUF of v[o .. 2r-1] + PRE of v[2r .. 2r+o]), squares by fma.
template <int R, int A, int LEN>
__device__ __forceinline__ void hsum_sq_run(const float* __restrict__ in, int c0, float* __restrict__ out) {
    constexpr int OFF = A - R;
    constexpr int NS = LEN < 2 * R ? LEN : 2 * R;
    float suf[NS];
    float acc = 0.f;
#pragma unroll
    for (int q = (OFF + 2 * R - 1) / 4; q >= 0; --q) {
        const float4 c = *reinterpret_cast<const float4*>(in + c0 + 4 * q);
        const float e[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 3; k >= 0; --k) {
            const int i = 4 * q + k - OFF;
            if (i >= 0 && i < 2 * R) {
                acc = fmaf(e[k], e[k], acc);
                if (i < NS) suf[i < NS ? i : 0] = acc;
            }
        }
    }
    float pre = 0.f;
#pragma unroll
    for (int q = (OFF + 2 * R) / 4; q <= (OFF + 2 * R + LEN - 1) / 4; ++q) {
        const float4 c = *reinterpret_cast<const float4*>(in + c0 + 4 * q);
        const float e[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = 4 * q + k - OFF;
            if (i >= 2 * R && i < 2 * R + LEN) {
                pre = fmaf(e[k], e[k], pre);
                const int o = i - 2 * R;
                out[c0 + o] = (o < NS) ? suf[o < NS ? o : 0] + pre : pre;
            }
        }
    }
}

// k_filter_res: per distinct row (blockIdx.y) and 128-column strip, streaming
// down in blocks of B rows of R = D - C held in a double buffer (block k being
// used, block k+1 being copied in):
//   2. all warps: horizontal window sums of R^2 (two stacks), warp w one run of
//      columns, lane = row                                               -> hE
//   3. warps 0-3, one column each: vertical window sum as the suffix of the
//      previous (2r+1)-row segment plus the prefix of the current one (exact)
//      -> S(ys), ys = row - r; snr = R(ys)/sqrt(S), stats.  The h values of a
//      segment stay in registers for its suffix sums, so each h slot of hE is
//      free once read: the snr is parked there, and candidates are resolved
//      once per block.  R(ys) of the first r rows lies in the last r rows of
//      block k-1, whose buffer is refilled during this pass: the column warps
//      read those r values first and then release the loader (named barrier 1).
//      warp 4 meanwhile issues the cp.async copies of block k+1.
//   One barrier per block publishes the copies and separates the vertical pass
//   of block k-1 from the horizontal pass of block k; a second one separates
//   the horizontal and vertical passes of block k.  A pixel outside the image
//   has a zero column or row factor, so S = 0 there and it is not valid.
template <int R, typename TS>
__global__ void __launch_bounds__(FiltGeom<R>::NT, 4) k_filter_res(ResArgs ra) {
    using G = FiltGeom<R>;
    constexpr int TX = G::TX, B = G::B, L = G::L, SD = G::SD, SX = G::SX, NT = G::NT;
    constexpr int NP = G::NP, RR = G::RR, NR = G::NR, A = G::A, WL = G::WL, NC = G::NC;
    extern __shared__ __align__(16) float sm[];
    float* Rb = sm;                     // [2][B][SD] R rows; col = x - (x0 - A)
    float* hE = Rb + 2 * B * SD;        // [B][SX]
    __shared__ float2 rowS[B];
    const FilterArgs& a = ra.a;
    const int strip = blockIdx.x, row = blockIdx.y;
    const int x0 = strip * TX;
    const int H = a.H, W = a.W;
    const float* Rimg = a.D + (int64_t)row * a.P;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const bool loader = t >= TX;        // warp 4: copies
    const int xs = x0 + t;
    const bool col_s = t < TX && xs < W;
    const int nx = col_s ? min(xs + R, W - 1) - max(xs - R, 0) + 1 : 0;
    const float inv_nx = col_s ? 1.0f / (float)nx : 0.f;
    // 16-byte copies need whole chunks inside the image and 16-byte aligned rows
    const bool vec_cols = x0 - A >= 0 && x0 - A + WL <= W && (W & 3) == 0;
    float suf[L];
#pragma unroll
    for (int i = 0; i < L; ++i) suf[i] = 0.f;
    float pre = 0.f;
    double d1 = 0.0, d2 = 0.0, dc = 0.0;
    const int m0 = a.member_start[row], nm = a.member_start[row + 1] - m0;

    // copies of block kk (rows kk*B ..) by the threads of [t0, t0 + nthr)
    auto load = [&](int kk, int t0, int nthr) {
        float* dst = Rb + (kk & 1) * B * SD;
        const int yb = kk * B;
        const int u = t - t0;
        if (vec_cols && yb + B <= H) {
            const float* src = Rimg + (int64_t)yb * W + (x0 - A);
            if (nthr == 32) {
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    cp_async16(dst + j * SD + 4 * u, src + (int64_t)j * W + 4 * u);
                    if (u + 32 < NC) cp_async16(dst + j * SD + 4 * (u + 32), src + (int64_t)j * W + 4 * (u + 32));
                }
            } else {
                for (int i = u; i < B * NC; i += nthr) {
                    const int j = i / NC, ch = i - j * NC;
                    cp_async16(dst + j * SD + 4 * ch, src + (int64_t)j * W + 4 * ch);
                }
            }
        } else {
            for (int c = u; c < WL; c += nthr) {
                const int x = x0 - A + c;
                const bool colok = x >= 0 && x < W;
                const float* src = Rimg + (int64_t)yb * W + x;
#pragma unroll 4
                for (int j = 0; j < B; ++j) {
                    bool in = colok && yb + j < H;
                    cp_async4(dst + j * SD + c, in ? src : Rimg, in);
                    src += W;
                }
            }
        }
    };
    // row segment blockIdx.z: blocks [k0, k1); a segment after the first starts one
    // block early, to build the suffix sums of the vertical two-stack (no output)
    const int nblk = (H + R + B - 1) / B;
    const int seg_blocks = (nblk + (int)gridDim.z - 1) / (int)gridDim.z;
    const int k0 = (int)blockIdx.z * seg_blocks, k1 = min(nblk, k0 + seg_blocks);
    double* partial = a.partials + (((int64_t)row * gridDim.z + blockIdx.z) * gridDim.x + strip) * 3;
    if (k0 >= k1) {
        if (t == 0) { partial[0] = 0.0; partial[1] = 0.0; partial[2] = 0.0; }
        return;
    }
    const int kbeg = k0 > 0 ? k0 - 1 : 0;
    load(kbeg, 0, NT);
    cp_async_commit();
    for (int k = kbeg; k < k1; ++k) {
        const int ybase = k * B;
        const float* cur = Rb + (k & 1) * B * SD;
        // one barrier both publishes the copies of block k and ends the vertical
        // pass of block k-1 (its reads of hE and rowS)
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();
        if (t < B) rowS[t] = row_count<R>(ybase + t - R, H);
        // ---- horizontal window sums of R^2 (output col x0 + c), warp = run, lane = row
        for (int ru = warp; ru < NR; ru += NT / 32) {
            if (lane < B) {
                if (ru < NR - 1) hsum_sq_run<R, A, RR>(cur + lane * SD, ru * RR, hE + lane * SX);
                else hsum_sq_run<R, A, G::LAST>(cur + lane * SD, (NR - 1) * RR, hE + lane * SX);
            }
        }
        __syncthreads();
        if (loader) {
            // ---- the next block's copies while the column warps run the vertical
            // pass, once they have read the last r rows of block k-1 (its buffer)
            asm volatile("bar.sync 1, %0;\n" ::"n"(NT));
            if (k + 1 < k1) load(k + 1, TX, NT - TX);
            cp_async_commit();
        } else if (k < k0) {
            asm volatile("bar.arrive 1, %0;\n" ::"n"(NT));
            // warm-up block: the suffix sums of its last (2r+1)-row segment
            float acc = 0.f;
#pragma unroll
            for (int i = L - 1; i >= 1; --i) { acc += hE[((NP - 1) * L + i) * SX + t]; suf[i] = acc; }
        } else {
            // R(ys) of the rows of block k-1 (ys = ybase - r .. ybase - 1): its last
            // r rows, zero above the image (the copies zero-fill rows outside it)
            float rvp[R];
            const float* prev = Rb + ((k + 1) & 1) * B * SD + t + A;
#pragma unroll
            for (int j = 0; j < R; ++j) rvp[j] = k > 0 ? prev[(B - R + j) * SD] : 0.f;
            asm volatile("bar.arrive 1, %0;\n" ::"n"(NT));
            // the snr of row j is parked in the hE slot of its own h value
            float* park = hE + t;
            // ---- vertical segment sums -> S for row ys = ybase + j - r
            float s1 = 0.f, s2 = 0.f, cnt = 0.f;
            unsigned cm = 0;
#pragma unroll
            for (int sgm = 0; sgm < NP; ++sgm) {
                float hv[L];                    // this segment's h, for its suffix sums
#pragma unroll
                for (int o = 0; o < L; ++o) {
                    const int j = sgm * L + o;
                    const float h = hE[j * SX + t];
                    hv[o] = h;
                    pre = (o == 0) ? h : pre + h;
                    const float Ssum = (o + 1 < L) ? suf[o + 1] + pre : pre;
                    const float S = Ssum * (rowS[j].y * inv_nx);
                    // a spread below the smallest normal FP32 number counts as none
                    const bool valid = S >= 1.17549435e-38f;
                    const float rv = (j >= R) ? cur[(j - R) * SD + t + A] : rvp[j < R ? j : 0];
                    // branch-free: an invalid pixel adds exactly +0 to the sums
                    const float snr = valid ? rv * rsqrt_normal(S) : 0.f;
                    s1 += snr;
                    s2 = fmaf(snr, snr, s2);
                    cnt += valid ? 1.f : 0.f;
                    cm |= (valid && snr > a.kappa) ? 1u << j : 0u;
                    park[j * SX] = snr;
                }
                // suffix sums of the finished segment for the next one
                float acc = 0.f;
#pragma unroll
                for (int i = L - 1; i >= 1; --i) { acc += hv[i]; suf[i] = acc; }
            }
            d1 += s1;
            d2 += s2;
            dc += cnt;
            // ---- threshold crossings of this block: one reservation per warp in
            // the crossing list (the 3x3 maximum of D is taken by k_lmax_res); a
            // warp whose reservation does not fit voids it and resolves its
            // crossings here, so every crossing is resolved exactly once
            if (__reduce_or_sync(0xffffffffu, cm)) {
                const unsigned mine = __popc(cm);
                unsigned incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
                unsigned long long base = 0;
                if (lane == 31) base = atomicAdd(ra.xcounter, (unsigned long long)total);
                base = __shfl_sync(0xffffffffu, base, 31);
                if (base + total <= (unsigned long long)ra.xcap) {
                    unsigned long long idx = base + incl - mine;
                    for (unsigned b = cm; b; b &= b - 1) {
                        const int j = __ffs(b) - 1;
                        ra.xkeys[idx] = ((uint64_t)row << 32) | ((uint64_t)(ybase + j - R) << 16) | (uint64_t)xs;
                        ra.xvals[idx] = park[j * SX];
                        ++idx;
                    }
                } else {
                    for (unsigned long long i = base + lane; i < base + total && i < (unsigned long long)ra.xcap; i += 32)
                        ra.xkeys[i] = kNoCrossing;
                    unsigned any = __reduce_or_sync(0xffffffffu, cm);
                    while (any) {
                        const int j = __ffs(any) - 1;
                        any &= any - 1;
                        const bool cand = (cm >> j) & 1u;
                        emit_res_candidates<TS>(ra, row, ybase + j - R, xs, cand ? park[j * SX] : 0.f, cand,
                                                m0, nm);
                    }
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
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
        partial[0] = q1; partial[1] = q2; partial[2] = qc;
    }
}

template <int R>
constexpr size_t res_filter_smem_bytes() {
    return ((size_t)2 * FiltGeom<R>::B * FiltGeom<R>::SD + (size_t)FiltGeom<R>::B * FiltGeom<R>::SX) * sizeof(float);
}

}  // namespace lpf
