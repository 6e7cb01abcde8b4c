// Iterated sigma clipping (Sec. 2.1.1) of the per-subband detector's band
// images, or of the dispersed search's D images (one per distinct delay row, on
// the direct-form path): at each iteration the local centre C and spread S of an
// image X are the
// kernel-weighted means over the window pixels not yet flagged (normalised by
// their kernel weight n), and the pixels with (X - C) / sqrt(S) > kappa join the
// flags; the loop stops when an iteration flags nothing new (each launch of a
// later iteration then returns at once) or after the iteration limit.
// Candidates are the flagged pixels that are (2k+1)^2 maxima of X (Sec. 2.1.2),
// with the S/N of the last iteration.
//
// The kernel on the (2r+1)^2 window is G(dy, dx) = w[|dy|] w[|dx|]: the uniform
// box (w = 1) or the Gaussian exp(-(dy^2 + dx^2) / (2 s^2)), which factorises
// into w[i] = exp(-i^2 / (2 s^2)).  With w = 1 every product below is exact, so
// the box sums are plain FP32 sums.
//
// Planes [F][P] (FP32 unless noted): X, flags (u8), T1, T2 (row sums), C, n, S.
// Window sums are direct weighted FP32 sums over the clipped window, rows then
// columns, tiled in shared memory (k_clip_hsum, k_clip_vsum).
#pragma once
#include "lpf_filter_stream.cuh"

#include <type_traits>

namespace lpf {

struct ClipArgs {
    float* X;
    uint8_t* flags;
    float *T1, *T2, *C, *N, *S;
    unsigned* changed;     // [iters]: bit set when iteration i flagged a new pixel
    const float* w;        // [r + 1] kernel factors w[|d|]
    int F, H, W, r;
    int64_t P;
    float kappa;
};

// iteration it runs unless the previous one flagged nothing new
__device__ __forceinline__ bool clip_active(const ClipArgs& c, int it) { return it == 0 || c.changed[it - 1] != 0u; }

template <typename TS>
__global__ void k_clip_init(ClipArgs c, const TS* __restrict__ slot) {
    const int64_t n = (int64_t)c.F * c.P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        c.X[i] = ld1(slot + i);
        c.flags[i] = 0;
    }
}

// ---------------------------------------------------------------------------
// Tiled window sums, ascending tap order.  R is a compile-time constant
// (with_radius instantiates 1..16), so every tap index and kernel factor is
// fixed.
// f(std::integral_constant<int, r>{}) for a runtime radius r in 1..16
template <typename Fn>
void with_radius(int r, Fn&& fn) {
    switch (r) {
        case 1: fn(std::integral_constant<int, 1>{}); break;
        case 2: fn(std::integral_constant<int, 2>{}); break;
        case 3: fn(std::integral_constant<int, 3>{}); break;
        case 4: fn(std::integral_constant<int, 4>{}); break;
        case 5: fn(std::integral_constant<int, 5>{}); break;
        case 6: fn(std::integral_constant<int, 6>{}); break;
        case 7: fn(std::integral_constant<int, 7>{}); break;
        case 8: fn(std::integral_constant<int, 8>{}); break;
        case 9: fn(std::integral_constant<int, 9>{}); break;
        case 10: fn(std::integral_constant<int, 10>{}); break;
        case 11: fn(std::integral_constant<int, 11>{}); break;
        case 12: fn(std::integral_constant<int, 12>{}); break;
        case 13: fn(std::integral_constant<int, 13>{}); break;
        case 14: fn(std::integral_constant<int, 14>{}); break;
        case 15: fn(std::integral_constant<int, 15>{}); break;
        default: fn(std::integral_constant<int, 16>{}); break;
    }
}

constexpr int kClipHX = 512;            // k_clip_hsum: output columns per CTA (one row)
constexpr int kClipVX = 64;             // k_clip_vsum: output columns per CTA
constexpr int kClipVY = 32;             // k_clip_vsum: output rows per CTA

template <int R>
__device__ __forceinline__ void clip_factors(const ClipArgs& c, float (&g)[R + 1]) {
#pragma unroll
    for (int i = 0; i <= R; ++i) g[i] = __ldg(c.w + i);
}

// Grid (ceil(W / 512) * H, F), 128 threads: one row segment of 512 outputs.  The
// masked inputs (pass 0: X m and m; pass 1: (X - C)^2 m; 0 outside the image)
// go to shared memory, column 0 = image column x0 - A (A = R rounded up to 4);
// thread t owns outputs x0 + 4t .. x0 + 4t + 3 and streams the float4 chunks
// t .. t + NQ - 1 once, each input into the outputs whose window holds it.
template <int R, int PASS>
__global__ void __launch_bounds__(128) k_clip_hsum(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    constexpr int A = (R + 3) & ~3;
    constexpr int NQ = (A + R + 3) / 4 + 1;          // float4 chunks a thread reads
    constexpr int WL = kClipHX + 4 * (NQ - 1);       // loaded columns
    __shared__ __align__(16) float sa[WL];
    __shared__ __align__(16) float sm[PASS == 0 ? WL : 4];
    const int nxb = (c.W + kClipHX - 1) / kClipHX;
    const int y = blockIdx.x / nxb, x0 = (blockIdx.x - y * nxb) * kClipHX;
    const int t = threadIdx.x, f = blockIdx.y;
    const int64_t row = (int64_t)f * c.P + (int64_t)y * c.W;
#pragma unroll
    for (int i = t; i < WL; i += 128) {
        const int x = x0 - A + i;
        const bool in = x >= 0 && x < c.W;
        const int64_t o = row + (in ? x : 0);
        // the flag, the value (and C) are loaded independently, then combined
        const uint8_t fl = in ? __ldg(c.flags + o) : (uint8_t)1;
        const float xv = in ? __ldg(c.X + o) : 0.f;
        const float cv = (PASS == 1 && in) ? __ldg(c.C + o) : 0.f;
        const bool keep = fl == 0;
        float a;
        if (PASS == 0) {
            a = keep ? xv : 0.f;
            sm[i] = keep ? 1.f : 0.f;
        } else {
            const float d = xv - cv;
            a = keep ? d * d : 0.f;
        }
        sa[i] = a;
    }
    float g[R + 1];
    clip_factors<R>(c, g);
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, accm[4] = {0.f, 0.f, 0.f, 0.f};
    const float4* a4 = reinterpret_cast<const float4*>(sa) + t;
    const float4* m4 = reinterpret_cast<const float4*>(sm) + t;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float4 va = a4[q];
        float4 vm = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PASS == 0) vm = m4[q];
        const float ea[4] = {va.x, va.y, va.z, va.w}, em[4] = {vm.x, vm.y, vm.z, vm.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            // shared column 4t + 4q + e holds image column x0 + 4t + 4q + e - A; for
            // output j (image column x0 + 4t + j) it is tap d = 4q + e - A - j
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int d = 4 * q + e - A - j;
                if (d >= -R && d <= R) {
                    const float w = g[d < 0 ? -d : d];
                    acc[j] = fmaf(w, ea[e], acc[j]);
                    if (PASS == 0) accm[j] = fmaf(w, em[e], accm[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = x0 + 4 * t + j;
        if (x < c.W) {
            c.T1[row + x] = acc[j];
            if (PASS == 0) c.T2[row + x] = accm[j];
        }
    }
}

// Grid (ceil(W / 64), ceil(H / 32), F), 128 threads: a 32 x 64 tile of outputs.
// The row sums of rows y0 - R .. y0 + 31 + R (0 outside the image) go to shared
// memory; thread (quad q = t % 16, group g = t / 16) owns rows y0 + 4g .. + 3 of
// columns x0 + 4q .. + 3 and streams its 2R + 4 float4 rows once.
// pass 0: n = the sums of T2, C = the sums of T1 / n (0 where n = 0);
// pass 1: S = the sums of T1 / n.
template <int R, int PASS>
__global__ void __launch_bounds__(128) k_clip_vsum(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    constexpr int NRW = kClipVY + 2 * R;
    __shared__ __align__(16) float s1[NRW][kClipVX];
    __shared__ __align__(16) float s2[PASS == 0 ? NRW : 1][kClipVX];
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kClipVX, y0 = blockIdx.y * kClipVY, f = blockIdx.z;
    const int64_t plane = (int64_t)f * c.P;
    // asynchronous 4-byte copies, zero-filled outside the image (the source address
    // then stays at the plane's first pixel and is not read)
#pragma unroll 4
    for (int i = t; i < NRW * kClipVX; i += 128) {
        const int rr = i / kClipVX, cc = i - rr * kClipVX;
        const int y = y0 - R + rr, x = x0 + cc;
        const bool in = y >= 0 && y < c.H && x < c.W;
        const int64_t o = plane + (in ? (int64_t)y * c.W + x : 0);
        cp_async4(&s1[rr][cc], c.T1 + o, in);
        if (PASS == 0) cp_async4(&s2[rr][cc], c.T2 + o, in);
    }
    cp_async_commit();
    float g[R + 1];
    clip_factors<R>(c, g);
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    const int q = t & 15, gr = t >> 4;
    float4 acc[4], acc2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc2[j] = acc[j];
    }
#pragma unroll
    for (int k = 0; k < 2 * R + 4; ++k) {
        // shared row 4 gr + k is image row y0 + 4 gr + k - R: tap d = k - R - j of output row j
        const float4 v = reinterpret_cast<const float4*>(s1[4 * gr + k])[q];
        float4 v2 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PASS == 0) v2 = reinterpret_cast<const float4*>(s2[4 * gr + k])[q];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int d = k - R - j;
            if (d >= -R && d <= R) {
                const float w = g[d < 0 ? -d : d];
                acc[j].x = fmaf(w, v.x, acc[j].x);
                acc[j].y = fmaf(w, v.y, acc[j].y);
                acc[j].z = fmaf(w, v.z, acc[j].z);
                acc[j].w = fmaf(w, v.w, acc[j].w);
                if (PASS == 0) {
                    acc2[j].x = fmaf(w, v2.x, acc2[j].x);
                    acc2[j].y = fmaf(w, v2.y, acc2[j].y);
                    acc2[j].z = fmaf(w, v2.z, acc2[j].z);
                    acc2[j].w = fmaf(w, v2.w, acc2[j].w);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = y0 + 4 * gr + j;
        if (y >= c.H) continue;
        const float a1[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
        const float a2[4] = {acc2[j].x, acc2[j].y, acc2[j].z, acc2[j].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int x = x0 + 4 * q + e;
            if (x >= c.W) continue;
            const int64_t o = plane + (int64_t)y * c.W + x;
            if (PASS == 0) {
                c.N[o] = a2[e];
                c.C[o] = a2[e] > 0.f ? a1[e] / a2[e] : 0.f;
            } else {
                const float cnt = c.N[o];
                c.S[o] = cnt > 0.f ? a1[e] / cnt : 0.f;
            }
        }
    }
}

// Pixels are taken four at a time (16-byte loads of X, C, S and 4-byte loads of
// the flags; the planes start on 32-byte boundaries); the last group of a band
// with H W not a multiple of 4 is read one pixel at a time.
struct ClipQuad {
    float X[4], C[4], S[4];
    uint8_t fl[4];
    int n;                     // pixels of the group inside the band (0..4)
};

__device__ __forceinline__ ClipQuad clip_quad(const ClipArgs& c, int64_t plane, int64_t i, int64_t HW) {
    ClipQuad q;
    q.n = HW - i >= 4 ? 4 : (int)(HW - i);
    if (q.n == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(c.X + plane + i));
        const float4 cc = __ldg(reinterpret_cast<const float4*>(c.C + plane + i));
        const float4 sv = __ldg(reinterpret_cast<const float4*>(c.S + plane + i));
        const uchar4 fl = *reinterpret_cast<const uchar4*>(c.flags + plane + i);
        q.X[0] = x.x; q.X[1] = x.y; q.X[2] = x.z; q.X[3] = x.w;
        q.C[0] = cc.x; q.C[1] = cc.y; q.C[2] = cc.z; q.C[3] = cc.w;
        q.S[0] = sv.x; q.S[1] = sv.y; q.S[2] = sv.z; q.S[3] = sv.w;
        q.fl[0] = fl.x; q.fl[1] = fl.y; q.fl[2] = fl.z; q.fl[3] = fl.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const bool in = e < q.n;
            const int64_t o = plane + i + (in ? e : 0);
            q.X[e] = in ? c.X[o] : 0.f;
            q.C[e] = in ? c.C[o] : 0.f;
            q.S[e] = in ? c.S[o] : 0.f;
            q.fl[e] = in ? c.flags[o] : (uint8_t)1;
        }
    }
    return q;
}

__device__ __forceinline__ float clip_snr_of(float X, float C, float S) { return S > 0.f ? (X - C) / sqrtf(S) : 0.f; }

// Grid (blocks, F): flags |= (snr > kappa) over the H W pixels of band
// blockIdx.y; changed[it] when a pixel is flagged for the first time.
__global__ void __launch_bounds__(256) k_clip_flag(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    const int64_t HW = (int64_t)c.H * c.W, plane = (int64_t)blockIdx.y * c.P;
    bool fresh = false;
    for (int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); i < HW;
         i += 4 * (int64_t)gridDim.x * blockDim.x) {
        const ClipQuad q = clip_quad(c, plane, i, HW);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e < q.n && !q.fl[e] && clip_snr_of(q.X[e], q.C[e], q.S[e]) > c.kappa) {
                c.flags[plane + i + e] = 1;
                fresh = true;
            }
        }
    }
    if (__syncthreads_or(fresh) && threadIdx.x == 0) atomicOr(c.changed + it, 1u);
}

// Grid (blocks per plane, planes): S/N of the last iteration, the per-plane
// statistics partials (FP32 per thread, FP64 per block), and the candidates:
// flagged pixels with S > 0 that are (2k+1)^2 maxima of X, one record per trial
// of the plane's row (a band: one trial; a distinct delay row: its members).
__global__ void __launch_bounds__(256) k_clip_emit(ClipArgs c, FilterArgs a, int k) {
    const int f = blockIdx.y;
    const int m0 = a.member_start[f], nm = a.member_start[f + 1] - m0;
    const int64_t HW = (int64_t)c.H * c.W, plane = (int64_t)f * c.P;
    const int lane = threadIdx.x & 31;
    float s1 = 0.f, s2 = 0.f, cnt = 0.f;
    const int64_t stride = 4 * (int64_t)gridDim.x * blockDim.x;
    // every thread of the block runs the same number of rounds (warp ballots)
    for (int64_t base = 4 * (int64_t)blockIdx.x * blockDim.x; base < HW; base += stride) {
        const int64_t i = base + 4 * threadIdx.x;
        ClipQuad q;
        q.n = 0;
        if (i < HW) q = clip_quad(c, plane, i, HW);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bool cand = false;
            int y = 0, x = 0;
            float snr = 0.f;
            if (e < q.n) {
                const bool valid = q.S[e] > 0.f;
                snr = clip_snr_of(q.X[e], q.C[e], q.S[e]);
                if (valid) {
                    s1 += snr;
                    s2 = fmaf(snr, snr, s2);
                    cnt += 1.f;
                }
                if (valid && q.fl[e]) {
                    const int64_t p = i + e;
                    y = (int)(p / c.W);
                    x = (int)(p - (int64_t)y * c.W);
                    const float* img = c.X + plane;
                    cand = window_is_max(y, x, k, c.H, c.W, q.X[e],
                                         [&](int yy, int xx) { return img[(int64_t)yy * c.W + xx]; });
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, cand);
            if (bal) {
                unsigned b0 = 0;
                const int leader = __ffs(bal) - 1;
                if (lane == leader) b0 = atomicAdd(a.counter, (unsigned)(__popc(bal) * nm));
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (cand) {
                    const unsigned base = b0 + __popc(bal & ((1u << lane) - 1u)) * (unsigned)nm;
                    const uint64_t pix = ((uint64_t)y << a.bx) | (uint64_t)x;
                    mark_zero_row(a, f, pix);
                    for (int m = 0; m < nm; ++m) {
                        const unsigned idx = base + (unsigned)m;
                        if (idx < (unsigned)a.cap) {
                            a.keys[idx] = ((uint64_t)a.member_ord[m0 + m] << (a.bx + a.by)) | pix;
                            a.vals[idx] = snr;
                        }
                    }
                }
            }
        }
    }
    double d1 = s1, d2 = s2, dc = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        dc += __shfl_down_sync(0xffffffffu, dc, o);
    }
    __shared__ double red[8][3];
    if (lane == 0) { red[threadIdx.x >> 5][0] = d1; red[threadIdx.x >> 5][1] = d2; red[threadIdx.x >> 5][2] = dc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double q1 = 0, q2 = 0, qc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { q1 += red[w][0]; q2 += red[w][1]; qc += red[w][2]; }
        double* p = a.partials + ((int64_t)f * gridDim.x + blockIdx.x) * 3;
        p[0] = q1; p[1] = q2; p[2] = qc;
    }
}

}  // namespace lpf
