// Iterated sigma clipping of the per-subband detector (Sec. 2.1.1): at each
// iteration the local centre C and spread S of a band image X are the
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
// columns.
#pragma once
#include "lpf_kernels.cuh"

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

// pass 0: T1 = weighted row sums of X m, T2 = of m (m = unflagged);
// pass 1: T1 = weighted row sums of (X - C)^2 m
template <int PASS>
__global__ void k_clip_rows(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    const int64_t n = (int64_t)c.F * c.H * c.W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % c.W);
        const int64_t fy = i / c.W;
        const int f = (int)(fy / c.H), y = (int)(fy - (int64_t)f * c.H);
        const int64_t row = (int64_t)f * c.P + (int64_t)y * c.W;
        float s1 = 0.f, s2 = 0.f;
        for (int xx = max(x - c.r, 0); xx <= min(x + c.r, c.W - 1); ++xx) {
            if (c.flags[row + xx]) continue;
            const float g = __ldg(c.w + abs(xx - x));
            if (PASS == 0) {
                s1 = fmaf(g, c.X[row + xx], s1);
                s2 += g;
            } else {
                const float d = c.X[row + xx] - c.C[row + xx];
                s1 = fmaf(g * d, d, s1);
            }
        }
        c.T1[row + x] = s1;
        if (PASS == 0) c.T2[row + x] = s2;
    }
}

// pass 0: n = weighted column sums of T2, C = weighted column sums of T1 / n
// (0 where n = 0); pass 1: S = weighted column sums of T1 / n
template <int PASS>
__global__ void k_clip_cols(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    const int64_t n = (int64_t)c.F * c.H * c.W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % c.W);
        const int64_t fy = i / c.W;
        const int f = (int)(fy / c.H), y = (int)(fy - (int64_t)f * c.H);
        const int64_t base = (int64_t)f * c.P + x;
        float s1 = 0.f, s2 = 0.f;
        for (int yy = max(y - c.r, 0); yy <= min(y + c.r, c.H - 1); ++yy) {
            const float g = __ldg(c.w + abs(yy - y));
            s1 = fmaf(g, c.T1[base + (int64_t)yy * c.W], s1);
            if (PASS == 0) s2 = fmaf(g, c.T2[base + (int64_t)yy * c.W], s2);
        }
        const int64_t o = base + (int64_t)y * c.W;
        if (PASS == 0) {
            c.N[o] = s2;
            c.C[o] = s2 > 0.f ? s1 / s2 : 0.f;
        } else {
            const float cnt = c.N[o];
            c.S[o] = cnt > 0.f ? s1 / cnt : 0.f;
        }
    }
}

__device__ __forceinline__ float clip_snr(const ClipArgs& c, int64_t o) {
    const float S = c.S[o];
    return S > 0.f ? (c.X[o] - c.C[o]) / sqrtf(S) : 0.f;
}

// flags |= (snr > kappa); changed[it] when a pixel is flagged for the first time
__global__ void k_clip_flag(ClipArgs c, int it) {
    if (!clip_active(c, it)) return;
    const int64_t n = (int64_t)c.F * c.H * c.W;
    bool fresh = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % c.W);
        const int64_t fy = i / c.W;
        const int f = (int)(fy / c.H), y = (int)(fy - (int64_t)f * c.H);
        const int64_t o = (int64_t)f * c.P + (int64_t)y * c.W + x;
        if (clip_snr(c, o) > c.kappa && !c.flags[o]) {
            c.flags[o] = 1;
            fresh = true;
        }
    }
    if (__syncthreads_or(fresh) && threadIdx.x == 0) atomicOr(c.changed + it, 1u);
}

// Grid (blocks per band, F): S/N of the last iteration, the per-band statistics
// partials (FP32 per thread, FP64 per block), and the candidates: flagged pixels
// with S > 0 that are (2k+1)^2 maxima of X, one record each (band f = trial f).
__global__ void __launch_bounds__(256) k_clip_emit(ClipArgs c, FilterArgs a, int k) {
    const int f = blockIdx.y;
    const int64_t HW = (int64_t)c.H * c.W;
    const int lane = threadIdx.x & 31;
    float s1 = 0.f, s2 = 0.f, cnt = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < HW; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool cand = false;
        int y = 0, x = 0;
        float snr = 0.f;
        if (i < HW) {
            y = (int)(i / c.W);
            x = (int)(i - (int64_t)y * c.W);
            const int64_t o = (int64_t)f * c.P + i;
            const bool valid = c.S[o] > 0.f;
            snr = clip_snr(c, o);
            if (valid) {
                s1 += snr;
                s2 = fmaf(snr, snr, s2);
                cnt += 1.f;
            }
            if (valid && c.flags[o]) {
                const float v = c.X[o];
                const float* plane = c.X + (int64_t)f * c.P;
                cand = true;
                for (int yy = max(y - k, 0); yy <= min(y + k, c.H - 1) && cand; ++yy)
                    for (int xx = max(x - k, 0); xx <= min(x + k, c.W - 1); ++xx)
                        if (plane[(int64_t)yy * c.W + xx] > v) { cand = false; break; }
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (bal) {
            unsigned b0 = 0;
            const int leader = __ffs(bal) - 1;
            if (lane == leader) b0 = atomicAdd(a.counter, (unsigned)__popc(bal));
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (cand) {
                const unsigned idx = b0 + __popc(bal & ((1u << lane) - 1u));
                if (idx < (unsigned)a.cap) {
                    a.keys[idx] = ((uint64_t)a.member_ord[f] << (a.bx + a.by)) | ((uint64_t)y << a.bx) | (uint64_t)x;
                    a.vals[idx] = snr;
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
