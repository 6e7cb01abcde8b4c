// Device kernels of the image-plane dispersed-transient search (sm_103a).
//
// Data layout in HBM (one stream):
//   ring     [depth][F][P]   storage type TS (float / __half / __nv_bfloat16), P = H*W
//                            rounded up to a multiple of 8 elements; frame T in slot T % depth
//   D        [n_distinct][P] FP32 dedispersed images, one per distinct delay row
//   keys/vals [cand_cap]     unsorted then sorted candidate records (u64 key, f32 snr)
//   out      [cand_cap]      lpf_candidate records of one result slot
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lpf {

constexpr int kTile = 64;             // output tile of the filter kernel (pixels per side)
constexpr int kFilterThreads = 256;
constexpr int kSortBlocks = 148;      // blocks of the candidate-ordering passes

// ------------------------------------------------------------------ storage I/O
__device__ __forceinline__ float4 ld4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const __half* p) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
// acc + *p: a 16-bit value is widened exactly inside the mixed-precision add, so
// the result is the FP32 sum rounded once, as ld1 followed by an FP32 add
__device__ __forceinline__ float add_ld1(const float* p, float acc) { return acc + __ldg(p); }
__device__ __forceinline__ float add_ld1(const __half* p, float acc) {
    float r;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(__half_as_ushort(__ldg(p))), "f"(acc));
    return r;
}
__device__ __forceinline__ float add_ld1(const __nv_bfloat16* p, float acc) {
    float r;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(__bfloat16_as_ushort(__ldg(p))), "f"(acc));
    return r;
}

__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__half* p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
// True when no pixel of the (2k+1)^2 window around (y, x), clipped to the H x W
// image, exceeds v (ties count as maxima, Sec. 2.1.2), reading pixels through
// ld(yy, xx).  The 3x3 ring is tested first: a pixel of a bright region that is
// not its peak usually has a larger neighbour there.
template <typename Ld>
__device__ __forceinline__ bool window_is_max(int y, int x, int k, int H, int W, float v, Ld&& ld) {
    const int k1 = k < 1 ? k : 1;
    for (int yy = max(y - k1, 0); yy <= min(y + k1, H - 1); ++yy)
        for (int xx = max(x - k1, 0); xx <= min(x + k1, W - 1); ++xx)
            if (ld(yy, xx) > v) return false;
    for (int yy = max(y - k, 0); yy <= min(y + k, H - 1); ++yy)
        for (int xx = max(x - k, 0); xx <= min(x + k, W - 1); ++xx)
            if ((yy - y > 1 || y - yy > 1 || xx - x > 1 || x - xx > 1) && ld(yy, xx) > v) return false;
    return true;
}

// v as the storage type TS holds it (round to nearest even, as st1 and st4 store)
template <typename TS> __device__ __forceinline__ float as_stored(float v);
template <> __device__ __forceinline__ float as_stored<float>(float v) { return v; }
template <> __device__ __forceinline__ float as_stored<__half>(float v) { return __half2float(__float2half_rn(v)); }
template <> __device__ __forceinline__ float as_stored<__nv_bfloat16>(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// ------------------------------------------------------------------ a2: ingest
// Convert frame [F][HW] (FP32, caller layout) into ring slot [F][P] (storage type,
// round to nearest even).  vec: frame pointer 16-B aligned and HW % 4 == 0.
template <typename TS>
__global__ void k_ingest(const float* __restrict__ frame, TS* __restrict__ slot, int F,
                         int64_t HW, int64_t P, int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const int64_t n4 = HW / 4;
        for (int64_t i = t0; i < (int64_t)F * n4; i += stride) {
            int64_t f = i / n4, q = i - f * n4;
            float4 v = __ldg(reinterpret_cast<const float4*>(frame + f * HW) + q);
            st4(slot + f * P + 4 * q, v);
        }
    } else {
        for (int64_t i = t0; i < (int64_t)F * HW; i += stride) {
            int64_t f = i / HW, q = i - f * HW;
            st1(slot + f * P + q, __ldg(frame + i));
        }
    }
}

// ------------------------------------------------------------------ a4-a6: filter + detect
// Window sum along a line without cancellation ("two stacks"): outputs
// j in [j0, j0 + R) of out[j] = sum_{k=0..2r} in[(j + k) * is], R <= 2r + 1.
// Every window contains the pivot m = j0 + 2r, so out[j] = SUF(j) + PRE(j + 2r)
// with SUF(a) = sum_{k=a}^{m-1} in[k] and PRE(b) = sum_{k=m}^{b} in[k]: each
// output is a sum of two sums of consecutive inputs, never a difference.
template <int RMAX, typename Epi>
__device__ __forceinline__ void window_run(const float* __restrict__ in, int is, int j0, int R,
                                           int r, Epi&& epi) {
    float suf[2 * RMAX + 1];
    float acc = 0.f;
#pragma unroll
    for (int i = 2 * RMAX; i >= 0; --i) {
        if (i < 2 * r) acc += in[(j0 + i) * is];
        if (i < R) suf[i] = acc;
    }
    float pre = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * RMAX + 1; ++i) {
        if (i < R) {
            pre += in[(j0 + 2 * r + i) * is];
            epi(j0 + i, suf[i] + pre);
        }
    }
}

__device__ __forceinline__ int clipped_count(int c, int r, int n) {
    return min(c + r, n - 1) - max(c - r, 0) + 1;
}

struct FilterArgs {
    const float* D;        // [n_rows][P]
    int64_t P;
    int H, W, r;
    float kappa;
    int tiles_x, tiles_y;
    const int* member_start;   // [n_distinct + 1]
    const int* member_ord;     // canonical (t0, d) rank of each member trial
    uint64_t* keys;
    float* vals;
    unsigned* counter;
    int cap;
    int bx, by;            // bits of x and y in the key
    double* partials;      // [n_rows][tiles][3]
    unsigned* zbits = nullptr;  // steady-source marks (null: off): one bit per key pixel y << bx | x
    int zrow = -1;              // the delay row that is all zero (no dispersion), -1 if none
};

// Steady-source marks: a candidate of the all-zero delay row sets its pixel's
// bit as it is found, whether or not its records fit the candidate list.
__device__ __forceinline__ void mark_zero_row(const FilterArgs& a, int row, uint64_t pix) {
    if (a.zbits != nullptr && row == a.zrow) atomicOr(&a.zbits[pix >> 5], 1u << (pix & 31));
}

__device__ __forceinline__ int odd_stride(int n) { return n | 1; }

// One CTA: one distinct delay row (blockIdx.y) x one 64x64 output tile.
// Shared memory (FP32): D region (64+4r)^2, horizontal sums of D, C and E on
// (64+2r)^2, horizontal sums of E.  E and the sums are zero outside the image,
// so every window is clipped to the image; C and S divide by the in-image count.
template <int RMAX>
__global__ void __launch_bounds__(kFilterThreads, 1) k_filter(FilterArgs a) {
    extern __shared__ float sm[];
    const int r = a.r;
    const int RY = kTile + 4 * r, RX = RY;
    const int nC = kTile + 2 * r;
    const int sD = odd_stride(RX), sA = odd_stride(nC), sC = odd_stride(nC), sB = odd_stride(kTile);
    float* bufD = sm;                    // [RY][sD]
    float* bufA = bufD + RY * sD;        // [RY][sA]  horizontal sums of D
    float* bufC = bufA + RY * sA;        // [nC][sC]  C
    float* bufE = bufC + nC * sC;        // [nC][sC]  E = (D - C)^2
    float* bufB = bufE + nC * sC;        // [nC][sB]  horizontal sums of E

    const int tile = blockIdx.x;
    const int row = blockIdx.y;
    const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
    const int y0 = ty * kTile, x0 = tx * kTile;
    const int H = a.H, W = a.W;
    const float* Dimg = a.D + (int64_t)row * a.P;
    const int tid = threadIdx.x;

    // 1. D region with a 2r halo, zero outside the image
    for (int idx = tid; idx < RY * RX; idx += blockDim.x) {
        int i = idx / RX, j = idx - i * RX;
        int gy = y0 - 2 * r + i, gx = x0 - 2 * r + j;
        float v = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = __ldg(Dimg + (int64_t)gy * W + gx);
        bufD[i * sD + j] = v;
    }
    __syncthreads();

    // 2. horizontal window sums of D: bufA[i][c], c <-> gx = x0 - r + c
    {
        const int nrun = (nC + 2 * r) / (2 * r + 1);
        const int R = (nC + nrun - 1) / nrun;
        for (int it = tid; it < RY * nrun; it += blockDim.x) {
            int i = it % RY, run = it / RY;
            int j0 = run * R, len = min(R, nC - j0);
            float* out = bufA + i * sA;
            window_run<RMAX>(bufD + i * sD, 1, j0, len, r, [&](int j, float s) { out[j] = s; });
        }
    }
    __syncthreads();

    // 3. vertical sums -> C, then E = (D - C)^2 on the (64+2r)^2 region
    {
        const int nrun = (nC + 2 * r) / (2 * r + 1);
        const int R = (nC + nrun - 1) / nrun;
        for (int it = tid; it < nC * nrun; it += blockDim.x) {
            int c = it % nC, run = it / nC;
            int j0 = run * R, len = min(R, nC - j0);
            int gx = x0 - r + c;
            bool xin = gx >= 0 && gx < W;
            int nx = xin ? clipped_count(gx, r, W) : 1;
            window_run<RMAX>(bufA + c, sA, j0, len, r, [&](int i2, float s) {
                int gy = y0 - r + i2;
                float Cv = 0.f, Ev = 0.f;
                if (xin && gy >= 0 && gy < H) {
                    Cv = s / (float)(clipped_count(gy, r, H) * nx);
                    float dv = bufD[(i2 + r) * sD + (c + r)] - Cv;
                    Ev = dv * dv;
                }
                bufC[i2 * sC + c] = Cv;
                bufE[i2 * sC + c] = Ev;
            });
        }
    }
    __syncthreads();

    // 4. horizontal sums of E: bufB[i2][j], j <-> gx = x0 + j
    {
        const int nrun = (kTile + 2 * r) / (2 * r + 1);
        const int R = (kTile + nrun - 1) / nrun;
        for (int it = tid; it < nC * nrun; it += blockDim.x) {
            int i2 = it % nC, run = it / nC;
            int j0 = run * R, len = min(R, kTile - j0);
            float* out = bufB + i2 * sB;
            window_run<RMAX>(bufE + i2 * sC, 1, j0, len, r, [&](int j, float s) { out[j] = s; });
        }
    }
    __syncthreads();

    // 5. vertical sums -> S, then snr, threshold, 3x3 local maximum, stats, emission
    float s1 = 0.f, s2 = 0.f;
    int cnt = 0;
    const int m0 = a.member_start[row], nm = a.member_start[row + 1] - m0;
    {
        const int nrun = (kTile + 2 * r) / (2 * r + 1);
        const int R = (kTile + nrun - 1) / nrun;
        const int nitems = kTile * nrun;
        const int nloop = (nitems + blockDim.x - 1) / blockDim.x;
        for (int l = 0; l < nloop; ++l) {
            int it = l * blockDim.x + tid;
            bool has = it < nitems;
            int j = has ? it % kTile : 0, run = has ? it / kTile : 0;
            int j0 = run * R, len = has ? min(R, kTile - j0) : 0;
            int x = x0 + j;
            bool xin = has && x < W;
            int nx = xin ? clipped_count(x, r, W) : 1;
            // all lanes iterate the same count so warp-wide ballots stay converged
            window_run<RMAX>(bufB + j, sB, j0, R, r, [&](int i, float s) {
                int y = y0 + i;
                bool in = xin && (i - j0) < len && y < H;
                bool cand = false;
                float snr = 0.f;
                if (in) {
                    float Sv = s / (float)(clipped_count(y, r, H) * nx);
                    float dv = bufD[(i + 2 * r) * sD + (j + 2 * r)];
                    float cv = bufC[(i + r) * sC + (j + r)];
                    if (Sv > 0.f) {
                        snr = (dv - cv) * rsqrtf(Sv);
                        s1 += snr;
                        s2 += snr * snr;
                        cnt += 1;
                        if (snr > a.kappa) {
                            bool mx = true;
#pragma unroll
                            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    if (dy == 0 && dx == 0) continue;
                                    int yy = y + dy, xx = x + dx;
                                    if (yy >= 0 && yy < H && xx >= 0 && xx < W &&
                                        bufD[(i + 2 * r + dy) * sD + (j + 2 * r + dx)] > dv)
                                        mx = false;
                                }
                            cand = mx;
                        }
                    }
                }
                unsigned act = __activemask();
                unsigned bal = __ballot_sync(act, cand);
                if (bal) {
                    int lane = threadIdx.x & 31;
                    int leader = __ffs(bal) - 1;
                    unsigned base = 0;
                    if (lane == leader) base = atomicAdd(a.counter, (unsigned)(__popc(bal) * nm));
                    base = __shfl_sync(act, base, leader);
                    if (cand) {
                        unsigned rank = __popc(bal & ((1u << lane) - 1u));
                        uint64_t pix = ((uint64_t)y << a.bx) | (uint64_t)x;
                        mark_zero_row(a, row, pix);
                        for (int m = 0; m < nm; ++m) {
                            unsigned idx = base + rank * nm + m;
                            if (idx < (unsigned)a.cap) {
                                a.keys[idx] = ((uint64_t)a.member_ord[m0 + m] << (a.bx + a.by)) | pix;
                                a.vals[idx] = snr;
                            }
                        }
                    }
                }
            });
        }
    }

    // 6. per-CTA stats partials in FP64 (fixed reduction order)
    double d1 = s1, d2 = s2, dc = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        dc += __shfl_down_sync(0xffffffffu, dc, o);
    }
    __shared__ double red[kFilterThreads / 32][3];
    int w = tid >> 5;
    if ((tid & 31) == 0) { red[w][0] = d1; red[w][1] = d2; red[w][2] = dc; }
    __syncthreads();
    if (tid == 0) {
        double t1 = 0, t2 = 0, tc = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t1 += red[k][0]; t2 += red[k][1]; tc += red[k][2]; }
        double* p = a.partials + ((int64_t)row * (a.tiles_x * a.tiles_y) + tile) * 3;
        p[0] = t1; p[1] = t2; p[2] = tc;
    }
}

// ------------------------------------------------------------------ a7: stats
// stats[r] = (sum snr, sum snr^2, count) over the tiles of row r, fixed order.
__global__ void k_stats(const double* __restrict__ partials, int n_tiles, double* __restrict__ stats) {
    const int row = blockIdx.x;
    __shared__ double red[3][256];
    double t[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < n_tiles; i += blockDim.x)
        for (int k = 0; k < 3; ++k) t[k] += partials[((int64_t)row * n_tiles + i) * 3 + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = t[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) stats[row * 3 + k] = red[k][0];
}

// ------------------------------------------------------------------ output records
struct CandidateRec {   // mirrors lpf_candidate (24 bytes)
    int64_t t0;
    int32_t dm_idx, y, x;
    float snr;
};

__global__ void k_zero_u32(unsigned* p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0u;
}

// ------------------------------------------------------------------ a8: dynspec gather
// out[i][f][tau] = X_f(T - Tw + 1 + tau) at (y_i, x_i) (max over the clipped box).
template <typename TS>
__global__ void k_dynspec(const TS* __restrict__ ring, const int2* __restrict__ yx, int n, int F,
                          int Tw, int depth, int slot_first, int64_t P, int H, int W, int box_r,
                          float* __restrict__ out) {
    const int64_t total = (int64_t)n * F * Tw;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int tau = (int)(idx % Tw);
        int64_t rest = idx / Tw;
        int f = (int)(rest % F);
        int i = (int)(rest / F);
        int slot = slot_first + tau;
        if (slot >= depth) slot -= depth;
        const TS* plane = ring + ((int64_t)slot * F + f) * P;
        int2 c = yx[i];
        float v;
        if (box_r == 0) {
            v = ld1(plane + (int64_t)c.x * W + c.y);
        } else {
            v = -INFINITY;
            int ylo = max(c.x - box_r, 0), yhi = min(c.x + box_r, H - 1);
            int xlo = max(c.y - box_r, 0), xhi = min(c.y + box_r, W - 1);
            for (int yy = ylo; yy <= yhi; ++yy)
                for (int xx = xlo; xx <= xhi; ++xx) v = fmaxf(v, ld1(plane + (int64_t)yy * W + xx));
        }
        out[idx] = v;
    }
}

}  // namespace lpf
