// Residual path: the box filter moved in front of the shift-sum.
//
// The local centre is linear in the image and the shift-sum only moves whole
// planes in time, so for every DM trial d and pixel p (Sec. 2.1.1, App. B.2)
//   C_d(p) = (1/n_p) sum_{q in W(p)} sum_f X_f(t_f)(q) = sum_f C(X_f(t_f))(p)
//   D_d(p) - C_d(p) = sum_f [X_f(t_f) - C(X_f(t_f))](p) = sum_f Xr_f(t_f)(p),
// with the same clipped window W(p) and count n_p for every plane.  So:
//   k_residual   once per frame and subband: Xr = X - C(X) into a residual ring
//   k_dedisperse over the residual ring gives R_d = D_d - C_d per distinct row
//   k_dedisperse over the raw ring gives D_d, read only at candidate windows
//   k_filter_res S_d = box mean of R_d^2, snr = R_d / sqrt(S_d), threshold,
//                stats, crossing list (lpf_filter_res.cuh)
//   k_lmax_res   3x3 local maximum of D_d at the crossings, emission.
// One box filter per trial instead of two, with a halo of r instead of 2r.
#pragma once
#include "lpf_filter_stream.cuh"

namespace lpf {

// 1/sqrt(x) for a normal FP32 x (x >= 2^-126): the approximate reciprocal
// square root instruction, whose relative error is a few units in the last
// place; no subnormal handling is needed on that range.
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int R>
struct ResGeom {
    static constexpr int TX = 128;
    static constexpr int L = 2 * R + 1;
    static constexpr int NP = 32 / L;
    static constexpr int B = NP * L;                 // rows per block
    static constexpr int WD = TX + 2 * R;             // columns carrying the input of one box pass
    static constexpr int SD = WD | 1;
    static constexpr int SX = TX | 1;
    static constexpr int NR = (TX + L - 1) / L;       // horizontal runs per row
    static constexpr int RR = (TX + NR - 1) / NR;
    static constexpr int NT = 160;
    static_assert(WD <= NT, "one thread per loaded column");
    static_assert(NT - TX == 32, "one copy warp beside the column warps");
};

// ---------------------------------------------------------------------------
// k_residual: Xr = X - C(X) for the F planes of one ring slot, C the clipped box
// mean of radius R (horizontal two-stack sums, vertical sliding sum, C by
// reciprocal plus one Newton step against the exact count, so a constant
// window gives Xr = 0 exactly).  X is read from the pushed frame [F][H][W]
// (FP32) and rounded to the storage type TS, the value the raw ring holds; a
// band whose bit is set in *drop (quality control) is all zeros.  Xr is written
// in the storage type.  Grid: (strips, F, row segments); a segment of seg_rows
// output rows streams from r rows above it (its vertical window starts there)
// to r rows below it.
template <int R, typename TS>
__global__ void __launch_bounds__(ResGeom<R>::NT) k_residual(const float* __restrict__ frame,
                                                             const unsigned* __restrict__ drop,
                                                             TS* __restrict__ res_slot, int H, int W,
                                                             int64_t P, int seg_rows) {
    using G = ResGeom<R>;
    constexpr int TX = G::TX, B = G::B, L = G::L, SD = G::SD, SX = G::SX, WD = G::WD;
    extern __shared__ float smr[];
    float(*Xb)[B][SD] = reinterpret_cast<float(*)[B][SD]>(smr);        // [2][B][SD] this and the previous block
    float(*hX)[SX] = reinterpret_cast<float(*)[SX]>(smr + 2 * B * SD);  // [B][SX]
    __shared__ float2 rowC[B];
    const int strip = blockIdx.x, f = blockIdx.y;
    const int x0 = strip * TX;
    const float* X = frame + (int64_t)f * H * W;
    TS* Xr = res_slot + (int64_t)f * P;
    const int t = threadIdx.x;
    const int xl = x0 - R + t;                  // loaded column of this thread
    const bool lcol = t < WD && xl >= 0 && xl < W && !(drop && ((*drop >> f) & 1u));
    const int xs = x0 + t;                      // output column of this thread
    const bool ocol = t < TX && xs < W;
    const int nx = ocol ? min(xs + R, W - 1) - max(xs - R, 0) + 1 : 0;
    const float nxf = (float)nx, inv_nx = ocol ? 1.0f / nxf : 0.f;
    float hist[L];
#pragma unroll
    for (int i = 0; i < L; ++i) hist[i] = 0.f;
    float v = 0.f;
    const int y0 = blockIdx.z * seg_rows, y1 = min(H, y0 + seg_rows);
    const int ys0 = max(0, y0 - R);             // first input row
    const int nblk = (y1 + R - ys0 + B - 1) / B;
    for (int k = 0; k < nblk; ++k) {
        const int ybase = ys0 + k * B;
        float(*cur)[SD] = Xb[k & 1];
        float(*prev)[SD] = Xb[(k + 1) & 1];
        if (t < WD) {
            // every load of the block first, then the rounding to the storage type:
            // all B loads are in flight at once for any TS
            const float* src = X + (int64_t)ybase * W + xl;
            float xv[B];
#pragma unroll
            for (int j = 0; j < B; ++j) xv[j] = (lcol && ybase + j < H) ? __ldg(src + (int64_t)j * W) : 0.f;
#pragma unroll
            for (int j = 0; j < B; ++j) cur[j][t] = as_stored<TS>(xv[j]);
        }
        if (t < B) rowC[t] = row_count<R>(ybase + t - R, H);
        __syncthreads();
        for (int it = t; it < B * G::NR; it += G::NT) {
            int j = it % B, run = it / B;
            int c0 = run * G::RR;
            int len = min(G::RR, TX - c0);
            const float* in = cur[j];
            float* out = hX[j];
            two_stack_run<R, G::RR>(c0, len, [&](int c) { return in[c]; },
                                    [&](int c, float val) { out[c] = val; });
        }
        __syncthreads();
        if (t < TX) {
#pragma unroll
            for (int j = 0; j < B; ++j) {
                float in = hX[j][t];
                float out = hist[j % L];
                hist[j % L] = in;
                v += in - out;
                const int yc = ybase + j - R;
                const float2 cy = rowC[j];
                const float n = cy.x * nxf, inv = cy.y * inv_nx;
                if (n > 0.f && yc >= y0 && yc < y1) {
                    const float c0 = v * inv;
                    const float C = fmaf(fmaf(-c0, n, v), inv, c0);
                    const float xv = (j >= R) ? cur[j - R][t + R] : prev[B + j - R][t + R];
                    st1(Xr + (int64_t)yc * W + xs, xv - C);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
struct ResArgs {
    FilterArgs a;            // R = D - C images in a.D, emission, stats
    const void* ring;        // raw ring [depth][F][P] (storage type), for D at 3x3 windows
    const int16_t* lag;      // [n_rows][F] frames back from the newest frame (slot Tmod)
    int F, depth, Tmod;
    uint64_t* xkeys;         // [xcap] threshold crossings (row << 32 | y << 16 | x) ...
    float* xvals;            // ... and their S/N
    unsigned long long* xcounter;   // crossings reserved (may exceed xcap)
    int64_t xcap;            // crossing list capacity
    int band_k;              // per-subband detector: local-maximum radius k on X_row (0: dispersed search)
};

// a crossing slot reserved by a warp that resolved its crossings itself
constexpr uint64_t kNoCrossing = ~0ull;

// D = sum_f X_f(t_f) of a delay row at a pixel is summed from the raw ring in
// the order f = 0 .. F-1 in FP32 (the arithmetic of the shift-sum, so the same
// values); -inf outside the image.  d_window3_lean: the 3x3 window one pixel at
// a time (few registers: the in-kernel resolution of an overflowing crossing
// list).
template <typename TS>
__device__ __forceinline__ void d_window3_lean(const ResArgs& ra, int row, int ys, int xs, float nb[9]) {
    const FilterArgs& a = ra.a;
    const TS* ring = static_cast<const TS*>(ra.ring);
    const int16_t* lr = ra.lag + (int64_t)row * ra.F;
#pragma unroll 1
    for (int k = 0; k < 9; ++k) {
        const int yy = ys + k / 3 - 1, xx = xs + k % 3 - 1;
        float v = -INFINITY;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
            const int64_t off = (int64_t)yy * a.W + xx;
#pragma unroll 1
            for (int f = 0; f < ra.F; ++f) {
                int slot = ra.Tmod - (int)__ldg(lr + f);
                if (slot < 0) slot += ra.depth;
                const float x = ld1(ring + ((int64_t)slot * ra.F + f) * a.P + off);
                v = (f == 0) ? x : v + x;
            }
        }
        nb[k] = v;
    }
}

// Sums D = sum_f X_f(t_f) (FP32, f = 0 .. F-1, as the shift-sum) at the NK
// pixels (ys + dy[k], xs + dx[k]) from the raw ring; -inf outside the image.
template <typename TS, int NK>
__device__ __forceinline__ void d_points(const ResArgs& ra, int row, int ys, int xs, const int (&dy)[NK],
                                         const int (&dx)[NK], float (&v)[NK]) {
    const FilterArgs& a = ra.a;
    const TS* ring = static_cast<const TS*>(ra.ring);
    const int16_t* lr = ra.lag + (int64_t)row * ra.F;
    int64_t off[NK];
    bool in[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int yy = ys + dy[k], xx = xs + dx[k];
        in[k] = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        off[k] = in[k] ? (int64_t)yy * a.W + xx : 0;
    }
    // unrolled by 4: the loads of four subbands are in flight together (the sum
    // still runs f = 0, 1, ... in order)
#pragma unroll 4
    for (int f = 0; f < ra.F; ++f) {
        int slot = ra.Tmod - (int)__ldg(lr + f);
        if (slot < 0) slot += ra.depth;
        const TS* plane = ring + ((int64_t)slot * ra.F + f) * a.P;
        // a point outside the image reads the plane's first value (off = 0); its
        // sum is replaced by -inf below
#pragma unroll
        for (int k = 0; k < NK; ++k) v[k] = (f == 0) ? ld1(plane + off[k]) : add_ld1(plane + off[k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < NK; ++k)
        if (!in[k]) v[k] = -INFINITY;
}

// Whether D(ys, xs) is the maximum of its 3x3 window clipped to the image (ties
// count), with the same D values as d_window3: the centre and its four edge
// neighbours first, the four diagonal ones only if none of those is larger
// (most crossings of a source's clump have a larger edge neighbour).
template <typename TS>
__device__ __forceinline__ bool d_is_max3(const ResArgs& ra, int row, int ys, int xs) {
    constexpr int ey[5] = {0, -1, 1, 0, 0}, ex[5] = {0, 0, 0, -1, 1};
    float v[5];
    d_points<TS, 5>(ra, row, ys, xs, ey, ex, v);
    if (v[1] > v[0] || v[2] > v[0] || v[3] > v[0] || v[4] > v[0]) return false;
    constexpr int gy[4] = {-1, -1, 1, 1}, gx[4] = {-1, 1, -1, 1};
    float g[4];
    d_points<TS, 4>(ra, row, ys, xs, gy, gx, g);
    return !(g[0] > v[0] || g[1] > v[0] || g[2] > v[0] || g[3] > v[0]);
}

// Per-subband detector: whether X_f(y, x) of the newest frame (ring slot Tmod,
// band f = row) is the maximum of its (2k+1)^2 window clipped to the image
// (ties count).
template <typename TS>
__device__ __forceinline__ bool band_is_max(const ResArgs& ra, int row, int ys, int xs) {
    const FilterArgs& a = ra.a;
    const TS* plane = static_cast<const TS*>(ra.ring) + ((int64_t)ra.Tmod * ra.F + row) * a.P;
    const float c = ld1(plane + (int64_t)ys * a.W + xs);
    return window_is_max(ys, xs, ra.band_k, a.H, a.W, c,
                         [&](int yy, int xx) { return ld1(plane + (int64_t)yy * a.W + xx); });
}

// Candidates of one image row of a warp (lanes with cand set): the 3x3 local
// maximum of D clipped to the image (ties count); then one warp-aggregated
// reservation and one record per DM trial of the delay row.  Every lane of the
// warp calls it.
template <typename TS>
__device__ __noinline__ void emit_res_candidates(const ResArgs& ra, int row, int ys, int xs, float snr,
                                                 bool cand, int m0, int nm) {
    const FilterArgs& a = ra.a;
    const int lane = threadIdx.x & 31;
    if (cand && ra.band_k > 0) {
        cand = band_is_max<TS>(ra, row, ys, xs);
    } else if (cand) {
        float nb[9];
        d_window3_lean<TS>(ra, row, ys, xs, nb);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (k != 4 && nb[k] > nb[4]) cand = false;
    }
    unsigned bal = __ballot_sync(0xffffffffu, cand);
    if (!bal) return;
    int leader = __ffs(bal) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(a.counter, (unsigned)(__popc(bal) * nm));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cand) {
        unsigned rank = __popc(bal & ((1u << lane) - 1u));
        uint64_t pix = ((uint64_t)ys << a.bx) | (uint64_t)xs;
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

// k_lmax_res: the 3x3 local maximum of D (clipped to the image, ties count) at
// every crossing of the list, one thread per crossing, D summed from the raw
// ring on the window; one candidate record per DM trial of a maximum's delay
// row (warp-aggregated reservations).  BAND: the per-subband detector, the
// (2k+1)^2 maximum of the band image X_row of the newest frame.
template <typename TS, bool BAND>
__global__ void __launch_bounds__(256) k_lmax_res(ResArgs ra) {
    const FilterArgs& a = ra.a;
    const unsigned long long nres = *ra.xcounter;
    const unsigned long long n = nres < (unsigned long long)ra.xcap ? nres : (unsigned long long)ra.xcap;
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = gridDim.x * (blockDim.x >> 5);
    const unsigned long long gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (unsigned long long i0 = gw * 32u; i0 < n; i0 += nwarps * 32u) {
        const unsigned long long i = i0 + lane;
        bool cand = false;
        int row = 0, ys = 0, xs = 0;
        float snr = 0.f;
        if (i < n) {
            const uint64_t key = ra.xkeys[i];
            if (key != kNoCrossing) {
                row = (int)(key >> 32);
                ys = (int)((key >> 16) & 0xffffu);
                xs = (int)(key & 0xffffu);
                snr = ra.xvals[i];
                if constexpr (BAND) {
                    cand = band_is_max<TS>(ra, row, ys, xs);
                } else {
                    cand = d_is_max3<TS>(ra, row, ys, xs);
                }
            }
        }
        const int m0 = cand ? a.member_start[row] : 0;
        const unsigned nm = cand ? (unsigned)(a.member_start[row + 1] - m0) : 0u;
        unsigned incl = nm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) continue;
        unsigned base = 0;
        if (lane == 31) base = atomicAdd(a.counter, total);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (cand) {
            const uint64_t pix = ((uint64_t)ys << a.bx) | (uint64_t)xs;
            mark_zero_row(a, row, pix);
            for (unsigned m = 0; m < nm; ++m) {
                const unsigned idx = base + incl - nm + m;
                if (idx < (unsigned)a.cap) {
                    a.keys[idx] = ((uint64_t)a.member_ord[m0 + m] << (a.bx + a.by)) | pix;
                    a.vals[idx] = snr;
                }
            }
        }
    }
}

template <int R>
constexpr size_t residual_smem_bytes() {
    return ((size_t)2 * ResGeom<R>::B * ResGeom<R>::SD + (size_t)ResGeom<R>::B * ResGeom<R>::SX) * sizeof(float);
}


}  // namespace lpf

namespace lpf {

// Per-subband detector with a 16-bit ring: the residual planes X_f - C(X_f) of
// the newest frame widened to FP32 (the images the filter reads).
template <typename TS>
__global__ void k_band_planes(const TS* __restrict__ res_slot, float* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = ld1(res_slot + i);
}

}  // namespace lpf
