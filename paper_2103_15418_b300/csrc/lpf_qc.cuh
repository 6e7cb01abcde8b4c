// Quality control of an incoming image cube before it enters the ring (App. A).
//
//   band test   b_f = mean of band image f; z_f = (b_f - median(b)) / MAD(b),
//               MAD the median absolute deviation from the median; a band with
//               |z_f| > z_thr is discarded.
//   pixel test  running per-pixel mean and sum of squared deviations m2 of the
//               kept band images (Welford); zeta = (x - mean) / s with the
//               sample deviation s = sqrt(m2 / (n - 1)) of the frames before this
//               one, once a band has min_frames frames folded in and where s > 0;
//               a band with any |zeta| > zeta_thr is discarded.
//   imputation  a discarded band image enters the ring as zeros; the kept ones
//               are folded into the running statistics.
//
// Three launches per push: k_qc_scan (band sums, pixel flags), k_qc_decide (one
// warp: median, MAD, mask, counts), k_ingest_qc (ring write + Welford update).
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

constexpr int kQcScanBlocks = 64;      // blocks per band in k_qc_scan

struct QcRecord {                      // per pushed frame, copied to the host with its results
    uint32_t discarded;                // bit f: band f imputed with zeros
    uint32_t pixel_flagged;            // bit f: some |zeta| > zeta_thr in band f
    float z[32];                       // band scores (0 for f >= F)
};

// Grid (kQcScanBlocks, F), 256 threads.  part[f * kQcScanBlocks + b]: the sum of
// block b's pixels of band f (compensated FP32 per thread over a strided share,
// FP64 over the block in a fixed order); bit f of *flags set when a pixel of band f fails
// the pixel test.
__global__ void __launch_bounds__(256) k_qc_scan(const float* __restrict__ frame, int64_t HW,
                                                 const float* __restrict__ mean, const float* __restrict__ m2,
                                                 const int* __restrict__ n, int64_t P, int min_frames,
                                                 float zeta_thr, double* __restrict__ part,
                                                 unsigned* __restrict__ flags) {
    const int f = blockIdx.y;
    const float* x = frame + (int64_t)f * HW;
    const float* mu = mean + (int64_t)f * P;
    const float* sq = m2 + (int64_t)f * P;
    const int nf = n[f];
    const bool test = nf >= min_frames && nf >= 2;
    const float inv_dof = test ? 1.0f / (float)(nf - 1) : 0.f;
    const float z2 = zeta_thr * zeta_thr;
    float acc = 0.f, comp = 0.f;        // compensated (Kahan) FP32 sum of the thread's share
    bool flag = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = __ldg(x + i);
        const float y = v - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
        if (test) {
            const float s2 = __ldg(sq + i) * inv_dof;
            const float d = v - __ldg(mu + i);
            flag |= s2 > 0.f && d * d > z2 * s2;
        }
    }
    double s = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = s;
    if (__syncthreads_or(flag) && threadIdx.x == 0) atomicOr(flags, 1u << f);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
        part[f * gridDim.x + blockIdx.x] = t;
    }
}

// Median of the F values v held by lanes 0..F-1 (ranked by (value, lane)); the
// mean of the two middle values for even F.  Every lane of the warp calls it.
__device__ __forceinline__ double warp_median(double v, int F) {
    const int lane = threadIdx.x & 31;
    int rank = 0;
    for (int g = 0; g < F; ++g) {
        const double u = __shfl_sync(0xffffffffu, v, g);
        rank += (lane < F) && (u < v || (u == v && g < lane));
    }
    const int lo = (F - 1) / 2, hi = F / 2;
    const unsigned blo = __ballot_sync(0xffffffffu, lane < F && rank == lo);
    const unsigned bhi = __ballot_sync(0xffffffffu, lane < F && rank == hi);
    const double a = __shfl_sync(0xffffffffu, v, __ffs(blo) - 1);
    const double b = __shfl_sync(0xffffffffu, v, __ffs(bhi) - 1);
    return lo == hi ? a : 0.5 * (a + b);
}

// One warp: band means, scores, the discard mask, the counts of the kept bands
// and 1/n for their Welford update; the record of this frame; clears *flags.
__global__ void k_qc_decide(const double* __restrict__ part, int F, int64_t HW, float z_thr,
                            unsigned* __restrict__ flags, int* __restrict__ n, float* __restrict__ inv_n,
                            unsigned* __restrict__ mask_out, QcRecord* __restrict__ rec) {
    const int f = threadIdx.x;
    double b = 0.0;
    if (f < F)
        for (int k = 0; k < kQcScanBlocks; ++k) b += part[f * kQcScanBlocks + k];
    b /= (double)HW;
    const double med = warp_median(b, F);
    const double dev = b - med;
    const double mad = warp_median(fabs(dev), F);
    const double z = mad > 0.0 ? dev / mad : (dev == 0.0 ? 0.0 : copysign((double)INFINITY, dev));
    const unsigned pix = *flags;
    const bool discard = f < F && (fabs(z) > (double)z_thr || ((pix >> f) & 1u));
    const unsigned mask = __ballot_sync(0xffffffffu, discard);
    if (f < F) {
        const int nn = n[f] + (discard ? 0 : 1);
        n[f] = nn;
        inv_n[f] = discard ? 0.f : 1.0f / (float)nn;
        rec->z[f] = (float)z;
    } else if (f < 32) {
        rec->z[f] = 0.f;
    }
    if (f == 0) {
        *mask_out = mask;
        rec->discarded = mask;
        rec->pixel_flagged = pix;
        *flags = 0u;
    }
}

// k_ingest with quality control: discarded bands enter the ring as zeros; kept
// bands as stored values, and their pixels are folded into the running
// statistics (Welford, FP32: mean += d / n, m2 += d (x - mean_new)).
template <typename TS>
__global__ void k_ingest_qc(const float* __restrict__ frame, TS* __restrict__ slot, int F, int64_t HW,
                            int64_t P, int vec, const unsigned* __restrict__ mask,
                            const float* __restrict__ inv_n, float* __restrict__ mean,
                            float* __restrict__ m2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned msk = *mask;
    if (vec) {
        const int64_t n4 = HW / 4;
        for (int64_t i = t0; i < (int64_t)F * n4; i += stride) {
            const int64_t f = i / n4, q = i - f * n4;
            const int64_t o = f * P + 4 * q;
            if ((msk >> f) & 1u) {
                st4(slot + o, make_float4(0.f, 0.f, 0.f, 0.f));
                continue;
            }
            const float4 v = __ldg(reinterpret_cast<const float4*>(frame + f * HW) + q);
            st4(slot + o, v);
            const float in = __ldg(inv_n + f);
            float4 m = *reinterpret_cast<float4*>(mean + o);
            float4 s = *reinterpret_cast<float4*>(m2 + o);
            float d;
            d = v.x - m.x; m.x = fmaf(d, in, m.x); s.x = fmaf(d, v.x - m.x, s.x);
            d = v.y - m.y; m.y = fmaf(d, in, m.y); s.y = fmaf(d, v.y - m.y, s.y);
            d = v.z - m.z; m.z = fmaf(d, in, m.z); s.z = fmaf(d, v.z - m.z, s.z);
            d = v.w - m.w; m.w = fmaf(d, in, m.w); s.w = fmaf(d, v.w - m.w, s.w);
            *reinterpret_cast<float4*>(mean + o) = m;
            *reinterpret_cast<float4*>(m2 + o) = s;
        }
    } else {
        for (int64_t i = t0; i < (int64_t)F * HW; i += stride) {
            const int64_t f = i / HW, q = i - f * HW;
            const int64_t o = f * P + q;
            if ((msk >> f) & 1u) {
                st1(slot + o, 0.f);
                continue;
            }
            const float v = __ldg(frame + i);
            st1(slot + o, v);
            const float d = v - mean[o];
            const float mn = fmaf(d, __ldg(inv_n + f), mean[o]);
            mean[o] = mn;
            m2[o] = fmaf(d, v - mn, m2[o]);
        }
    }
}

}  // namespace lpf
