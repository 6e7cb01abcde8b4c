// Candidate ordering (sm_103a): the records of a push sorted by (t0, d, y, x)
// and written out as lpf_candidate records.
//
// A record's key is (rank << (bx + by)) | (y << bx) | x, where rank is the
// canonical trial rank (t0 ascending, then d), so the output order is the key
// order.  Within one rank every pixel occurs at most once, so the keys of a
// rank are distinct and any correct sort gives the same order.  The ordering
// is a counting sort on the rank followed by one block-level sort per rank:
//   k_ord_count    records per rank (shared-memory histograms)
//   k_ord_scan     exclusive scan of the counts -> bucket starts (one block);
//                  the counts are cleared for the lane's next use
//   k_ord_scatter  every record into its rank's bucket (warp-aggregated cursor
//                  reservations; order inside a bucket arbitrary)
//   k_ord_sort_format  one block per bucket: bitonic sort of the bucket's
//                  keys (shared memory up to kOrdCap records, global memory
//                  above), then the records, formatted (t0, d, y, x, snr)
#pragma once
#include "lpf_kernels.cuh"

namespace lpf {

constexpr int kOrdThreads = 256;
constexpr uint64_t kDropped = ~0ull;  // a record dropped by the steady-source mask (skipped below)
constexpr int kOrdHist = 4096;      // ranks counted in shared memory (more: global atomics)
constexpr int kOrdCap = 4096;       // bucket size sorted in shared memory

__global__ void __launch_bounds__(kOrdThreads) k_ord_count(const uint64_t* __restrict__ keys,
                                                           const unsigned* __restrict__ n_ptr, int cap,
                                                           int shift, int n_ord, unsigned* __restrict__ counts) {
    __shared__ unsigned h[kOrdHist];
    const bool local = n_ord <= kOrdHist;
    if (local)
        for (int i = threadIdx.x; i < n_ord; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const unsigned n = min(*n_ptr, (unsigned)cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        if (key == kDropped) continue;
        const unsigned r = (unsigned)(key >> shift);
        if (local) atomicAdd(&h[r], 1u);
        else atomicAdd(&counts[r], 1u);
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < n_ord; i += blockDim.x)
            if (h[i]) atomicAdd(&counts[i], h[i]);
}

// start[r] = cursor[r] = sum of counts below r; counts cleared.  One block of
// 1024 threads, each owning a run of consecutive ranks.
__global__ void __launch_bounds__(1024) k_ord_scan(unsigned* __restrict__ counts, int n_ord,
                                                   unsigned* __restrict__ start, unsigned* __restrict__ cursor) {
    __shared__ unsigned wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n_ord + 1023) / 1024;
    const int r0 = min(n_ord, t * per), r1 = min(n_ord, r0 + per);
    unsigned own = 0;
    for (int r = r0; r < r1; ++r) own += counts[r];
    unsigned inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    unsigned run = wsum[warp] + inc - own;
    for (int r = r0; r < r1; ++r) {
        const unsigned c = counts[r];
        start[r] = run;
        cursor[r] = run;
        counts[r] = 0u;
        run += c;
    }
}

// Every record into its rank's bucket.  The loop runs in whole tiles of the
// grid so that every lane of a warp takes part in the match; lanes past the end
// carry an impossible rank.
__global__ void __launch_bounds__(kOrdThreads) k_ord_scatter(const uint64_t* __restrict__ kin,
                                                             const float* __restrict__ vin,
                                                             const unsigned* __restrict__ n_ptr, int cap, int shift,
                                                             unsigned* __restrict__ cursor,
                                                             uint64_t* __restrict__ kout, float* __restrict__ vout) {
    const unsigned n = min(*n_ptr, (unsigned)cap);
    const int lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const unsigned i = i0 + threadIdx.x;
        const uint64_t key = i < n ? kin[i] : kDropped;
        const bool valid = key != kDropped;
        const unsigned r = valid ? (unsigned)(key >> shift) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (valid && lane == leader) base = atomicAdd(&cursor[r], (unsigned)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) {
            const unsigned pos = base + __popc(peers & ((1u << lane) - 1u));
            kout[pos] = key;
            vout[pos] = vin[i];
        }
    }
}

// Bitonic sorting network of N = 2^p >= m elements with every comparator
// ascending (min to the lower index): in the merge of blocks of size k the
// first step compares i with its mirror i ^ (k - 1), the later steps i with
// i + j.  Elements at or past m act as +infinity: a comparator whose upper
// index is >= m is skipped, so no padding is stored.  cmpswap(i, l) orders one
// pair (shared or global memory); sync separates the steps.
template <typename Cmp, typename Sync>
__device__ __forceinline__ void bitonic_network(unsigned m, Cmp&& cmpswap, Sync&& sync) {
    unsigned N = 2;
    while (N < m) N <<= 1;
    for (unsigned k = 2; k <= N; k <<= 1) {
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
                const unsigned i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                const unsigned l = (j == (k >> 1)) ? (i ^ (k - 1)) : (i + j);
                if (l < m) cmpswap(i, l);
            }
            sync();
        }
    }
}

__global__ void __launch_bounds__(kOrdThreads) k_ord_sort_format(
    uint64_t* __restrict__ kin, float* __restrict__ vin, const unsigned* __restrict__ start,
    const unsigned* __restrict__ cursor, int n_ord, CandidateRec* __restrict__ out,
    const int* __restrict__ ord2d, const int* __restrict__ dmax_of_d, int64_t T, int bx, int by) {
    extern __shared__ __align__(16) unsigned char ord_sm[];
    uint64_t* sk = reinterpret_cast<uint64_t*>(ord_sm);             // [kOrdCap]
    float* sv = reinterpret_cast<float*>(sk + kOrdCap);              // [kOrdCap]
    for (int r = blockIdx.x; r < n_ord; r += gridDim.x) {
        const unsigned s0 = start[r], m = cursor[r] - s0;
        if (m == 0) continue;
        const int d = ord2d[r];
        const int64_t t0 = T - dmax_of_d[d];
        const uint64_t xm = (1ull << bx) - 1, ym = (1ull << by) - 1;
        auto emit = [&](unsigned i, uint64_t k, float v) {
            CandidateRec c;
            c.t0 = t0;
            c.dm_idx = d;
            c.y = (int)((k >> bx) & ym);
            c.x = (int)(k & xm);
            c.snr = v;
            out[s0 + i] = c;
        };
        if (m <= (unsigned)kOrdCap) {
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) {
                sk[i] = kin[s0 + i];
                sv[i] = vin[s0 + i];
            }
            __syncthreads();
            bitonic_network(m, [&](unsigned i, unsigned l) {
                const uint64_t a = sk[i], b = sk[l];
                if (b < a) {
                    sk[i] = b; sk[l] = a;
                    const float va = sv[i];
                    sv[i] = sv[l]; sv[l] = va;
                }
            }, [] { __syncthreads(); });
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) emit(i, sk[i], sv[i]);
        } else {
            // a bucket larger than shared memory: the same network in place in global
            // memory (rare: a trial with more than kOrdCap candidates)
            uint64_t* gk = kin + s0;
            float* gv = vin + s0;
            bitonic_network(m, [&](unsigned i, unsigned l) {
                const uint64_t a = gk[i], b = gk[l];
                if (b < a) {
                    gk[i] = b; gk[l] = a;
                    const float va = gv[i];
                    gv[i] = gv[l]; gv[l] = va;
                }
            }, [] { __threadfence_block(); __syncthreads(); });
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) emit(i, gk[i], gv[i]);
        }
        __syncthreads();
    }
}

constexpr size_t ord_sort_smem_bytes() { return (size_t)kOrdCap * (sizeof(uint64_t) + sizeof(float)); }

// ---------------------------------------------------------------------------
// Opt-in steady-source suppression (between the 3x3 pass and the ordering; see
// suppress_steady in lpf.h).  Pixels are indexed by the key's low bits (y << bx
// | x), so the per-pixel state has 2^shift entries.  The kernels that find the
// candidates set the bit of every pixel with a candidate of the all-zero delay
// row of the push (mark_zero_row), stored in the list or not; then
//   k_steady_update  run[p] = bit ? min(run[p] + 1, 255) : 0: the pushes in a
//                    row with such a candidate, in push order (tail stream);
//                    each word of the bit map is cleared once its warp has read
//                    it, ready for the lane's next push
//   k_steady_apply   records of the other trials at pixels with run >= K get
//                    the key kDropped (the ordering skips them); their number
//                    is added to *dropped (one atomic per warp)
// The lanes of a warp take the 32 pixels of one word (blockDim and the grid
// stride are multiples of 32, npix is a power of two).
__global__ void __launch_bounds__(kOrdThreads) k_steady_update(unsigned* __restrict__ bits,
                                                               uint8_t* __restrict__ run, int64_t npix) {
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < npix; p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        const bool valid = p < npix;                          // false only when npix < 32
        unsigned w = 0u;
        if (valid) {
            w = bits[p >> 5];
            const bool hit = (w >> (p & 31)) & 1u;
            const unsigned r = run[p];
            run[p] = hit ? (uint8_t)min(r + 1u, 255u) : (uint8_t)0;
        }
        __syncwarp();                                         // every lane has read the word
        if (valid && (p & 31) == 0 && w != 0u) bits[p >> 5] = 0u;
    }
}

__global__ void __launch_bounds__(kOrdThreads) k_steady_apply(uint64_t* __restrict__ keys,
                                                              const unsigned* __restrict__ n_ptr, int cap,
                                                              int shift, const int* __restrict__ ord2d,
                                                              const int* __restrict__ dmax_of_d,
                                                              const uint8_t* __restrict__ run, int K,
                                                              unsigned* __restrict__ dropped) {
    const unsigned n = min(*n_ptr, (unsigned)cap);
    const uint64_t pm = (1ull << shift) - 1;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const unsigned i = i0 + threadIdx.x;
        bool drop = false;
        if (i < n) {
            const uint64_t key = keys[i];
            drop = dmax_of_d[ord2d[key >> shift]] != 0 && run[key & pm] >= K;
            if (drop) keys[i] = kDropped;
        }
        const unsigned b = __ballot_sync(0xffffffffu, drop);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(dropped, (unsigned)__popc(b));
    }
}

}  // namespace lpf
