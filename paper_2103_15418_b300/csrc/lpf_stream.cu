// Host runtime and C ABI of the dispersed-transient search (see include/lpf.h).
//
// One lpf_stream owns: the FP64-built integer delay table and its distinct-row
// plan, the device ring buffer, the dedispersed-image scratch, the candidate
// sort buffers and a small ring of result slots (pushed-but-unpolled frames).
// Every push enqueues ingest -> shift-sum -> filter/detect -> 3x3 maximum ->
// ordering -> stats and records an event; poll waits on that event with a
// deadline.  On the residual path three CUDA streams carry a push: the main
// stream (residuals, shift-sum, raw-ring write), a filter stream (the filter
// of push T runs beside the residuals and shift-sum of push T + 1) and a tail
// stream (3x3 maximum, ordering, statistics, result copies).
#include "../../include/lpf.h"
#include "lpf_kernels.cuh"
#include "lpf_dedisperse.cuh"
#include "lpf_residual.cuh"
#include "lpf_filter_res.cuh"
#include "lpf_qc.cuh"
#include "lpf_clip.cuh"
#include "lpf_order.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr double kCdmSeconds = 4.148808e3;   // s MHz^2 cm^3 / pc (Sec. 3.2)
using lpf::kSortBlocks;
constexpr int kMaxSlots = 16;
constexpr int kLmaxEv = 16;            // ring of per-push events: the 3x3 pass of push n done
constexpr int kSpareSlots = 2;         // raw/residual ring slots beyond the requested depth (residual path)

// Stages in the order their marks are recorded.  The residual path writes the
// raw ring after the shift-sum (ring_write); the tiled and clipping paths write
// it at ingest (ring_write then empty).
enum Stage { ST_INGEST, ST_DEDISP, ST_RINGW, ST_FILTER, ST_LMAX, ST_SORT, ST_FORMAT, ST_STATS, ST_N };
const char* kStageNames[ST_N] = {"ingest", "dedisperse", "ring_write", "filter_detect", "lmax", "sort", "format",
                                 "stats"};

int ceil_log2(int64_t v) {
    int b = 0;
    while ((int64_t(1) << b) < v) ++b;
    return b;
}

// words of one steady-source bit map (a bit per pixel of the key space)
size_t steady_words(int bx, int by) { return std::max<size_t>(((size_t)1 << (bx + by)) / 32, 1); }

// Candidate buffers of one push.  Consecutive pushes alternate between two
// lanes, so that the ordering, formatting and statistics of push T (its tail,
// on a second stream) overlap the ingest and search of push T + 1.
struct PushLane {
    uint64_t* keys[2] = {nullptr, nullptr};
    float* vals[2] = {nullptr, nullptr};
    unsigned* counter = nullptr;       // [4]: candidates, dropped by the steady mask, crossings (u64 at word 2)
    uint64_t* xkeys = nullptr;         // threshold crossings of the residual path (row, y, x) ...
    float* xvals = nullptr;            // ... and their S/N
    unsigned* ord = nullptr;           // [3][n ranks]: records per trial rank, bucket starts, cursors
    double* partials = nullptr;        // [n_distinct][filter blocks][3]
    cudaEvent_t dd_done = nullptr;     // the push's shift-sum finished: its filter may start
    cudaEvent_t rw_done = nullptr;     // the push's raw-ring write finished: its 3x3 pass may read the frame
    cudaEvent_t filter_done = nullptr; // the push's filter finished: its tail may start
    cudaEvent_t tail_done = nullptr;   // the push's tail finished: the lane may be reused
};

struct Slot {
    int64_t T = -1;
    int n_active = 0;
    lpf::CandidateRec* d_out = nullptr;
    double* d_stats = nullptr;     // [n_distinct][3]
    lpf::QcRecord* d_qc = nullptr; // quality-control record of the frame (qc on)
    cudaEvent_t done = nullptr;
};

}  // namespace

struct lpf_stream {
    int dev = 0;
    int H = 0, W = 0, F = 0, n_dm = 0, depth = 0;
    int ring_n = 0;                  // ring slots: depth (+ kSpareSlots on the residual path)
    lpf_params prm{};
    int64_t HW = 0, P = 0;
    size_t elem = 4;

    std::vector<int32_t> delay;      // [n_dm][F]
    std::vector<int> dmax;           // per trial
    int max_delay = 0;
    // distinct delay rows, sorted by (max delay, first trial)
    int n_distinct = 0;
    std::vector<int> row_dmax;       // per distinct row
    std::vector<int> row_of_d;
    std::vector<int> member_start;   // [n_distinct + 1]
    std::vector<int> member_ord;     // canonical rank of each member
    std::vector<int> ord2d;          // canonical rank -> trial
    int bx = 0, by = 0, bo = 0, key_bits = 0;

    // device memory
    void* ring = nullptr;
    float* D = nullptr;
    float* D2 = nullptr;            // second image buffer of the residual path (lane 1)
    int64_t xcap = 0;               // crossing capacity (per lane)
    float* stage = nullptr;          // host-push staging frames [2][F][HW]
    cudaStream_t h2d_st = nullptr;   // uploads of host frames
    cudaEvent_t stage_ready[2] = {nullptr, nullptr};   // upload into stage i done
    cudaEvent_t stage_free[2] = {nullptr, nullptr};    // push that read stage i done
    int stage_next = 0;
    int16_t* d_lag = nullptr;
    uint32_t* d_chg = nullptr;      // per distinct row: subbands whose lag differs from the previous row
    int* d_member_start = nullptr;
    int* d_member_ord = nullptr;
    int* d_ord2d = nullptr;
    int* d_dmax = nullptr;
    PushLane lanes[2];
    int lane_next = 0;
    cudaStream_t tail_st = nullptr;  // ordering, formatting, statistics, result copies
    cudaStream_t filt_st = nullptr;  // residual path: the filters
    cudaEvent_t lmax_ev[kLmaxEv] = {};   // [push n % kLmaxEv]: its 3x3 pass done
    int2* d_yx = nullptr;
    int yx_cap = 0;
    int2* h_yx = nullptr;           // page-locked staging of the dynspec coordinates
    int h_yx_cap = 0;
    cudaEvent_t yx_copied = nullptr; // the last staging copy has been read
    size_t device_bytes = 0;

    // opt-in steady-source suppression (suppress_steady > 0): per pixel of the key
    // space (2^(bx + by)), the push's zero-delay candidates (one bit map per push
    // lane, set by the kernels that find the candidates) and the run length
    unsigned* steady_bits = nullptr; // [2][steady_words]
    uint8_t* steady_run = nullptr;   // [2^(bx+by)]
    int zero_row = -1;               // the distinct delay row that is all zero, -1 if none
    // host pinned
    unsigned* h_count = nullptr;     // [slots][2]: records emitted, records dropped by the steady mask
    // quality control (App. A), when prm.qc: running per-pixel statistics of the
    // kept band images and the scratch of the three QC launches
    float* qc_mean = nullptr;        // [F][P]
    float* qc_m2 = nullptr;          // [F][P] sum of squared deviations
    int* qc_n = nullptr;             // [F] frames folded in
    float* qc_invn = nullptr;        // [F] 1/n of this frame's update
    double* qc_part = nullptr;       // [F][kQcScanBlocks] band sums
    unsigned* qc_words = nullptr;    // [2] pixel flags, discard mask
    lpf::QcRecord* h_qc = nullptr;   // [slots] pinned
    lpf::QcRecord last_qc{};
    // clipping path of the per-subband detector (clip_iters > 1 or the Gaussian kernel)
    bool clip = false;
    float* clip_w = nullptr;         // [box_r + 1] kernel factors g(|d|) (1 for the box)
    int clip_planes_n = 0;           // planes clipped per push: F (per-subband) or n_distinct (dispersed)
    uint8_t* clip_flags = nullptr;   // [clip_planes_n][P]
    float* clip_planes = nullptr;    // T1, T2, C, N, S: 5 x [clip_planes_n][P]
    unsigned* clip_changed = nullptr;  // [clip_iters]
    int64_t last_qc_T = -1;
    double* h_stats = nullptr;       // [slots][n_distinct][3]

    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t copy_st = nullptr;
    Slot slots[kMaxSlots];
    int n_slots = 2;
    std::deque<int> pending;         // slot indices in push order
    int next_slot = 0;

    bool any_push = false;
    int64_t T_first = 0, last_T = -1, frames_pushed = 0;
    bool polled = false;
    int64_t polled_T = -1;
    int polled_slot = -1;
    std::vector<double> last_stats; // [n_dm][2]

    int tiles_x = 0, tiles_y = 0;
    size_t filter_smem = 0;
    int filter_rmax = 16;
    bool stream_filter = false;     // residual path: k_residual + k_filter_res (box_r 7 or 15)
    int fseg = 1;                   // row segments per strip of the streaming filter
    void* resring = nullptr;        // [depth][F][P] per-subband residual X - C(X), storage type
    int n_strips = 0;

    bool profiling = false;
    cudaEvent_t ev[kMaxSlots][ST_N][2] = {};   // begin / end of every stage of a slot
    bool prof_slot[kMaxSlots] = {};
    double prof_ms[ST_N] = {};
    int64_t prof_n[ST_N] = {};
};

namespace {

int cuda_fail(cudaError_t e) {
    return e == cudaSuccess ? LPF_OK : LPF_E_CUDA;
}

#define LPF_TRY(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return LPF_E_CUDA;       \
    } while (0)

template <typename T>
int dev_alloc(lpf_stream* s, T** p, size_t count) {
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LPF_E_OOM;
    }
    s->device_bytes += bytes;
    return LPF_OK;
}

void free_all(lpf_stream* s) {
    if (!s) return;
    cudaSetDevice(s->dev);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->tail_st) cudaStreamSynchronize(s->tail_st);
    if (s->filt_st) cudaStreamSynchronize(s->filt_st);
    void* ptrs[] = {s->ring, s->resring, s->D, s->D2, s->stage, s->d_lag, s->d_chg, s->d_member_start, s->d_member_ord,
                    s->d_ord2d, s->d_dmax, s->d_yx};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& L : s->lanes) {
        void* lp[] = {L.keys[0], L.keys[1], L.vals[0], L.vals[1], L.counter, L.ord, L.partials, L.xkeys, L.xvals};
        for (void* p : lp)
            if (p) cudaFree(p);
        for (cudaEvent_t e : {L.dd_done, L.rw_done, L.filter_done, L.tail_done})
            if (e) cudaEventDestroy(e);
    }
    for (int i = 0; i < kMaxSlots; ++i) {
        if (s->slots[i].d_out) cudaFree(s->slots[i].d_out);
        if (s->slots[i].d_stats) cudaFree(s->slots[i].d_stats);
        if (s->slots[i].done) cudaEventDestroy(s->slots[i].done);
    }
    for (auto& row : s->ev)
        for (auto& st : row)
            for (auto& e : st)
                if (e) cudaEventDestroy(e);
    for (auto& e : s->lmax_ev)
        if (e) cudaEventDestroy(e);
    if (s->h_count) cudaFreeHost(s->h_count);
    if (s->steady_bits) cudaFree(s->steady_bits);
    if (s->steady_run) cudaFree(s->steady_run);
    if (s->h_yx) cudaFreeHost(s->h_yx);
    if (s->yx_copied) cudaEventDestroy(s->yx_copied);
    if (s->h_qc) cudaFreeHost(s->h_qc);
    if (s->clip_w) cudaFree(s->clip_w);
    if (s->clip_flags) cudaFree(s->clip_flags);
    if (s->clip_planes) cudaFree(s->clip_planes);
    if (s->clip_changed) cudaFree(s->clip_changed);
    {
        void* q[] = {s->qc_mean, s->qc_m2, s->qc_n, s->qc_invn, s->qc_part, s->qc_words};
        for (void* p : q)
            if (p) cudaFree(p);
        for (int i = 0; i < kMaxSlots; ++i)
            if (s->slots[i].d_qc) cudaFree(s->slots[i].d_qc);
    }
    if (s->h_stats) cudaFreeHost(s->h_stats);
    for (int i = 0; i < 2; ++i) {
        if (s->stage_ready[i]) cudaEventDestroy(s->stage_ready[i]);
        if (s->stage_free[i]) cudaEventDestroy(s->stage_free[i]);
    }
    if (s->h2d_st) {
        cudaStreamSynchronize(s->h2d_st);
        cudaStreamDestroy(s->h2d_st);
    }
    if (s->copy_st) cudaStreamDestroy(s->copy_st);
    if (s->tail_st) cudaStreamDestroy(s->tail_st);
    if (s->filt_st) cudaStreamDestroy(s->filt_st);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
}

// Sec. 3.2 delay law, FP64 on the host: floor(C_DM DM (nu^-2 - nu_ref^-2) / cadence + 1/2).
void build_delay_table(lpf_stream* s, const double* freqs, const double* dms) {
    double ref = freqs[0];
    for (int f = 1; f < s->F; ++f) ref = std::max(ref, freqs[f]);
    s->delay.assign((size_t)s->n_dm * s->F, 0);
    s->dmax.assign(s->n_dm, 0);
    for (int d = 0; d < s->n_dm; ++d) {
        int mx = 0;
        for (int f = 0; f < s->F; ++f) {
            double seconds = kCdmSeconds * dms[d] * (std::pow(freqs[f], -2.0) - std::pow(ref, -2.0));
            int v = (int)std::floor(seconds / s->prm.cadence_s + 0.5);
            s->delay[(size_t)d * s->F + f] = v;
            mx = std::max(mx, v);
        }
        s->dmax[d] = mx;
    }
    s->max_delay = *std::max_element(s->dmax.begin(), s->dmax.end());
}

// Group trials with identical delay rows; order rows by (max delay, first trial);
// canonical trial order is (t0 ascending = max delay descending, trial index).
void build_plan(lpf_stream* s) {
    std::map<std::vector<int32_t>, int> ids;
    std::vector<std::vector<int>> groups;
    std::vector<int> first_row_of_group;
    for (int d = 0; d < s->n_dm; ++d) {
        std::vector<int32_t> row(s->delay.begin() + (size_t)d * s->F, s->delay.begin() + (size_t)(d + 1) * s->F);
        auto it = ids.find(row);
        if (it == ids.end()) {
            ids.emplace(row, (int)groups.size());
            groups.push_back({d});
        } else {
            groups[it->second].push_back(d);
        }
    }
    std::vector<int> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        int da = s->dmax[groups[a][0]], db = s->dmax[groups[b][0]];
        if (da != db) return da < db;
        return groups[a][0] < groups[b][0];
    });
    // Inside each run of equal largest delay (any order there keeps the rows of
    // a warm-up prefix), order the rows greedily so that consecutive rows differ
    // in as few subbands as possible: the shift-sum reloads only those planes.
    auto lag_of = [&](int g, int f) { int d = groups[g][0]; return s->dmax[d] - s->delay[(size_t)d * s->F + f]; };
    for (size_t a = 0; a < order.size();) {
        size_t b = a;
        while (b < order.size() && s->dmax[groups[order[b]][0]] == s->dmax[groups[order[a]][0]]) ++b;
        for (size_t i = a; i < b && b - a <= 4096; ++i) {
            if (i == 0) continue;
            const int prev = order[i - 1];
            size_t best = i;
            int best_cost = s->F + 1;
            for (size_t j = i; j < b; ++j) {
                int c = 0;
                for (int f = 0; f < s->F; ++f) c += lag_of(order[j], f) != lag_of(prev, f);
                if (c < best_cost || (c == best_cost && order[j] < order[best])) { best_cost = c; best = j; }
            }
            std::swap(order[i], order[best]);
        }
        a = b;
    }
    s->n_distinct = (int)groups.size();
    // canonical trial ranks
    std::vector<int> tr(s->n_dm);
    for (int d = 0; d < s->n_dm; ++d) tr[d] = d;
    std::stable_sort(tr.begin(), tr.end(), [&](int a, int b) {
        if (s->dmax[a] != s->dmax[b]) return s->dmax[a] > s->dmax[b];
        return a < b;
    });
    s->ord2d = tr;
    std::vector<int> ord_of_d(s->n_dm);
    for (int i = 0; i < s->n_dm; ++i) ord_of_d[tr[i]] = i;
    s->row_of_d.assign(s->n_dm, 0);
    s->row_dmax.clear();
    s->member_start.assign(1, 0);
    s->member_ord.clear();
    for (int rr = 0; rr < s->n_distinct; ++rr) {
        const auto& g = groups[order[rr]];
        s->row_dmax.push_back(s->dmax[g[0]]);
        for (int d : g) {
            s->row_of_d[d] = rr;
            s->member_ord.push_back(ord_of_d[d]);
        }
        s->member_start.push_back((int)s->member_ord.size());
    }
}

// Per-subband detector: one row per band image of the newest frame (no delays),
// "trial" f = band f.
void build_band_plan(lpf_stream* s) {
    const int F = s->F;
    s->delay.assign((size_t)F * F, 0);
    s->dmax.assign(F, 0);
    s->max_delay = 0;
    s->n_distinct = F;
    s->ord2d.resize(F);
    s->row_of_d.resize(F);
    s->row_dmax.assign(F, 0);
    s->member_start.resize(F + 1);
    s->member_ord.resize(F);
    for (int f = 0; f < F; ++f) {
        s->ord2d[f] = f;
        s->row_of_d[f] = f;
        s->member_start[f] = f;
        s->member_ord[f] = f;
    }
    s->member_start[F] = F;
}

int n_active_rows(const lpf_stream* s, int64_t T) {
    int64_t span = T - s->T_first;
    int n = 0;
    while (n < s->n_distinct && s->row_dmax[n] <= span) ++n;
    return n;
}

template <typename TS>
void launch_ingest(lpf_stream* s, const float* frame, int64_t slot) {
    TS* dst = reinterpret_cast<TS*>(s->ring) + slot * s->F * s->P;
    int vec = ((reinterpret_cast<uintptr_t>(frame) & 15u) == 0 && (s->HW % 4) == 0) ? 1 : 0;
    int64_t work = vec ? s->F * s->HW / 4 : s->F * s->HW;
    int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 16);
    if (s->prm.qc)
        lpf::k_ingest_qc<TS><<<blocks, 256, 0, s->st>>>(frame, dst, s->F, s->HW, s->P, vec, s->qc_words + 1,
                                                         s->qc_invn, s->qc_mean, s->qc_m2);
    else
        lpf::k_ingest<TS><<<blocks, 256, 0, s->st>>>(frame, dst, s->F, s->HW, s->P, vec);
}

template <typename TS>
void launch_residual(lpf_stream* s, const float* frame, int64_t slot) {
    const unsigned* drop = s->prm.qc ? s->qc_words + 1 : nullptr;
    TS* res = reinterpret_cast<TS*>(s->resring) + slot * s->F * s->P;
    // row segments so that about two waves of CTAs (4 per SM) run; a segment
    // keeps at least 4 row blocks so that its 2r halo rows stay a small share
    const int B = s->prm.box_r == 7 ? lpf::ResGeom<7>::B : lpf::ResGeom<15>::B;
    const int per_plane = s->n_strips * s->F;
    int nseg = std::max(1, (2 * 4 * 148 + per_plane - 1) / per_plane);
    nseg = std::min(nseg, std::max(1, s->H / (4 * B)));
    const int seg_rows = (s->H + nseg - 1) / nseg;
    nseg = (s->H + seg_rows - 1) / seg_rows;
    dim3 grid((unsigned)s->n_strips, (unsigned)s->F, (unsigned)nseg);
    if (s->prm.box_r == 7)
        lpf::k_residual<7, TS><<<grid, lpf::ResGeom<7>::NT, lpf::residual_smem_bytes<7>(), s->st>>>(
            frame, drop, res, s->H, s->W, s->P, seg_rows);
    else
        lpf::k_residual<15, TS><<<grid, lpf::ResGeom<15>::NT, lpf::residual_smem_bytes<15>(), s->st>>>(
            frame, drop, res, s->H, s->W, s->P, seg_rows);
}

lpf::ResArgs res_args(lpf_stream* s, const lpf::FilterArgs& a, int Tmod, const PushLane& L) {
    lpf::ResArgs ra;
    ra.a = a;
    ra.ring = s->ring;
    ra.lag = s->d_lag;
    ra.F = s->F;
    ra.depth = s->ring_n;
    ra.Tmod = Tmod;
    ra.xkeys = L.xkeys;
    ra.xvals = L.xvals;
    ra.xcounter = reinterpret_cast<unsigned long long*>(L.counter + 2);
    ra.xcap = s->xcap;
    ra.band_k = s->prm.mode == LPF_MODE_SUBBAND ? s->prm.lmax_r : 0;
    return ra;
}

template <typename TS>
void launch_filter_res(lpf_stream* s, const lpf::FilterArgs& a, int n_rows, int Tmod, const PushLane& L,
                       cudaStream_t st) {
    const lpf::ResArgs ra = res_args(s, a, Tmod, L);
    dim3 grid((unsigned)s->n_strips, (unsigned)n_rows, (unsigned)s->fseg);
    if (s->prm.box_r == 7)
        lpf::k_filter_res<7, TS><<<grid, lpf::FiltGeom<7>::NT, lpf::res_filter_smem_bytes<7>(), st>>>(ra);
    else
        lpf::k_filter_res<15, TS><<<grid, lpf::FiltGeom<15>::NT, lpf::res_filter_smem_bytes<15>(), st>>>(ra);
}

template <typename TS>
void launch_lmax_res(lpf_stream* s, const lpf::FilterArgs& a, int Tmod, const PushLane& L, cudaStream_t st) {
    if (s->prm.mode == LPF_MODE_SUBBAND)
        lpf::k_lmax_res<TS, true><<<148 * 8, 256, 0, st>>>(res_args(s, a, Tmod, L));
    else
        lpf::k_lmax_res<TS, false><<<148 * 8, 256, 0, st>>>(res_args(s, a, Tmod, L));
}

template <typename TS>
int set_res_attributes() {
    if (cudaFuncSetAttribute(lpf::k_residual<7, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lpf::residual_smem_bytes<7>()) != cudaSuccess ||
        cudaFuncSetAttribute(lpf::k_residual<15, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lpf::residual_smem_bytes<15>()) != cudaSuccess ||
        cudaFuncSetAttribute(lpf::k_filter_res<7, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lpf::res_filter_smem_bytes<7>()) != cudaSuccess ||
        cudaFuncSetAttribute(lpf::k_filter_res<15, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lpf::res_filter_smem_bytes<15>()) != cudaSuccess)
        return LPF_E_CUDA;
    return LPF_OK;
}

// Shift-sum of a ring (raw: D; residual: R = D - C) into out; the rows are
// split into segments (each restarts its register state) for parallelism.
template <typename TS>
void launch_dedisperse_ring(lpf_stream* s, const void* ring_v, float* out, int n_rows, int Tmod) {
    // three row segments for FP32 rings, four for 16-bit rings (whose threads own 8
    // pixels, so half as many CTAs per segment; measured against 1-2 and 4-5);
    // more where one segment's plane table would exceed 48 KB of shared memory
    int nseg = n_rows >= 32 ? (sizeof(TS) == 4 ? 3 : 4) : 1;
    while (lpf::dedisperse_smem_bytes((n_rows + nseg - 1) / nseg, s->F) > 48 * 1024) ++nseg;
    const int seg = (n_rows + nseg - 1) / nseg;
    const size_t smem = lpf::dedisperse_smem_bytes(seg, s->F);
    const int F = s->F;
    auto go = [&](auto kern, int px) {
        dim3 grid((unsigned)((s->P / px + 255) / 256), (unsigned)nseg);
        kern<<<grid, 256, smem, s->st>>>(reinterpret_cast<const TS*>(ring_v), out, s->d_lag, s->d_chg, F,
                                         s->ring_n, Tmod, n_rows, seg, s->P);
    };
    if constexpr (sizeof(TS) == 4) {
        if (F == 8) go(lpf::k_dedisperse<8, true>, 4);
        else if (F == 16) go(lpf::k_dedisperse<16, true>, 4);
        else if (F == 32) go(lpf::k_dedisperse<32, true>, 4);
        else if (F < 8) go(lpf::k_dedisperse<8, false>, 4);
        else if (F < 16) go(lpf::k_dedisperse<16, false>, 4);
        else go(lpf::k_dedisperse<32, false>, 4);
    } else {
        if (F == 8) go(lpf::k_dedisperse16<8, true, TS>, 8);
        else if (F == 16) go(lpf::k_dedisperse16<16, true, TS>, 8);
        else if (F == 32) go(lpf::k_dedisperse16<32, true, TS>, 8);
        else if (F < 8) go(lpf::k_dedisperse16<8, false, TS>, 8);
        else if (F < 16) go(lpf::k_dedisperse16<16, false, TS>, 8);
        else go(lpf::k_dedisperse16<32, false, TS>, 8);
    }
}

// Tiled path: D from the raw ring.  Residual path: R = D - C from the residual
// ring (D itself is summed from the raw ring only on the 3x3 windows of the
// threshold crossings).
template <typename TS>
void launch_dedisperse(lpf_stream* s, float* out, int n_rows, int Tmod) {
    if (s->stream_filter) {
        launch_dedisperse_ring<TS>(s, s->resring, out, n_rows, Tmod);
    } else {
        launch_dedisperse_ring<TS>(s, s->ring, out, n_rows, Tmod);
    }
}

template <typename TS>
void launch_dynspec(lpf_stream* s, int n, int Tw, int slot_first, float* out) {
    int64_t total = (int64_t)n * s->F * Tw;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 32);
    if (blocks < 1) blocks = 1;
    lpf::k_dynspec<TS><<<blocks, 256, 0, s->st>>>(reinterpret_cast<const TS*>(s->ring), s->d_yx, n,
                                                  s->F, Tw, s->ring_n, slot_first, s->P, s->H, s->W,
                                                  s->prm.dyn_box_r, out);
}

int n_filter_blocks(const lpf_stream* s) {
    return s->stream_filter ? s->n_strips * s->fseg : s->tiles_x * s->tiles_y;
}

size_t filter_smem_bytes(int r, int rmax) {
    auto odd = [](int n) { return n | 1; };
    int RY = lpf::kTile + 4 * r, nC = lpf::kTile + 2 * r;
    size_t floats = (size_t)RY * odd(RY) + (size_t)RY * odd(nC) + 2 * (size_t)nC * odd(nC) +
                    (size_t)(nC + 2 * rmax + 2) * odd(lpf::kTile);
    return floats * sizeof(float);
}

// begin / end of stage i of slot sl on the stream the stage runs on
void prof_begin(lpf_stream* s, int sl, int i, cudaStream_t st) {
    if (s->profiling) cudaEventRecord(s->ev[sl][i][0], st);
}
void prof_end(lpf_stream* s, int sl, int i, cudaStream_t st) {
    if (s->profiling) cudaEventRecord(s->ev[sl][i][1], st);
}

// Accumulate the stage times of a finished slot (its done event has completed).
void prof_collect(lpf_stream* s, int sl) {
    if (!s->prof_slot[sl]) return;
    for (int i = 0; i < ST_N; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev[sl][i][0], s->ev[sl][i][1]) == cudaSuccess) {
            s->prof_ms[i] += ms;
            s->prof_n[i] += 1;
        } else {
            cudaGetLastError();
        }
    }
    s->prof_slot[sl] = false;
}

int enqueue_push(lpf_stream* s, const float* frame_dev, int64_t T) {
    const int sl = s->next_slot;
    Slot& slot = s->slots[sl];
    const int64_t ring_slot = T % s->ring_n;
    const int Tmod = (int)ring_slot;
    const int n_rows = n_active_rows(s, T);
    const int p = s->lane_next;
    PushLane& L = s->lanes[p];
    const int64_t seq = s->frames_pushed;      // push sequence number
    cudaGetLastError();

    const bool clip = s->clip;
    // Residual path: the residuals and their shift-sum come from the pushed frame
    // and the residual ring, so the raw ring write of this frame follows the
    // shift-sum; the filter runs on its own stream, beside the next push's
    // residuals and shift-sum, on this lane's image buffer and crossing list.
    const bool late_ring = s->stream_filter && !clip;
    cudaStream_t fs = late_ring ? s->filt_st : s->st;
    cudaStream_t ts = s->tail_st;
    float* images = (late_ring && p == 1) ? s->D2 : s->D;

    prof_begin(s, sl, ST_INGEST, s->st);
    if (s->prm.qc) {
        lpf::k_qc_scan<<<dim3(lpf::kQcScanBlocks, s->F), 256, 0, s->st>>>(
            frame_dev, s->HW, s->qc_mean, s->qc_m2, s->qc_n, s->P, s->prm.qc_min_frames, s->prm.qc_zeta,
            s->qc_part, s->qc_words);
        lpf::k_qc_decide<<<1, 32, 0, s->st>>>(s->qc_part, s->F, s->HW, s->prm.qc_z, s->qc_words, s->qc_n,
                                              s->qc_invn, s->qc_words + 1, slot.d_qc);
    }
    auto ingest = [&]() {
        switch (s->prm.dtype) {
            case LPF_FP32: launch_ingest<float>(s, frame_dev, ring_slot); break;
            case LPF_FP16: launch_ingest<__half>(s, frame_dev, ring_slot); break;
            default: launch_ingest<__nv_bfloat16>(s, frame_dev, ring_slot); break;
        }
    };
    if (late_ring) {
        switch (s->prm.dtype) {
            case LPF_FP32: launch_residual<float>(s, frame_dev, ring_slot); break;
            case LPF_FP16: launch_residual<__half>(s, frame_dev, ring_slot); break;
            default: launch_residual<__nv_bfloat16>(s, frame_dev, ring_slot); break;
        }
    } else {
        ingest();
    }
    // this lane's image buffer was last read by the filter of the push two back
    LPF_TRY(cudaStreamWaitEvent(s->st, L.filter_done, 0));
    prof_end(s, sl, ST_INGEST, s->st);
    prof_begin(s, sl, ST_DEDISP, s->st);
    // images the filter reads: D - C per distinct delay row, or (per-subband
    // detector) the residual planes of the newest frame, in place for FP32
    const float* filter_images = images;
    lpf::ClipArgs ca{};
    if (clip) {
        // planes clipped: the F band images of the newest frame (per-subband
        // detector), or the D images of the active distinct delay rows (dispersed
        // search, direct form: the shift-sum of the raw ring)
        const bool band = s->prm.mode == LPF_MODE_SUBBAND;
        const int np = band ? s->F : n_rows;
        const int64_t ns = (int64_t)s->clip_planes_n * s->P;   // stride of the scratch plane sets
        ca.X = s->D;
        ca.flags = s->clip_flags;
        ca.T1 = s->clip_planes;
        ca.T2 = ca.T1 + ns;
        ca.C = ca.T2 + ns;
        ca.N = ca.C + ns;
        ca.S = ca.N + ns;
        ca.changed = s->clip_changed;
        ca.w = s->clip_w;
        ca.F = np; ca.H = s->H; ca.W = s->W; ca.r = s->prm.box_r; ca.P = s->P; ca.kappa = s->prm.kappa;
        if (np > 0) {
            const int g = 148 * 8;
            const int64_t n = (int64_t)s->F * s->P;             // one ring slot
            lpf::k_zero_u32<<<1, 32, 0, s->st>>>(s->clip_changed, s->prm.clip_iters);
            if (band) {
                switch (s->prm.dtype) {
                    case LPF_FP32:
                        lpf::k_clip_init<float><<<g, 256, 0, s->st>>>(
                            ca, reinterpret_cast<const float*>(s->ring) + ring_slot * n);
                        break;
                    case LPF_FP16:
                        lpf::k_clip_init<__half><<<g, 256, 0, s->st>>>(
                            ca, reinterpret_cast<const __half*>(s->ring) + ring_slot * n);
                        break;
                    default:
                        lpf::k_clip_init<__nv_bfloat16><<<g, 256, 0, s->st>>>(
                            ca, reinterpret_cast<const __nv_bfloat16*>(s->ring) + ring_slot * n);
                        break;
                }
            } else {
                switch (s->prm.dtype) {
                    case LPF_FP32: launch_dedisperse<float>(s, s->D, n_rows, Tmod); break;
                    case LPF_FP16: launch_dedisperse<__half>(s, s->D, n_rows, Tmod); break;
                    default: launch_dedisperse<__nv_bfloat16>(s, s->D, n_rows, Tmod); break;
                }
                LPF_TRY(cudaMemsetAsync(s->clip_flags, 0, (size_t)np * s->P, s->st));
            }
            // window sums: shared-memory tiles, the radius a compile-time constant
            const dim3 gh((unsigned)(((s->W + lpf::kClipHX - 1) / lpf::kClipHX) * s->H), (unsigned)np);
            const dim3 gv((unsigned)((s->W + lpf::kClipVX - 1) / lpf::kClipVX),
                          (unsigned)((s->H + lpf::kClipVY - 1) / lpf::kClipVY), (unsigned)np);
            for (int it = 0; it < s->prm.clip_iters; ++it) {
                lpf::with_radius(ca.r, [&](auto rc) {
                    constexpr int R = decltype(rc)::value;
                    lpf::k_clip_hsum<R, 0><<<gh, 128, 0, s->st>>>(ca, it);
                    lpf::k_clip_vsum<R, 0><<<gv, 128, 0, s->st>>>(ca, it);
                    lpf::k_clip_hsum<R, 1><<<gh, 128, 0, s->st>>>(ca, it);
                    lpf::k_clip_vsum<R, 1><<<gv, 128, 0, s->st>>>(ca, it);
                });
                lpf::k_clip_flag<<<dim3((unsigned)std::min<int64_t>((s->HW + 1023) / 1024, 65535), (unsigned)np),
                                    256, 0, s->st>>>(ca, it);
            }
        }
    } else if (s->prm.mode == LPF_MODE_SUBBAND) {
        const int64_t n = (int64_t)s->F * s->P;
        if (s->prm.dtype == LPF_FP32) {
            filter_images = reinterpret_cast<const float*>(s->resring) + ring_slot * n;
        } else if (s->prm.dtype == LPF_FP16) {
            lpf::k_band_planes<__half><<<148 * 8, 256, 0, s->st>>>(
                reinterpret_cast<const __half*>(s->resring) + ring_slot * n, images, n);
        } else {
            lpf::k_band_planes<__nv_bfloat16><<<148 * 8, 256, 0, s->st>>>(
                reinterpret_cast<const __nv_bfloat16*>(s->resring) + ring_slot * n, images, n);
        }
    } else if (n_rows > 0) {
        switch (s->prm.dtype) {
            case LPF_FP32: launch_dedisperse<float>(s, images, n_rows, Tmod); break;
            case LPF_FP16: launch_dedisperse<__half>(s, images, n_rows, Tmod); break;
            default: launch_dedisperse<__nv_bfloat16>(s, images, n_rows, Tmod); break;
        }
    }
    prof_end(s, sl, ST_DEDISP, s->st);
    if (late_ring) LPF_TRY(cudaEventRecord(L.dd_done, s->st));
    prof_begin(s, sl, ST_RINGW, s->st);
    if (late_ring) {
        // the raw ring write replaces the frame T - slots, which the 3x3 passes of
        // the pushes up to T - slots + max_delay read: wait for the last of them (the
        // tail stream runs them in order; an event re-recorded by a later push is a
        // later pass, so waiting on it is safe)
        const int64_t back = (int64_t)s->ring_n - s->max_delay;
        if (seq >= back) LPF_TRY(cudaStreamWaitEvent(s->st, s->lmax_ev[(seq - back) % kLmaxEv], 0));
        ingest();
        LPF_TRY(cudaEventRecord(L.rw_done, s->st));
    }
    prof_end(s, sl, ST_RINGW, s->st);
    if (late_ring) LPF_TRY(cudaStreamWaitEvent(fs, L.dd_done, 0));
    // the lane's crossing list, counters, candidate buffers and partials were last
    // used by the tail of the push two back
    LPF_TRY(cudaStreamWaitEvent(fs, L.tail_done, 0));
    lpf::k_zero_u32<<<1, 32, 0, fs>>>(L.counter, 4);   // candidates, dropped, crossings (u64 at word 2)
    // this lane's zero-delay marks (cleared by the lane's previous run-length update)
    unsigned* zbits = s->prm.suppress_steady > 0 ? s->steady_bits + p * steady_words(s->bx, s->by) : nullptr;
    prof_begin(s, sl, ST_FILTER, fs);
    lpf::FilterArgs a;
    if (n_rows > 0) {
        a.D = filter_images; a.P = s->P; a.H = s->H; a.W = s->W; a.r = s->prm.box_r; a.kappa = s->prm.kappa;
        a.tiles_x = s->tiles_x; a.tiles_y = s->tiles_y;
        a.member_start = s->d_member_start; a.member_ord = s->d_member_ord;
        a.keys = L.keys[0]; a.vals = L.vals[0]; a.counter = L.counter; a.cap = s->prm.cand_cap;
        a.bx = s->bx; a.by = s->by; a.partials = L.partials;
        a.zbits = zbits; a.zrow = s->zero_row;
        if (clip) {
            lpf::k_clip_emit<<<dim3((unsigned)n_filter_blocks(s), (unsigned)ca.F), 256, 0, s->st>>>(
                ca, a, s->prm.lmax_r);
        } else if (s->stream_filter) {
            switch (s->prm.dtype) {
                case LPF_FP32: launch_filter_res<float>(s, a, n_rows, Tmod, L, fs); break;
                case LPF_FP16: launch_filter_res<__half>(s, a, n_rows, Tmod, L, fs); break;
                default: launch_filter_res<__nv_bfloat16>(s, a, n_rows, Tmod, L, fs); break;
            }
        } else {
            a.D = s->D;
            dim3 grid((unsigned)(s->tiles_x * s->tiles_y), (unsigned)n_rows);
            if (s->filter_rmax == 8)
                lpf::k_filter<8><<<grid, lpf::kFilterThreads, s->filter_smem, s->st>>>(a);
            else
                lpf::k_filter<16><<<grid, lpf::kFilterThreads, s->filter_smem, s->st>>>(a);
        }
    }
    prof_end(s, sl, ST_FILTER, fs);
    // the tail of this push (3x3 pass, ordering, formatting, statistics, copies)
    // on the tail stream once its filter (and raw ring write) is done, after the
    // tail of the previous push (same stream, other lane)
    LPF_TRY(cudaEventRecord(L.filter_done, fs));
    LPF_TRY(cudaStreamWaitEvent(ts, L.filter_done, 0));
    if (late_ring) LPF_TRY(cudaStreamWaitEvent(ts, L.rw_done, 0));
    prof_begin(s, sl, ST_LMAX, ts);
    if (n_rows > 0 && late_ring) {
        switch (s->prm.dtype) {
            case LPF_FP32: launch_lmax_res<float>(s, a, Tmod, L, ts); break;
            case LPF_FP16: launch_lmax_res<__half>(s, a, Tmod, L, ts); break;
            default: launch_lmax_res<__nv_bfloat16>(s, a, Tmod, L, ts); break;
        }
    }
    prof_end(s, sl, ST_LMAX, ts);
    LPF_TRY(cudaEventRecord(s->lmax_ev[seq % kLmaxEv], ts));
    // opt-in steady-source suppression, in push order on the tail stream
    if (s->prm.suppress_steady > 0) {
        const int shift = s->bx + s->by;
        const int64_t npix = (int64_t)1 << shift;
        lpf::k_steady_update<<<(unsigned)std::min<int64_t>((npix + 255) / 256, 148 * 16), 256, 0, ts>>>(
            zbits, s->steady_run, npix);
        lpf::k_steady_apply<<<kSortBlocks, lpf::kOrdThreads, 0, ts>>>(L.keys[0], L.counter, s->prm.cand_cap, shift,
                                                                      s->d_ord2d, s->d_dmax, s->steady_run,
                                                                      s->prm.suppress_steady, L.counter + 1);
    }
    // ordering: counting sort on the trial rank, then each rank's bucket sorted by
    // pixel and formatted (lpf_order.cuh)
    {
        const int shift = s->bx + s->by, n_ord = s->n_dm;
        unsigned* counts = L.ord;
        unsigned* start = L.ord + n_ord;
        unsigned* cursor = L.ord + 2 * n_ord;
        prof_begin(s, sl, ST_SORT, ts);
        lpf::k_ord_count<<<kSortBlocks, lpf::kOrdThreads, 0, ts>>>(L.keys[0], L.counter, s->prm.cand_cap, shift,
                                                                   n_ord, counts);
        lpf::k_ord_scan<<<1, 1024, 0, ts>>>(counts, n_ord, start, cursor);
        lpf::k_ord_scatter<<<kSortBlocks, lpf::kOrdThreads, 0, ts>>>(L.keys[0], L.vals[0], L.counter,
                                                                     s->prm.cand_cap, shift, cursor, L.keys[1],
                                                                     L.vals[1]);
        prof_end(s, sl, ST_SORT, ts);
        prof_begin(s, sl, ST_FORMAT, ts);
        lpf::k_ord_sort_format<<<std::min(n_ord, 148 * 8), lpf::kOrdThreads, lpf::ord_sort_smem_bytes(), ts>>>(
            L.keys[1], L.vals[1], start, cursor, n_ord, slot.d_out, s->d_ord2d, s->d_dmax, T, s->bx, s->by);
        prof_end(s, sl, ST_FORMAT, ts);
    }
    prof_begin(s, sl, ST_STATS, ts);
    if (n_rows > 0)
        lpf::k_stats<<<n_rows, 256, 0, ts>>>(L.partials, n_filter_blocks(s), slot.d_stats);
    prof_end(s, sl, ST_STATS, ts);
    if (cudaGetLastError() != cudaSuccess) return LPF_E_CUDA;
    LPF_TRY(cudaMemcpyAsync(s->h_count + 2 * sl, L.counter, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, ts));
    if (s->prm.qc)
        LPF_TRY(cudaMemcpyAsync(s->h_qc + sl, slot.d_qc, sizeof(lpf::QcRecord), cudaMemcpyDeviceToHost, ts));
    if (n_rows > 0)
        LPF_TRY(cudaMemcpyAsync(s->h_stats + (size_t)sl * s->n_distinct * 3, slot.d_stats,
                                (size_t)n_rows * 3 * sizeof(double), cudaMemcpyDeviceToHost, ts));
    LPF_TRY(cudaEventRecord(L.tail_done, ts));
    LPF_TRY(cudaEventRecord(slot.done, ts));
    s->lane_next = p ^ 1;
    s->prof_slot[sl] = s->profiling;
    slot.T = T;
    slot.n_active = n_rows;
    s->pending.push_back(sl);
    s->next_slot = (sl + 1) % s->n_slots;
    if (!s->any_push) {
        s->any_push = true;
        s->T_first = T;
    }
    s->last_T = T;
    s->frames_pushed += 1;
    return LPF_OK;
}

int check_push(lpf_stream* s, int64_t T) {
    if (!s || T < 0) return LPF_E_ARG;
    if (s->any_push && T != s->last_T + 1) return LPF_E_ORDER;
    if ((int)s->pending.size() >= s->n_slots) return LPF_E_BUSY;
    return LPF_OK;
}

}  // namespace

extern "C" {

void lpf_default_params(lpf_params* p) {
    if (!p) return;
    p->cadence_s = 1.0;
    p->kappa = 6.0f;
    p->box_r = 15;
    p->lmax_r = 1;
    p->dtype = LPF_FP32;
    p->cand_cap = 1 << 20;
    p->dyn_box_r = 0;
    p->result_slots = 2;
    p->cuda_stream = nullptr;
    p->filter_impl = 0;
    p->qc = 0;
    p->qc_z = 5.0f;
    p->qc_zeta = 20.0f;
    p->qc_min_frames = 128;
    p->mode = LPF_MODE_DISPERSED;
    p->clip_iters = 1;
    p->kernel = LPF_KERNEL_BOX;
    p->gauss_sigma = 0.f;
    p->suppress_steady = 0;
}

const char* lpf_strerror(int code) {
    switch (code) {
        case LPF_OK: return "ok";
        case LPF_E_ARG: return "invalid argument";
        case LPF_E_DEPTH: return "buffer depth too small for the delay table or window";
        case LPF_E_ORDER: return "frame index out of order";
        case LPF_E_OOM: return "out of memory";
        case LPF_E_BUDGET: return "stream exceeds the HBM budget";
        case LPF_E_TRUNCATED: return "candidate list truncated";
        case LPF_E_STALE: return "frames no longer in the ring buffer";
        case LPF_E_TIMEOUT: return "timed out";
        case LPF_E_CUDA: return "CUDA error";
        case LPF_E_BUSY: return "all result slots are unpolled";
        case LPF_E_NODATA: return "no frame to poll";
        case LPF_E_CAPACITY: return "request exceeds the fixed staging capacity";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// Validate the arguments and build the host-side plan (delay table, distinct
// rows, launch geometry) of a stream; no CUDA call.
int plan_stream(lpf_stream** out, int H, int W, int F, const double* freqs_mhz, int n_dm,
                const double* dm_grid, int buffer_depth, const lpf_params* params) {
    *out = nullptr;
    lpf_params prm;
    lpf_default_params(&prm);
    if (params) prm = *params;
    if (prm.mode != LPF_MODE_DISPERSED && prm.mode != LPF_MODE_SUBBAND) return LPF_E_ARG;
    const bool band = prm.mode == LPF_MODE_SUBBAND;
    if (H <= 0 || W <= 0 || F <= 0 || !freqs_mhz || buffer_depth <= 0) return LPF_E_ARG;
    if (!band && (n_dm <= 0 || !dm_grid)) return LPF_E_ARG;
    if (H > (1 << 16) || W > (1 << 16) || buffer_depth > 32767 || F > 32) return LPF_E_ARG;
    if (!(prm.cadence_s > 0) || prm.box_r < 1 || prm.box_r > 16) return LPF_E_ARG;
    if (band ? (prm.lmax_r < 1 || prm.lmax_r > 3) : prm.lmax_r != 1) return LPF_E_ARG;
    // the Gaussian kernel: per-subband detector, on the clipping path (any box_r)
    if (prm.kernel != LPF_KERNEL_BOX && prm.kernel != LPF_KERNEL_GAUSS) return LPF_E_ARG;
    const bool gauss = prm.kernel == LPF_KERNEL_GAUSS;
    if (gauss && (!band || !(prm.gauss_sigma > 0) || !std::isfinite(prm.gauss_sigma))) return LPF_E_ARG;
    if (prm.suppress_steady < 0 || prm.suppress_steady > 255 || (prm.suppress_steady > 0 && band)) return LPF_E_ARG;
    // the per-subband detector with the box runs on the residual planes: streaming filter only
    if (band && !gauss && (prm.filter_impl == 1 || (prm.box_r != 7 && prm.box_r != 15))) return LPF_E_ARG;
    // iterated clipping: the per-subband detector, or the dispersed search on the
    // direct-form path (D itself per delay row; the box kernel)
    if (prm.clip_iters < 1 || prm.clip_iters > 16) return LPF_E_ARG;
    if (!band && prm.clip_iters > 1 && prm.filter_impl == 2) return LPF_E_ARG;
    if (prm.dtype < LPF_FP32 || prm.dtype > LPF_BF16 || prm.cand_cap < 1 || prm.dyn_box_r < 0) return LPF_E_ARG;
    if (prm.result_slots < 1 || prm.result_slots > kMaxSlots) return LPF_E_ARG;
    if (!std::isfinite(prm.kappa)) return LPF_E_ARG;
    if (prm.filter_impl < 0 || prm.filter_impl > 2) return LPF_E_ARG;
    if (prm.filter_impl == 2 && prm.box_r != 7 && prm.box_r != 15) return LPF_E_ARG;
    if (prm.qc != 0 && prm.qc != 1) return LPF_E_ARG;
    if (prm.qc && (!(prm.qc_z > 0) || !(prm.qc_zeta > 0) || !std::isfinite(prm.qc_z) ||
                   !std::isfinite(prm.qc_zeta) || prm.qc_min_frames < 2))
        return LPF_E_ARG;
    for (int f = 0; f < F; ++f)
        if (!(freqs_mhz[f] > 0) || !std::isfinite(freqs_mhz[f])) return LPF_E_ARG;
    for (int d = 0; !band && d < n_dm; ++d)
        if (!(dm_grid[d] >= 0) || !std::isfinite(dm_grid[d])) return LPF_E_ARG;

    lpf_stream* s = new (std::nothrow) lpf_stream();
    if (!s) return LPF_E_OOM;
    s->H = H; s->W = W; s->F = F; s->n_dm = band ? F : n_dm; s->depth = buffer_depth; s->prm = prm;
    s->HW = (int64_t)H * W;
    s->P = (s->HW + 7) / 8 * 8;
    s->elem = prm.dtype == LPF_FP32 ? 4 : 2;
    s->n_slots = prm.result_slots;
    if (band) {
        build_band_plan(s);
    } else {
        build_delay_table(s, freqs_mhz, dm_grid);
        if (buffer_depth < s->max_delay + 1) {
            delete s;
            return LPF_E_DEPTH;
        }
        build_plan(s);
    }
    s->bx = std::max(1, ceil_log2(W));
    s->by = std::max(1, ceil_log2(H));
    for (int rr = 0; rr < s->n_distinct && !band; ++rr)
        if (s->row_dmax[rr] == 0) s->zero_row = rr;      // max delay 0: every delay is 0
    s->bo = std::max(1, ceil_log2(s->n_dm));
    s->key_bits = s->bx + s->by + s->bo;
    if (s->key_bits > 64) {
        delete s;
        return LPF_E_ARG;
    }
    s->tiles_x = (W + lpf::kTile - 1) / lpf::kTile;
    s->tiles_y = (H + lpf::kTile - 1) / lpf::kTile;
    s->filter_rmax = prm.box_r <= 8 ? 8 : 16;
    s->filter_smem = filter_smem_bytes(prm.box_r, s->filter_rmax);
    // the clipping path (per-subband detector, clip_iters > 1 or the Gaussian kernel)
    // sums its windows directly from the raw ring: no residual ring, no crossing list
    s->clip = prm.clip_iters > 1 || gauss;
    // clipping planes: one per band image (per-subband detector) or per distinct delay row
    s->clip_planes_n = band ? F : s->n_distinct;
    s->stream_filter = !s->clip && (band || prm.filter_impl == 2 ||
                                    (prm.filter_impl == 0 && (prm.box_r == 7 || prm.box_r == 15)));
    // the residual path writes the raw ring after the shift-sum, while 3x3 passes of
    // earlier pushes may still read it: two spare slots keep that write from
    // waiting on the pass just before it
    s->ring_n = buffer_depth + ((s->stream_filter && !s->clip) ? kSpareSlots : 0);
    s->n_strips = (W + lpf::kStreamTX - 1) / lpf::kStreamTX;
    // the per-subband detector has only F rows: split each strip into row segments
    // so that about two waves of 4 CTAs per SM run (each segment after the first
    // re-reads one block of rows); the dispersed search has enough rows
    if (band) {
        const int B = prm.box_r == 7 ? lpf::FiltGeom<7>::B : lpf::FiltGeom<15>::B;
        const int nblk = (H + prm.box_r + B - 1) / B;
        const int want = (2 * 4 * 148 + s->n_strips * F - 1) / (s->n_strips * F);
        s->fseg = std::max(1, std::min(want, nblk / 2));
    }
    // crossing list of the residual path: room for 1/32 of all pixels of all
    // delay rows above the threshold (a swamped frame overflows into the slower
    // in-kernel resolution, with the same results)
    if (s->stream_filter)
        s->xcap = std::max<int64_t>(prm.cand_cap, (int64_t)s->n_distinct * s->HW / 32);

    *out = s;
    return LPF_OK;
}

// Device bytes lpf_stream_open requests for a planned stream (the sum of the
// allocation sizes; the allocator may round each one up).
size_t footprint_bytes(const lpf_stream* s) {
    auto b = [](size_t n) { return std::max<size_t>(n, 16); };
    const size_t nd = (size_t)s->n_distinct, cap = (size_t)s->prm.cand_cap;
    const bool two = s->stream_filter && !s->clip;   // filter beside the next push: two image buffers
    size_t t = (size_t)s->ring_n * s->F * s->P * s->elem * (s->stream_filter ? 2 : 1);
    t += b(nd * s->P * 4) * (two ? 2 : 1) + b(2 * (size_t)s->F * s->HW * 4) + b(nd * s->F * 2) + b(nd * 4);
    if (s->xcap > 0) t += 2 * (b((size_t)s->xcap * 8) + b((size_t)s->xcap * 4));
    if (s->clip)
        t += b((size_t)s->clip_planes_n * s->P) + b(5 * (size_t)s->clip_planes_n * s->P * 4) +
             b((size_t)s->prm.clip_iters * 4) +
             b((size_t)(s->prm.box_r + 1) * 4);
    if (s->prm.qc) {
        t += 2 * b((size_t)s->F * s->P * 4) + b((size_t)s->F * 4) + b((size_t)s->F * 4) +
             b((size_t)s->F * lpf::kQcScanBlocks * 8) + b(2 * 4);
        t += (size_t)s->n_slots * b(sizeof(lpf::QcRecord));
    }
    t += b(s->member_start.size() * 4) + b(s->member_ord.size() * 4) + 2 * b((size_t)s->n_dm * 4);
    // two push lanes: keys and values (x2 for the ordering), counter, rank buckets, partials
    t += 2 * (2 * (b(cap * 8) + b(cap * 4)) + b(16) + b((size_t)3 * s->n_dm * 4) +
              b(nd * n_filter_blocks(s) * 3 * 8));
    t += (size_t)s->n_slots * (b(cap * sizeof(lpf::CandidateRec)) + b(nd * 3 * 8));
    if (s->prm.suppress_steady > 0) {
        const size_t npix = (size_t)1 << (s->bx + s->by);
        t += b(2 * steady_words(s->bx, s->by) * 4) + b(npix);
    }
    return t;
}

}  // namespace

extern "C" {

int lpf_stream_footprint(int H, int W, int F, const double* freqs_mhz, int n_dm, const double* dm_grid,
                         int buffer_depth, const lpf_params* params, size_t* bytes) {
    if (!bytes) return LPF_E_ARG;
    lpf_stream* s = nullptr;
    int rc = plan_stream(&s, H, W, F, freqs_mhz, n_dm, dm_grid, buffer_depth, params);
    if (rc != LPF_OK) return rc;
    *bytes = footprint_bytes(s);
    delete s;
    return LPF_OK;
}

int lpf_stream_open(lpf_stream** out, int H, int W, int F, const double* freqs_mhz, int n_dm,
                    const double* dm_grid, int buffer_depth, const lpf_params* params) {
    if (!out) return LPF_E_ARG;
    *out = nullptr;
    lpf_stream* s = nullptr;
    {
        int prc = plan_stream(&s, H, W, F, freqs_mhz, n_dm, dm_grid, buffer_depth, params);
        if (prc != LPF_OK) return prc;
    }
    const lpf_params prm = s->prm;

    int rc = LPF_OK;
    if (cudaGetDevice(&s->dev) != cudaSuccess) { cudaGetLastError(); delete s; return LPF_E_CUDA; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { cudaGetLastError(); delete s; return LPF_E_CUDA; }
    if (prm.cuda_stream) {
        s->st = (cudaStream_t)prm.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return LPF_E_CUDA; }
        s->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK && cudaStreamCreateWithFlags(&s->h2d_st, cudaStreamNonBlocking) != cudaSuccess) rc = LPF_E_CUDA;
    // the tail stream at the highest priority: its short launches (3x3 pass,
    // ordering, statistics) take SMs ahead of the next pushes' shift-sums and
    // filters, so the lane they hold is freed sooner (measured: 1.13 against
    // 1.14-1.18 ms per push, and steadier)
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (rc == LPF_OK && cudaStreamCreateWithPriority(&s->tail_st, cudaStreamNonBlocking, hi) != cudaSuccess) rc = LPF_E_CUDA;
    }
    if (rc == LPF_OK && cudaStreamCreateWithFlags(&s->filt_st, cudaStreamNonBlocking) != cudaSuccess) rc = LPF_E_CUDA;
    for (int i = 0; i < kLmaxEv && rc == LPF_OK; ++i)
        if (cudaEventCreateWithFlags(&s->lmax_ev[i], cudaEventDisableTiming) != cudaSuccess) rc = LPF_E_CUDA;
    for (int i = 0; i < 2 && rc == LPF_OK; ++i)
        if (cudaEventCreateWithFlags(&s->stage_ready[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->stage_free[i], cudaEventDisableTiming) != cudaSuccess)
            rc = LPF_E_CUDA;
    if (rc == LPF_OK && cudaFuncSetAttribute(lpf::k_filter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)filter_smem_bytes(8, 8)) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK && cudaFuncSetAttribute(lpf::k_filter<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)filter_smem_bytes(16, 16)) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK) rc = set_res_attributes<float>();
    if (rc == LPF_OK) rc = set_res_attributes<__half>();
    if (rc == LPF_OK) rc = set_res_attributes<__nv_bfloat16>();
    const size_t ring_elems = (size_t)s->ring_n * F * s->P;
    if (rc == LPF_OK) {
        if (cudaMalloc(&s->ring, ring_elems * s->elem) != cudaSuccess) { cudaGetLastError(); rc = LPF_E_OOM; }
        else s->device_bytes += ring_elems * s->elem;
    }
    if (rc == LPF_OK && cudaMemsetAsync(s->ring, 0, ring_elems * s->elem, s->st) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK && s->stream_filter) {
        if (cudaMalloc(&s->resring, ring_elems * s->elem) != cudaSuccess) { cudaGetLastError(); rc = LPF_E_OOM; }
        else s->device_bytes += ring_elems * s->elem;
        if (rc == LPF_OK && cudaMemsetAsync(s->resring, 0, ring_elems * s->elem, s->st) != cudaSuccess) rc = LPF_E_CUDA;
    }
    if (rc == LPF_OK) rc = dev_alloc(s, &s->D, (size_t)s->n_distinct * s->P);
    if (rc == LPF_OK && s->stream_filter && !s->clip) rc = dev_alloc(s, &s->D2, (size_t)s->n_distinct * s->P);
    if (rc == LPF_OK) rc = dev_alloc(s, &s->stage, 2 * (size_t)F * s->HW);
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_lag, (size_t)s->n_distinct * F);
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_chg, (size_t)s->n_distinct);
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_member_start, s->member_start.size());
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_member_ord, s->member_ord.size());
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_ord2d, (size_t)s->n_dm);
    if (rc == LPF_OK) rc = dev_alloc(s, &s->d_dmax, (size_t)s->n_dm);
    for (auto& L : s->lanes) {
        for (int i = 0; i < 2 && rc == LPF_OK; ++i) {
            rc = dev_alloc(s, &L.keys[i], (size_t)prm.cand_cap);
            if (rc == LPF_OK) rc = dev_alloc(s, &L.vals[i], (size_t)prm.cand_cap);
        }
        if (rc == LPF_OK) rc = dev_alloc(s, &L.counter, 4);
        if (rc == LPF_OK && s->xcap > 0) rc = dev_alloc(s, &L.xkeys, (size_t)s->xcap);
        if (rc == LPF_OK && s->xcap > 0) rc = dev_alloc(s, &L.xvals, (size_t)s->xcap);
        if (rc == LPF_OK) rc = dev_alloc(s, &L.ord, (size_t)3 * s->n_dm);
        // the rank counts start at zero; the scan clears them after every push
        if (rc == LPF_OK && cudaMemsetAsync(L.ord, 0, (size_t)3 * s->n_dm * 4, s->st) != cudaSuccess) rc = LPF_E_CUDA;
        if (rc == LPF_OK) rc = dev_alloc(s, &L.partials, (size_t)s->n_distinct * n_filter_blocks(s) * 3);
        if (rc == LPF_OK && (cudaEventCreateWithFlags(&L.filter_done, cudaEventDisableTiming) != cudaSuccess ||
                             cudaEventCreateWithFlags(&L.dd_done, cudaEventDisableTiming) != cudaSuccess ||
                             cudaEventCreateWithFlags(&L.rw_done, cudaEventDisableTiming) != cudaSuccess ||
                             cudaEventCreateWithFlags(&L.tail_done, cudaEventDisableTiming) != cudaSuccess))
            rc = LPF_E_CUDA;
    }
    if (rc == LPF_OK && prm.suppress_steady > 0) {
        const size_t npix = (size_t)1 << (s->bx + s->by);
        rc = dev_alloc(s, &s->steady_bits, 2 * steady_words(s->bx, s->by));
        if (rc == LPF_OK) rc = dev_alloc(s, &s->steady_run, npix);
        // no pixel has a run yet, no lane a mark
        if (rc == LPF_OK && (cudaMemsetAsync(s->steady_run, 0, npix, s->st) != cudaSuccess ||
                             cudaMemsetAsync(s->steady_bits, 0, 2 * steady_words(s->bx, s->by) * sizeof(unsigned),
                                             s->st) != cudaSuccess))
            rc = LPF_E_CUDA;
    }
    for (int i = 0; i < s->n_slots && rc == LPF_OK; ++i) {
        rc = dev_alloc(s, &s->slots[i].d_out, (size_t)prm.cand_cap);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->slots[i].d_stats, (size_t)s->n_distinct * 3);
        if (rc == LPF_OK && cudaEventCreateWithFlags(&s->slots[i].done, cudaEventDisableTiming) != cudaSuccess)
            rc = LPF_E_CUDA;
    }
    if (s->clip) {
        // g(i) = exp(-i^2 / (2 s^2)) in FP64, stored as FP32 (1 for the box)
        std::vector<float> g(prm.box_r + 1, 1.0f);
        if (prm.kernel == LPF_KERNEL_GAUSS)
            for (int i = 0; i <= prm.box_r; ++i)
                g[i] = (float)std::exp(-(double)i * i / (2.0 * (double)prm.gauss_sigma * prm.gauss_sigma));
        if (rc == LPF_OK) rc = dev_alloc(s, &s->clip_w, g.size());
        if (rc == LPF_OK && cudaMemcpy(s->clip_w, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice) !=
                                cudaSuccess)
            rc = LPF_E_CUDA;
        if (rc == LPF_OK) rc = dev_alloc(s, &s->clip_flags, (size_t)s->clip_planes_n * s->P);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->clip_planes, 5 * (size_t)s->clip_planes_n * s->P);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->clip_changed, (size_t)prm.clip_iters);
    }
    if (prm.qc) {
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_mean, (size_t)F * s->P);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_m2, (size_t)F * s->P);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_n, (size_t)F);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_invn, (size_t)F);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_part, (size_t)F * lpf::kQcScanBlocks);
        if (rc == LPF_OK) rc = dev_alloc(s, &s->qc_words, 2);
        for (int i = 0; i < s->n_slots && rc == LPF_OK; ++i) rc = dev_alloc(s, &s->slots[i].d_qc, 1);
        if (rc == LPF_OK && (cudaMemsetAsync(s->qc_mean, 0, (size_t)F * s->P * 4, s->st) != cudaSuccess ||
                             cudaMemsetAsync(s->qc_m2, 0, (size_t)F * s->P * 4, s->st) != cudaSuccess ||
                             cudaMemsetAsync(s->qc_n, 0, (size_t)F * 4, s->st) != cudaSuccess ||
                             cudaMemsetAsync(s->qc_words, 0, 2 * 4, s->st) != cudaSuccess))
            rc = LPF_E_CUDA;
        if (rc == LPF_OK && cudaMallocHost(&s->h_qc, sizeof(lpf::QcRecord) * kMaxSlots) != cudaSuccess) {
            cudaGetLastError();
            rc = LPF_E_OOM;
        }
    }
    for (int k = 0; k < s->n_slots && rc == LPF_OK; ++k)
        for (int i = 0; i < ST_N && rc == LPF_OK; ++i)
            for (int e = 0; e < 2 && rc == LPF_OK; ++e)
                if (cudaEventCreate(&s->ev[k][i][e]) != cudaSuccess) rc = LPF_E_CUDA;
    if (rc == LPF_OK) {
        if (cudaMallocHost(&s->h_count, 2 * sizeof(unsigned) * kMaxSlots) != cudaSuccess ||
            cudaMallocHost(&s->h_stats, sizeof(double) * kMaxSlots * s->n_distinct * 3) != cudaSuccess) {
            cudaGetLastError();
            rc = LPF_E_OOM;
        }
    }
    if (rc == LPF_OK) {
        std::vector<int16_t> lag((size_t)s->n_distinct * F);
        for (int rr = 0; rr < s->n_distinct; ++rr) {
            int d = s->ord2d[s->member_ord[s->member_start[rr]]];
            for (int f = 0; f < F; ++f)
                lag[(size_t)rr * F + f] = (int16_t)(s->dmax[d] - s->delay[(size_t)d * F + f]);
        }
        std::vector<uint32_t> chg(s->n_distinct, 0);
        for (int rr = 0; rr < s->n_distinct; ++rr)
            for (int f = 0; f < F; ++f)
                if (rr == 0 || lag[(size_t)rr * F + f] != lag[(size_t)(rr - 1) * F + f]) chg[rr] |= 1u << f;
        std::vector<int> dm32(s->dmax.begin(), s->dmax.end());
        if (cudaMemcpy(s->d_lag, lag.data(), lag.size() * sizeof(int16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_chg, chg.data(), chg.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_member_start, s->member_start.data(), s->member_start.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_member_ord, s->member_ord.data(), s->member_ord.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_ord2d, s->ord2d.data(), s->ord2d.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_dmax, dm32.data(), dm32.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaStreamSynchronize(s->st) != cudaSuccess)
            rc = LPF_E_CUDA;
    }
    if (rc != LPF_OK) {
        free_all(s);
        delete s;
        return rc;
    }
    s->last_stats.assign((size_t)s->n_dm * 2, std::nan(""));
    *out = s;
    return LPF_OK;
}

int lpf_push_frame(lpf_stream* s, const float* frame_dev, int64_t T) {
    int rc = check_push(s, T);
    if (rc != LPF_OK) return rc;
    if (!frame_dev) return LPF_E_ARG;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    return enqueue_push(s, frame_dev, T);
}

int lpf_push_frame_host(lpf_stream* s, const float* frame_host, int64_t T) {
    int rc = check_push(s, T);
    if (rc != LPF_OK) return rc;
    if (!frame_host) return LPF_E_ARG;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    // Double-buffered upload on its own stream: the copy of this frame overlaps
    // the search of the previous one; the stream's work waits for the copy, and
    // the next upload into this buffer waits for this push to finish reading it.
    const int i = s->stage_next;
    float* stage = s->stage + (size_t)i * s->F * s->HW;
    LPF_TRY(cudaStreamWaitEvent(s->h2d_st, s->stage_free[i], 0));
    LPF_TRY(cudaMemcpyAsync(stage, frame_host, sizeof(float) * s->F * s->HW, cudaMemcpyHostToDevice, s->h2d_st));
    LPF_TRY(cudaEventRecord(s->stage_ready[i], s->h2d_st));
    LPF_TRY(cudaStreamWaitEvent(s->st, s->stage_ready[i], 0));
    rc = enqueue_push(s, stage, T);
    if (rc != LPF_OK) return rc;
    LPF_TRY(cudaEventRecord(s->stage_free[i], s->st));
    s->stage_next = i ^ 1;
    return LPF_OK;
}

int lpf_poll_candidates(lpf_stream* s, lpf_candidate* out_host, int cap, int* n_out, int64_t* T_out,
                        int timeout_ms) {
    if (!s || cap < 0 || (cap > 0 && !out_host)) return LPF_E_ARG;
    if (s->pending.empty()) return LPF_E_NODATA;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    const int sl = s->pending.front();
    Slot& slot = s->slots[sl];
    auto t_start = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(slot.done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return LPF_E_CUDA;
        if (timeout_ms >= 0) {
            double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            if (el >= timeout_ms) return LPF_E_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    prof_collect(s, sl);
    if (s->prm.qc) {
        s->last_qc = s->h_qc[sl];
        s->last_qc_T = slot.T;
    }
    // records emitted (may exceed the list), and those the steady mask dropped
    // (among the stored ones); the stored records left are the ones formatted.
    // Without the mask the total found is the emitted count.  With it, records
    // past cand_cap were never checked against the mask, so the total of kept
    // candidates is known only without overflow; with overflow it is reported as
    // the kept records stored, so that out_host always holds min(cap, found).
    const unsigned emitted = s->h_count[2 * sl], dropped = s->h_count[2 * sl + 1];
    const unsigned stored = std::min<unsigned>(emitted, (unsigned)s->prm.cand_cap) - dropped;
    const unsigned found = s->prm.suppress_steady > 0 ? stored : emitted;
    const unsigned ncopy = std::min<unsigned>(stored, (unsigned)cap);
    if (ncopy > 0) {
        LPF_TRY(cudaMemcpyAsync(out_host, slot.d_out, (size_t)ncopy * sizeof(lpf_candidate),
                                cudaMemcpyDeviceToHost, s->copy_st));
        LPF_TRY(cudaStreamSynchronize(s->copy_st));
    }
    // stats of this frame
    std::fill(s->last_stats.begin(), s->last_stats.end(), std::nan(""));
    const double* hs = s->h_stats + (size_t)sl * s->n_distinct * 3;
    for (int rr = 0; rr < slot.n_active; ++rr) {
        double n = hs[rr * 3 + 2];
        double mean = n > 0 ? hs[rr * 3 + 0] / n : 0.0;
        double rms = n > 0 ? std::sqrt(hs[rr * 3 + 1] / n) : 0.0;
        for (int m = s->member_start[rr]; m < s->member_start[rr + 1]; ++m) {
            int d = s->ord2d[s->member_ord[m]];
            s->last_stats[(size_t)d * 2] = mean;
            s->last_stats[(size_t)d * 2 + 1] = rms;
        }
    }
    if (n_out) *n_out = (int)found;
    if (T_out) *T_out = slot.T;
    s->polled = true;
    s->polled_T = slot.T;
    s->polled_slot = sl;
    s->pending.pop_front();
    if (emitted > (unsigned)s->prm.cand_cap || found > (unsigned)cap) return LPF_E_TRUNCATED;
    return LPF_OK;
}

int lpf_extract_dynspec(lpf_stream* s, const lpf_candidate* c_host, int n, int Tw, float* out_dev) {
    if (!s || n < 0 || Tw < 1 || (n > 0 && (!c_host || !out_dev))) return LPF_E_ARG;
    if (Tw > s->depth) return LPF_E_DEPTH;
    if (!s->polled) return LPF_E_NODATA;
    const int64_t T = s->polled_T;
    if (T - Tw + 1 < s->T_first) return LPF_E_STALE;
    if (s->last_T - s->depth + 1 > T - Tw + 1) return LPF_E_STALE;
    if (n == 0) return LPF_OK;
    for (int i = 0; i < n; ++i)
        if (c_host[i].y < 0 || c_host[i].y >= s->H || c_host[i].x < 0 || c_host[i].x >= s->W) return LPF_E_ARG;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    // coordinates staged in page-locked memory, so the copy and the gather stay
    // asynchronous; the staging buffer is refilled once the previous copy has read it
    if (!s->yx_copied && cudaEventCreateWithFlags(&s->yx_copied, cudaEventDisableTiming) != cudaSuccess)
        return LPF_E_CUDA;
    LPF_TRY(cudaEventSynchronize(s->yx_copied));
    if (n > s->h_yx_cap) {
        if (s->h_yx) cudaFreeHost(s->h_yx);
        s->h_yx = nullptr;
        s->h_yx_cap = 0;
        if (cudaMallocHost((void**)&s->h_yx, (size_t)n * sizeof(int2)) != cudaSuccess) {
            cudaGetLastError();
            s->h_yx = nullptr;
            return LPF_E_OOM;
        }
        s->h_yx_cap = n;
    }
    for (int i = 0; i < n; ++i) s->h_yx[i] = make_int2(c_host[i].y, c_host[i].x);
    if (n > s->yx_cap) {
        LPF_TRY(cudaStreamSynchronize(s->st));
        if (s->d_yx) { cudaFree(s->d_yx); s->device_bytes -= (size_t)s->yx_cap * sizeof(int2); }
        s->d_yx = nullptr;
        s->yx_cap = 0;
        int rc = dev_alloc(s, &s->d_yx, (size_t)n);
        if (rc != LPF_OK) return rc;
        s->yx_cap = n;
    }
    LPF_TRY(cudaMemcpyAsync(s->d_yx, s->h_yx, (size_t)n * sizeof(int2), cudaMemcpyHostToDevice, s->st));
    LPF_TRY(cudaEventRecord(s->yx_copied, s->st));
    int slot_first = (int)((T - Tw + 1) % s->ring_n);
    cudaGetLastError();
    switch (s->prm.dtype) {
        case LPF_FP32: launch_dynspec<float>(s, n, Tw, slot_first, out_dev); break;
        case LPF_FP16: launch_dynspec<__half>(s, n, Tw, slot_first, out_dev); break;
        default: launch_dynspec<__nv_bfloat16>(s, n, Tw, slot_first, out_dev); break;
    }
    if (cudaGetLastError() != cudaSuccess) return LPF_E_CUDA;
    return LPF_OK;
}

int lpf_get_delay_table(const lpf_stream* s, int32_t* out) {
    if (!s || !out) return LPF_E_ARG;
    std::memcpy(out, s->delay.data(), s->delay.size() * sizeof(int32_t));
    return LPF_OK;
}

int lpf_get_stats(const lpf_stream* s, double* out) {
    if (!s || !out) return LPF_E_ARG;
    if (!s->polled) return LPF_E_NODATA;
    std::memcpy(out, s->last_stats.data(), s->last_stats.size() * sizeof(double));
    return LPF_OK;
}

int lpf_get_qc(const lpf_stream* s, int64_t* T_out, uint32_t* discarded, float* z) {
    if (!s) return LPF_E_ARG;
    if (!s->prm.qc || s->last_qc_T < 0) return LPF_E_NODATA;
    if (T_out) *T_out = s->last_qc_T;
    if (discarded) *discarded = s->last_qc.discarded;
    if (z) std::memcpy(z, s->last_qc.z, sizeof(float) * s->F);
    return LPF_OK;
}

int lpf_stream_info(const lpf_stream* s, lpf_stream_info_t* out) {
    if (!s || !out) return LPF_E_ARG;
    out->H = s->H; out->W = s->W; out->F = s->F; out->n_dm = s->n_dm; out->depth = s->depth;
    out->dtype = s->prm.dtype; out->n_distinct = s->n_distinct; out->max_delay = s->max_delay;
    out->ring_bytes = (size_t)s->ring_n * s->F * s->P * s->elem;
    out->device_bytes = s->device_bytes;
    out->frames_pushed = s->frames_pushed;
    out->last_T = s->last_T;
    return LPF_OK;
}

int lpf_stream_sync(lpf_stream* s) {
    if (!s) return LPF_E_ARG;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    int rc = cuda_fail(cudaStreamSynchronize(s->st));
    if (rc == LPF_OK && s->filt_st) rc = cuda_fail(cudaStreamSynchronize(s->filt_st));
    if (rc == LPF_OK && s->tail_st) rc = cuda_fail(cudaStreamSynchronize(s->tail_st));
    return rc;
}

int lpf_stream_close(lpf_stream* s) {
    if (!s) return LPF_OK;
    free_all(s);
    delete s;
    return LPF_OK;
}

int lpf_set_profiling(lpf_stream* s, int on) {
    if (!s) return LPF_E_ARG;
    s->profiling = on != 0;
    return LPF_OK;
}

int lpf_get_kernel_times(lpf_stream* s, const char** names, double* total_ms, int64_t* launches, int n,
                         int reset) {
    if (!s) return LPF_E_ARG;
    for (int i = 0; i < ST_N && i < n; ++i) {
        if (names) names[i] = kStageNames[i];
        if (total_ms) total_ms[i] = s->prof_ms[i];
        if (launches) launches[i] = s->prof_n[i];
    }
    if (reset)
        for (int i = 0; i < ST_N; ++i) { s->prof_ms[i] = 0; s->prof_n[i] = 0; }
    return ST_N;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Dynamic-spectrum gather for callers that cannot allocate device memory.
//
// lpf_extract_dynspec copies the caller's candidate list to a device buffer
// that it grows with cudaMalloc when a call brings more candidates than any
// earlier one.  This variant stages the candidate records in a fixed array in
// device global memory instead, declared at file scope below, so the call
// itself allocates nothing.  The array (LPF_STATIC_DYNSPEC_MAX records of 24
// bytes, 1.5 MiB) exists on every GPU that loads the library, until exit.
namespace {

static_assert(sizeof(lpf::CandidateRec) == sizeof(lpf_candidate), "record layouts differ");

static __device__ __align__(256) lpf::CandidateRec g_dynspec_records[LPF_STATIC_DYNSPEC_MAX];

constexpr int kMaxDevices = 64;
std::mutex g_records_mu;
lpf::CandidateRec* g_records_ptr[kMaxDevices] = {};

// Device address of g_dynspec_records on the current device `dev`.  In host
// code the array's name is only a host-side stand-in, so the address is looked
// up once per device (cudaGetSymbolAddress, with that device current) and kept.
int records_on_device(int dev, lpf::CandidateRec** out) {
    if (dev < 0 || dev >= kMaxDevices) return LPF_E_CUDA;
    std::lock_guard<std::mutex> lock(g_records_mu);
    if (!g_records_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dynspec_records) != cudaSuccess || !p) {
            cudaGetLastError();
            return LPF_E_CUDA;
        }
        g_records_ptr[dev] = static_cast<lpf::CandidateRec*>(p);
    }
    *out = g_records_ptr[dev];
    return LPF_OK;
}

// Same gather as lpf::k_dynspec, reading each pixel from a candidate record.
template <typename TS>
__global__ void k_dynspec_records(const TS* __restrict__ ring, const lpf::CandidateRec* __restrict__ c,
                                  int n, int F, int Tw, int depth, int slot_first, int64_t P, int H,
                                  int W, int box_r, float* __restrict__ out) {
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
        const int y = c[i].y, x = c[i].x;
        float v;
        if (box_r == 0) {
            v = lpf::ld1(plane + (int64_t)y * W + x);
        } else {
            v = -INFINITY;
            int ylo = max(y - box_r, 0), yhi = min(y + box_r, H - 1);
            int xlo = max(x - box_r, 0), xhi = min(x + box_r, W - 1);
            for (int yy = ylo; yy <= yhi; ++yy)
                for (int xx = xlo; xx <= xhi; ++xx) v = fmaxf(v, lpf::ld1(plane + (int64_t)yy * W + xx));
        }
        out[idx] = v;
    }
}

template <typename TS>
void launch_dynspec_records(lpf_stream* s, const lpf::CandidateRec* rec, int n, int Tw, int slot_first,
                            float* out) {
    int64_t total = (int64_t)n * s->F * Tw;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 32);
    if (blocks < 1) blocks = 1;
    k_dynspec_records<TS><<<blocks, 256, 0, s->st>>>(reinterpret_cast<const TS*>(s->ring), rec, n, s->F, Tw,
                                                     s->ring_n, slot_first, s->P, s->H, s->W,
                                                     s->prm.dyn_box_r, out);
}

}  // namespace

extern "C" int lpf_extract_dynspec_static(lpf_stream* s, const lpf_candidate* c_host, int n, int Tw,
                                          float* out_dev) {
    // the checks of lpf_extract_dynspec, in its order; the capacity last
    if (!s || n < 0 || Tw < 1 || (n > 0 && (!c_host || !out_dev))) return LPF_E_ARG;
    if (Tw > s->depth) return LPF_E_DEPTH;
    if (!s->polled) return LPF_E_NODATA;
    const int64_t T = s->polled_T;
    if (T - Tw + 1 < s->T_first) return LPF_E_STALE;
    if (s->last_T - s->depth + 1 > T - Tw + 1) return LPF_E_STALE;
    if (n == 0) return LPF_OK;
    for (int i = 0; i < n; ++i)
        if (c_host[i].y < 0 || c_host[i].y >= s->H || c_host[i].x < 0 || c_host[i].x >= s->W) return LPF_E_ARG;
    if (n > LPF_STATIC_DYNSPEC_MAX) return LPF_E_CAPACITY;
    if (cudaSetDevice(s->dev) != cudaSuccess) return LPF_E_CUDA;
    lpf::CandidateRec* rec = nullptr;
    int rc = records_on_device(s->dev, &rec);
    if (rc != LPF_OK) return rc;
    // every call writes the records it reads: nothing carries over between calls
    LPF_TRY(cudaMemcpyAsync(rec, c_host, (size_t)n * sizeof(lpf_candidate), cudaMemcpyHostToDevice, s->st));
    const int slot_first = (int)((T - Tw + 1) % s->ring_n);
    cudaGetLastError();
    switch (s->prm.dtype) {
        case LPF_FP32: launch_dynspec_records<float>(s, rec, n, Tw, slot_first, out_dev); break;
        case LPF_FP16: launch_dynspec_records<__half>(s, rec, n, Tw, slot_first, out_dev); break;
        default: launch_dynspec_records<__nv_bfloat16>(s, rec, n, Tw, slot_first, out_dev); break;
    }
    if (cudaGetLastError() != cudaSuccess) return LPF_E_CUDA;
    // the shared staging array is free for the next call once this returns
    LPF_TRY(cudaStreamSynchronize(s->st));
    return LPF_OK;
}
