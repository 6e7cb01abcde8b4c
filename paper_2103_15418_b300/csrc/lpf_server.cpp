// Serving loop: several concurrent image streams on one GPU (see include/lpf.h).
//
// A persistent worker thread owns every lpf_stream handle.  Each tick it
//   1. admits requested streams, in request order, while the next one's device
//      footprint fits the HBM budget left by the admitted streams;
//   2. for every admitted stream, moves queued frames onto the GPU while the
//      stream has a free result slot (each stream runs on its own CUDA stream,
//      so the work of different streams overlaps on the device: a frame that
//      arrives while others are on the GPU starts as soon as its stream has a
//      free slot, not after the others finish);
//   3. polls in-flight frames without blocking and moves finished ones to the
//      stream's result queue with their submit-to-done latency;
//   4. closes streams whose close was requested once they are drained, which
//      returns their budget to the streams still waiting.
// Callers only touch queues under the server mutex; no CUDA call is made on
// their threads except the pinned-buffer allocation at request time.
#include "../../include/lpf.h"

#include <cuda_runtime_api.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Frame {
    float* host = nullptr;        // pinned buffer of the stream's pool
    int64_t T = 0;
    Clock::time_point submitted;
};

struct Result {
    int64_t T = 0;
    int rc = LPF_OK;
    int n_found = 0;
    double latency_ms = 0.0;
    std::vector<lpf_candidate> cands;
};

struct ServedStream {
    int id = 0;
    int state = LPF_SERVE_PENDING;
    // request
    int H = 0, W = 0, F = 0, n_dm = 0, depth = 0;
    std::vector<double> freqs, dms;
    lpf_params prm{};
    size_t footprint = 0;
    // runtime
    lpf_stream* s = nullptr;
    std::vector<float*> pool;      // pinned frame buffers
    std::vector<float*> free_bufs;
    std::deque<Frame> queued;      // submitted, not yet on the GPU
    std::deque<Frame> inflight;    // pushed, not yet polled
    std::deque<Result> done;       // finished, not yet fetched
    lpf_candidate* poll_buf = nullptr;     // pinned, cand_cap records, reused by every poll
    bool close_requested = false;
    int last_rc = LPF_OK;
    std::vector<double> latencies;
    int64_t frames_done = 0;
    Clock::time_point first_submit{};
    Clock::time_point last_done{};
    bool any_submit = false;
};

}  // namespace

struct lpf_server {
    size_t budget = 0;
    size_t used = 0;
    int max_streams = 0;
    int queue_frames = 4;
    int dev = 0;
    std::mutex mu;
    std::condition_variable cv;        // wakes the worker
    std::condition_variable done_cv;   // wakes fetchers
    std::vector<std::unique_ptr<ServedStream>> streams;
    std::thread worker;
    bool stop = false;
    int worker_error = LPF_OK;
};

namespace {

ServedStream* find(lpf_server* srv, int id) {
    if (id < 0 || id >= (int)srv->streams.size()) return nullptr;
    return srv->streams[id].get();
}

void release_pool(ServedStream* st) {
    for (float* p : st->pool) cudaFreeHost(p);
    st->pool.clear();
    st->free_bufs.clear();
    if (st->poll_buf) cudaFreeHost(st->poll_buf);
    st->poll_buf = nullptr;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    double pos = q * (v.size() - 1);
    size_t lo = (size_t)pos;
    size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

// One pass of the worker over every stream; returns true if anything progressed.
bool tick(lpf_server* srv, std::unique_lock<std::mutex>& lk) {
    bool progress = false;
    // 1. admission in request order
    for (auto& up : srv->streams) {
        ServedStream* st = up.get();
        if (st->state != LPF_SERVE_PENDING) continue;
        if (st->close_requested && st->queued.empty()) {
            st->state = LPF_SERVE_CLOSED;
            release_pool(st);
            progress = true;
            continue;
        }
        if (srv->used + st->footprint > srv->budget) break;      // keep request order
        lpf_stream* s = nullptr;
        lpf_params p = st->prm;
        p.cuda_stream = nullptr;                                 // each stream its own CUDA stream
        lk.unlock();
        int rc = lpf_stream_open(&s, st->H, st->W, st->F, st->freqs.data(), st->n_dm, st->dms.data(),
                                 st->depth, &p);
        lk.lock();
        if (rc != LPF_OK) {
            st->state = LPF_SERVE_CLOSED;
            st->last_rc = rc;
            release_pool(st);
        } else {
            st->s = s;
            // pinned, so that the candidate copy of every poll is a plain DMA
            if (cudaMallocHost((void**)&st->poll_buf, sizeof(lpf_candidate) * (size_t)st->prm.cand_cap) !=
                cudaSuccess) {
                cudaGetLastError();
                st->poll_buf = nullptr;
                lpf_stream_close(s);
                st->s = nullptr;
                st->state = LPF_SERVE_CLOSED;
                st->last_rc = LPF_E_OOM;
                release_pool(st);
            } else {
                st->state = LPF_SERVE_ACTIVE;
                srv->used += st->footprint;
            }
        }
        progress = true;
    }
    // 2. + 3. feed and poll the admitted streams
    for (auto& up : srv->streams) {
        ServedStream* st = up.get();
        if (st->state != LPF_SERVE_ACTIVE) continue;
        while (!st->queued.empty() && (int)st->inflight.size() < st->prm.result_slots) {
            Frame fr = st->queued.front();
            int rc = lpf_push_frame_host(st->s, fr.host, fr.T);
            if (rc == LPF_E_BUSY) break;
            st->queued.pop_front();
            if (rc != LPF_OK) {
                Result r;
                r.T = fr.T;
                r.rc = rc;
                st->done.push_back(std::move(r));
                st->free_bufs.push_back(fr.host);
                srv->done_cv.notify_all();
            } else {
                st->inflight.push_back(fr);
            }
            progress = true;
        }
        while (!st->inflight.empty()) {
            Result r;
            int n = 0;
            int64_t T = -1;
            int rc = lpf_poll_candidates(st->s, st->poll_buf, st->prm.cand_cap, &n, &T, 0);
            if (rc == LPF_E_TIMEOUT) break;
            Frame fr = st->inflight.front();
            st->inflight.pop_front();
            auto now = Clock::now();
            r.T = fr.T;
            r.rc = rc;
            r.n_found = n;
            r.latency_ms = std::chrono::duration<double, std::milli>(now - fr.submitted).count();
            r.cands.assign(st->poll_buf, st->poll_buf + std::min(n, st->prm.cand_cap));
            st->latencies.push_back(r.latency_ms);
            st->frames_done += 1;
            st->last_done = now;
            st->done.push_back(std::move(r));
            st->free_bufs.push_back(fr.host);
            srv->done_cv.notify_all();
            progress = true;
        }
        // 4. drained close
        if (st->close_requested && st->queued.empty() && st->inflight.empty()) {
            lpf_stream_close(st->s);
            st->s = nullptr;
            srv->used -= st->footprint;
            st->state = LPF_SERVE_CLOSED;
            release_pool(st);
            srv->done_cv.notify_all();
            progress = true;
        }
    }
    return progress;
}

void worker_main(lpf_server* srv) {
    cudaSetDevice(srv->dev);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (!srv->stop) {
        bool progress = tick(srv, lk);
        if (!progress) srv->cv.wait_for(lk, std::chrono::microseconds(50));
    }
    // shut down: wait for every admitted stream's work, then release everything
    for (auto& up : srv->streams) {
        ServedStream* st = up.get();
        if (st->s) {
            lpf_stream_close(st->s);
            st->s = nullptr;
        }
        release_pool(st);
        st->state = LPF_SERVE_CLOSED;
    }
}

}  // namespace

extern "C" {

int lpf_server_open(lpf_server** out, size_t hbm_budget_bytes, int max_streams) {
    if (!out || hbm_budget_bytes == 0 || max_streams < 1) return LPF_E_ARG;
    *out = nullptr;
    int dev = 0, ndev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return LPF_E_CUDA;
    }
    lpf_server* srv = new (std::nothrow) lpf_server();
    if (!srv) return LPF_E_OOM;
    srv->budget = hbm_budget_bytes;
    srv->max_streams = max_streams;
    srv->dev = dev;
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return LPF_OK;
}

int lpf_server_open_stream(lpf_server* srv, int H, int W, int F, const double* freqs_mhz, int n_dm,
                           const double* dm_grid, int buffer_depth, const lpf_params* params,
                           int* id_out) {
    if (!srv || !id_out) return LPF_E_ARG;
    size_t fp = 0;
    int rc = lpf_stream_footprint(H, W, F, freqs_mhz, n_dm, dm_grid, buffer_depth, params, &fp);
    if (rc != LPF_OK) return rc;
    if (fp > srv->budget) return LPF_E_BUDGET;
    auto st = std::make_unique<ServedStream>();
    st->H = H; st->W = W; st->F = F; st->n_dm = n_dm; st->depth = buffer_depth;
    st->freqs.assign(freqs_mhz, freqs_mhz + F);
    st->dms.assign(dm_grid, dm_grid + n_dm);
    lpf_default_params(&st->prm);
    if (params) st->prm = *params;
    st->footprint = fp;
    // pinned frame buffers: one per result slot plus the submit queue
    const int nbuf = st->prm.result_slots + srv->queue_frames;
    for (int i = 0; i < nbuf; ++i) {
        float* p = nullptr;
        if (cudaMallocHost((void**)&p, sizeof(float) * (size_t)F * H * W) != cudaSuccess) {
            cudaGetLastError();
            release_pool(st.get());
            return LPF_E_OOM;
        }
        st->pool.push_back(p);
        st->free_bufs.push_back(p);
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    int live = 0;
    for (auto& up : srv->streams)
        if (up->state != LPF_SERVE_CLOSED) ++live;
    if (live >= srv->max_streams) {
        release_pool(st.get());
        return LPF_E_BUSY;
    }
    st->id = (int)srv->streams.size();
    *id_out = st->id;
    srv->streams.push_back(std::move(st));
    srv->cv.notify_all();
    return LPF_OK;
}

int lpf_server_submit(lpf_server* srv, int id, const float* frame_host, int64_t T) {
    if (!srv || !frame_host) return LPF_E_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    ServedStream* st = find(srv, id);
    if (!st || st->state == LPF_SERVE_CLOSED || st->close_requested) return LPF_E_ARG;
    if (st->free_bufs.empty()) return LPF_E_BUSY;
    float* buf = st->free_bufs.back();
    st->free_bufs.pop_back();
    lk.unlock();
    std::memcpy(buf, frame_host, sizeof(float) * (size_t)st->F * st->H * st->W);
    lk.lock();
    Frame fr;
    fr.host = buf;
    fr.T = T;
    fr.submitted = Clock::now();
    if (!st->any_submit) {
        st->any_submit = true;
        st->first_submit = fr.submitted;
    }
    st->queued.push_back(fr);
    srv->cv.notify_all();
    return LPF_OK;
}

int lpf_server_fetch(lpf_server* srv, int id, lpf_candidate* out_host, int cap, int* n_out, int64_t* T_out,
                     double* latency_ms, int timeout_ms) {
    if (!srv || cap < 0 || (cap > 0 && !out_host)) return LPF_E_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    ServedStream* st = find(srv, id);
    if (!st) return LPF_E_ARG;
    auto ready = [&] { return !st->done.empty(); };
    if (!ready()) {
        if (st->state == LPF_SERVE_CLOSED && st->queued.empty() && st->inflight.empty())
            return st->last_rc != LPF_OK ? st->last_rc : LPF_E_NODATA;
        if (timeout_ms < 0) srv->done_cv.wait(lk, [&] { return ready() || st->state == LPF_SERVE_CLOSED; });
        else srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
        if (!ready()) return st->state == LPF_SERVE_CLOSED ? LPF_E_NODATA : LPF_E_TIMEOUT;
    }
    Result r = std::move(st->done.front());
    st->done.pop_front();
    lk.unlock();
    int k = std::min<int>((int)r.cands.size(), cap);
    if (k > 0) std::memcpy(out_host, r.cands.data(), sizeof(lpf_candidate) * (size_t)k);
    if (n_out) *n_out = r.n_found;
    if (T_out) *T_out = r.T;
    if (latency_ms) *latency_ms = r.latency_ms;
    if (r.rc != LPF_OK) return r.rc;
    return r.n_found > cap ? LPF_E_TRUNCATED : LPF_OK;
}

int lpf_server_close_stream(lpf_server* srv, int id) {
    if (!srv) return LPF_E_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    ServedStream* st = find(srv, id);
    if (!st) return LPF_E_ARG;
    st->close_requested = true;
    srv->cv.notify_all();
    return LPF_OK;
}

int lpf_server_stream_state(lpf_server* srv, int id, int* state) {
    if (!srv || !state) return LPF_E_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    ServedStream* st = find(srv, id);
    if (!st) return LPF_E_ARG;
    *state = st->state;
    return LPF_OK;
}

int lpf_server_stats(lpf_server* srv, int id, lpf_serve_stats_t* out) {
    if (!srv || !out) return LPF_E_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<double> lat;
    double pixdm = 0.0;
    Clock::time_point t0 = Clock::time_point::max(), t1 = Clock::time_point::min();
    int64_t frames = 0;
    for (auto& up : srv->streams) {
        ServedStream* st = up.get();
        if (id >= 0 && st->id != id) continue;
        lat.insert(lat.end(), st->latencies.begin(), st->latencies.end());
        frames += st->frames_done;
        pixdm += (double)st->H * st->W * st->n_dm * st->frames_done;
        if (st->any_submit && st->frames_done > 0) {
            t0 = std::min(t0, st->first_submit);
            t1 = std::max(t1, st->last_done);
        }
    }
    out->frames = frames;
    out->p50_ms = percentile(lat, 0.50);
    out->p99_ms = percentile(lat, 0.99);
    out->max_ms = lat.empty() ? 0.0 : *std::max_element(lat.begin(), lat.end());
    double secs = frames > 0 ? std::chrono::duration<double>(t1 - t0).count() : 0.0;
    out->pixel_dm_per_s = secs > 0 ? pixdm / secs : 0.0;
    out->budget_bytes = srv->budget;
    out->used_bytes = srv->used;
    return LPF_OK;
}

int lpf_server_close(lpf_server* srv) {
    if (!srv) return LPF_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return LPF_OK;
}

}  // extern "C"
