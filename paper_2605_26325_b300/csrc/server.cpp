// Serving loop for many reslice sessions (dare_server_*): continuous batching
// over a few stream lanes, live frame ingestion on its own stream; the
// dispatcher thread stamps each completion when it sees the stream's event
// (polled every 20 us while work is in flight).
//
// Ordering.  Each lane runs one batch at a time; a batch first waits on the
// "last ingest" event of every session it reads.  An ingest first waits on
// every busy lane, then calls dare_build_volume on the ingest stream and
// records that session's "last ingest" event.  Requests submitted after an
// ingest therefore see the new frames; requests submitted before it do not.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "dare_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    dare_reslice_req req;
    uint64_t tag;
    double submit_s;
};

struct Ingest {
    dare_session s;
    const uint8_t* frames;
    int32_t n, w, h;
    double px[2];
    std::vector<double> poses;
    uint64_t tag;
    double submit_s;
};

// One queue entry, kept in submission order: a reslice request or an ingest.
struct Item {
    bool is_ingest;
    Pending req;
    Ingest ingest;
};

struct DoneBatch;  // a batch or ingest in flight

}  // namespace

struct dare_server_s {
    dare_server_config cfg{};
    struct Lane {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        void* ws = nullptr;
        size_t ws_bytes = 0;
        void* pin = nullptr;
        size_t pin_bytes = 0;
        bool busy = false;
        DoneBatch* pending = nullptr;  // the batch in flight on this lane
    };
    std::vector<Lane> lanes;
    cudaStream_t ingest_st = nullptr;
    std::map<dare_session, cudaEvent_t> write_ev;
    std::deque<std::pair<cudaEvent_t, DoneBatch*>> ingests_in_flight;  // in stream order
    std::vector<cudaEvent_t> spare_events;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Item> queue;  // submission order
    bool stop = false;
    int64_t in_flight = 0;  // submitted, not yet completed
    std::mutex done_mu;
    std::condition_variable done_cv;
    std::vector<dare_completion> done;
    dare_server_stats stats{};
};

namespace {

struct DoneBatch {
    dare_server sv;
    std::vector<std::pair<uint64_t, double>> items;  // tag, submit time
    int32_t kind;
    int32_t status;
    double issue_s = 0.0;
    int32_t lane = -1;
};

// Hands a finished batch's completions to dare_server_poll; t is when the
// dispatcher saw its stream reach the end of it.  Called without sv->mu held.
void finish(DoneBatch* d, double t) {
    {
        std::lock_guard<std::mutex> lk(d->sv->done_mu);
        for (auto& it : d->items)
            d->sv->done.push_back({it.first, d->status, d->kind, it.second, t, d->issue_s,
                                   static_cast<int32_t>(d->items.size()), d->lane});
        d->sv->stats.completed += static_cast<int64_t>(d->items.size());
    }
    {
        std::lock_guard<std::mutex> lk(d->sv->mu);
        d->sv->in_flight -= static_cast<int64_t>(d->items.size());
    }
    d->sv->done_cv.notify_all();
    d->sv->cv.notify_all();
    delete d;
}

// Completes requests that never reached the GPU.
void complete_now(dare_server sv, DoneBatch* d) {
    (void)sv;
    finish(d, now_s());
}

// A lane's device workspace and pinned staging, allocated once at server creation.
dare_status lane_alloc(dare_server_s::Lane& L, size_t ws_need, size_t pin_need) {
    dare_status rc = dare::reserve_bytes(static_cast<int64_t>(ws_need));
    if (rc != DARE_OK) return rc;
    if (cudaMalloc(&L.ws, ws_need) != cudaSuccess) {
        cudaGetLastError();
        dare::release_bytes(static_cast<int64_t>(ws_need));
        L.ws = nullptr;
        return dare::set_error(DARE_E_OOM, "server lane workspace allocation failed");
    }
    L.ws_bytes = ws_need;
    if (cudaHostAlloc(&L.pin, pin_need, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        L.pin = nullptr;
        return dare::set_error(DARE_E_OOM, "server lane staging allocation failed");
    }
    L.pin_bytes = pin_need;
    return DARE_OK;
}

// The session's last ingest is still running on the device.
bool ingest_running(dare_server sv, dare_session s) {
    auto it = sv->write_ev.find(s);
    return it != sv->write_ev.end() && cudaEventQuery(it->second) == cudaErrorNotReady;
}

// wait_ingests: the batch holds requests of sessions whose last ingest may still
// be running; the lane waits for those ingests first.
void issue_batch(dare_server sv, dare_server_s::Lane& L, std::vector<Pending>& batch, bool wait_ingests) {
    auto* d = new DoneBatch{sv, {}, 0, DARE_OK};
    d->issue_s = now_s();
    d->lane = static_cast<int32_t>(&L - sv->lanes.data());
    std::vector<dare_reslice_req> reqs;
    reqs.reserve(batch.size());
    for (auto& p : batch) {
        reqs.push_back(p.req);
        d->items.push_back({p.tag, p.submit_s});
    }
    const int32_t n = static_cast<int32_t>(reqs.size());
    size_t ws_need = 0, pin_need = 0;
    dare::batch_sizes(reqs.data(), n, &sv->cfg.params, &ws_need, &pin_need);
    if (ws_need > L.ws_bytes || pin_need > L.pin_bytes) {  // excluded by the checks at submission
        d->status = DARE_E_STATE;
        complete_now(sv, d);
        return;
    }
    for (auto& r : reqs) {
        if (wait_ingests) {
            auto it = sv->write_ev.find(r.session);
            if (it != sv->write_ev.end()) cudaStreamWaitEvent(L.st, it->second, 0);
        }
        dare::settle_session(r.session, L.st);  // a reset volume not yet cleared
    }
    dare_status rc = dare::queue_batch(reqs.data(), n, &sv->cfg.params, L.st, static_cast<uint8_t*>(L.ws),
                                       static_cast<uint8_t*>(L.pin));
    if (rc != DARE_OK) d->status = rc;
    if (cudaEventRecord(L.ev, L.st) != cudaSuccess) {
        cudaGetLastError();
        d->status = DARE_E_CUDA;
        cudaStreamSynchronize(L.st);
        complete_now(sv, d);
        return;
    }
    L.pending = d;  // the dispatcher completes it when L.ev is reached
    L.busy = true;
    std::lock_guard<std::mutex> lk(sv->done_mu);
    sv->stats.batches += 1;
    sv->stats.max_batch_seen = std::max<int64_t>(sv->stats.max_batch_seen, n);
}

void run_ingest(dare_server sv, Ingest& g) {
    auto* d = new DoneBatch{sv, {{g.tag, g.submit_s}}, 1, DARE_OK};
    d->issue_s = now_s();
    for (auto& L : sv->lanes)
        if (L.busy) cudaStreamWaitEvent(sv->ingest_st, L.ev, 0);
    dare_status rc = dare_build_volume(g.s, g.frames, g.n, g.w, g.h, g.px, g.poses.data(), sv->ingest_st);
    if (rc != DARE_OK) d->status = rc;
    cudaEvent_t& ev = sv->write_ev[g.s];
    if (!ev) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, sv->ingest_st);
    cudaEvent_t done_ev = nullptr;
    if (!sv->spare_events.empty()) {
        done_ev = sv->spare_events.back();
        sv->spare_events.pop_back();
    } else if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        done_ev = nullptr;
    }
    if (!done_ev || cudaEventRecord(done_ev, sv->ingest_st) != cudaSuccess) {
        cudaGetLastError();
        if (done_ev) sv->spare_events.push_back(done_ev);
        d->status = DARE_E_CUDA;
        cudaStreamSynchronize(sv->ingest_st);
        complete_now(sv, d);
    } else {
        sv->ingests_in_flight.push_back({done_ev, d});
    }
    std::lock_guard<std::mutex> lk(sv->done_mu);
    sv->stats.ingests += 1;
}

// Requests at the front of the queue that can go out as one batch: consecutive,
// up to max_batch, stopping at an ingest.
size_t front_batch(dare_server sv, bool* ingest_follows) {
    size_t n = 0;
    *ingest_follows = false;
    for (const Item& it : sv->queue) {
        if (it.is_ingest) {
            *ingest_follows = true;
            break;
        }
        if (++n == static_cast<size_t>(sv->cfg.max_batch)) break;
    }
    return n;
}

void worker_main(dare_server sv) {
    cudaSetDevice(sv->cfg.device);
    const double window = sv->cfg.coalesce_us * 1e-6;
    std::unique_lock<std::mutex> lk(sv->mu);
    std::vector<DoneBatch*> finished;
    for (;;) {
        // completions: lanes and ingests whose streams have reached their events
        bool any_busy = false;
        for (auto& L : sv->lanes) {
            if (L.busy && cudaEventQuery(L.ev) == cudaSuccess) {
                L.busy = false;
                finished.push_back(L.pending);
                L.pending = nullptr;
            }
            any_busy = any_busy || L.busy;
        }
        while (!sv->ingests_in_flight.empty() && cudaEventQuery(sv->ingests_in_flight.front().first) == cudaSuccess) {
            finished.push_back(sv->ingests_in_flight.front().second);
            sv->spare_events.push_back(sv->ingests_in_flight.front().first);
            sv->ingests_in_flight.pop_front();
        }
        any_busy = any_busy || !sv->ingests_in_flight.empty();
        if (!finished.empty()) {
            const double t = now_s();
            lk.unlock();
            for (DoneBatch* d : finished) finish(d, t);
            lk.lock();
            finished.clear();
        }
        if (sv->stop && sv->queue.empty() && !any_busy) break;
        bool did = false;
        // an ingest runs once every request submitted before it has been issued
        if (!sv->queue.empty() && sv->queue.front().is_ingest) {
            Ingest g = std::move(sv->queue.front().ingest);
            sv->queue.pop_front();
            lk.unlock();
            run_ingest(sv, g);
            lk.lock();
            did = true;
        }
        double wake = 0.0;  // when the front batch's coalescing window closes
        for (auto& L : sv->lanes) {
            if (L.busy || sv->queue.empty() || sv->queue.front().is_ingest) continue;
            // coalescing: a batch that is not full waits until its oldest request is
            // `window` old, unless an ingest behind it or a stop ends the wait
            bool ingest_follows = false;
            const size_t n = front_batch(sv, &ingest_follows);
            const double close = sv->queue.front().req.submit_s + window;
            if (window > 0 && n < static_cast<size_t>(sv->cfg.max_batch) && !ingest_follows && !sv->stop &&
                now_s() < close) {
                wake = close;
                break;
            }
            // requests of a session whose last ingest is still running must wait for it;
            // the others go out at once in a batch of their own, so that an ingest
            // holds up only its own session's requests
            std::vector<Pending> ready, waiting;
            for (size_t k = 0; k < n; ++k) {
                Pending& p = sv->queue.front().req;
                (ingest_running(sv, p.req.session) ? waiting : ready).push_back(p);
                sv->queue.pop_front();
            }
            dare_server_s::Lane* lw = ready.empty() ? &L : nullptr;
            for (auto& L2 : sv->lanes)
                if (!lw && &L2 != &L && !L2.busy) lw = &L2;
            if (!waiting.empty() && !lw)  // no second lane free: back to the front, in order
                for (auto it = waiting.rbegin(); it != waiting.rend(); ++it) sv->queue.push_front(Item{false, *it, Ingest{}});
            lk.unlock();
            if (!ready.empty()) issue_batch(sv, L, ready, false);
            if (!waiting.empty() && lw) issue_batch(sv, *lw, waiting, true);
            lk.lock();
            did = true;
        }
        if (did) continue;
        if (wake > 0) {
            // a batch is coalescing: wait for its window (new work or a stop ends the wait early)
            const double dt = std::min(wake - now_s(), any_busy ? 20e-6 : 1.0);
            if (dt > 0) sv->cv.wait_for(lk, std::chrono::duration<double>(dt));
        } else if (any_busy) {
            // lanes still running: poll again shortly (a free lane or new work ends the wait)
            sv->cv.wait_for(lk, std::chrono::microseconds(20));
        } else {
            sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
        }
    }
}

dare_status err(dare_status st, const char* msg) { return dare::set_error(st, msg); }

}  // namespace

extern "C" {

double dare_clock_seconds(void) { return now_s(); }

dare_status dare_server_create(const dare_server_config* cfg, dare_server* out) {
    if (!cfg || !out) return err(DARE_E_INVALID, "NULL argument");
    *out = nullptr;
    dare_server_config c = *cfg;
    if (c.lanes == 0) c.lanes = 2;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.lanes < 1 || c.lanes > 8 || c.max_batch < 1 || c.max_batch > 4096)
        return err(DARE_E_INVALID, "lanes must be 1..8, max_batch 1..4096");
    if (c.coalesce_us < 0 || c.coalesce_us > 1000000) return err(DARE_E_INVALID, "coalesce_us must be 0..1000000");
    if (c.max_frames == 0) c.max_frames = DARE_MAX_FRAMES;
    if (c.max_frames < 1 || c.max_frames > DARE_MAX_FRAMES) return err(DARE_E_INVALID, "max_frames must be 0..65535");
    dare_status prc = dare::check_batch(nullptr, 0, &c.params);
    if (prc != DARE_OK) return prc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return err(DARE_E_INVALID, "device not available");
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c.device);
    auto* sv = new dare_server_s();
    sv->cfg = c;
    sv->stats.lanes = c.lanes;
    sv->lanes.resize(c.lanes);
    bool ok = cudaStreamCreateWithFlags(&sv->ingest_st, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& L : sv->lanes) {
        ok = ok && cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) == cudaSuccess;
    }
    dare_status arc = DARE_OK;
    if (ok) {
        size_t ws_b = 0, pin_b = 0;
        dare::batch_sizes_bound(c.max_batch, c.max_frames, &ws_b, &pin_b);
        for (auto& L : sv->lanes)
            if (arc == DARE_OK) arc = lane_alloc(L, ws_b, pin_b);
    }
    if (prev != c.device) cudaSetDevice(prev);
    if (!ok) {
        cudaGetLastError();
        dare_server_destroy(sv);
        return err(DARE_E_CUDA, "server stream/event creation failed");
    }
    if (arc != DARE_OK) {
        const std::string msg = dare_last_error();
        dare_server_destroy(sv);
        return err(arc, msg.c_str());
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return DARE_OK;
}

dare_status dare_server_submit(dare_server sv, const dare_reslice_req* req, uint64_t tag) {
    if (!sv || !req) return err(DARE_E_INVALID, "NULL argument");
    dare_status rc = dare::check_batch(req, 1, &sv->cfg.params);
    if (rc != DARE_OK) return rc;
    if (dare::session_device(req->session) != sv->cfg.device) return err(DARE_E_INVALID, "session on another device");
    if (dare::session_max_frames(req->session) > sv->cfg.max_frames)
        return err(DARE_E_INVALID, "the session allows more frames than the server's lanes were sized for");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return err(DARE_E_STATE, "server is stopping");
        sv->queue.push_back(Item{false, Pending{*req, tag, now_s()}, Ingest{}});
        sv->in_flight += 1;
    }
    {
        std::lock_guard<std::mutex> lk(sv->done_mu);
        sv->stats.submitted += 1;
    }
    sv->cv.notify_all();
    return DARE_OK;
}

dare_status dare_server_ingest(dare_server sv, dare_session s, const uint8_t* frames_dev, int32_t n, int32_t width,
                               int32_t height, const double px_mm[2], const double* image_to_world, uint64_t tag) {
    if (!sv || !s || !frames_dev || !px_mm || !image_to_world || n <= 0)
        return err(DARE_E_INVALID, "bad ingest arguments");
    if (dare::session_device(s) != sv->cfg.device) return err(DARE_E_INVALID, "session on another device");
    Ingest g{s, frames_dev, n, width, height, {px_mm[0], px_mm[1]},
             std::vector<double>(image_to_world, image_to_world + 16 * size_t(n)), tag, now_s()};
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return err(DARE_E_STATE, "server is stopping");
        sv->queue.push_back(Item{true, Pending{}, std::move(g)});
        sv->in_flight += 1;
    }
    {
        std::lock_guard<std::mutex> lk(sv->done_mu);
        sv->stats.submitted += 1;
    }
    sv->cv.notify_all();
    return DARE_OK;
}

dare_status dare_server_poll(dare_server sv, dare_completion* out, int32_t capacity, int32_t* n_out) {
    if (!sv || !n_out || capacity < 0 || (capacity > 0 && !out)) return err(DARE_E_INVALID, "bad arguments");
    std::lock_guard<std::mutex> lk(sv->done_mu);
    const int32_t n = static_cast<int32_t>(std::min<size_t>(sv->done.size(), static_cast<size_t>(capacity)));
    std::copy(sv->done.begin(), sv->done.begin() + n, out);
    sv->done.erase(sv->done.begin(), sv->done.begin() + n);
    *n_out = n;
    return DARE_OK;
}

dare_status dare_server_drain(dare_server sv, double timeout_s) {
    if (!sv) return err(DARE_E_INVALID, "server is NULL");
    const double end = now_s() + timeout_s;
    std::unique_lock<std::mutex> lk(sv->mu);
    while (sv->in_flight > 0) {
        if (now_s() > end) return err(DARE_E_TIMEOUT, "drain timed out with requests in flight");
        sv->done_cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    return DARE_OK;
}

dare_status dare_server_stats_get(dare_server sv, dare_server_stats* out) {
    if (!sv || !out) return err(DARE_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->done_mu);
    *out = sv->stats;
    return DARE_OK;
}

dare_status dare_server_destroy(dare_server sv) {
    if (!sv) return DARE_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->cfg.device);
    if (sv->ingest_st) cudaStreamSynchronize(sv->ingest_st);
    for (auto& L : sv->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        if (L.ws) {
            cudaFree(L.ws);
            dare::release_bytes(static_cast<int64_t>(L.ws_bytes));
        }
        if (L.pin) cudaFreeHost(L.pin);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.st) cudaStreamDestroy(L.st);
    }
    for (auto& kv : sv->write_ev) cudaEventDestroy(kv.second);
    for (cudaEvent_t e : sv->spare_events) cudaEventDestroy(e);
    if (sv->ingest_st) cudaStreamDestroy(sv->ingest_st);
    if (prev != sv->cfg.device) cudaSetDevice(prev);
    delete sv;
    return DARE_OK;
}

}  // extern "C"
