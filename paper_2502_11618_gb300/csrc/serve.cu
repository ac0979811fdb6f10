// Serving loop: continuous batching of render requests on one GPU.
//
// Requests (pose, resolution, n_levels, filter_strength) are queued by lnr_submit from any
// thread.  A scheduler thread owns `slots` workspaces with their buffers.  Whenever a slot
// is free it takes the oldest queued request and up to max_batch - 1 more of the same
// resolution and pyramid depth, admits them if their activation memory fits the budget next
// to the requests already on the GPU, and launches the batch (a replayed CUDA graph once the
// configuration has been seen).  The frames of all slots run in launch order on one compute
// stream: the conv kernels are persistent (one CTA per SM), and two frames sharing the SMs
// would leave each with part of the GPU and a long tail.  The device-to-host copy of every
// result, into its own pinned buffer, goes on the slot's copy stream after its frame, and
// overlaps the next frames.  Completed requests are picked up by lnr_poll.
//
// Memory: a slot's buffers grow to the largest batch it has run.  Under a budget
// (lnr_set_memory_budget) admission counts the bytes the slots actually hold: a batch is
// launched when the busy slots' buffers plus the batch's own need fit, and before the
// launch the slot's buffers, then idle slots' buffers, are released while the total the
// slots would hold exceeds the budget.  So the device memory of all slots stays within the
// budget whenever one batch of one request fits in it.
// Every wait is bounded: the scheduler polls events, and lnr_serve_stop gives the device a
// deadline before reporting a timeout.
#include <chrono>
#include <cstring>

#include "lnr_internal.h"

namespace lnr {

struct Slot {
    Workspace ws;                     // ws.stream is the server's compute stream (not owned)
    cudaStream_t copy = nullptr;      // the results' device-to-host copies
    cudaEvent_t computed = nullptr;   // the frame is done on the compute stream
    cudaEvent_t done = nullptr;       // and its results are in host memory
    std::vector<uint64_t> tickets;
    bool busy = false;
};

struct PinnedPool {
    std::multimap<size_t, float*> free_;
    float* get(size_t bytes) {
        auto it = free_.lower_bound(bytes);
        if (it != free_.end() && it->first < 2 * bytes) {
            float* p = it->second;
            free_.erase(it);
            return p;
        }
        void* p = nullptr;
        if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
        return static_cast<float*>(p);
    }
    void put(float* p, size_t bytes) { free_.emplace(bytes, p); }
    void release() {
        for (auto& kv : free_) cudaFreeHost(kv.second);
        free_.clear();
    }
};

// Host copy of finished results into the caller's buffer, split across a few persistent
// worker threads: one 1080p RGB frame is 24.9 MB, and a single core's memcpy (~16-27 GB/s
// on the Grace host) would otherwise cap a polling thread near 600 frames/s.
struct CopyPool {
    struct Part {
        char* dst;
        const char* src;
        size_t n;
        std::atomic<int>* left;
    };
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Part> q;
    bool stop = false;

    void start() {
        const unsigned hw = std::thread::hardware_concurrency();
        const int n = (int)std::min(7u, hw > 1 ? hw - 1 : 0u);
        for (int i = 0; i < n; ++i)
            th.emplace_back([this] {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    cv.wait(lk, [this] { return stop || !q.empty(); });
                    if (q.empty()) return;  // stop requested and nothing left
                    Part pt = q.front();
                    q.pop_front();
                    lk.unlock();
                    std::memcpy(pt.dst, pt.src, pt.n);
                    lk.lock();
                    pt.left->fetch_sub(1);
                    done_cv.notify_all();
                }
            });
    }
    void finish() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto& t : th) t.join();
        th.clear();
    }
    // Copies n bytes; returns when every part is done.  Parts of at least 2 MB, one done by
    // the calling thread.
    void copy(void* dst, const void* src, size_t n) {
        const size_t kMin = 2u << 20;
        const int parts = (int)std::min<size_t>(th.size() + 1, std::max<size_t>(1, n / kMin));
        if (parts <= 1) {
            std::memcpy(dst, src, n);
            return;
        }
        const size_t step = (n / parts + 63) & ~(size_t)63;
        std::atomic<int> left(0);
        {
            std::lock_guard<std::mutex> g(mu);
            for (int i = 1; i < parts; ++i) {
                const size_t off = step * i;
                if (off >= n) break;
                left.fetch_add(1);
                q.push_back({static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, std::min(step, n - off), &left});
            }
        }
        cv.notify_all();
        std::memcpy(dst, src, std::min(step, n));
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return left.load() == 0; });
    }
};

struct ServeReq {
    lnr_view view;
    lnr_intrinsics intr;
    int W, H, nlev;
    float fs;
    double t_submit = 0, t_done = 0;
    bool done = false, failed = false;
    float* host = nullptr;  // pinned result, H*W*3 floats
    size_t bytes = 0;
    float* user = nullptr;  // lnr_submit_into: the caller's destination
    bool user_pinned = false;  // ... page-locked: the result is copied straight into it
};

struct Server {
    lnr_ctx* c = nullptr;
    int max_batch = 1;
    cudaStream_t compute = nullptr;  // every slot's frames, in launch order
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, ServeReq> reqs;
    std::thread th;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    PinnedPool pool;
    CopyPool copier;
    lnr_precision prec = LNR_FP32;
    // stats
    uint64_t n_done = 0, n_launch = 0, max_b = 0, peak_bytes = 0, peak_alloc = 0, peak_busy = 0;
    std::string err;

    void loop();
    bool launch(Slot& s, std::vector<uint64_t>& batch, size_t need);
    size_t busy_bytes(const Slot* except) const;
    void make_room(Slot& s, size_t need);
};

// Device bytes a batch of B requests of W x H needs: its U-Net activations and its raster
// buffers (the network input and output included).
static size_t request_bytes(const lnr_ctx* c, int B, int W, int H, lnr_precision p) {
    return unet_act_bytes(c->unet, B, W, H, p) + frame_bytes(c, B, W, H, c->soft_rel > 0.0f);
}

size_t Server::busy_bytes(const Slot* except) const {
    size_t n = 0;
    for (const auto& sp : slots)
        if (sp.get() != except && sp->busy) n += sp->ws.device_bytes();
    return n;
}

// Under a budget: release this slot's buffers when they outgrow the batch, then idle slots'
// buffers, while the slots together would hold more than the budget.
void Server::make_room(Slot& s, size_t need) {
    const size_t budget = c->mem_budget;
    if (!budget) return;
    auto total = [&] {
        size_t n = 0;
        for (const auto& sp : slots) n += sp.get() == &s ? std::max(sp->ws.device_bytes(), need) : sp->ws.device_bytes();
        return n;
    };
    if (total() > budget && s.ws.device_bytes() > need) s.ws.release();
    for (auto& sp : slots) {
        if (total() <= budget) break;
        if (sp.get() != &s && !sp->busy && sp->ws.device_bytes()) sp->ws.release();
    }
}

bool Server::launch(Slot& s, std::vector<uint64_t>& batch, size_t need) {
    const int B = (int)batch.size();
    std::vector<lnr_view> views(B);
    std::vector<lnr_intrinsics> intr(B);
    std::vector<float> fs(B);
    int W, H, nlev;
    {
        std::lock_guard<std::mutex> g(mu);
        for (int i = 0; i < B; ++i) {
            const ServeReq& r = reqs[batch[i]];
            views[i] = r.view;
            intr[i] = r.intr;
            fs[i] = r.fs;
        }
        const ServeReq& r0 = reqs[batch[0]];
        W = r0.W;
        H = r0.H;
        nlev = r0.nlev;
    }
    make_room(s, need);
    if (prepare_views(c, s.ws, B, views.data(), intr.data(), W, H, nlev, fs.data(), prec) != LNR_OK) return false;
    {
        size_t held = 0;
        for (const auto& sp : slots) held += sp->ws.device_bytes();
        std::lock_guard<std::mutex> g(mu);
        peak_alloc = std::max<uint64_t>(peak_alloc, held);
    }
    if (run_frame(c, s.ws, prec, true) != cudaSuccess) return false;
    const size_t per = (size_t)W * H * 3;
    for (int i = 0; i < B; ++i) {
        float* dst;
        {
            std::lock_guard<std::mutex> g(mu);
            ServeReq& r = reqs[batch[i]];
            r.bytes = per * 4;
            if (r.user_pinned) {
                dst = r.user;
            } else {
                if (!r.host) r.host = pool.get(r.bytes);
                dst = r.host;
            }
        }
        if (i == 0 && (cudaEventRecord(s.computed, s.ws.stream) != cudaSuccess ||
                       cudaStreamWaitEvent(s.copy, s.computed, 0) != cudaSuccess))
            return false;
        if (!dst || cudaMemcpyAsync(dst, s.ws.out.as<float>() + i * per, per * 4, cudaMemcpyDeviceToHost, s.copy))
            return false;
    }
    if (cudaEventRecord(s.done, s.copy) != cudaSuccess) return false;
    s.tickets = batch;
    s.busy = true;
    return true;
}

void Server::loop() {
    cudaSetDevice(c->device);
    while (!stop.load()) {
        bool progressed = false;
        // completions
        for (auto& sp : slots) {
            Slot& s = *sp;
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            const double t = now_s();
            std::lock_guard<std::mutex> g(mu);
            for (uint64_t tk : s.tickets) {
                auto it = reqs.find(tk);
                if (it == reqs.end()) continue;
                it->second.done = true;
                it->second.failed = q != cudaSuccess;
                it->second.t_done = t;
                ++n_done;
            }
            if (q != cudaSuccess) err = cudaGetErrorString(q);
            s.busy = false;
            s.tickets.clear();
            progressed = true;
        }
        // admission: the oldest request plus up to max_batch-1 more of its configuration
        for (auto& sp : slots) {
            Slot& s = *sp;
            if (s.busy) continue;
            std::vector<uint64_t> batch;
            size_t bytes = 0;
            {
                std::lock_guard<std::mutex> g(mu);
                if (queue.empty()) break;
                const ServeReq& h = reqs[queue.front()];
                std::vector<size_t> take;
                for (size_t i = 0; i < queue.size() && (int)take.size() < max_batch; ++i) {
                    const ServeReq& r = reqs[queue[i]];
                    if (r.W == h.W && r.H == h.H && r.nlev == h.nlev) take.push_back(i);
                }
                bytes = request_bytes(c, (int)take.size(), h.W, h.H, prec);
                const size_t busy = busy_bytes(&s);
                if (c->mem_budget && busy > 0 && busy + bytes > c->mem_budget) {
                    // shrink the batch until it fits next to the buffers of the busy slots
                    while (take.size() > 1 && busy + request_bytes(c, (int)take.size(), h.W, h.H, prec) > c->mem_budget)
                        take.pop_back();
                    bytes = request_bytes(c, (int)take.size(), h.W, h.H, prec);
                    if (busy + bytes > c->mem_budget) break;  // wait for completions
                }
                for (size_t k = take.size(); k-- > 0;) {
                    batch.insert(batch.begin(), queue[take[k]]);
                    queue.erase(queue.begin() + (long)take[k]);
                }
                peak_bytes = std::max<uint64_t>(peak_bytes, busy + bytes);
            }
            if (!launch(s, batch, bytes)) {
                std::lock_guard<std::mutex> g(mu);
                for (uint64_t tk : batch) {
                    reqs[tk].done = true;
                    reqs[tk].failed = true;
                }
                err = c->err.empty() ? "launch failed" : c->err;
                s.busy = false;
            } else {
                ++n_launch;
                max_b = std::max<uint64_t>(max_b, batch.size());
                uint64_t nb = 0;
                for (const auto& sp : slots) nb += sp->busy ? 1 : 0;
                std::lock_guard<std::mutex> g(mu);
                peak_busy = std::max(peak_busy, nb);
            }
            progressed = true;
        }
        if (!progressed) {
            bool in_flight = false;
            for (const auto& sp : slots) in_flight = in_flight || sp->busy;
            if (in_flight) {
                // frames on the device: poll their events without sleeping.  A thread that
                // sleeps can take milliseconds to run again on a loaded host, and the GPU
                // idles until the next batch is launched.
                std::this_thread::yield();
            } else {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait_for(lk, std::chrono::microseconds(500), [&] { return stop.load() || !queue.empty(); });
            }
        }
    }
}

}  // namespace lnr

using namespace lnr;

extern "C" {

lnr_status lnr_serve_start(lnr_ctx* c, int max_batch, int nslots) {
    if (!c) return LNR_E_ARG;
    if (c->server) return fail(c, LNR_E_STATE, "serving already started");
    if (!c->grid_ok || !c->unet_ok) return fail(c, LNR_E_STATE, "serving needs build_grid and set_unet");
    if (max_batch < 1 || max_batch > 64 || nslots < 1 || nslots > 16) return fail(c, LNR_E_ARG, "bad batch or slot count");
    cudaSetDevice(c->device);
    Server* s = new Server();
    s->c = c;
    s->max_batch = max_batch;
    s->prec = c->prec;
    if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(c, LNR_E_CUDA, "serving streams");
    }
    for (int i = 0; i < nslots; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->ws.stream = s->compute;
        const bool ok = cudaStreamCreateWithFlags(&sl->copy, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaEventCreateWithFlags(&sl->computed, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) == cudaSuccess;
        s->slots.push_back(std::move(sl));
        if (!ok) {
            for (auto& x : s->slots) {
                if (x->copy) cudaStreamDestroy(x->copy);
                if (x->computed) cudaEventDestroy(x->computed);
                if (x->done) cudaEventDestroy(x->done);
            }
            cudaStreamDestroy(s->compute);
            delete s;
            return fail(c, LNR_E_CUDA, "serving streams");
        }
    }
    c->server = s;
    s->copier.start();
    s->th = std::thread([s] { s->loop(); });
    return LNR_OK;
}

lnr_status lnr_serve_stop(lnr_ctx* c) {
    if (!c) return LNR_E_ARG;
    Server* s = c->server;
    if (!s) return LNR_OK;
    s->stop = true;
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    s->copier.finish();
    lnr_status st = LNR_OK;
    cudaSetDevice(c->device);
    const double deadline = now_s() + 10.0;
    auto drain = [&](cudaStream_t q) {
        while (st == LNR_OK && cudaStreamQuery(q) == cudaErrorNotReady) {
            if (now_s() > deadline) {
                st = fail(c, LNR_E_TIMEOUT, "serving stop: device work did not finish in 10 s");
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    };
    drain(s->compute);
    for (auto& sl : s->slots) drain(sl->copy);
    for (auto& sl : s->slots) {
        sl->ws.release();
        cudaStreamDestroy(sl->copy);
        cudaEventDestroy(sl->computed);
        cudaEventDestroy(sl->done);
    }
    cudaStreamDestroy(s->compute);
    for (auto& kv : s->reqs)
        if (kv.second.host) cudaFreeHost(kv.second.host);
    s->pool.release();
    c->server = nullptr;
    delete s;
    return st;
}

lnr_status lnr_set_memory_budget(lnr_ctx* c, size_t bytes) {
    if (!c) return LNR_E_ARG;
    c->mem_budget = bytes;
    return LNR_OK;
}

lnr_status lnr_submit(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* intr, int W, int H, int nlev, float fs,
                      uint64_t* ticket) {
    return lnr_submit_into(c, view, intr, W, H, nlev, fs, nullptr, ticket);
}

lnr_status lnr_submit_into(lnr_ctx* c, const lnr_view* view, const lnr_intrinsics* intr, int W, int H, int nlev,
                           float fs, float* out_rgb, uint64_t* ticket) {
    if (!c || !ticket) return LNR_E_ARG;
    Server* s = c->server;
    if (!s) return fail(c, LNR_E_STATE, "serving not started");
    std::lock_guard<std::mutex> g(s->mu);
    lnr_status st = check_frame_args(c, 1, view, intr, W, H, nlev, &fs, true);
    if (st != LNR_OK) return st;
    ServeReq r;
    r.view = *view;
    r.intr = *intr;
    r.W = W;
    r.H = H;
    r.nlev = nlev;
    r.fs = fs;
    r.user = out_rgb;
    if (out_rgb) {
        cudaPointerAttributes at{};
        r.user_pinned = cudaPointerGetAttributes(&at, out_rgb) == cudaSuccess && at.type == cudaMemoryTypeHost;
        cudaGetLastError();  // a pageable pointer may leave an error behind
    }
    r.t_submit = now_s();
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->queue.push_back(t);
    *ticket = t;
    s->cv.notify_one();
    return LNR_OK;
}

lnr_status lnr_poll(lnr_ctx* c, uint64_t ticket, float* out, double* latency_s) {
    if (!c) return LNR_E_ARG;
    Server* s = c->server;
    if (!s) return fail(c, LNR_E_STATE, "serving not started");
    ServeReq r;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(c, LNR_E_ARG, "unknown ticket");
        if (!it->second.done) return LNR_E_BUSY;
        r = it->second;
        s->reqs.erase(it);
    }
    lnr_status st = LNR_OK;
    if (!out && !r.user_pinned) out = r.user;  // lnr_submit_into with a pageable destination
    if (r.failed) st = fail(c, LNR_E_CUDA, "request failed: " + s->err);
    else if (out && r.host) s->copier.copy(out, r.host, r.bytes);
    else if (out && r.user_pinned && out != r.user) std::memcpy(out, r.user, r.bytes);
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    if (r.host) {
        std::lock_guard<std::mutex> g(s->mu);
        s->pool.put(r.host, r.bytes);
    }
    return st;
}

lnr_status lnr_serve_stats(lnr_ctx* c, uint64_t out[6]) {
    if (!c || !out) return LNR_E_ARG;
    Server* s = c->server;
    if (!s) {
        for (int i = 0; i < 6; ++i) out[i] = 0;
        return LNR_OK;
    }
    std::lock_guard<std::mutex> g(s->mu);
    out[0] = s->n_done;
    out[1] = s->n_launch;
    out[2] = s->max_b;
    out[3] = s->peak_bytes;
    out[4] = s->peak_alloc;
    out[5] = s->peak_busy;
    return LNR_OK;
}

}  // extern "C"
