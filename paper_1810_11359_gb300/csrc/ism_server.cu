// ism_server.cu -- continuous batching of RIR requests on one GPU (the
// serving loop of include/ism.h).  Host code only: every request is computed
// by ism_simulate_batch, so the arithmetic is that of the other entry points.
//
// Memory: one device pool and one pinned host pool, allocated at create and
// carved by first-fit arenas (256-byte granules, coalescing on release).  A
// request holds, from admission to completion, a device block (its RIRs and
// positions) and a pinned block (positions in, RIRs out); a batch holds a
// device block for its workspace and a pinned word for its status flags.
//
// Threads: the caller's (submit / poll / wait), a launcher and a completer.
// The launcher admits queued requests in arrival order into a batch while
// memory and a stream are free, copies their positions to the device, runs
// the batch on the stream and queues the copies of the results to pinned
// memory, then an event.  The completer polls the events of the batches on
// the GPU, copies finished results to the callers' buffers, frees the
// memory and wakes the launcher and the waiters.  One mutex guards the
// queues, the arenas and the request table.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ism_internal.h"

namespace {

size_t g256(size_t x) { return (x + 255) & ~(size_t)255; }

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, cap) in 256-byte granules.
class Arena {
public:
    void init(size_t cap)
    {
        free_.clear();
        cap_ = cap & ~(size_t)255;
        if (cap_) free_[0] = cap_;
        used_ = 0;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = g256(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                size_t rest = it->second - n;
                size_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = g256(n ? n : 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t cap() const { return cap_; }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0;
};

struct Request {
    ism_ticket id = 0;
    ism_job job{};               // host view: positions point into `pos`, out is the caller's
    std::vector<float> pos;      // n_src * 3 source then n_rcv * 3 receiver coordinates
    size_t out_bytes = 0, pos_bytes = 0;
    size_t dev_off = 0, pin_off = 0;
    bool direct = false;         // out is page-locked: the kernels write the results there
    float* out_dev = nullptr;    // its device-side address (direct requests)
    bool admitted = false, done = false;
    ism_status status = ISM_OK;
    std::string message;
    double t_submit = 0.0, t_ready = 0.0;
};

struct Batch {
    std::vector<Request*> reqs;
    size_t ws_off = 0, ws_bytes = 0, flag_off = 0;
    int stream = -1;
    cudaEvent_t ev = nullptr;
};

}  // namespace

struct ism_server {
    ism_server_config cfg{};
    char* dev = nullptr;
    char* pin = nullptr;
    Arena dev_arena, pin_arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<int> stream_busy;
    std::mutex mu;
    std::condition_variable cv_launch, cv_done, cv_complete;
    std::deque<Request*> queue;
    std::deque<Batch*> inflight;
    std::unordered_map<ism_ticket, Request*> table;
    ism_ticket next_id = 1;
    bool stopping = false;
    bool launcher_done = false;
    bool retry_now = false;        // form_batch failed a request: look at the queue again at once
    std::thread launcher, completer;
    ism_server_stats st{};
    size_t dev_peak = 0;

    void finish(Request* r, ism_status s, const std::string& msg)
    {
        r->status = s;
        r->message = msg;
        r->done = true;
        r->t_ready = now_s();
        if (s == ISM_OK) ++st.completed;
        else ++st.failed;
    }

    void release_request(Request* r)
    {
        if (!r->admitted) return;
        dev_arena.release(r->dev_off, dev_bytes(r));
        pin_arena.release(r->pin_off, pin_bytes(r));
        r->admitted = false;
    }

    // Staging bytes of a request in the pinned pool: [results | positions], or
    // the positions alone when the results go straight to a page-locked `out`.
    static size_t pin_bytes(const Request* r) { return (r->direct ? 0 : g256(r->out_bytes)) + g256(r->pos_bytes); }
    static size_t pin_pos(const Request* r) { return r->pin_off + (r->direct ? 0 : g256(r->out_bytes)); }
    // Device bytes of a request: [results | positions], or the positions alone when the
    // kernels write the results straight into a page-locked `out`.
    static size_t dev_bytes(const Request* r) { return (r->direct ? 0 : g256(r->out_bytes)) + g256(r->pos_bytes); }
    static size_t dev_pos(const Request* r) { return r->dev_off + (r->direct ? 0 : g256(r->out_bytes)); }

    // Admits requests from the head of the queue into a batch (lock held).
    // Returns nullptr when nothing can start now.
    Batch* form_batch()
    {
        int s = -1;
        for (int i = 0; i < (int)stream_busy.size(); ++i)
            if (!stream_busy[i]) {
                s = i;
                break;
            }
        if (s < 0 || queue.empty()) return nullptr;
        Batch* b = new Batch();
        while (!queue.empty() && (int)b->reqs.size() < cfg.max_batch) {
            Request* r = queue.front();
            const size_t need = dev_bytes(r);
            size_t doff = 0, poff = 0;
            if (!dev_arena.alloc(need, &doff)) break;
            if (!pin_arena.alloc(pin_bytes(r), &poff)) {
                dev_arena.release(doff, need);
                break;
            }
            r->dev_off = doff;
            r->pin_off = poff;
            r->admitted = true;
            queue.pop_front();
            b->reqs.push_back(r);
        }
        // the workspace of the batch; shrink the batch until it fits
        while (!b->reqs.empty()) {
            std::vector<ism_job> jobs = device_jobs(b);
            size_t ws = 0;
            if (ism_batch_workspace_size(jobs.data(), (int)jobs.size(), cfg.prec, &ws) != ISM_OK) ws = 0;
            size_t woff = 0, foff = 0;
            if (ws && dev_arena.alloc(ws, &woff)) {
                if (pin_arena.alloc(256, &foff)) {
                    b->ws_off = woff;
                    b->ws_bytes = ws;
                    b->flag_off = foff;
                    break;
                }
                dev_arena.release(woff, ws);
            }
            Request* last = b->reqs.back();
            b->reqs.pop_back();
            release_request(last);
            queue.push_front(last);
        }
        if (b->reqs.empty()) {
            delete b;
            // nothing in flight and the head still does not fit: it never will
            if (inflight.empty() && !queue.empty()) {
                Request* r = queue.front();
                queue.pop_front();
                finish(r, ISM_ERR_OOM, "request does not fit the server's memory budget with its workspace");
                cv_done.notify_all();
                retry_now = true;
            }
            return nullptr;
        }
        b->stream = s;
        b->ev = events[s];
        stream_busy[s] = 1;
        size_t in_use = dev_arena.used();
        if (in_use > dev_peak) dev_peak = in_use;
        return b;
    }

    std::vector<ism_job> device_jobs(Batch* b)
    {
        std::vector<ism_job> jobs;
        for (Request* r : b->reqs) {
            ism_job j = r->job;
            j.out = r->direct ? r->out_dev : reinterpret_cast<float*>(dev + r->dev_off);
            j.pos_src = reinterpret_cast<const float*>(dev + dev_pos(r));
            j.pos_rcv = j.pos_src + 3 * r->job.n_src;
            j.orient_rcv = r->job.mic_pattern != ISM_MIC_OMNI ? j.pos_rcv + 3 * r->job.n_rcv : nullptr;
            j.env_amp = nullptr;
            jobs.push_back(j);
        }
        return jobs;
    }

    // Enqueues the work of a batch on its stream (lock not held).
    ism_status launch(Batch* b, std::string* msg)
    {
        cudaStream_t s = streams[b->stream];
        for (Request* r : b->reqs) {
            char* h = pin + pin_pos(r);
            std::memcpy(h, r->pos.data(), r->pos_bytes);
            if (cudaMemcpyAsync(dev + dev_pos(r), h, r->pos_bytes, cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
                *msg = "position copy failed";
                return ISM_ERR_CUDA;
            }
        }
        std::vector<ism_job> jobs = device_jobs(b);
        ism_status st = ism_simulate_batch(jobs.data(), (int)jobs.size(), cfg.prec, dev + b->ws_off, b->ws_bytes, s);
        if (st != ISM_OK) {
            *msg = ism_last_error_message();
            return st;
        }
        if (cudaMemcpyAsync(pin + b->flag_off, dev + b->ws_off, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess) {
            *msg = "status copy failed";
            return ISM_ERR_CUDA;
        }
        for (Request* r : b->reqs)
            if (!r->direct && cudaMemcpyAsync(pin + r->pin_off, dev + r->dev_off, r->out_bytes, cudaMemcpyDeviceToHost,
                                              s) != cudaSuccess) {
                *msg = "result copy failed";
                return ISM_ERR_CUDA;
            }
        if (cudaEventRecord(b->ev, s) != cudaSuccess) {
            *msg = "event record failed";
            return ISM_ERR_CUDA;
        }
        return ISM_OK;
    }

    void free_batch(Batch* b)
    {
        for (Request* r : b->reqs) release_request(r);
        dev_arena.release(b->ws_off, b->ws_bytes);
        pin_arena.release(b->flag_off, 256);
        stream_busy[b->stream] = 0;
        delete b;
    }

    void launcher_loop()
    {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            Batch* b = stopping ? nullptr : form_batch();
            if (!b) {
                if (stopping) {
                    launcher_done = true;
                    cv_complete.notify_all();
                    break;
                }
                if (retry_now) {
                    retry_now = false;
                    continue;
                }
                cv_launch.wait(lk);
                continue;
            }
            lk.unlock();
            std::string msg;
            ism_status s = launch(b, &msg);
            if (s != ISM_OK) cudaStreamSynchronize(streams[b->stream]);  // nothing of it may still run
            lk.lock();
            ++st.batches;
            if (s != ISM_OK) {
                for (Request* r : b->reqs) finish(r, s, msg);
                free_batch(b);
                cv_done.notify_all();
                continue;
            }
            inflight.push_back(b);
            if ((int)inflight.size() > st.inflight_peak) st.inflight_peak = (int)inflight.size();
            cv_complete.notify_one();
        }
    }

    void completer_loop()
    {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            if (inflight.empty()) {
                if (stopping && launcher_done) break;
                cv_complete.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            // poll the batches in flight without the lock (only this thread removes them),
            // yielding between polls rather than sleeping: a sleep of a few microseconds
            // lasts tens with the kernel's timer slack, and every batch's latency would pay it
            std::vector<Batch*> snap(inflight.begin(), inflight.end());
            lk.unlock();
            std::vector<Batch*> ready;
            for (Batch* b : snap) {
                cudaError_t e = cudaEventQuery(b->ev);
                if (e != cudaErrorNotReady) ready.push_back(b);
            }
            if (ready.empty()) {
                std::this_thread::yield();
                lk.lock();
                continue;
            }
            lk.lock();
            for (Batch* b : ready) inflight.erase(std::find(inflight.begin(), inflight.end(), b));
            lk.unlock();
            std::vector<std::pair<ism_status, std::string>> res;
            for (Batch* b : ready) {
                cudaError_t e = cudaEventQuery(b->ev);
                uint32_t flags = 0;
                std::memcpy(&flags, pin + b->flag_off, sizeof flags);
                ism_status s = ISM_OK;
                std::string msg;
                if (e != cudaSuccess) {
                    s = ISM_ERR_CUDA;
                    msg = cudaGetErrorString(e);
                } else if (flags) {
                    s = ISM_ERR_DEVICE_CHECK;
                    msg = "device check flags set";
                }
                if (s == ISM_OK)
                    for (Request* r : b->reqs)
                        if (!r->direct) std::memcpy(r->job.out, pin + r->pin_off, r->out_bytes);
                res.emplace_back(s, msg);
            }
            lk.lock();
            for (size_t i = 0; i < ready.size(); ++i) {
                for (Request* r : ready[i]->reqs) finish(r, res[i].first, res[i].second);
                free_batch(ready[i]);
            }
            cv_done.notify_all();
            cv_launch.notify_one();
        }
    }
};

namespace {

// Checks one job (arguments as for ism_simulate, host positions strictly
// inside the room, a budget it can fit) and builds its request with copies of
// its positions; nothing is queued.
ism_status prepare_request(ism_server* s, const ism_job* job, Request** out)
{
    *out = nullptr;
    if (!job) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL job");
    if (!job->pos_src || !job->pos_rcv || !job->out)
        return ism_fail_message(ISM_ERR_INVALID_ARG, "pos_src, pos_rcv and out must be host pointers, not NULL");
    if (job->env_amp) return ism_fail_message(ISM_ERR_INVALID_ARG, "env_amp is not available through the server");
    if (job->beta_dev)
        return ism_fail_message(ISM_ERR_INVALID_ARG, "beta_dev is not available through the server (host jobs)");
    if (job->n_src < 1 || job->n_rcv < 1) return ism_fail_message(ISM_ERR_INVALID_ARG, "need n_src, n_rcv >= 1");
    const bool patterned = job->mic_pattern != ISM_MIC_OMNI;
    if (patterned && !job->orient_rcv)
        return ism_fail_message(ISM_ERR_INVALID_ARG, "a polar pattern needs orient_rcv (host pointer, [n_rcv][3])");
    for (int i = 0; patterned && i < job->n_rcv; ++i) {
        const float* o = job->orient_rcv + 3 * i;
        const double oo = (double)o[0] * o[0] + (double)o[1] * o[1] + (double)o[2] * o[2];
        if (!(oo > 0.0) || !(oo < 1e300))
            return ism_fail_message(ISM_ERR_INVALID_ARG, "receiver %d has a zero or non-finite orientation", i);
    }
    for (int i = 0; i < job->n_src; ++i)
        for (int a = 0; a < 3; ++a)
            if (!(job->pos_src[3 * i + a] > 0.0f && (double)job->pos_src[3 * i + a] < job->room.L[a]))
                return ism_fail_message(ISM_ERR_INVALID_ARG, "source %d lies outside the room", i);
    for (int i = 0; i < job->n_rcv; ++i)
        for (int a = 0; a < 3; ++a)
            if (!(job->pos_rcv[3 * i + a] > 0.0f && (double)job->pos_rcv[3 * i + a] < job->room.L[a]))
                return ism_fail_message(ISM_ERR_INVALID_ARG, "receiver %d lies outside the room", i);
    // full validation (and the workspace this job alone would need)
    ism_job probe = *job;
    probe.pos_src = probe.pos_rcv = nullptr;
    probe.orient_rcv = nullptr;
    probe.out = nullptr;
    size_t ws1 = 0;
    ism_status v = ism_batch_workspace_size(&probe, 1, s->cfg.prec, &ws1);
    if (v != ISM_OK) return v;
    int n_S = 0;
    if ((v = ism_rir_length(job->Tmax, job->fs, &n_S)) != ISM_OK) return v;
    Request* r = new Request();
    r->job = *job;
    r->out_bytes = (size_t)job->n_src * job->n_rcv * (size_t)n_S * sizeof(float);
    const int n_vec = job->n_src + job->n_rcv + (patterned ? job->n_rcv : 0);   // positions, then orientations
    r->pos_bytes = (size_t)n_vec * 3 * sizeof(float);
    const size_t need = g256(r->out_bytes) + g256(r->pos_bytes);
    if (need + g256(ws1) > s->dev_arena.cap() || need + 256 > s->pin_arena.cap()) {
        delete r;
        return ism_fail_message(ISM_ERR_OOM, "request needs %zu device bytes with its workspace; the budget is %zu",
                                need + g256(ws1), s->dev_arena.cap());
    }
    r->pos.resize((size_t)n_vec * 3);
    std::memcpy(r->pos.data(), job->pos_src, (size_t)job->n_src * 3 * sizeof(float));
    if (patterned)
        std::memcpy(r->pos.data() + 3 * (job->n_src + job->n_rcv), job->orient_rcv,
                    (size_t)job->n_rcv * 3 * sizeof(float));
    std::memcpy(r->pos.data() + 3 * job->n_src, job->pos_rcv, (size_t)job->n_rcv * 3 * sizeof(float));
    // The kernels run on the server's device, so a page-locked `out` is written directly only
    // if it has an address there: it is looked up with that device current (memory pinned in
    // another device's context without the portable flag has none and takes the staging copy).
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev == s->cfg.device || cudaSetDevice(s->cfg.device) == cudaSuccess) {
        cudaPointerAttributes attr{};
        void* dp = nullptr;
        if (cudaPointerGetAttributes(&attr, job->out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            cudaHostGetDevicePointer(&dp, static_cast<void*>(job->out), 0) == cudaSuccess && dp != nullptr) {
            r->direct = true;
            r->out_dev = static_cast<float*>(dp);
        }
        if (prev >= 0 && prev != s->cfg.device) cudaSetDevice(prev);
    }
    cudaGetLastError();   // a pageable or foreign pointer leaves an error behind
    *out = r;
    return ISM_OK;
}

}  // namespace

extern "C" {

ism_status ism_server_create(const ism_server_config* cfg, ism_server** server)
{
    if (!cfg || !server) return ism_fail_message(ISM_ERR_INVALID_ARG, "cfg and server must not be NULL");
    *server = nullptr;
    ism_server_config c = *cfg;
    if (c.max_inflight == 0) c.max_inflight = 3;
    if (c.max_batch == 0) c.max_batch = 32;
    if (c.host_budget == 0) c.host_budget = c.hbm_budget / 4;
    if (c.max_inflight < 1 || c.max_inflight > 16 || c.max_batch < 1 || c.max_batch > 256)
        return ism_fail_message(ISM_ERR_INVALID_ARG, "need 1 <= max_inflight <= 16 and 1 <= max_batch <= 256");
    if (c.hbm_budget < ((size_t)16 << 20) || c.host_budget < ((size_t)1 << 20))
        return ism_fail_message(ISM_ERR_INVALID_ARG, "hbm_budget must be >= 16 MiB and host_budget >= 1 MiB");
    if (c.prec != ISM_PREC_FP32 && c.prec != ISM_PREC_FP16X2 && c.prec != ISM_PREC_BF16X2 && c.prec != ISM_PREC_LUT &&
        c.prec != ISM_PREC_FP32_DIRECT && c.prec != ISM_PREC_LUT_TEX)
        return ism_fail_message(ISM_ERR_INVALID_ARG, "unknown precision");
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || c.device < 0 || c.device >= n_dev) {
        cudaGetLastError();
        return ism_fail_message(ISM_ERR_CUDA, "CUDA device %d is not available", c.device);
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return ism_fail_message(ISM_ERR_CUDA, "cudaSetDevice failed");
    ism_server* s = new ism_server();
    s->cfg = c;
    if (cudaMalloc(&s->dev, c.hbm_budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ism_fail_message(ISM_ERR_OOM, "cannot allocate %zu device bytes", c.hbm_budget);
    }
    if (cudaHostAlloc(&s->pin, c.host_budget, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->dev);
        delete s;
        return ism_fail_message(ISM_ERR_OOM, "cannot allocate %zu pinned host bytes", c.host_budget);
    }
    s->dev_arena.init(c.hbm_budget);
    s->pin_arena.init(c.host_budget);
    for (int i = 0; i < c.max_inflight; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        s->streams.push_back(st);
        s->events.push_back(ev);
        s->stream_busy.push_back(0);
    }
    s->launcher = std::thread([s] { s->launcher_loop(); });
    s->completer = std::thread([s] { s->completer_loop(); });
    *server = s;
    return ISM_OK;
}

ism_status ism_server_submit(ism_server* s, const ism_job* job, ism_ticket* ticket)
{
    if (!s || !job || !ticket) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL argument");
    return ism_server_submit_batch(s, job, 1, ticket);
}

ism_status ism_server_submit_batch(ism_server* s, const ism_job* jobs, int n_jobs, ism_ticket* tickets)
{
    if (!s || !jobs || !tickets || n_jobs < 1) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL argument or no job");
    std::vector<Request*> rs((size_t)n_jobs, nullptr);
    for (int k = 0; k < n_jobs; ++k) {
        ism_status v = prepare_request(s, jobs + k, &rs[k]);
        if (v != ISM_OK) {
            for (Request* r : rs) delete r;
            if (n_jobs > 1) {
                const std::string m = ism_last_error_message();
                return ism_fail_message(v, "job %d: %s", k, m.c_str());
            }
            return v;
        }
    }
    const double t = now_s();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stopping) {
            for (Request* r : rs) delete r;
            return ism_fail_message(ISM_ERR_CANCELLED, "the server is shutting down");
        }
        for (int k = 0; k < n_jobs; ++k) {
            Request* r = rs[k];
            r->t_submit = t;
            r->id = s->next_id++;
            s->table[r->id] = r;
            s->queue.push_back(r);
            ++s->st.submitted;
            tickets[k] = r->id;
        }
    }
    s->cv_launch.notify_one();
    return ISM_OK;
}

ism_status ism_server_poll(ism_server* s, ism_ticket t, int* done)
{
    if (!s || !done) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->table.find(t);
    if (it == s->table.end()) return ism_fail_message(ISM_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)t);
    *done = it->second->done ? 1 : 0;
    return ISM_OK;
}

ism_status ism_server_wait(ism_server* s, ism_ticket t, double timeout_s, double* latency_s)
{
    if (!s) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(t);
    if (it == s->table.end()) return ism_fail_message(ISM_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)t);
    Request* r = it->second;
    auto pred = [r] { return r->done; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return ism_fail_message(ISM_ERR_TIMEOUT, "request %llu still running", (unsigned long long)t);
    if (latency_s) *latency_s = r->t_ready - r->t_submit;
    ism_status st = r->status;
    std::string msg = r->message;
    s->table.erase(it);
    delete r;
    lk.unlock();
    if (st != ISM_OK) return ism_fail_message(st, "%s", msg.c_str());
    return ISM_OK;
}

ism_status ism_server_stats_read(ism_server* s, ism_server_stats* out)
{
    if (!s || !out) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->dev_in_use = s->dev_arena.used();
    out->dev_peak = s->dev_peak;
    out->host_in_use = s->pin_arena.used();
    out->inflight = (int)s->inflight.size();
    out->queued = (int)s->queue.size();
    return ISM_OK;
}

ism_status ism_server_destroy(ism_server* s)
{
    if (!s) return ism_fail_message(ISM_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stopping = true;
        for (Request* r : s->queue) s->finish(r, ISM_ERR_CANCELLED, "cancelled by ism_server_destroy");
        s->queue.clear();
    }
    s->cv_launch.notify_all();
    s->cv_complete.notify_all();
    s->launcher.join();
    s->completer.join();   // returns once every batch on the GPU has been retired
    s->cv_done.notify_all();
    for (auto& kv : s->table) delete kv.second;
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    cudaFreeHost(s->pin);
    cudaFree(s->dev);
    delete s;
    return ISM_OK;
}

}  // extern "C"
