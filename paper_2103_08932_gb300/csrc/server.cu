// server.cu — served relaxation with continuous batching.
//
// Requests (lattice body descriptions) arrive on any host thread and wait in
// a bounded queue.  One worker thread owns the GPU work: it admits requests
// while slots and the device-memory budget allow, builds their bodies on
// the server stream, relaxes every live body together as one batch in
// chunks of steps (batch.cu: shared launches, colour-synchronised damping
// sweep, per-body retirement), and after every chunk retires the bodies
// that met their own KE criterion (their displacement goes to the host,
// their memory back to the budget) and admits waiting requests into the
// freed slots.  A body's result is bitwise the same whether it ran alone or
// in the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "srdr_internal.cuh"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    srdr_body_desc desc;
    double t_submit;
    size_t est_bytes;
};

struct Result {
    srdr_status status;
    std::vector<double> disp;
    double latency;
    int64_t steps;
};

struct Live {
    uint64_t ticket;
    srdr_body* body;
    double t_submit;
    size_t bytes;
    int64_t steps;
};

// device bytes of a body of n particles, before it exists (admission)
size_t estimate_bytes(const srdr_body_desc& d, int64_t n)
{
    const double k = d.dim == 3 ? 80.0 : 20.0;       // neighbours per particle
    const double t = d.precision == SRDR_FP64 ? 8.0 : 4.0;
    const double per_pair = (4 + 2 + t) + 1.15 * (4 + 3 * t);  // CSR + padded sliced ELL
    const double per_particle = 24 + 8 + 1 + 4 * t + 3 * t * 2 + 9 * t * 2 + 12 * t + 64 + 32;
    return (size_t)(n * (per_particle + k * per_pair)) + (1u << 20);
}

}  // namespace

struct srdr_server {
    size_t budget = 0;
    size_t in_use = 0;
    size_t queue_cap = 4096;
    int max_bodies = 256;
    double ke_ratio = 1e-8;
    int64_t max_steps = 1000000;
    int64_t chunk = 256;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::map<uint64_t, Result> results;
    std::map<uint64_t, int> in_flight;  // admitted, not finished
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    // statistics
    std::vector<double> latencies;
    int64_t submitted = 0, completed = 0, refused = 0;
    int64_t not_converged = 0, failed = 0;
    int peak_live = 0;
    double t_first_submit = 0, t_last_done = 0;
    int64_t particle_steps = 0;
};

namespace {

void finish(srdr_server* s, Live& l, srdr_status st)
{
    Result r;
    r.status = st;
    r.steps = l.steps;
    if (l.body) {
        if (st == SRDR_OK || st == SRDR_ERR_NOT_CONVERGED) {
            r.disp.resize((size_t)l.body->n * 3);
            srdr_status rs = srdr_body_read_displacement(l.body, r.disp.data(), r.disp.size());
            if (rs != SRDR_OK) r.status = rs;
        }
        srdr_body_destroy(l.body);
        l.body = nullptr;
    }
    const double t = now_s();
    r.latency = t - l.t_submit;
    std::lock_guard<std::mutex> lock(s->mu);
    s->in_use -= std::min(s->in_use, l.bytes);
    s->in_flight.erase(l.ticket);
    // only a request that met its KE criterion counts as a solve (and in the
    // latency percentiles); one retired at the step cap or by an error is
    // counted apart
    if (r.status == SRDR_OK) {
        s->latencies.push_back(t - l.t_submit);
        s->completed += 1;
    } else if (r.status == SRDR_ERR_NOT_CONVERGED) {
        s->not_converged += 1;
    } else {
        s->failed += 1;
    }
    s->results[l.ticket] = std::move(r);
    s->t_last_done = t;
    s->cv_done.notify_all();
}

void worker_main(srdr_server* s)
{
    cudaSetDevice(s->device);
    std::vector<Live> live;
    srdr_batch* batch = nullptr;
    bool dirty = true;
    int tuning[4] = {0, 0, 0, 0};  // the tuned launch configuration, once a batch has one
    for (;;) {
        // admission: slots and device-memory budget
        std::vector<Request> take;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (live.empty())
                s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) break;
            while (!s->queue.empty() && (int)(live.size() + take.size()) < s->max_bodies &&
                   s->in_use + s->queue.front().est_bytes <= s->budget) {
                take.push_back(s->queue.front());
                s->in_use += s->queue.front().est_bytes;
                s->in_flight[s->queue.front().ticket] = 1;
                s->queue.pop_front();
            }
        }
        for (Request& r : take) {
            Live l{r.ticket, nullptr, r.t_submit, r.est_bytes, 0};
            srdr_status st = srdr_body_create(&r.desc, s->stream, &l.body);
            if (st != SRDR_OK) {
                l.body = nullptr;
                finish(s, l, st);
                continue;
            }
            live.push_back(l);
            dirty = true;
        }
        if (live.empty()) continue;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->peak_live = std::max(s->peak_live, (int)live.size());
        }
        if (dirty) {
            // the new batch keeps the launch configuration the first batch
            // tuned (its bodies have moved, so it cannot tune itself)
            if (batch) {
                int cfg[4];
                srdr::batch_get_tuning(batch, cfg);
                if (cfg[0]) std::copy(cfg, cfg + 4, tuning);
                srdr_batch_destroy(batch);
            }
            batch = nullptr;
            std::vector<srdr_body*> bodies;
            for (Live& l : live) bodies.push_back(l.body);
            srdr_status st = srdr_batch_create(bodies.data(), (int)bodies.size(), s->stream, &batch);
            if (st != SRDR_OK) {
                for (Live& l : live) finish(s, l, st);
                live.clear();
                batch = nullptr;
                continue;
            }
            srdr::batch_set_tuning(batch, tuning);
            dirty = false;
        }
        // one chunk of batched steps; every body stops at its own criterion
        std::vector<srdr_status> per(live.size(), SRDR_OK);
        std::vector<int64_t> steps(live.size(), 0);
        srdr_status st = srdr_batch_run(batch, s->ke_ratio, s->chunk, per.data(), steps.data());
        if (st == SRDR_ERR_TIMEOUT || st == SRDR_ERR_CUDA || st == SRDR_ERR_INVALID) {
            for (Live& l : live) finish(s, l, st);
            live.clear();
            srdr_batch_destroy(batch);
            batch = nullptr;
            dirty = true;
            continue;
        }
        std::vector<Live> keep;
        for (size_t k = 0; k < live.size(); ++k) {
            Live& l = live[k];
            l.steps += steps[k];
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->particle_steps += steps[k] * l.body->n;
            }
            if (per[k] == SRDR_OK) {
                finish(s, l, SRDR_OK);
            } else if (per[k] == SRDR_ERR_NONFINITE) {
                finish(s, l, SRDR_ERR_NONFINITE);
            } else if (l.steps >= s->max_steps) {
                finish(s, l, SRDR_ERR_NOT_CONVERGED);
            } else {
                keep.push_back(l);
            }
        }
        if (keep.size() != live.size()) dirty = true;
        live.swap(keep);
    }
    if (batch) srdr_batch_destroy(batch);
    for (Live& l : live) finish(s, l, SRDR_ERR_NOT_CONVERGED);
}

}  // namespace

using namespace srdr;

extern "C" {

srdr_status srdr_server_create(size_t device_mem_budget, void* cuda_stream, srdr_server** out)
{
    if (!out || device_mem_budget == 0) {
        set_error("need an output handle and a non-zero memory budget");
        return SRDR_ERR_INVALID;
    }
    *out = nullptr;
    srdr_server* s = new (std::nothrow) srdr_server();
    if (!s) {
        set_error("host allocation failed");
        return SRDR_ERR_NO_MEMORY;
    }
    s->budget = device_mem_budget;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        set_error("no CUDA device");
        return SRDR_ERR_CUDA;
    }
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            set_error("cudaStreamCreate failed");
            return SRDR_ERR_CUDA;
        }
        s->own_stream = true;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SRDR_OK;
}

srdr_status srdr_server_configure(srdr_server* s, double ke_ratio, int64_t max_steps, int max_bodies,
                                  int64_t chunk_steps, size_t queue_capacity)
{
    if (!s || !(ke_ratio > 0) || max_steps < 1 || max_bodies < 1 || chunk_steps < 1 ||
        queue_capacity < 1) {
        set_error("bad server configuration");
        return SRDR_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->ke_ratio = ke_ratio;
    s->max_steps = max_steps;
    s->max_bodies = max_bodies;
    s->chunk = chunk_steps;
    s->queue_cap = queue_capacity;
    return SRDR_OK;
}

srdr_status srdr_server_submit(srdr_server* s, const srdr_body_desc* desc, uint64_t* ticket)
{
    if (!s || !desc || !ticket) {
        set_error("NULL argument");
        return SRDR_ERR_INVALID;
    }
    int64_t n = 0;
    SRDR_TRY(srdr_desc_particle_count(desc, &n));
    const size_t est = estimate_bytes(*desc, n);
    std::lock_guard<std::mutex> lock(s->mu);
    if (est > s->budget) {
        s->refused += 1;
        set_error("request needs about %zu bytes of device memory, budget is %zu", est, s->budget);
        return SRDR_ERR_NO_MEMORY;
    }
    if (s->queue.size() >= s->queue_cap) {
        s->refused += 1;
        set_error("request queue full (%zu)", s->queue_cap);
        return SRDR_ERR_BUSY;
    }
    Request r{s->next_ticket++, *desc, now_s(), est};
    if (s->submitted == 0) s->t_first_submit = r.t_submit;
    s->submitted += 1;
    *ticket = r.ticket;
    s->queue.push_back(r);
    s->cv_work.notify_one();
    return SRDR_OK;
}

static srdr_status take_result(srdr_server* s, uint64_t ticket, double* out, size_t n, double* latency,
                               int64_t* steps)
{
    auto it = s->results.find(ticket);
    Result& r = it->second;
    if (out && n < r.disp.size()) {
        set_error("output buffer too small (need %zu doubles)", r.disp.size());
        return SRDR_ERR_INVALID;
    }
    if (out) std::copy(r.disp.begin(), r.disp.end(), out);
    if (latency) *latency = r.latency;
    if (steps) *steps = r.steps;
    srdr_status st = r.status;
    s->results.erase(it);
    if (st != SRDR_OK) set_error("request %llu finished with status %d", (unsigned long long)ticket, st);
    return st;
}

srdr_status srdr_server_poll(srdr_server* s, uint64_t ticket, double* host_disp_out, size_t n,
                             double* latency_s)
{
    if (!s) {
        set_error("server is NULL");
        return SRDR_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->results.count(ticket)) return take_result(s, ticket, host_disp_out, n, latency_s, nullptr);
    if (ticket == 0 || ticket >= s->next_ticket) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return SRDR_ERR_INVALID;
    }
    set_error("request %llu not finished", (unsigned long long)ticket);
    return SRDR_ERR_BUSY;
}

srdr_status srdr_server_wait(srdr_server* s, uint64_t ticket, double timeout_s, double* host_disp_out,
                             size_t n, double* latency_s, int64_t* steps)
{
    if (!s || ticket == 0) {
        set_error("bad server or ticket");
        return SRDR_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    if (ticket >= s->next_ticket) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return SRDR_ERR_INVALID;
    }
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->results.count(ticket) > 0; });
    if (!ok) {
        set_error("request %llu not finished after %.3f s", (unsigned long long)ticket, timeout_s);
        return SRDR_ERR_BUSY;
    }
    return take_result(s, ticket, host_disp_out, n, latency_s, steps);
}

srdr_status srdr_server_stats(srdr_server* s, srdr_server_report* out)
{
    if (!s || !out) {
        set_error("NULL argument");
        return SRDR_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    *out = srdr_server_report{};
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->refused = s->refused;
    out->queued = (int64_t)s->queue.size();
    out->in_flight = (int64_t)s->in_flight.size();
    out->peak_concurrent = s->peak_live;
    out->bytes_in_use = s->in_use;
    out->particle_steps = s->particle_steps;
    out->not_converged = s->not_converged;
    out->failed = s->failed;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            size_t k = (size_t)std::min<double>(l.size() - 1, std::ceil(p * l.size()) - 1);
            return l[k];
        };
        out->p50_latency_s = pct(0.50);
        out->p99_latency_s = pct(0.99);
    }
    const double span = s->t_last_done - s->t_first_submit;
    out->solves_per_s = span > 0 ? s->completed / span : 0.0;
    return SRDR_OK;
}

void srdr_server_destroy(srdr_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
