// serve.cu -- the request server of include/rubix.h: one resident SSP state,
// a host thread running a continuous-batching loop, stream-ordered device
// memory, and per-request completion events.
//
// Loop (one iteration):
//   1. completions: requests whose done event has fired are finished (device
//      error word checked, host copy for pageable output, plan freed
//      stream-ordered, budget and slot returned);
//   2. admission: FIFO queue head admitted while a slot is free and its
//      footprint fits the budget; its plan is allocated from the pool and
//      its pre stage (stage, keys, sort, setup, work items) enqueued on the
//      slot's stream, followed by an event;
//   3. batching: when at most one deposit launch is still in flight, every
//      request whose pre stage is enqueued (up to max_batch) joins one
//      deposit launch on the deposit stream, which waits on their events;
//      each request's stream then waits on the launch and runs its combine,
//      PSF/LSF/noise and output copy, and records its done event.
// The loop only queries events: it never synchronises the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rubix.h"
#include "engine.h"

using namespace rubix;

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kQueued, kPre, kLaunched, kFinished };

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_pre = nullptr, ev_done = nullptr;
    unsigned* h_err = nullptr;  // pinned copy of the device error word after the request
};

struct Request {
    uint64_t ticket = 0;
    rubix_telescope tel{};
    rubix_particles p{};
    uint64_t seed = 0;
    float s2n = 0.f;
    float* out = nullptr;
    bool out_dev = false, out_pinned = false;
    size_t bytes = 0;
    double work = 0;           // estimated GPU work: deposits + kVoxelWork per cube voxel
    Clock::time_point t_submit, t_done;
    ReqState state = kQueued;
    rubix_status status = RUBIX_ERR_NOT_READY;
    std::string message;
    // while on the GPU
    int slot = -1;
    Plan plan;
    float* target = nullptr;   // deposit target
    float* dout = nullptr;     // device cube the post stage writes
};

using ReqPtr = std::shared_ptr<Request>;

// Batch formation: a request joins the launch being formed while the launch's
// estimated work stays within max(kBatchWork, work of its first request), so
// small requests share launches but never wait behind a large one that was
// queued after them. Work unit: one deposit (particle x wavelength bin); a
// cube voxel (zero fill, combine, PSF/LSF) costs about kVoxelWork deposits.
constexpr double kBatchWork = 2e9;
constexpr double kVoxelWork = 2.0;

struct Batch {
    cudaEvent_t ev = nullptr;
    bool busy = false;
};

}  // namespace

struct rubix_server {
    SspState* S = nullptr;
    int device = 0;
    size_t budget = 0;
    int max_slots = 1, max_batch = 1;
    cudaMemPool_t pool = nullptr;
    cudaStream_t dep_stream = nullptr;
    long long* d_job_cost = nullptr;
    std::vector<Slot> slots;
    std::vector<Batch> batch_ev;  // deposit launches in flight (at most 2 used)

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<ReqPtr> queue;                          // guarded by mu
    std::unordered_map<uint64_t, ReqPtr> reqs;         // guarded by mu
    uint64_t next_ticket = 1;                          // guarded by mu
    int64_t n_submitted = 0, n_ok = 0, n_rejected = 0, n_cancelled = 0, n_failed = 0;  // guarded by mu
    int64_t n_dep_launches = 0, max_jobs = 0;          // guarded by mu
    size_t in_use = 0, peak = 0;                       // guarded by mu
    int n_active = 0;                                  // guarded by mu

    // loop-thread state
    std::vector<int> free_slots;
    std::vector<ReqPtr> active;   // admitted, not finished
    std::vector<ReqPtr> ready;    // pre stage enqueued, waiting for a deposit launch
    std::thread th;
};

namespace {

// Ends a request (loop or client thread) and wakes its waiters. Caller holds mu.
void finish_locked(rubix_server* srv, Request& r, rubix_status st, const char* msg) {
    r.status = st;
    r.message = msg ? msg : "";
    r.state = kFinished;
    r.t_done = Clock::now();
    if (st == RUBIX_OK) ++srv->n_ok;
    else if (st == RUBIX_ERR_CANCELLED) ++srv->n_cancelled;
    else ++srv->n_failed;
    srv->cv_done.notify_all();
}

// Returns an admitted request's budget and slot and ends it.
void retire(rubix_server* srv, const ReqPtr& r, rubix_status st, const char* msg) {
    plan_release(&r->plan);  // stream-ordered on the slot's stream
    if (r->slot >= 0) srv->free_slots.push_back(r->slot);
    r->slot = -1;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->in_use -= r->bytes;
    --srv->n_active;
    finish_locked(srv, *r, st, msg);
}

// Plan allocation and the pre stage of one admitted request.
void admit(rubix_server* srv, const ReqPtr& r) {
    Slot& sl = srv->slots[r->slot];
    Alloc a;
    a.async = true;
    a.stream = sl.stream;
    a.pool = srv->pool;
    a.staging = !r->p.on_device;
    rubix_status s = plan_init(&r->plan, srv->S, &r->tel, std::max<int64_t>(r->p.n, 1), a, !r->out_dev, false);
    if (s == RUBIX_OK) {
        r->dout = r->out_dev ? r->out : r->plan.d_out;
        r->target = deposit_target(r->plan, r->dout, r->s2n > 0.f);
        s = enqueue_pre(r->plan, &r->p, sl.stream);
    }
    if (s == RUBIX_OK && cudaEventRecord(sl.ev_pre, sl.stream) != cudaSuccess)
        s = fail(RUBIX_ERR_CUDA, "event record: %s", cudaGetErrorString(cudaGetLastError()));
    if (s != RUBIX_OK) {
        retire(srv, r, s, last_error());
        return;
    }
    srv->active.push_back(r);
    srv->ready.push_back(r);
}

// Deposit launches still running; frees the events of finished ones.
int launches_in_flight(rubix_server* srv) {
    int n = 0;
    for (Batch& b : srv->batch_ev) {
        if (!b.busy) continue;
        if (cudaEventQuery(b.ev) == cudaErrorNotReady) ++n;
        else b.busy = false;
    }
    return n;
}

// One shared deposit launch for the ready requests, then each one's post stage.
bool launch_batch(rubix_server* srv) {
    if (srv->ready.empty() || launches_in_flight(srv) > 1) return false;
    NvtxRange nvtx("rubix: serving batch");
    Batch* B = nullptr;
    for (Batch& b : srv->batch_ev)
        if (!b.busy) {
            B = &b;
            break;
        }
    if (!B) return false;
    int n = 1;
    double work = srv->ready[0]->work;
    const double cap = std::max(kBatchWork, work);
    while (n < std::min<int>((int)srv->ready.size(), srv->max_batch) && work + srv->ready[n]->work <= cap)
        work += srv->ready[n++]->work;
    std::vector<ReqPtr> batch(srv->ready.begin(), srv->ready.begin() + n);
    srv->ready.erase(srv->ready.begin(), srv->ready.begin() + n);
    DepJob jobs[kMaxJobs];
    for (int j = 0; j < n; ++j) {
        cudaStreamWaitEvent(srv->dep_stream, srv->slots[batch[j]->slot].ev_pre, 0);
        jobs[j] = plan_job(batch[j]->plan, batch[j]->target);
    }
    const int l = enqueue_deposit(*srv->S, jobs, n, srv->d_job_cost, srv->dep_stream);
    if (l < 0 || cudaEventRecord(B->ev, srv->dep_stream) != cudaSuccess) {
        const char* m = cudaGetErrorString(cudaGetLastError());
        for (const ReqPtr& r : batch) {
            srv->active.erase(std::find(srv->active.begin(), srv->active.end(), r));
            retire(srv, r, RUBIX_ERR_CUDA, m);
        }
        return true;
    }
    B->busy = true;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        ++srv->n_dep_launches;
        srv->max_jobs = std::max<int64_t>(srv->max_jobs, n);
    }
    for (const ReqPtr& r : batch) {
        Slot& sl = srv->slots[r->slot];
        cudaStreamWaitEvent(sl.stream, B->ev, 0);
        enqueue_post(r->plan, r->target, r->dout, r->seed, r->s2n, sl.stream);
        if (!r->out_dev && r->out_pinned)
            cudaMemcpyAsync(r->out, r->dout, (size_t)r->plan.n_s * r->tel.n_lambda * sizeof(float),
                            cudaMemcpyDeviceToHost, sl.stream);
        cudaMemcpyAsync(sl.h_err, srv->S->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, sl.stream);
        cudaEventRecord(sl.ev_done, sl.stream);
        r->state = kLaunched;
    }
    return true;
}

// Finishes the requests whose done event has fired.
bool completions(rubix_server* srv) {
    bool any = false;
    for (size_t i = 0; i < srv->active.size();) {
        const ReqPtr r = srv->active[i];
        if (r->state != kLaunched) {
            ++i;
            continue;
        }
        const Slot& sl = srv->slots[r->slot];
        const cudaError_t q = cudaEventQuery(sl.ev_done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        any = true;
        rubix_status st = RUBIX_OK;
        char msg[160] = "";
        if (q != cudaSuccess) {
            st = RUBIX_ERR_CUDA;
            snprintf(msg, sizeof(msg), "request: %s", cudaGetErrorString(q));
        } else if (*sl.h_err != 0) {
            st = RUBIX_ERR_DEVICE;
            snprintf(msg, sizeof(msg), "device error word 0x%x", *sl.h_err);
        } else if (!r->out_dev && !r->out_pinned) {
            // pageable host output: a synchronous copy from the loop thread
            const cudaError_t e = cudaMemcpy(r->out, r->dout, (size_t)r->plan.n_s * r->tel.n_lambda * sizeof(float),
                                             cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                st = RUBIX_ERR_CUDA;
                snprintf(msg, sizeof(msg), "output copy: %s", cudaGetErrorString(e));
            }
        }
        srv->active.erase(srv->active.begin() + i);
        retire(srv, r, st, msg);
    }
    return any;
}

void serve_loop(rubix_server* srv) {
    cudaSetDevice(srv->device);
    while (true) {
        bool progressed = completions(srv);
        std::vector<ReqPtr> adm;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop && srv->queue.empty() && srv->active.empty()) break;
            while (!srv->queue.empty() && !srv->free_slots.empty()) {
                const ReqPtr& h = srv->queue.front();
                if (srv->in_use + h->bytes > srv->budget) break;  // FIFO: nothing overtakes the head
                srv->in_use += h->bytes;
                srv->peak = std::max(srv->peak, srv->in_use);
                ++srv->n_active;
                h->state = kPre;
                h->slot = srv->free_slots.back();
                srv->free_slots.pop_back();
                adm.push_back(h);
                srv->queue.pop_front();
            }
        }
        for (const ReqPtr& r : adm) admit(srv, r);
        progressed |= !adm.empty();
        progressed |= launch_batch(srv);
        if (!progressed) {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->active.empty()) {
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(10),
                                      [&] { return srv->stop || !srv->queue.empty(); });
            } else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
}

}  // namespace

#define SCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            st = fail(e_ == cudaErrorMemoryAllocation ? RUBIX_ERR_OOM : RUBIX_ERR_CUDA, "%s: %s", #call,   \
                      cudaGetErrorString(e_));                                                            \
            goto done;                                                                                    \
        }                                                                                                 \
    } while (0)

static void free_server(rubix_server* srv) {
    if (!srv) return;
    cudaSetDevice(srv->device);
    cudaDeviceSynchronize();
    for (Slot& sl : srv->slots) {
        if (sl.ev_pre) cudaEventDestroy(sl.ev_pre);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_err) cudaFreeHost(sl.h_err);
    }
    for (Batch& b : srv->batch_ev)
        if (b.ev) cudaEventDestroy(b.ev);
    if (srv->d_job_cost) cudaFree(srv->d_job_cost);
    if (srv->dep_stream) cudaStreamDestroy(srv->dep_stream);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    ssp_state_destroy(srv->S);
    delete srv;
}

extern "C" rubix_status rubix_serve_create(const rubix_ssp_grid* ssp, const rubix_telescope* wavelength_grid,
                                           size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                                           rubix_server_t** out) {
    if (!out) return fail(RUBIX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ssp || !wavelength_grid) return fail(RUBIX_ERR_INVALID_ARG, "ssp or wavelength grid is NULL");
    if (max_slots < 1 || max_slots > 256) return fail(RUBIX_ERR_INVALID_ARG, "max_slots must be in [1, 256]");
    if (max_batch < 1 || max_batch > kMaxJobs) return fail(RUBIX_ERR_INVALID_ARG, "max_batch must be in [1, 64]");
    if (hbm_budget_bytes == 0) return fail(RUBIX_ERR_INVALID_ARG, "hbm_budget_bytes is 0");
    rubix_server* srv = new rubix_server();
    rubix_status st = RUBIX_OK;
    srv->budget = hbm_budget_bytes;
    srv->max_slots = max_slots;
    srv->max_batch = max_batch;
    cudaGetDevice(&srv->device);
    {
        st = ssp_state_create(ssp, wavelength_grid, &srv->S);
        if (st != RUBIX_OK) goto done;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = srv->device;
        SCK(cudaMemPoolCreate(&srv->pool, &props));
        // keep up to the budget cached in the pool between requests
        cuuint64_t keep = hbm_budget_bytes;
        SCK(cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        SCK(cudaStreamCreateWithFlags(&srv->dep_stream, cudaStreamNonBlocking));
        SCK(cudaMalloc(&srv->d_job_cost, sizeof(long long) * (kMaxJobs + 1)));
        srv->slots.resize(max_slots);
        for (int i = 0; i < max_slots; ++i) {
            Slot& sl = srv->slots[i];
            SCK(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
            SCK(cudaEventCreateWithFlags(&sl.ev_pre, cudaEventDisableTiming));
            SCK(cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming));
            SCK(cudaHostAlloc(&sl.h_err, sizeof(unsigned), cudaHostAllocDefault));
            *sl.h_err = 0;
            srv->free_slots.push_back(max_slots - 1 - i);
        }
        srv->batch_ev.resize(4);
        for (Batch& b : srv->batch_ev) SCK(cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming));
        SCK(cudaDeviceSynchronize());
        srv->th = std::thread(serve_loop, srv);
    }
done:
    if (st != RUBIX_OK) {
        free_server(srv);
        return st;
    }
    *out = srv;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_serve_submit(rubix_server_t* srv, const rubix_telescope* tel, const rubix_particles* p,
                                           uint64_t noise_seed, float noise_s2n, float* cube_out,
                                           int32_t cube_on_device, uint64_t* ticket) {
    if (!srv || !tel || !ticket || !cube_out) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    *ticket = 0;
    rubix_status s = check_particles(p);
    if (s != RUBIX_OK) return s;
    s = validate_telescope(tel, srv->S->ssp.dls);
    if (s != RUBIX_OK) return s;
    if (!same_wavelength_grid(*srv->S, tel))
        return fail(RUBIX_ERR_INVALID_ARG, "the request's wavelength grid differs from the server's");
    auto r = std::make_shared<Request>();
    r->tel = *tel;
    r->p = *p;
    r->seed = noise_seed;
    r->s2n = noise_s2n;
    r->out = cube_out;
    r->out_dev = cube_on_device != 0;
    if (!r->out_dev) {
        cudaPointerAttributes at{};
        r->out_pinned = cudaPointerGetAttributes(&at, cube_out) == cudaSuccess && at.type == cudaMemoryTypeHost;
        cudaGetLastError();
    }
    r->bytes = plan_bytes(*srv->S, tel, std::max<int64_t>(p->n, 1), !r->out_dev, false, !p->on_device);
    r->work = ((double)p->n + kVoxelWork * (double)tel->nx * tel->ny) * tel->n_lambda;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return fail(RUBIX_ERR_INVALID_ARG, "server is shutting down");
    ++srv->n_submitted;
    if (r->bytes > srv->budget) {
        ++srv->n_rejected;
        return fail(RUBIX_ERR_REJECTED, "request footprint %zu bytes exceeds the server budget of %zu bytes",
                    r->bytes, srv->budget);
    }
    r->ticket = srv->next_ticket++;
    srv->reqs[r->ticket] = r;
    srv->queue.push_back(r);
    *ticket = r->ticket;
    srv->cv_work.notify_one();
    return RUBIX_OK;
}

extern "C" rubix_status rubix_serve_footprint(rubix_server_t* srv, const rubix_telescope* tel,
                                              const rubix_particles* p, int32_t cube_on_device, size_t* bytes) {
    if (!srv || !tel || !bytes) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    rubix_status s = check_particles(p);
    if (s != RUBIX_OK) return s;
    s = validate_telescope(tel, srv->S->ssp.dls);
    if (s != RUBIX_OK) return s;
    *bytes = plan_bytes(*srv->S, tel, std::max<int64_t>(p->n, 1), cube_on_device == 0, false, !p->on_device);
    return RUBIX_OK;
}

// Final status of a finished request (caller holds mu).
static rubix_status report_locked(const Request& r, double* latency_s) {
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    if (r.status != RUBIX_OK) return fail(r.status, "%s", r.message.empty() ? "request failed" : r.message.c_str());
    return RUBIX_OK;
}

extern "C" rubix_status rubix_serve_poll(rubix_server_t* srv, uint64_t ticket, double* latency_s) {
    if (!srv) return fail(RUBIX_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(RUBIX_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const Request& r = *it->second;
    if (r.state != kFinished) return fail(RUBIX_ERR_NOT_READY, "request %llu is not finished", (unsigned long long)ticket);
    return report_locked(r, latency_s);
}

extern "C" rubix_status rubix_serve_wait(rubix_server_t* srv, uint64_t ticket, double timeout_s) {
    if (!srv) return fail(RUBIX_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(RUBIX_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const ReqPtr r = it->second;
    auto done = [&] { return r->state == kFinished; };
    if (timeout_s < 0) {
        srv->cv_done.wait(lk, done);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return fail(RUBIX_ERR_TIMEOUT, "request %llu not finished after %.3f s", (unsigned long long)ticket, timeout_s);
    }
    return report_locked(*r, nullptr);
}

extern "C" rubix_status rubix_serve_cancel(rubix_server_t* srv, uint64_t ticket) {
    if (!srv) return fail(RUBIX_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail(RUBIX_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const ReqPtr r = it->second;
    if (r->state == kQueued) {
        srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), r));
        finish_locked(srv, *r, RUBIX_ERR_CANCELLED, "cancelled");
        return RUBIX_OK;
    }
    if (r->state == kFinished) return report_locked(*r, nullptr);
    return fail(RUBIX_ERR_NOT_READY, "request %llu is already on the GPU", (unsigned long long)ticket);
}

extern "C" rubix_status rubix_serve_stats(rubix_server_t* srv, int64_t* stats, int32_t* n_inout) {
    if (!srv || !stats || !n_inout) return fail(RUBIX_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    const int64_t v[11] = {srv->n_submitted, srv->n_ok,           srv->n_rejected,    srv->n_cancelled,
                           srv->n_failed,    srv->n_dep_launches, srv->max_jobs,      (int64_t)srv->in_use,
                           (int64_t)srv->peak, srv->n_active,     (int64_t)srv->queue.size()};
    const int n = std::min<int>(*n_inout, 11);
    for (int i = 0; i < n; ++i) stats[i] = v[i];
    *n_inout = n;
    return RUBIX_OK;
}

extern "C" rubix_status rubix_serve_destroy(rubix_server_t* srv) {
    if (!srv) return fail(RUBIX_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (const ReqPtr& r : srv->queue) finish_locked(srv, *r, RUBIX_ERR_CANCELLED, "server destroyed");
        srv->queue.clear();
        srv->cv_work.notify_all();
    }
    if (srv->th.joinable()) srv->th.join();
    free_server(srv);
    return RUBIX_OK;
}
