// Serving loop: continuous batching of PMACE reconstruction jobs on one GPU.
//
// Jobs (each a full problem: image size, probe, scan, amplitudes, iteration
// count, alpha, rho) are submitted from any host thread and queued.  An
// admitter thread creates queued jobs in arrival order while the device
// bytes of the admitted jobs stay within the budget, a slot is free and the
// admitted jobs do not already fill a tick; a worker thread runs the ticks.
// Every job keeps its whole state resident (stacks, consensus image,
// amplitudes).  One tick runs one iteration of Algorithm 1 for the admitted
// jobs it steps: one agent launch per (probe size, amplitude format, plan)
// group, whose clusters cover the windows of all the stepped jobs in the
// group, and one consensus launch whose CTAs cover their image tiles.  A
// tick steps every admitted job while they fit the device; when they hold
// more work than that, it steps the jobs with the least remaining work
// first (see tick()).  A job that reaches its iteration count is read out
// and retired at the end of the tick, which frees its memory and slot for
// the next queued job.  Each window and each pixel is computed by the same
// code as in a job run alone, so a job's result does not depend on what it
// was batched with or on which ticks stepped it.
#include "job.h"
#include "pmace.h"
#include "pmace_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <tuple>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace pmace;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    pmace_dims dims{};
    pmace_amp_format fmt = PMACE_AMP_F32;
    pmace_step step{};
    int32_t iterations = 0;
    std::vector<float> probe;
    std::vector<int32_t> offsets;
    std::vector<char> amps;
    std::vector<float> scales, init;
    double submit_ms = 0.0;
};

struct Active {
    Request req;
    pmace_job* job = nullptr;
    double start_ms = 0.0;
    int64_t bytes = 0;
    int32_t skipped = 0;   // consecutive ticks this job waited for shorter ones
};

// A job is stepped at the latest after this many consecutive ticks in
// which shorter jobs filled the device.
constexpr int32_t kMaxSkippedTicks = 64;

struct Result {
    pmace_status status = PMACE_OK;
    std::string error;
    double submit_ms = 0.0, start_ms = 0.0, finish_ms = 0.0;
    int64_t device_bytes = 0;
    int32_t n1 = 0, n2 = 0;
    std::vector<float> image;
};

// Device bytes a job will hold (stacks, amplitudes, images and tables).
int64_t footprint(const pmace_dims& d, pmace_amp_format fmt) {
    const int64_t P = (int64_t)d.np * d.np, JP = (int64_t)d.J * P, NI = (int64_t)d.n1 * d.n2;
    // gather scratch: one slot of at most 32 x 32 pixels per unit of a split
    // tile; the block length keeps the units near 3072 (a little over, where
    // the 8- and 32-row tiles cut differently than the 16-row ones)
    const int64_t per_window = (int64_t)(d.np / 8 + 2) * (d.np / 32 + 2);
    const int64_t slots = std::min<int64_t>(8192, (int64_t)d.J * per_window / 8);
    return JP * 16 + JP * (fmt == PMACE_AMP_F16_SCALED ? 2 : 4) + NI * (8 + 4 + 8) + P * 24 +
           (int64_t)d.J * (16 * 4 * 8 + 8 + 4) + NI / 64 * 8 + slots * 32 * 32 * 8 + (1 << 20);
}

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t c = std::max<size_t>(n, 2 * cap + 64);
        cudaError_t e = cudaMalloc(&p, c * sizeof(T));
        if (e == cudaSuccess) cap = c;
        return e;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

struct pmace_server {
    int device = 0;
    int64_t budget = 0;
    int32_t max_active = 0;
    int32_t tile_h = 16;
    int64_t fill_pixels = 0;           // admit while the active jobs' window pixels per tick stay below this
    int64_t tick_pixels = 0;           // window pixels per tick that fill the device
    cudaStream_t stream = nullptr;     // ticks and readouts
    cudaStream_t admit_stream = nullptr;  // job creation, so admission does not wait for queued ticks

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<Request> queue;
    std::vector<Active> ready;           // created by the admitter, not yet picked up by the worker
    std::vector<pmace_job*> graveyard;   // retired jobs the admitter frees
    int64_t committed_px = 0;            // window pixels per tick of created or creating jobs
    int32_t committed_n = 0;             // jobs created or being created
    std::map<int64_t, Result> results;
    int64_t next_id = 1;
    int64_t used = 0;
    int64_t ticks = 0, retired = 0;
    int32_t n_active = 0;
    bool stop = false;
    std::string error;
    std::thread worker, admitter;

    // worker-only state
    std::vector<Active> active;
    DevBuf<AgentArgs> d_adesc;
    DevBuf<int2> d_awork;
    DevBuf<GatherArgs> d_gdesc;
    DevBuf<int2> d_gwork;

    void run();
    void admit_loop();
    pmace_status tick();
    void retire_finished();
};

namespace {

cudaError_t agent_batched(int np, const AgentArgs* descs, const int2* work, int nclusters, int v, int amp,
                          cudaStream_t s) {
    switch (np) {
        case 32: return agent_entry_batched_32(descs, work, nclusters, v, amp, s);
        case 64: return agent_entry_batched_64(descs, work, nclusters, v, amp, s);
        case 128: return agent_entry_batched_128(descs, work, nclusters, v, amp, s);
        case 256: return agent_entry_batched_256(descs, work, nclusters, v, amp, s);
        default: return cudaErrorInvalidValue;
    }
}

void finish_with_error(pmace_server* sv, const Request& r, pmace_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lock(sv->mu);
    Result& res = sv->results[r.id];
    res.status = st;
    res.error = msg;
    res.submit_ms = r.submit_ms;
    res.finish_ms = now_ms();
    res.n1 = r.dims.n1;
    res.n2 = r.dims.n2;
    sv->retired++;
    sv->cv_done.notify_all();
}

}  // namespace

// Admitter thread: creates queued jobs in arrival order (on its own stream)
// while they fit the budget, a slot and the fill target, and hands them to
// the worker; it also frees retired jobs, so that neither creation nor the
// device synchronisation of freeing ever stalls the worker's ticks.
void pmace_server::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        Request r;
        std::vector<pmace_job*> dead;
        int64_t px = 0;
        {
            std::unique_lock<std::mutex> lock(mu);
            for (;;) {
                if (stop) break;
                if (!graveyard.empty()) break;
                if (!queue.empty() && committed_n < max_active) {
                    const Request& f = queue.front();
                    const int64_t need = footprint(f.dims, f.fmt);
                    if (committed_n == 0 || (used + need <= budget && committed_px < fill_pixels)) break;
                }
                cv_admit.wait_for(lock, std::chrono::milliseconds(20));
            }
            if (stop) break;
            dead.swap(graveyard);
            if (!queue.empty() && committed_n < max_active) {
                const Request& f = queue.front();
                const int64_t need = footprint(f.dims, f.fmt);
                if (committed_n == 0 || (used + need <= budget && committed_px < fill_pixels)) {
                    r = std::move(queue.front());
                    queue.pop_front();
                    px = (int64_t)r.dims.J * r.dims.np * r.dims.np;
                    committed_n++;
                    committed_px += px;
                    used += need;   // reserved until the job's real size is known
                }
            }
        }
        for (pmace_job* j : dead) pmace_destroy(j);
        if (r.id == 0) continue;
        const int64_t reserved = footprint(r.dims, r.fmt);
        auto release = [&]() {
            std::lock_guard<std::mutex> lock(mu);
            committed_n--;
            committed_px -= px;
            used -= reserved;
        };
        if (reserved > budget) {
            release();
            finish_with_error(this, r, PMACE_ERR_OOM, "job does not fit the server's device-memory budget");
            continue;
        }
        pmace_job* job = nullptr;
        const double t0 = now_ms();
        pmace_status st = pmace_create(&r.dims, r.probe.data(), r.offsets.data(), r.amps.data(), r.fmt,
                                       r.scales.empty() ? nullptr : r.scales.data(),
                                       r.init.empty() ? nullptr : r.init.data(), 0, admit_stream, &job);
        if (st == PMACE_OK && job->tile_h != tile_h) {
            st = pmace_set_plan(job, job->variant, tile_h, admit_stream);
            if (st != PMACE_OK) {
                const std::string msg = pmace_last_error(job);
                pmace_destroy(job);
                release();
                finish_with_error(this, r, st, msg);
                continue;
            }
        }
        if (st != PMACE_OK) {
            const std::string msg = pmace_last_error(nullptr);
            release();
            finish_with_error(this, r, st, msg);
            continue;
        }
        Active a;
        a.job = job;
        a.start_ms = t0;
        a.bytes = pmace_device_bytes(job);
        r.probe.clear();
        r.probe.shrink_to_fit();
        r.amps.clear();
        r.amps.shrink_to_fit();
        r.init.clear();
        r.init.shrink_to_fit();
        a.req = std::move(r);
        std::lock_guard<std::mutex> lock(mu);
        used += a.bytes - reserved;
        ready.push_back(std::move(a));
        cv_work.notify_all();
    }
}

// One iteration for admitted jobs that still have iterations to run: the
// jobs with the least remaining work first (window pixels times remaining
// iterations, then arrival order), as many as fill the device
// (tick_pixels window pixels); a job that has waited kMaxSkippedTicks ticks
// is stepped regardless.  Short jobs then finish without waiting behind
// long ones, while the device stays full.  Which ticks step a job does not
// change its arithmetic.
pmace_status pmace_server::tick() {
    std::vector<int> cand;
    for (int i = 0; i < (int)active.size(); ++i)
        if (active[i].job->iterations < active[i].req.iterations) cand.push_back(i);
    auto remaining = [&](int i) {
        const pmace_job* h = active[i].job;
        return (int64_t)h->dims.J * h->dims.np * h->dims.np * (active[i].req.iterations - h->iterations);
    };
    std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
        const int64_t rx = remaining(x), ry = remaining(y);
        return rx != ry ? rx < ry : active[x].req.id < active[y].req.id;
    });
    // agent launches, one per (probe size, amplitude format, variant) group
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    int64_t px = 0;
    for (int i : cand) {
        Active& a = active[i];
        const pmace_job* h = a.job;
        if (px < tick_pixels || a.skipped >= kMaxSkippedTicks) {
            groups[std::make_tuple(h->dims.np, h->amp_f16, h->variant)].push_back(i);
            px += (int64_t)h->dims.J * h->dims.np * h->dims.np;
            a.skipped = 0;
        } else {
            a.skipped++;
        }
    }
    if (groups.empty()) return PMACE_OK;
    std::vector<AgentArgs> adesc;
    std::vector<int2> awork;
    struct Launch {
        int np, amp, variant, first_cluster, nclusters;
    };
    std::vector<Launch> launches;
    std::vector<int> stepping;
    for (auto& g : groups) {
        Launch L{std::get<0>(g.first), std::get<1>(g.first), std::get<2>(g.first), (int)awork.size(), 0};
        for (int i : g.second) {
            const Active& a = active[i];
            const int jd = (int)adesc.size();
            adesc.push_back(agent_args(a.job, a.req.step.alpha, a.req.step.rho));
            adesc.back().residual = a.job->iterations + 1 >= a.req.iterations ? 1 : 0;   // the job's last iteration
            for (int j0 = 0; j0 < a.job->dims.J; j0 += a.job->wpc) awork.push_back(make_int2(jd, j0));
            stepping.push_back(i);
        }
        L.nclusters = (int)awork.size() - L.first_cluster;
        launches.push_back(L);
    }
    // consensus over the tiles of every stepping job
    std::vector<GatherArgs> gdesc;
    std::vector<int2> gwork;
    for (int i : stepping) {
        const pmace_job* h = active[i].job;
        GatherArgs g = gather_args(h);
        g.src = h->u;
        g.out = h->xbar;
        const int gd = (int)gdesc.size();
        gdesc.push_back(g);
        for (int t = 0; t < h->nunits; ++t) gwork.push_back(make_int2(gd, t));
    }
    cudaError_t e = d_adesc.reserve(adesc.size());
    if (e == cudaSuccess) e = d_awork.reserve(awork.size());
    if (e == cudaSuccess) e = d_gdesc.reserve(gdesc.size());
    if (e == cudaSuccess) e = d_gwork.reserve(gwork.size());
    // pageable copies: stream-ordered, and the host vectors may be reused on return
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_adesc.p, adesc.data(), adesc.size() * sizeof(AgentArgs), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_awork.p, awork.data(), awork.size() * sizeof(int2), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_gdesc.p, gdesc.data(), gdesc.size() * sizeof(GatherArgs), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_gwork.p, gwork.data(), gwork.size() * sizeof(int2), cudaMemcpyHostToDevice, stream);
    for (const Launch& L : launches) {
        if (e != cudaSuccess) break;
        e = agent_batched(L.np, d_adesc.p, d_awork.p + L.first_cluster, L.nclusters, L.variant, L.amp, stream);
    }
    if (e == cudaSuccess) e = launch_gather_consensus_batched(d_gdesc.p, d_gwork.p, (int)gwork.size(), tile_h, stream);
    if (e != cudaSuccess) {
        error = std::string("tick: ") + cudaGetErrorString(e);
        return PMACE_ERR_CUDA;
    }
    for (int i : stepping) {
        pmace_job* h = active[i].job;
        h->rho_pending = active[i].req.step.rho;
        h->iterations++;
    }
    ticks++;
    return PMACE_OK;
}

// Read out and free every job that has run all its iterations.
void pmace_server::retire_finished() {
    for (size_t i = 0; i < active.size();) {
        Active& a = active[i];
        if (a.job->iterations < a.req.iterations) {
            ++i;
            continue;
        }
        Result res;
        res.submit_ms = a.req.submit_ms;
        res.start_ms = a.start_ms;
        res.device_bytes = a.bytes;
        res.n1 = a.req.dims.n1;
        res.n2 = a.req.dims.n2;
        res.image.resize((size_t)res.n1 * res.n2 * 2);
        res.status = pmace_get_image(a.job, res.image.data(), 0, stream);   // synchronises the stream
        if (res.status != PMACE_OK) res.error = pmace_last_error(a.job);
        res.finish_ms = now_ms();
        {
            std::lock_guard<std::mutex> lock(mu);
            used -= a.bytes;
            committed_n--;
            committed_px -= (int64_t)a.job->dims.J * a.job->dims.np * a.job->dims.np;
            graveyard.push_back(a.job);   // freed by the admitter thread
            results[a.req.id] = std::move(res);
            retired++;
            active.erase(active.begin() + i);
            n_active = (int32_t)active.size();
        }
        cv_done.notify_all();
        cv_admit.notify_all();
    }
}

void pmace_server::run() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(mu);
            if (stop) break;
            if (active.empty() && ready.empty()) {
                cv_work.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
            for (Active& a : ready) active.push_back(std::move(a));
            ready.clear();
            n_active = (int32_t)active.size();
        }
        // jobs admitted with zero iterations retire at once
        pmace_status st = tick();
        if (st != PMACE_OK) {
            // a launch failed: fail every active job and keep serving the queue
            for (Active& a : active) finish_with_error(this, a.req, st, error);
            std::lock_guard<std::mutex> lock(mu);
            for (Active& a : active) {
                used -= a.bytes;
                committed_n--;
                committed_px -= (int64_t)a.job->dims.J * a.job->dims.np * a.job->dims.np;
                graveyard.push_back(a.job);
            }
            active.clear();
            n_active = 0;
            cudaGetLastError();
            cv_admit.notify_all();
            continue;
        }
        retire_finished();
    }
}

extern "C" {

pmace_status pmace_server_create(const pmace_server_config* cfg, pmace_server_handle* out) {
    if (!out) return PMACE_ERR_INVALID_ARG;
    *out = nullptr;
    pmace_server* sv = new (std::nothrow) pmace_server();
    if (!sv) return PMACE_ERR_OOM;
    cudaGetDevice(&sv->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete sv;
        set_unbound_error(cudaGetErrorString(e));
        return PMACE_ERR_CUDA;
    }
    sv->budget = (cfg && cfg->hbm_budget_bytes > 0) ? cfg->hbm_budget_bytes : (int64_t)(0.8 * (double)free_b);
    sv->max_active = (cfg && cfg->max_active_jobs > 0) ? cfg->max_active_jobs : 64;
    const int th = cfg ? cfg->tile_h : 0;
    sv->tile_h = (th == 8 || th == 16 || th == 32) ? th : 16;
    sv->fill_pixels = (cfg && cfg->fill_pixels > 0) ? cfg->fill_pixels : ((int64_t)1 << 27);
    // about a thousand 128 x 128 windows fill every SM with agent clusters
    // more than once (PMACE_SERVER_TICK_PIXELS overrides)
    sv->tick_pixels = (int64_t)1 << 24;
    if (const char* env = std::getenv("PMACE_SERVER_TICK_PIXELS")) {
        const long long v = std::atoll(env);
        if (v > 0) sv->tick_pixels = v;
    }
    e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->admit_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete sv;
        set_unbound_error(cudaGetErrorString(e));
        return PMACE_ERR_CUDA;
    }
    sv->worker = std::thread([sv] { sv->run(); });
    sv->admitter = std::thread([sv] { sv->admit_loop(); });
    *out = sv;
    return PMACE_OK;
}

pmace_status pmace_server_submit(pmace_server_handle sv, const pmace_request* req, int64_t* id) {
    if (!sv || !req || !id) return PMACE_ERR_INVALID_ARG;
    const pmace_dims& d = req->dims;
    if (!req->probe || !req->offsets || !req->amps || d.np <= 0 || d.J <= 0 || d.n1 <= 0 || d.n2 <= 0 ||
        req->iterations < 0 || (req->fmt == PMACE_AMP_F16_SCALED && !req->scales)) {
        set_unbound_error("invalid request");
        return PMACE_ERR_INVALID_ARG;
    }
    Request r;
    r.dims = d;
    r.fmt = req->fmt;
    r.step = req->step;
    r.iterations = req->iterations;
    const size_t P = (size_t)d.np * d.np, JP = (size_t)d.J * P, NI = (size_t)d.n1 * d.n2;
    r.probe.assign(req->probe, req->probe + 2 * P);
    r.offsets.assign(req->offsets, req->offsets + 2 * (size_t)d.J);
    const size_t ab = JP * (req->fmt == PMACE_AMP_F16_SCALED ? 2 : 4);
    r.amps.assign(static_cast<const char*>(req->amps), static_cast<const char*>(req->amps) + ab);
    if (req->scales) r.scales.assign(req->scales, req->scales + d.J);
    if (req->init) r.init.assign(req->init, req->init + 2 * NI);
    r.submit_ms = now_ms();
    std::lock_guard<std::mutex> lock(sv->mu);
    r.id = sv->next_id++;
    *id = r.id;
    sv->queue.push_back(std::move(r));
    sv->cv_admit.notify_all();
    return PMACE_OK;
}

static pmace_status take_result(pmace_server* sv, int64_t id, pmace_job_result* res, float* image) {
    auto it = sv->results.find(id);
    if (it == sv->results.end()) {
        if (res) res->done = 0;
        return PMACE_OK;
    }
    const Result& r = it->second;
    if (res) {
        res->done = 1;
        res->status = r.status;
        res->submit_ms = r.submit_ms;
        res->start_ms = r.start_ms;
        res->finish_ms = r.finish_ms;
        res->device_bytes = r.device_bytes;
    }
    if (image && r.status == PMACE_OK)
        std::memcpy(image, r.image.data(), r.image.size() * sizeof(float));
    if (r.status != PMACE_OK) set_unbound_error(r.error.c_str());
    return PMACE_OK;
}

pmace_status pmace_server_poll(pmace_server_handle sv, int64_t id, pmace_job_result* res, float* image) {
    if (!sv) return PMACE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    return take_result(sv, id, res, image);
}

pmace_status pmace_server_wait(pmace_server_handle sv, int64_t id, int32_t timeout_ms, pmace_job_result* res,
                               float* image) {
    if (!sv) return PMACE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(sv->mu);
    const bool ok = sv->cv_done.wait_for(lock, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                         [&] { return sv->results.count(id) > 0; });
    if (!ok) {
        if (res) res->done = 0;
        set_unbound_error("timed out waiting for the job");
        return PMACE_ERR_TIMEOUT;
    }
    return take_result(sv, id, res, image);
}

pmace_status pmace_server_release(pmace_server_handle sv, int64_t id) {
    if (!sv) return PMACE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->results.erase(id);
    return PMACE_OK;
}

pmace_status pmace_server_stats(pmace_server_handle sv, pmace_server_counters* st) {
    if (!sv || !st) return PMACE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(sv->mu);
    st->queued = (int64_t)sv->queue.size();
    st->active = sv->n_active;
    st->completed = sv->retired;
    st->ticks = sv->ticks;
    st->device_bytes = sv->used;
    st->budget_bytes = sv->budget;
    return PMACE_OK;
}

void pmace_server_destroy(pmace_server_handle sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
        sv->cv_admit.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->admitter.joinable()) sv->admitter.join();
    for (Active& a : sv->active) pmace_destroy(a.job);
    for (Active& a : sv->ready) pmace_destroy(a.job);
    for (pmace_job* j : sv->graveyard) pmace_destroy(j);
    cudaStreamSynchronize(sv->stream);
    cudaStream_t s = sv->stream, s2 = sv->admit_stream;
    delete sv;   // frees the launch tables
    cudaStreamDestroy(s);
    cudaStreamDestroy(s2);
}

}  // extern "C"
