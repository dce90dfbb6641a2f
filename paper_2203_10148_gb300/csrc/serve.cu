// Serving runtime: continuous batching of PiTSBiCG solves on one GPU.
//
// Requests (a problem description, Section 2, plus solve options) are copied
// at submission and queued.  `max_slots` worker threads each own a CUDA
// stream; a free worker admits the first queued request whose device
// footprint fits the HBM budget next to the requests already running, builds
// the problem on its stream with stream-ordered allocations from a pool of
// the server's own, runs the mixed-precision BiCGStab solve (Algorithm 1 on
// the preconditioned system, Eq. 8) and copies the result to host memory.
// Solves of different N and grid size therefore run concurrently on the
// device, and requests that arrive while others run are admitted as soon as
// a slot and memory are free.  Each request's arithmetic does not depend on
// what else runs: kernels, launch shapes and reduction orders are chosen
// from the request alone, so a result is the same alone and in the mix.
//
// Admission is first-fit in arrival order with a bypass limit: a request
// that does not fit may be overtaken by later, smaller ones at most
// kMaxBypass times, after which admission waits for it (no starvation).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pit_internal.h"

namespace pit {
namespace {

constexpr int kMaxBypass = 16;
constexpr size_t kMaxQueued = 1u << 20;

using Clock = std::chrono::steady_clock;

double since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    pit_problem_desc desc{};
    std::vector<double> y0;
    pit_solve_opts opts{};
    size_t footprint = 0;
    double t_submit = 0, t_start = 0, t_done = 0;   // seconds since server start
    std::vector<double> X;
    std::vector<pit_solve_info> info;
    pit_status status = PIT_PENDING;
    int state = QUEUED;
    volatile int cancel = 0;
    int bypassed = 0;
    size_t device_peak = 0;
    std::string error;
};

struct Slot {
    cudaStream_t stream = nullptr;
    AllocCtx ctx;
    std::thread thread;
};

// Nearest-rank percentile (the smallest value with at least q of the
// samples at or below it).
double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t k = (size_t)ceil(q * (double)v.size());
    k = std::min(std::max<size_t>(k, 1), v.size());
    return v[k - 1];
}

}  // namespace

// Device bytes one request holds while it runs (an upper bound of the
// buffers the problem allocates): eight Krylov block vectors (X, R, R~, P,
// S, D, K and the refinement's outer iterate), the FP32 fine output and the
// sine-mode work of the 2D heat sweep, set-up tables and the reduction
// partials.
size_t serve_footprint(const pit_problem_desc *d) {
    const size_t M = (size_t)d->op.nx * d->op.ny;
    const size_t nblk = (size_t)d->N + 1;
    const size_t vlen = nblk * M * d->batch;
    size_t b = 64 * vlen;                                    // Krylov vectors
    b += vlen / 32 + 4096;                                   // reduction partials
    if (d->op.kind == PIT_OP_HEAT2D) {
        const size_t nn = M;
        const size_t ends = (size_t)d->batch * ((nblk + 15) / 16) * nn * 8;
        b += 4 * vlen + 16 * vlen + ends;                    // FP32 fine output, sweep modes
        b += 32 * nn;                                        // sine bases (FP64, FP32, TF32 parts), mode factors
        b = std::max(b, 16 * vlen + 32 * nn + 4096);         // set-up (variant autotuning)
    } else {
        b += 72 * M;                                         // Thomas factors (FP64, FP32, float-float)
        // FP64: the stored fine propagator, powers of G and the sweep's products
        b += heat1d_table_bytes((int)M, d->N, d->batch, d->fine.steps, d->coarse.steps, d->precision);
        if (d->precision == PIT_MIXED) {
            // sine-basis sweep: TF32 parts of S, two padded FP32 row sets,
            // chunk ends and mode factors
            const size_t Mp = (M + 31) / 32 * 32;
            const size_t rows = nblk * d->batch;
            b += 8 * Mp * Mp + 8 * rows * Mp + (size_t)d->batch * ((nblk + 15) / 16) * Mp * 8 + 8 * Mp;
        }
    }
    return b + (256u << 10);                                 // small buffers
}

}  // namespace pit

using namespace pit;

struct pit_server_s {
    int device = 0;
    size_t budget = 0, reserved = 0, reserved_peak = 0;
    cudaMemPool_t pool = nullptr;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::unique_ptr<Slot>> slots;
    // statistics since creation or the last reset
    std::vector<double> lat_total, lat_queue, lat_service;
    long long submitted = 0, completed = 0, failed = 0, cancelled = 0;
    long long slice_steps = 0;
    double t_first = -1.0, t_last = 0.0;
    int running = 0, max_running = 0;

    // Next request to run, or nullptr; called with mu held.
    Request *pick_locked() {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            Request *r = *it;
            if (r->footprint + reserved <= budget) {
                for (auto jt = queue.begin(); jt != it; ++jt) (*jt)->bypassed += 1;
                queue.erase(it);
                return r;
            }
            if (r->bypassed >= kMaxBypass) return nullptr;   // it goes next
        }
        return nullptr;
    }

    void record_locked(Request *r) {
        if (r->status == PIT_E_CANCELLED) {
            cancelled += 1;
            return;
        }
        if (r->status != PIT_OK) failed += 1;
        completed += 1;
        lat_total.push_back(r->t_done - r->t_submit);
        lat_queue.push_back(r->t_start - r->t_submit);
        lat_service.push_back(r->t_done - r->t_start);
        for (const auto &i : r->info) slice_steps += i.fine_slice_steps;
        t_last = std::max(t_last, r->t_done);
    }

    void run(Request *r, Slot &slot) {
        pit_problem_t h = nullptr;
        slot.ctx.cur = 0;
        slot.ctx.peak = 0;
        const int B = r->desc.batch;
        r->info.assign(B, pit_solve_info{});
        pit_status st = problem_create(&r->desc, slot.stream, &h);
        if (st == PIT_OK) {
            h->p.cancel = &r->cancel;
            pit_solve_opts o = r->opts;
            o.stream = slot.stream;
            o.history = nullptr;
            o.history_len = 0;
            r->X.assign(h->p.vlen, 0.0);
            st = pit_bicgstab_solve(h, &o, r->X.data(), 0, r->info.data());
        }
        if (st != PIT_OK) {
            char buf[512];
            pit_last_error(buf, sizeof buf);
            r->error = buf;
            if (st != PIT_E_MAXITER && st != PIT_E_BREAKDOWN && st != PIT_E_NONFINITE) {
                r->X.clear();
                for (auto &i : r->info) i.status = st;
            }
        }
        if (h) pit_problem_destroy(h);
        r->device_peak = slot.ctx.peak;
        r->status = st;
    }

    void worker(Slot *slot) {
        cudaSetDevice(device);
        tl_alloc = &slot->ctx;
        tl_tune_fallback = true;   // no timing runs per request shape
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Request *r = nullptr;
            cv_work.wait(lk, [&] { return stop || (r = pick_locked()) != nullptr; });
            if (!r) break;   // stopping
            r->state = RUNNING;
            r->t_start = since(t0);
            reserved += r->footprint;
            reserved_peak = std::max(reserved_peak, reserved);
            running += 1;
            max_running = std::max(max_running, running);
            lk.unlock();
            run(r, *slot);
            const double td = since(t0);
            lk.lock();
            r->t_done = td;
            for (auto &i : r->info) {
                i.queue_seconds = r->t_start - r->t_submit;
                i.latency_seconds = r->t_done - r->t_submit;
                i.device_bytes = (long long)r->device_peak;
            }
            r->state = DONE;
            reserved -= r->footprint;
            running -= 1;
            record_locked(r);
            cv_done.notify_all();
            cv_work.notify_all();   // memory was released: others may fit now
        }
        tl_alloc = nullptr;
    }
};

namespace {

pit_status validate(const pit_problem_desc *d, const pit_solve_opts *o) {
    if (!d || !o || !d->y0) {
        set_error("pit_serve_submit: null argument");
        return PIT_E_INVALID;
    }
    if (d->op.kind != PIT_OP_HEAT1D && d->op.kind != PIT_OP_HEAT2D) {
        set_error("pit_serve_submit: the server takes HEAT1D and HEAT2D problems");
        return PIT_E_UNSUPPORTED;
    }
    if (d->op.nx < 1 || d->op.ny < 1 || d->N < 1 || d->batch < 1 || !(d->T > 0.0)) {
        set_error("pit_serve_submit: invalid sizes or T");
        return PIT_E_INVALID;
    }
    return PIT_OK;
}

}  // namespace

extern "C" {

pit_status pit_serve_footprint(const pit_problem_desc *d, size_t *bytes) {
    if (!d || !bytes || d->op.nx < 1 || d->op.ny < 1 || d->N < 1 || d->batch < 1) {
        set_error("pit_serve_footprint: bad argument");
        return PIT_E_INVALID;
    }
    *bytes = serve_footprint(d);
    return PIT_OK;
}

pit_status pit_server_create(size_t hbm_budget_bytes, int max_slots, pit_server_t *out) {
    if (!out || max_slots < 1 || max_slots > 64) {
        set_error("pit_server_create: null out or max_slots outside 1..64");
        return PIT_E_INVALID;
    }
    *out = nullptr;
    std::unique_ptr<pit_server_s> s(new (std::nothrow) pit_server_s());
    if (!s) {
        set_error("pit_server_create: host allocation failed");
        return PIT_E_NOMEM;
    }
    PIT_CUDA(cudaGetDevice(&s->device));
    size_t free_b = 0, total_b = 0;
    PIT_CUDA(cudaMemGetInfo(&free_b, &total_b));
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    PIT_CUDA(cudaMemPoolCreate(&s->pool, &props));
    // keep freed memory (up to the budget) for the next requests
    uint64_t thr = (uint64_t)s->budget;
    PIT_CUDA(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr));
    s->t0 = Clock::now();
    for (int i = 0; i < max_slots; ++i) {
        std::unique_ptr<Slot> sl(new Slot());
        cudaError_t e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            pit_server_destroy(s.release());
            return cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
        }
        sl->ctx.pool = s->pool;
        sl->ctx.stream = sl->stream;
        s->slots.push_back(std::move(sl));
    }
    for (auto &sl : s->slots) {
        Slot *raw = sl.get();
        pit_server_s *srv = s.get();
        raw->thread = std::thread([srv, raw] { srv->worker(raw); });
    }
    *out = s.release();
    return PIT_OK;
}

pit_status pit_server_destroy(pit_server_t s) {
    if (!s) return PIT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request *r : s->queue) {
            r->status = PIT_E_CANCELLED;
            r->state = DONE;
        }
        s->queue.clear();
        for (auto &kv : s->reqs)
            if (kv.second->state == RUNNING) kv.second->cancel = 1;
    }
    s->cv_work.notify_all();
    for (auto &sl : s->slots)
        if (sl->thread.joinable()) sl->thread.join();
    cudaSetDevice(s->device);
    for (auto &sl : s->slots)
        if (sl->stream) {
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return PIT_OK;
}

pit_status pit_serve_submit(pit_server_t s, const pit_problem_desc *d, const pit_solve_opts *o,
                            uint64_t *ticket) {
    if (!s || !ticket) {
        set_error("pit_serve_submit: null argument");
        return PIT_E_INVALID;
    }
    PIT_TRY(validate(d, o));
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) {
        set_error("pit_serve_submit: host allocation failed");
        return PIT_E_NOMEM;
    }
    r->desc = *d;
    const size_t M = (size_t)d->op.nx * d->op.ny;
    r->y0.assign(d->y0, d->y0 + M * d->batch);
    r->desc.y0 = r->y0.data();
    r->desc.op.vx = r->desc.op.vy = r->desc.op.A = nullptr;
    r->opts = *o;
    r->footprint = serve_footprint(d);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        set_error("pit_serve_submit: the server is shutting down");
        return PIT_E_INVALID;
    }
    if (r->footprint > s->budget) {
        set_error("pit_serve_submit: the request alone exceeds the HBM budget");
        return PIT_E_NOMEM;
    }
    if (s->queue.size() >= kMaxQueued) {
        set_error("pit_serve_submit: the queue is full");
        return PIT_E_BUSY;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = since(s->t0);
    if (s->t_first < 0.0) s->t_first = r->t_submit;
    s->submitted += 1;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->ticket, std::move(r));
    s->cv_work.notify_one();
    return PIT_OK;
}

// Shared by poll and wait: with mu held and the request DONE, hands the
// result over and releases the request.
static pit_status take_locked(pit_server_t s, Request *r, double *X_out, pit_solve_info *info) {
    const pit_status st = r->status;
    if (X_out && !r->X.empty()) memcpy(X_out, r->X.data(), r->X.size() * sizeof(double));
    if (info) {
        for (size_t b = 0; b < r->info.size(); ++b) info[b] = r->info[b];
        if (r->info.empty()) {
            memset(info, 0, sizeof *info);
            info->status = st;
        }
    }
    if (st != PIT_OK) set_error(r->error.empty() ? "request failed" : r->error);
    s->reqs.erase(r->ticket);
    return st;
}

pit_status pit_serve_poll(pit_server_t s, uint64_t ticket, double *X_out, pit_solve_info *info) {
    if (!s) {
        set_error("pit_serve_poll: null server");
        return PIT_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("pit_serve_poll: unknown ticket (never issued, or already taken)");
        return PIT_E_INVALID;
    }
    Request *r = it->second.get();
    if (r->state != DONE) return PIT_PENDING;
    return take_locked(s, r, X_out, info);
}

pit_status pit_serve_wait(pit_server_t s, uint64_t ticket, double timeout_s, double *X_out,
                          pit_solve_info *info) {
    if (!s) {
        set_error("pit_serve_wait: null server");
        return PIT_E_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("pit_serve_wait: unknown ticket (never issued, or already taken)");
        return PIT_E_INVALID;
    }
    // the request is looked up again after every wake-up: another thread
    // waiting on the same ticket may have taken (and released) it meanwhile
    auto done = [&] {
        auto jt = s->reqs.find(ticket);
        return jt == s->reqs.end() || jt->second->state == DONE;
    };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return PIT_PENDING;
    }
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("pit_serve_wait: the result was taken by another caller");
        return PIT_E_INVALID;
    }
    return take_locked(s, it->second.get(), X_out, info);
}

pit_status pit_serve_cancel(pit_server_t s, uint64_t ticket) {
    if (!s) {
        set_error("pit_serve_cancel: null server");
        return PIT_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("pit_serve_cancel: unknown ticket");
        return PIT_E_INVALID;
    }
    Request *r = it->second.get();
    if (r->state == QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        r->status = PIT_E_CANCELLED;
        r->error = "the request was cancelled before it started";
        r->state = DONE;
        r->t_start = r->t_done = since(s->t0);
        s->record_locked(r);
        s->cv_done.notify_all();
    } else if (r->state == RUNNING) {
        r->cancel = 1;   // the solve stops at its next iteration boundary
    }
    return PIT_OK;
}

pit_status pit_server_stats(pit_server_t s, int reset, pit_server_stats_t *out) {
    if (!s || !out) {
        set_error("pit_server_stats: null argument");
        return PIT_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->cancelled = s->cancelled;
    out->queued = (long long)s->queue.size();
    out->running = s->running;
    out->max_running = s->max_running;
    out->latency_p50 = percentile(s->lat_total, 0.50);
    out->latency_p99 = percentile(s->lat_total, 0.99);
    double sum = 0;
    for (double v : s->lat_total) sum += v;
    out->latency_mean = s->lat_total.empty() ? 0.0 : sum / (double)s->lat_total.size();
    out->queue_p50 = percentile(s->lat_queue, 0.50);
    out->queue_p99 = percentile(s->lat_queue, 0.99);
    out->service_p50 = percentile(s->lat_service, 0.50);
    out->service_p99 = percentile(s->lat_service, 0.99);
    const double win = (s->t_first >= 0.0 && s->t_last > s->t_first) ? s->t_last - s->t_first : 0.0;
    out->window_seconds = win;
    out->solves_per_s = win > 0 ? (double)(s->completed - s->failed) / win : 0.0;
    out->slice_steps_per_s = win > 0 ? (double)s->slice_steps / win : 0.0;
    out->hbm_budget = s->budget;
    out->hbm_reserved = s->reserved;
    out->hbm_reserved_peak = s->reserved_peak;
    uint64_t high = 0;
    if (cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemHigh, &high) == cudaSuccess)
        out->pool_peak = (size_t)high;
    out->slots = (int)s->slots.size();
    if (reset) {
        s->lat_total.clear();
        s->lat_queue.clear();
        s->lat_service.clear();
        s->submitted = s->completed = s->failed = s->cancelled = 0;
        s->slice_steps = 0;
        s->t_first = -1.0;
        s->t_last = 0.0;
        s->max_running = s->running;
        s->reserved_peak = s->reserved;
        uint64_t zero = 0;
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReservedMemHigh, &zero);
    }
    return PIT_OK;
}

}  // extern "C"
