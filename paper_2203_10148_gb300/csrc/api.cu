// C-ABI entry points of libpit and the solver engine: PiTSBiCG (Algorithm 1,
// Sec. 3) and parareal (eq. (6), Sec. 2) driven from the host with every
// vector operation and every Krylov scalar on the device.  The host reads a
// few bytes of per-member state once per iteration to decide whether any
// member is still iterating.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "pit_internal.h"

namespace pit {

std::atomic<unsigned long long> g_launches{0};
thread_local unsigned long long tl_launches = 0;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

pit_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e),
             what, file, line);
    set_error(buf);
    if (e == cudaErrorMemoryAllocation) return PIT_E_NOMEM;
    return PIT_E_CUDA;
}

thread_local AllocCtx *tl_alloc = nullptr;
thread_local bool tl_capturing = false;

pit_status smem_limit_raw(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limits;   // (device, kernel) -> limit set
    int dev = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limits[std::make_pair(dev, func)];
    if (bytes <= cur) return PIT_OK;
    PIT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return PIT_OK;
}

pit_status DevBuf::ensure(size_t n) {
    if (n <= bytes && ptr) return PIT_OK;
    release();
    if (n == 0) return PIT_OK;
    if (tl_capturing) {
        set_error("device allocation requested during CUDA graph capture");
        return PIT_E_CUDA;
    }
    AllocCtx *ctx = tl_alloc;
    cudaError_t e = ctx ? cudaMallocFromPoolAsync(&ptr, n, ctx->pool, ctx->stream)
                        : cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        (void)cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", n,
                 cudaGetErrorString(e));
        set_error(buf);
        return PIT_E_NOMEM;
    }
    bytes = n;
    if (ctx) {
        astream = ctx->stream;
        ctx->cur += n;
        ctx->peak = std::max(ctx->peak, ctx->cur);
    }
    return PIT_OK;
}

void DevBuf::release() {
    if (ptr) {
        if (astream) {
            cudaFreeAsync(ptr, astream);
            if (tl_alloc && tl_alloc->stream == astream)
                tl_alloc->cur -= std::min(tl_alloc->cur, bytes);
        } else {
            cudaFree(ptr);
        }
    }
    ptr = nullptr;
    bytes = 0;
    astream = nullptr;
}

// ------------------------------------------------------------ op timing
cudaEvent_t OpTimer::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

pit_status OpTimer::begin(int cls, cudaStream_t s, Rec &r) {
    if (pending.size() > 4096 && !capture_into) PIT_TRY(resolve());
    r.cls = cls;
    r.a = get();
    r.b = get();
    if (!r.a || !r.b) {
        set_error("cudaEventCreate failed");
        return PIT_E_CUDA;
    }
    if (capture_into) PIT_CUDA(cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal));
    else PIT_CUDA(cudaEventRecord(r.a, s));
    return PIT_OK;
}

pit_status OpTimer::end(Rec &r, cudaStream_t s) {
    if (capture_into) {
        PIT_CUDA(cudaEventRecordWithFlags(r.b, s, cudaEventRecordExternal));
        capture_into->push_back(r);
        return PIT_OK;
    }
    PIT_CUDA(cudaEventRecord(r.b, s));
    pending.push_back(r);
    return PIT_OK;
}

pit_status OpTimer::collect(const std::vector<Rec> &recs) {
    for (const Rec &r : recs) {
        PIT_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        PIT_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.cls] += t;
        calls[r.cls] += 1;
    }
    return PIT_OK;
}

void OpTimer::release(std::vector<Rec> &recs) {
    for (Rec &r : recs) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

pit_status OpTimer::resolve() {
    for (Rec &r : pending) {
        PIT_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        PIT_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.cls] += t;
        calls[r.cls] += 1;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    return PIT_OK;
}

void OpTimer::reset() {
    for (Rec &r : pending) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    for (int i = 0; i < PIT_TIME_CLASSES; ++i) {
        calls[i] = 0;
        ms[i] = 0.0;
    }
}

void OpTimer::destroy() {
    reset();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

#define PIT_TIMED(p, cls, s, call)                                            \
    do {                                                                      \
        ::pit::OpTimer::Rec r_{};                                             \
        const bool on_ = (p)->timer.enabled;                                  \
        if (on_) PIT_TRY((p)->timer.begin((cls), (s), r_));                   \
        PIT_TRY(call);                                                        \
        if (on_) PIT_TRY((p)->timer.end(r_, (s)));                            \
    } while (0)

static int fine_cls(int prec) {
    return prec == PIT_FP64 ? PIT_TIME_FINE_FP64
         : prec == PIT_FF ? PIT_TIME_FINE_FF
         : prec == PIT_SPLIT ? PIT_TIME_FINE_SPLIT : PIT_TIME_FINE_FP32;
}

// PIT_SPLIT is the split RK4 arithmetic of the 2D heat stepper and the
// product by error-free splitting of DENSE (where its tensor-core kernel
// serves the problem); elsewhere it means float-float (which DENSE outside
// its product runs in FP64).
static int split_or_ff(const Problem *p, int prec) {
    if (prec != PIT_SPLIT) return prec;
    return (p->kind == PIT_OP_HEAT2D || (p->kind == PIT_OP_DENSE && p->oz_on)) ? PIT_SPLIT : PIT_FF;
}
static int sweep_cls(int prec) { return prec == PIT_MIXED ? PIT_TIME_SWEEP_MIXED : PIT_TIME_SWEEP_FP64; }

// --------------------------------------------------------- operator switch
pit_status op_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                      const MemberState *st, cudaStream_t s) {
    prec = split_or_ff(p, prec);
    pit_status st_ = PIT_E_INVALID;
    switch (p->kind) {
    case PIT_OP_HEAT1D: st_ = heat1d_apply_F(p, x, y, mode, prec, st, s); break;
    case PIT_OP_HEAT2D: st_ = heat2d_apply_F(p, x, y, mode, prec, st, s); break;
    case PIT_OP_ADVDIFF2D: st_ = advdiff_apply_F(p, x, y, mode, prec, st, s); break;
    case PIT_OP_DENSE: st_ = dense_apply_F(p, x, y, mode, prec, st, s); break;
    default: set_error("unknown operator kind"); return PIT_E_INVALID;
    }
    // residual B - F x with a source: rows n >= 1 gain c (F_f(x) = F(x) + c)
    if (st_ == PIT_OK && p->has_src && mode == FINE_RESIDUAL) st_ = add_source_rows(p, y, s);
    return st_;
}

pit_status op_sweep(Problem *p, const double *q, double *z, int prec, const MemberState *st,
                    cudaStream_t s) {
    switch (p->kind) {
    case PIT_OP_HEAT1D: return heat1d_sweep(p, q, z, prec, st, s);
    case PIT_OP_HEAT2D: return heat2d_sweep(p, q, z, prec, st, s);
    case PIT_OP_ADVDIFF2D: return advdiff_sweep(p, q, z, prec, st, s);
    case PIT_OP_DENSE: return dense_sweep(p, q, z, prec, st, s);
    }
    set_error("unknown operator kind");
    return PIT_E_INVALID;
}

static pit_status fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s) {
    prec = split_or_ff(p, prec);
    if ((prec == PIT_FF || prec == PIT_SPLIT) && p->kind == PIT_OP_DENSE) prec = PIT_FP64;
    switch (p->kind) {
    case PIT_OP_HEAT1D: return heat1d_fine_one(p, x, y, prec, s);
    case PIT_OP_HEAT2D: return heat2d_fine_one(p, x, y, prec, s);
    case PIT_OP_ADVDIFF2D: return advdiff_fine_one(p, x, y, prec, s);
    case PIT_OP_DENSE: return dense_fine_one(p, x, y, prec, s);
    }
    set_error("unknown operator kind");
    return PIT_E_INVALID;
}

// y = B for every member: block 0 = y0, other blocks 0.
// y[b][n][i] += c[b][i] for blocks n in [n0, n1) of every member
__global__ void k_add_source(double *y, const double *c, int M, int n0, int n1, size_t blen,
                             int batch) {
    const size_t per = (size_t)(n1 - n0) * M;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < per * batch;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t b = t / per, r = t % per;
        const size_t n = n0 + r / M, i = r % M;
        y[b * blen + n * M + i] += c[b * M + i];
    }
}

static pit_status add_source_blocks(Problem *p, double *y, int n0, int n1, cudaStream_t s) {
    const size_t work = (size_t)(n1 - n0) * p->M * p->batch;
    const int blocks = (int)std::min<size_t>((work + 255) / 256, 152 * 8);
    if (work == 0) return PIT_OK;
    k_add_source<<<blocks, 256, 0, s>>>(y, p->cvec.as<double>(), p->M, n0, n1, p->blen, p->batch);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

pit_status add_source_rows(Problem *p, double *y, cudaStream_t s) {
    return add_source_blocks(p, y, 1, p->N + 1, s);
}

// B = (y0, 0, ..., 0), or (y0, c, ..., c) with a source (rows n >= 1 of eq. (4))
pit_status build_rhs(Problem *p, double *B, cudaStream_t s) {
    PIT_CUDA(cudaMemsetAsync(B, 0, p->vlen * sizeof(double), s));
    PIT_CUDA(cudaMemcpy2DAsync(B, p->blen * sizeof(double), p->y0.ptr, p->M * sizeof(double),
                               p->M * sizeof(double), p->batch, cudaMemcpyDeviceToDevice, s));
    if (p->has_src) PIT_TRY(add_source_rows(p, B, s));
    return PIT_OK;
}

pit_status op_serial(Problem *p, double *Lam, int prec, cudaStream_t s) {
    PIT_TRY(build_rhs(p, Lam, s));
    for (int n = 1; n <= p->N; ++n) {
        PIT_TRY(fine_one(p, Lam + (size_t)(n - 1) * p->M, Lam + (size_t)n * p->M, prec, s));
        // with a source: lam_n = F(lam_{n-1}) + c
        if (p->has_src) PIT_TRY(add_source_blocks(p, Lam, n, n + 1, s));
    }
    return PIT_OK;
}

// The offset c = F_f(0) of a source f (time-independent, y' = L y + f): both
// steppers keep the steady state y* (L y* = -f) fixed, and F_f(x) - y* =
// F(x - y*), so c = y* - F(y*) with the linear fine propagator F (FP64).
// y*: Thomas solve (1D heat), sine-basis solve (2D heat), LU (dense).
pit_status source_offset(Problem *p, const double *f) {
    const int M = p->M, B = p->batch;
    std::vector<double> ys((size_t)B * M, 0.0);
    if (p->kind == PIT_OP_HEAT1D || p->kind == PIT_OP_HEAT2D) {
        if (!(p->nu > 0.0)) {
            set_error("source: nu = 0 leaves no steady state");
            return PIT_E_UNSUPPORTED;
        }
    }
    if (p->kind == PIT_OP_HEAT1D) {
        // (nu/h^2)(y_{i-1} - 2 y_i + y_{i+1}) = -f_i, y_{-1} = y_M = 0
        const double h = 1.0 / (M + 1), k = p->nu / (h * h);
        std::vector<double> cp(M), dp(M);
        for (int b = 0; b < B; ++b) {
            const double *fb = f + (size_t)b * M;
            for (int i = 0; i < M; ++i) {
                const double den = -2.0 * k - (i > 0 ? k * cp[i - 1] : 0.0);
                cp[i] = k / den;
                dp[i] = (-fb[i] - (i > 0 ? k * dp[i - 1] : 0.0)) / den;
            }
            double *yb = ys.data() + (size_t)b * M;
            yb[M - 1] = dp[M - 1];
            for (int i = M - 2; i >= 0; --i) yb[i] = dp[i] - cp[i] * yb[i + 1];
        }
    } else if (p->kind == PIT_OP_HEAT2D) {
        // sine basis: Fh = S F S, Yh = -Fh / (nu (mu_a + mu_b)), Y = (2/(n+1))^2 S Yh S
        const int n = p->nx;
        const double h = 1.0 / (n + 1);
        std::vector<double> S((size_t)n * n), mu(n), T1((size_t)n * n), T2((size_t)n * n);
        for (int a = 0; a < n; ++a) {
            for (int j = 0; j < n; ++j)
                S[(size_t)a * n + j] = sin(M_PI * (double)(a + 1) * (double)(j + 1) / (n + 1));
            const double sk = sin(M_PI * (a + 1) * h / 2.0);
            mu[a] = -4.0 / (h * h) * sk * sk;
        }
        auto mul = [&](const double *X, const double *Y, double *Z) {   // Z = X Y (n x n)
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c) {
                    double acc = 0.0;
                    for (int k2 = 0; k2 < n; ++k2) acc += X[(size_t)r * n + k2] * Y[(size_t)k2 * n + c];
                    Z[(size_t)r * n + c] = acc;
                }
        };
        const double sc = (2.0 / (n + 1)) * (2.0 / (n + 1));
        for (int b = 0; b < B; ++b) {
            mul(S.data(), f + (size_t)b * M, T1.data());
            mul(T1.data(), S.data(), T2.data());
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < n; ++c) T2[(size_t)a * n + c] *= -1.0 / (p->nu * (mu[a] + mu[c]));
            mul(S.data(), T2.data(), T1.data());
            mul(T1.data(), S.data(), ys.data() + (size_t)b * M);
            for (int i = 0; i < M; ++i) ys[(size_t)b * M + i] *= sc;
        }
    } else if (p->kind == PIT_OP_DENSE) {
        PIT_TRY(dense_steady_state(p, f, ys.data()));
    } else {
        set_error("source: supported for HEAT1D, HEAT2D and DENSE");
        return PIT_E_UNSUPPORTED;
    }
    // F(y*) on the device: y* in block 0 of each member, F(y*) into block 1
    cudaStream_t s = p->stream;
    DevBuf tmp;
    PIT_TRY(tmp.ensure(p->vlen * sizeof(double)));
    PIT_CUDA(cudaMemsetAsync(tmp.ptr, 0, p->vlen * sizeof(double), s));
    PIT_CUDA(cudaMemcpy2DAsync(tmp.ptr, p->blen * sizeof(double), ys.data(), M * sizeof(double),
                               M * sizeof(double), B, cudaMemcpyHostToDevice, s));
    PIT_TRY(fine_one(p, tmp.as<double>(), tmp.as<double>() + M, PIT_FP64, s));
    std::vector<double> fy((size_t)B * M);
    PIT_CUDA(cudaMemcpy2DAsync(fy.data(), M * sizeof(double), tmp.as<double>() + M,
                               p->blen * sizeof(double), M * sizeof(double), B,
                               cudaMemcpyDeviceToHost, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < fy.size(); ++i) fy[i] = ys[i] - fy[i];
    PIT_TRY(p->cvec.ensure((size_t)B * M * sizeof(double)));
    PIT_CUDA(cudaMemcpyAsync(p->cvec.ptr, fy.data(), fy.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    return PIT_OK;
}

// Reads (and clears) the problem's device error word; PIT_E_TIMEOUT when a
// bounded device-side wait gave up.  Synchronises the stream.
static pit_status check_errword(Problem *p, cudaStream_t s) {
    int w = 0;
    PIT_CUDA(cudaMemcpyAsync(&w, p->errword.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    if (w != 0) {
        PIT_CUDA(cudaMemsetAsync(p->errword.ptr, 0, sizeof(int), s));
        set_error("a bounded device-side wait (grid barrier) expired; results are invalid");
        return PIT_E_TIMEOUT;
    }
    return PIT_OK;
}

// Sweep arithmetic: FP32 transforms / FP64 running sums for PIT_MIXED, FP64 otherwise.
static int sweep_prec(int prec) { return prec == PIT_MIXED ? PIT_MIXED : PIT_FP64; }

static pit_status timed_F(Problem *p, const double *x, double *y, int mode, int prec,
                          const MemberState *st, cudaStream_t s) {
    PIT_TIMED(p, fine_cls(split_or_ff(p, prec)), s, op_apply_F(p, x, y, mode, prec, st, s));
    return PIT_OK;
}

static pit_status timed_sweep(Problem *p, const double *q, double *z, int prec,
                              const MemberState *st, cudaStream_t s) {
    PIT_TIMED(p, sweep_cls(sweep_prec(prec)), s, op_sweep(p, q, z, sweep_prec(prec), st, s));
    return PIT_OK;
}

static pit_status apply_GinvF(Problem *p, const double *x, double *y, int prec,
                              const MemberState *st, cudaStream_t s) {
    if (p->kind == PIT_OP_HEAT2D && prec == PIT_MIXED) {
        // the FP32 sweep consumes FP32 rows: the fine kernel writes them directly
        PIT_TRY(p->q32.ensure(p->vlen * sizeof(float)));
        float *q = p->q32.as<float>();
        PIT_TIMED(p, PIT_TIME_FINE_FP32, s, heat2d_fine_f32out(p, x, q, st, s));
        PIT_TIMED(p, PIT_TIME_SWEEP_MIXED, s, heat2d_sweep_f32in(p, q, y, st, s));
        return PIT_OK;
    }
    PIT_TRY(timed_F(p, x, y, FINE_APPLY, prec, st, s));
    return timed_sweep(p, y, y, prec, st, s);
}

// ------------------------------------------------------------ the engine
namespace {

// Pinned staging for the per-iteration state read-back, one per host thread
// and kept for the thread's life: allocating and freeing pinned memory per
// solve would synchronise the whole device (and stall concurrent solves).
struct PinnedStates {
    MemberState *ptr = nullptr;
    int cap = 0;
    ~PinnedStates() {
        if (ptr) cudaFreeHost(ptr);
    }
};
thread_local PinnedStates tl_pinned;

struct HostStates {
    std::vector<MemberState> v;
    MemberState *pinned = nullptr;
    int batch = 0;
    pit_status init(int b) {
        batch = b;
        v.resize(b);
        // one record more than the batch: its first bytes take the loop
        // graph's iteration count
        if (tl_pinned.cap < b + 1) {
            if (tl_pinned.ptr) cudaFreeHost(tl_pinned.ptr);
            tl_pinned.ptr = nullptr;
            tl_pinned.cap = 0;
            PIT_CUDA(cudaMallocHost(&tl_pinned.ptr, sizeof(MemberState) * (b + 1)));
            tl_pinned.cap = b + 1;
        }
        pinned = tl_pinned.ptr;
        return PIT_OK;
    }
    // The member states and, with `count_dev`, the int it points to (into
    // *count), after one stream synchronisation.
    pit_status fetch(Problem *p, cudaStream_t s, const int *count_dev = nullptr,
                     int *count = nullptr) {
        int *cnt_pinned = reinterpret_cast<int *>(pinned + batch);
        if (count_dev)
            PIT_CUDA(cudaMemcpyAsync(cnt_pinned, count_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        PIT_CUDA(cudaMemcpyAsync(pinned, p->states.ptr, sizeof(MemberState) * batch,
                                 cudaMemcpyDeviceToHost, s));
        PIT_CUDA(cudaStreamSynchronize(s));
        std::copy(pinned, pinned + batch, v.begin());
        if (count_dev && count) *count = *cnt_pinned;
        return PIT_OK;
    }
    bool any_active() const {
        for (const auto &m : v)
            if (m.active) return true;
        return false;
    }
};

// CUDA graphs for the iteration: 2D and 1D heat (their launches are plain
// and cluster kernel launches on one stream).
bool graphs_apply(const Problem *p) {
    return p->use_graphs && (p->kind == PIT_OP_HEAT1D || p->kind == PIT_OP_HEAT2D);
}

void iter_graph_drop(Problem *p, IterGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    p->timer.release(g.recs);
}

// Captures (or re-captures, when the stream, the buffers or the timing mode
// changed) the iteration; on a stream that cannot be captured the graph is
// marked failed and the iterations run eagerly.
template <class Fn>
pit_status iter_graph_ready(Problem *p, IterGraph &g, cudaStream_t s, Fn &&iteration) {
    const void *ptrs[5] = {p->P.ptr, p->D.ptr, p->S.ptr, p->K.ptr, p->states.ptr};
    const bool same = g.exec && g.stream == s && g.timed == p->timer.enabled &&
                      std::equal(ptrs, ptrs + 5, g.ptrs);
    if (same) return PIT_OK;
    iter_graph_drop(p, g);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        g.failed = true;
        return PIT_OK;
    }
    tl_capturing = true;
    p->timer.capture_into = p->timer.enabled ? &g.recs : nullptr;
    const unsigned long long k0 = tl_launches;
    const pit_status st = iteration();
    // captured launches do not run: the counter counts each replay instead
    g.kernels = tl_launches - k0;
    g_launches -= g.kernels;
    p->timer.capture_into = nullptr;
    tl_capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != PIT_OK || e != cudaSuccess || !graph) {
        (void)cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        p->timer.release(g.recs);
        g.failed = true;
        return PIT_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        (void)cudaGetLastError();
        g.exec = nullptr;
        p->timer.release(g.recs);
        g.failed = true;
        return PIT_OK;
    }
    g.stream = s;
    g.timed = p->timer.enabled;
    std::copy(ptrs, ptrs + 5, g.ptrs);
    return PIT_OK;
}

// Condition of the loop graph's while node, run after every iteration of
// its body: count the iteration and go on while some member is active and
// fewer than `limit` iterations ran in this launch (the host reads the
// states and the count between launches: cancellation, the iteration guard).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const MemberState *__restrict__ st,
                            int batch, int *count, int limit) {
    int any = 0;
    for (int b = threadIdx.x; b < batch; b += 32) any |= st[b].active;
    any = __any_sync(0xffffffffu, any);
    if (threadIdx.x == 0) {
        const int c = *count + 1;
        *count = c;
        cudaGraphSetConditional(h, (any && c < limit) ? 1u : 0u);
    }
}

// The iteration loop as one graph: a conditional while node (its value set
// to 1 at every launch) whose body is the captured iteration followed by
// k_loop_cond, so that up to p->loop_chunk iterations run per launch with
// no host round trip between them.  The host clears p->loopctl before each
// launch.  Event-record nodes cannot sit in a conditional body, so timed
// solves keep the per-iteration graph; where the loop graph cannot be built
// it is marked failed and the per-iteration graph runs instead.
template <class Fn>
pit_status loop_graph_ready(Problem *p, IterGraph &g, cudaStream_t s, Fn &&iteration) {
    const void *ptrs[5] = {p->P.ptr, p->D.ptr, p->S.ptr, p->K.ptr, p->states.ptr};
    if (g.exec && g.stream == s && std::equal(ptrs, ptrs + 5, g.ptrs)) return PIT_OK;
    iter_graph_drop(p, g);
    cudaGraph_t graph = nullptr;
    auto give_up = [&]() {
        (void)cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        g.failed = true;
        return PIT_OK;
    };
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return give_up();
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return give_up();
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) return give_up();
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return give_up();
    tl_capturing = true;
    const unsigned long long k0 = tl_launches;
    pit_status st = iteration();
    if (st == PIT_OK) {
        k_loop_cond<<<1, 32, 0, s>>>(h, p->states.as<MemberState>(), p->batch,
                                     p->loopctl.as<int>(), p->loop_chunk);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        ++tl_launches;
        if (cudaGetLastError() != cudaSuccess) st = PIT_E_CUDA;
    }
    // captured launches do not run: the counter counts each iteration instead
    g.kernels = tl_launches - k0;
    g_launches -= g.kernels;
    tl_capturing = false;
    cudaGraph_t captured = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &captured);
    if (st != PIT_OK || e != cudaSuccess || captured != body) return give_up();
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    graph = nullptr;
    if (ei != cudaSuccess) {
        g.exec = nullptr;
        return give_up();
    }
    g.stream = s;
    g.timed = false;
    std::copy(ptrs, ptrs + 5, g.ptrs);
    return PIT_OK;
}

pit_status check_cancel(const Problem *p) {
    if (p->cancel && *p->cancel) {
        set_error("the solve was cancelled");
        return PIT_E_CANCELLED;
    }
    return PIT_OK;
}

struct LoopOut {
    std::vector<MemberState> final_states;
    int history_count = 0;
    int graph_iterations = 0;     // iterations run as replays of the captured graph
};

// Algorithm 1 on the workspace: X holds X^0.  If r_given, R already holds
// R^0 (inner solves of the refinement); otherwise R^0 = G^{-1}(B - F X^0) is
// computed here in precision `prec`.
pit_status run_bicgstab(Problem *p, int prec, double tol_rel, const double *abs_thresh,
                        double eps0, int max_iter, bool r_given, cudaStream_t s, double *history,
                        int history_len, int history_offset, LoopOut &out) {
    double *X = p->X.as<double>(), *R = p->R.as<double>();
    MemberState *st = p->states.as<MemberState>();
    if (!r_given) {
        PIT_TRY(timed_F(p, X, R, FINE_RESIDUAL, prec, nullptr, s));
        PIT_TRY(timed_sweep(p, R, R, prec, nullptr, s));
    }
    PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_init(p, tol_rel, abs_thresh, eps0, max_iter, s));
    // top-level timing: the iterations run untimed (and so as the loop
    // graph), each of their launches timed as a whole
    const bool inner_whole = p->timer.enabled && p->timer.top_only;
    struct TimerOff {
        OpTimer *t;
        bool on;
        ~TimerOff() {
            if (on) t->enabled = true;
        }
    } timer_off{&p->timer, inner_whole};
    if (inner_whole) p->timer.enabled = false;
    auto inner_begin = [&](OpTimer::Rec &r) -> pit_status {
        return inner_whole ? p->timer.begin(PIT_TIME_INNER, s, r) : PIT_OK;
    };
    auto inner_end = [&](OpTimer::Rec &r) -> pit_status {
        return inner_whole ? p->timer.end(r, s) : PIT_OK;
    };
    HostStates hs;
    PIT_TRY(hs.init(p->batch));
    int hc = history_offset;
    int last_iter = -1;
    // one iteration: every launch depends on device state only (members that
    // converged or restarted are masked on the device), so it is replayable
    auto iteration = [&]() -> pit_status {
        PIT_TRY(apply_GinvF(p, p->P.as<double>(), p->D.as<double>(), prec, st, s));   // D = G^-1 F P
        PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_sigma(p, s));                             // alpha
        PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_update_S(p, s));                          // S = R - alpha D
        PIT_TRY(apply_GinvF(p, p->S.as<double>(), p->K.as<double>(), prec, st, s));   // K = G^-1 F S
        PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_omega(p, s));                             // omega
        PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_update_XR(p, s));                         // X, R, beta
        PIT_TIMED(p, PIT_TIME_KRYLOV, s, kr_update_P(p, s));                          // P
        return PIT_OK;
    };
    IterGraph *g = graphs_apply(p) ? &p->igraph[prec == PIT_FP64 ? 0 : 1] : nullptr;
    // the loop graph runs several iterations per launch: not where the host
    // records member 0's residual after every iteration, nor with event timing
    IterGraph *lg = (g && p->loop_chunk > 0 && !history && !p->timer.enabled)
                        ? &p->lgraph[prec == PIT_FP64 ? 0 : 1]
                        : nullptr;
    bool collect = false, looped = false;
    // iteration guard: every member stops by max_iter, plus one restart per iteration
    const long guard = 2L * (max_iter + 2) + 4;
    long done = 0;                        // iterations run
    for (;;) {
        int ran = 0;
        PIT_TRY(hs.fetch(p, s, looped ? p->loopctl.as<int>() : nullptr, &ran));
        if (looped) {
            looped = false;
            if (ran <= 0 || ran > p->loop_chunk) {
                // not the count the condition kernel keeps: stop using the loop graph
                lg->failed = true;
                set_error("the loop graph reported " + std::to_string(ran) + " iterations");
                return PIT_E_CUDA;
            }
            g_launches += (unsigned long long)ran * lg->kernels;
            out.graph_iterations += ran;
            done += ran;
        }
        if (collect) PIT_TRY(p->timer.collect(g->recs));
        collect = false;
        if (history && hc < history_len && hs.v[0].iter != last_iter) {
            history[hc++] = hs.v[0].rnorm;       // ||R^k||_{N,inf} of member 0
            last_iter = hs.v[0].iter;
        }
        if (!hs.any_active() || done >= guard) break;
        PIT_TRY(check_cancel(p));
        // the first iteration runs eagerly (it allocates every buffer the
        // iteration uses); later ones replay a captured graph: the loop graph
        // where it applies, else one graph per iteration
        if (g && done > 0) {
            if (lg && !lg->failed) {
                PIT_TRY(loop_graph_ready(p, *lg, s, iteration));
                if (lg->exec) {
                    PIT_CUDA(cudaMemsetAsync(p->loopctl.ptr, 0, sizeof(int), s));
                    OpTimer::Rec ri{};
                    PIT_TRY(inner_begin(ri));
                    PIT_CUDA(cudaGraphLaunch(lg->exec, s));
                    PIT_TRY(inner_end(ri));
                    looped = true;
                    continue;
                }
            }
            if (!g->failed) {
                PIT_TRY(iter_graph_ready(p, *g, s, iteration));
                if (g->exec) {
                    OpTimer::Rec ri{};
                    PIT_TRY(inner_begin(ri));
                    PIT_CUDA(cudaGraphLaunch(g->exec, s));
                    PIT_TRY(inner_end(ri));
                    g_launches += g->kernels;
                    out.graph_iterations += 1;
                    collect = g->timed;
                    ++done;
                    continue;
                }
            }
        }
        {
            OpTimer::Rec ri{};
            PIT_TRY(inner_begin(ri));
            PIT_TRY(iteration());
            PIT_TRY(inner_end(ri));
        }
        ++done;
    }
    out.final_states = hs.v;
    out.history_count = hc - history_offset;
    return PIT_OK;
}

// Copies between a caller block vector and a device buffer.
pit_status to_device(Problem *p, double *dst, const double *src, int on_device, cudaStream_t s) {
    PIT_CUDA(cudaMemcpyAsync(dst, src, p->vlen * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return PIT_OK;
}
pit_status from_device(Problem *p, double *dst, const double *src, int on_device, cudaStream_t s) {
    PIT_CUDA(cudaMemcpyAsync(dst, src, p->vlen * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return PIT_OK;
}

// The copy stream and events of the early copy of a solution to host memory.
pit_status ensure_copy_stream(Problem *p) {
    if (p->copy_stream) return PIT_OK;
    PIT_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    PIT_CUDA(cudaEventCreateWithFlags(&p->x_ready, cudaEventDisableTiming));
    PIT_CUDA(cudaEventCreateWithFlags(&p->x_copied, cudaEventDisableTiming));
    return PIT_OK;
}

bool all_finite(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

int worst_status(const std::vector<int> &st) {
    int w = PIT_OK;
    for (int s : st) {
        if (s == PIT_E_NONFINITE) return s;
        if (s == PIT_E_BREAKDOWN) w = s;
        else if (s == PIT_E_MAXITER && w == PIT_OK) w = s;
    }
    return w;
}

// Per-member ||U||_{N,inf} on the host.
pit_status member_norms(Problem *p, const double *U, std::vector<double> &out, cudaStream_t s) {
    double *d = p->fine_tmp.as<double>();
    PIT_TRY(kr_block_norm(p, U, d, s));
    out.resize(p->batch);
    PIT_CUDA(cudaMemcpyAsync(out.data(), d, sizeof(double) * p->batch, cudaMemcpyDeviceToHost, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    return PIT_OK;
}

}  // namespace
}  // namespace pit

using namespace pit;

// ================================================================== C ABI
extern "C" {

void pit_default_opts(pit_solve_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->tol = 1e-10;
    o->restart_eps0 = 1e-8;
    o->max_iter = 500;
    o->x0_mode = PIT_X0_COARSE;
    o->refine_max = 8;
    o->inner_tol = 1e-4;
    o->residual_precision = PIT_SPLIT;
    o->tol_mode = PIT_TOL_R0;
}

const char *pit_version(void) { return "libpit 0.1 (sm_103a)"; }

size_t pit_last_error(char *buf, size_t n) {
    const std::string &e = g_last_error;
    if (buf && n) {
        const size_t k = std::min(n - 1, e.size());
        memcpy(buf, e.data(), k);
        buf[k] = 0;
    }
    return e.size();
}

}  // extern "C"

namespace pit {

pit_status problem_create(const pit_problem_desc *d, cudaStream_t ext_stream,
                          pit_problem_t *out) {
    if (!d || !out) {
        set_error("pit_problem_create: null argument");
        return PIT_E_INVALID;
    }
    *out = nullptr;
    const pit_operator_desc &op = d->op;
    if (op.kind < PIT_OP_HEAT1D || op.kind > PIT_OP_DENSE) {
        set_error("pit_problem_create: unknown operator kind");
        return PIT_E_INVALID;
    }
    if (op.nx < 1 || op.ny < 1 || d->N < 1 || d->batch < 1 || !(d->T > 0.0) ||
        d->fine.steps < 1 || d->coarse.steps < 1 || !d->y0 ||
        d->coarse.inner < 0 || d->coarse.inner > 64 ||
        (d->precision != PIT_FP64 && d->precision != PIT_MIXED && d->precision != PIT_MIXED_BF16)) {
        set_error("pit_problem_create: invalid sizes, steps, T, precision or null y0");
        return PIT_E_INVALID;
    }
    if (d->N + 1 > PIT_MAX_BLOCKS || d->batch > PIT_MAX_BLOCKS) {
        set_error("pit_problem_create: N + 1 and batch must be <= 65535 (grid rows of the "
                  "vector kernels)");
        return PIT_E_INVALID;
    }
    if ((op.kind == PIT_OP_HEAT1D || op.kind == PIT_OP_DENSE) && op.ny != 1) {
        set_error("pit_problem_create: HEAT1D and DENSE need ny = 1");
        return PIT_E_INVALID;
    }
    if (op.kind == PIT_OP_ADVDIFF2D && (!op.vx || !op.vy)) {
        set_error("pit_problem_create: ADVDIFF2D needs vx and vy");
        return PIT_E_INVALID;
    }
    if (op.kind == PIT_OP_DENSE && !op.A) {
        set_error("pit_problem_create: DENSE needs A");
        return PIT_E_INVALID;
    }
    if (op.kind != PIT_OP_DENSE && !(op.nu >= 0.0 && std::isfinite(op.nu))) {
        set_error("pit_problem_create: nu must be finite and >= 0");
        return PIT_E_INVALID;
    }
    const size_t M = (size_t)op.nx * op.ny;
    if (!all_finite(d->y0, M * d->batch) ||
        (op.kind == PIT_OP_DENSE && !all_finite(op.A, M * M)) ||
        (op.kind == PIT_OP_ADVDIFF2D && (!all_finite(op.vx, M) || !all_finite(op.vy, M)))) {
        set_error("pit_problem_create: non-finite value in y0, A or v");
        return PIT_E_NONFINITE;
    }
    pit_problem_s *h = new (std::nothrow) pit_problem_s();
    if (!h) {
        set_error("pit_problem_create: host allocation failed");
        return PIT_E_NOMEM;
    }
    Problem *p = &h->p;
    p->kind = op.kind;
    p->nx = op.nx;
    p->ny = op.ny;
    p->M = (int)M;
    p->N = d->N;
    p->batch = d->batch;
    p->T = d->T;
    p->dT = d->T / d->N;
    p->nu = op.nu;
    p->fine_kind = d->fine.kind;
    p->fine_steps = d->fine.steps;
    p->coarse_kind = d->coarse.kind;
    p->coarse_steps = d->coarse.steps;
    p->coarse_inner = d->coarse.inner;
    // PIT_MIXED_BF16 is the mixed path with the dense product split in BF16
    p->precision = d->precision == PIT_MIXED_BF16 ? PIT_MIXED : d->precision;
    p->dense_bf16 = d->precision == PIT_MIXED_BF16 && op.kind == PIT_OP_DENSE;
    p->blen = (size_t)(p->N + 1) * M;
    p->vlen = p->blen * p->batch;
    {
        const char *g = getenv("PIT_GRAPHS");
        p->use_graphs = !(g && g[0] == '0');
        // PIT_GRAPH_LOOP=k: k iterations per launch of the loop graph (0: off)
        const char *l = getenv("PIT_GRAPH_LOOP");
        if (l && l[0]) p->loop_chunk = std::max(0, std::min(4096, atoi(l)));
        // PIT_KRYLOV_CLUSTERS=1: a block's chunk sums reduced in a cluster
        const char *kc = getenv("PIT_KRYLOV_CLUSTERS");
        p->kr_cluster = kc && kc[0] == '1';
    }
    pit_status s = PIT_OK;
    auto fail = [&](pit_status e) {
        pit_problem_destroy(h);
        return e;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__));
    if (ext_stream) {
        p->stream = ext_stream;
        p->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&p->stream, cudaStreamDefault);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__));
    }
    if ((s = p->y0.ensure(M * d->batch * sizeof(double))) != PIT_OK) return fail(s);
    e = cudaMemcpyAsync(p->y0.ptr, d->y0, M * d->batch * sizeof(double), cudaMemcpyHostToDevice,
                        p->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "copy y0", __FILE__, __LINE__));
    if ((s = p->fine_tmp.ensure(std::max<size_t>(4096, 64 * (size_t)d->batch))) != PIT_OK)
        return fail(s);
    if ((s = p->errword.ensure(sizeof(int))) != PIT_OK) return fail(s);
    if ((s = p->loopctl.ensure(sizeof(int))) != PIT_OK) return fail(s);
    e = cudaMemsetAsync(p->errword.ptr, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "clear error word", __FILE__, __LINE__));
    switch (p->kind) {
    case PIT_OP_HEAT1D: s = heat1d_setup(p); break;
    case PIT_OP_HEAT2D: s = heat2d_setup(p); break;
    case PIT_OP_ADVDIFF2D: {
        if ((s = p->vx64.ensure(M * sizeof(double))) != PIT_OK) return fail(s);
        if ((s = p->vy64.ensure(M * sizeof(double))) != PIT_OK) return fail(s);
        e = cudaMemcpy(p->vx64.ptr, op.vx, M * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->vy64.ptr, op.vy, M * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "copy v", __FILE__, __LINE__));
        s = advdiff_setup(p);
        break;
    }
    case PIT_OP_DENSE: {
        if ((s = p->PhiF64.ensure(M * M * sizeof(double))) != PIT_OK) return fail(s);
        // A is staged in PhiF64; dense_setup replaces it by the propagator
        e = cudaMemcpy(p->PhiF64.ptr, op.A, M * M * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "copy A", __FILE__, __LINE__));
        s = dense_setup(p);
        break;
    }
    }
    if (s != PIT_OK) return fail(s);
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "setup", __FILE__, __LINE__));
    *out = h;
    return PIT_OK;
}

}  // namespace pit

extern "C" {

pit_status pit_problem_create(const pit_problem_desc *d, pit_problem_t *out) {
    return problem_create(d, nullptr, out);
}

pit_status pit_problem_destroy(pit_problem_t h) {
    if (!h) return PIT_OK;
    Problem *p = &h->p;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    DevBuf *bufs[] = {&p->y0, &p->fine_inv64, &p->fine_cp64, &p->coarse_inv64, &p->coarse_cp64,
                      &p->fine_inv32, &p->fine_cp32, &p->coarse_inv32, &p->coarse_cp32, &p->fine_invff,
                      &p->S64, &p->S32, &p->gmode, &p->hat, &p->vx64, &p->vy64, &p->vx32,
                      &p->vy32, &p->vxff, &p->vyff, &p->A64, &p->cvec, &p->adv_scratch, &p->PhiF64, &p->G64, &p->PhiF_hi,
                      &p->PhiF_lo, &p->G32, &p->dense_scratch, &p->X, &p->R, &p->Rt,
                      &p->P, &p->S, &p->D, &p->K, &p->W, &p->partials, &p->states,
                      &p->flags_host_mirror, &p->fine_tmp, &p->q32, &p->GL32, &p->GLL32, &p->xtc_S,
                      &p->errword, &p->loopctl, &p->PhiTh, &p->PhiTl, &p->tc_split,
                      &p->PhiBh, &p->PhiBl, &p->dtc_mats, &p->dtc_buf, &p->oz_phi, &p->oz_ephi,
                      &p->oz_x, &p->oz_ex, &p->h1_phiT, &p->h1_powT, &p->h1_sweep_t};
    for (IterGraph &g : p->igraph) iter_graph_drop(p, g);
    for (IterGraph &g : p->lgraph) iter_graph_drop(p, g);
    for (DevBuf *b : bufs) b->release();
    dense_teardown(p);
    p->timer.destroy();
    if (p->x_ready) cudaEventDestroy(p->x_ready);
    if (p->x_copied) cudaEventDestroy(p->x_copied);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->stream && p->own_stream) cudaStreamDestroy(p->stream);
    delete h;
    return PIT_OK;
}

pit_status pit_problem_shape(pit_problem_t h, int *M, int *N, int *batch) {
    if (!h) {
        set_error("pit_problem_shape: null problem");
        return PIT_E_INVALID;
    }
    if (M) *M = h->p.M;
    if (N) *N = h->p.N;
    if (batch) *batch = h->p.batch;
    return PIT_OK;
}

pit_status pit_apply_operator(pit_problem_t h, int which, int precision, const double *x,
                              double *y, int on_device, void *stream) {
    if (!h || !x || !y) {
        set_error("pit_apply_operator: null argument");
        return PIT_E_INVALID;
    }
    if (which < PIT_APPLY_F || which > PIT_APPLY_RESIDUAL ||
        (precision != PIT_FP64 && precision != PIT_MIXED && precision != PIT_FF &&
         precision != PIT_SPLIT)) {
        set_error("pit_apply_operator: bad operator or precision");
        return PIT_E_INVALID;
    }
    Problem *p = &h->p;
    PIT_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
    const double *dx = x;
    double *dy = y;
    if (!on_device) {
        PIT_TRY(p->X.ensure(p->vlen * sizeof(double)));
        PIT_TRY(p->W.ensure(p->vlen * sizeof(double)));
        PIT_TRY(to_device(p, p->X.as<double>(), x, 0, s));
        dx = p->X.as<double>();
        dy = p->W.as<double>();
    }
    switch (which) {
    case PIT_APPLY_F: PIT_TRY(op_apply_F(p, dx, dy, FINE_APPLY, precision, nullptr, s)); break;
    case PIT_APPLY_GINV: PIT_TRY(op_sweep(p, dx, dy, sweep_prec(precision), nullptr, s)); break;
    case PIT_APPLY_GINV_F: PIT_TRY(apply_GinvF(p, dx, dy, precision, nullptr, s)); break;
    case PIT_APPLY_RESIDUAL:
        PIT_TRY(op_apply_F(p, dx, dy, FINE_RESIDUAL, precision, nullptr, s));
        PIT_TRY(op_sweep(p, dy, dy, sweep_prec(precision), nullptr, s));
        break;
    }
    if (!on_device) {
        PIT_TRY(from_device(p, y, dy, 0, s));
        PIT_TRY(check_errword(p, s));
    }
    return PIT_OK;
}

pit_status pit_serial_fine(pit_problem_t h, int precision, double *Lam, int on_device) {
    if (!h || !Lam || (precision != PIT_FP64 && precision != PIT_MIXED && precision != PIT_FF &&
                       precision != PIT_SPLIT)) {
        set_error("pit_serial_fine: bad argument");
        return PIT_E_INVALID;
    }
    Problem *p = &h->p;
    PIT_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = p->stream;
    double *d = Lam;
    if (!on_device) {
        PIT_TRY(p->W.ensure(p->vlen * sizeof(double)));
        d = p->W.as<double>();
    }
    PIT_TRY(op_serial(p, d, precision, s));
    if (!on_device) PIT_TRY(from_device(p, Lam, d, 0, s));
    return check_errword(p, s);
}

pit_status pit_bicgstab_solve(pit_problem_t h, const pit_solve_opts *o, double *Xu,
                              int on_device, pit_solve_info *info) {
    if (!h || !o || !Xu) {
        set_error("pit_bicgstab_solve: null argument");
        return PIT_E_INVALID;
    }
    if (!(o->tol >= 0.0) || o->max_iter < 0 || o->x0_mode < PIT_X0_COARSE ||
        o->x0_mode > PIT_X0_GIVEN || !(o->restart_eps0 >= 0.0) ||
        (o->tol_mode != PIT_TOL_R0 && o->tol_mode != PIT_TOL_RHS) ||
        (o->residual_precision != PIT_FF && o->residual_precision != PIT_FP64 &&
         o->residual_precision != PIT_SPLIT)) {
        set_error("pit_bicgstab_solve: invalid options");
        return PIT_E_INVALID;
    }
    auto t0 = std::chrono::steady_clock::now();
    Problem *p = &h->p;
    PIT_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = o->stream ? (cudaStream_t)o->stream : p->stream;
    PIT_TRY(krylov_prepare(p));
    const size_t vb = p->vlen * sizeof(double);
    const int B = p->batch;
    std::vector<pit_solve_info> inf(B);
    for (auto &i : inf) memset(&i, 0, sizeof i);
    std::vector<int> status(B, PIT_OK);
    const long long steps_per_matvec = (long long)p->N * p->fine_steps;

    // ||G^{-1} B||_{N,inf} per member when the tolerance is relative to it
    // (with X^0 = G^{-1} B it is the norm of X^0, computed after X^0)
    std::vector<double> rhsn(B, 0.0);
    double *d_thr = p->fine_tmp.as<double>() + B;
    if (o->tol_mode == PIT_TOL_RHS && o->x0_mode != PIT_X0_COARSE) {
        double *tmp = p->D.as<double>();
        PIT_TRY(build_rhs(p, tmp, s));
        PIT_TRY(op_sweep(p, tmp, tmp, sweep_prec(p->precision), nullptr, s));
        PIT_TRY(member_norms(p, tmp, rhsn, s));
    }
    if (p->precision == PIT_FP64) {
        double *X = p->X.as<double>();
        if (o->x0_mode == PIT_X0_GIVEN) PIT_TRY(to_device(p, X, Xu, on_device, s));
        else if (o->x0_mode == PIT_X0_ZERO) PIT_CUDA(cudaMemsetAsync(X, 0, vb, s));
        else {
            PIT_TRY(build_rhs(p, X, s));
            PIT_TRY(op_sweep(p, X, X, PIT_FP64, nullptr, s));
            if (o->tol_mode == PIT_TOL_RHS) PIT_TRY(member_norms(p, X, rhsn, s));
        }
        const double *thr = nullptr;
        if (o->tol_mode == PIT_TOL_RHS) {
            std::vector<double> t(B);
            for (int b = 0; b < B; ++b) t[b] = o->tol * rhsn[b];
            PIT_CUDA(cudaMemcpyAsync(d_thr, t.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
            PIT_CUDA(cudaStreamSynchronize(s));
            thr = d_thr;
        }
        LoopOut lo;
        PIT_TRY(run_bicgstab(p, PIT_FP64, o->tol, thr, o->restart_eps0, o->max_iter, false, s,
                             o->history, o->history_len, 0, lo));
        PIT_TRY(from_device(p, Xu, X, on_device, s));
        PIT_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) {
            const MemberState &m = lo.final_states[b];
            inf[b].iterations = m.iter;
            inf[b].matvecs = m.matvecs;
            inf[b].restarts = m.restarts;
            inf[b].refinements = 0;
            inf[b].fine_slice_steps = (long long)m.matvecs * steps_per_matvec;
            inf[b].r0 = m.r0;
            inf[b].precond_resid = m.rnorm;
            inf[b].status = m.status;
            inf[b].history_count = (b == 0) ? lo.history_count : 0;
            inf[b].graph_iterations = lo.graph_iterations;
            status[b] = m.status;
        }
    } else {
        // Iterative refinement: FP64 true residual, FP32-fine inner solve.
        const int rprec = o->residual_precision;
        PIT_TRY(p->W.ensure(vb));
        double *Xo = p->W.as<double>();   // outer solution lives in W
        double *Wr = p->R.as<double>();   // true residual goes straight into R
        if (o->x0_mode == PIT_X0_GIVEN) PIT_TRY(to_device(p, Xo, Xu, on_device, s));
        else if (o->x0_mode == PIT_X0_ZERO) PIT_CUDA(cudaMemsetAsync(Xo, 0, vb, s));
        else {
            PIT_TRY(build_rhs(p, Xo, s));
            PIT_TRY(op_sweep(p, Xo, Xo, PIT_MIXED, nullptr, s));
            if (o->tol_mode == PIT_TOL_RHS) PIT_TRY(member_norms(p, Xo, rhsn, s));
        }
        std::vector<double> rtrue, r0(B, 0.0);
        std::vector<char> done(B, 0);
        int hc = 0;
        const int rounds = std::max(1, o->refine_max);
        // To host memory, the solution goes out while its own true residual
        // is computed (after the first correction): the check reads X and
        // the copy reads X, and a round that goes on waits for the copy
        // before it changes X.  When the check passes, the copy is the
        // result; the call returns once it has landed.
        bool copy_in_flight = false;
        // whatever way the call leaves, no copy may still be writing the
        // caller's buffer
        struct CopyWait {
            Problem *p;
            const bool *live;
            ~CopyWait() {
                if (*live) cudaEventSynchronize(p->x_copied);
            }
        } copy_wait{p, &copy_in_flight};
        for (int round = 0; round <= rounds; ++round) {
            if (!on_device && round > 0) {
                PIT_TRY(ensure_copy_stream(p));
                PIT_CUDA(cudaEventRecord(p->x_ready, s));
                PIT_CUDA(cudaStreamWaitEvent(p->copy_stream, p->x_ready, 0));
                PIT_CUDA(cudaMemcpyAsync(Xu, Xo, vb, cudaMemcpyDeviceToHost, p->copy_stream));
                PIT_CUDA(cudaEventRecord(p->x_copied, p->copy_stream));
                copy_in_flight = true;
            }
            PIT_TRY(timed_F(p, Xo, Wr, FINE_RESIDUAL, rprec, nullptr, s));
            PIT_TRY(timed_sweep(p, Wr, Wr, PIT_MIXED, nullptr, s));
            PIT_TRY(member_norms(p, Wr, rtrue, s));
            bool any = false;
            for (int b = 0; b < B; ++b) {
                if (done[b]) continue;
                inf[b].matvecs += 1;
                inf[b].fine_slice_steps += steps_per_matvec;
                if (round == 0) r0[b] = rtrue[b];
                inf[b].r0 = r0[b];
                inf[b].precond_resid = rtrue[b];
                if (!std::isfinite(rtrue[b])) {
                    done[b] = 1;
                    status[b] = PIT_E_NONFINITE;
                } else if (rtrue[b] <= o->tol * (o->tol_mode == PIT_TOL_RHS ? rhsn[b] : r0[b])) {
                    done[b] = 1;
                    status[b] = PIT_OK;
                } else if (round == rounds) {
                    done[b] = 1;
                    status[b] = PIT_E_MAXITER;
                } else {
                    any = true;
                }
            }
            if (o->history && hc < o->history_len) o->history[hc++] = rtrue[0];
            if (!any) break;
            PIT_TRY(check_cancel(p));
            for (int b = 0; b < B; ++b)
                if (done[b])
                    PIT_CUDA(cudaMemsetAsync(Wr + (size_t)b * p->blen, 0,
                                             p->blen * sizeof(double), s));
            PIT_CUDA(cudaMemsetAsync(p->X.ptr, 0, vb, s));
            if (copy_in_flight) {
                // X changes at the end of this round: the copy must have read it
                PIT_CUDA(cudaStreamWaitEvent(s, p->x_copied, 0));
                copy_in_flight = false;
            }
            LoopOut lo;
            PIT_TRY(run_bicgstab(p, PIT_MIXED, o->inner_tol, nullptr, o->restart_eps0,
                                 o->max_iter, true, s, nullptr, 0, 0, lo));
            for (int b = 0; b < B; ++b) {
                if (done[b]) continue;
                const MemberState &m = lo.final_states[b];
                inf[b].iterations += m.iter;
                inf[b].graph_iterations += lo.graph_iterations;
                inf[b].matvecs += m.matvecs - 1;   // R^0 was given: no matvec
                inf[b].restarts += m.restarts;
                inf[b].refinements += 1;
                inf[b].fine_slice_steps += (long long)(m.matvecs - 1) * steps_per_matvec;
                if (m.status == PIT_E_NONFINITE || m.status == PIT_E_BREAKDOWN) {
                    // a failed inner solve still leaves a usable correction of
                    // the last iterate; a non-finite one does not
                    if (m.status == PIT_E_NONFINITE) {
                        done[b] = 1;
                        status[b] = m.status;
                    }
                }
            }
            PIT_TRY(kr_axpy(p, Xo, p->X.as<double>(), s));
        }
        if (copy_in_flight) {
            copy_in_flight = false;
            PIT_CUDA(cudaEventSynchronize(p->x_copied));   // the final X, already on its way
        } else {
            PIT_TRY(from_device(p, Xu, Xo, on_device, s));
        }
        PIT_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) {
            inf[b].status = status[b];
            inf[b].history_count = (b == 0) ? hc : 0;
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (auto &i : inf) i.seconds = secs;
    const pit_status ew = check_errword(p, s);
    if (ew != PIT_OK)
        for (auto &i : inf) i.status = ew;
    if (info) std::copy(inf.begin(), inf.end(), info);
    return ew != PIT_OK ? ew : worst_status(status);
}

pit_status pit_parareal_solve(pit_problem_t h, int kmax, double tol, double *Xu, int on_device,
                              pit_solve_info *info) {
    if (!h || !Xu || kmax < 0 || !(tol >= 0.0)) {
        set_error("pit_parareal_solve: bad argument");
        return PIT_E_INVALID;
    }
    auto t0 = std::chrono::steady_clock::now();
    Problem *p = &h->p;
    PIT_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = p->stream;
    PIT_TRY(krylov_prepare(p));
    const int B = p->batch;
    const int sp = sweep_prec(p->precision);
    double *X = p->X.as<double>(), *Wr = p->R.as<double>();
    PIT_TRY(build_rhs(p, X, s));
    PIT_TRY(op_sweep(p, X, X, sp, nullptr, s));       // X^0 = G^{-1} B
    std::vector<pit_solve_info> inf(B);
    for (auto &i : inf) memset(&i, 0, sizeof i);
    std::vector<char> done(B, 0);
    std::vector<int> status(B, PIT_OK);
    std::vector<double> rn, r0(B, 0.0);
    const long long steps_per_matvec = (long long)p->N * p->fine_steps;
    for (int k = 0;; ++k) {
        PIT_TRY(timed_F(p, X, Wr, FINE_RESIDUAL, PIT_FP64, nullptr, s));
        PIT_TRY(timed_sweep(p, Wr, Wr, sp, nullptr, s));
        PIT_TRY(member_norms(p, Wr, rn, s));
        bool any = false;
        for (int b = 0; b < B; ++b) {
            if (done[b]) continue;
            inf[b].matvecs += 1;
            inf[b].fine_slice_steps += steps_per_matvec;
            if (k == 0) r0[b] = rn[b];
            inf[b].r0 = r0[b];
            inf[b].precond_resid = rn[b];
            inf[b].iterations = k;
            if (!std::isfinite(rn[b])) {
                done[b] = 1;
                status[b] = PIT_E_NONFINITE;
            } else if (rn[b] <= tol * r0[b]) {
                done[b] = 1;
            } else if (k >= kmax) {
                done[b] = 1;
                status[b] = tol > 0.0 ? PIT_E_MAXITER : PIT_OK;
            } else {
                any = true;
            }
        }
        if (!any) break;
        for (int b = 0; b < B; ++b)
            if (done[b])
                PIT_CUDA(cudaMemsetAsync(Wr + (size_t)b * p->blen, 0, p->blen * sizeof(double), s));
        PIT_TRY(kr_axpy(p, X, Wr, s));                 // X^{k+1} = X^k + G^{-1}(B - F X^k)
    }
    PIT_TRY(from_device(p, Xu, X, on_device, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const pit_status ew = check_errword(p, s);
    for (int b = 0; b < B; ++b) {
        inf[b].status = ew != PIT_OK ? ew : status[b];
        inf[b].seconds = secs;
    }
    if (info) std::copy(inf.begin(), inf.end(), info);
    return ew != PIT_OK ? ew : worst_status(status);
}

pit_status pit_problem_set_y0(pit_problem_t h, const double *y0, int on_device) {
    if (!h || !y0) {
        set_error("pit_problem_set_y0: null argument");
        return PIT_E_INVALID;
    }
    Problem *p = &h->p;
    const size_t n = (size_t)p->M * p->batch;
    if (!on_device && !all_finite(y0, n)) {
        set_error("pit_problem_set_y0: non-finite value in y0");
        return PIT_E_NONFINITE;
    }
    PIT_CUDA(cudaSetDevice(p->device));
    PIT_CUDA(cudaMemcpyAsync(p->y0.ptr, y0, n * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             p->stream));
    PIT_CUDA(cudaStreamSynchronize(p->stream));
    return PIT_OK;
}

pit_status pit_problem_set_source(pit_problem_t h, const double *f, int on_device) {
    if (!h) {
        set_error("pit_problem_set_source: null problem");
        return PIT_E_INVALID;
    }
    Problem *p = &h->p;
    PIT_CUDA(cudaSetDevice(p->device));
    if (!f) {
        p->has_src = false;
        return PIT_OK;
    }
    const size_t n = (size_t)p->M * p->batch;
    std::vector<double> fh(n);
    if (on_device) {
        PIT_CUDA(cudaMemcpy(fh.data(), f, n * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::copy(f, f + n, fh.begin());
    }
    if (!all_finite(fh.data(), n)) {
        set_error("pit_problem_set_source: non-finite value in f");
        return PIT_E_NONFINITE;
    }
    p->has_src = false;
    PIT_TRY(source_offset(p, fh.data()));
    p->has_src = true;
    return PIT_OK;
}

unsigned long long pit_kernel_launches(void) { return g_launches.load(); }

pit_status pit_set_timing(pit_problem_t h, int enable) {
    if (!h) {
        set_error("pit_set_timing: null problem");
        return PIT_E_INVALID;
    }
    h->p.timer.reset();
    h->p.timer.enabled = enable != 0;
    h->p.timer.top_only = enable == 2;
    return PIT_OK;
}

pit_status pit_get_timing(pit_problem_t h, int cls, long long *calls, double *ms) {
    if (!h || cls < 0 || cls >= PIT_TIME_CLASSES) {
        set_error("pit_get_timing: bad argument");
        return PIT_E_INVALID;
    }
    PIT_TRY(h->p.timer.resolve());
    if (calls) *calls = h->p.timer.calls[cls];
    if (ms) *ms = h->p.timer.ms[cls];
    return PIT_OK;
}

pit_status pit_block_reduce(const double *U, const double *V, int nblocks, int M, double *dot,
                            double *norms, double *norm_inf) {
    if (!U || !V || !dot || !norm_inf || nblocks < 1 || M < 1) {
        set_error("pit_block_reduce: bad argument");
        return PIT_E_INVALID;
    }
    if (nblocks > PIT_MAX_BLOCKS) {
        set_error("pit_block_reduce: nblocks exceeds 65535 (one grid row per block)");
        return PIT_E_INVALID;
    }
    PIT_TRY(block_reduce(U, V, nblocks, M, dot, norms, norm_inf, 0));
    PIT_CUDA(cudaStreamSynchronize(0));
    return PIT_OK;
}

}  // extern "C"
