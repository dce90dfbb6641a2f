// Internal declarations shared by the libpit translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "pit.h"

namespace pit {

// The vector kernels put one grid row (gridDim.y) per block of a block
// vector and one grid layer (gridDim.z) per batch member; both are limited
// to 65535.
constexpr int PIT_MAX_BLOCKS = 65535;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
pit_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define PIT_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::pit::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define PIT_TRY(call)                                                         \
    do {                                                                      \
        pit_status s_ = (call);                                               \
        if (s_ != PIT_OK) return s_;                                          \
    } while (0)

extern std::atomic<unsigned long long> g_launches;   // all threads
extern thread_local unsigned long long tl_launches;   // this thread

#define PIT_LAUNCH_CHECK()                                                    \
    do {                                                                      \
        g_launches.fetch_add(1, std::memory_order_relaxed);                   \
        ++tl_launches;                                                        \
        PIT_CUDA(cudaGetLastError());                                         \
    } while (0)

// Raises the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes` (cudaFuncAttributeMaxDynamicSharedMemorySize).
// The limit belongs to the function for the whole process, so solves that
// run at once on several host threads and set it to different values would
// race: one could lower it between another's set and that one's launch,
// which then fails.  Here the limit only grows, under a lock, so every
// launch after the call sees a limit no smaller than its request; a limit
// already large enough costs a table lookup and no driver call.
pit_status smem_limit_raw(const void *func, size_t bytes);
template <class F>
pit_status smem_limit(F *func, size_t bytes) {
    return smem_limit_raw(reinterpret_cast<const void *>(func), bytes);
}

// ------------------------------------------------------- device buffers
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t astream = nullptr;   // stream of a pool allocation (nullptr: cudaMalloc)
    pit_status ensure(size_t n);   // grows (never shrinks) the allocation
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Allocation context of the calling host thread.  When set (a serving slot),
// DevBuf allocations are stream-ordered allocations from `pool` on `stream`
// (no device-wide synchronisation on free, memory reused across requests)
// and are counted in cur / peak.
struct AllocCtx {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
    size_t cur = 0, peak = 0;
};
extern thread_local AllocCtx *tl_alloc;
// Set while this thread captures a CUDA graph: DevBuf::ensure must not
// allocate then (the capture is abandoned and the work runs eagerly).
extern thread_local bool tl_capturing;


// Per-member solver state, resident on the device (Algorithm 1 scalars).
struct MemberState {
    double rho;        // <R^k, R~>
    double sigma;      // <D^k, R~>
    double alpha, omega, beta;
    double dd;         // <D, D>
    double ks, kk;     // <K, S>, <K, K>
    double rho_new;    // <R^{k+1}, R~>
    double r2;         // <R^{k+1}, R^{k+1}>
    double rt2;        // <R~, R~>
    double r0;         // ||R^0||_{N,inf}
    double rnorm;      // ||R^k||_{N,inf}
    double snorm;      // ||S^k||_{N,inf}
    double thresh;     // stopping threshold
    double eps0, eps_b;
    int active;        // 1 while iterating
    int status;        // PIT_OK / PIT_E_*
    int iter, restarts, matvecs;
    int skip;          // this iteration restarts after a vanishing sigma (no update)
    int half;          // this iteration exits after the half step
    int just_restarted;
    int do_restart;    // update of P restarts R~ and P
    int max_iter;
    int pad_;
};

// Reduction scratch: partial sums of Q quantities per (member, block, chunk).
struct ReduceLayout {
    int Q;        // quantities
    int nblk;     // N + 1
    int chunks;   // chunks per block
    int chunk;    // elements per chunk
};

// Event timing of operator applications (diagnostics).
struct OpTimer {
    bool enabled = false;
    bool top_only = false;   // pit_set_timing(prob, 2): BiCGStab iterations timed as a whole
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    // while a CUDA graph is captured: records go here (external event-record
    // nodes that fire at every replay) instead of `pending`
    std::vector<Rec> *capture_into = nullptr;
    long long calls[PIT_TIME_CLASSES] = {};
    double ms[PIT_TIME_CLASSES] = {};
    cudaEvent_t get();
    pit_status begin(int cls, cudaStream_t s, Rec &r);
    pit_status end(Rec &r, cudaStream_t s);
    pit_status resolve();
    pit_status collect(const std::vector<Rec> &recs);   // one replay of a timed graph
    void release(std::vector<Rec> &recs);              // events back to the pool
    void reset();
    void destroy();
};

// One BiCGStab iteration (Algorithm 1: two applications of G^{-1}F and the
// fused vector updates) captured as a CUDA graph and replayed.
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    const void *ptrs[5] = {};     // buffers the captured kernels use
    bool timed = false;
    bool failed = false;          // capture not possible on this stream: run eagerly
    unsigned long long kernels = 0;   // kernel launches one replay stands for
    std::vector<OpTimer::Rec> recs;
};

// ---------------------------------------------------------------- problem
struct Problem {
    // description
    int kind = 0, nx = 0, ny = 0, M = 0, N = 0, batch = 0;
    double T = 0, dT = 0, nu = 0;
    int fine_kind = 0, fine_steps = 0, coarse_kind = 0, coarse_steps = 0;
    int coarse_inner = 0;   // advdiff coarse IE: Chebyshev steps per solve (0: default)
    int precision = PIT_FP64;
    size_t blen = 0;              // (N+1)*M
    size_t vlen = 0;              // batch*(N+1)*M
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = true;       // false: the stream belongs to a serving slot
    cudaStream_t copy_stream = nullptr;   // copy of the solution to host memory, beside the last check
    cudaEvent_t x_ready = nullptr, x_copied = nullptr;
    const volatile int *cancel = nullptr;   // serving: nonzero asks the solve to stop

    DevBuf y0;                    // batch*M

    // heat1d: Thomas factors of (I - dt L) for the fine and coarse steps
    DevBuf fine_inv64, fine_cp64, coarse_inv64, coarse_cp64;
    DevBuf fine_inv32, fine_cp32, coarse_inv32, coarse_cp32;
    DevBuf fine_invff;            // heat1d: fine Thomas factors as float-float (hi, lo) pairs
    int heat1d_small = 0;         // heat1d, M <= 256: one-warp kernels (else CTA-wide scans)
    int h1_phi_on = 0;            // heat1d FP64 fine batch through the propagator matrix A^{-m}
    DevBuf h1_phiT;               // ... its columns (M x M, FP64)
    int h1_pow_on = 0;            // heat1d FP64 sweep through the powers G^j (independent products)
    DevBuf h1_powT, h1_sweep_t;   // ... G^1..G^N by columns, and the products G^(n-k) q_k
    double fine_off = 0, coarse_off = 0;   // off-diagonal -dt nu / h^2

    // heat2d: sine basis S_jk = sin(pi j k/(n+1)) and coarse mode factors
    DevBuf S64, S32, gmode;       // gmode: (1 - dTc nu (mu_k + mu_l))^{-c}
    DevBuf xtc_S;                 // TF32 parts (hi, lo) of S for the tensor-core transforms
    int xform_tc = 0;             // 2D / 1D heat sweeps transform on the tensor cores
    int split_fold = 0;           // 2D heat split RK4 residual: the Z u_lo term among the FP32 terms
    DevBuf hat;                   // sweep scratch: transformed blocks

    // advdiff2d: per-point velocities (FP64 and FP32)
    DevBuf vx64, vy64, vx32, vy32;   // after set-up: ax = vx/h, ay = vy/h
    DevBuf vxff, vyff;            // advdiff coefficients as float-float (hi, lo) pairs
    DevBuf adv_scratch;
    int adv_K = 8;                // Chebyshev steps of the coarse IE step
    long long adv_spin = 1LL << 26;   // polls of each bounded wait of the advdiff sweep
    int adv_coef32 = 0;           // every coefficient v / h is an FP32 value (float-float lo parts zero)
    int adv_rx = 4;               // columns of the fine kernel's thread tiles (4, or 8 for n >= 256)
    double adv_inv_theta = 1.0, adv_c1[64] = {}, adv_c2[64] = {};   // Chebyshev coefficients

    // dense: fine propagator Phi and coarse matrix G (FP64 + split FP32)
    DevBuf PhiF64, G64, PhiF_hi, PhiF_lo, G32;
    DevBuf A64;                   // dense: a copy of A (steady states of a source)
    // source f of y' = L y + f (time-independent): the fine propagator is
    // affine, F_f(x) = F(x) + c, c = F_f(0) per member (batch x M, FP64)
    DevBuf cvec;
    bool has_src = false;
    DevBuf dense_scratch;
    void *blas = nullptr;         // cuBLAS handle (dense set-up and FP64 products)
    DevBuf GL32;                  // G^L (FP32) for the chunked dense sweep
    DevBuf GLL32;                 // G^(L L2) (FP32): carries across super-chunks
    int sweep_L = 1;              // chunk length of the dense sweep
    int sweep_L2 = 1;             // chunks per super-chunk of the carry scan
    DevBuf errword;               // device-side error word of bounded waits (0 = none)
    DevBuf PhiTh, PhiTl, tc_split;  // TF32 splits of Phi and of the input block vector
    bool use_tc = false;          // dense FP32-class product on the tensor cores
    bool dense_bf16 = false;      // ... in split BF16 (PIT_MIXED_BF16) instead of split TF32
    DevBuf PhiBh, PhiBl;          // BF16 splits of Phi
    bool dtc_on = false;          // dense mixed sweep on the tensor cores (dense_sweep_tc.cu)
    DevBuf dtc_mats;              // its TF32 (hi, lo) splits of G and of G^(L 2^s), s < S
    DevBuf dtc_buf;               // its chunk states (ping-pong hi, lo, FP32) and barrier words
    bool oz_on = false;           // dense true residual (PIT_SPLIT) by error-free splitting on the tensor cores
    DevBuf oz_phi, oz_ephi;       // ... BF16 digit slices of Phi and its row exponents
    DevBuf oz_x, oz_ex;           // ... slices and row exponents of the block vector (per product)

    // Krylov workspace
    DevBuf X, R, Rt, P, S, D, K, W;
    DevBuf partials, states, flags_host_mirror;
    DevBuf fine_tmp;              // serial / misc scratch
    DevBuf q32;                   // FP32 block-operator rows of the mixed G^{-1}F
    // heat2d fine-kernel variant for n <= 128 (autotuned for FP32 and
    // float-float): 0 one CTA of 4-column tiles, 1 one CTA of 8-column
    // tiles (FP32 only), 2 a cluster of CTAs with 8 x 4 tiles
    int fine_var32 = 0, fine_var_ff = 0;
    bool kr_cluster = false;      // Krylov partials of 2..8-chunk blocks reduced per cluster
    int fine_var32_big = 0, fine_var_ff_big = 0;   // n > 128: 8-column clusters (0) or wide 4-column ones (1)
    ReduceLayout rl{};
    OpTimer timer;
    IterGraph igraph[2];          // [0]: FP64 iterations, [1]: mixed (FP32 fine) iterations
    // the iteration loop as one graph (a conditional while node around the
    // captured iteration): [0] FP64, [1] mixed
    IterGraph lgraph[2];
    DevBuf loopctl;               // iterations run by the current loop-graph launch (one int)
    int loop_chunk = 16;          // iterations per loop-graph launch; 0: per-iteration graphs
    bool use_graphs = true;       // PIT_GRAPHS=0 in the environment turns graphs off
};

// Modes of the fused block-operator epilogue.
enum { FINE_APPLY = 0, FINE_RESIDUAL = 1 };

// ---------------------------------------------------------- operator API
// y = F x (mode FINE_APPLY) or y = B - F x (mode FINE_RESIDUAL); every block.
// `states` (may be null) masks inactive members.
pit_status op_apply_F(Problem *p, const double *x, double *y, int mode, int precision,
                      const MemberState *states, cudaStream_t s);
// z = G^{-1} q (in place allowed: z == q).
pit_status op_sweep(Problem *p, const double *q, double *z, int precision,
                    const MemberState *states, cudaStream_t s);
// Lam = serial fine trajectory.
pit_status op_serial(Problem *p, double *Lam, int precision, cudaStream_t s);

// per-family implementations
pit_status heat1d_setup(Problem *p);
// 1D heat, FP64: whether set-up stores the fine propagator matrix A^{-m}
// and the powers G^j of the coarse propagator (the environment switches
// aside), and the device bytes those tables and the sweep's products take.
bool heat1d_phi_wanted(int M, int fine_steps, int precision);
bool heat1d_pow_wanted(int M, int N, int coarse_steps, int precision);
size_t heat1d_table_bytes(int M, int N, int batch, int fine_steps, int coarse_steps, int precision);
pit_status heat1d_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                          const MemberState *st, cudaStream_t s);
pit_status heat1d_sweep(Problem *p, const double *q, double *z, int prec,
                        const MemberState *st, cudaStream_t s);
pit_status heat1d_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s);

pit_status heat2d_setup(Problem *p);
pit_status heat2d_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                          const MemberState *st, cudaStream_t s);
pit_status heat2d_sweep(Problem *p, const double *q, double *z, int prec,
                        const MemberState *st, cudaStream_t s);
pit_status heat2d_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s);
// mixed G^{-1}F: FP32 fine batch writing FP32 rows, then the FP32-input sweep
pit_status heat2d_fine_f32out(Problem *p, const double *x, float *q32, const MemberState *st,
                              cudaStream_t s);
pit_status heat2d_sweep_f32in(Problem *p, const float *q32, double *z, const MemberState *st,
                              cudaStream_t s);

pit_status advdiff_setup(Problem *p);
pit_status advdiff_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                           const MemberState *st, cudaStream_t s);
pit_status advdiff_sweep(Problem *p, const double *q, double *z, int prec,
                         const MemberState *st, cudaStream_t s);
pit_status advdiff_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s);

pit_status dense_setup(Problem *p);
pit_status dense_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                         const MemberState *st, cudaStream_t s);
pit_status dense_sweep(Problem *p, const double *q, double *z, int prec,
                       const MemberState *st, cudaStream_t s);
pit_status dense_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s);
pit_status dense_steady_state(Problem *p, const double *f_host, double *ys_host);
// c = F_f(0) per member for a source f (host, batch x M); see source.cu
pit_status source_offset(Problem *p, const double *f_host);
// y[b][n][:] += c[b][:] for n = 1..N of every member (forced rows of eq. (4))
pit_status add_source_rows(Problem *p, double *y, cudaStream_t s);
void dense_teardown(Problem *p);
bool dense_tc_supported(const Problem *p);
pit_status dense_tc_split_phi(Problem *p);
bool dense_oz_supported(const Problem *p);
pit_status dense_oz_setup(Problem *p);
pit_status dense_oz_apply(Problem *p, const double *x, double *y, int mode, const MemberState *st,
                          cudaStream_t s);
// TF32 (hi, lo) parts of the rows_src x M row-major FP64 x into rows_out x Mp
// arrays (zero outside x)
pit_status tc_split_tf32(const double *x, float *hi, float *lo, int rows_src, int rows_out, int M,
                         int Mp, cudaStream_t s);
// dense mixed sweep on the tensor cores: at most 2^DTC_SMAX chunks
constexpr int DTC_SMAX = 7;
void dense_tc_sweep_shape(int N, int &L, int &C, int &S);
int dense_tc_sweep_padded(int M);
bool dense_tc_sweep_fits(const Problem *p);
pit_status dense_tc_sweep(Problem *p, const double *q, double *z, const MemberState *st,
                          cudaStream_t s, bool *launched);
pit_status dense_tc_apply(Problem *p, const double *x, double *y, float *y32, int mode,
                          const MemberState *st, cudaStream_t s);
// 2D heat sine transforms on the tensor cores (xform_tc.cu), 96 <= n <= 256,
// n % 4 == 0: out_b = scale (A_b S)^T for every n x n block b of A (FP32,
// 16-byte aligned), out FP32 or FP64.
bool heat2d_tc_usable(const Problem *p);
// 1D heat sweep in the sine basis on the tensor cores (mixed path): rows of
// length M padded to heat1d_tc_padded(M); S generated on the device.
int heat1d_tc_padded(int M);
pit_status heat1d_tc_setup(Problem *p);
pit_status heat1d_tc_pack(Problem *p, const double *q, float *out, cudaStream_t s);
pit_status heat1d_tc_xform(Problem *p, const float *A, void *out, bool out64, int nout, int ldo,
                           double scale, const MemberState *st, cudaStream_t s);
// per-mode recurrence of the sine-basis sweeps (heat2d.cu)
pit_status sine_mode_recurrence(Problem *p, float *hat, double *ends, int nn, const MemberState *st,
                                cudaStream_t s);
pit_status heat2d_tc_setup(Problem *p, const double *S);
pit_status heat2d_tc_xform(Problem *p, const float *A, void *out, bool out64, double scale,
                           const MemberState *st, cudaStream_t s);

// Autotuner (tune.cu): index of the fastest of ncand variants run(c), timed
// with CUDA events on stream s; cached per key, device SM count and process.
pit_status autotune(const std::string &key, int ncand, const std::function<pit_status(int)> &run,
                    cudaStream_t s, int *choice, int fallback = 0);
extern thread_local bool tl_tune_fallback;

// ------------------------------------------------------------ Krylov API
// pit_problem_create with an optional caller stream (not owned; nullptr: a
// stream of the problem's own).
pit_status problem_create(const pit_problem_desc *d, cudaStream_t ext_stream,
                          pit_problem_t *out);
pit_status krylov_prepare(Problem *p);   // allocates vectors, partials, states
// block copy of y0 into block 0 of each member and zeros elsewhere
pit_status build_rhs(Problem *p, double *B, cudaStream_t s);

// Kernel launchers (krylov.cu); every one masks inactive members.
// R computed: R~ = P = R; rho, r0; thresh = abs_thresh[b] (device array) if
// given, else tol_rel * r0
pit_status kr_init(Problem *p, double tol_rel, const double *abs_thresh, double eps0,
                   int max_iter, cudaStream_t s);
pit_status kr_sigma(Problem *p, cudaStream_t s);     // sigma = <D,R~>, alpha
pit_status kr_update_S(Problem *p, cudaStream_t s);  // S = R - alpha D, ||S||, half exit
pit_status kr_omega(Problem *p, cudaStream_t s);     // <K,S>, <K,K>, omega
pit_status kr_update_XR(Problem *p, cudaStream_t s); // X, R, rho_new, ||R||, beta, tests
pit_status kr_update_P(Problem *p, cudaStream_t s);  // P update or restart
pit_status kr_block_norm(Problem *p, const double *U, double *out_norm_per_member,
                         cudaStream_t s);            // ||U||_{N,inf} per member (device out)
pit_status kr_axpy(Problem *p, double *X, const double *Y, cudaStream_t s);  // X += Y
pit_status block_reduce(const double *U, const double *V, int nblocks, int M, double *dot,
                        double *norms, double *norm_inf, cudaStream_t s);

}  // namespace pit

struct pit_problem_s {
    pit::Problem p;
};
