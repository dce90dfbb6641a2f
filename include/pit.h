/*
 * pit.h -- C ABI of libpit: the parallel-in-time hot path of PiTSBiCG
 * (Riahi, "PiTSBiCG: Parallel in Time Stable Bi-Conjugate Gradient
 * Algorithm", arXiv 2203.10148) on NVIDIA GB300 (sm_103a).
 *
 * The problem (Sec. 2, eqs. (1)-(2)): a linear ODE or semi-discrete PDE
 * y' = L y on [0, T] with y(0) = y0, cut into N equal slices of length
 * dT = T/N.  A fine propagator F and a coarse propagator G advance a state
 * over one slice.  The unknown is Lambda = (lambda_0, ..., lambda_N), the
 * states at the slice boundaries (N+1 blocks of M values).  The all-at-once
 * system of eq. (4) is  F Lambda = B  with (F Lambda)_0 = lambda_0,
 * (F Lambda)_n = lambda_n - F(lambda_{n-1}) and B = (y0, 0, ..., 0); its
 * exact solution is the serial fine trajectory lambda_n = F^n y0.
 * PiTSBiCG (Algorithm 1) runs BiCGStab on the left-preconditioned system
 * G^{-1} F Lambda = G^{-1} B of eq. (8), where G^{-1} is the forward
 * substitution of eq. (7), right.
 *
 * Conventions for every call:
 *   - Every call returns a pit_status; PIT_OK (0) on success, a negative
 *     code on error.  No call aborts or exits the process.
 *     pit_last_error() returns a message for the calling thread's last error.
 *   - A "block vector" holds batch * (N+1) * M doubles, member-major, then
 *     slice-major: element (b, n, i) is at index (b*(N+1) + n)*M + i.
 *     2D states are row-major: point (i, j) of an nx-by-ny grid is i + j*nx.
 *   - on_device = 1: the pointer is CUDA device memory (for instance a torch
 *     tensor's data_ptr) on the current device; on_device = 0: host memory.
 *     Caller-owned arrays are never retained after a call returns.
 *   - stream: a cudaStream_t cast to void*, or NULL for the problem's own
 *     stream.  Calls taking a stream are asynchronous with respect to the
 *     host when on_device = 1 unless stated otherwise.
 *   - Calls on one problem must be serialised by the caller.
 */
#ifndef PIT_H
#define PIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pit_status;

#define PIT_OK              0
#define PIT_PENDING         1   /* serving: the request has not finished yet */
#define PIT_E_INVALID      -1   /* bad argument or descriptor */
#define PIT_E_NOMEM        -2   /* device or host allocation failed / over budget */
#define PIT_E_CUDA         -3   /* a CUDA runtime call failed */
#define PIT_E_BREAKDOWN    -4   /* BiCGStab breakdown: <D,R~> vanished twice, or omega = 0 */
#define PIT_E_MAXITER      -5   /* iteration limit reached before the tolerance */
#define PIT_E_NONFINITE    -6   /* NaN or Inf in an input or a Krylov scalar */
#define PIT_E_TIMEOUT      -7   /* a bounded device-side wait expired */
#define PIT_E_BUSY         -8   /* serving: no free slot and the queue is full */
#define PIT_E_UNSUPPORTED  -9   /* valid but not implemented combination */
#define PIT_E_CANCELLED   -10   /* serving: the request was cancelled */

/* Spatial operator families (the operator L of eq. (1), f = 0). */
#define PIT_OP_HEAT1D       1   /* nu u_xx, Dirichlet 0, nx interior points, h = 1/(nx+1) */
#define PIT_OP_HEAT2D       2   /* nu (u_xx + u_yy), 5-point, Dirichlet 0, nx = ny interior, h = 1/(n+1) */
#define PIT_OP_ADVDIFF2D    3   /* nu Lap u - v.grad u, periodic nx x ny, h = 1/nx, upwind advection */
#define PIT_OP_DENSE        4   /* y' = A y with a dense M x M matrix A */

/* Time steppers over one slice (fine F and coarse G). */
#define PIT_STEP_IE         1   /* implicit Euler: (I - dt L) u+ = u, dt = dT/steps */
#define PIT_STEP_RK4        2   /* classical RK4, dt = dT/steps; for PIT_OP_DENSE the
                                   fine RK4 propagator R(dt A)^steps is precomputed once
                                   and applied to all slices as one GEMM */

/* Arithmetic of the fine propagator. */
#define PIT_FP64            0   /* FP64 throughout */
#define PIT_MIXED           1   /* FP32 fine stepping (split-precision tensor-core GEMM for
                                   PIT_OP_DENSE), FP64 Krylov vectors and scalars, and
                                   iterative refinement on true residuals computed in
                                   PIT_SPLIT by default (PIT_FF or PIT_FP64 on request) */
#define PIT_FF              2   /* float-float fine arithmetic: each value an unevaluated sum
                                   of two FP32 numbers (about 48 significant bits) on the
                                   FP32 pipe, FP64 inputs and outputs: stepping for HEAT2D
                                   and ADVDIFF2D, the Thomas recurrences for HEAT1D, a
                                   compensated product for DENSE */
#define PIT_MIXED_BF16      4   /* problem precision only: PIT_MIXED with the dense fine
                                   product split in BF16 instead of TF32 ("3xBF16": x = xh + xl
                                   and Phi = ph + pl with BF16 parts, xh ph + xh pl + xl ph on
                                   tcgen05 kind::f16 with FP32 accumulation; about 2^-16
                                   relative per product against 2^-21 for split TF32, twice
                                   the MMA rate and half the operand bytes); refinement keeps
                                   results within the tolerance.  Other operators: PIT_MIXED */
#define PIT_SPLIT           3   /* split arithmetic of the true residual.  DENSE: the
                                   product Phi x by error-free splitting (Ozaki et al. 2012):
                                   7 BF16 slices of 6-bit digits per row of Phi and of the
                                   block vector, the slice products of each anti-diagonal
                                   summed exactly in FP32 on the tensor cores, the sums
                                   added in float-float (within about 2^-42 of
                                   sum |phi| |x|); for M <= 1024, PIT_FF above.  HEAT2D:
                                   split RK4 (other operators treat it as PIT_FF):
                                   each step u + Z u + Z^2 u/2 + Z^3 u/6 + Z^4 u/24 (Z = dt L)
                                   takes the first-order term Z u in float-float and the
                                   others in FP32 (nested form) and keeps the state in
                                   float-float: about 68 FP32 operations per point and step
                                   against 179.  Used where ||Z|| = 8 nu dt / h^2 <= 1/8, so
                                   that the FP32 terms are <= 8.1e-3 |u| and their rounding
                                   costs <= about 5e-10 |u| per step (1.4e-3 and 1e-10 on the
                                   128^2 workload; far less on smooth components, where the
                                   terms scale with |Z|^2); larger steps run PIT_FF */

/* pit_apply_operator: which operator. */
#define PIT_APPLY_F         1   /* y = F x, the block operator of eq. (4) */
#define PIT_APPLY_GINV      2   /* y = G^{-1} x, the forward substitution of eq. (7), right */
#define PIT_APPLY_GINV_F    3   /* y = G^{-1} F x, the preconditioned operator of eq. (8) */
#define PIT_APPLY_RESIDUAL  4   /* y = G^{-1}(B - F x), Algorithm 1, first line */

/* Initial guess X^0 of Algorithm 1. */
#define PIT_X0_COARSE       0   /* G^{-1} B: lambda_n = G^n y0 (the parareal predictor) */
#define PIT_X0_ZERO         1
#define PIT_X0_GIVEN        2   /* X holds the initial guess on entry */

typedef struct pit_problem_s *pit_problem_t;
typedef struct pit_server_s *pit_server_t;

typedef struct {
    int kind;              /* PIT_OP_* */
    int nx, ny;            /* grid; HEAT1D and DENSE: nx = M, ny = 1 */
    double nu;             /* diffusion coefficient (unused for DENSE) */
    const double *vx;      /* ADVDIFF2D: host arrays of nx*ny velocities; copied at create */
    const double *vy;
    const double *A;       /* DENSE: host M*M row-major matrix; copied at create */
} pit_operator_desc;

typedef struct {
    int kind;              /* PIT_STEP_* */
    int steps;             /* steps per slice, >= 1 */
    int inner;             /* coarse IE of PIT_OP_ADVDIFF2D: Chebyshev steps replacing
                              each linear solve (Saad, Sec. 12.3), 1 .. 64; 0 takes 48.
                              Ignored elsewhere (the other coarse solves are exact). */
} pit_stepper_desc;

typedef struct {
    pit_operator_desc op;
    const double *y0;      /* host, batch * M initial values; copied at create */
    int batch;             /* independent initial values sharing the operator, >= 1 */
    double T;              /* end time, > 0 */
    int N;                 /* number of time slices, >= 1 */
    pit_stepper_desc fine;
    pit_stepper_desc coarse;
    int precision;         /* PIT_FP64, PIT_MIXED or PIT_MIXED_BF16 */
} pit_problem_desc;

typedef struct {
    double tol;            /* stop when ||R^k||_{N,inf} <= tol * ||R^0||_{N,inf} */
    double restart_eps0;   /* restart when |<R^{k+1},R~>| <= eps0 ||R^{k+1}||_2 ||R~||_2 */
    int max_iter;          /* BiCGStab iterations (per refinement round in PIT_MIXED) */
    int x0_mode;           /* PIT_X0_* */
    int refine_max;        /* PIT_MIXED: outer refinement rounds, >= 1 */
    double inner_tol;      /* PIT_MIXED: relative tolerance of each inner solve */
    void *stream;          /* cudaStream_t or NULL */
    double *history;       /* optional host array: ||R^k||_{N,inf} of member 0 per
                              iteration (PIT_FP64) or per refinement round (PIT_MIXED) */
    int history_len;
    int residual_precision; /* PIT_MIXED: arithmetic of the fine propagations inside the
                               true residual, PIT_SPLIT (default), PIT_FF or PIT_FP64 */
    int tol_mode;          /* PIT_TOL_R0 (default) or PIT_TOL_RHS */
} pit_solve_opts;

/* Reference of the relative tolerance. */
#define PIT_TOL_R0          0   /* tol * ||R^0||_{N,inf}, R^0 the first (true) residual */
#define PIT_TOL_RHS         1   /* tol * ||G^{-1} B||_{N,inf}, independent of X^0 */

typedef struct {
    int iterations;        /* BiCGStab iterations (summed over refinement rounds) */
    int matvecs;           /* applications of G^{-1} F (FP32 and FP64) */
    int restarts;
    int refinements;       /* PIT_MIXED: outer rounds taken */
    long long fine_slice_steps;  /* slices propagated x fine steps per slice */
    double r0;             /* ||R^0||_{N,inf} */
    double precond_resid;  /* final ||R||_{N,inf}: recursive (FP64) or true (PIT_MIXED) */
    double seconds;        /* wall time of the call */
    int status;            /* pit_status of this member */
    int history_count;     /* entries written to opts->history */
    double queue_seconds;  /* serving: submission to admission (0 otherwise) */
    double latency_seconds;  /* serving: submission to result on the host (0 otherwise) */
    long long device_bytes;  /* serving: peak device bytes the request held (0 otherwise) */
    int graph_iterations;  /* BiCGStab iterations run as replays of the captured CUDA graph */
} pit_solve_info;

/* Fills *opts with defaults: tol 1e-10, eps0 1e-8, max_iter 500, X0 coarse,
 * refine_max 8, inner_tol 1e-4, default stream, no history, PIT_SPLIT true
 * residuals (split RK4 for HEAT2D where its bound holds, error-free
 * splitting for DENSE with M <= 1024, float-float otherwise), tolerance
 * relative to ||R^0||. */
void pit_default_opts(pit_solve_opts *opts);

/* Version string of the library. */
const char *pit_version(void);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to n bytes); returns the length of the full message. */
size_t pit_last_error(char *buf, size_t n);

/*
 * Creates a problem on the current CUDA device (Sec. 2, eqs. (1)-(4)).
 * Copies y0, A, vx, vy into library-owned device memory (the caller may free
 * its arrays on return) and runs the set-up: stepper factorisations, the
 * sine-basis tables of the 2D heat coarse solver, or the dense propagator
 * (R(dt A) or (I - dt A)^{-1})^steps and G = (I - dT A)^{-1} for PIT_OP_DENSE.
 * Supported: HEAT1D with IE fine and IE coarse; HEAT2D (nx = ny <= 256) with
 * RK4 fine and IE coarse; ADVDIFF2D (n = 32 .. 512, a power of two) with RK4
 * fine and one IE coarse step; DENSE with RK4 or IE fine and IE coarse.
 * The ADVDIFF2D coarse step (I - dT L) w = b has variable coefficients and
 * no fast exact solver: G maps b to the iterate after coarse.inner steps of
 * Chebyshev acceleration on the Jacobi-scaled system D^{-1}(I - dT L),
 * started from w = b, for the interval [1 - rho, 1 + rho], rho =
 * max_p (D_p - 1)/D_p (Gershgorin).  G is a fixed linear operator, so the
 * solution of eq. (4) does not depend on coarse.inner; the iteration count
 * does.  The default 48 solves the implicit-Euler system to a relative
 * residual below 1e-6 on the 512^2 workload (white noise and its smooth
 * initial value), so G is the implicit-Euler step to that accuracy; 16 is
 * faster there (same iteration count, inner residual 3e-2 on white noise,
 * 2e-5 on the smooth data), 8 leaves 0.7 and 7e-4.  Where advection
 * dominates a stiff step (cell Peclet number |v| h / nu and dT |v| / h both
 * well above 1) the scaled spectrum leaves the real interval and large
 * counts stop converging to the implicit-Euler step.
 * Others return PIT_E_UNSUPPORTED.
 * Set-up reads these environment variables (none changes a result beyond
 * rounding: every choice computes the same operator):
 *   PIT_GRAPHS=0           CUDA graphs of the iterations off (pit_bicgstab_solve);
 *   PIT_GRAPH_LOOP=k       iterations per launch of the loop graph (default
 *                          16; 0: one graph launch per iteration);
 *   PIT_HEAT2D_TC=0        mixed 2D heat sweeps (96 <= n <= 256) on the FP32
 *                          pipe instead of the tensor cores;
 *   PIT_HEAT1D_TC=0        mixed 1D heat sweeps as sequential FP32 Thomas
 *                          solves instead of sine transforms on the tensor cores;
 *   PIT_HEAT1D_SMALL=cta   1D heat grids of M <= 256 on the CTA-wide scans
 *                          instead of the one-warp kernels;
 *   PIT_HEAT1D_PHI=0       FP64 1D heat fine batch by its m implicit-Euler
 *                          steps instead of one product with the stored
 *                          propagator matrix A^-m (small grids);
 *   PIT_HEAT1D_POW=0       FP64 1D heat sweep as N dependent coarse solves
 *                          instead of the independent products with stored
 *                          powers of G (small grids, N <= 128);
 *   PIT_SPLIT_FOLD=1       2D heat split RK4 residual with the low word's
 *                          first-order term among the FP32 terms (off by
 *                          default: not yet run on a GPU);
 *   PIT_ADV_COEF32=0       ADVDIFF2D float-float stages keep the velocity
 *                          coefficients' low parts even when all are FP32 values;
 *   PIT_ADV_RX=8           ADVDIFF2D fine kernels on 8 x 8 thread tiles for
 *                          n >= 256 (default 8 x 4);
 *   PIT_DENSE_OZ=0         DENSE true residual by the float-float product
 *                          instead of error-free splitting on the tensor cores;
 *   PIT_DENSE_SWEEP_TC=0   DENSE sweep on the CUDA cores instead of the
 *                          tensor-core chunked scan;
 *   PIT_HEAT2D_VARIANTS=a,b  2D heat fine-kernel variants for n <= 128 (FP32
 *                          a in 0..3, float-float b in {0, 2}) instead of the
 *                          autotuner's choice (bit-identical results);
 *   PIT_AUTOTUNE=0         untuned shapes take the built-in variant;
 *   PIT_AUTOTUNE_CACHE=f   persist the autotuner's choices in file f;
 *   PIT_KRYLOV_CLUSTERS=1  the Krylov kernels reduce a block's 2..8 chunks
 *                          of 2048 values in a thread-block cluster
 *                          (distributed shared memory, one partial per
 *                          block) instead of storing one partial per chunk
 *                          (the same results bit for bit; measured 6% slower
 *                          on the Krylov kernels of the 128^2 workload, so
 *                          off by default);
 *   PIT_SPIN_LIMIT=k       polls of each bounded wait of the ADVDIFF2D coarse
 *                          sweep (neighbouring bands' progress flags) before
 *                          the call reports PIT_E_TIMEOUT (default 2^26; a
 *                          small k exercises the timeout path: the sweep's
 *                          CTAs all return, the call fails with
 *                          PIT_E_TIMEOUT and the context stays usable).
 * Errors: PIT_E_INVALID (bad sizes, including N + 1 > 65535 or batch > 65535:
 * the vector kernels put one grid row per block and one grid layer per
 * member), PIT_E_NONFINITE (non-finite values), PIT_E_NOMEM, PIT_E_CUDA.
 */
pit_status pit_problem_create(const pit_problem_desc *desc, pit_problem_t *out);

/* Frees every resource of the problem.  NULL is accepted. */
pit_status pit_problem_destroy(pit_problem_t prob);

/* Sizes of a problem: M values per state, N slices, batch members. */
pit_status pit_problem_shape(pit_problem_t prob, int *M, int *N, int *batch);

/*
 * Applies one operator to a block vector x, writing y (both batch*(N+1)*M):
 * PIT_APPLY_F (eq. (4)), PIT_APPLY_GINV (eq. (7) right, sequential in n),
 * PIT_APPLY_GINV_F (eq. (8)), PIT_APPLY_RESIDUAL (G^{-1}(B - F x)).
 * precision selects the fine arithmetic (PIT_FP64, PIT_MIXED = FP32 fine
 * stepping from FP64 inputs, or PIT_FF = float-float arithmetic, about 48
 * significant bits on the FP32 pipe: stepping for PIT_OP_HEAT2D and
 * PIT_OP_ADVDIFF2D, a compensated product for PIT_OP_DENSE; PIT_SPLIT is
 * split RK4 for PIT_OP_HEAT2D, the product by error-free splitting on the
 * tensor cores for PIT_OP_DENSE with M <= 1024, and PIT_FF elsewhere; PIT_FF is the
 * float-float Thomas recurrence for PIT_OP_HEAT1D).  Every dense product runs on the library's kernels for
 * any M (tcgen05 split TF32 for PIT_MIXED, rows padded to 128; float-float
 * for PIT_FF, padded to 64; FP64 tiles for PIT_FP64).  G^{-1} runs
 * in reduced precision for PIT_MIXED (2D heat and 1D heat: split-TF32 sine
 * transforms on the tensor cores with float-float running sums in the sine
 * basis; advection-diffusion and dense: FP32) and in FP64 otherwise.
 * x and y may not overlap.
 * With on_device = 0 the call copies through device memory and synchronises.
 */
pit_status pit_apply_operator(pit_problem_t prob, int which, int precision,
                              const double *x, double *y, int on_device, void *stream);

/*
 * The serial fine trajectory lambda_n = F^n y0 (eq. (7), left: F^{-1} B),
 * computed on the device one slice after the other in the given precision.
 * Lam holds batch*(N+1)*M values.  Synchronous.
 */
pit_status pit_serial_fine(pit_problem_t prob, int precision, double *Lam, int on_device);

/*
 * PiTSBiCG (Algorithm 1) on G^{-1} F X = G^{-1} B for every batch member.
 * X (batch*(N+1)*M): initial guess on entry when x0_mode = PIT_X0_GIVEN,
 * the solution on return.  info: array of batch entries (may be NULL).
 * PIT_FP64: every step in FP64 on the device.  PIT_MIXED: iterative
 * refinement: the true residual G^{-1}(B - F X) with the fine propagations
 * in opts.residual_precision (PIT_SPLIT by default: split RK4 for HEAT2D,
 * error-free splitting on the tensor cores for DENSE with M <= 1024,
 * float-float on the FP32 pipe elsewhere; PIT_FF or PIT_FP64 on request),
 * an FP32-fine /
 * FP64-Krylov inner solve of the correction to inner_tol, X += correction,
 * until the true preconditioned residual is <= tol * its reference
 * (opts.tol_mode).
 * For PIT_OP_HEAT1D and PIT_OP_HEAT2D one iteration (two applications of
 * G^{-1}F and the fused vector kernels) is captured as a CUDA graph after
 * the first, eager, iteration of each inner solve and replayed for the
 * others; the graph is kept with the problem (re-captured when the stream
 * or the timing mode changes) and info.graph_iterations counts the
 * replays.  By default the replays run as a loop graph: a conditional
 * while node around the captured iteration and a one-warp condition kernel
 * that stops it once no member is active or after PIT_GRAPH_LOOP (16)
 * iterations, so that the host reads the member states once per launch
 * instead of once per iteration (cancellation and the iteration guard are
 * checked between launches).  With event timing (pit_set_timing)
 * or a residual history (opts.history) one graph launch runs one
 * iteration.  Results are bit for bit those of eager launches; the loop
 * graph launches one condition kernel more per iteration.  The
 * environment variable PIT_GRAPHS=0, read by pit_problem_create, turns the
 * graphs off; a stream that cannot be captured (the legacy default stream)
 * runs every iteration eagerly.
 * Synchronous.  Returns the worst member status (PIT_E_MAXITER,
 * PIT_E_BREAKDOWN, PIT_E_NONFINITE) or PIT_OK.
 */
pit_status pit_bicgstab_solve(pit_problem_t prob, const pit_solve_opts *opts, double *X,
                              int on_device, pit_solve_info *info);

/*
 * Parareal in the algebraic form of eq. (6):
 * X^{k+1} = X^k + G^{-1}(B - F X^k), X^0 = G^{-1} B, in the problem's fine
 * precision (FP64 true residual in PIT_FP64), stopping when the preconditioned
 * residual is <= tol * its initial value or after kmax corrections.
 * Synchronous.
 */
pit_status pit_parareal_solve(pit_problem_t prob, int kmax, double tol, double *X,
                              int on_device, pit_solve_info *info);

/*
 * Deterministic block reductions used by the Krylov kernels, exposed for
 * testing: for block vectors U, V of nblocks blocks of M values,
 * *dot = sum of U.V over all entries (the block inner product, Sec. 3 text
 * after Algorithm 1), norms[n] = ||U_n||_2, *norm_inf = max_n norms[n]
 * (the ||.||_{N,inf} of Algorithm 1).  Device pointers; synchronous.
 * norms may be NULL.  1 <= nblocks <= 65535 (one grid row per block) and
 * M >= 1, else PIT_E_INVALID before any device call.
 */
pit_status pit_block_reduce(const double *U, const double *V, int nblocks, int M,
                            double *dot, double *norms, double *norm_inf);

/*
 * Allocation-free variant of pit_block_reduce, with the same arguments,
 * results and synchronisation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory, for
 * instance a process whose device memory is all reserved by another
 * allocator (so cudaMalloc would fail), or a latency-bound thread that
 * cannot pay for cudaMalloc/cudaFree.  The partial sums live in a fixed
 * 1 MiB array compiled into the library, which every device that loads the
 * library keeps until the process exits; it holds nblocks * ceil(M/2048)
 * <= 65536 chunks, and larger sizes (or nblocks > 65535, as for
 * pit_block_reduce) return PIT_E_INVALID without touching the device.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (from several threads or streams) race and must be
 * serialised by the caller.  Nothing in the array needs to start at zero.
 */
pit_status pit_block_reduce_noalloc(const double *U, const double *V, int nblocks, int M,
                                    double *dot, double *norms, double *norm_inf);

/*
 * Replaces the initial values y0 (batch * M doubles, host or device) of an
 * existing problem; the operator and its set-up are kept.  Synchronous.
 * Errors: PIT_E_INVALID, PIT_E_NONFINITE (host arrays only), PIT_E_CUDA.
 */
pit_status pit_problem_set_y0(pit_problem_t prob, const double *y0, int on_device);

/* -------------------------------------------------------------- serving */
/*
 * A request server on the current device: continuous batching of PiTSBiCG
 * solves (the mixed-precision or FP64 solve of pit_bicgstab_solve, Algorithm
 * 1 on eq. (8)) of different sizes N and grids, submitted while others run.
 *
 * max_slots (1..64) worker threads each own a CUDA stream.  A free worker
 * admits the first queued request whose device footprint
 * (pit_serve_footprint) fits hbm_budget_bytes next to the running ones,
 * builds its problem with stream-ordered allocations from a memory pool of
 * the server, solves it and copies the result to host memory; the GPU work
 * of up to max_slots requests overlaps.  A request that does not fit may be
 * overtaken by later, smaller ones 16 times at most.  hbm_budget_bytes = 0
 * takes 80% of the device's free memory.  Freed pool memory is kept (up to
 * the budget) for later requests.  Each result does not depend on the
 * other requests: it equals the result of pit_bicgstab_solve on the same
 * problem and options alone.
 *
 * The server is thread-safe: any thread may submit, poll, wait or cancel.
 * Kinds served: PIT_OP_HEAT1D and PIT_OP_HEAT2D (PIT_E_UNSUPPORTED
 * otherwise).  Errors: PIT_E_INVALID (max_slots, null out), PIT_E_CUDA.
 */
pit_status pit_server_create(size_t hbm_budget_bytes, int max_slots, pit_server_t *out);

/* Cancels queued requests, asks running ones to stop at their next
 * iteration, joins the workers and frees everything; results not yet taken
 * are dropped.  NULL is a no-op. */
pit_status pit_server_destroy(pit_server_t server);

/*
 * Queues one request.  Everything is copied: desc (with y0; vx, vy and A are
 * not used by the served kinds) and opts (its stream, history and
 * history_len are ignored: the server uses its slot's stream).  *ticket
 * identifies the request in poll / wait / cancel.  Validation of the
 * operator's values (finite y0, supported steppers) happens when the
 * request runs and is reported by poll.
 * Errors: PIT_E_INVALID (null argument, bad sizes, server stopping),
 * PIT_E_UNSUPPORTED (kind), PIT_E_NOMEM (the footprint alone exceeds the
 * budget), PIT_E_BUSY (2^20 requests queued).
 */
pit_status pit_serve_submit(pit_server_t server, const pit_problem_desc *desc,
                            const pit_solve_opts *opts, uint64_t *ticket);

/*
 * Non-blocking: PIT_PENDING while the request is queued or running.
 * Otherwise the request's final status (that of pit_bicgstab_solve, or
 * PIT_E_CANCELLED, or the set-up error), with the result copied to X_out
 * (host, batch*(N+1)*M doubles; may be NULL) and one pit_solve_info per
 * member to info (may be NULL; queue_seconds, latency_seconds and
 * device_bytes filled in); the request is then released and its ticket
 * becomes unknown (PIT_E_INVALID).  X_out is left untouched when the solve
 * failed before producing an iterate.
 */
pit_status pit_serve_poll(pit_server_t server, uint64_t ticket, double *X_out,
                          pit_solve_info *info);

/* pit_serve_poll that blocks until the request is done or timeout_s seconds
 * have passed (PIT_PENDING); timeout_s < 0 waits without limit.  Where
 * several callers wait on one ticket, the first to wake takes the result and
 * the others return PIT_E_INVALID. */
pit_status pit_serve_wait(pit_server_t server, uint64_t ticket, double timeout_s,
                          double *X_out, pit_solve_info *info);

/* A queued request is removed (its poll returns PIT_E_CANCELLED); a running
 * one stops at its next BiCGStab iteration or refinement round and reports
 * PIT_E_CANCELLED.  Errors: PIT_E_INVALID (unknown ticket). */
pit_status pit_serve_cancel(pit_server_t server, uint64_t ticket);

/* Device bytes the server reserves for a request of this description: an
 * upper bound of what its problem allocates (eight Krylov block vectors,
 * the FP32 fine output and sine-mode work of the 2D sweep, set-up tables,
 * reduction partials; for FP64 1D heat on small grids also the stored fine
 * propagator matrix, the powers of the coarse propagator and the sweep's
 * (N+1)(N+2)/2 products per member).  Host-only. */
pit_status pit_serve_footprint(const pit_problem_desc *desc, size_t *bytes);

typedef struct {
    long long submitted, completed, failed, cancelled;  /* failed: completed with status != OK */
    long long queued, running;
    int max_running;       /* most requests running at once */
    int slots;
    double latency_p50, latency_p99, latency_mean;  /* submission to result, seconds */
    double queue_p50, queue_p99;                    /* submission to admission */
    double service_p50, service_p99;                /* admission to result */
    double window_seconds;  /* first submission to last completion */
    double solves_per_s;    /* successful solves / window */
    double slice_steps_per_s;  /* fine slice-steps of completed solves / window */
    size_t hbm_budget, hbm_reserved, hbm_reserved_peak;  /* admission footprints */
    size_t pool_peak;       /* high-water mark of the pool's reserved device memory */
} pit_server_stats_t;

/* Statistics of the requests completed since creation or the last reset
 * (percentiles by nearest rank); reset = 1 starts a new window. */
pit_status pit_server_stats(pit_server_t server, int reset, pit_server_stats_t *out);

/*
 * A time-independent source: the problem becomes y' = L y + f (eq. (1) with
 * f != 0), f holding batch * M values (host or device; NULL removes the
 * source).  The fine propagator is then affine, F_f(x) = F(x) + c with
 * c = F_f(0), so the rows n >= 1 of eq. (4) read lambda_n - F(lambda_{n-1})
 * = c and B = (y0, c, ..., c); the Krylov operator G^{-1} F stays linear.
 * c is computed here in FP64 as y* - F(y*) from the steady state y*
 * (L y* = -f), which both fine steppers keep fixed.  Afterwards every
 * residual, right-hand side and serial trajectory includes the source.
 * Supported for PIT_OP_HEAT1D, PIT_OP_HEAT2D (nu > 0) and PIT_OP_DENSE (A
 * invertible).  Synchronous.
 * Errors: PIT_E_INVALID, PIT_E_NONFINITE, PIT_E_UNSUPPORTED, PIT_E_CUDA.
 */
pit_status pit_problem_set_source(pit_problem_t prob, const double *f, int on_device);

/* ---------------------------------------------------------- diagnostics */

/* Number of kernels libpit has launched in this process (all problems). */
unsigned long long pit_kernel_launches(void);

/* Self-test of the integer-pipe FP64 -> FP32 (round to nearest even) and
 * FP32 -> FP64 conversions the kernels use in place of the hardware
 * conversion: f32[i] = convert(in[i]), back[i] = convert(f32[i]).  Device
 * pointers, n values; synchronous. */
pit_status pit_selftest_convert(const double *in, int n, float *f32, double *back);

/* Operator classes timed by pit_get_timing. */
#define PIT_TIME_FINE_FP32   0   /* fine batch, FP32 stepping (one kernel per call) */
#define PIT_TIME_FINE_FP64   1   /* fine batch, FP64 stepping (one kernel per call) */
#define PIT_TIME_SWEEP_MIXED 2   /* coarse sweep, FP32 transforms */
#define PIT_TIME_SWEEP_FP64  3   /* coarse sweep, FP64 */
#define PIT_TIME_KRYLOV      4   /* fused BiCGStab vector kernels and finishers */
#define PIT_TIME_FINE_FF     5   /* fine batch, float-float stepping (one kernel per call) */
#define PIT_TIME_FINE_SPLIT  6   /* fine batch, split RK4 stepping (one kernel per call) */
#define PIT_TIME_INNER       7   /* with pit_set_timing(prob, 2): each launch of a solve's
                                    BiCGStab iterations as a whole (loop graph, iteration
                                    graph or eager iteration) */
#define PIT_TIME_CLASSES     8

/*
 * enable = 1: every later operator application of this problem is bracketed
 * by CUDA events on the stream it runs on, and the elapsed times are summed
 * per class (the BiCGStab iterations then replay one graph per iteration,
 * so that each application inside them can be timed); enable = 2: only the
 * applications outside the iterations (true residuals, the initial sweep)
 * are timed by class, and each launch of the iterations -- which then run
 * as the loop graph, as without timing -- as a whole, in PIT_TIME_INNER;
 * enable = 0 stops recording.  Resets the sums.
 */
pit_status pit_set_timing(pit_problem_t prob, int enable);

/* Calls and summed milliseconds of one class since pit_set_timing(prob, 1).
 * Synchronises the problem's pending events. */
pit_status pit_get_timing(pit_problem_t prob, int cls, long long *calls, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* PIT_H */
