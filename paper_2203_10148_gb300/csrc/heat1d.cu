// 1D heat u_t = nu u_xx (Dirichlet 0, M interior points, h = 1/(M+1)):
// implicit-Euler fine propagator over all N slices at once (the N
// independent problems of eq. (2)), fused with the shift-subtract of the
// block operator of eq. (4), and the sequential coarse sweep G^{-1} of
// eq. (7), right.
//
// Each implicit-Euler step solves the tridiagonal system (I - dt nu D2) u+ = u.
// The Thomas elimination is two first-order linear recurrences,
//   forward  d'_i = -a inv_i d'_{i-1} + inv_i d_i,
//   backward x_i  = -c'_i x_{i+1} + d'_i,
// with inv_i and c'_i precomputed once on the host.  A linear recurrence is
// a composition of affine maps, so one CTA evaluates it with a parallel
// scan: every thread composes the maps of its E contiguous points, the CTA
// scans the per-thread maps (warp shuffles, then a short pass over warps),
// and every thread replays its points from the scanned prefix.  A slice's
// state stays in registers across all fine steps.  The fine kernel runs in
// FP64, FP32 or float-float (the true residual of the mixed path: every
// product and sum of the recurrences as float-float operations on the FP32
// pipe, Thomas factors stored as (hi, lo) pairs).
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "pit_internal.h"
#include "stencil_arith.cuh"

namespace pit {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// The arithmetic the recurrences need, for FP32 / FP64 and float-float.
template <class T> __device__ __forceinline__ T one() { return T(1); }
template <class T> __device__ __forceinline__ T zero() { return T(0); }
template <> __device__ __forceinline__ ff one<ff>() { return ff{1.f, 0.f}; }
template <> __device__ __forceinline__ ff zero<ff>() { return ff{0.f, 0.f}; }
__device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff operator-(ff a) { return ff{-a.hi, -a.lo}; }
template <class T> __device__ __forceinline__ T fmaT(T a, T b, T c) { return fma(a, b, c); }
template <> __device__ __forceinline__ ff fmaT<ff>(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

template <class T>
struct Aff {
    T a, c;
};

// later o earlier
template <class T>
__device__ __forceinline__ Aff<T> comp(Aff<T> later, Aff<T> earlier) {
    return Aff<T>{later.a * earlier.a, fmaT(later.a, earlier.c, later.c)};
}

template <class T>
__device__ __forceinline__ T shfl_dir(T v, int o, bool rev) {
    return rev ? __shfl_down_sync(FULL, v, o) : __shfl_up_sync(FULL, v, o);
}
template <>
__device__ __forceinline__ ff shfl_dir<ff>(ff v, int o, bool rev) {
    return ff{shfl_dir(v.hi, o, rev), shfl_dir(v.lo, o, rev)};
}

// Exclusive scan of affine maps over the CTA.  Scan order is thread order
// (REV = false) or reversed thread order (REV = true).  sh: 4*NT/32 values.
template <class T, int NT, bool REV>
__device__ Aff<T> cta_affine_excl(Aff<T> v, T *sh) {
    constexpr int W = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Aff<T> inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T a = shfl_dir(inc.a, o, REV);
        const T c = shfl_dir(inc.c, o, REV);
        const bool ok = REV ? (lane + o < 32) : (lane >= o);
        if (ok) inc = comp(inc, Aff<T>{a, c});
    }
    const T ea = shfl_dir(inc.a, 1, REV);
    const T ec = shfl_dir(inc.c, 1, REV);
    const bool first = REV ? (lane == 31) : (lane == 0);
    Aff<T> exw = first ? Aff<T>{one<T>(), zero<T>()} : Aff<T>{ea, ec};
    if (W == 1) return exw;
    const int last = REV ? 0 : 31;
    __syncthreads();
    if (lane == last) {
        sh[warp] = inc.a;
        sh[W + warp] = inc.c;
    }
    __syncthreads();
    // prefix over the warps' aggregates: warp 0 scans them with shuffles
    // (lane l holds warp l's map, W <= 32) and leaves each warp's exclusive
    // prefix in shared memory
    if (warp == 0) {
        Aff<T> wv = (lane < W) ? Aff<T>{sh[lane], sh[W + lane]} : Aff<T>{one<T>(), zero<T>()};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T a = shfl_dir(wv.a, o, REV);
            const T c = shfl_dir(wv.c, o, REV);
            const bool ok = REV ? (lane + o < 32) : (lane >= o);
            if (ok) wv = comp(wv, Aff<T>{a, c});
        }
        // inclusive prefix at lane l -/+ 1 is the exclusive prefix of warp l
        const T pa = shfl_dir(wv.a, 1, REV);
        const T pc = shfl_dir(wv.c, 1, REV);
        const bool none = REV ? (lane == W - 1) : (lane == 0);
        __syncwarp();
        if (lane < W) {
            sh[2 * W + lane] = none ? one<T>() : pa;
            sh[3 * W + lane] = none ? zero<T>() : pc;
        }
    }
    __syncthreads();
    const Aff<T> wp{sh[2 * W + warp], sh[3 * W + warp]};
    return comp(exw, wp);
}

// Thomas factors of this thread's E points, loaded once per kernel:
// fm_i = -a inv_i, inv_i, ncp_i = -c'_i; padding points (i >= M) get the
// identity map (fm = 1, inv = 0, ncp = 1) and never feed a valid point.
template <class T, int E>
struct Factors {
    T fm[E], inv[E], ncp[E];
    bool ok[E];
    __device__ void load(const T *__restrict__ fmg, const T *__restrict__ invg,
                         const T *__restrict__ cpg, int M) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            ok[e] = i < M;
            const int ic = min(i, M - 1);
            fm[e] = ok[e] ? fmg[ic] : one<T>();
            inv[e] = ok[e] ? invg[ic] : zero<T>();
            ncp[e] = ok[e] ? -cpg[ic] : one<T>();
        }
    }
};

// One implicit-Euler step on the CTA-distributed state u (E points per
// thread, thread t owns points t*E .. t*E+E-1).
template <class T, int E, int NT>
__device__ __forceinline__ void ie_step(T (&u)[E], const Factors<T, E> &f, T *sh) {
    // forward: d'_i = fm_i d'_{i-1} + inv_i d_i
    Aff<T> agg{one<T>(), zero<T>()};
    T lc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        lc[e] = f.inv[e] * u[e];
        agg = comp(Aff<T>{f.fm[e], lc[e]}, agg);
    }
    Aff<T> pre = cta_affine_excl<T, NT, false>(agg, sh);
    T y = pre.c;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        y = fmaT(f.fm[e], y, lc[e]);
        u[e] = y;                       // d'_i
    }
    // backward: x_i = -cp_i x_{i+1} + d'_i, scanned from the last point
    agg = Aff<T>{one<T>(), zero<T>()};
#pragma unroll
    for (int e = E - 1; e >= 0; --e) {
        lc[e] = f.ok[e] ? u[e] : zero<T>();
        agg = comp(Aff<T>{f.ncp[e], lc[e]}, agg);
    }
    pre = cta_affine_excl<T, NT, true>(agg, sh + 4 * (NT / 32));
    y = pre.c;
#pragma unroll
    for (int e = E - 1; e >= 0; --e) {
        y = fmaT(f.ncp[e], y, lc[e]);
        u[e] = y;
    }
}

struct Heat1dArgs {
    const double *x;
    double *y;
    const double *y0;
    int M, N, batch;
    size_t blen;
    int n_first;    // output slice index of blockIdx.x == 0
    int mode;       // FINE_APPLY, FINE_RESIDUAL, or 2 = plain (y_n = F(x_{n-1}))
    int steps;
    const MemberState *st;
};

__device__ __forceinline__ bool runs(const MemberState *st, int b) {
    return st == nullptr || (st[b].active && !st[b].skip && !st[b].half);
}

// Fine batch: CTA (slice n, member b) propagates x_{n-1} over `steps` IE
// steps and writes the block-operator row n.
template <class T, int E, int NT>
__global__ void __launch_bounds__(NT) k_heat1d_fine(Heat1dArgs a, const T *__restrict__ fm,
                                                    const T *__restrict__ inv,
                                                    const T *__restrict__ cp) {
    __shared__ T sh[8 * (NT / 32)];
    const int b = blockIdx.y;
    if (!runs(a.st, b)) return;
    const int n = a.n_first + blockIdx.x;    // output block, 1..N
    const size_t mb = (size_t)b * a.blen;
    const double *xin = a.x + mb + (size_t)(n - 1) * a.M;
    T u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        T ld;
        if constexpr (std::is_same<T, float>::value) ld = d2f_rn(xin[min(i, a.M - 1)]);  // integer pipe
        else if constexpr (std::is_same<T, ff>::value) ld = ff_from_double(xin[min(i, a.M - 1)]);
        else ld = xin[min(i, a.M - 1)];
        u[e] = (i < a.M) ? ld : zero<T>();
    }
    Factors<T, E> f;
    f.load(fm, inv, cp, a.M);
    for (int s = 0; s < a.steps; ++s) ie_step<T, E, NT>(u, f, sh);
    double *yo = a.y + mb + (size_t)n * a.M;
    const double *xn = a.x + mb + (size_t)n * a.M;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        if (i < a.M) {
            double f;
            if constexpr (std::is_same<T, float>::value) f = f2d(u[e]);
            else if constexpr (std::is_same<T, ff>::value) f = ff_to_double(u[e]);
            else f = u[e];
            if (a.mode == FINE_APPLY) yo[i] = xn[i] - f;
            else if (a.mode == FINE_RESIDUAL) yo[i] = f - xn[i];
            else yo[i] = f;
        }
    }
    if (n == 1 && a.mode != 2) {
        // row 0 of eq. (4): (F X)_0 = x_0; residual: y0 - x_0
        const double *x0 = a.x + mb;
        double *y0o = a.y + mb;
        for (int i = threadIdx.x; i < a.M; i += NT)
            y0o[i] = (a.mode == FINE_APPLY) ? x0[i] : a.y0[(size_t)b * a.M + i] - x0[i];
    }
}

// Coarse sweep z_0 = q_0, z_n = q_n + G(z_{n-1}), one CTA per member,
// sequential in n.  G is `steps` IE steps in arithmetic T.  FP64: the
// running sum z_n is FP64.  FP32 (the mixed path): everything is FP32 and
// the FP64 <-> FP32 conversions run on the integer pipe, so a step has no
// FP64-pipe work (one CTA runs the whole sweep, and the FP64 pipe of one SM
// is 2 lanes wide); G(z_{n-1}) is an FP32 solve in both forms, so the FP32
// running sum costs no accuracy the FP64 one had.
template <int E, int NT>
__global__ void __launch_bounds__(NT) k_heat1d_sweep_f32(const double *q, double *z, int M, int N,
                                                        size_t blen, int steps,
                                                        const float *__restrict__ fm,
                                                        const float *__restrict__ inv,
                                                        const float *__restrict__ cp,
                                                        const MemberState *st) {
    __shared__ float sh[8 * (NT / 32)];
    const int b = blockIdx.x;
    if (!runs(st, b)) return;
    const size_t mb = (size_t)b * blen;
    Factors<float, E> fac;
    fac.load(fm, inv, cp, M);
    float zz[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        const double ld = q[mb + min(i, M - 1)];
        zz[e] = (i < M) ? d2f_rn(ld) : 0.f;
        if (i < M) z[mb + i] = ld;          // z_0 = q_0 exactly
    }
    // q_n is loaded one slice ahead so that its latency overlaps a solve
    double qnext[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        qnext[e] = (i < M && N >= 1) ? q[mb + (size_t)M + i] : 0.0;
    }
    for (int n = 1; n <= N; ++n) {
        const size_t off = mb + (size_t)n * M;
        float qn[E];
#pragma unroll
        for (int e = 0; e < E; ++e) qn[e] = d2f_rn(qnext[e]);
        if (n < N) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = threadIdx.x * E + e;
                qnext[e] = (i < M) ? q[off + (size_t)M + i] : 0.0;
            }
        }
        float u[E];
#pragma unroll
        for (int e = 0; e < E; ++e) u[e] = zz[e];
        for (int s = 0; s < steps; ++s) ie_step<float, E, NT>(u, fac, sh);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            if (i < M) {
                zz[e] = qn[e] + u[e];
                z[off + i] = f2d(zz[e]);
            } else {
                zz[e] = 0.f;
            }
        }
    }
}

template <class T, int E, int NT>
__global__ void __launch_bounds__(NT) k_heat1d_sweep(const double *q, double *z, int M, int N,
                                                     size_t blen, int steps,
                                                     const T *__restrict__ fm,
                                                     const T *__restrict__ inv,
                                                     const T *__restrict__ cp,
                                                     const MemberState *st) {
    __shared__ T sh[8 * (NT / 32)];
    const int b = blockIdx.x;
    if (!runs(st, b)) return;
    const size_t mb = (size_t)b * blen;
    Factors<T, E> fac;
    fac.load(fm, inv, cp, M);
    double zz[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        const double ld = q[mb + min(i, M - 1)];
        zz[e] = (i < M) ? ld : 0.0;
        if (i < M) z[mb + i] = zz[e];
    }
    for (int n = 1; n <= N; ++n) {
        const size_t off = mb + (size_t)n * M;
        // q_n is loaded before the solve so that its latency overlaps it
        double qn[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            qn[e] = (i < M) ? q[off + i] : 0.0;
        }
        T u[E];
#pragma unroll
        for (int e = 0; e < E; ++e) u[e] = (T)zz[e];
        for (int s = 0; s < steps; ++s) ie_step<T, E, NT>(u, fac, sh);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            if (i < M) {
                zz[e] = qn[e] + (double)u[e];
                z[off + i] = zz[e];
            } else {
                zz[e] = 0.0;
            }
        }
    }
}

// ------------------------------------------------- small grids (M <= 256)
// One warp per slice, E points per lane.  The multiplier halves of the
// affine maps in both Thomas scans are products of the constant factors, so
// the kernel forms, once per launch, each lane's multiplier for every level
// of the two warp scans and the products of its own points' factors; an
// implicit-Euler step then carries only data: a lane composes its E points
// (E - 1 dependent operations), the warp scan takes one fused multiply-add
// per level, and every point's value is one independent multiply-add from
// the lane's incoming value.  The state between steps is w = inv .* u (the
// right-hand side of the forward recurrence), formed in the backward fix-up
// off the dependent chain.  Per step: 2 (E - 1) + 12 dependent operations
// and 12 warp shuffles; the small-grid solves are bound by that chain (FP64
// result latency and shuffles), not by the FP64 pipe's throughput.
constexpr int WARP_MAXM = 256;

template <class T, int E>
struct WarpThomas {
    T fm[E], ncp[E], inv[E];
    T P[E], Q[E], iQ[E];  // prod_{k<=e} fm_k, prod_{k>=e} ncp_k, inv_e Q_e (this lane's points)
    T fa[5], ba[5];       // level multipliers of the forward / backward scans (0: no partner)

    // Padding points (i >= M) get fm = ncp = inv = 0: they hold 0 and cut
    // every chain through them.
    __device__ void load(const T *__restrict__ fmg, const T *__restrict__ invg,
                         const T *__restrict__ cpg, int M) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane * E + e;
            const bool ok = i < M;
            const int ic = min(i, M - 1);
            fm[e] = ok ? fmg[ic] : zero<T>();
            inv[e] = ok ? invg[ic] : zero<T>();
            ncp[e] = ok ? -cpg[ic] : zero<T>();
        }
        P[0] = fm[0];
#pragma unroll
        for (int e = 1; e < E; ++e) P[e] = fm[e] * P[e - 1];
        Q[E - 1] = ncp[E - 1];
#pragma unroll
        for (int e = E - 2; e >= 0; --e) Q[e] = ncp[e] * Q[e + 1];
#pragma unroll
        for (int e = 0; e < E; ++e) iQ[e] = inv[e] * Q[e];
        T A = P[E - 1], B = Q[0];
        // inclusive scans of the multipliers; level l combines with the lane
        // 2^l before (forward) / after (backward)
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            const int o = 1 << l;
            const bool fwd = lane >= o, bwd = lane + o < 32;
            fa[l] = fwd ? A : zero<T>();
            ba[l] = bwd ? B : zero<T>();
            const T Ao = shfl_dir(A, o, false);
            const T Bo = shfl_dir(B, o, true);
            if (fwd) A = A * Ao;
            if (bwd) B = B * Bo;
        }
    }

    // One implicit-Euler step: w = inv .* u in, w of the new u out (and the
    // new u in x when X).  Lane owns points lane*E .. lane*E+E-1.
    template <bool X>
    __device__ __forceinline__ void step(T (&w)[E], T (&x)[E]) const {
        const int lane = threadIdx.x & 31;
        // forward: d_i = fm_i d_{i-1} + w_i
        T L[E];
        L[0] = w[0];
#pragma unroll
        for (int e = 1; e < E; ++e) L[e] = fmaT(fm[e], L[e - 1], w[e]);
        T c = L[E - 1];
#pragma unroll
        for (int l = 0; l < 5; ++l) c = fmaT(fa[l], shfl_dir(c, 1 << l, false), c);
        T pre = shfl_dir(c, 1, false);
        if (lane == 0) pre = zero<T>();
        T d[E];
#pragma unroll
        for (int e = 0; e < E; ++e) d[e] = fmaT(P[e], pre, L[e]);
        // backward: x_i = -cp_i x_{i+1} + d_i
        L[E - 1] = d[E - 1];
#pragma unroll
        for (int e = E - 2; e >= 0; --e) L[e] = fmaT(ncp[e], L[e + 1], d[e]);
        c = L[0];
#pragma unroll
        for (int l = 0; l < 5; ++l) c = fmaT(ba[l], shfl_dir(c, 1 << l, true), c);
        pre = shfl_dir(c, 1, true);
        if (lane == 31) pre = zero<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            w[e] = fmaT(iQ[e], pre, inv[e] * L[e]);
            if (X) x[e] = fmaT(Q[e], pre, L[e]);
        }
    }

    // `steps` implicit-Euler steps on x.
    __device__ __forceinline__ void run(T (&x)[E], int steps) const {
        T w[E];
#pragma unroll
        for (int e = 0; e < E; ++e) w[e] = inv[e] * x[e];
        for (int s = 0; s + 1 < steps; ++s) step<false>(w, x);
        if (steps > 0) step<true>(w, x);
    }
};

template <class T>
__device__ __forceinline__ T load_as(const double *p) {
    if constexpr (std::is_same<T, float>::value) return d2f_rn(*p);
    else if constexpr (std::is_same<T, ff>::value) return ff_from_double(*p);
    else return *p;
}
template <class T>
__device__ __forceinline__ double store_as(T v) {
    if constexpr (std::is_same<T, float>::value) return f2d(v);
    else if constexpr (std::is_same<T, ff>::value) return ff_to_double(v);
    else return v;
}

// Fine batch on small grids: warp (slice n, member b).
template <class T, int E>
__global__ void __launch_bounds__(32) k_heat1d_fine_warp(Heat1dArgs a, const T *__restrict__ fm,
                                                         const T *__restrict__ inv,
                                                         const T *__restrict__ cp) {
    const int b = blockIdx.y;
    if (!runs(a.st, b)) return;
    const int n = a.n_first + blockIdx.x;
    const int M = a.M;
    const size_t mb = (size_t)b * a.blen;
    const double *xin = a.x + mb + (size_t)(n - 1) * M;
    T u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        const T ld = load_as<T>(xin + min(i, M - 1));
        u[e] = (i < M) ? ld : zero<T>();
    }
    WarpThomas<T, E> f;
    f.load(fm, inv, cp, M);
    f.run(u, a.steps);
    double *yo = a.y + mb + (size_t)n * M;
    const double *xn = a.x + mb + (size_t)n * M;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        if (i < M) {
            const double v = store_as<T>(u[e]);
            if (a.mode == FINE_APPLY) yo[i] = xn[i] - v;
            else if (a.mode == FINE_RESIDUAL) yo[i] = v - xn[i];
            else yo[i] = v;
        }
    }
    if (n == 1 && a.mode != 2) {
        // row 0 of eq. (4): (F X)_0 = x_0; residual: y0 - x_0
        const double *x0 = a.x + mb;
        double *y0o = a.y + mb;
        for (int i = threadIdx.x; i < M; i += 32)
            y0o[i] = (a.mode == FINE_APPLY) ? x0[i] : a.y0[(size_t)b * M + i] - x0[i];
    }
}

// y_i = sum_j A_ij x_j for row i = threadIdx.x (the CTA has at least M
// threads; A stored by columns, At[j * M + i]; x in shared memory): jb
// columns at a time (contiguous in At; jb a multiple of 4, every column of a
// small matrix at once) are copied into shared memory with asynchronous
// 16-byte copies issued back to back by all threads (one memory latency per
// block of columns, not one per load), then each thread adds its row over
// them in four partial sums (columns j mod 4, in order); returns (s0 + s1) +
// (s2 + s3).  `as` is 16-byte aligned.  Every thread of the CTA must call it.
constexpr int H1_JB = 32;   // columns per block at M = 256 (the shared-memory budget below)
constexpr int H1_SMEM_MAX = (258 + H1_JB * 256) * (int)sizeof(double);   // M <= 256
// columns per staged block: as many as the budget takes, a multiple of 4
inline int h1_jb(int M) {
    const int jb = (H1_SMEM_MAX / (int)sizeof(double) - 258) / M / 4 * 4;
    return std::max(4, std::min(jb, (M + 3) / 4 * 4));
}
// stride of the matrices G^j: M^2 rounded up to even, so that every matrix
// (and so every block of its columns) starts on a 16-byte boundary
__host__ __device__ __forceinline__ size_t h1_pow_stride(int M) { return ((size_t)M * M + 1) & ~(size_t)1; }
__device__ __forceinline__ double h1_matvec_row(const double *__restrict__ At, const double *xs, double *as,
                                                int M, int jb) {
    const int i = threadIdx.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int j0 = 0; j0 < M; j0 += jb) {
        const int jn = min(jb, M - j0);
        const int nd = jn * M;
        const double *src = At + (size_t)j0 * M;   // 16-byte aligned: j0 M is even
        __syncthreads();   // the previous block's reads are done (and x is stored)
        for (int t = threadIdx.x; t < nd / 2; t += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (unsigned)__cvta_generic_to_shared(as + 2 * t)),
                         "l"(src + 2 * t)
                         : "memory");
        if ((nd & 1) && threadIdx.x == 0) as[nd - 1] = src[nd - 1];
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (i < M) {
            int j = 0;
            for (; j + 3 < jn; j += 4) {
                a0 = fma(as[j * M + i], xs[j0 + j], a0);
                a1 = fma(as[(j + 1) * M + i], xs[j0 + j + 1], a1);
                a2 = fma(as[(j + 2) * M + i], xs[j0 + j + 2], a2);
                a3 = fma(as[(j + 3) * M + i], xs[j0 + j + 3], a3);
            }
            for (; j < jn; ++j) a0 = fma(as[j * M + i], xs[j0 + j], a0);
        }
    }
    return (a0 + a1) + (a2 + a3);
}

// FP64 fine batch through the propagator matrix (small grids): the m
// implicit-Euler steps of a slice are one fixed linear map Phi = A^{-m},
// formed once on the host; one CTA per (slice, member) forms Phi x_{n-1},
// a row per thread, with x_{n-1} in shared memory and Phi stored by columns
// (phiT[j * M + i] = Phi_ij: at each j the threads read consecutive words).
__global__ void __launch_bounds__(256) k_heat1d_fine_phi(Heat1dArgs a, const double *__restrict__ phiT, int jb) {
    extern __shared__ __align__(16) double xs[];   // x_{n-1}, then 32 columns of Phi
    const int b = blockIdx.y;
    if (!runs(a.st, b)) return;
    const int n = a.n_first + blockIdx.x;
    const int M = a.M;
    const size_t mb = (size_t)b * a.blen;
    const double *xin = a.x + mb + (size_t)(n - 1) * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) xs[i] = xin[i];
    const double v = h1_matvec_row(phiT, xs, xs + ((M + 1) & ~1), M, jb);
    double *yo = a.y + mb + (size_t)n * M;
    const double *xn = a.x + mb + (size_t)n * M;
    if (const int i = threadIdx.x; i < M) {
        if (a.mode == FINE_APPLY) yo[i] = xn[i] - v;
        else if (a.mode == FINE_RESIDUAL) yo[i] = v - xn[i];
        else yo[i] = v;
    }
    if (n == 1 && a.mode != 2) {
        // row 0 of eq. (4): (F X)_0 = x_0; residual: y0 - x_0
        const double *x0 = a.x + mb;
        double *y0o = a.y + mb;
        for (int i = threadIdx.x; i < M; i += blockDim.x)
            y0o[i] = (a.mode == FINE_APPLY) ? x0[i] : a.y0[(size_t)b * M + i] - x0[i];
    }
}

// FP64 coarse sweep on small grids through the powers of G: the solution
// of eq. (7)'s block-bidiagonal system is z_n = sum_{k <= n} G^(n-k) q_k, so
// with G^j formed once (j = 1..N, by columns: powT[(j-1) S + c M + r] =
// (G^j)_rc, S = M^2 rounded up to even) every product t_{n,k} = G^(n-k) q_k
// is independent: one CTA per (n, k) forms it (stage 1), one CTA per n sums
// t_{n,0..n} in that order (stage 2).  t is laid out per member as (N+1)(N+2)/2 rows of M, pair
// (n, k) at row n(n+1)/2 + k.  q and z may be the same array.
__global__ void __launch_bounds__(256) k_heat1d_sweep_pow1(const double *__restrict__ q, double *__restrict__ t,
                                                           const double *__restrict__ powT, int M, int N,
                                                           size_t blen, const MemberState *st, int jb) {
    extern __shared__ __align__(16) double qs[];   // q_k, then 32 columns of G^(n-k)
    const int b = blockIdx.y;
    if (!runs(st, b)) return;
    const int pidx = blockIdx.x;
    // pair index -> (n, k): n(n+1)/2 <= pidx < (n+1)(n+2)/2
    int n = (int)((sqrt(8.0 * pidx + 1.0) - 1.0) * 0.5);
    while ((n + 1) * (n + 2) / 2 <= pidx) ++n;
    while (n * (n + 1) / 2 > pidx) --n;
    const int k = pidx - n * (n + 1) / 2;
    const size_t npairs = (size_t)(N + 1) * (N + 2) / 2;
    const double *qk = q + (size_t)b * blen + (size_t)k * M;
    double *tp = t + ((size_t)b * npairs + pidx) * M;
    if (k == n) {
        for (int i = threadIdx.x; i < M; i += blockDim.x) tp[i] = qk[i];
        return;
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) qs[i] = qk[i];
    const double v = h1_matvec_row(powT + (size_t)(n - k - 1) * h1_pow_stride(M), qs, qs + ((M + 1) & ~1), M, jb);
    if (threadIdx.x < M) tp[threadIdx.x] = v;
}

__global__ void __launch_bounds__(256) k_heat1d_sweep_pow2(const double *__restrict__ t, double *__restrict__ z,
                                                           int M, int N, size_t blen, const MemberState *st) {
    const int b = blockIdx.y;
    if (!runs(st, b)) return;
    const int n = blockIdx.x;
    const size_t npairs = (size_t)(N + 1) * (N + 2) / 2;
    const double *tn = t + ((size_t)b * npairs + (size_t)n * (n + 1) / 2) * M;
    double *zn = z + (size_t)b * blen + (size_t)n * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k <= n; ++k) acc += tn[(size_t)k * M + i];
        zn[i] = acc;
    }
}

// FP64 coarse sweep on small grids, one warp per member:
// z_0 = q_0, z_n = q_n + G z_{n-1}.
template <int E>
__global__ void __launch_bounds__(32) k_heat1d_sweep_warp(const double *q, double *z, int M, int N,
                                                          size_t blen, int steps,
                                                          const double *__restrict__ fm,
                                                          const double *__restrict__ inv,
                                                          const double *__restrict__ cp,
                                                          const MemberState *st) {
    const int b = blockIdx.x;
    if (!runs(st, b)) return;
    const size_t mb = (size_t)b * blen;
    WarpThomas<double, E> f;
    f.load(fm, inv, cp, M);
    double zz[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = threadIdx.x * E + e;
        const double ld = q[mb + min(i, M - 1)];
        zz[e] = (i < M) ? ld : 0.0;
        if (i < M) z[mb + i] = ld;
    }
    for (int n = 1; n <= N; ++n) {
        const size_t off = mb + (size_t)n * M;
        double qn[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            qn[e] = (i < M) ? q[off + i] : 0.0;
        }
        f.run(zz, steps);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = threadIdx.x * E + e;
            if (i < M) {
                zz[e] += qn[e];
                z[off + i] = zz[e];
            } else {
                zz[e] = 0.0;
            }
        }
    }
}

// Thomas factors of tridiag(a, 1 - 2a, a), a = -dt nu/h^2.
void thomas_factors(int M, double r, std::vector<double> &fm, std::vector<double> &inv,
                    std::vector<double> &cp) {
    const double a = -r, b = 1.0 + 2.0 * r;
    fm.assign(M, 0.0);
    inv.assign(M, 0.0);
    cp.assign(M, 0.0);
    double cprev = 0.0;
    for (int i = 0; i < M; ++i) {
        const double den = (i == 0) ? b : b - a * cprev;
        inv[i] = 1.0 / den;
        fm[i] = (i == 0) ? 0.0 : -a * inv[i];
        cp[i] = (i == M - 1) ? 0.0 : a * inv[i];
        cprev = cp[i];
    }
}

pit_status upload_factors(int M, double r, DevBuf &b64, DevBuf &b32, cudaStream_t s,
                          DevBuf *bff = nullptr) {
    std::vector<double> fm, inv, cp;
    thomas_factors(M, r, fm, inv, cp);
    std::vector<double> all(3 * (size_t)M);
    std::vector<float> all32(3 * (size_t)M);
    for (int i = 0; i < M; ++i) {
        all[i] = fm[i];
        all[M + i] = inv[i];
        all[2 * M + i] = cp[i];
    }
    for (size_t i = 0; i < all.size(); ++i) all32[i] = (float)all[i];
    PIT_TRY(b64.ensure(all.size() * sizeof(double)));
    PIT_TRY(b32.ensure(all32.size() * sizeof(float)));
    PIT_CUDA(cudaMemcpyAsync(b64.ptr, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    PIT_CUDA(cudaMemcpyAsync(b32.ptr, all32.data(), all32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    if (bff) {
        // float-float factors: (hi, lo) with hi = RN32(x), lo = RN32(x - hi)
        std::vector<float> allff(2 * all.size());
        for (size_t i = 0; i < all.size(); ++i) {
            const float hi = (float)all[i];
            allff[2 * i] = hi;
            allff[2 * i + 1] = (float)(all[i] - (double)hi);
        }
        PIT_TRY(bff->ensure(allff.size() * sizeof(float)));
        PIT_CUDA(cudaMemcpyAsync(bff->ptr, allff.data(), allff.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, s));
        PIT_CUDA(cudaStreamSynchronize(s));   // allff is a local buffer
    }
    return PIT_OK;
}

template <class T>
const T *fptr(const DevBuf &b, int M, int which) {
    return b.as<T>() + (size_t)which * M;
}

// Threads and points per thread for a state of M points.
template <class F>
pit_status dispatch_1d(int M, F &&f) {
    // a few points per thread: the CTA scans cost shuffles per warp, the
    // per-thread compositions cost a dependent chain per point
    if (M <= 64) return f.template run<1, 64>();
    if (M <= 256) return f.template run<2, 128>();
    if (M <= 1024) return f.template run<4, 256>();
    if (M <= 2048) return f.template run<8, 256>();
    if (M <= 4096) return f.template run<8, 512>();
    if (M <= 8192) return f.template run<8, 1024>();
    set_error("heat1d: M > 8192 is not supported");
    return PIT_E_UNSUPPORTED;
}

template <class T>
struct FineLaunch {
    Problem *p;
    Heat1dArgs a;
    int nslices;
    const DevBuf *fac;
    cudaStream_t s;
    template <int E, int NT>
    pit_status run() {
        const T *base = fac->as<T>();
        const int M = p->M;
        k_heat1d_fine<T, E, NT><<<dim3(nslices, p->batch), NT, 0, s>>>(a, base, base + M,
                                                                        base + 2 * M);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
};

template <class T>
struct SweepLaunch {
    Problem *p;
    const double *q;
    double *z;
    const DevBuf *fac;
    const MemberState *st;
    cudaStream_t s;
    template <int E, int NT>
    pit_status run() {
        const T *base = fac->as<T>();
        const int M = p->M;
        if constexpr (std::is_same<T, float>::value) {
            k_heat1d_sweep_f32<E, NT><<<p->batch, NT, 0, s>>>(q, z, M, p->N, p->blen,
                                                              p->coarse_steps, base, base + M,
                                                              base + 2 * M, st);
        } else {
            k_heat1d_sweep<T, E, NT><<<p->batch, NT, 0, s>>>(q, z, M, p->N, p->blen,
                                                              p->coarse_steps, base, base + M,
                                                              base + 2 * M, st);
        }
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
};

template <class T>
struct FineWarpLaunch {
    Problem *p;
    Heat1dArgs a;
    int nslices;
    const DevBuf *fac;
    cudaStream_t s;
    template <int E>
    pit_status run() {
        const T *base = fac->as<T>();
        const int M = p->M;
        k_heat1d_fine_warp<T, E><<<dim3(nslices, p->batch), 32, 0, s>>>(a, base, base + M,
                                                                         base + 2 * M);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
};

struct SweepWarpLaunch {
    Problem *p;
    const double *q;
    double *z;
    const MemberState *st;
    cudaStream_t s;
    template <int E>
    pit_status run() {
        const double *base = p->coarse_inv64.as<double>();
        const int M = p->M;
        k_heat1d_sweep_warp<E><<<p->batch, 32, 0, s>>>(q, z, M, p->N, p->blen, p->coarse_steps,
                                                       base, base + M, base + 2 * M, st);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
};

// Points per lane of the one-warp kernels (M <= 256).
template <class F>
pit_status dispatch_warp(int M, F &&f) {
    if (M <= 64) return f.template run<2>();
    if (M <= 128) return f.template run<4>();
    return f.template run<8>();
}

pit_status fine_launch(Problem *p, Heat1dArgs a, int nslices, int prec, cudaStream_t s) {
    if (prec == PIT_FP64 && p->h1_phi_on) {
        const int nt = std::min(256, (p->M + 31) / 32 * 32);
        const int jb = h1_jb(p->M);
        const size_t sm = (size_t)(((p->M + 1) & ~1) + jb * p->M) * sizeof(double);
        PIT_TRY(smem_limit(k_heat1d_fine_phi, H1_SMEM_MAX));
        k_heat1d_fine_phi<<<dim3(nslices, p->batch), nt, sm, s>>>(
            a, p->h1_phiT.as<double>(), jb);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
    if (p->M <= WARP_MAXM && p->heat1d_small) {
        if (prec == PIT_FP64) {
            FineWarpLaunch<double> f{p, a, nslices, &p->fine_inv64, s};
            return dispatch_warp(p->M, f);
        }
        if (prec == PIT_FF) {
            FineWarpLaunch<ff> f{p, a, nslices, &p->fine_invff, s};
            return dispatch_warp(p->M, f);
        }
        FineWarpLaunch<float> f{p, a, nslices, &p->fine_inv32, s};
        return dispatch_warp(p->M, f);
    }
    if (prec == PIT_FP64) {
        FineLaunch<double> f{p, a, nslices, &p->fine_inv64, s};
        return dispatch_1d(p->M, f);
    }
    if (prec == PIT_FF) {
        FineLaunch<ff> f{p, a, nslices, &p->fine_invff, s};
        return dispatch_1d(p->M, f);
    }
    FineLaunch<float> f{p, a, nslices, &p->fine_inv32, s};
    return dispatch_1d(p->M, f);
}

// Phi = A^{-m}, A = tridiag(-r, 1 + 2r, -r): column j is m Thomas solves of
// the unit vector e_j in FP64 (A^{-1} contracts, so the rounding of each
// solve is not amplified); uploaded by columns (phiT[j * M + i] = Phi_ij).
// `times` implicit-Euler solves A d <- d in place (Thomas, FP64).
void solve_times(const std::vector<double> &fm, const std::vector<double> &inv, const std::vector<double> &cp,
                 std::vector<double> &d, int times) {
    const int M = (int)d.size();
    for (int s = 0; s < times; ++s) {
        d[0] = inv[0] * d[0];
        for (int i = 1; i < M; ++i) d[i] = fm[i] * d[i - 1] + inv[i] * d[i];
        for (int i = M - 2; i >= 0; --i) d[i] = d[i] - cp[i] * d[i + 1];
    }
}

pit_status upload_fine_matrix(Problem *p, double r) {
    const int M = p->M, m = p->fine_steps;
    std::vector<double> fm, inv, cp;
    thomas_factors(M, r, fm, inv, cp);
    std::vector<double> phiT((size_t)M * M), d(M);
    for (int j = 0; j < M; ++j) {
        for (int i = 0; i < M; ++i) d[i] = (i == j) ? 1.0 : 0.0;
        solve_times(fm, inv, cp, d, m);
        for (int i = 0; i < M; ++i) phiT[(size_t)j * M + i] = d[i];
    }
    PIT_TRY(p->h1_phiT.ensure(phiT.size() * sizeof(double)));
    PIT_CUDA(cudaMemcpyAsync(p->h1_phiT.ptr, phiT.data(), phiT.size() * sizeof(double), cudaMemcpyHostToDevice,
                             p->stream));
    PIT_CUDA(cudaStreamSynchronize(p->stream));   // phiT is a local buffer
    return PIT_OK;
}

// G^j = (A_c^{-c})^j for j = 1..N by columns: column c of G^j is c more
// coarse solves of column c of G^(j-1), so each carries only the rounding
// of j c contracting solves.
pit_status upload_sweep_powers(Problem *p, double r) {
    const int M = p->M, N = p->N, c = p->coarse_steps;
    std::vector<double> fm, inv, cp;
    thomas_factors(M, r, fm, inv, cp);
    const size_t S = h1_pow_stride(M);
    std::vector<double> powT((size_t)N * S, 0.0), d(M);
    for (int col = 0; col < M; ++col) {
        for (int i = 0; i < M; ++i) d[i] = (i == col) ? 1.0 : 0.0;
        for (int j = 1; j <= N; ++j) {
            solve_times(fm, inv, cp, d, c);
            for (int i = 0; i < M; ++i) powT[(size_t)(j - 1) * S + (size_t)col * M + i] = d[i];
        }
    }
    PIT_TRY(p->h1_powT.ensure(powT.size() * sizeof(double)));
    PIT_CUDA(cudaMemcpyAsync(p->h1_powT.ptr, powT.data(), powT.size() * sizeof(double), cudaMemcpyHostToDevice,
                             p->stream));
    PIT_CUDA(cudaStreamSynchronize(p->stream));   // powT is a local buffer
    return PIT_OK;
}

}  // namespace

// FP64 problems: the fine batch as one matrix product where that is cheaper
// than the steps: M^2 multiply-adds per slice against m steps of the
// one-warp Thomas kernel (about 32 (5E + 8) lane operations each, E = 2, 4,
// 8 points per lane), with the matrix formed on the host in bounded time.
bool heat1d_phi_wanted(int M, int fine_steps, int precision) {
    const int E = M <= 64 ? 2 : M <= 128 ? 4 : 8;
    return precision == PIT_FP64 && M <= WARP_MAXM &&
           (double)M * M < 0.5 * fine_steps * 32.0 * (5 * E + 8) && (double)M * M * fine_steps <= 1e8;
}

// FP64 problems: the sweep through the powers of G where the (N+1)(N+2)/2
// independent products stay small and the powers are formed on the host in
// bounded time.
bool heat1d_pow_wanted(int M, int N, int coarse_steps, int precision) {
    const double pairs = 0.5 * (N + 1.0) * (N + 2.0);
    return precision == PIT_FP64 && M <= WARP_MAXM && N <= 128 && pairs * M * M <= 4e6 &&
           (double)N * M * M * coarse_steps <= 1e8;
}

size_t heat1d_table_bytes(int M, int N, int batch, int fine_steps, int coarse_steps, int precision) {
    size_t b = 0;
    if (heat1d_phi_wanted(M, fine_steps, precision)) b += (size_t)M * M * sizeof(double);
    if (heat1d_pow_wanted(M, N, coarse_steps, precision))
        b += ((size_t)N * h1_pow_stride(M) + (size_t)batch * ((size_t)(N + 1) * (N + 2) / 2) * M) *
             sizeof(double);
    return b;
}

pit_status heat1d_setup(Problem *p) {
    if (p->fine_kind != PIT_STEP_IE || p->coarse_kind != PIT_STEP_IE) {
        set_error("heat1d: fine and coarse steppers must be implicit Euler");
        return PIT_E_UNSUPPORTED;
    }
    if (p->M > 8192) {
        set_error("heat1d: M > 8192 is not supported");
        return PIT_E_UNSUPPORTED;
    }
    // grids of M <= 256 points run the one-warp kernels unless
    // PIT_HEAT1D_SMALL=cta selects the CTA-wide scans
    const char *sq = getenv("PIT_HEAT1D_SMALL");
    p->heat1d_small = !(sq && !strcmp(sq, "cta"));
    const double h = 1.0 / (p->M + 1);
    const double rf = (p->dT / p->fine_steps) * p->nu / (h * h);
    const double rc = (p->dT / p->coarse_steps) * p->nu / (h * h);
    // fine factors in fine_inv64/32, coarse in coarse_inv64/32 (fm | inv | cp)
    PIT_TRY(upload_factors(p->M, rf, p->fine_inv64, p->fine_inv32, p->stream, &p->fine_invff));
    // FP64 problems: the fine batch as one product with the propagator
    // matrix where heat1d_phi_wanted says so (PIT_HEAT1D_PHI=0 keeps the
    // steps).  The matrices are formed on the host at set-up, so mixed
    // problems, whose solves run no FP64 fine batch, keep the steps for the
    // FP64 calls they may make
    {
        const char *pe = getenv("PIT_HEAT1D_PHI");
        p->h1_phi_on = heat1d_phi_wanted(p->M, p->fine_steps, p->precision) && !(pe && pe[0] == '0');
        if (p->h1_phi_on) PIT_TRY(upload_fine_matrix(p, rf));
    }
    // FP64 sweep through the powers of G where heat1d_pow_wanted says so
    // (PIT_HEAT1D_POW=0 keeps the sequential solves)
    {
        const char *pe = getenv("PIT_HEAT1D_POW");
        p->h1_pow_on = heat1d_pow_wanted(p->M, p->N, p->coarse_steps, p->precision) && !(pe && pe[0] == '0');
        if (p->h1_pow_on) PIT_TRY(upload_sweep_powers(p, rc));
    }
    PIT_TRY(upload_factors(p->M, rc, p->coarse_inv64, p->coarse_inv32, p->stream));
    // mixed path: the coarse step (I - dTc nu D2)^{-c} is diagonal in the sine
    // basis (eigenvalues mu_k = -4/h^2 sin^2(k pi h / 2), k = 1..M), so the
    // FP32 sweep runs as two sine transforms on the tensor cores around a
    // per-mode recurrence over the slices (PIT_HEAT1D_TC=0 keeps the
    // sequential Thomas sweep)
    const char *env = getenv("PIT_HEAT1D_TC");
    p->xform_tc = (p->precision == PIT_MIXED && p->M >= 16 && !(env && env[0] == '0') &&
                   heat1d_tc_setup(p) == PIT_OK) ? 1 : 0;
    if (p->xform_tc) {
        const int Mp = heat1d_tc_padded(p->M);
        const double dtc = p->dT / p->coarse_steps;
        std::vector<double> g(Mp, 0.0);
        for (int k = 0; k < p->M; ++k) {
            const double sk = sin(M_PI * (k + 1) * h / 2.0);
            const double mu = -4.0 / (h * h) * sk * sk;
            g[k] = pow(1.0 - dtc * p->nu * mu, -(double)p->coarse_steps);
        }
        PIT_TRY(p->gmode.ensure(Mp * sizeof(double)));
        PIT_CUDA(cudaMemcpyAsync(p->gmode.ptr, g.data(), Mp * sizeof(double), cudaMemcpyHostToDevice,
                                 p->stream));
        PIT_CUDA(cudaStreamSynchronize(p->stream));
    }
    return PIT_OK;
}

pit_status heat1d_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                          const MemberState *st, cudaStream_t s) {
    Heat1dArgs a{x, y, p->y0.as<double>(), p->M, p->N, p->batch, p->blen, 1, mode,
                 p->fine_steps, st};
    return fine_launch(p, a, p->N, prec, s);
}

pit_status heat1d_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s) {
    // y (block n) = F(x (block n-1)) for every member: x and y point at
    // consecutive blocks of the same block vector.
    Heat1dArgs a{x, y - p->M, p->y0.as<double>(), p->M, p->N, p->batch, p->blen, 1, 2,
                 p->fine_steps, nullptr};
    return fine_launch(p, a, 1, prec, s);
}

pit_status heat1d_sweep(Problem *p, const double *q, double *z, int prec, const MemberState *st,
                        cudaStream_t s) {
    if (prec == PIT_FP64 && p->h1_pow_on) {
        const int M = p->M, N = p->N;
        const size_t npairs = (size_t)(N + 1) * (N + 2) / 2;
        PIT_TRY(p->h1_sweep_t.ensure((size_t)p->batch * npairs * M * sizeof(double)));
        const int nt = std::min(256, (M + 31) / 32 * 32);
        const int jb = h1_jb(M);
        const size_t sm = (size_t)(((M + 1) & ~1) + jb * M) * sizeof(double);
        PIT_TRY(smem_limit(k_heat1d_sweep_pow1, H1_SMEM_MAX));
        k_heat1d_sweep_pow1<<<dim3((unsigned)npairs, p->batch), nt, sm, s>>>(
            q, p->h1_sweep_t.as<double>(), p->h1_powT.as<double>(), M, N, p->blen, st, jb);
        PIT_LAUNCH_CHECK();
        k_heat1d_sweep_pow2<<<dim3((unsigned)(N + 1), p->batch), nt, 0, s>>>(p->h1_sweep_t.as<double>(), z, M, N,
                                                                             p->blen, st);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
    if (prec == PIT_FP64 && p->M <= WARP_MAXM && p->heat1d_small) {
        SweepWarpLaunch f{p, q, z, st, s};
        return dispatch_warp(p->M, f);
    }
    if (prec == PIT_FP64) {
        SweepLaunch<double> f{p, q, z, &p->coarse_inv64, st, s};
        return dispatch_1d(p->M, f);
    }
    if (p->xform_tc) {
        // q -> padded FP32 rows -> qhat = q S -> recurrence per mode -> z = (2/(M+1)) zhat S
        const int M = p->M, Mp = heat1d_tc_padded(M);
        const size_t R = (size_t)p->batch * (p->N + 1);
        const int nchunks = (p->N + 1 + 15) / 16;
        const size_t ends_bytes = (size_t)p->batch * nchunks * Mp * sizeof(double);
        PIT_TRY(p->hat.ensure(2 * R * Mp * sizeof(float) + ends_bytes));
        float *h1 = p->hat.as<float>(), *h2 = h1 + R * Mp;
        double *ends = reinterpret_cast<double *>(h2 + R * Mp);
        PIT_TRY(heat1d_tc_pack(p, q, h1, s));
        PIT_TRY(heat1d_tc_xform(p, h1, h2, false, Mp, Mp, 1.0, st, s));
        PIT_TRY(sine_mode_recurrence(p, h2, ends, Mp, st, s));
        return heat1d_tc_xform(p, h2, z, true, M, M, 2.0 / (M + 1), st, s);
    }
    SweepLaunch<float> f{p, q, z, &p->coarse_inv32, st, s};
    return dispatch_1d(p->M, f);
}

}  // namespace pit
