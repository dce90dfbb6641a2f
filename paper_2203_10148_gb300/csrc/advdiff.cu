// 2D advection-diffusion u_t = nu Lap u - v . grad u on the periodic unit
// square, n x n points x_i = i/n, h = 1/n: central 5-point diffusion,
// first-order upwind advection (backward difference where the velocity
// component is >= 0, forward where < 0).  With ax = vx/h, ay = vy/h and
// nu_d = nu/h^2:
//   L v = nu_d (vE + vW + vN + vS - 4 vC) - ax dX - ay dY,
//   dX = vC - vW (ax >= 0) or vE - vC,  dY = vC - vN (ay >= 0) or vS - vC,
// with N the row above (j - 1) and S the row below (j + 1).
//
// Fine batch (eq. (2), fused with the shift-subtract of eq. (4)): one
// thread-block cluster per slice.  The n/32 CTAs of a cluster each hold 32
// rows of the slice on chip for all RK4 steps (Horner form, as for the heat
// equation); a thread owns a 4 x 8 tile; west/east halos come from the
// neighbouring lanes by shuffle (across a warp boundary through a small
// shared column buffer), north/south halos through a shared row buffer,
// and the two rows at a CTA boundary from the neighbouring CTA's shared
// memory (DSMEM), periodic across the cluster.  One cluster barrier per RK4
// stage.
//
// Coarse sweep (eq. (7), right): G is one implicit-Euler step,
// (I - dT L) w = b.  L has variable coefficients and is not symmetric, so no
// transform diagonalises it; G is applied as a fixed linear operator: K
// (the coarse stepper's inner count, 48 by default) steps of the Chebyshev
// semi-iteration on the Jacobi-scaled system
// D^{-1} (I - dT L) w = D^{-1} b, started from w = b, for the eigenvalue
// interval [1 - rho, 1 + rho] with rho = max_p (D_p - 1) / D_p (the
// Gershgorin bound of the scaled system).  The coefficients depend on the
// problem only, so G is a fixed polynomial in D^{-1}(I - dT L): any fixed
// linear preconditioner leaves the solution of eq. (4) unchanged, and only
// the iteration count depends on it.  The sweep runs in one cooperative
// launch: each CTA owns a band of rows, and exchanges its edge rows with the
// two neighbouring bands through global memory as tagged words: every 8-byte
// word carries a 32-bit part of a value and the exchange's sequence number,
// so that a reader polls the data itself (bounded waits) and one L2 round
// trip delivers both the value and the news that it is there.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "pit_internal.h"
#include "stencil_arith.cuh"

namespace cg = cooperative_groups;

namespace pit {
namespace {

constexpr int AD_RY = 4, AD_RX = 8;          // thread tile
constexpr int AD_ROWS = 32;                  // rows per CTA (cluster size = n / 32)
constexpr int AD_TY = AD_ROWS / AD_RY;       // 8 thread rows per CTA

struct AdvArgs {
    const double *x;
    double *y;
    float *y32;
    const double *y0;
    const void *ax, *ay;   // per-point coefficients (float or double), row-major n x n
    int n, N, batch;
    size_t blen;
    int n_first, mode, steps;
    double c[4];           // stage coefficients dt/4, dt/3, dt/2, dt
    double nud;            // nu / h^2
    const MemberState *st;
};

__device__ __forceinline__ bool adv_runs(const MemberState *st, int b) {
    return st == nullptr || (st[b].active && !st[b].skip && !st[b].half);
}

template <class T>
__device__ __forceinline__ T adv_stage(T vn, T vs, T vw, T ve, T vc, T u, T cc, T nud, T ax,
                                       T ay) {
    const T lap = fma(T(-4), vc, (ve + vw) + (vn + vs));
    const T dX = (ax >= T(0)) ? (vc - vw) : (ve - vc);
    const T dY = (ay >= T(0)) ? (vc - vn) : (vs - vc);
    const T adv = fma(ay, dY, ax * dX);
    return fma(cc, fma(nud, lap, -adv), u);
}

// Float-float stage (the residual arithmetic, about 48 significant bits on
// the FP32 pipe): the sums of high parts are exact TwoSums, their errors and
// the low parts are summed in FP32, products keep their exact FMA error
// terms, one renormalisation at the end.  The upwind side follows the sign
// of the coefficient's high part (the sign of the FP64 coefficient).
template <>
__device__ __forceinline__ ff adv_stage<ff>(ff vn, ff vs, ff vw, ff ve, ff vc, ff u, ff cc,
                                            ff nud, ff ax, ff ay) {
    // Laplacian sum vE + vW + vN + vS - 4 vC
    const ff a = two_sum(ve.hi, vw.hi);
    const ff b = two_sum(vn.hi, vs.hi);
    const ff c = two_sum(a.hi, b.hi);
    const ff d = two_sum(c.hi, __fmul_rn(-4.f, vc.hi));
    const float lap_lo = fmaf(-4.f, vc.lo, ((a.lo + b.lo) + (c.lo + d.lo)) +
                                              ((ve.lo + vw.lo) + (vn.lo + vs.lo)));
    // upwind differences
    const ff x1 = ax.hi >= 0.f ? vc : ve, x2 = ax.hi >= 0.f ? vw : vc;
    const ff y1 = ay.hi >= 0.f ? vc : vs, y2 = ay.hi >= 0.f ? vn : vc;
    const ff dx = two_sum(x1.hi, -x2.hi);
    const float dx_lo = dx.lo + (x1.lo - x2.lo);
    const ff dy = two_sum(y1.hi, -y2.hi);
    const float dy_lo = dy.lo + (y1.lo - y2.lo);
    // nud lap - ax dX - ay dY, each product with its exact error term
    const float p1 = __fmul_rn(nud.hi, d.hi);
    float e1 = fmaf(nud.hi, d.hi, -p1);
    e1 = fmaf(nud.hi, lap_lo, e1);
    e1 = fmaf(nud.lo, d.hi, e1);
    const float p2 = __fmul_rn(ax.hi, dx.hi);
    float e2 = fmaf(ax.hi, dx.hi, -p2);
    e2 = fmaf(ax.hi, dx_lo, e2);
    e2 = fmaf(ax.lo, dx.hi, e2);
    const float p3 = __fmul_rn(ay.hi, dy.hi);
    float e3 = fmaf(ay.hi, dy.hi, -p3);
    e3 = fmaf(ay.hi, dy_lo, e3);
    e3 = fmaf(ay.lo, dy.hi, e3);
    const ff s1 = two_sum(p1, -p2);
    const ff s2 = two_sum(s1.hi, -p3);
    const float l_lo = (s1.lo + s2.lo) + ((e1 - e2) - e3);
    // u + cc L
    const float p = __fmul_rn(cc.hi, s2.hi);
    float e = fmaf(cc.hi, s2.hi, -p);
    e = fmaf(cc.hi, l_lo, e);
    e = fmaf(cc.lo, s2.hi, e);
    const ff t = two_sum(u.hi, p);
    return fast_two_sum(t.hi, t.lo + (u.lo + e));
}

// The same stage for coefficients that are FP32 values (low parts zero):
// the low-part terms of the two coefficient products vanish (90 operations).
__device__ __forceinline__ ff adv_stage_c32(ff vn, ff vs, ff vw, ff ve, ff vc, ff u, ff cc, ff nud,
                                            float ax, float ay) {
    const ff a = two_sum(ve.hi, vw.hi);
    const ff b = two_sum(vn.hi, vs.hi);
    const ff c = two_sum(a.hi, b.hi);
    const ff d = two_sum(c.hi, __fmul_rn(-4.f, vc.hi));
    const float lap_lo = fmaf(-4.f, vc.lo, ((a.lo + b.lo) + (c.lo + d.lo)) +
                                              ((ve.lo + vw.lo) + (vn.lo + vs.lo)));
    const ff x1 = ax >= 0.f ? vc : ve, x2 = ax >= 0.f ? vw : vc;
    const ff y1 = ay >= 0.f ? vc : vs, y2 = ay >= 0.f ? vn : vc;
    const ff dx = two_sum(x1.hi, -x2.hi);
    const float dx_lo = dx.lo + (x1.lo - x2.lo);
    const ff dy = two_sum(y1.hi, -y2.hi);
    const float dy_lo = dy.lo + (y1.lo - y2.lo);
    const float p1 = __fmul_rn(nud.hi, d.hi);
    float e1 = fmaf(nud.hi, d.hi, -p1);
    e1 = fmaf(nud.hi, lap_lo, e1);
    e1 = fmaf(nud.lo, d.hi, e1);
    const float p2 = __fmul_rn(ax, dx.hi);
    float e2 = fmaf(ax, dx.hi, -p2);
    e2 = fmaf(ax, dx_lo, e2);
    const float p3 = __fmul_rn(ay, dy.hi);
    float e3 = fmaf(ay, dy.hi, -p3);
    e3 = fmaf(ay, dy_lo, e3);
    const ff s1 = two_sum(p1, -p2);
    const ff s2 = two_sum(s1.hi, -p3);
    const float l_lo = (s1.lo + s2.lo) + ((e1 - e2) - e3);
    const float p = __fmul_rn(cc.hi, s2.hi);
    float e = fmaf(cc.hi, s2.hi, -p);
    e = fmaf(cc.hi, l_lo, e);
    e = fmaf(cc.lo, s2.hi, e);
    const ff t = two_sum(u.hi, p);
    return fast_two_sum(t.hi, t.lo + (u.lo + e));
}

template <class T>
__device__ __forceinline__ T adv_zero() { return T(0); }
template <>
__device__ __forceinline__ ff adv_zero<ff>() { return ff{0.f, 0.f}; }

template <class T>
__device__ __forceinline__ T adv_from_d(double x) { return (T)x; }
template <>
__device__ __forceinline__ float adv_from_d<float>(double x) { return d2f_rn(x); }
template <>
__device__ __forceinline__ ff adv_from_d<ff>(double x) { return ff_from_double(x); }

__device__ __forceinline__ double adv_to_d(float v) { return f2d(v); }
__device__ __forceinline__ double adv_to_d(double v) { return v; }
__device__ __forceinline__ double adv_to_d(ff v) { return f2d(v.hi) + f2d(v.lo); }

template <class T>
__device__ __forceinline__ T shfl_idx(T v, int src) { return __shfl_sync(kFullMask, v, src); }
template <class T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(kFullMask, v, 1); }
template <class T>
__device__ __forceinline__ T shfl_down1(T v) { return __shfl_down_sync(kFullMask, v, 1); }
template <>
__device__ __forceinline__ ff shfl_idx<ff>(ff v, int src) {
    return ff{__shfl_sync(kFullMask, v.hi, src), __shfl_sync(kFullMask, v.lo, src)};
}
template <>
__device__ __forceinline__ ff shfl_up1<ff>(ff v) {
    return ff{__shfl_up_sync(kFullMask, v.hi, 1), __shfl_up_sync(kFullMask, v.lo, 1)};
}
template <>
__device__ __forceinline__ ff shfl_down1<ff>(ff v) {
    return ff{__shfl_down_sync(kFullMask, v.hi, 1), __shfl_down_sync(kFullMask, v.lo, 1)};
}

// A thread's 8 consecutive values of a row buffer are stored as 16-byte
// chunks in chunk-major order: chunk q of thread column tx at element
// q * TX * CW + tx * CW (CW values per 16 bytes), so that a warp's 16-byte
// accesses to one chunk are contiguous (no shared-memory bank conflicts).
template <class T>
struct RowChunks;
template <>
struct RowChunks<float> {
    __device__ static void store(float *row, int tx, int TX, const float (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
            *reinterpret_cast<float4 *>(row + (size_t)q * TX * 4 + (size_t)tx * 4) =
                make_float4(v[q * 4], v[q * 4 + 1], v[q * 4 + 2], v[q * 4 + 3]);
    }
    __device__ static void load(const float *row, int tx, int TX, float (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float4 t = *reinterpret_cast<const float4 *>(row + (size_t)q * TX * 4 + (size_t)tx * 4);
            v[q * 4] = t.x;
            v[q * 4 + 1] = t.y;
            v[q * 4 + 2] = t.z;
            v[q * 4 + 3] = t.w;
        }
    }
};
template <>
struct RowChunks<double> {
    __device__ static void store(double *row, int tx, int TX, const double (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<double2 *>(row + (size_t)q * TX * 2 + (size_t)tx * 2) =
                make_double2(v[q * 2], v[q * 2 + 1]);
    }
    __device__ static void load(const double *row, int tx, int TX, double (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 t = *reinterpret_cast<const double2 *>(row + (size_t)q * TX * 2 + (size_t)tx * 2);
            v[q * 2] = t.x;
            v[q * 2 + 1] = t.y;
        }
    }
};
template <>
struct RowChunks<ff> {
    __device__ static void store(ff *row, int tx, int TX, const ff (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4 *>(row + (size_t)q * TX * 2 + (size_t)tx * 2) =
                make_float4(v[q * 2].hi, v[q * 2].lo, v[q * 2 + 1].hi, v[q * 2 + 1].lo);
    }
    __device__ static void load(const ff *row, int tx, int TX, ff (&v)[AD_RX]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = *reinterpret_cast<const float4 *>(row + (size_t)q * TX * 2 + (size_t)tx * 2);
            v[q * 2] = ff{t.x, t.y};
            v[q * 2 + 1] = ff{t.z, t.w};
        }
    }
};

// One cluster of CS = n/32 CTAs per (slice, member).  Threads: TX * 8 with
// TX = n/8 thread columns (n <= 512).  T = float (state in registers,
// coefficients in shared memory), double or float-float (state in shared
// memory, coefficients read through L1; float-float coefficients are
// (hi, lo) float pairs).
template <class T, bool DBUF, bool C32 = false>
__global__ void __launch_bounds__(512, 1) k_advdiff_fine(AdvArgs a) {
    constexpr bool FP32 = std::is_same<T, float>::value;
    constexpr bool FF = std::is_same<T, ff>::value;
    constexpr int NB = DBUF ? 2 : 1;               // row-buffer copies
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int n = a.n;
    const int CS = n / AD_ROWS;
    const int rank = (int)cluster.block_rank();
    const int slice_lin = blockIdx.x / CS;          // cluster index = (member, slice)
    const int b = slice_lin / a.N;
    const int slice = a.n_first + slice_lin % a.N;  // output block
    // inactive member: the whole cluster leaves before any cluster barrier
    if (!adv_runs(a.st, b)) return;
    const bool active = true;
    const int TX = n / AD_RX;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int lane = tid & 31, warp_in_row = tx / 32;
    const int i0 = tx * AD_RX;
    const int jl0 = ty * AD_RY;                      // local row
    const int j0 = rank * AD_ROWS + jl0;             // global row
    // shared memory: [cc 4][rowbuf NB x 2 x TY x n][colbuf NB x TY x 4 x RY][u or coefficients]
    T *ccs = reinterpret_cast<T *>(smem_raw);
    T *rowbuf = reinterpret_cast<T *>(smem_raw + 32);
    T *colbuf = rowbuf + (size_t)NB * 2 * AD_TY * n;
    T *tail = colbuf + NB * AD_TY * 4 * AD_RY;
    if (tid < 4) ccs[tid] = adv_from_d<T>(tid == 0 ? a.c[0] : tid == 1 ? a.c[1] : tid == 2 ? a.c[2] : a.c[3]);
    const size_t mb = (size_t)b * a.blen;
    const size_t nn = (size_t)n * n;
    const double *xin = a.x + mb + (size_t)(slice - 1) * nn;

    T v[AD_RY][AD_RX];
    T ur[FP32 ? AD_RY : 1][FP32 ? AD_RX : 1];
    T *us = tail;                                    // double: u thread-private
    T *cax = tail, *cay = tail + (size_t)AD_RY * AD_RX * nthr;   // float: coefficients
    const T *gax = reinterpret_cast<const T *>(a.ax);
    const T *gay = reinterpret_cast<const T *>(a.ay);
    [[maybe_unused]] const float2 *gax2 = reinterpret_cast<const float2 *>(a.ax);
    [[maybe_unused]] const float2 *gay2 = reinterpret_cast<const float2 *>(a.ay);
#pragma unroll
    for (int r = 0; r < AD_RY; ++r)
#pragma unroll
        for (int c = 0; c < AD_RX; ++c) {
            const size_t k = (size_t)(j0 + r) * n + (i0 + c);
            const int slot = (r * AD_RX + c) * nthr + tid;
            T val = adv_zero<T>();
            if (active) val = adv_from_d<T>(xin[k]);
            v[r][c] = val;
            if constexpr (FP32) {
                ur[FP32 ? r : 0][FP32 ? c : 0] = val;
                cax[slot] = gax[k];
                cay[slot] = gay[k];
            } else {
                us[slot] = val;
            }
        }
    const T nud = adv_from_d<T>(a.nud);
    int buf = 0;
    const int up_rank = (rank + CS - 1) % CS, down_rank = (rank + 1) % CS;
    for (int s = 0; s < a.steps; ++s) {
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
            // single buffer: every read of the previous stage's rows is done first
            if (!DBUF) cluster.sync();
            // publish top / bottom rows and the warp-edge columns
            RowChunks<T>::store(rowbuf + ((size_t)(buf * 2 + 0) * AD_TY + ty) * n, tx, TX, v[0]);
            RowChunks<T>::store(rowbuf + ((size_t)(buf * 2 + 1) * AD_TY + ty) * n, tx, TX, v[AD_RY - 1]);
            if (lane == 0 || lane == 31) {
                // colbuf[buf][ty][slot][r]: slot 0/1 = west column of warp 0/1,
                // slot 2/3 = east column of warp 0/1
                T *cb = colbuf + ((size_t)(buf * AD_TY + ty) * 4 + (lane == 0 ? 0 : 2) + warp_in_row) * AD_RY;
#pragma unroll
                for (int r = 0; r < AD_RY; ++r) cb[r] = (lane == 0) ? v[r][0] : v[r][AD_RX - 1];
            }
            cluster.sync();
            const T cc = ccs[stage];
            // north / south rows: from the thread row above / below, across the
            // CTA edge from the neighbouring CTA's shared memory (periodic)
            T prev[AD_RX];
            {
                const T *src = (ty > 0) ? rowbuf + ((size_t)(buf * 2 + 1) * AD_TY + (ty - 1)) * n
                                        : cluster.map_shared_rank(rowbuf, up_rank) +
                                              ((size_t)(buf * 2 + 1) * AD_TY + (AD_TY - 1)) * n;
                RowChunks<T>::load(src, tx, TX, prev);
            }
            // west/east neighbours of the tile's first/last column (periodic in x)
            const int row_base = (tid / 32) * 32;   // lanes of this warp
            const bool row_in_warp = TX <= 32;
#pragma unroll
            for (int r = 0; r < AD_RY; ++r) {
                T w_in, e_in;
                if (row_in_warp) {
                    // the thread row lies in one warp: lanes tx-1 / tx+1 modulo TX
                    const int seg = (lane / TX) * TX;
                    w_in = shfl_idx(v[r][AD_RX - 1], seg + (tx + TX - 1) % TX);
                    e_in = shfl_idx(v[r][0], seg + (tx + 1) % TX);
                } else {
                    // two warps per thread row: the edge lanes read the other warp's column
                    w_in = shfl_up1(v[r][AD_RX - 1]);
                    e_in = shfl_down1(v[r][0]);
                    const int other = 1 - warp_in_row;
                    if (lane == 0)
                        w_in = colbuf[((size_t)(buf * AD_TY + ty) * 4 + 2 + other) * AD_RY + r];
                    if (lane == 31)
                        e_in = colbuf[((size_t)(buf * AD_TY + ty) * 4 + 0 + other) * AD_RY + r];
                }
                (void)row_base;
                T cur[AD_RX];
#pragma unroll
                for (int c = 0; c < AD_RX; ++c) cur[c] = v[r][c];
                T srow[AD_RX];
                if (r == AD_RY - 1) {
                    const T *srs = (ty < AD_TY - 1) ? rowbuf + ((size_t)(buf * 2 + 0) * AD_TY + (ty + 1)) * n
                                                    : cluster.map_shared_rank(rowbuf, down_rank) +
                                                          ((size_t)(buf * 2 + 0) * AD_TY + 0) * n;
                    RowChunks<T>::load(srs, tx, TX, srow);
                }
#pragma unroll
                for (int c = 0; c < AD_RX; ++c) {
                    const T vn = prev[c];
                    const T vs = (r < AD_RY - 1) ? v[r + 1][c] : srow[c];
                    const T vw = (c > 0) ? cur[c - 1] : w_in;
                    const T ve = (c < AD_RX - 1) ? cur[c + 1] : e_in;
                    const int slot = (r * AD_RX + c) * nthr + tid;
                    T u, ax, ay;
                    if constexpr (FP32) {
                        u = ur[FP32 ? r : 0][FP32 ? c : 0];
                        ax = cax[slot];
                        ay = cay[slot];
                    } else if constexpr (FF) {
                        u = us[slot];
                        const size_t k = (size_t)(j0 + r) * n + (i0 + c);
                        if constexpr (C32) {
                            // FP32 coefficients: the low parts are zero
                            const float* fx = reinterpret_cast<const float *>(a.ax);
                            const float* fy = reinterpret_cast<const float *>(a.ay);
                            v[r][c] = adv_stage_c32(vn, vs, vw, ve, cur[c], u, cc, nud, __ldg(fx + k),
                                                    __ldg(fy + k));
                            continue;
                        }
                        const float2 cx = __ldg(gax2 + k), cy = __ldg(gay2 + k);
                        ax = ff{cx.x, cx.y};
                        ay = ff{cy.x, cy.y};
                    } else {
                        u = us[slot];
                        const size_t k = (size_t)(j0 + r) * n + (i0 + c);
                        ax = __ldg(gax + k);
                        ay = __ldg(gay + k);
                    }
                    v[r][c] = adv_stage(vn, vs, vw, ve, cur[c], u, cc, nud, ax, ay);
                }
#pragma unroll
                for (int c = 0; c < AD_RX; ++c) prev[c] = cur[c];
            }
            if (DBUF) buf ^= 1;
        }
#pragma unroll
        for (int r = 0; r < AD_RY; ++r)
#pragma unroll
            for (int c = 0; c < AD_RX; ++c) {
                if constexpr (FP32) ur[FP32 ? r : 0][FP32 ? c : 0] = v[r][c];
                else us[(r * AD_RX + c) * nthr + tid] = v[r][c];
            }
    }
    // all remote reads of this CTA's row buffer are done before anyone exits
    cluster.sync();
    const double *xn = a.x + mb + (size_t)slice * nn;
#pragma unroll
    for (int r = 0; r < AD_RY; ++r)
#pragma unroll
        for (int c = 0; c < AD_RX; ++c) {
            const size_t k = (size_t)(j0 + r) * n + (i0 + c);
            if constexpr (FP32) {
                if (a.y32) {
                    a.y32[mb + (size_t)slice * nn + k] = d2f_rn(xn[k]) - v[r][c];
                    continue;
                }
            }
            const double f = adv_to_d(v[r][c]);
            double *yo = a.y + mb + (size_t)slice * nn;
            if (a.mode == FINE_APPLY) yo[k] = xn[k] - f;
            else if (a.mode == FINE_RESIDUAL) yo[k] = f - xn[k];
            else yo[k] = f;
        }
    if (slice == 1 && a.mode != 2) {
        // row 0 of eq. (4) for this CTA's rows
        const double *x0 = a.x + mb;
        const size_t k0 = (size_t)rank * AD_ROWS * n, k1 = k0 + (size_t)AD_ROWS * n;
        for (size_t k = k0 + tid; k < k1; k += nthr) {
            if constexpr (FP32) {
                if (a.y32) {
                    a.y32[mb + k] = d2f_rn(x0[k]);
                    continue;
                }
            }
            a.y[mb + k] = (a.mode == FINE_APPLY) ? x0[k] : a.y0[(size_t)b * nn + k] - x0[k];
        }
    }
}

// x = hi + lo with hi = RN32(x), lo = RN32(x - hi)
__global__ void k_split_ff(const double *__restrict__ x, float2 *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float hi = __double2float_rn(x[i]);
        out[i] = make_float2(hi, __double2float_rn(x[i] - (double)hi));
    }
}

template <class T, bool DBUF>
size_t adv_smem(int n) {
    const size_t nthr = (size_t)n;   // TX * 8 = n
    const size_t nb = DBUF ? 2 : 1;
    size_t s = 32 + (nb * 2 * AD_TY * (size_t)n + nb * AD_TY * 4 * AD_RY) * sizeof(T);
    if (std::is_same<T, float>::value) s += 2 * (size_t)AD_RY * AD_RX * nthr * sizeof(T);
    else s += (size_t)AD_RY * AD_RX * nthr * sizeof(T);
    return s;
}

// coefficient arrays: prec = PIT_MIXED (float), PIT_FP64 (double) or PIT_FF
// ((hi, lo) float pairs)
AdvArgs adv_args(Problem *p, const double *x, double *y, float *y32, int mode,
                 const MemberState *st, int prec) {
    AdvArgs a{};
    a.x = x;
    a.y = y;
    a.y32 = y32;
    a.y0 = p->y0.as<double>();
    a.ax = prec == PIT_MIXED ? p->vx32.ptr : prec == PIT_FF ? p->vxff.ptr : p->vx64.ptr;
    a.ay = prec == PIT_MIXED ? p->vy32.ptr : prec == PIT_FF ? p->vyff.ptr : p->vy64.ptr;
    a.n = p->nx;
    a.N = p->N;
    a.batch = p->batch;
    a.blen = p->blen;
    a.n_first = 1;
    a.mode = mode;
    a.steps = p->fine_steps;
    const double dt = p->dT / p->fine_steps;
    a.c[0] = dt / 4.0;
    a.c[1] = dt / 3.0;
    a.c[2] = dt / 2.0;
    a.c[3] = dt;
    const double h = 1.0 / p->nx;
    a.nud = p->nu / (h * h);
    a.st = st;
    return a;
}

template <class T, bool DBUF, bool C32 = false>
pit_status launch_adv_fine_v(Problem *p, AdvArgs a, int nslices, cudaStream_t s) {
    const int n = p->nx;
    const int CS = n / AD_ROWS;
    const size_t sm = adv_smem<T, DBUF>(n);
    auto kern = k_advdiff_fine<T, DBUF, C32>;
    PIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (CS > 8)
        PIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    a.N = nslices;   // slices in this launch (output blocks n_first .. n_first + nslices - 1)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CS * nslices * p->batch), 1, 1);
    cfg.blockDim = dim3((unsigned)n, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PIT_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

constexpr size_t kSmemLimit = 227 * 1024;

// double-buffered row exchange when it fits, single-buffered otherwise;
// float-float with FP32 coefficients reads them as FP32 values
template <class T>
pit_status launch_adv_fine(Problem *p, AdvArgs a, int nslices, cudaStream_t s) {
    if constexpr (std::is_same<T, ff>::value) {
        if (p->adv_coef32) {
            a.ax = p->vx32.ptr;
            a.ay = p->vy32.ptr;
            if (adv_smem<T, true>(p->nx) <= kSmemLimit) return launch_adv_fine_v<T, true, true>(p, a, nslices, s);
            if (adv_smem<T, false>(p->nx) <= kSmemLimit) return launch_adv_fine_v<T, false, true>(p, a, nslices, s);
        }
    }
    if (adv_smem<T, true>(p->nx) <= kSmemLimit) return launch_adv_fine_v<T, true>(p, a, nslices, s);
    if (adv_smem<T, false>(p->nx) <= kSmemLimit) return launch_adv_fine_v<T, false>(p, a, nslices, s);
    set_error("advdiff2d: the slice does not fit the cluster's shared memory");
    return PIT_E_UNSUPPORTED;
}

// ------------------------------------------------------------------ sweep
constexpr int SWA_THREADS = 512;               // 16 warps per SM: the steps' short chains interleave
constexpr int SWA_PPT = 4;                     // points per thread: bands of <= 2048 points
constexpr int SWA_KMAX = 64;     // Chebyshev steps per coarse solve, at most

template <class T>
struct AdSweepArgs {
    const double *q;
    double *z;
    int n, N, batch, K, R;     // grid, slices, members, Chebyshev steps, rows per CTA
    long long spin;            // polls of a neighbour's flag before PIT_E_TIMEOUT
    size_t blen;
    double dT, nud;
    double inv_theta;          // first direction d_0 = D^{-1} r_0 / theta
    double c1[SWA_KMAX], c2[SWA_KMAX];   // d_{k+1} = c1_k d_k + c2_k D^{-1} r_{k+1}
    const T *ax, *ay;
    unsigned long long *halo;  // [2 parity][G][2 top/bottom][n][W] tagged words, W = sizeof(T)/4
    int *err;
    const MemberState *st;
};

// (A w)_p = w_p - dT (L w)_p on this CTA's band; wb holds the band with one
// halo row above (row 0) and below (row R+1).
template <class T>
__device__ __forceinline__ T apply_A(const T *wb, int n, int rl, int i, T ax, T ay, T dT, T nud) {
    const T *row = wb + (size_t)(rl + 1) * n;
    const T vc = row[i];
    const T vw = row[i == 0 ? n - 1 : i - 1], ve = row[i == n - 1 ? 0 : i + 1];
    const T vn = wb[(size_t)rl * n + i], vs = wb[(size_t)(rl + 2) * n + i];
    const T lap = fma(T(-4), vc, (ve + vw) + (vn + vs));
    const T dX = (ax >= T(0)) ? (vc - vw) : (ve - vc);
    const T dY = (ay >= T(0)) ? (vc - vn) : (vs - vc);
    const T Lw = fma(nud, lap, -fma(ay, dY, ax * dX));
    return fma(-dT, Lw, vc);
}

// A 32-bit part of a halo value with its exchange's sequence number in the
// other half of one 8-byte word: a single-copy-atomic store and load at GPU
// scope, so a reader that sees the number also sees the value.
__device__ __forceinline__ void st_tagged(unsigned long long *p, unsigned v, unsigned tag) {
    const unsigned long long w = ((unsigned long long)tag << 32) | v;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long *p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

template <class T> struct Words;
template <> struct Words<float> {
    static constexpr int W = 1;
    __device__ static void split(float v, unsigned (&u)[1]) { u[0] = __float_as_uint(v); }
    __device__ static float join(const unsigned (&u)[1]) { return __uint_as_float(u[0]); }
};
template <> struct Words<double> {
    static constexpr int W = 2;
    __device__ static void split(double v, unsigned (&u)[2]) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        u[0] = (unsigned)b;
        u[1] = (unsigned)(b >> 32);
    }
    __device__ static double join(const unsigned (&u)[2]) {
        return __longlong_as_double((long long)(((unsigned long long)u[1] << 32) | u[0]));
    }
};

// Puts this thread's points of a vector into the band buffer and the band's
// edge rows, tagged with the exchange number, into the band's global halo
// slot; then reads the neighbouring bands' edge rows of the same exchange
// into the halo rows of the band buffer, each word polled until it carries
// the exchange number (bounded: PIT_E_TIMEOUT after a.spin polls, or at once
// when another CTA reported an error), and synchronises the CTA.  The slots
// alternate by the exchange number's parity: a band rewrites a slot only two
// exchanges later, after both neighbours have published the exchange in
// between, which they can only do after reading this one.
template <class T>
__device__ bool exchange(const AdSweepArgs<T> &a, T *wb, const T (&val)[SWA_PPT], unsigned &step,
                         int g, int G, int up, int down, int *ok) {
    using Wd = Words<T>;
    constexpr int W = Wd::W;
    const int n = a.n, band = a.R * n;
    const unsigned tag = step + 1;
    unsigned long long *hslot = a.halo + ((size_t)((step & 1u) * G + g) * 2) * n * W;
#pragma unroll
    for (int e = 0; e < SWA_PPT; ++e) {
        const int p = threadIdx.x + e * SWA_THREADS;
        if (p < band) {
            wb[n + p] = val[e];
            unsigned u[W];
            Wd::split(val[e], u);
            if (p < n) {
#pragma unroll
                for (int w = 0; w < W; ++w) st_tagged(hslot + (size_t)p * W + w, u[w], tag);
            }
            if (p >= band - n) {
                const size_t q = (size_t)n + (p - (band - n));
#pragma unroll
                for (int w = 0; w < W; ++w) st_tagged(hslot + q * W + w, u[w], tag);
            }
        }
    }
    const unsigned long long *hu = a.halo + ((size_t)((step & 1u) * G + up) * 2) * n * W;
    const unsigned long long *hd = a.halo + ((size_t)((step & 1u) * G + down) * 2) * n * W;
    // this thread's halo words: columns i = tid + k * SWA_THREADS (n <= 512), the
    // row above (the upper band's bottom row) and below (the lower band's top
    // row); all loads issued first, then the late ones polled again
    constexpr int KI = 512 / SWA_THREADS;
    const unsigned long long *src[KI][2];
    unsigned long long x[KI][2][W];
#pragma unroll
    for (int k = 0; k < KI; ++k) {
        const int i = threadIdx.x + k * SWA_THREADS;
        src[k][0] = hu + ((size_t)n + (i < n ? i : 0)) * W;
        src[k][1] = hd + (size_t)(i < n ? i : 0) * W;
#pragma unroll
        for (int sd = 0; sd < 2; ++sd)
#pragma unroll
            for (int w = 0; w < W; ++w) x[k][sd][w] = (i < n) ? ld_tagged(src[k][sd] + w) : 0ull;
    }
    bool good = true;
    long long spins = 0;
    for (;;) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            if (threadIdx.x + k * SWA_THREADS >= n) continue;
#pragma unroll
            for (int sd = 0; sd < 2; ++sd)
#pragma unroll
                for (int w = 0; w < W; ++w)
                    if ((unsigned)(x[k][sd][w] >> 32) != tag) {
                        all = false;
                        x[k][sd][w] = ld_tagged(src[k][sd] + w);
                    }
        }
        if (all) break;
        if (++spins > a.spin || ((spins & 255) == 0 && *(volatile int *)a.err)) {
            atomicExch(a.err, PIT_E_TIMEOUT);
            good = false;
            break;
        }
    }
    if (good) {
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            const int i = threadIdx.x + k * SWA_THREADS;
            if (i >= n) continue;
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                unsigned u[W];
#pragma unroll
                for (int w = 0; w < W; ++w) u[w] = (unsigned)x[k][sd][w];
                wb[sd == 0 ? (size_t)i : (size_t)(a.R + 1) * n + i] = Wd::join(u);
            }
        }
    } else {
        *ok = 0;
    }
    __syncthreads();
    if (!*ok) return false;
    ++step;
    return true;
}

// z_0 = q_0, z_n = q_n + G z_{n-1}, G b ~ (I - dT L)^{-1} b by K Chebyshev
// steps on the Jacobi-scaled system from x = b (fixed coefficients, so G is
// a fixed polynomial in D^{-1} A).
template <class T>
__global__ void __launch_bounds__(SWA_THREADS, 1) k_advdiff_sweep(AdSweepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *wb = reinterpret_cast<T *>(smem_raw);          // (R + 2) x n band with halos
    __shared__ int ok;
    const int g = blockIdx.x, G = gridDim.x;
    const int up = (g + G - 1) % G, down = (g + 1) % G;
    const int n = a.n, R = a.R;
    const int band = R * n;
    const int r0 = g * R;
    const T dT = (T)a.dT, nud = (T)a.nud;
    T bv[SWA_PPT], x[SWA_PPT], r[SWA_PPT], d[SWA_PPT], Dinv[SWA_PPT], axv[SWA_PPT], ayv[SWA_PPT];
    int rlv[SWA_PPT], iv[SWA_PPT];
#pragma unroll
    for (int e = 0; e < SWA_PPT; ++e) {
        const int p = min(threadIdx.x + e * SWA_THREADS, band - 1);
        rlv[e] = p / n;
        iv[e] = p % n;
        const size_t k = (size_t)(r0 + rlv[e]) * n + iv[e];
        axv[e] = a.ax[k];
        ayv[e] = a.ay[k];
        Dinv[e] = T(1) / fma(dT, fma(T(4), nud, fabs(axv[e]) + fabs(ayv[e])), T(1));
    }
    unsigned step = 0;
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int mbr = 0; mbr < a.batch; ++mbr) {
        if (!(a.st == nullptr || (a.st[mbr].active && !a.st[mbr].skip && !a.st[mbr].half))) continue;
        const size_t mb = (size_t)mbr * a.blen;
#pragma unroll
        for (int e = 0; e < SWA_PPT; ++e) {
            const int p = threadIdx.x + e * SWA_THREADS;
            if (p < band) {
                const size_t k = mb + (size_t)r0 * n + p;
                const double q0 = a.q[k];
                a.z[k] = q0;
                bv[e] = (T)q0;
            }
        }
        for (int sl = 1; sl <= a.N; ++sl) {
            // x = b; r = b - A b; d = D^{-1} r / theta
            if (!exchange(a, wb, bv, step, g, G, up, down, &ok)) return;
#pragma unroll
            for (int e = 0; e < SWA_PPT; ++e) {
                x[e] = bv[e];
                r[e] = bv[e] - apply_A(wb, n, rlv[e], iv[e], axv[e], ayv[e], dT, nud);
                d[e] = (T)a.inv_theta * Dinv[e] * r[e];
            }
            for (int k = 0; k < a.K; ++k) {
#pragma unroll
                for (int e = 0; e < SWA_PPT; ++e) x[e] += d[e];
                if (k == a.K - 1) break;
                __syncthreads();                      // band buffer reused for d
                if (!exchange(a, wb, d, step, g, G, up, down, &ok)) return;
                const T c1 = (T)a.c1[k], c2 = (T)a.c2[k];
#pragma unroll
                for (int e = 0; e < SWA_PPT; ++e) {
                    r[e] -= apply_A(wb, n, rlv[e], iv[e], axv[e], ayv[e], dT, nud);
                    d[e] = fma(c1, d[e], c2 * Dinv[e] * r[e]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < SWA_PPT; ++e) {
                const int p = threadIdx.x + e * SWA_THREADS;
                if (p < band) {
                    const size_t k = mb + (size_t)sl * n * n + (size_t)r0 * n + p;
                    const double zz = a.q[k] + (double)x[e];
                    a.z[k] = zz;
                    bv[e] = (T)zz;
                }
            }
        }
    }
}

template <class T>
pit_status launch_adv_sweep(Problem *p, const double *q, double *z, const T *ax, const T *ay,
                            const MemberState *st, cudaStream_t s) {
    const int n = p->nx;
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // bands of R rows with R * n <= SWA_PPT * SWA_THREADS, as many bands as fit
    int R = 1;
    while (R * n < n * n && (n / R) > sms) R *= 2;
    if (R * n > SWA_PPT * SWA_THREADS || n % R != 0 || n / R > sms) {
        set_error("advdiff sweep: grid does not fit the band decomposition");
        return PIT_E_UNSUPPORTED;
    }
    const int G = n / R;
    auto kern = k_advdiff_sweep<T>;
    const size_t smem = (size_t)(R + 2) * n * sizeof(T);
    PIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PIT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SWA_THREADS, smem));
    if (per_sm * sms < G) {
        set_error("advdiff sweep: bands cannot all be resident");
        return PIT_E_UNSUPPORTED;
    }
    // tagged halo words; zero tags never match an exchange number (they start at 1)
    const size_t hbytes = (size_t)2 * G * 2 * n * (sizeof(T) / 4) * sizeof(unsigned long long);
    PIT_TRY(p->adv_scratch.ensure(hbytes + 256));
    unsigned long long *halo = p->adv_scratch.as<unsigned long long>();
    PIT_CUDA(cudaMemsetAsync(halo, 0, hbytes, s));
    AdSweepArgs<T> a{};
    a.q = q;
    a.z = z;
    a.n = n;
    a.N = p->N;
    a.batch = p->batch;
    a.K = p->adv_K;
    a.spin = p->adv_spin;
    a.R = R;
    a.blen = p->blen;
    a.dT = p->dT / p->coarse_steps;
    a.nud = p->nu * n * (double)n;
    a.inv_theta = p->adv_inv_theta;
    for (int k = 0; k < SWA_KMAX; ++k) {
        a.c1[k] = p->adv_c1[k];
        a.c2[k] = p->adv_c2[k];
    }
    a.ax = ax;
    a.ay = ay;
    a.halo = halo;
    a.err = p->errword.as<int>();
    a.st = st;
    void *args[] = {&a};
    PIT_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(SWA_THREADS), args, smem, s));
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

__global__ void k_scale_coeff(const double *v, double *o64, float *o32, double scale, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double x = v[i] * scale;
        o64[i] = x;
        o32[i] = d2f_rn(x);
    }
}

}  // namespace

pit_status advdiff_setup(Problem *p) {
    if (p->nx != p->ny) {
        set_error("advdiff2d: only square grids are supported");
        return PIT_E_UNSUPPORTED;
    }
    const int n = p->nx;
    if (!(n == 32 || n == 64 || n == 128 || n == 256 || n == 512)) {
        set_error("advdiff2d: n must be 32, 64, 128, 256 or 512");
        return PIT_E_UNSUPPORTED;
    }
    if (p->fine_kind != PIT_STEP_RK4 || p->coarse_kind != PIT_STEP_IE || p->coarse_steps != 1) {
        set_error("advdiff2d: fine must be RK4 and coarse one implicit-Euler step");
        return PIT_E_UNSUPPORTED;
    }
    // coefficients ax = vx / h, ay = vy / h (FP64 in place, FP32 copies)
    const size_t M = p->M;
    PIT_TRY(p->vx32.ensure(M * sizeof(float)));
    PIT_TRY(p->vy32.ensure(M * sizeof(float)));
    k_scale_coeff<<<256, 256, 0, p->stream>>>(p->vx64.as<double>(), p->vx64.as<double>(),
                                              p->vx32.as<float>(), (double)n, M);
    PIT_LAUNCH_CHECK();
    k_scale_coeff<<<256, 256, 0, p->stream>>>(p->vy64.as<double>(), p->vy64.as<double>(),
                                              p->vy32.as<float>(), (double)n, M);
    PIT_LAUNCH_CHECK();
    // float-float copies (hi, lo) for the residual arithmetic
    PIT_TRY(p->vxff.ensure(M * sizeof(float2)));
    PIT_TRY(p->vyff.ensure(M * sizeof(float2)));
    k_split_ff<<<256, 256, 0, p->stream>>>(p->vx64.as<double>(), p->vxff.as<float2>(), M);
    PIT_LAUNCH_CHECK();
    k_split_ff<<<256, 256, 0, p->stream>>>(p->vy64.as<double>(), p->vyff.as<float2>(), M);
    PIT_LAUNCH_CHECK();
    // Chebyshev coefficients on the Jacobi-scaled IE system: the spectrum of
    // D^{-1} A lies in the Gershgorin disc |z - 1| <= rho, rho = max (D - 1)/D,
    // taken as the real interval [1 - rho, 1 + rho]
    {
        std::vector<double> vx(M), vy(M);
        PIT_CUDA(cudaMemcpy(vx.data(), p->vx64.ptr, M * sizeof(double), cudaMemcpyDeviceToHost));
        PIT_CUDA(cudaMemcpy(vy.data(), p->vy64.ptr, M * sizeof(double), cudaMemcpyDeviceToHost));
        const double dtc = p->dT / p->coarse_steps, nud = p->nu * n * (double)n;
        // every coefficient an FP32 value: the float-float stage can drop their low parts
        bool c32 = !(getenv("PIT_ADV_COEF32") && getenv("PIT_ADV_COEF32")[0] == '0');
        for (size_t i = 0; i < M && c32; ++i)
            c32 = (double)(float)vx[i] == vx[i] && (double)(float)vy[i] == vy[i];
        p->adv_coef32 = c32 ? 1 : 0;
        // PIT_SPIN_LIMIT: polls of each bounded wait of the sweep (tests of the timeout path)
        if (const char *sl = getenv("PIT_SPIN_LIMIT")) {
            char *end = nullptr;
            const long long v = strtoll(sl, &end, 10);
            if (end != sl && v >= 0) p->adv_spin = v;
        }
        double rho = 0.0;
        for (size_t i = 0; i < M; ++i) {
            const double D = 1.0 + dtc * (4.0 * nud + fabs(vx[i]) + fabs(vy[i]));
            rho = std::max(rho, (D - 1.0) / D);
        }
        const double lmin = 1.0 - rho, lmax = 1.0 + rho;
        const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
        p->adv_K = p->coarse_inner > 0 ? p->coarse_inner : 48;
        p->adv_inv_theta = 1.0 / theta;
        double r = 1.0 / sigma;
        for (int k = 0; k < SWA_KMAX; ++k) {
            const double rn = 1.0 / (2.0 * sigma - r);
            p->adv_c1[k] = rn * r;
            p->adv_c2[k] = 2.0 * rn / delta;
            r = rn;
        }
        if (!(delta > 0.0)) {
            // nu = 0 and v = 0: I - dT L = I, and w = b after one step is exact
            p->adv_K = 1;
            for (int k = 0; k < SWA_KMAX; ++k) p->adv_c1[k] = p->adv_c2[k] = 0.0;
        }
    }
    // the cluster shape must be schedulable (n / 32 CTAs of one SM each)
    const int CS = n / AD_ROWS > 0 ? n / AD_ROWS : 1;
    const size_t sm = adv_smem<float, true>(n);
    PIT_CUDA(cudaFuncSetAttribute(k_advdiff_fine<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (CS > 8)
        PIT_CUDA(cudaFuncSetAttribute(k_advdiff_fine<float, true>,
                                      cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CS, 1, 1);
    cfg.blockDim = dim3((unsigned)n, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    PIT_CUDA(cudaOccupancyMaxActiveClusters(&clusters, k_advdiff_fine<float, true>, &cfg));
    if (clusters < 1) {
        set_error("advdiff2d: the " + std::to_string(CS) + "-CTA cluster of the fine kernel cannot be scheduled");
        return PIT_E_UNSUPPORTED;
    }
    return PIT_OK;
}

pit_status advdiff_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                           const MemberState *st, cudaStream_t s) {
    const AdvArgs a = adv_args(p, x, y, nullptr, mode, st, prec);
    if (prec == PIT_MIXED) return launch_adv_fine<float>(p, a, p->N, s);
    if (prec == PIT_FF) return launch_adv_fine<ff>(p, a, p->N, s);
    return launch_adv_fine<double>(p, a, p->N, s);
}

pit_status advdiff_fine_f32out(Problem *p, const double *x, float *q32, const MemberState *st,
                               cudaStream_t s) {
    return launch_adv_fine<float>(p, adv_args(p, x, nullptr, q32, FINE_APPLY, st, PIT_MIXED), p->N, s);
}

pit_status advdiff_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s) {
    const AdvArgs a = adv_args(p, x, y - (size_t)p->M, nullptr, 2, nullptr, prec);
    if (prec == PIT_MIXED) return launch_adv_fine<float>(p, a, 1, s);
    if (prec == PIT_FF) return launch_adv_fine<ff>(p, a, 1, s);
    return launch_adv_fine<double>(p, a, 1, s);
}

pit_status advdiff_sweep(Problem *p, const double *q, double *z, int prec, const MemberState *st,
                         cudaStream_t s) {
    if (prec == PIT_MIXED)
        return launch_adv_sweep<float>(p, q, z, p->vx32.as<float>(), p->vy32.as<float>(), st, s);
    return launch_adv_sweep<double>(p, q, z, p->vx64.as<double>(), p->vy64.as<double>(), st, s);
}

}  // namespace pit
