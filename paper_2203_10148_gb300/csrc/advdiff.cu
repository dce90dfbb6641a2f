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

constexpr int AD_RY = 8;                     // rows of a thread tile
constexpr int AD_H = AD_RY / 2;              // rows r and r + AD_H share a packed pair
constexpr int AD_ROWS = 32;                  // rows per CTA (cluster size = n / 32)
constexpr int AD_TY = AD_ROWS / AD_RY;       // 4 thread rows per CTA

struct AdvArgs {
    const double *x;
    double *y;
    float *y32;
    const double *y0;
    const void *ax, *ay;   // per-point coefficients (float, double or (hi, lo) float pairs), row-major n x n
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

// Scalar stage (FP64): w = u + cc L v at one point.
__device__ __forceinline__ double adv_stage(double vn, double vs, double vw, double ve, double vc,
                                            double u, double cc, double nud, double ax, double ay) {
    const double lap = fma(-4.0, vc, (ve + vw) + (vn + vs));
    const double dX = (ax >= 0.0) ? (vc - vw) : (ve - vc);
    const double dY = (ay >= 0.0) ? (vc - vn) : (vs - vc);
    const double adv = fma(ay, dY, ax * dX);
    return fma(cc, fma(nud, lap, -adv), u);
}

// FP32 stage on two points per packed instruction, with the scalar stage's
// roundings: lap = (ve + vw) + (vn + vs) - 4 vc, adv = ay dY + fl(ax dX),
// w = u + cc (nud lap - adv).  The coefficients come negated (nax = -ax):
// -fl(ax dX) = fl(nax dX) and -adv = fl(nay dY + fl(nax dX)) exactly, so
// no negation is issued; ax >= 0 is nax <= 0 (also for signed zeros).
__device__ __forceinline__ float2 adv_stage_f2(float2 vn, float2 vs, float2 vw, float2 ve, float2 vc,
                                               float2 u, float2 cc, float2 nud, float2 nax, float2 nay) {
    const float2 lap = __ffma2_rn(make_float2(-4.f, -4.f), vc,
                                  __fadd2_rn(__fadd2_rn(ve, vw), __fadd2_rn(vn, vs)));
    const float2 dW = f2_sub(vc, vw), dE = f2_sub(ve, vc);
    const float2 dN = f2_sub(vc, vn), dS = f2_sub(vs, vc);
    const float2 dX = make_float2(nax.x <= 0.f ? dW.x : dE.x, nax.y <= 0.f ? dW.y : dE.y);
    const float2 dY = make_float2(nay.x <= 0.f ? dN.x : dS.x, nay.y <= 0.f ? dN.y : dS.y);
    const float2 nadv = __ffma2_rn(nay, dY, __fmul2_rn(nax, dX));
    return __ffma2_rn(cc, __ffma2_rn(nud, lap, nadv), u);
}

// TwoSum(a, -b) on packed pairs: s = fl(a - b) and e = (a - b) - s exactly.
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2 &s, float2 &e) {
    s = f2_sub(a, b);
    const float2 bb = f2_sub(s, a);   // the -b actually added
    e = f2_sub(f2_sub(a, f2_sub(s, bb)), __fadd2_rn(b, bb));
}

// Float-float stage on two points per packed instruction (the residual
// arithmetic, about 48 significant bits on the FP32 pipe).  The upwind term
// is written |ax| (vc - ux) with ux the upwind neighbour (vw where ax >= 0,
// else ve), which equals ax dX exactly.  High parts are summed with exact
// TwoSums, products keep their exact FMA error terms, the errors and the low
// parts are summed in FP32; the result is left unnormalised (its low part a
// few ulp of its high part at most, summed in FP32 next to exact sums of high
// parts by the next stage) and renormalised once per time step.  A
// coefficient pair is (hi, lo) per lane; C32: coefficients that are FP32
// values, whose low parts are zero and skipped.
struct AdCoefFF {
    float2 hi, lo;
};

template <bool C32>
__device__ __forceinline__ ff2 adv_stage_ff2(const ff2 &vn, const ff2 &vs, const ff2 &vw, const ff2 &ve,
                                             const ff2 &vc, const ff2 &u, float2 cch, float2 ncch, float2 ccl,
                                             float2 nudh, float2 nnudh, float2 nudl, const AdCoefFF &ax,
                                             const AdCoefFF &ay) {
    const float2 m4 = make_float2(-4.f, -4.f);
    // vn + vs + vw + ve - 4 vc = dh + lap_lo
    float2 ah, al, bh, bl, ch, cl;
    two_sum2(vn.hi, vs.hi, ah, al);
    two_sum2(vw.hi, ve.hi, bh, bl);
    two_sum2(ah, bh, ch, cl);
    const float2 dh = __ffma2_rn(m4, vc.hi, ch);
    const float2 nbb = f2_sub(ch, dh);
    const float2 dl = __fadd2_rn(f2_sub(ch, __fadd2_rn(dh, nbb)), __ffma2_rn(m4, vc.hi, nbb));
    const float2 lap_lo = __ffma2_rn(
        m4, vc.lo,
        __fadd2_rn(__fadd2_rn(__fadd2_rn(al, bl), __fadd2_rn(cl, dl)),
                   __fadd2_rn(__fadd2_rn(vn.lo, vs.lo), __fadd2_rn(vw.lo, ve.lo))));
    // upwind neighbours and coefficient magnitudes, per lane
    const bool px0 = ax.hi.x >= 0.f, px1 = ax.hi.y >= 0.f;
    const bool py0 = ay.hi.x >= 0.f, py1 = ay.hi.y >= 0.f;
    const float2 uxh = make_float2(px0 ? vw.hi.x : ve.hi.x, px1 ? vw.hi.y : ve.hi.y);
    const float2 uxl = make_float2(px0 ? vw.lo.x : ve.lo.x, px1 ? vw.lo.y : ve.lo.y);
    const float2 uyh = make_float2(py0 ? vn.hi.x : vs.hi.x, py1 ? vn.hi.y : vs.hi.y);
    const float2 uyl = make_float2(py0 ? vn.lo.x : vs.lo.x, py1 ? vn.lo.y : vs.lo.y);
    const float2 axh = make_float2(fabsf(ax.hi.x), fabsf(ax.hi.y));
    const float2 ayh = make_float2(fabsf(ay.hi.x), fabsf(ay.hi.y));
    const float2 naxh = make_float2(-axh.x, -axh.y), nayh = make_float2(-ayh.x, -ayh.y);
    // dx = vc - ux, dy = vc - uy
    float2 dxh, dxe, dyh, dye;
    two_diff2(vc.hi, uxh, dxh, dxe);
    two_diff2(vc.hi, uyh, dyh, dye);
    const float2 dxl = __fadd2_rn(dxe, f2_sub(vc.lo, uxl));
    const float2 dyl = __fadd2_rn(dye, f2_sub(vc.lo, uyl));
    // p1 = fl(nud dh), p2 = fl(|ax| dx), p3 = fl(|ay| dy) taken negated; e_i
    // collect the products' exact rounding errors and their low-part terms
    const float2 np1 = __fmul2_rn(nnudh, dh);
    float2 e1 = __ffma2_rn(nudh, dh, np1);
    e1 = __ffma2_rn(nudh, lap_lo, e1);
    e1 = __ffma2_rn(nudl, dh, e1);
    const float2 np2 = __fmul2_rn(naxh, dxh);
    float2 e2 = __ffma2_rn(axh, dxh, np2);
    e2 = __ffma2_rn(axh, dxl, e2);
    const float2 np3 = __fmul2_rn(nayh, dyh);
    float2 e3 = __ffma2_rn(ayh, dyh, np3);
    e3 = __ffma2_rn(ayh, dyl, e3);
    if constexpr (!C32) {
        // |ax| = -ax where ax.hi < 0: the low part follows the high part's sign
        const float2 axl = make_float2(px0 ? ax.lo.x : -ax.lo.x, px1 ? ax.lo.y : -ax.lo.y);
        const float2 ayl = make_float2(py0 ? ay.lo.x : -ay.lo.x, py1 ? ay.lo.y : -ay.lo.y);
        e2 = __ffma2_rn(axl, dxh, e2);
        e3 = __ffma2_rn(ayl, dyh, e3);
    }
    // L = p1 - p2 - p3 + (e1 - e2 - e3) = s2h + l_lo
    float2 s1h, s1e, s2h, s2e;
    two_diff2(np2, np1, s1h, s1e);   // p1 - p2
    two_sum2(s1h, np3, s2h, s2e);    // - p3
    const float2 l_lo = __fadd2_rn(__fadd2_rn(s1e, s2e), f2_sub(f2_sub(e1, e2), e3));
    // u + cc L, p = fl(cc.hi s2h) taken negated
    const float2 pn = __fmul2_rn(ncch, s2h);
    float2 e = __ffma2_rn(cch, s2h, pn);
    e = __ffma2_rn(cch, l_lo, e);
    e = __ffma2_rn(ccl, s2h, e);
    const float2 sh = f2_sub(u.hi, pn);
    const float2 nb2 = f2_sub(u.hi, sh);
    const float2 sl = __fadd2_rn(f2_sub(u.hi, __fadd2_rn(sh, nb2)), f2_sub(nb2, pn));
    ff2 w;
    w.hi = sh;
    w.lo = __fadd2_rn(sl, __fadd2_rn(u.lo, e));
    return w;
}

template <class T>
__device__ __forceinline__ T adv_from_d(double x) { return (T)x; }
template <>
__device__ __forceinline__ float adv_from_d<float>(double x) { return d2f_rn(x); }
template <>
__device__ __forceinline__ ff adv_from_d<ff>(double x) { return ff_from_double(x); }

__device__ __forceinline__ double adv_to_d(float v) { return f2d(v); }
__device__ __forceinline__ double adv_to_d(double v) { return v; }
__device__ __forceinline__ double adv_to_d(ff v) { return f2d(v.hi) + f2d(v.lo); }

// A pair of points of a thread tile, rows r and r + AD_H of one column: the
// two lanes of every packed instruction.
template <class T>
struct AdPair;
template <>
struct AdPair<float> {
    using P = float2;
    __device__ static P make(float a, float b) { return make_float2(a, b); }
    __device__ static float x(const P &p) { return p.x; }
    __device__ static float y(const P &p) { return p.y; }
    __device__ static P shfl_idx(const P &p, int s) {
        return make_float2(__shfl_sync(kFullMask, p.x, s), __shfl_sync(kFullMask, p.y, s));
    }
    __device__ static P shfl_up(const P &p) {
        return make_float2(__shfl_up_sync(kFullMask, p.x, 1), __shfl_up_sync(kFullMask, p.y, 1));
    }
    __device__ static P shfl_down(const P &p) {
        return make_float2(__shfl_down_sync(kFullMask, p.x, 1), __shfl_down_sync(kFullMask, p.y, 1));
    }
};
template <>
struct AdPair<double> {
    using P = double2;
    __device__ static P make(double a, double b) { return make_double2(a, b); }
    __device__ static double x(const P &p) { return p.x; }
    __device__ static double y(const P &p) { return p.y; }
    __device__ static P shfl_idx(const P &p, int s) {
        return make_double2(__shfl_sync(kFullMask, p.x, s), __shfl_sync(kFullMask, p.y, s));
    }
    __device__ static P shfl_up(const P &p) {
        return make_double2(__shfl_up_sync(kFullMask, p.x, 1), __shfl_up_sync(kFullMask, p.y, 1));
    }
    __device__ static P shfl_down(const P &p) {
        return make_double2(__shfl_down_sync(kFullMask, p.x, 1), __shfl_down_sync(kFullMask, p.y, 1));
    }
};
template <>
struct AdPair<ff> {
    using P = ff2;
    __device__ static P make(ff a, ff b) { return ff_pair(a, b); }
    __device__ static ff x(const P &p) { return ff{p.hi.x, p.lo.x}; }
    __device__ static ff y(const P &p) { return ff{p.hi.y, p.lo.y}; }
    __device__ static P shfl_idx(const P &p, int s) {
        return ff2{AdPair<float>::shfl_idx(p.hi, s), AdPair<float>::shfl_idx(p.lo, s)};
    }
    __device__ static P shfl_up(const P &p) {
        return ff2{AdPair<float>::shfl_up(p.hi), AdPair<float>::shfl_up(p.lo)};
    }
    __device__ static P shfl_down(const P &p) {
        return ff2{AdPair<float>::shfl_down(p.hi), AdPair<float>::shfl_down(p.lo)};
    }
};

// A thread's RX consecutive values of a row buffer are stored as 16-byte
// chunks in chunk-major order: chunk q of thread column tx at element
// q * TX * CW + tx * CW (CW values per 16 bytes), so that a warp's 16-byte
// accesses to one chunk are contiguous (no shared-memory bank conflicts).
__device__ __forceinline__ float4 adv_chunk(const float *v) { return make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ float4 adv_chunk(const ff *v) { return make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo); }
__device__ __forceinline__ double2 adv_chunk(const double *v) { return make_double2(v[0], v[1]); }
__device__ __forceinline__ void adv_unchunk(float4 t, float *v) {
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void adv_unchunk(float4 t, ff *v) {
    v[0] = ff{t.x, t.y};
    v[1] = ff{t.z, t.w};
}
__device__ __forceinline__ void adv_unchunk(double2 t, double *v) {
    v[0] = t.x;
    v[1] = t.y;
}

template <class T, int RX>
struct RowChunks {
    static constexpr int CW = 16 / (int)sizeof(T);
    static_assert(RX % CW == 0, "a thread's row segment is whole 16-byte chunks");
    using C = typename std::conditional<std::is_same<T, double>::value, double2, float4>::type;
    __device__ static void store(T *row, int tx, int TX, const T (&v)[RX]) {
#pragma unroll
        for (int q = 0; q < RX / CW; ++q)
            *reinterpret_cast<C *>(row + (size_t)q * TX * CW + (size_t)tx * CW) = adv_chunk(&v[q * CW]);
    }
    __device__ static void load(const T *row, int tx, int TX, T (&v)[RX]) {
#pragma unroll
        for (int q = 0; q < RX / CW; ++q)
            adv_unchunk(*reinterpret_cast<const C *>(row + (size_t)q * TX * CW + (size_t)tx * CW), &v[q * CW]);
    }
};

// u records of the thread-private shared-memory layout, one 16-byte store each
__device__ __forceinline__ void adv_store_u(ff2 *p, const ff2 &v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y);
}
__device__ __forceinline__ void adv_store_u(double2 *p, const double2 &v) { *p = v; }
__device__ __forceinline__ void adv_store_u(float2 *, const float2 &) {}

// One cluster of CS = n/32 CTAs per (slice, member); each CTA holds 32 rows
// for all RK4 steps.  A thread owns an 8 x RX tile (RX = 4: n threads per
// CTA; RX = 8: n/2) kept as AD_H x RX pairs (rows r and r + 4 of a column).
// T = float (state, u and stage values in registers, coefficients negated in
// shared memory, packed f32x2 arithmetic), ff (state in registers, u in
// shared memory, coefficients read through L1 as 16-byte vectors, packed
// float-float arithmetic) or double (u in shared memory, scalar arithmetic
// on each lane).  Row buffers and the warp-edge column buffers are double
// buffered: one cluster barrier per RK4 stage.
template <class T, int RX, bool C32 = false>
__global__ void __launch_bounds__(RX == 4 ? 512 : 256, 1) k_advdiff_fine(AdvArgs a) {
    using PA = AdPair<T>;
    using P = typename PA::P;
    constexpr bool FP32 = std::is_same<T, float>::value;
    constexpr bool FF = std::is_same<T, ff>::value;
    constexpr int H = AD_H;
    constexpr int NT = 2048 / RX;                   // slot stride of u / coefficient records (threads at n = 512)
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
    const int TX = n / RX;                          // thread columns
    const int nthr = blockDim.x;                    // TX * AD_TY
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int lane = tid & 31;
    const int W = TX >> 5;                          // warps per thread row (0: part of one warp)
    const int Wc = W > 0 ? W : 1;
    const int wir = tx >> 5;                        // warp within the thread row
    const int i0 = tx * RX;
    const int j0 = rank * AD_ROWS + ty * AD_RY;     // global row of the tile's row 0
    // shared memory: [cc 4][rowbuf 2 buf x 2 top/bottom x TY x n]
    // [colbuf 2 buf x TY x 2 west/east x Wc x H pairs][u or coefficients]
    T *ccs = reinterpret_cast<T *>(smem_raw);
    T *rowbuf = reinterpret_cast<T *>(smem_raw + 32);
    P *colbuf = reinterpret_cast<P *>(rowbuf + (size_t)4 * AD_TY * n);
    unsigned char *tail = reinterpret_cast<unsigned char *>(colbuf + (size_t)4 * AD_TY * Wc * H);
    [[maybe_unused]] P *us = reinterpret_cast<P *>(tail);                  // u: [H x RX][NT]
    [[maybe_unused]] float4 *cx4 = reinterpret_cast<float4 *>(tail);       // FP32: [H x RX/2][NT]
    [[maybe_unused]] float4 *cy4 = cx4 + (size_t)H * (RX / 2) * NT;
    if (tid < 4) ccs[tid] = adv_from_d<T>(tid == 0 ? a.c[0] : tid == 1 ? a.c[1] : tid == 2 ? a.c[2] : a.c[3]);
    const size_t mb = (size_t)b * a.blen;
    const size_t nn = (size_t)n * n;
    const double *xin = a.x + mb + (size_t)(slice - 1) * nn;

    P v[H][RX];
    [[maybe_unused]] P ur[FP32 ? H : 1][FP32 ? RX : 1];
#pragma unroll
    for (int r = 0; r < H; ++r)
#pragma unroll
        for (int c = 0; c < RX; ++c) {
            const size_t kA = (size_t)(j0 + r) * n + (i0 + c), kB = kA + (size_t)H * n;
            v[r][c] = PA::make(adv_from_d<T>(xin[kA]), adv_from_d<T>(xin[kB]));
            if constexpr (FP32) ur[FP32 ? r : 0][FP32 ? c : 0] = v[r][c];
            else adv_store_u(us + (size_t)(r * RX + c) * NT + tid, v[r][c]);
        }
    if constexpr (FP32) {
        // negated coefficients of the tile, a float4 per two columns of a pair row
        const float *gx = reinterpret_cast<const float *>(a.ax);
        const float *gy = reinterpret_cast<const float *>(a.ay);
#pragma unroll
        for (int r = 0; r < H; ++r)
#pragma unroll
            for (int q = 0; q < RX / 2; ++q) {
                const size_t kA = (size_t)(j0 + r) * n + (i0 + 2 * q), kB = kA + (size_t)H * n;
                const size_t slot = (size_t)(r * (RX / 2) + q) * NT + tid;
                cx4[slot] = make_float4(-gx[kA], -gx[kB], -gx[kA + 1], -gx[kB + 1]);
                cy4[slot] = make_float4(-gy[kA], -gy[kB], -gy[kA + 1], -gy[kB + 1]);
            }
    }
    const T nud = adv_from_d<T>(a.nud);
    // north halo: the bottom row of the thread row above (periodic across the
    // cluster); south halo: the top row of the thread row below
    const int up_rank = (rank + CS - 1) % CS, down_rank = (rank + 1) % CS;
    const T *nsrc = (ty > 0) ? rowbuf : cluster.map_shared_rank(rowbuf, up_rank);
    const T *ssrc = (ty < AD_TY - 1) ? rowbuf : cluster.map_shared_rank(rowbuf, down_rank);
    const int nty = (ty > 0) ? ty - 1 : AD_TY - 1;
    const int sty = (ty < AD_TY - 1) ? ty + 1 : 0;
    int buf = 0;
    for (int s = 0; s < a.steps; ++s) {
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
            // publish the tile's top row (row 0) and bottom row (row 7)
            {
                T top[RX], bot[RX];
#pragma unroll
                for (int c = 0; c < RX; ++c) {
                    top[c] = PA::x(v[0][c]);
                    bot[c] = PA::y(v[H - 1][c]);
                }
                RowChunks<T, RX>::store(rowbuf + ((size_t)(buf * 2 + 0) * AD_TY + ty) * n, tx, TX, top);
                RowChunks<T, RX>::store(rowbuf + ((size_t)(buf * 2 + 1) * AD_TY + ty) * n, tx, TX, bot);
            }
            if (W > 1 && (lane == 0 || lane == 31)) {
                // colbuf[buf][ty][0: west column of warp w, 1: east column][w][pair row]
                P *cb = colbuf + ((((size_t)buf * AD_TY + ty) * 2 + (lane == 0 ? 0 : 1)) * Wc + wir) * H;
#pragma unroll
                for (int r = 0; r < H; ++r) cb[r] = (lane == 0) ? v[r][0] : v[r][RX - 1];
            }
            cluster.sync();
            const T cc = ccs[stage];
            [[maybe_unused]] float2 cc2, nud2, cch, ncch, ccl, nudh, nnudh, nudl;
            if constexpr (FP32) {
                cc2 = make_float2(cc, cc);
                nud2 = make_float2(nud, nud);
            } else if constexpr (FF) {
                cch = make_float2(cc.hi, cc.hi);
                ncch = make_float2(-cc.hi, -cc.hi);
                ccl = make_float2(cc.lo, cc.lo);
                nudh = make_float2(nud.hi, nud.hi);
                nnudh = make_float2(-nud.hi, -nud.hi);
                nudl = make_float2(nud.lo, nud.lo);
            }
            // north pair of pair row 0: rows -1 (halo) and H - 1 (not yet updated)
            P prev[RX];
            {
                T nh[RX];
                RowChunks<T, RX>::load(nsrc + ((size_t)(buf * 2 + 1) * AD_TY + nty) * n, tx, TX, nh);
#pragma unroll
                for (int c = 0; c < RX; ++c) prev[c] = PA::make(nh[c], PA::x(v[H - 1][c]));
            }
            // row H before its update: the south neighbour of row H - 1
            T rowH[RX];
#pragma unroll
            for (int c = 0; c < RX; ++c) rowH[c] = PA::y(v[0][c]);
            const P *cbt = colbuf + ((size_t)buf * AD_TY + ty) * 2 * Wc * H;
#pragma unroll
            for (int r = 0; r < H; ++r) {
                // west / east neighbours of the tile's first / last column (periodic in x)
                P w_in, e_in;
                if (W <= 1) {
                    // the thread row lies in one warp: lanes tx - 1 / tx + 1 modulo TX
                    const int seg = lane - tx;
                    w_in = PA::shfl_idx(v[r][RX - 1], seg + (tx + TX - 1) % TX);
                    e_in = PA::shfl_idx(v[r][0], seg + (tx + 1) % TX);
                } else {
                    w_in = PA::shfl_up(v[r][RX - 1]);
                    e_in = PA::shfl_down(v[r][0]);
                    if (lane == 0) w_in = cbt[(1 * Wc + (wir + W - 1) % W) * H + r];   // east column, warp to the west
                    if (lane == 31) e_in = cbt[(0 * Wc + (wir + 1) % W) * H + r];      // west column, warp to the east
                }
                [[maybe_unused]] T sh[RX];
                if (r == H - 1)
                    RowChunks<T, RX>::load(ssrc + ((size_t)(buf * 2 + 0) * AD_TY + sty) * n, tx, TX, sh);
                const size_t kA = (size_t)(j0 + r) * n + i0, kB = kA + (size_t)H * n;
                // Column by column, in place: prev[c] holds the north pair (pair
                // row r - 1 before its update) until column c is done, then the
                // old values of column c, which are the west pair of column c + 1
                // and the north pair of pair row r + 1.
                [[maybe_unused]] float4 f4x, f4y;
#pragma unroll
                for (int c = 0; c < RX; ++c) {
                    const P vw = (c > 0) ? prev[c > 0 ? c - 1 : 0] : w_in;
                    const P ve = (c < RX - 1) ? v[r][c < RX - 1 ? c + 1 : 0] : e_in;
                    const P vs = (r < H - 1) ? v[r < H - 1 ? r + 1 : 0][c] : PA::make(rowH[c], sh[c]);
                    P nv;
                    if constexpr (FP32) {
                        // negated coefficients of columns c, c + 1 (one float4)
                        if ((c & 1) == 0) {
                            const size_t slot = (size_t)(r * (RX / 2) + c / 2) * NT + tid;
                            f4x = cx4[slot];
                            f4y = cy4[slot];
                        }
                        const float2 nax = (c & 1) ? make_float2(f4x.z, f4x.w) : make_float2(f4x.x, f4x.y);
                        const float2 nay = (c & 1) ? make_float2(f4y.z, f4y.w) : make_float2(f4y.x, f4y.y);
                        nv = adv_stage_f2(prev[c], vs, vw, ve, v[r][c], ur[FP32 ? r : 0][FP32 ? c : 0], cc2, nud2,
                                          nax, nay);
                    } else if constexpr (FF) {
                        AdCoefFF qx, qy;
                        if constexpr (C32) {
                            const float *gx = reinterpret_cast<const float *>(a.ax);
                            const float *gy = reinterpret_cast<const float *>(a.ay);
                            qx = AdCoefFF{make_float2(__ldg(gx + kA + c), __ldg(gx + kB + c)), make_float2(0.f, 0.f)};
                            qy = AdCoefFF{make_float2(__ldg(gy + kA + c), __ldg(gy + kB + c)), make_float2(0.f, 0.f)};
                        } else {
                            const float2 *gx = reinterpret_cast<const float2 *>(a.ax);
                            const float2 *gy = reinterpret_cast<const float2 *>(a.ay);
                            const float2 xa = __ldg(gx + kA + c), xb = __ldg(gx + kB + c);
                            const float2 ya = __ldg(gy + kA + c), yb = __ldg(gy + kB + c);
                            qx = AdCoefFF{make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)};
                            qy = AdCoefFF{make_float2(ya.x, yb.x), make_float2(ya.y, yb.y)};
                        }
                        const float4 u4 = *reinterpret_cast<const float4 *>(us + (size_t)(r * RX + c) * NT + tid);
                        const ff2 u = ff2{make_float2(u4.x, u4.y), make_float2(u4.z, u4.w)};
                        nv = adv_stage_ff2<C32>(prev[c], vs, vw, ve, v[r][c], u, cch, ncch, ccl, nudh, nnudh, nudl,
                                                qx, qy);
                    } else {
                        const double *gx = reinterpret_cast<const double *>(a.ax);
                        const double *gy = reinterpret_cast<const double *>(a.ay);
                        const double qxa = __ldg(gx + kA + c), qxb = __ldg(gx + kB + c);
                        const double qya = __ldg(gy + kA + c), qyb = __ldg(gy + kB + c);
                        const P u = us[(size_t)(r * RX + c) * NT + tid];
                        const P vn = prev[c], vc = v[r][c];
                        nv = make_double2(adv_stage(vn.x, vs.x, vw.x, ve.x, vc.x, u.x, cc, nud, qxa, qya),
                                          adv_stage(vn.y, vs.y, vw.y, ve.y, vc.y, u.y, cc, nud, qxb, qyb));
                    }
                    prev[c] = v[r][c];
                    v[r][c] = nv;
                }
            }
            buf ^= 1;
        }
        // end of the step: the stage value becomes u (float-float renormalised)
#pragma unroll
        for (int r = 0; r < H; ++r)
#pragma unroll
            for (int c = 0; c < RX; ++c) {
                if constexpr (FF) v[r][c] = ff_renorm2(v[r][c]);
                if constexpr (FP32) ur[FP32 ? r : 0][FP32 ? c : 0] = v[r][c];
                else adv_store_u(us + (size_t)(r * RX + c) * NT + tid, v[r][c]);
            }
    }
    // all remote reads of this CTA's row buffers are done before anyone exits
    cluster.sync();
    const double *xn = a.x + mb + (size_t)slice * nn;
    double *yo = a.y + mb + (size_t)slice * nn;
#pragma unroll
    for (int r = 0; r < AD_RY; ++r)
#pragma unroll
        for (int c = 0; c < RX; ++c) {
            const size_t k = (size_t)(j0 + r) * n + (i0 + c);
            const T val = (r < H) ? PA::x(v[r < H ? r : 0][c]) : PA::y(v[r < H ? 0 : r - H][c]);
            if constexpr (FP32) {
                if (a.y32) {
                    a.y32[mb + (size_t)slice * nn + k] = d2f_rn(xn[k]) - val;
                    continue;
                }
            }
            const double f = adv_to_d(val);
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

// dynamic shared memory of k_advdiff_fine<T, RX>: [cc][row buffers][column
// buffers][u (ff, double) or the negated coefficients (float)]
template <class T, int RX>
size_t adv_smem(int n) {
    const size_t nthr = 2048 / RX;   // the kernel's record stride
    const size_t TX = (size_t)n / RX;
    const size_t Wc = TX >= 64 ? TX / 32 : 1;
    const size_t pair = 2 * sizeof(T);
    size_t s = 32 + 4 * AD_TY * (size_t)n * sizeof(T) + 4 * AD_TY * Wc * AD_H * pair;
    if (std::is_same<T, float>::value) s += 2 * (size_t)AD_H * RX * nthr * pair;
    else s += (size_t)AD_H * RX * nthr * pair;
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

template <class T, int RX, bool C32 = false>
pit_status launch_adv_fine_v(Problem *p, AdvArgs a, int nslices, cudaStream_t s) {
    const int n = p->nx;
    const int CS = n / AD_ROWS;
    const size_t sm = adv_smem<T, RX>(n);
    auto kern = k_advdiff_fine<T, RX, C32>;
    PIT_TRY(smem_limit(kern, sm));
    if (CS > 8)
        PIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    a.N = nslices;   // slices in this launch (output blocks n_first .. n_first + nslices - 1)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CS * nslices * p->batch), 1, 1);
    cfg.blockDim = dim3((unsigned)(n / RX * AD_TY), 1, 1);
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

// 8 x 4 thread tiles (n threads per CTA), or 8 x 8 (n/2 threads, n >= 256)
// where the problem selects them; float-float with FP32 coefficients reads
// them as FP32 values
template <class T, int RX>
pit_status launch_adv_fine_rx(Problem *p, AdvArgs a, int nslices, cudaStream_t s) {
    if (adv_smem<T, RX>(p->nx) > kSmemLimit) {
        set_error("advdiff2d: the slice does not fit the cluster's shared memory");
        return PIT_E_UNSUPPORTED;
    }
    if constexpr (std::is_same<T, ff>::value) {
        if (p->adv_coef32) {
            a.ax = p->vx32.ptr;
            a.ay = p->vy32.ptr;
            return launch_adv_fine_v<T, RX, true>(p, a, nslices, s);
        }
    }
    return launch_adv_fine_v<T, RX>(p, a, nslices, s);
}

template <class T>
pit_status launch_adv_fine(Problem *p, AdvArgs a, int nslices, cudaStream_t s) {
    if (p->adv_rx == 8 && p->nx >= 256) return launch_adv_fine_rx<T, 8>(p, a, nslices, s);
    return launch_adv_fine_rx<T, 4>(p, a, nslices, s);
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
    PIT_TRY(smem_limit(kern, smem));
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

template <class T, int RX>
pit_status adv_check_cluster(int n) {
    const int CS = n / AD_ROWS;
    const size_t sm = adv_smem<T, RX>(n);
    auto kern = k_advdiff_fine<T, RX, false>;
    PIT_TRY(smem_limit(kern, sm));
    if (CS > 8) PIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CS, 1, 1);
    cfg.blockDim = dim3((unsigned)(n / RX * AD_TY), 1, 1);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    PIT_CUDA(cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg));
    if (clusters < 1) {
        set_error("advdiff2d: the " + std::to_string(CS) + "-CTA cluster of the fine kernel cannot be scheduled");
        return PIT_E_UNSUPPORTED;
    }
    return PIT_OK;
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
    // PIT_ADV_RX=8: 8 x 8 thread tiles (n/2 threads per CTA) for n >= 256
    if (const char *rx = getenv("PIT_ADV_RX")) p->adv_rx = atoi(rx) == 8 ? 8 : 4;
    // the cluster shapes must be schedulable (n / 32 CTAs of one SM each);
    // the float-float kernel holds the most shared memory
    if (p->adv_rx == 8 && n >= 256) {
        PIT_TRY((adv_check_cluster<ff, 8>(n)));
    } else {
        PIT_TRY((adv_check_cluster<ff, 4>(n)));
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
