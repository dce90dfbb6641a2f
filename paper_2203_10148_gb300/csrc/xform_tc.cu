// Sine transforms of the 2D heat coarse sweep on the tensor cores.
//
// The exact implicit-Euler coarse step of the 5-point Laplacian is diagonal
// in the discrete sine basis, S[k][i] = sin(pi (k+1)(i+1) / (n+1)), so the
// sweep G^{-1} of eq. (7) runs as  qhat = S q S,  a recurrence per mode over
// the slices, and  z = (2/(n+1))^2 S zhat S.  Each of the four passes is
//     out_b[k][j] = scale * sum_i S[k][i] A_b[j][i]      (out_b = scale (A_b S)^T)
// for every n x n block b of the block vector: one GEMM of all blocks' rows
// (r = b * n + j) against S, stored transposed per block so that the next
// pass contracts the other index.
//
// Arithmetic: split TF32 (3xTF32), A = Ah + Al and S = Sh + Sl with every
// part a TF32 value rounded to nearest, C = Ah Sh^T + Ah Sl^T + Al Sh^T in
// FP32 (Al Sl^T is below FP32 resolution) -- the accuracy class of the FP32
// transforms it replaces.  The sweep only preconditions (its FP32 error
// enters the inner solve's operator, not the float-float true residual).
//
// Kernel: persistent, one CTA per SM, output tiles t = blockIdx.x,
// +gridDim.x, ... of 128 x 128 (one per block for 96 <= n <= 128, 2 x 2 for
// 128 < n <= 256; n % 4 == 0; rows and columns beyond n read as zero or are
// not stored).  Warp roles:
//   warp 0      TMA: for n <= 128 Sh and Sl once (resident, 128 KB), then
//               each tile's chunks of A (32 columns) into a 6-stage ring of
//               raw chunks; for n > 128 each chunk of A with the matching
//               chunks of Sh and Sl into a 3-stage ring;
//   warp 1      one thread issues tcgen05.mma (kind::tf32, M = N = 128,
//               K = 8) into one of two TMEM accumulators (2 x 128 columns);
//   warps 2..9  split each landed chunk into Ah and Al.  S resident: each
//               thread reads its row of the chunk (the 128-byte swizzle
//               undone in the address) and writes its parts into one of two
//               A buffers in tensor memory (tcgen05.st, 2 x 64 columns), the
//               raw stage freed at once; the products read A from tensor
//               memory, so splitting the next chunk overlaps them and the
//               shared-memory port carries only the TMA writes, the split's
//               reads and the B operand.  S streamed: in place in the stage;
//   warps 10..17 drain an accumulator with tcgen05.ld (one row per thread;
//               two warps per 32-lane quarter of TMEM, 64 columns each) and
//               write the block transposed: for each k the 32 lanes of a
//               warp store 32 consecutive j (coalesced), scaled, FP32 or FP64.
// Stage and accumulator hand-offs are mbarriers; every wait is bounded and
// reports PIT_E_TIMEOUT through the problem's error word.
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "pit_internal.h"
#include "stencil_arith.cuh"
#include "tc_common.cuh"

namespace pit {
namespace {

constexpr int XT_T = 128;                              // tile rows (TMEM lanes) = columns
constexpr int XT_BK = 32;                              // K per chunk (128 bytes of FP32)
constexpr int XT_STAGES = 3;                           // S streamed: stages of [Ah][Al][Sh][Sl]
constexpr int XT_RAW = 6;                              // S resident: raw A chunks in flight
constexpr int XT_ABUF = 2 * XT_T;                      // S resident: first TMEM column of the A buffers
constexpr int XT_CH = XT_T * XT_BK * 4;                // 16 KB: one chunk of one operand part
constexpr int XT_S_BYTES = (XT_T / XT_BK) * XT_CH;     // 64 KB: one part of a resident S (n <= 128)
constexpr int XT_CONV_WARPS = 8;                       // split a 16 KB chunk: 4 float4 per thread
constexpr int XT_EPI_WARPS = 8;                        // two per TMEM lane quarter
constexpr int XT_THREADS = 32 * (2 + XT_CONV_WARPS + XT_EPI_WARPS);
constexpr int XT_CONV_THREADS = 32 * XT_CONV_WARPS;
constexpr int XT_EPI0 = 2 + XT_CONV_WARPS;             // first epilogue warp
constexpr uint32_t kXtIdesc = tc_idesc_tf32(XT_T, XT_T);

// Shared memory: S resident (n <= 128): [Sh 64 KB][Sl 64 KB] + 6 raw A
// chunks; S streamed (n > 128): 3 stages of [Ah][Al][Sh][Sl].  Then 26
// mbarriers and the TMEM address.  Tensor memory: two accumulators (256
// columns) and, S resident, two A buffers [Ah 32 columns][Al 32 columns].
template <bool SRES>
struct XtLayout {
    static constexpr int kStages = SRES ? XT_RAW : XT_STAGES;
    static constexpr int kStage = SRES ? XT_CH : 4 * XT_CH;
    static constexpr int kRing = SRES ? 2 * XT_S_BYTES : 0;
    static constexpr int kBar = kRing + kStages * kStage;
    static constexpr int kSmem = 1024 + kBar + 256;
    static constexpr uint32_t kTmemCols = SRES ? 4 * XT_T : 2 * XT_T;
};

__device__ __forceinline__ bool xt_live(const MemberState *st, int b) {
    if (st == nullptr) return true;
    const MemberState &m = st[b];
    return m.active && !m.skip && !m.half;
}

// x rounded to TF32 (10 mantissa bits), to nearest with ties away from
// zero: half a TF32 ulp added to the magnitude bits, the 13 low bits
// cleared (a carry moves into the next binade; overflow gives infinity).
// Infinities and NaNs pass unchanged.  Integer-pipe work only.
__device__ __forceinline__ float tf32_rna(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t r = (b + 0x1000u) & 0xffffe000u;
    return __uint_as_float((b & 0x7f800000u) == 0x7f800000u ? b : r);
}

// Output tiles t = (block, tj, tk), TN x TN of them per block (TN = 1 for
// n <= 128, 2 for n <= 256): rows j = 128 tj + lane, columns k = 128 tk + ...;
// K in KC = ceil(n / 32) chunks.
//
// ROW1D (1D heat): one matrix of R = batch (N+1) rows of length n (padded),
// out[r][k] = scale sum_i S[k][i] A[r][i] for k < nout, stored row-major with
// stride ldo; tiles t = (tk, ti) over 128 modes x 128 rows, the tensor core
// computing D[k][r] (S as the A operand, the data as B) so that TMEM lanes
// are modes and a warp's stores cover 32 consecutive k of one row.
template <bool OUT64, bool SRES, bool ROW1D>
__global__ void __launch_bounds__(XT_THREADS, 1)
    k_xform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmSh,
               const __grid_constant__ CUtensorMap tmSl, void *out_raw, int n, int total_tiles,
               int TN, int nblk, int R, int nout, int ldo, float scale, const MemberState *st,
               int *err) {
    static_assert(!(ROW1D && SRES), "the 1D transform streams S");
    using LY = XtLayout<SRES>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *Sres = base;                          // resident Sh, then Sl (SRES)
    unsigned char *ring = base + LY::kRing;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + LY::kBar);
    constexpr int NS = LY::kStages;
    // S streamed: full (TMA landed), conv (split in place), empty (consumed
    // by the tensor core) per stage.  S resident: full (raw chunk landed)
    // and empty (raw chunk read by the converters) per stage, conv[a] (A
    // buffer a written) and conv[2 + a] (A buffer a consumed by the
    // tensor core) for the two TMEM A buffers.
    uint64_t *full = bars;
    uint64_t *empty = bars + 8;
    uint64_t *conv = bars + 16;
    uint64_t *tfull = bars + 20;                 // accumulator complete, 2 buffers
    uint64_t *tempty = tfull + 2;                // accumulator drained, 2 buffers
    uint64_t *sbar = tempty + 2;                 // resident S landed
    uint64_t *mdone = sbar + 1;                  // all products issued have finished
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // K chunks per tile: all four for a resident S (n <= 128, chunks past n
    // read as zero), ceil(n / 32) otherwise
    const int KC = SRES ? XT_T / XT_BK : (n + XT_BK - 1) / XT_BK;
    const int tpb = TN * TN;                     // tiles per block

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], SRES ? XT_CONV_THREADS : 1);
            if (!SRES) mbar_init(&conv[s], XT_CONV_THREADS);
        }
        if (SRES) {
            for (int a = 0; a < 2; ++a) {
                mbar_init(&conv[a], XT_CONV_THREADS);
                mbar_init(&conv[2 + a], 1);
            }
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], XT_EPI_WARPS);
        }
        mbar_init(sbar, 1);
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(LY::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            if constexpr (SRES) {
                mbar_expect_tx(sbar, 2 * XT_S_BYTES);
                for (int c = 0; c < XT_T / XT_BK; ++c) {
                    tma_load_2d(Sres + c * XT_CH, &tmSh, c * XT_BK, 0, sbar);
                    tma_load_2d(Sres + XT_S_BYTES + c * XT_CH, &tmSl, c * XT_BK, 0, sbar);
                }
            }
            int last_use[NS];
            for (int s = 0; s < NS; ++s) last_use[s] = -1;
            int q = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
                int arow, srow;       // first data row and first S row of the tile
                if constexpr (ROW1D) {
                    arow = (t % TN) * XT_T;
                    srow = (t / TN) * XT_T;
                } else {
                    const int b = t / tpb, tj = (t % tpb) / TN, tk = t % TN;
                    if (!xt_live(st, b / nblk)) continue;
                    arow = b * n + tj * XT_T;
                    srow = tk * XT_T;
                }
                for (int c = 0; c < KC; ++c, ++q) {
                    const int s = q % NS, u = q / NS;
                    if (!tc_mbar_wait(&empty[s], (uint32_t)(u & 1) ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    unsigned char *stg = ring + s * LY::kStage;
                    mbar_expect_tx(&full[s], SRES ? XT_CH : 3 * XT_CH);
                    tma_load_2d(stg, &tmA, c * XT_BK, arow, &full[s]);
                    if constexpr (!SRES) {
                        tma_load_2d(stg + 2 * XT_CH, &tmSh, c * XT_BK, srow, &full[s]);
                        tma_load_2d(stg + 3 * XT_CH, &tmSl, c * XT_BK, srow, &full[s]);
                    }
                    last_use[s] = u;
                }
            }
            // no copy of this CTA may still be writing shared memory at exit
            if constexpr (SRES) tc_mbar_drain(sbar, 0u);
            for (int s = 0; s < NS; ++s)
                if (last_use[s] >= 0) tc_mbar_drain(&full[s], (uint32_t)(last_use[s] & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            bool ok = SRES ? tc_mbar_wait(sbar, 0u, err) : true;
            int q = 0, L = 0;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
                if (!ROW1D && !xt_live(st, (t / tpb) / nblk)) continue;
                const int buf = L & 1, v = L >> 1;
                if (!tc_mbar_wait(&tempty[buf], (uint32_t)(v & 1) ^ 1u, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * XT_T);
                for (int c = 0; c < KC; ++c, ++q) {
                    const int s = q % NS, u = q / NS;
                    if constexpr (SRES) {
                        // A parts of chunk q in TMEM buffer q & 1
                        const int a = q & 1, ua = q >> 1;
                        if (!tc_mbar_wait(&conv[a], (uint32_t)(ua & 1), err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t ahi = tmem + (uint32_t)(XT_ABUF + a * 2 * XT_BK);
                        const uint64_t bh = smem_desc(Sres + c * XT_CH);
                        const uint64_t bl = smem_desc(Sres + XT_S_BYTES + c * XT_CH);
#pragma unroll
                        for (int j = 0; j < XT_BK / 8; ++j) {
                            const uint64_t adv = (uint64_t)(j * 32) >> 4;   // 8 TF32 = 32 bytes along K
                            const uint32_t acol = (uint32_t)(j * 8);        // 8 TF32 = 8 TMEM columns
                            tc_mma_tf32_ts(d, ahi + acol, bh + adv, kXtIdesc, (c > 0 || j > 0) ? 1u : 0u);
                            tc_mma_tf32_ts(d, ahi + acol, bl + adv, kXtIdesc, 1u);
                            tc_mma_tf32_ts(d, ahi + XT_BK + acol, bh + adv, kXtIdesc, 1u);
                        }
                        mma_commit(&conv[2 + a]);    // A buffer free once these products finish
                        continue;
                    }
                    if (!tc_mbar_wait(&conv[s], (uint32_t)(u & 1), err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *stg = ring + s * LY::kStage;
                    const uint64_t ah = smem_desc(stg), al = smem_desc(stg + XT_CH);
                    const uint64_t bh = smem_desc(stg + 2 * XT_CH), bl = smem_desc(stg + 3 * XT_CH);
#pragma unroll
                    for (int j = 0; j < XT_BK / 8; ++j) {
                        const uint64_t adv = (uint64_t)(j * 32) >> 4;   // 8 TF32 = 32 bytes along K
                        if constexpr (ROW1D) {
                            // D[k][r]: S rows as the A operand, data rows as B
                            tc_mma_tf32(d, bh + adv, ah + adv, kXtIdesc, (c > 0 || j > 0) ? 1u : 0u);
                            tc_mma_tf32(d, bl + adv, ah + adv, kXtIdesc, 1u);
                            tc_mma_tf32(d, bh + adv, al + adv, kXtIdesc, 1u);
                        } else {
                            tc_mma_tf32(d, ah + adv, bh + adv, kXtIdesc, (c > 0 || j > 0) ? 1u : 0u);
                            tc_mma_tf32(d, ah + adv, bl + adv, kXtIdesc, 1u);
                            tc_mma_tf32(d, al + adv, bh + adv, kXtIdesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);    // stage free once these products finish
                }
                if (!ok) break;
                mma_commit(&tfull[buf]);      // accumulator complete
                ++L;
            }
            mma_commit(mdone);
            tc_mbar_drain(mdone, 0u);
        }
    } else if (warp < XT_EPI0) {
        // ---- split: Ah = rna_tf32(a), Al = rna_tf32(a - Ah)
        if constexpr (SRES) {
            // into TMEM: warp quarter (warp % 4) owns rows 32 quarter .. +31
            // (its TMEM lanes); two warps per quarter, 16 columns each
            const int quarter = warp & 3, half = (warp - 2) >> 2;
            const int r = quarter * 32 + lane;
            const uint32_t tl = (uint32_t)(quarter * 32) << 16;
            int q = 0;
            for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
                if (!xt_live(st, (t / tpb) / nblk)) continue;
                bool ok = true;
                for (int c = 0; c < KC; ++c, ++q) {
                    const int s = q % NS, u = q / NS, a = q & 1, ua = q >> 1;
                    // chunk landed, and the products that read A buffer a
                    // (chunk q - 2) have finished
                    ok = __all_sync(0xffffffffu, tc_mbar_wait(&full[s], (uint32_t)(u & 1), err) &&
                                                     tc_mbar_wait(&conv[2 + a], (uint32_t)(ua & 1) ^ 1u, err)) != 0;
                    if (!ok) break;
                    // row r of the chunk: 16-byte granule g sits at g ^ (r % 8)
                    const unsigned char *row = ring + s * LY::kStage + r * (XT_BK * 4);
                    uint32_t h[16], l[16];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        const float4 x = *reinterpret_cast<const float4 *>(
                            row + (((half * 4 + g) ^ (r & 7)) << 4));
                        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float hv = tf32_rna(xs[e]);
                            h[4 * g + e] = __float_as_uint(hv);
                            l[4 * g + e] = __float_as_uint(tf32_rna(xs[e] - hv));
                        }
                    }
                    mbar_arrive(&empty[s]);   // raw chunk read: the TMA may refill it
                    const uint32_t col = tmem + tl + (uint32_t)(XT_ABUF + a * 2 * XT_BK + half * 16);
                    tmem_st16(col, h);
                    tmem_st16(col + XT_BK, l);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&conv[a]);
                }
                if (!ok) break;
            }
        } else {
            // in place in the stage (S streamed)
            const int ct = threadIdx.x - 64;
            int q = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
                if (!ROW1D && !xt_live(st, (t / tpb) / nblk)) continue;
                for (int c = 0; c < KC; ++c, ++q) {
                    const int s = q % NS, u = q / NS;
                    if (!tc_mbar_wait(&full[s], (uint32_t)(u & 1), err)) {
                        ok = false;
                        break;
                    }
                    float4 *hi = reinterpret_cast<float4 *>(ring + s * LY::kStage);
                    float4 *lo = reinterpret_cast<float4 *>(ring + s * LY::kStage + XT_CH);
#pragma unroll
                    for (int i = ct; i < XT_CH / 16; i += XT_CONV_THREADS) {
                        const float4 a = hi[i];
                        float4 h, l;
                        h.x = tf32_rna(a.x);
                        h.y = tf32_rna(a.y);
                        h.z = tf32_rna(a.z);
                        h.w = tf32_rna(a.w);
                        l.x = tf32_rna(a.x - h.x);
                        l.y = tf32_rna(a.y - h.y);
                        l.z = tf32_rna(a.z - h.z);
                        l.w = tf32_rna(a.w - h.w);
                        hi[i] = h;
                        lo[i] = l;
                    }
                    // generic-proxy writes become visible to the tensor core
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(&conv[s]);
                }
            }
        }
    } else {
        // ---- epilogue: TMEM lanes 32 (warp % 4) .. +31 are the tile rows;
        // this warp drains columns 64 half .. 64 half + 63
        const int quad = warp & 3, half = (warp - XT_EPI0) >> 2;
        constexpr int CPW = XT_T / 32 / (XT_EPI_WARPS / 4);   // 32-column groups per warp
        const size_t nn = (size_t)n * n;
        int L = 0;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
            const int b = t / tpb, tj = (t % tpb) / TN, tk = t % TN;
            if (!ROW1D && !xt_live(st, b / nblk)) continue;
            const int buf = L & 1, v = L >> 1;
            const bool ok = __all_sync(0xffffffffu, tc_mbar_wait(&tfull[buf], (uint32_t)(v & 1), err) ? 1 : 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if constexpr (ROW1D) {
                // lane = mode k, columns = rows r of the data
                const int k = (t / TN) * XT_T + quad * 32 + lane;
                const int rbase = (t % TN) * XT_T;
#pragma unroll 1
                for (int cc = half * CPW; cc < (half + 1) * CPW; ++cc) {
                    float vals[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * XT_T + cc * 32), vals);
                    if (k < nout) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int r = rbase + cc * 32 + i;
                            if (r < R && xt_live(st, r / nblk)) {
                                if constexpr (OUT64)
                                    reinterpret_cast<double *>(out_raw)[(size_t)r * ldo + k] = f2d(scale * vals[i]);
                                else
                                    reinterpret_cast<float *>(out_raw)[(size_t)r * ldo + k] = scale * vals[i];
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                ++L;
                continue;
            }
            const int j = tj * XT_T + quad * 32 + lane;
#pragma unroll 1
            for (int cc = half * CPW; cc < (half + 1) * CPW; ++cc) {
                float vals[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * XT_T + cc * 32), vals);
                const int k0 = tk * XT_T + cc * 32;
                if (j < n) {
                    if constexpr (OUT64) {
                        double *ob = reinterpret_cast<double *>(out_raw) + (size_t)b * nn + j;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (k0 + i < n) ob[(size_t)(k0 + i) * n] = f2d(scale * vals[i]);
                    } else {
                        float *ob = reinterpret_cast<float *>(out_raw) + (size_t)b * nn + j;
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (k0 + i < n) ob[(size_t)(k0 + i) * n] = scale * vals[i];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++L;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LY::kTmemCols));
    }
}

template <bool OUT64, bool SRES, bool ROW1D = false>
pit_status launch_xform_tc(const CUtensorMap &tA, const CUtensorMap &tSh, const CUtensorMap &tSl,
                           void *out, int n, int total_tiles, int TN, int nblk, float scale,
                           const MemberState *st, int *err, int grid, cudaStream_t s, int R = 0,
                           int nout = 0, int ldo = 0) {
    auto kern = k_xform_tc<OUT64, SRES, ROW1D>;
    PIT_TRY(smem_limit(kern, XtLayout<SRES>::kSmem));
    kern<<<grid, XT_THREADS, XtLayout<SRES>::kSmem, s>>>(tA, tSh, tSl, out, n, total_tiles, TN, nblk,
                                                          R, nout, ldo, scale, st, err);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

uint32_t tf32_rna_host(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    // round the magnitude to 10 mantissa bits, ties away from zero
    if ((b & 0x7f800000u) != 0x7f800000u) b += 0x1000u;
    return b & 0xffffe000u;
}

float bits_to_float(uint32_t b) {
    float x;
    memcpy(&x, &b, 4);
    return x;
}

}  // namespace

bool heat2d_tc_usable(const Problem *p) {
    return p->nx >= 96 && p->nx <= 2 * XT_T && p->nx % 4 == 0 && tc_encode_fn() != nullptr;
}

pit_status heat2d_tc_setup(Problem *p, const double *S) {
    const int n = p->nx;
    const size_t nn = (size_t)n * n;
    std::vector<float> parts(2 * nn);
    for (size_t i = 0; i < nn; ++i) {
        const float h = bits_to_float(tf32_rna_host((float)S[i]));
        parts[i] = h;
        parts[nn + i] = bits_to_float(tf32_rna_host((float)(S[i] - (double)h)));
    }
    PIT_TRY(p->xtc_S.ensure(2 * nn * sizeof(float)));
    PIT_CUDA(cudaMemcpyAsync(p->xtc_S.ptr, parts.data(), 2 * nn * sizeof(float),
                             cudaMemcpyHostToDevice, p->stream));
    PIT_CUDA(cudaStreamSynchronize(p->stream));
    return PIT_OK;
}

pit_status heat2d_tc_xform(Problem *p, const float *A, void *out, bool out64, double scale,
                           const MemberState *st, cudaStream_t s) {
    const int n = p->nx;
    const int blocks = p->batch * (p->N + 1);
    const int TN = (n + XT_T - 1) / XT_T;
    const int total_tiles = blocks * TN * TN;
    const float *Sh = p->xtc_S.as<float>();
    CUtensorMap tA, tSh, tSl;
    PIT_TRY(tc_make_map(&tA, A, blocks * n, n, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSh, Sh, n, n, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSl, Sh + (size_t)n * n, n, n, XT_BK, XT_T));
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(total_tiles, sms);
    int *err = p->errword.as<int>();
    const float sc = (float)scale;
    if (TN == 1) {
        if (out64) return launch_xform_tc<true, true>(tA, tSh, tSl, out, n, total_tiles, TN, p->N + 1, sc, st, err, grid, s);
        return launch_xform_tc<false, true>(tA, tSh, tSl, out, n, total_tiles, TN, p->N + 1, sc, st, err, grid, s);
    }
    if (out64) return launch_xform_tc<true, false>(tA, tSh, tSl, out, n, total_tiles, TN, p->N + 1, sc, st, err, grid, s);
    return launch_xform_tc<false, false>(tA, tSh, tSl, out, n, total_tiles, TN, p->N + 1, sc, st, err, grid, s);
}

// ------------------------------------------------------------ 1D heat
namespace {

// S[k][i] = sin(pi (k+1)(i+1) / (M+1)) for k, i < M, zero padding to Mp;
// split into TF32 parts hi = rna(fl32(S)), lo = rna(fl32(S - hi)).  The
// argument is reduced exactly in integers, (k+1)(i+1) mod 2(M+1).
__global__ void k_make_dst1d(float *Sh, float *Sl, int M, int Mp) {
    const size_t total = (size_t)Mp * Mp;
    const long long period = 2LL * (M + 1);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / Mp), i = (int)(e % Mp);
        float h = 0.f, l = 0.f;
        if (k < M && i < M) {
            const long long m = ((long long)(k + 1) * (i + 1)) % period;
            const double v = sinpi((double)m / (double)(M + 1));
            h = tf32_rna(__double2float_rn(v));
            l = tf32_rna(__double2float_rn(v - (double)h));
        }
        Sh[e] = h;
        Sl[e] = l;
    }
}

// rows of length M (FP64 or FP32) into rows of length Mp (FP32, zero padded)
template <class Tin>
__global__ void k_pack_rows(const Tin *__restrict__ q, float *__restrict__ out, int R, int M, int Mp) {
    const size_t total = (size_t)R * Mp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Mp), i = (int)(e % Mp);
        float v = 0.f;
        if (i < M) {
            if constexpr (std::is_same<Tin, double>::value) v = d2f_rn(q[(size_t)r * M + i]);
            else v = q[(size_t)r * M + i];
        }
        out[e] = v;
    }
}

}  // namespace

int heat1d_tc_padded(int M) { return (M + 31) / 32 * 32; }

pit_status heat1d_tc_setup(Problem *p) {
    const int M = p->M, Mp = heat1d_tc_padded(M);
    PIT_TRY(p->xtc_S.ensure(2 * (size_t)Mp * Mp * sizeof(float)));
    float *Sh = p->xtc_S.as<float>();
    k_make_dst1d<<<1024, 256, 0, p->stream>>>(Sh, Sh + (size_t)Mp * Mp, M, Mp);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

// out = scale * (S A^T)^T for the rows of A: A (R x Mp FP32, zero padded),
// out R x nout with row stride ldo (FP32 or FP64)
pit_status heat1d_tc_xform(Problem *p, const float *A, void *out, bool out64, int nout, int ldo,
                           double scale, const MemberState *st, cudaStream_t s) {
    const int M = p->M, Mp = heat1d_tc_padded(M);
    const int R = p->batch * (p->N + 1);
    const int RT = (R + XT_T - 1) / XT_T, KT = (Mp + XT_T - 1) / XT_T;
    const int total_tiles = RT * KT;
    const float *Sh = p->xtc_S.as<float>();
    CUtensorMap tA, tSh, tSl;
    PIT_TRY(tc_make_map(&tA, A, R, Mp, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSh, Sh, Mp, Mp, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSl, Sh + (size_t)Mp * Mp, Mp, Mp, XT_BK, XT_T));
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(total_tiles, sms);
    int *err = p->errword.as<int>();
    const float sc = (float)scale;
    if (out64)
        return launch_xform_tc<true, false, true>(tA, tSh, tSl, out, Mp, total_tiles, RT, p->N + 1, sc,
                                                  st, err, grid, s, R, nout, ldo);
    return launch_xform_tc<false, false, true>(tA, tSh, tSl, out, Mp, total_tiles, RT, p->N + 1, sc,
                                               st, err, grid, s, R, nout, ldo);
}

pit_status heat1d_tc_pack(Problem *p, const double *q, float *out, cudaStream_t s) {
    const int M = p->M, Mp = heat1d_tc_padded(M);
    const int R = p->batch * (p->N + 1);
    k_pack_rows<double><<<1024, 256, 0, s>>>(q, out, R, M, Mp);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

}  // namespace pit
