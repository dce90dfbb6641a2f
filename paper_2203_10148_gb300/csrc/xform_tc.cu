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
// Kernel: persistent, one CTA per SM, blocks b = blockIdx.x, +gridDim.x, ...
// for 96 <= n <= 128 (n % 4 == 0: one 128 x 128 tile per block, rows and
// columns beyond n read as zero or are not stored).  Warp roles:
//   warp 0      TMA: Sh and Sl once (resident, 128 KB), then the block's
//               four 32-column chunks of A into a 3-stage ring;
//   warp 1      one thread issues tcgen05.mma (kind::tf32, M = N = 128,
//               K = 8) into one of two TMEM accumulators (2 x 128 columns);
//   warps 2..5  split each landed chunk in place into Ah and Al;
//   warps 6..9  drain an accumulator with tcgen05.ld (one row per thread)
//               and write the block transposed: for each k the 32 lanes of a
//               warp store 32 consecutive j (coalesced), scaled, FP32 or FP64.
// Stage and accumulator hand-offs are mbarriers; every wait is bounded and
// reports PIT_E_TIMEOUT through the problem's error word.
#include <string.h>

#include <algorithm>
#include <vector>

#include "pit_internal.h"
#include "stencil_arith.cuh"
#include "tc_common.cuh"

namespace pit {
namespace {

constexpr int XT_T = 128;                              // tile rows (TMEM lanes) = columns
constexpr int XT_BK = 32;                              // K per chunk (128 bytes of FP32)
constexpr int XT_KCH = XT_T / XT_BK;                   // chunks per tile
constexpr int XT_STAGES = 3;
constexpr int XT_CH = XT_T * XT_BK * 4;                // 16 KB: one chunk of one operand part
constexpr int XT_S_BYTES = XT_KCH * XT_CH;             // 64 KB: one part of S
constexpr int XT_STAGE_BYTES = 2 * XT_CH;              // Ah (landed by TMA, split in place) + Al
constexpr int XT_BAR_OFF = 2 * XT_S_BYTES + XT_STAGES * XT_STAGE_BYTES;
constexpr int XT_SMEM = 1024 + XT_BAR_OFF + 128;       // alignment slack + ring + barriers
constexpr int XT_THREADS = 320;
constexpr int XT_CONV_THREADS = 128;
constexpr uint32_t kXtIdesc = tc_idesc_tf32(XT_T, XT_T);

__device__ __forceinline__ bool xt_live(const MemberState *st, int t, int nblk) {
    if (st == nullptr) return true;
    const MemberState &m = st[t / nblk];
    return m.active && !m.skip && !m.half;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
}

template <bool OUT64>
__global__ void __launch_bounds__(XT_THREADS, 1)
    k_xform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmSh,
               const __grid_constant__ CUtensorMap tmSl, void *out_raw, int n, int total, int nblk,
               float scale, const MemberState *st, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *Sh = base, *Sl = base + XT_S_BYTES;
    unsigned char *ring = base + 2 * XT_S_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + XT_BAR_OFF);
    uint64_t *full = bars;                       // chunk landed (TMA)
    uint64_t *conv = bars + XT_STAGES;           // chunk split (converters)
    uint64_t *empty = bars + 2 * XT_STAGES;      // chunk consumed (tensor core)
    uint64_t *tfull = bars + 3 * XT_STAGES;      // accumulator complete, 2 buffers
    uint64_t *tempty = tfull + 2;                // accumulator drained, 2 buffers
    uint64_t *sbar = tempty + 2;                 // S resident
    uint64_t *mdone = sbar + 1;                  // all products issued have finished
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XT_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], XT_CONV_THREADS);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(sbar, 1);
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2 * XT_T));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            mbar_expect_tx(sbar, 2 * XT_S_BYTES);
            for (int c = 0; c < XT_KCH; ++c) {
                tma_load_2d(Sh + c * XT_CH, &tmSh, c * XT_BK, 0, sbar);
                tma_load_2d(Sl + c * XT_CH, &tmSl, c * XT_BK, 0, sbar);
            }
            int last_use[XT_STAGES];
            for (int s = 0; s < XT_STAGES; ++s) last_use[s] = -1;
            int q = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                if (!xt_live(st, t, nblk)) continue;
                for (int c = 0; c < XT_KCH; ++c, ++q) {
                    const int s = q % XT_STAGES, u = q / XT_STAGES;
                    if (!tc_mbar_wait(&empty[s], (uint32_t)(u & 1) ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], XT_CH);
                    tma_load_2d(ring + s * XT_STAGE_BYTES, &tmA, c * XT_BK, t * n, &full[s]);
                    last_use[s] = u;
                }
            }
            // no copy of this CTA may still be writing shared memory at exit
            tc_mbar_drain(sbar, 0u);
            for (int s = 0; s < XT_STAGES; ++s)
                if (last_use[s] >= 0) tc_mbar_drain(&full[s], (uint32_t)(last_use[s] & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            bool ok = tc_mbar_wait(sbar, 0u, err);
            int q = 0, L = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                if (!xt_live(st, t, nblk)) continue;
                const int buf = L & 1, v = L >> 1;
                if (!tc_mbar_wait(&tempty[buf], (uint32_t)(v & 1) ^ 1u, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * XT_T);
                for (int c = 0; c < XT_KCH; ++c, ++q) {
                    const int s = q % XT_STAGES, u = q / XT_STAGES;
                    if (!tc_mbar_wait(&conv[s], (uint32_t)(u & 1), err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *stg = ring + s * XT_STAGE_BYTES;
                    const uint64_t ah = smem_desc(stg), al = smem_desc(stg + XT_CH);
                    const uint64_t bh = smem_desc(Sh + c * XT_CH), bl = smem_desc(Sl + c * XT_CH);
#pragma unroll
                    for (int j = 0; j < XT_BK / 8; ++j) {
                        const uint64_t adv = (uint64_t)(j * 32) >> 4;   // 8 TF32 = 32 bytes along K
                        tc_mma_tf32(d, ah + adv, bh + adv, kXtIdesc, (c > 0 || j > 0) ? 1u : 0u);
                        tc_mma_tf32(d, ah + adv, bl + adv, kXtIdesc, 1u);
                        tc_mma_tf32(d, al + adv, bh + adv, kXtIdesc, 1u);
                    }
                    mma_commit(&empty[s]);    // chunk free once these products finish
                }
                if (!ok) break;
                mma_commit(&tfull[buf]);      // accumulator complete
                ++L;
            }
            mma_commit(mdone);
            tc_mbar_drain(mdone, 0u);
        }
    } else if (warp < 6) {
        // ---- split: Ah = rna_tf32(a) in place, Al = rna_tf32(a - Ah)
        const int ct = threadIdx.x - 64;
        int q = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            if (!xt_live(st, t, nblk)) continue;
            for (int c = 0; c < XT_KCH; ++c, ++q) {
                const int s = q % XT_STAGES, u = q / XT_STAGES;
                if (!tc_mbar_wait(&full[s], (uint32_t)(u & 1), err)) {
                    ok = false;
                    break;
                }
                float4 *hi = reinterpret_cast<float4 *>(ring + s * XT_STAGE_BYTES);
                float4 *lo = reinterpret_cast<float4 *>(ring + s * XT_STAGE_BYTES + XT_CH);
#pragma unroll 4
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
    } else {
        // ---- epilogue: TMEM lanes 32 (warp % 4) .. +31 are the tile rows j
        const int quad = warp & 3;
        const int j = quad * 32 + lane;
        const size_t nn = (size_t)n * n;
        int L = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            if (!xt_live(st, t, nblk)) continue;
            const int buf = L & 1, v = L >> 1;
            const bool ok = __all_sync(0xffffffffu, tc_mbar_wait(&tfull[buf], (uint32_t)(v & 1), err) ? 1 : 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int cc = 0; cc < XT_T / 32; ++cc) {
                float vals[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * XT_T + cc * 32), vals);
                if (j < n) {
                    if constexpr (OUT64) {
                        double *ob = reinterpret_cast<double *>(out_raw) + (size_t)t * nn + j;
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int k = cc * 32 + i;
                            if (k < n) ob[(size_t)k * n] = f2d(scale * vals[i]);
                        }
                    } else {
                        float *ob = reinterpret_cast<float *>(out_raw) + (size_t)t * nn + j;
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int k = cc * 32 + i;
                            if (k < n) ob[(size_t)k * n] = scale * vals[i];
                        }
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * XT_T));
    }
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
    return p->nx >= 96 && p->nx <= XT_T && p->nx % 4 == 0 && tc_encode_fn() != nullptr;
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
    const int total = p->batch * (p->N + 1);
    const float *Sh = p->xtc_S.as<float>();
    CUtensorMap tA, tSh, tSl;
    PIT_TRY(tc_make_map(&tA, A, total * n, n, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSh, Sh, n, n, XT_BK, XT_T));
    PIT_TRY(tc_make_map(&tSl, Sh + (size_t)n * n, n, n, XT_BK, XT_T));
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(total, sms);
    if (out64) {
        PIT_CUDA(cudaFuncSetAttribute(k_xform_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, XT_SMEM));
        k_xform_tc<true><<<grid, XT_THREADS, XT_SMEM, s>>>(tA, tSh, tSl, out, n, total, p->N + 1,
                                                           (float)scale, st, p->errword.as<int>());
    } else {
        PIT_CUDA(cudaFuncSetAttribute(k_xform_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, XT_SMEM));
        k_xform_tc<false><<<grid, XT_THREADS, XT_SMEM, s>>>(tA, tSh, tSl, out, n, total, p->N + 1,
                                                            (float)scale, st, p->errword.as<int>());
    }
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

}  // namespace pit
