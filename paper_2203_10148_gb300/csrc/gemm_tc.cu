// Dense fine propagator on the 5th-generation tensor cores (tcgen05):
//   C[r][c] = sum_k X[r][k] Phi[c][k]      (r = member * (N+1) + slice, c = state index)
// i.e. C row r = Phi x_r, for all slices of all members at once, in split
// TF32 ("3xTF32"): X = Xh + Xl and Phi = Ph + Pl with each part a TF32
// value, and C = Xh Ph^T + Xh Pl^T + Xl Ph^T accumulated in FP32 (the Xl Pl^T
// term is below FP32 resolution).  The epilogue writes the block-operator
// rows of eq. (4): y_{n+1} = x_{n+1} - C[r] (or the residual form).
//
// Any M: the TF32 parts of X and Phi are stored with rows of Mp = M rounded
// up to 128 (zero columns, and for Phi zero rows, beyond M), K runs over Mp
// and the epilogue writes the first M columns only.
//
// The same kernel runs the split in BF16 ("3xBF16", kind::f16 with BF16 A
// and B): X = Xh + Xl and Phi = Ph + Pl with BF16 parts, the same three
// products, K in 64-element (128-byte) stages; about 2^-16 relative per
// product against about 2^-21 for split TF32, at twice the MMA rate and half
// the operand bytes.
//
// Kernel structure: 128 x 128 output tiles, K in 32-element (128-byte)
// stages through a 3-stage shared-memory ring filled by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) and drained by tcgen05.mma
// (kind::tf32, M = N = 128, K = 8 per instruction) issued by one thread; one
// persistent CTA per SM loops over the tiles with two FP32 accumulators in
// tensor memory (128 columns each), so four epilogue warps read one back
// with tcgen05.ld while the next tile's products fill the other.  mbarriers
// hand stages and accumulators between the TMA thread, the MMA thread, the
// tensor core and the epilogue; every wait is bounded and reports
// PIT_E_TIMEOUT through the problem's error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

#include "pit_internal.h"
#include "stencil_arith.cuh"
#include "tc_common.cuh"

namespace pit {
namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32, TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;                  // 16 KB per operand tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;                 // Ah, Al, Bh, Bl
// Instruction descriptors: D = F32, A = B = TF32 (or BF16), both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = tc_idesc_tf32(TC_BM, TC_BN);
constexpr uint32_t kIdescBf = tc_idesc_bf16(TC_BM, TC_BN);
constexpr int TC_BK_BF = 64;   // BF16 elements per 128-byte stage row

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
    tc_mma_tf32(tmem, a, b, kIdesc, accum);
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err) {
    return tc_mbar_wait(bar, parity, err);
}

pit_status make_map(CUtensorMap *tm, const void *ptr, int rows, int cols, bool bf16) {
    return tc_make_map(tm, ptr, rows, cols, bf16 ? TC_BK_BF : TC_BK, TC_BM, bf16);
}

struct TcEpilogue {
    const double *x;      // block vector (batch x (N+1) x M)
    double *y;            // FP64 rows (or null)
    float *y32;           // FP32 rows (or null): q = fl32(x_{n+1}) - C
    const double *y0;
    int N, M, batch, mode;   // M: columns written (the product runs over the padded width)
    size_t blen;
    const MemberState *st;
};

// Epilogue of one warp: the 32 tile rows m0 + row0 + lane (TMEM lanes of
// the warp's quarter, from column address `taddr`) times 128 columns from n0,
// 32 columns at a time (nchunks of them): tcgen05.ld gives a lane one row; the values go
// through the warp's padded shared-memory tile `stg` (32 x 33 floats) so
// that, row by row, the 32 lanes read x and write y as 32 consecutive
// columns (coalesced).
__device__ __forceinline__ void store_tile_rows(const TcEpilogue &ep, float *stg, uint32_t taddr,
                                                int m0, int row0, int n0, int R, int lane,
                                                int nchunks = TC_BN / 32) {
    // this lane's tile row (member, slice, liveness), broadcast row by row below
    const int nb1 = ep.N + 1;
    const int myrow = m0 + row0 + lane;
    const int myb = myrow / nb1, myn = myrow % nb1;
    const bool mylive = myrow < R && myn < ep.N &&
                        (ep.st == nullptr || (ep.st[myb].active && !ep.st[myb].skip && !ep.st[myb].half));
    const unsigned livemask = __ballot_sync(0xffffffffu, mylive);
    for (int cchunk = 0; cchunk < nchunks; ++cchunk) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(cchunk * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[i];
        __syncwarp();
        const int c = n0 + cchunk * 32 + lane;
        const bool col_ok = c < ep.M;
        // all x loads of the 32 rows first (independent, in flight together)
        double xn[32];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int b = __shfl_sync(0xffffffffu, myb, rr), n = __shfl_sync(0xffffffffu, myn, rr);
            const bool ok = ((livemask >> rr) & 1u) && col_ok;
            xn[rr] = ok ? ep.x[(size_t)b * ep.blen + (size_t)(n + 1) * ep.M + c] : 0.0;
        }
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int b = __shfl_sync(0xffffffffu, myb, rr), n = __shfl_sync(0xffffffffu, myn, rr);
            if (!((livemask >> rr) & 1u) || !col_ok) continue;
            const float cv = stg[rr * 33 + lane];
            const size_t mb = (size_t)b * ep.blen;
            if (ep.y32) {
                ep.y32[mb + (size_t)(n + 1) * ep.M + c] = d2f_rn(xn[rr]) - cv;
                if (n == 0) ep.y32[mb + c] = d2f_rn(ep.x[mb + c]);   // row 0 of eq. (4): x_0
            } else {
                const double f = f2d(cv);
                ep.y[mb + (size_t)(n + 1) * ep.M + c] = (ep.mode == FINE_APPLY) ? xn[rr] - f : f - xn[rr];
                if (n == 0) {
                    // row 0 of eq. (4): x_0 (or y0 - x_0)
                    const double x0 = ep.x[mb + c];
                    ep.y[mb + c] = (ep.mode == FINE_APPLY) ? x0 : ep.y0[(size_t)b * ep.M + c] - x0;
                }
            }
        }
        __syncwarp();
    }
}

// Persistent form: one CTA per SM loops over the output tiles (tile t =
// blockIdx.x, + gridDim.x, ...).  Warp 0 (one thread) streams the K stages
// of every tile through the 3-stage ring by TMA; warp 1 (one thread) issues
// the products into one of two tensor-memory accumulators (128 columns each)
// in turn; warps 2-9 drain the other accumulator through the epilogue (warp
// w reads the TMEM lanes of quarter w % 4, columns 0-63 for w < 6 and 64-127
// above), so a tile's stores overlap the next tile's products.  mbarriers: stage full / empty, accumulator full
// (the MMA commit) / empty (one arrival per epilogue warp).  Every wait is
// bounded; at exit the copies and products still in flight are drained.
constexpr int TP_EPI = 8;                                          // epilogue warps: 2 per TMEM quarter
constexpr int TP_THREADS = 64 + 32 * TP_EPI;
constexpr int TP_STG = TP_EPI * 32 * 33 * 4;                       // epilogue staging tiles
constexpr int TP_SMEM = TC_STAGES * TC_STAGE_BYTES + TP_STG + 1024 + 256;

template <bool BF>
__global__ void __launch_bounds__(TP_THREADS, 1)
    k_gemm_tf32x3_p(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                    int K, int R, int ntn, int ntiles, TcEpilogue ep, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *stg_all = reinterpret_cast<float *>(base + TC_STAGES * TC_STAGE_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + TC_STAGES * TC_STAGE_BYTES + TP_STG);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *accf = empty + TC_STAGES;     // [2] accumulator complete
    uint64_t *acce = accf + 2;              // [2] accumulator drained
    uint64_t *fin = acce + 2;               // the MMA thread's last products, at exit
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int BKE = BF ? TC_BK_BF : TC_BK;   // K elements per stage
    const int KB = K / BKE;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], TP_EPI);
        }
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2 * TC_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer over every tile's K stages
        int it = 0;
        int last_it[TC_STAGES];
#pragma unroll
        for (int s = 0; s < TC_STAGES; ++s) last_it[s] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = (tile / ntn) * TC_BM, n0 = (tile % ntn) * TC_BN;
            for (int kb = 0; kb < KB; ++kb, ++it) {
                const int s = it % TC_STAGES;
                const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, err)) {
                    ok = false;
                    break;
                }
                unsigned char *st = base + s * TC_STAGE_BYTES;
                mbar_expect_tx(&full[s], TC_STAGE_BYTES);
                tma_load_2d(st, &tmAh, kb * BKE, m0, &full[s]);
                tma_load_2d(st + TC_TILE_BYTES, &tmAl, kb * BKE, m0, &full[s]);
                tma_load_2d(st + 2 * TC_TILE_BYTES, &tmBh, kb * BKE, n0, &full[s]);
                tma_load_2d(st + 3 * TC_TILE_BYTES, &tmBl, kb * BKE, n0, &full[s]);
                last_it[s] = it;
            }
        }
        // no copy of this CTA may still be writing shared memory at exit
#pragma unroll
        for (int s = 0; s < TC_STAGES; ++s)
            if (last_it[s] >= 0) tc_mbar_drain(&full[s], (uint32_t)(last_it[s] / TC_STAGES) & 1u);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: three products per K step into accumulator b = tile count % 2
        int it = 0, tc = 0;
        bool ok = true, issued = false;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tc) {
            const int b = tc & 1;
            const uint32_t use = (uint32_t)(tc >> 1);
            if (!mbar_wait(&acce[b], (use & 1u) ^ 1u, err)) break;   // the epilogue drained b
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(b * TC_BN);
            for (int kb = 0; kb < KB; ++kb, ++it) {
                const int s = it % TC_STAGES;
                const uint32_t ph = (uint32_t)(it / TC_STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char *st = base + s * TC_STAGE_BYTES;
                const uint64_t ah = smem_desc(st), al = smem_desc(st + TC_TILE_BYTES);
                const uint64_t bh = smem_desc(st + 2 * TC_TILE_BYTES), bl = smem_desc(st + 3 * TC_TILE_BYTES);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t adv = (uint64_t)(j * 32) >> 4;   // 32 bytes along K
                    if constexpr (BF) {
                        tc_mma_f16(acc, ah + adv, bh + adv, kIdescBf, (kb > 0 || j > 0) ? 1u : 0u);
                        tc_mma_f16(acc, ah + adv, bl + adv, kIdescBf, 1u);
                        tc_mma_f16(acc, al + adv, bh + adv, kIdescBf, 1u);
                    } else {
                        mma_tf32(acc, ah + adv, bh + adv, (kb > 0 || j > 0) ? 1u : 0u);
                        mma_tf32(acc, ah + adv, bl + adv, 1u);
                        mma_tf32(acc, al + adv, bh + adv, 1u);
                    }
                }
                issued = true;
                mma_commit(&empty[s]);          // the stage is free once these products finish
            }
            if (!ok) break;
            mma_commit(&accf[b]);               // accumulator b complete
        }
        if (issued) {
            // every product of this CTA done before the accumulators are freed
            mma_commit(fin);
            tc_mbar_drain(fin, 0u);
        }
    } else if (warp >= 2) {
        // epilogue warps: quarter q of the tile rows, half h of its columns
        const int q = warp & 3, h = (warp - 2) >> 2;
        float *stg = stg_all + (warp - 2) * 32 * 33;
        int tc = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tc) {
            const int b = tc & 1;
            const uint32_t use = (uint32_t)(tc >> 1);
            const bool have = __all_sync(0xffffffffu, mbar_wait(&accf[b], use & 1u, err) ? 1 : 0) != 0;
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / ntn) * TC_BM, n0 = (tile % ntn) * TC_BN;
            store_tile_rows(ep, stg,
                            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TC_BN + h * (TC_BN / 2)),
                            m0, q * 32, n0 + h * (TC_BN / 2), R, lane, TC_BN / 64);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN));
    }
}

// hi = TF32 rounding of fl32(x), lo = TF32 rounding of the FP32 remainder,
// for an rows_out x Mp array from the rows_src x M row-major x (zero where
// r >= rows_src or c >= M).
__global__ void k_split_tf32(const double *x, float *hi, float *lo, int rows_src, int rows_out, int M,
                             int Mp) {
    const size_t n = (size_t)rows_out * Mp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Mp, col = i % Mp;
        const float v = (row < (size_t)rows_src && col < (size_t)M) ? d2f_rn(x[row * M + col]) : 0.f;
        uint32_t h, l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
        const float r = v - __uint_as_float(h);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
        hi[i] = __uint_as_float(h);
        lo[i] = __uint_as_float(l);
    }
}

// hi = BF16 rounding of fl32(x), lo = BF16 rounding of the FP32 remainder,
// padded like k_split_tf32.
__global__ void k_split_bf16(const double *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int rows_src,
                             int rows_out, int M, int Mp) {
    const size_t n = (size_t)rows_out * Mp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / Mp, col = i % Mp;
        const float v = (row < (size_t)rows_src && col < (size_t)M) ? d2f_rn(x[row * M + col]) : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = h;
        lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

}  // namespace

static int padded(int M) { return (M + TC_BN - 1) / TC_BN * TC_BN; }

pit_status tc_split_tf32(const double *x, float *hi, float *lo, int rows_src, int rows_out, int M,
                         int Mp, cudaStream_t s) {
    k_split_tf32<<<1024, 256, 0, s>>>(x, hi, lo, rows_src, rows_out, M, Mp);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

bool dense_tc_supported(const Problem *p) {
    (void)p;   // any M (padded to 128 columns); needs the tensor-map encoder
    return tc_encode_fn() != nullptr;
}

pit_status dense_tc_split_phi(Problem *p) {
    const int Mp = padded(p->M);
    const size_t mm2 = (size_t)Mp * Mp;
    PIT_TRY(p->PhiTh.ensure(mm2 * sizeof(float)));
    PIT_TRY(p->PhiTl.ensure(mm2 * sizeof(float)));
    k_split_tf32<<<1024, 256, 0, p->stream>>>(p->PhiF64.as<double>(), p->PhiTh.as<float>(),
                                              p->PhiTl.as<float>(), p->M, Mp, p->M, Mp);
    PIT_LAUNCH_CHECK();
    if (p->dense_bf16) {
        PIT_TRY(p->PhiBh.ensure(mm2 * sizeof(__nv_bfloat16)));
        PIT_TRY(p->PhiBl.ensure(mm2 * sizeof(__nv_bfloat16)));
        k_split_bf16<<<1024, 256, 0, p->stream>>>(p->PhiF64.as<double>(), p->PhiBh.as<__nv_bfloat16>(),
                                                  p->PhiBl.as<__nv_bfloat16>(), p->M, Mp, p->M, Mp);
        PIT_LAUNCH_CHECK();
    }
    return PIT_OK;
}

// Block-operator rows of the dense fine batch on the tensor cores: y (FP64)
// or y32 (FP32 rows for the mixed sweep); split BF16 when the problem was
// created with PIT_MIXED_BF16, split TF32 otherwise.
pit_status dense_tc_apply(Problem *p, const double *x, double *y, float *y32, int mode,
                          const MemberState *st, cudaStream_t s) {
    const int M = p->M, Mp = padded(M);
    const int R = p->batch * (p->N + 1);
    const size_t n = (size_t)R * Mp;
    const bool bf = p->dense_bf16;
    const unsigned sgrid = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    CUtensorMap tAh, tAl, tBh, tBl;
    if (bf) {
        PIT_TRY(p->tc_split.ensure(2 * n * sizeof(__nv_bfloat16)));
        __nv_bfloat16 *xh = p->tc_split.as<__nv_bfloat16>(), *xl = xh + n;
        k_split_bf16<<<sgrid, 256, 0, s>>>(x, xh, xl, R, R, M, Mp);
        PIT_LAUNCH_CHECK();
        PIT_TRY(make_map(&tAh, xh, R, Mp, true));
        PIT_TRY(make_map(&tAl, xl, R, Mp, true));
        PIT_TRY(make_map(&tBh, p->PhiBh.ptr, Mp, Mp, true));
        PIT_TRY(make_map(&tBl, p->PhiBl.ptr, Mp, Mp, true));
    } else {
        PIT_TRY(p->tc_split.ensure(2 * n * sizeof(float)));
        float *xh = p->tc_split.as<float>(), *xl = xh + n;
        k_split_tf32<<<sgrid, 256, 0, s>>>(x, xh, xl, R, R, M, Mp);
        PIT_LAUNCH_CHECK();
        PIT_TRY(make_map(&tAh, xh, R, Mp, false));
        PIT_TRY(make_map(&tAl, xl, R, Mp, false));
        PIT_TRY(make_map(&tBh, p->PhiTh.as<float>(), Mp, Mp, false));
        PIT_TRY(make_map(&tBl, p->PhiTl.as<float>(), Mp, Mp, false));
    }
    TcEpilogue ep{x, y, y32, p->y0.as<double>(), p->N, M, p->batch, mode, p->blen, st};
    // persistent: one CTA per SM over all output tiles
    const int ntn = Mp / TC_BN, ntiles = (R + TC_BM - 1) / TC_BM * ntn;
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kern = bf ? k_gemm_tf32x3_p<true> : k_gemm_tf32x3_p<false>;
    PIT_TRY(smem_limit(kern, TP_SMEM));
    kern<<<std::min(ntiles, sms), TP_THREADS, TP_SMEM, s>>>(tAh, tAl, tBh, tBl, Mp, R, ntn, ntiles, ep,
                                                           p->errword.as<int>());
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

}  // namespace pit
