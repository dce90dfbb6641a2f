// Dense true residual on the tensor cores by error-free splitting.
//
// The product C[g][c] = sum_k X[g][k] Phi[c][k] (row g = member * (N+1) +
// slice of the block vector, c = state index: C row g = Phi x_g) in the
// accuracy class of the float-float product, from BF16 products with FP32
// accumulation: the error-free splitting of Ozaki, Ogita, Oishi and Rump
// ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012), which Mukunoki, Ozaki, Ogita and Imamura ran on
// tensor cores with FP32 accumulation ("DGEMM using Tensor Cores, and Its
// Accurate and Reproducible Versions", ISC 2020).
//
// Splitting: every row g of X is written 2^E_g sum_{i=1..S} d_gi 2^(-i b)
// with 2^E_g above the row's largest magnitude and balanced integer digits
// (|d_1| <= 2^b, |d_i| <= 2^(b-1) for i > 1), taken from the value as a
// 62-bit fixed-point integer; the part below the S-th digit is dropped
// (at most 2^(E_g - S b - 1) per entry).  Phi's rows likewise with F_c.
// Slice i holds d_i 2^(-i b), a BF16 value exactly.
//
// Exactness: the products of slices i and j are integer multiples of
// 2^(-(i+j) b); over one anti-diagonal s = i + j and k < K their absolute
// sum is at most K 2^(2b - 2) max(s + 1, 4) such units (the two end pairs
// with the leading digit and s - 3 inner pairs; for s = 2 the one pair of
// leading digits), so with b = 6, K <= 1024 and the diagonals formed
// (s <= 8) it stays below 2^24 units: the tensor core's FP32 accumulation of
// a whole diagonal (every pair, every K step) is exact, whatever order it
// adds in.
// The S diagonal sums (s = 2 .. S + 1) are added in float-float, scaled by
// 2^(E_g + F_c) and written as FP64 block-operator rows of eq. (4).  Pairs
// beyond the last diagonal are not formed; with S = 7 the result is within
// about 2^-42 of K max_k |x_gk| max_k |phi_ck| (the rows' maxima).
//
// Kernel: persistent, one CTA per SM over 128 x 64 output tiles.  For slice
// i of X, each 64-wide K stage brings X_i's tile and the tiles of the S - i
// slices of Phi it pairs with (TMA, 128-byte swizzle), so an X tile is read
// once for all its pairs; one thread issues tcgen05.mma (kind::f16, BF16, M
// = 128, N = 64, K = 16) into the S diagonal accumulators in tensor memory
// (S x 64 columns); four epilogue warps add them in float-float, release
// tensor memory, then write the tile's rows in FP64 while the next tile's
// products run.  Every wait is bounded and reports PIT_E_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "pit_internal.h"
#include "stencil_arith.cuh"
#include "tc_common.cuh"

namespace pit {
namespace {

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64;     // tile rows, tile columns, BF16 K per stage
constexpr int OZ_SMAX = 7;                              // slices per operand
constexpr int OZ_BETA = 6;                              // bits per digit
constexpr int OZ_KMAX = 1024;                           // K for which every diagonal sum is exact
constexpr int OZ_STAGES = 2;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;           // 16 KB
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;           // 8 KB
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_SMAX * OZ_B_BYTES;   // 72 KB
constexpr int OZ_EPI = 4;                               // epilogue warps: one per TMEM lane quarter
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI;
constexpr int OZ_STG = OZ_EPI * 32 * 33 * 8;            // per-warp staging tiles (float2)
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + OZ_STG + 1024 + 256;
constexpr int OZ_TMEM_COLS = 512;                       // S x 64 accumulator columns, rounded up

// Digits of the rows of a rows_src x M row-major FP64 matrix (rows_out x Kp
// outputs, zero beyond rows_src / M): slices[i][g][k] = d_(i+1) 2^(-(i+1) b)
// as BF16 and expo[g] = E_g.  One warp per row.  Rows whose largest
// magnitude is zero or subnormal get E = 0 and zero digits (and so do
// subnormal entries of other rows).
__global__ void k_oz_split(const double *__restrict__ x, int rows_src, int rows_out, int M, int Kp,
                           int S, __nv_bfloat16 *__restrict__ slices, int *__restrict__ expo) {
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= rows_out) return;
    const bool row_ok = g < rows_src;
    const double *xr = x + (size_t)(row_ok ? g : 0) * M;
    // the row's largest magnitude: the bit patterns of |x| order like the values
    unsigned long long mx = 0;
    for (int k = lane; k < M; k += 32) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(row_ok ? xr[k] : 0.0) &
                                     0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    const int efield = (int)(mx >> 52);
    const int E = efield == 0 ? 0 : efield - 1023 + 1;   // |x| < 2^E over the row
    if (lane == 0) expo[g] = E;
    const size_t plane = (size_t)rows_out * Kp;
    __nv_bfloat16 *out = slices + (size_t)g * Kp;
    for (int k = lane; k < Kp; k += 32) {
        long long V = 0;
        if (row_ok && k < M && efield != 0) {
            const long long bits = __double_as_longlong(xr[k]);
            const int ef = (int)((bits >> 52) & 0x7ff);
            if (ef != 0) {
                const long long m = (bits & 0xfffffffffffffll) | 0x10000000000000ll;
                // x / 2^E = m 2^(ef - 1023 - 52 - E), as an integer over 2^62
                const int sh = ef - 1023 - 52 + 62 - E;          // <= 9
                const long long mag = sh >= 0 ? (m << sh) : (sh > -63 ? (m >> -sh) : 0ll);
                V = bits < 0 ? -mag : mag;
            }
        }
        long long r = V;
        float unit = 1.f;
        for (int i = 1; i <= S; ++i) {
            const int sh = 62 - i * OZ_BETA;
            const long long d = (r + (1ll << (sh - 1))) >> sh;   // round half up: balanced digit
            r -= d << sh;
            unit *= 1.f / (float)(1 << OZ_BETA);
            out[(size_t)(i - 1) * plane + k] = __float2bfloat16_rn((float)d * unit);
        }
    }
}

struct OzEpilogue {
    const double *x;      // block vector (batch x (N+1) x M)
    double *y;            // FP64 block-operator rows
    const double *y0;
    const int *ex, *ephi; // row exponents of X and of Phi
    int N, M, batch, mode;
    size_t blen;
    const MemberState *st;
};

// v * 2^k exactly (exponent arithmetic; ldexp where the result leaves the normal range)
__device__ __forceinline__ double oz_scale(double v, int k) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (v == 0.0 || e == 0 || e + k <= 0 || e + k >= 2047) return ldexp(v, k);
    return __longlong_as_double(b + ((long long)k << 52));
}

// Warps: 0 = TMA (one thread), 1 = MMA issue (one thread), 2-5 = epilogue
// (warp w reads the tensor-memory lanes of quarter w % 4).  Stage layout:
// X_i's tile, then Phi_0 .. Phi_(S-1-i)'s tiles.  mbarriers: stage full /
// empty, accumulators full (the MMA commit) / empty (one arrival per
// epilogue warp), and a final commit drained before exit.
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_gemm_oz(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int Kp,
              int R, int Rp, int Mp, int S, int ntn, int ntiles, OzEpilogue ep, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *stg_all = reinterpret_cast<float2 *>(base + OZ_STAGES * OZ_STAGE_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + OZ_STAGES * OZ_STAGE_BYTES + OZ_STG);
    uint64_t *empty = full + OZ_STAGES;
    uint64_t *accf = empty + OZ_STAGES;
    uint64_t *acce = accf + 1;
    uint64_t *fin = acce + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KB = Kp / OZ_BK;
    constexpr uint32_t idesc = tc_idesc_bf16(OZ_BM, OZ_BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, OZ_EPI);
        mbar_init(fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(OZ_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: per tile, per slice i of X, per K stage
        int it = 0;
        int last_it[OZ_STAGES];
#pragma unroll
        for (int s = 0; s < OZ_STAGES; ++s) last_it[s] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = (tile / ntn) * OZ_BM, n0 = (tile % ntn) * OZ_BN;
            for (int i = 0; i < S && ok; ++i) {
                const int nb = S - i;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % OZ_STAGES;
                    const uint32_t ph = (uint32_t)(it / OZ_STAGES) & 1u;
                    if (!tc_mbar_wait(&empty[s], ph ^ 1u, err)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = base + s * OZ_STAGE_BYTES;
                    mbar_expect_tx(&full[s], (uint32_t)(OZ_A_BYTES + nb * OZ_B_BYTES));
                    tma_load_2d(st, &tmA, kb * OZ_BK, i * Rp + m0, &full[s]);
                    for (int j = 0; j < nb; ++j)
                        tma_load_2d(st + OZ_A_BYTES + j * OZ_B_BYTES, &tmB, kb * OZ_BK, j * Mp + n0, &full[s]);
                    last_it[s] = it;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < OZ_STAGES; ++s)
            if (last_it[s] >= 0) tc_mbar_drain(&full[s], (uint32_t)(last_it[s] / OZ_STAGES) & 1u);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: pair (i, j) accumulates into diagonal i + j (columns (i + j) x 64);
        // the i = 0 pairs come first and start every diagonal
        int it = 0, tc = 0;
        bool ok = true, issued = false;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tc) {
            if (!tc_mbar_wait(acce, ((uint32_t)tc & 1u) ^ 1u, err)) break;   // the epilogue drained them
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int i = 0; i < S && ok; ++i) {
                const int nb = S - i;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % OZ_STAGES;
                    const uint32_t ph = (uint32_t)(it / OZ_STAGES) & 1u;
                    if (!tc_mbar_wait(&full[s], ph, err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *st = base + s * OZ_STAGE_BYTES;
                    const uint64_t ad = smem_desc(st);
#pragma unroll
                    for (int sub = 0; sub < OZ_BK / 16; ++sub) {
                        const uint64_t adv = (uint64_t)(sub * 32) >> 4;   // 32 bytes along K
                        const uint32_t acc_flag = (kb > 0 || sub > 0 || i > 0) ? 1u : 0u;
                        for (int j = 0; j < nb; ++j) {
                            const uint64_t bd = smem_desc(st + OZ_A_BYTES + j * OZ_B_BYTES);
                            tc_mma_f16(tmem + (uint32_t)((i + j) * OZ_BN), ad + adv, bd + adv, idesc, acc_flag);
                        }
                    }
                    issued = true;
                    mma_commit(&empty[s]);
                }
            }
            if (!ok) break;
            mma_commit(accf);
        }
        if (issued) {
            mma_commit(fin);
            tc_mbar_drain(fin, 0u);
        }
    } else if (warp >= 2) {
        const int q = warp & 3;
        float2 *stg = stg_all + (warp - 2) * 32 * 33;
        const int nb1 = ep.N + 1;
        int tc = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tc) {
            const bool have = __all_sync(0xffffffffu, tc_mbar_wait(accf, (uint32_t)tc & 1u, err) ? 1 : 0) != 0;
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / ntn) * OZ_BM, n0 = (tile % ntn) * OZ_BN;
            // the S diagonal sums of this lane's row, smallest first, into float-float
            float hs[OZ_BN], ls[OZ_BN];
#pragma unroll
            for (int c = 0; c < OZ_BN; ++c) {
                hs[c] = 0.f;
                ls[c] = 0.f;
            }
            for (int d = S - 1; d >= 0; --d) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * OZ_BN + half * 32), v);
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const ff sum = two_sum(hs[half * 32 + t], v[t]);
                        hs[half * 32 + t] = sum.hi;
                        ls[half * 32 + t] += sum.lo;
                    }
                }
            }
            // tensor memory free for the next tile's products
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce);
            // rows m0 + q * 32 + lane: member, slice, liveness, exponent
            const int myrow = m0 + q * 32 + lane;
            const int myb = myrow / nb1, myn = myrow % nb1;
            const bool mylive = myrow < R && myn < ep.N &&
                                (ep.st == nullptr ||
                                 (ep.st[myb].active && !ep.st[myb].skip && !ep.st[myb].half));
            const unsigned livemask = __ballot_sync(0xffffffffu, mylive);
            const int myE = mylive ? ep.ex[myrow] : 0;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int t = 0; t < 32; ++t) stg[lane * 33 + t] = make_float2(hs[half * 32 + t], ls[half * 32 + t]);
                __syncwarp();
                const int c = n0 + half * 32 + lane;
                const bool col_ok = c < ep.M;
                const int F = col_ok ? ep.ephi[c] : 0;
                for (int rr = 0; rr < 32; ++rr) {
                    const int b = __shfl_sync(0xffffffffu, myb, rr), n = __shfl_sync(0xffffffffu, myn, rr);
                    const int E = __shfl_sync(0xffffffffu, myE, rr);
                    if (!((livemask >> rr) & 1u) || !col_ok) continue;
                    const float2 hl = stg[rr * 33 + lane];
                    const double C = oz_scale(f2d(hl.x) + f2d(hl.y), E + F);
                    const size_t mb = (size_t)b * ep.blen;
                    const double xn = ep.x[mb + (size_t)(n + 1) * ep.M + c];
                    ep.y[mb + (size_t)(n + 1) * ep.M + c] = (ep.mode == FINE_APPLY) ? xn - C : C - xn;
                    if (n == 0) {
                        // row 0 of eq. (4): x_0 (or y0 - x_0)
                        const double x0 = ep.x[mb + c];
                        ep.y[mb + c] = (ep.mode == FINE_APPLY) ? x0 : ep.y0[(size_t)b * ep.M + c] - x0;
                    }
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
    }
}

int oz_pad(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

bool dense_oz_supported(const Problem *p) {
    return oz_pad(p->M, 128) <= OZ_KMAX && tc_encode_fn() != nullptr;
}

// Slices and row exponents of Phi (once per problem).
pit_status dense_oz_setup(Problem *p) {
    const int M = p->M, Kp = oz_pad(M, 128), Mp = Kp;
    PIT_TRY(p->oz_phi.ensure((size_t)OZ_SMAX * Mp * Kp * sizeof(__nv_bfloat16)));
    PIT_TRY(p->oz_ephi.ensure((size_t)Mp * sizeof(int)));
    k_oz_split<<<(Mp + 7) / 8, 256, 0, p->stream>>>(p->PhiF64.as<double>(), M, Mp, M, Kp, OZ_SMAX,
                                                    p->oz_phi.as<__nv_bfloat16>(), p->oz_ephi.as<int>());
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

// Block-operator rows (FINE_APPLY: x_{n+1} - Phi x_n; FINE_RESIDUAL: the
// negation; row 0 as eq. (4)) with the product by error-free splitting.
pit_status dense_oz_apply(Problem *p, const double *x, double *y, int mode, const MemberState *st,
                          cudaStream_t s) {
    const int M = p->M, Kp = oz_pad(M, 128), Mp = Kp;
    const int Rall = p->batch * (p->N + 1);
    const int R = Rall - 1;                  // the last member's row N is no product's input
    const int Rp = oz_pad(Rall, OZ_BM);
    PIT_TRY(p->oz_x.ensure((size_t)OZ_SMAX * Rp * Kp * sizeof(__nv_bfloat16)));
    PIT_TRY(p->oz_ex.ensure((size_t)Rp * sizeof(int)));
    k_oz_split<<<(Rp + 7) / 8, 256, 0, s>>>(x, Rall, Rp, M, Kp, OZ_SMAX, p->oz_x.as<__nv_bfloat16>(),
                                            p->oz_ex.as<int>());
    PIT_LAUNCH_CHECK();
    CUtensorMap tA, tB;
    PIT_TRY(tc_make_map(&tA, p->oz_x.ptr, OZ_SMAX * Rp, Kp, OZ_BK, OZ_BM, true));
    PIT_TRY(tc_make_map(&tB, p->oz_phi.ptr, OZ_SMAX * Mp, Kp, OZ_BK, OZ_BN, true));
    OzEpilogue ep{x, y, p->y0.as<double>(), p->oz_ex.as<int>(), p->oz_ephi.as<int>(), p->N, M, p->batch, mode,
                  p->blen, st};
    const int ntn = Mp / OZ_BN, ntiles = (R + OZ_BM - 1) / OZ_BM * ntn;
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PIT_TRY(smem_limit(k_gemm_oz, OZ_SMEM));
    k_gemm_oz<<<std::min(ntiles, sms), OZ_THREADS, OZ_SMEM, s>>>(tA, tB, Kp, R, Rp, Mp, OZ_SMAX, ntn, ntiles, ep,
                                                              p->errword.as<int>());
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

}  // namespace pit
