// Coarse sweep of the dense mode on the tensor cores: z_0 = q_0,
// z_n = q_n + G z_{n-1} (eq. (7) with a dense coarse propagator G), for one
// member, as a chunked scan whose every dependent step is one product of a
// matrix with all chunk states at once:
//
//   phase 1  the N + 1 slices in C <= 128 chunks of L: each chunk's local
//            recurrence from zero, w_{c,i} = q_{cL+i} + G w_{c,i-1} (L steps);
//   phase 2  the carries E_c = z_{cL-1} = u_c + A E_{c-1} with A = G^L and
//            u_c = w_{c-1,L-1} (u_0 = 0): a doubling scan, V_c <- V_c +
//            A^(2^s) V_{c-2^s} for s = 0 .. S-1, 2^S >= C (S steps, the
//            powers formed at set-up);
//   phase 3  every chunk again from its carry, z_{cL+i} = q_{cL+i} + G
//            z_{cL+i-1} with z_{cL-1} = E_c, storing z (L steps).
//
// One persistent cooperative launch runs all 2L + S steps.  The CTAs form
// clusters of 8: cluster j owns state rows 80j .. 80j+79, and its CTAs split
// K (the M columns of the matrix) in eight (80-row blocks: at M = 1024, 13
// clusters, where this part keeps at most 15 clusters of 8 CTAs with about
// 200 KB of shared memory each resident).  A step: TMA loads the split
// TF32 parts (hi, lo) of the chunk states (the A operand, 128 rows = chunk
// columns, K-major, 128-byte swizzle; a row shift of -2^s reads zeros above
// the first chunk) and, when the step's matrix is not the one already in
// shared memory, of the matrix rows (the B operand; G stays for the 2L
// steps that use it); one thread issues the 3xTF32 tcgen05.mma products
// (M = 128, N = 80, K = 8) into a tensor-memory accumulator stage by stage as
// the copies land; the eight warps move it to shared memory, the cluster
// sums its eight partial tiles through distributed shared memory in a fixed
// order (each CTA 16 chunk columns), adds the step's term, writes the next
// chunk states (split again) and, in phase 3, z; a bounded grid barrier
// ends the step.  Every wait is bounded; the CTAs of a cluster post their
// status before each cluster barrier and leave together.  Arithmetic: split
// TF32 products (about 2^-21 relative per product) accumulated in FP32, FP32
// sums: an FP32-class sweep, like the CUDA-core one it replaces (the sweep
// only preconditions).
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "pit_internal.h"
#include "stencil_arith.cuh"
#include "tc_common.cuh"

namespace pit {
namespace {

namespace cg = cooperative_groups;

constexpr int DS_BM = 128;                         // MMA M: chunk columns
constexpr int DS_BN = 80;                          // MMA N: state rows per cluster
constexpr int DS_TMEM = 128;                       // tensor-memory columns allocated (power of 2)
constexpr int DS_BK = 32;                          // K per stage (128 bytes of FP32)
constexpr int DS_CL = 8;                           // CTAs per cluster (K splits)
constexpr int DS_THREADS = 256;                    // 8 warps: two per 32-lane quarter of TMEM
constexpr int DS_A_BYTES = DS_BM * DS_BK * 4;      // 16 KB per part
constexpr int DS_B_BYTES = DS_BN * DS_BK * 4;      // 10 KB per part (1024-byte multiple)
constexpr int DS_PLD = DS_BN + 1;                  // padded row of the partial tile
constexpr int DS_COLS = DS_BM / DS_CL;             // chunk columns reduced per CTA
constexpr int DS_KBMAX = 1024 / DS_CL / DS_BK;     // K stages per CTA, at most (M <= 1024)
constexpr long long DS_SPIN = 1LL << 24;           // polls of the grid barrier
constexpr uint32_t kIdescDs = tc_idesc_tf32(DS_BM, DS_BN);

struct DsMaps {
    CUtensorMap ph[2], pl[2];                      // chunk states, ping-pong (hi, lo)
    CUtensorMap gh, gl;                            // G
    CUtensorMap ah[DTC_SMAX], al[DTC_SMAX];        // G^(L 2^s)
};

struct DsArgs {
    const double *q;
    double *z;
    int M, Mp, N, L, C, S;
    float *ph[2], *pl[2];   // the arrays behind the maps: DS_BM rows of Mp
    float *vf[2];           // FP32 carries of the doubling scan, DS_BM rows of Mp
    unsigned *bar;          // [0] arrivals at the grid barrier, all barriers counted
    int *err;
    const MemberState *st;
};

__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    const float r = v - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    hi = __uint_as_float(h);
    lo = __uint_as_float(l);
}

// Grid-wide barrier with a bounded wait: every CTA adds one to a counter
// that only grows (a release reduction, no reply awaited) and polls it with
// acquire loads until it holds every CTA's arrivals so far (`target`, the
// barrier's number times the grid size); false when the wait gave up or
// another CTA reported an error.  The caller does not leave on a false
// return at once: the CTAs of a cluster share their status at the next
// step's cluster barrier and leave together.
__device__ bool ds_grid_barrier(unsigned *bar, int *err, unsigned target) {
    __shared__ int res;
    __syncthreads();
    if (threadIdx.x == 0) {
        res = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long long spins = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if (++spins > DS_SPIN || ((spins & 63) == 0 && *(volatile int *)err)) {
                atomicExch(err, PIT_E_TIMEOUT);
                res = 0;
                break;
            }
        }
    }
    __syncthreads();
    return res != 0;
}

enum DsKind { DS_LOCAL = 0, DS_LOCAL_LAST = 1, DS_SCAN = 2, DS_FINAL = 3 };

__global__ void __launch_bounds__(DS_THREADS, 1)
    k_dense_sweep_tc(const __grid_constant__ DsMaps mp, DsArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int Kc = a.Mp / DS_CL, KB = Kc / DS_BK;
    // the matrix parts of all K stages (kept while consecutive steps use the
    // same matrix), then the chunk-state parts; the partial tile aliases the
    // latter once the products are done
    unsigned char *bsm = base;
    unsigned char *asm_ = base + (size_t)KB * 2 * DS_B_BYTES;
    float *part = reinterpret_cast<float *>(asm_);
    __shared__ uint64_t full_bar[DS_KBMAX], acc_bar;   // a K stage landed; the products are done
    __shared__ uint32_t tmem_slot;
    __shared__ int okflag[2]; // this CTA's status, posted for the cluster (by step parity)
    cg::cluster_group cluster = cg::this_cluster();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cluster.block_rank();
    const int n0 = (blockIdx.x / DS_CL) * DS_BN;
    const int k0 = rank * Kc;
    const unsigned nblocks = gridDim.x;
    // one member: every CTA takes the same decision
    if (!(a.st == nullptr || (a.st[0].active && !a.st[0].skip && !a.st[0].half))) return;

    if (threadIdx.x == 0) {
        for (int kb = 0; kb < DS_KBMAX; ++kb) mbar_init(&full_bar[kb], 1);
        mbar_init(&acc_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(DS_TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    uint32_t uses = 0;        // completed phases of full_bar and acc_bar
    bool local_ok = true;     // this CTA's waits all ended in time
    int nstep = 0;
    unsigned nbar = 0;        // grid barriers passed
    int resident = -1;        // matrix in bsm: 0 = G, 1 + s = G^(L 2^s), -1 none
    bool loads_out = false;   // a TMA copy of this CTA may be in flight (thread 0)

    // One step: out[c][n] = add(c, n) + sum_k Mat[n][k] in[c - shift][k] for
    // this cluster's rows n and this CTA's 16 chunk columns c.
    auto step = [&](bool has_in, int cur, int shift, const CUtensorMap *mh, const CUtensorMap *ml,
                    int mat, int kind, int i) -> bool {
        if (has_in && local_ok) {
            const uint32_t par = uses & 1u;
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                const bool loadb = mat != resident;
                for (int kb = 0; kb < KB; ++kb) {
                    const int x = k0 + kb * DS_BK;
                    uint64_t *fb = &full_bar[kb];
                    mbar_expect_tx(fb, (uint32_t)(2 * DS_A_BYTES + (loadb ? 2 * DS_B_BYTES : 0)));
                    unsigned char *sa = asm_ + kb * 2 * DS_A_BYTES;
                    tma_load_2d(sa, &mp.ph[cur], x, -shift, fb);
                    tma_load_2d(sa + DS_A_BYTES, &mp.pl[cur], x, -shift, fb);
                    if (loadb) {
                        unsigned char *sb = bsm + kb * 2 * DS_B_BYTES;
                        tma_load_2d(sb, mh, x, n0, fb);
                        tma_load_2d(sb + DS_B_BYTES, ml, x, n0, fb);
                    }
                }
                loads_out = true;
            }
            if (threadIdx.x == 32) {
                // stage by stage as the copies land; a wait that gives up sets
                // the error word and the cluster stops at the step's barrier
                for (int kb = 0; kb < KB; ++kb) {
                    if (!tc_mbar_wait(&full_bar[kb], par, a.err)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *sa = asm_ + kb * 2 * DS_A_BYTES;
                    unsigned char *sb = bsm + kb * 2 * DS_B_BYTES;
                    const uint64_t ah = smem_desc(sa), al = smem_desc(sa + DS_A_BYTES);
                    const uint64_t bh = smem_desc(sb), bl = smem_desc(sb + DS_B_BYTES);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint64_t adv = (uint64_t)(j * 32) >> 4;   // 8 TF32 along K
                        tc_mma_tf32(tmem, ah + adv, bh + adv, kIdescDs, (kb > 0 || j > 0) ? 1u : 0u);
                        tc_mma_tf32(tmem, ah + adv, bl + adv, kIdescDs, 1u);
                        tc_mma_tf32(tmem, al + adv, bh + adv, kIdescDs, 1u);
                    }
                }
                mma_commit(&acc_bar);   // arrives once the products issued above are done
            }
            __syncwarp();
            const bool have = __all_sync(0xffffffffu, tc_mbar_wait(&acc_bar, par, a.err) ? 1 : 0) != 0;
            if (!have) local_ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (threadIdx.x == 0 && have) loads_out = false;   // the products consumed every copy
            resident = have ? mat : -1;
            if (have) {
                // warp w reads TMEM lanes 32 (w % 4) .. + 31 (chunk columns);
                // warps 0-3 take columns 0-31 and 64-79, warps 4-7 columns 32-63
                const int q4 = warp & 3;
                for (int cc = warp >> 2; cc < (DS_BN + 31) / 32; cc += 2) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cc * 32), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (cc * 32 + j < DS_BN) part[(q4 * 32 + lane) * DS_PLD + cc * 32 + j] = v[j];
                }
            }
            ++uses;
        }
        const int fp = nstep & 1;
        ++nstep;
        local_ok = __syncthreads_or(!local_ok) == 0;   // CTA-uniform from here on
        if (threadIdx.x == 0) okflag[fp] = local_ok ? 1 : 0;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        cluster.sync();   // every partial tile of the cluster is in shared memory
        const int c0 = rank * DS_COLS;
        const float *pr[DS_CL];
#pragma unroll
        for (int r = 0; r < DS_CL; ++r) pr[r] = cluster.map_shared_rank(part, r);
        // this thread's elements: t = threadIdx.x + e * DS_THREADS (n fastest);
        // every partial of every element is loaded before any is summed, so
        // the distributed-shared-memory latency is paid about once
        constexpr int EPT = DS_COLS * DS_BN / DS_THREADS;
        static_assert(EPT * DS_THREADS == DS_COLS * DS_BN, "whole elements per thread");
        float sums[EPT], addv[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            // the step's added term, loaded ahead of the partial sums and every store
            const int t = threadIdx.x + e * DS_THREADS;
            const int c = rank * DS_COLS + t / DS_BN, n = n0 + t % DS_BN;
            const int blk = c * a.L + i;
            sums[e] = 0.f;
            addv[e] = 0.f;
            if (n < a.M) {
                if (kind == DS_SCAN) {
                    if (c < a.C) addv[e] = a.vf[cur][(size_t)c * a.Mp + n];
                } else if (c < a.C && blk <= a.N) {
                    addv[e] = (float)a.q[(size_t)blk * a.M + n];
                }
            }
        }
        // one decision for the cluster: every CTA reads the same eight statuses
        // (a CTA rewrites its flag of this parity only after the next
        // barrier), loaded with the partial tiles; no CTA of the cluster has
        // left before this point, so every load reads a live CTA
        int flg[DS_CL];
#pragma unroll
        for (int r = 0; r < DS_CL; ++r) flg[r] = *cluster.map_shared_rank(&okflag[fp], r);
        if (has_in) {
            float pv[EPT][DS_CL];
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int t = threadIdx.x + e * DS_THREADS;
                const int off = (c0 + t / DS_BN) * DS_PLD + t % DS_BN;
#pragma unroll
                for (int r = 0; r < DS_CL; ++r) pv[e][r] = pr[r][off];
            }
#pragma unroll
            for (int e = 0; e < EPT; ++e)
#pragma unroll
                for (int r = 0; r < DS_CL; ++r) sums[e] += pv[e][r];   // ranks in a fixed order
        }
        bool all_ok = true;
#pragma unroll
        for (int r = 0; r < DS_CL; ++r) all_ok = all_ok && flg[r] != 0;
        if (!all_ok) return false;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int t = threadIdx.x + e * DS_THREADS;
            const int c = c0 + t / DS_BN, nl = t % DS_BN, n = n0 + nl;
            if (n >= a.M) continue;
            const float sum = sums[e];
            const int nx = cur ^ 1;
            float val = 0.f, hi, lo;
            if (kind == DS_SCAN) {
                if (c < a.C) val = addv[e] + sum;
                a.vf[nx][(size_t)c * a.Mp + n] = val;
                split_tf32(val, hi, lo);
                a.ph[nx][(size_t)c * a.Mp + n] = hi;
                a.pl[nx][(size_t)c * a.Mp + n] = lo;
                continue;
            }
            const int blk = c * a.L + i;
            const bool live = c < a.C && blk <= a.N;
            if (live) val = addv[e] + sum;
            if (kind == DS_FINAL && live) a.z[(size_t)blk * a.M + n] = (double)val;
            split_tf32(val, hi, lo);
            if (kind == DS_LOCAL_LAST) {
                // the chunk ends seed the scan one column on: V_{c+1} = w_{c,L-1}, V_0 = 0
                if (c + 1 < DS_BM) {
                    a.vf[nx][(size_t)(c + 1) * a.Mp + n] = val;
                    a.ph[nx][(size_t)(c + 1) * a.Mp + n] = hi;
                    a.pl[nx][(size_t)(c + 1) * a.Mp + n] = lo;
                }
                if (c == 0) {
                    a.vf[nx][n] = 0.f;
                    a.ph[nx][n] = 0.f;
                    a.pl[nx][n] = 0.f;
                }
            } else {
                a.ph[nx][(size_t)c * a.Mp + n] = hi;
                a.pl[nx][(size_t)c * a.Mp + n] = lo;
            }
        }
        // the next step's TMA copies (async proxy) read what these stores wrote
        asm volatile("fence.proxy.async.global;" ::: "memory");
        ++nbar;
        if (!ds_grid_barrier(a.bar, a.err, nbar * nblocks)) local_ok = false;
        return true;
    };

    int cur = 0;
    bool good = true;
    for (int i = 0; i < a.L && good; ++i, cur ^= 1)
        good = step(i > 0, cur, 0, &mp.gh, &mp.gl, 0, i == a.L - 1 ? DS_LOCAL_LAST : DS_LOCAL, i);
    for (int s = 0; s < a.S && good; ++s, cur ^= 1)
        good = step(true, cur, 1 << s, &mp.ah[s], &mp.al[s], 1 + s, DS_SCAN, s);
    for (int i = 0; i < a.L && good; ++i, cur ^= 1)
        good = step(true, cur, 0, &mp.gh, &mp.gl, 0, DS_FINAL, i);

    // exit: no TMA copy may still be writing shared memory, and the peers of
    // the cluster must be done reading this CTA's partial tile
    if (threadIdx.x == 0 && loads_out)
        for (int kb = 0; kb < KB; ++kb) tc_mbar_drain(&full_bar[kb], (uses - 1) & 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster.sync();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(DS_TMEM));
    }
}

}  // namespace

// Chunk length L, chunk count C and doubling steps S of the tensor-core
// sweep for N + 1 slices: L = ceil((N + 1) / 128), so C <= 128.
void dense_tc_sweep_shape(int N, int &L, int &C, int &S) {
    L = (N + 1 + DS_BM - 1) / DS_BM;
    C = (N + 1 + L - 1) / L;
    S = 0;
    while ((1 << S) < C) ++S;
}

int dense_tc_sweep_padded(int M) { return (M + 255) / 256 * 256; }

bool dense_tc_sweep_fits(const Problem *p) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    const int Mp = dense_tc_sweep_padded(p->M);
    return p->batch == 1 && Mp <= 1024 && (Mp + DS_BN - 1) / DS_BN * DS_CL <= sms &&
           tc_encode_fn() != nullptr;
}

pit_status dense_tc_sweep(Problem *p, const double *q, double *z, const MemberState *st,
                          cudaStream_t s, bool *launched) {
    *launched = false;
    const int M = p->M, Mp = dense_tc_sweep_padded(M);
    int L, C, S;
    dense_tc_sweep_shape(p->N, L, C, S);
    if (S > DTC_SMAX) {
        p->dtc_on = false;
        return PIT_OK;
    }
    const size_t rows = (size_t)DS_BM * Mp;
    float *buf = p->dtc_buf.as<float>();
    DsArgs a{};
    a.q = q;
    a.z = z;
    a.M = M;
    a.Mp = Mp;
    a.N = p->N;
    a.L = L;
    a.C = C;
    a.S = S;
    for (int k = 0; k < 2; ++k) {
        a.ph[k] = buf + (size_t)(3 * k) * rows;
        a.pl[k] = buf + (size_t)(3 * k + 1) * rows;
        a.vf[k] = buf + (size_t)(3 * k + 2) * rows;
    }
    a.bar = reinterpret_cast<unsigned *>(buf + 6 * rows);
    a.err = p->errword.as<int>();
    a.st = st;
    DsMaps mp;
    for (int k = 0; k < 2; ++k) {
        PIT_TRY(tc_make_map(&mp.ph[k], a.ph[k], DS_BM, Mp, DS_BK, DS_BM));
        PIT_TRY(tc_make_map(&mp.pl[k], a.pl[k], DS_BM, Mp, DS_BK, DS_BM));
    }
    const size_t mm2 = (size_t)Mp * Mp;
    const float *mats = p->dtc_mats.as<float>();
    PIT_TRY(tc_make_map(&mp.gh, mats, Mp, Mp, DS_BK, DS_BN));
    PIT_TRY(tc_make_map(&mp.gl, mats + mm2, Mp, Mp, DS_BK, DS_BN));
    for (int k = 0; k < DTC_SMAX; ++k) {
        const int j = std::min(k, std::max(S - 1, 0));   // unused maps repeat a valid one
        PIT_TRY(tc_make_map(&mp.ah[k], mats + (size_t)(2 + 2 * j) * mm2, Mp, Mp, DS_BK, DS_BN));
        PIT_TRY(tc_make_map(&mp.al[k], mats + (size_t)(3 + 2 * j) * mm2, Mp, Mp, DS_BK, DS_BN));
    }
    PIT_CUDA(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s));
    const int KB = Mp / DS_CL / DS_BK;
    const size_t smem = (size_t)KB * 2 * DS_B_BYTES +
                        std::max((size_t)KB * 2 * DS_A_BYTES, (size_t)DS_BM * DS_PLD * 4) + 1024;
    PIT_TRY(smem_limit(k_dense_sweep_tc, smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((Mp + DS_BN - 1) / DS_BN * DS_CL));
    cfg.blockDim = dim3(DS_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = DS_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    int nclusters = 0;
    {
        cudaLaunchConfig_t q1 = cfg;
        q1.numAttrs = 1;   // the occupancy query takes the cluster shape
        PIT_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, k_dense_sweep_tc, &q1));
    }
    if (nclusters * DS_CL < (int)cfg.gridDim.x) {
        p->dtc_on = false;   // the CUDA-core sweep takes over
        return PIT_OK;
    }
    // only a cooperative launch guarantees that every CTA of the grid
    // barrier is resident; where the runtime refuses it (a profiler, a
    // device shared with other work) the CUDA-core sweep takes over
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_dense_sweep_tc, mp, a);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        p->dtc_on = false;
        return PIT_OK;
    }
    PIT_LAUNCH_CHECK();
    *launched = true;
    return PIT_OK;
}

}  // namespace pit
