// Fused BiCGStab vector work and device-side scalar control of Algorithm 1
// (PiTSBiCG, Sec. 3).  All vectors are FP64 block vectors of
// batch x (N+1) x M values; every reduction is deterministic: a fixed
// warp-shuffle / shared-memory tree per CTA, partial sums per (member,
// quantity, block), and one finishing CTA per member that adds the partials
// in a fixed order.  Optionally (PIT_KRYLOV_CLUSTERS=1) a block of 2 to 8
// chunks of 2048 values is one thread-block cluster: its CTAs' sums meet in
// distributed shared memory and the first CTA adds them in rank order, so
// one partial per block reaches global memory.  Both forms add the chunks'
// sums in chunk order: the results are the same bit for bit.
//
// Block inner product (Sec. 3, text after Algorithm 1): the sum of the
// Euclidean products of all N+1 blocks.  ||.||_{N,inf} (Algorithm 1, the
// while test): the largest Euclidean block norm.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include <cooperative_groups.h>

#include "pit_internal.h"

namespace pit {

namespace {

constexpr int VT = 256;        // threads per vector CTA
constexpr int EPT = 8;         // elements per thread
constexpr int CHUNK = VT * EPT;
constexpr int FT = 256;        // threads of a finishing CTA
constexpr int QMAX = 2;        // partial quantities per kernel

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the CTA (fixed tree); result valid in thread 0.
template <int NT>
__device__ double cta_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    return r;
}
template <int NT>
__device__ double cta_max(double v, double *sh) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_max(r);
    }
    return r;
}

struct VecGeom {
    int M, nblk, chunks;
    size_t blen;   // nblk * M
    int cl = 0;    // 1: the chunks of a block form a cluster, one partial per block
};

// partial slots per block: one per chunk, or one per block with clusters
__device__ __host__ __forceinline__ int pslots(const VecGeom &g) { return g.cl ? 1 : g.chunks; }

__device__ __forceinline__ bool member_runs(const MemberState *st, int b) {
    const MemberState &m = st[b];
    return m.active && !m.skip;
}

__device__ __forceinline__ size_t pidx(const VecGeom &g, int b, int q, int Q, int n, int c) {
    return (((size_t)b * Q + q) * g.nblk + n) * pslots(g) + c;
}

// Writes this CTA's Q partial sums (fixed order: warp q sums quantity q,
// lane l first over threads l, l + 32, ..., then a shuffle tree).  One
// barrier and 12 FP64 adds per quantity on the 2-lane-per-SM FP64 pipe,
// against 45 adds per quantity for a shuffle tree in every warp.
template <int Q>
__device__ void store_partials(const VecGeom &g, double *part, const double (&acc)[Q]) {
    static_assert(Q <= VT / 32, "one warp per quantity");
    __shared__ double sh[Q][VT];
    __shared__ double csum[8][Q];   // the first CTA of a cluster: every chunk's sums
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
#pragma unroll
    for (int q = 0; q < Q; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    double r = 0.0;
    if (w < Q) {
        r = sh[w][l];
#pragma unroll
        for (int i = 1; i < VT / 32; ++i) r += sh[w][l + 32 * i];
        r = warp_sum(r);
        if (l == 0 && !g.cl) part[pidx(g, b, w, Q, n, c)] = r;
    }
    if (g.cl) {
        // the block's chunks are the cluster's CTAs (rank = chunk): each CTA
        // writes its sums into the first CTA's shared memory (distributed
        // shared memory), one cluster barrier, and the first CTA adds them in
        // rank order; the others may leave at once
        namespace cg = cooperative_groups;
        cg::cluster_group cluster = cg::this_cluster();
        if (w < Q && l == 0) cluster.map_shared_rank(&csum[0][0], 0)[c * Q + w] = r;
        cluster.sync();
        if (c == 0 && threadIdx.x < Q) {
            double s = 0.0;
            for (int k = 0; k < g.chunks; ++k) s += csum[k][threadIdx.x];
            part[pidx(g, b, threadIdx.x, Q, n, 0)] = s;
        }
    }
}

// ---------------------------------------------------------------- kernels

// R~ = P = R; partial: ||R_n||^2.
__global__ void __launch_bounds__(VT) k_init(VecGeom g, const double *__restrict__ R,
                                             double *__restrict__ Rt, double *__restrict__ P,
                                             double *__restrict__ part, const MemberState *st) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
    double acc[1] = {0.0};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) {
            const double r = R[base + i];
            Rt[base + i] = r;
            P[base + i] = r;
            acc[0] = fma(r, r, acc[0]);
        }
    }
    store_partials<1>(g, part, acc);
}

// partials: <U, V>, <U, U> per block (masked by the member's run flag).
__global__ void __launch_bounds__(VT) k_dot2(VecGeom g, const double *__restrict__ U,
                                             const double *__restrict__ V,
                                             double *__restrict__ part, const MemberState *st) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    if (st && !member_runs(st, b)) return;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
    double acc[2] = {0.0, 0.0};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) {
            const double u = U[base + i];
            acc[0] = fma(u, V[base + i], acc[0]);
            acc[1] = fma(u, u, acc[1]);
        }
    }
    store_partials<2>(g, part, acc);
}

// S = R - alpha D; partial ||S_n||^2.
__global__ void __launch_bounds__(VT) k_update_S(VecGeom g, const double *__restrict__ R,
                                                 const double *__restrict__ D,
                                                 double *__restrict__ S, double *__restrict__ part,
                                                 const MemberState *st) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    if (!member_runs(st, b)) return;
    const double alpha = st[b].alpha;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
    double acc[1] = {0.0};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) {
            const double s = fma(-alpha, D[base + i], R[base + i]);
            S[base + i] = s;
            acc[0] = fma(s, s, acc[0]);
        }
    }
    store_partials<1>(g, part, acc);
}

// X += alpha P + omega S; R = S - omega K   (half-step exit: X += alpha P; R = S)
// partials: <R, R~>, ||R_n||^2.
__global__ void __launch_bounds__(VT) k_update_XR(VecGeom g, double *__restrict__ X,
                                                  double *__restrict__ R,
                                                  const double *__restrict__ P,
                                                  const double *__restrict__ S,
                                                  const double *__restrict__ K,
                                                  const double *__restrict__ Rt,
                                                  double *__restrict__ part,
                                                  const MemberState *st) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    if (!member_runs(st, b)) return;
    const double alpha = st[b].alpha;
    const bool half = st[b].half != 0;
    const double omega = half ? 0.0 : st[b].omega;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
    double acc[2] = {0.0, 0.0};
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) {
            const size_t j = base + i;
            const double s = S[j];
            double x = fma(alpha, P[j], X[j]);
            double r = s;
            if (!half) {
                x = fma(omega, s, x);
                r = fma(-omega, K[j], s);
            }
            X[j] = x;
            R[j] = r;
            acc[0] = fma(r, Rt[j], acc[0]);
            acc[1] = fma(r, r, acc[1]);
        }
    }
    store_partials<2>(g, part, acc);
}

// P = R + beta (P - omega D), or on restart P = R~ = R.
__global__ void __launch_bounds__(VT) k_update_P(VecGeom g, const double *__restrict__ R,
                                                 double *__restrict__ P,
                                                 const double *__restrict__ D,
                                                 double *__restrict__ Rt, const MemberState *st) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    if (!st[b].active) return;
    const bool restart = st[b].do_restart != 0;
    const double beta = st[b].beta, omega = st[b].omega;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) {
            const size_t j = base + i;
            const double r = R[j];
            if (restart) {
                P[j] = r;
                Rt[j] = r;
            } else {
                P[j] = fma(beta, fma(-omega, D[j], P[j]), r);
            }
        }
    }
}

// X += Y for active members (refinement correction).
__global__ void __launch_bounds__(VT) k_axpy(VecGeom g, double *__restrict__ X,
                                             const double *__restrict__ Y) {
    const int b = blockIdx.z, n = blockIdx.y, c = blockIdx.x;
    const size_t base = (size_t)b * g.blen + (size_t)n * g.M;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int i = c * CHUNK + e * VT + threadIdx.x;
        if (i < g.M) X[base + i] += Y[base + i];
    }
}

// Sum over the chunks of block n (fixed order) of quantity q.
__device__ __forceinline__ double block_value(const VecGeom &g, const double *part, int b,
                                              int q, int Q, int n) {
    if (g.cl) return part[pidx(g, b, q, Q, n, 0)];   // already summed in chunk order
    double s = 0.0;
    for (int c = 0; c < g.chunks; ++c) s += part[pidx(g, b, q, Q, n, c)];
    return s;
}

// For quantity q: total over blocks and the largest block value.
__device__ void reduce_q(const VecGeom &g, const double *part, int b, int q, int Q,
                         double *sum_out, double *max_out) {
    __shared__ double sh[32];
    double s = 0.0, m = 0.0;
    for (int n = threadIdx.x; n < g.nblk; n += FT) {
        const double v = block_value(g, part, b, q, Q, n);
        s += v;
        m = fmax(m, v);
    }
    s = cta_sum<FT>(s, sh);
    m = cta_max<FT>(m, sh);
    if (threadIdx.x == 0) {
        *sum_out = s;
        *max_out = m;
    }
}

enum FinishKind { F_INIT, F_SIGMA, F_S, F_OMEGA, F_R, F_NORM };

struct InitArgs {
    double tol_rel;
    const double *abs_thresh;   // per-member absolute thresholds (device) or null
    double eps0, eps_b;
    int max_iter;
};

__global__ void __launch_bounds__(FT) k_finish(VecGeom g, const double *__restrict__ part,
                                               MemberState *st, int kind, InitArgs ia,
                                               double *out) {
    const int b = blockIdx.x;
    MemberState &m = st[b];
    __shared__ double s0, m0, s1, m1;
    if (kind == F_INIT) {
        reduce_q(g, part, b, 0, 1, &s0, &m0);
        __syncthreads();
        if (threadIdx.x == 0) {
            m.rho = s0;
            m.rt2 = s0;
            m.r2 = s0;
            m.r0 = sqrt(m0);
            m.rnorm = m.r0;
            m.thresh = ia.abs_thresh ? ia.abs_thresh[b] : ia.tol_rel * m.r0;
            m.eps0 = ia.eps0;
            m.eps_b = ia.eps_b;
            m.max_iter = ia.max_iter;
            m.iter = 0;
            m.restarts = 0;
            m.matvecs = 1;
            m.skip = m.half = m.just_restarted = m.do_restart = 0;
            m.alpha = m.omega = m.beta = 0.0;
            m.status = PIT_OK;
            m.active = 1;
            if (!isfinite(s0)) {
                m.status = PIT_E_NONFINITE;
                m.active = 0;
            } else if (!(m.rnorm > m.thresh)) {
                m.active = 0;
            } else if (ia.max_iter <= 0) {
                m.status = PIT_E_MAXITER;
                m.active = 0;
            }
        }
        return;
    }
    if (kind == F_NORM) {
        reduce_q(g, part, b, 0, 2, &s0, &m0);
        __syncthreads();
        if (threadIdx.x == 0) out[b] = sqrt(m0);
        return;
    }
    if (!m.active) return;
    if (kind == F_SIGMA) {
        reduce_q(g, part, b, 0, 2, &s0, &m0);
        reduce_q(g, part, b, 1, 2, &s1, &m1);
        __syncthreads();
        if (threadIdx.x == 0) {
            m.do_restart = 0;
            m.matvecs += 1;
            m.sigma = s0;
            m.dd = s1;
            const double lim = m.eps_b * sqrt(m.dd) * sqrt(m.rt2);
            if (!isfinite(s0) || !isfinite(s1)) {
                m.status = PIT_E_NONFINITE;
                m.active = 0;
            } else if (fabs(m.sigma) <= lim) {
                if (m.just_restarted) {
                    m.status = PIT_E_BREAKDOWN;
                    m.active = 0;
                } else {
                    m.skip = 1;
                    m.do_restart = 1;
                    m.just_restarted = 1;
                    m.restarts += 1;
                }
            } else {
                m.just_restarted = 0;
                m.alpha = m.rho / m.sigma;
            }
        }
        return;
    }
    if (m.skip) {
        if (kind == F_R && threadIdx.x == 0) {
            // restart after a vanishing sigma: R~ <- R, P <- R (done by k_update_P)
            m.rho = m.r2;
            m.rt2 = m.r2;
            m.skip = 0;
        }
        return;
    }
    if (kind == F_S) {
        reduce_q(g, part, b, 0, 1, &s0, &m0);
        __syncthreads();
        if (threadIdx.x == 0) {
            m.snorm = sqrt(m0);
            m.half = (m.snorm <= m.thresh) ? 1 : 0;
            if (!isfinite(m0)) {
                m.status = PIT_E_NONFINITE;
                m.active = 0;
            }
        }
        return;
    }
    if (kind == F_OMEGA) {
        if (m.half) return;
        reduce_q(g, part, b, 0, 2, &s0, &m0);
        reduce_q(g, part, b, 1, 2, &s1, &m1);
        __syncthreads();
        if (threadIdx.x == 0) {
            m.matvecs += 1;
            m.ks = s0;
            m.kk = s1;
            m.omega = m.ks / m.kk;
            if (!isfinite(m.omega)) {
                m.status = PIT_E_NONFINITE;
                m.active = 0;
            } else if (m.omega == 0.0) {
                m.status = PIT_E_BREAKDOWN;
                m.active = 0;
            }
        }
        return;
    }
    if (kind == F_R) {
        reduce_q(g, part, b, 0, 2, &s0, &m0);
        reduce_q(g, part, b, 1, 2, &s1, &m1);
        __syncthreads();
        if (threadIdx.x == 0) {
            m.rho_new = s0;
            m.r2 = s1;
            m.rnorm = sqrt(m1);
            m.iter += 1;
            if (m.half) {
                m.half = 0;
                m.active = 0;
                m.status = PIT_OK;
                return;
            }
            m.beta = (m.alpha / m.omega) * (m.rho_new / m.rho);
            if (fabs(m.rho_new) <= m.eps0 * sqrt(m.r2) * sqrt(m.rt2)) {
                m.do_restart = 1;
                m.restarts += 1;
                m.rho = m.r2;
                m.rt2 = m.r2;
            } else {
                m.do_restart = 0;
                m.rho = m.rho_new;
            }
            if (!isfinite(m.r2) || !isfinite(m.rho_new)) {
                m.status = PIT_E_NONFINITE;
                m.active = 0;
            } else if (m.rnorm <= m.thresh) {
                m.active = 0;
                m.status = PIT_OK;
            } else if (m.iter >= m.max_iter) {
                m.active = 0;
                m.status = PIT_E_MAXITER;
            }
        }
        return;
    }
}

VecGeom geom(const Problem *p) {
    VecGeom g;
    g.M = p->M;
    g.nblk = p->N + 1;
    g.chunks = (p->M + CHUNK - 1) / CHUNK;
    g.blen = p->blen;
    g.cl = (g.chunks >= 2 && g.chunks <= 8 && p->kr_cluster) ? 1 : 0;
    return g;
}

dim3 vgrid(const Problem *p, const VecGeom &g) { return dim3(g.chunks, g.nblk, p->batch); }

// A vector kernel that stores partial sums: with g.cl, launched as clusters
// of the block's chunks.
template <class... KArgs, class... Args>
pit_status vlaunch(const Problem *p, const VecGeom &g, cudaStream_t s, void (*kern)(KArgs...),
                   Args &&...args) {
    if (!g.cl) {
        kern<<<vgrid(p, g), VT, 0, s>>>(std::forward<Args>(args)...);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = vgrid(p, g);
    cfg.blockDim = dim3(VT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g.chunks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PIT_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

pit_status finish(Problem *p, int kind, cudaStream_t s, InitArgs ia = InitArgs{},
                  double *out = nullptr) {
    VecGeom g = geom(p);
    k_finish<<<p->batch, FT, 0, s>>>(g, p->partials.as<double>(), p->states.as<MemberState>(),
                                     kind, ia, out);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

}  // namespace

pit_status krylov_prepare(Problem *p) {
    const size_t vb = p->vlen * sizeof(double);
    PIT_TRY(p->X.ensure(vb));
    PIT_TRY(p->R.ensure(vb));
    PIT_TRY(p->Rt.ensure(vb));
    PIT_TRY(p->P.ensure(vb));
    PIT_TRY(p->S.ensure(vb));
    PIT_TRY(p->D.ensure(vb));
    PIT_TRY(p->K.ensure(vb));
    VecGeom g = geom(p);
    PIT_TRY(p->partials.ensure((size_t)p->batch * QMAX * g.nblk * g.chunks * sizeof(double)));
    PIT_TRY(p->states.ensure((size_t)p->batch * sizeof(MemberState)));
    return PIT_OK;
}

pit_status kr_init(Problem *p, double tol_rel, const double *abs_thresh, double eps0,
                   int max_iter, cudaStream_t s) {
    VecGeom g = geom(p);
    PIT_TRY(vlaunch(p, g, s, k_init, g, (const double *)p->R.as<double>(), p->Rt.as<double>(),
                    p->P.as<double>(), p->partials.as<double>(), (const MemberState *)nullptr));
    InitArgs ia{tol_rel, abs_thresh, eps0, 1e-14, max_iter};
    return finish(p, F_INIT, s, ia);
}

pit_status kr_sigma(Problem *p, cudaStream_t s) {
    VecGeom g = geom(p);
    MemberState *st = p->states.as<MemberState>();
    PIT_TRY(vlaunch(p, g, s, k_dot2, g, (const double *)p->D.as<double>(),
                    (const double *)p->Rt.as<double>(), p->partials.as<double>(),
                    (const MemberState *)st));
    return finish(p, F_SIGMA, s);
}

pit_status kr_update_S(Problem *p, cudaStream_t s) {
    VecGeom g = geom(p);
    MemberState *st = p->states.as<MemberState>();
    PIT_TRY(vlaunch(p, g, s, k_update_S, g, (const double *)p->R.as<double>(),
                    (const double *)p->D.as<double>(), p->S.as<double>(), p->partials.as<double>(),
                    (const MemberState *)st));
    return finish(p, F_S, s);
}

pit_status kr_omega(Problem *p, cudaStream_t s) {
    VecGeom g = geom(p);
    MemberState *st = p->states.as<MemberState>();
    PIT_TRY(vlaunch(p, g, s, k_dot2, g, (const double *)p->K.as<double>(),
                    (const double *)p->S.as<double>(), p->partials.as<double>(),
                    (const MemberState *)st));
    return finish(p, F_OMEGA, s);
}

pit_status kr_update_XR(Problem *p, cudaStream_t s) {
    VecGeom g = geom(p);
    MemberState *st = p->states.as<MemberState>();
    PIT_TRY(vlaunch(p, g, s, k_update_XR, g, p->X.as<double>(), p->R.as<double>(),
                    (const double *)p->P.as<double>(), (const double *)p->S.as<double>(),
                    (const double *)p->K.as<double>(), (const double *)p->Rt.as<double>(),
                    p->partials.as<double>(), (const MemberState *)st));
    return finish(p, F_R, s);
}

pit_status kr_update_P(Problem *p, cudaStream_t s) {
    VecGeom g = geom(p);
    k_update_P<<<vgrid(p, g), VT, 0, s>>>(g, p->R.as<double>(), p->P.as<double>(),
                                          p->D.as<double>(), p->Rt.as<double>(),
                                          p->states.as<MemberState>());
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

pit_status kr_block_norm(Problem *p, const double *U, double *out, cudaStream_t s) {
    VecGeom g = geom(p);
    // k_dot2(U, U) stores <U,U> per block as quantity 0 of a Q = 2 layout
    PIT_TRY(vlaunch(p, g, s, k_dot2, g, U, U, p->partials.as<double>(), (const MemberState *)nullptr));
    return finish(p, F_NORM, s, InitArgs{}, out);
}

pit_status kr_axpy(Problem *p, double *X, const double *Y, cudaStream_t s) {
    VecGeom g = geom(p);
    k_axpy<<<vgrid(p, g), VT, 0, s>>>(g, X, Y);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

// ---------------------------------------------------- standalone reduction
namespace {
__global__ void __launch_bounds__(FT) k_reduce_final(VecGeom g, const double *__restrict__ part,
                                                     double *dot, double *norms,
                                                     double *norm_inf) {
    __shared__ double sh[32];
    double s = 0.0, m = 0.0;
    for (int n = threadIdx.x; n < g.nblk; n += FT) {
        const double d = block_value(g, part, 0, 0, 2, n);
        const double u = block_value(g, part, 0, 1, 2, n);
        s += d;
        m = fmax(m, u);
        if (norms) norms[n] = sqrt(u);
    }
    s = cta_sum<FT>(s, sh);
    m = cta_max<FT>(m, sh);
    if (threadIdx.x == 0) {
        *dot = s;
        *norm_inf = sqrt(m);
    }
}
}  // namespace

pit_status block_reduce(const double *U, const double *V, int nblocks, int M, double *dot,
                        double *norms, double *norm_inf, cudaStream_t s) {
    VecGeom g;
    g.M = M;
    g.nblk = nblocks;
    g.chunks = (M + CHUNK - 1) / CHUNK;
    g.blen = (size_t)nblocks * M;
    double *part = nullptr;
    PIT_CUDA(cudaMallocAsync(&part, (size_t)2 * nblocks * g.chunks * sizeof(double), s));
    k_dot2<<<dim3(g.chunks, g.nblk, 1), VT, 0, s>>>(g, U, V, part, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_reduce_final<<<1, FT, 0, s>>>(g, part, dot, norms, norm_inf);
        e = cudaGetLastError();
    }
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return cuda_fail(e, "block_reduce launch", __FILE__, __LINE__);
    return PIT_OK;
}

}  // namespace pit

// ------------------------------------------------ allocation-free variant
// pit_block_reduce_noalloc: the same two kernels as pit_block_reduce, but
// the partial sums live in a fixed array compiled into the library instead
// of memory allocated per call.  Meant for callers that may not allocate
// device memory: a process whose device memory is entirely handed to another
// allocator (so cudaMalloc would fail), or a latency-bound host thread that
// cannot afford cudaMalloc/cudaFree and the device-wide synchronisation
// cudaFree implies.
namespace pit {
namespace {

// Two partial sums per chunk of CHUNK values, per block: 131072 doubles
// (1 MiB) hold nblocks * ceil(M / 2048) <= 65536 chunks.  Every device that
// loads the library keeps this array until the process exits.
constexpr size_t NOALLOC_DOUBLES = 131072;
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_partials on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
pit_status noalloc_scratch(double **out) {
    int dev = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("pit_block_reduce_noalloc: device ordinal out of range");
        return PIT_E_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *addr = nullptr;
        PIT_CUDA(cudaGetSymbolAddress(&addr, g_noalloc_partials));
        g_noalloc_addr[dev] = static_cast<double *>(addr);
    }
    *out = g_noalloc_addr[dev];
    return PIT_OK;
}

}  // namespace
}  // namespace pit

extern "C" pit_status pit_block_reduce_noalloc(const double *U, const double *V, int nblocks,
                                               int M, double *dot, double *norms,
                                               double *norm_inf) {
    using namespace pit;
    if (!U || !V || !dot || !norm_inf || nblocks < 1 || M < 1) {
        set_error("pit_block_reduce_noalloc: bad argument");
        return PIT_E_INVALID;
    }
    if (nblocks > PIT_MAX_BLOCKS) {
        set_error("pit_block_reduce_noalloc: nblocks exceeds 65535 (one grid row per block)");
        return PIT_E_INVALID;
    }
    VecGeom g;
    g.M = M;
    g.nblk = nblocks;
    g.chunks = (M + CHUNK - 1) / CHUNK;
    g.blen = (size_t)nblocks * M;
    const size_t need = (size_t)2 * nblocks * g.chunks;
    if (need > NOALLOC_DOUBLES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "pit_block_reduce_noalloc: nblocks * ceil(M/2048) = %zu chunks exceeds the "
                 "fixed scratch of %zu chunks; use pit_block_reduce",
                 need / 2, NOALLOC_DOUBLES / 2);
        set_error(buf);
        return PIT_E_INVALID;
    }
    double *part = nullptr;
    PIT_TRY(noalloc_scratch(&part));
    // every partial read by k_reduce_final is written by k_dot2 in this call,
    // so the array needs no clearing between calls
    k_dot2<<<dim3(g.chunks, g.nblk, 1), VT, 0, 0>>>(g, U, V, part, nullptr);
    PIT_LAUNCH_CHECK();
    k_reduce_final<<<1, FT, 0, 0>>>(g, part, dot, norms, norm_inf);
    PIT_LAUNCH_CHECK();
    PIT_CUDA(cudaStreamSynchronize(0));
    return PIT_OK;
}
