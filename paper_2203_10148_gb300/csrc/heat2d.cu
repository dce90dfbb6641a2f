// 2D heat u_t = nu (u_xx + u_yy) on the unit square, Dirichlet 0, n x n
// interior points, h = 1/(n+1), 5-point Laplacian.
//
// Fine batch (the N independent slice problems of eq. (2), fused with the
// shift-subtract of eq. (4)): one CTA per slice keeps the slice's whole
// state on chip across all RK4 steps.  Thread (tx, ty) owns an RY x RX tile
// of points; the west/east halo columns come from the neighbouring lanes
// by warp shuffle (a row of thread tiles never straddles a warp) and the
// north/south halo rows through a double-buffered shared-memory row buffer,
// so each RK4 stage costs one CTA barrier.  RK4 for the linear autonomous
// u' = L u is applied in nested (Horner) form
//   w = u + (dt/4) L u;  w = u + (dt/3) L w;  w = u + (dt/2) L w;  u <- u + dt L w,
// which is the same polynomial 1 + Z + Z^2/2 + Z^3/6 + Z^4/24 of Z = dt L as the
// classical four-stage form.  FP32 keeps u and the stage value in
// registers; FP64 keeps u in shared memory.  Inputs and outputs are FP64.
//
// Coarse sweep (eq. (7), right): G is one implicit-Euler step, which the
// sine basis S_jk = sin(pi (j+1)(k+1)/(n+1)) diagonalises exactly
// (S D2 S^{-1} = diag(mu_k), mu_k = -(4/h^2) sin^2(pi (k+1) h/2), S^2 = (n+1)/2 I).
// So z_n = q_n + G z_{n-1} becomes, mode by mode,
//   zhat_n = qhat_n + g_kl zhat_{n-1},  g_kl = (1 - dTc nu (mu_k + mu_l))^{-c},
// with qhat = S q S and z = (2/(n+1))^2 S zhat S.  The transforms are batched
// block products; the recurrence is a chunked scan over n.
#include <math.h>

#include <vector>

#include "pit_internal.h"

namespace pit {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RY = 8;   // rows per thread tile
constexpr int RX = 4;   // columns per thread tile

struct Heat2dArgs {
    const double *x;
    double *y;
    const double *y0;
    int n, N, batch;
    size_t blen;
    int n_first;    // output slice of blockIdx.x == 0
    int mode;       // FINE_APPLY, FINE_RESIDUAL, 2 = plain
    int steps;
    double c[4];    // stage coefficients dt/4, dt/3, dt/2, dt times nu/h^2
    int TX, TXp, TY;
    const MemberState *st;
};

__device__ __forceinline__ bool runs(const MemberState *st, int b) {
    return st == nullptr || (st[b].active && !st[b].skip && !st[b].half);
}

template <class T>
__device__ __forceinline__ T lap5(T vn, T vs, T vw, T ve, T vc) {
    const T a = vn + vs;
    const T b = vw + ve;
    return fma(T(-4), vc, a + b);
}

// One CTA per (slice, member).  Threads: TXp * TYp (multiple of 32);
// thread tiles with tx >= TX or ty >= TY hold zeros.
template <class T>
__global__ void __launch_bounds__(512, 1) k_heat2d_fine(Heat2dArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.y;
    if (!runs(a.st, b)) return;
    const int n = a.n;
    const int tid = threadIdx.x;
    const int tx = tid % a.TXp, ty = tid / a.TXp;
    const int TYp = blockDim.x / a.TXp;
    const int W = a.TXp * RX;                     // row buffer width
    T *rows = reinterpret_cast<T *>(smem_raw);    // [2 buf][2 top/bot][TYp][W]
    T *us = rows + 4 * (size_t)TYp * W;           // FP64 only: u[n][n]
    constexpr bool U_SMEM = sizeof(T) == 8;

    const int i0 = tx * RX, j0 = ty * RY;
    const bool edge = (i0 + RX > n) || (j0 + RY > n);
    const int slice = a.n_first + blockIdx.x;     // output block 1..N
    const size_t mb = (size_t)b * a.blen;
    const double *xin = a.x + mb + (size_t)(slice - 1) * n * n;

    T v[RY][RX];
    T ur[U_SMEM ? 1 : RY][U_SMEM ? 1 : RX];
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int c = 0; c < RX; ++c) {
            const int i = i0 + c, j = j0 + r;
            const bool ok = (i < n && j < n);
            const T ld = (T)xin[(size_t)min(j, n - 1) * n + min(i, n - 1)];
            const T val = ok ? ld : T(0);
            v[r][c] = val;
            if constexpr (U_SMEM) {
                if (i < n && j < n) us[(size_t)j * n + i] = val;
            } else {
                ur[r][c] = val;
            }
        }
    const bool west_zero = (tx == 0), east_zero = (tx == a.TXp - 1);
    const bool north_zero = (ty == 0), south_zero = (ty == TYp - 1);
    int buf = 0;
    for (int s = 0; s < a.steps; ++s) {
#pragma unroll 1
        for (int stage = 0; stage < 4; ++stage) {
            const double cd = stage == 0 ? a.c[0] : stage == 1 ? a.c[1] : stage == 2 ? a.c[2] : a.c[3];
            const T cc = (T)cd;
            // publish the top and bottom rows of v
            T *top = rows + ((size_t)(buf * 2 + 0) * TYp + ty) * W + i0;
            T *bot = rows + ((size_t)(buf * 2 + 1) * TYp + ty) * W + i0;
#pragma unroll
            for (int c = 0; c < RX; ++c) {
                top[c] = v[0][c];
                bot[c] = v[RY - 1][c];
            }
            __syncthreads();
            T nrow[RX], srow[RX];
            const T *nsrc = rows + ((size_t)(buf * 2 + 1) * TYp + (ty - 1)) * W + i0;
            const T *ssrc = rows + ((size_t)(buf * 2 + 0) * TYp + (ty + 1)) * W + i0;
#pragma unroll
            for (int c = 0; c < RX; ++c) {
                nrow[c] = north_zero ? T(0) : nsrc[c];
                srow[c] = south_zero ? T(0) : ssrc[c];
            }
            T prev[RX];
#pragma unroll
            for (int c = 0; c < RX; ++c) prev[c] = nrow[c];
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                T w_in = __shfl_up_sync(FULL, v[r][RX - 1], 1);
                T e_in = __shfl_down_sync(FULL, v[r][0], 1);
                if (west_zero) w_in = T(0);
                if (east_zero) e_in = T(0);
                T cur[RX];
#pragma unroll
                for (int c = 0; c < RX; ++c) cur[c] = v[r][c];
#pragma unroll
                for (int c = 0; c < RX; ++c) {
                    const T vn = prev[c];
                    const T vs = (r < RY - 1) ? v[r + 1][c] : srow[c];
                    const T vw = (c > 0) ? cur[c - 1] : w_in;
                    const T ve = (c < RX - 1) ? cur[c + 1] : e_in;
                    T u;
                    if constexpr (U_SMEM) {
                        const int i = i0 + c, j = j0 + r;
                        const T uu = us[(size_t)min(j, n - 1) * n + min(i, n - 1)];
                        u = (i < n && j < n) ? uu : T(0);
                    } else {
                        u = ur[U_SMEM ? 0 : r][U_SMEM ? 0 : c];
                    }
                    v[r][c] = fma(cc, lap5(vn, vs, vw, ve, cur[c]), u);
                }
#pragma unroll
                for (int c = 0; c < RX; ++c) prev[c] = cur[c];
            }
            if (edge) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int c = 0; c < RX; ++c)
                        if (i0 + c >= n || j0 + r >= n) v[r][c] = T(0);
            }
            buf ^= 1;
        }
        // end of step: u <- v
        if constexpr (U_SMEM) {
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int c = 0; c < RX; ++c) {
                    const int i = i0 + c, j = j0 + r;
                    if (i < n && j < n) us[(size_t)j * n + i] = v[r][c];
                }
        } else {
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int c = 0; c < RX; ++c) ur[U_SMEM ? 0 : r][U_SMEM ? 0 : c] = v[r][c];
        }
    }
    // epilogue: row `slice` of the block operator, FP64
    double *yo = a.y + mb + (size_t)slice * n * n;
    const double *xn = a.x + mb + (size_t)slice * n * n;
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int c = 0; c < RX; ++c) {
            const int i = i0 + c, j = j0 + r;
            if (i < n && j < n) {
                const size_t k = (size_t)j * n + i;
                const double f = (double)v[r][c];
                if (a.mode == FINE_APPLY) yo[k] = xn[k] - f;
                else if (a.mode == FINE_RESIDUAL) yo[k] = f - xn[k];
                else yo[k] = f;
            }
        }
    if (slice == 1 && a.mode != 2) {
        const double *x0 = a.x + mb;
        double *y0o = a.y + mb;
        const int nn = n * n;
        for (int k = tid; k < nn; k += blockDim.x)
            y0o[k] = (a.mode == FINE_APPLY) ? x0[k] : a.y0[(size_t)b * nn + k] - x0[k];
    }
}

// ------------------------------------------------------- sine transforms
// out_b = scale * (A_b S)^T for every n x n block b, i.e.
// out_b[k][j] = scale * sum_i A_b[j][i] S[i][k].  Applied twice it gives
// scale^2 S A S (S symmetric).  One CTA (256 threads, 8x8 outputs each) per
// block; A_b is staged transposed in shared memory; S is staged in shared
// memory (FP32) or read through L1/L2 (FP64).
constexpr int PT = 256;

template <class Tin, class T, class Tout>
__global__ void __launch_bounds__(PT) k_block_xS_T(const Tin *__restrict__ A, Tout *__restrict__ out,
                                                   const T *__restrict__ S, int n, int nblk,
                                                   double scale, const MemberState *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool S_SMEM = sizeof(T) == 4;
    const int blk = blockIdx.x;
    const int member = blk / nblk;
    if (!runs(st, member)) return;
    const int ld = n + 4;                          // padded row of At
    T *At = reinterpret_cast<T *>(smem_raw);       // At[i][j] = A[j][i]
    T *Ss = At + (size_t)n * ld;                   // S[i][k] (FP32 only)
    const size_t nn = (size_t)n * n;
    const Tin *Ab = A + (size_t)blk * nn;
    for (size_t q = threadIdx.x; q < nn; q += PT) {
        const int j = (int)(q / n), i = (int)(q % n);
        At[(size_t)i * ld + j] = (T)Ab[q];
    }
    if (S_SMEM)
        for (size_t q = threadIdx.x; q < nn; q += PT) Ss[(q / n) * ld + (q % n)] = S[q];
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int j0 = ty * 8, k0 = tx * 8;
    if (j0 >= n || k0 >= n) return;
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = T(0);
    const int jn = min(8, n - j0), kn = min(8, n - k0);
    for (int i = 0; i < n; ++i) {
        T av[8], sv[8];
        const T *arow = At + (size_t)i * ld + j0;
#pragma unroll
        for (int r = 0; r < 8; ++r) av[r] = (r < jn) ? arow[min(r, jn - 1)] : T(0);
        if (S_SMEM) {
            const T *srow = Ss + (size_t)i * ld + k0;
#pragma unroll
            for (int c = 0; c < 8; ++c) sv[c] = (c < kn) ? srow[min(c, kn - 1)] : T(0);
        } else {
            const T *srow = S + (size_t)i * n + k0;
#pragma unroll
            for (int c = 0; c < 8; ++c) sv[c] = (c < kn) ? __ldg(srow + min(c, kn - 1)) : T(0);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = fma(av[r], sv[c], acc[r][c]);
    }
    Tout *ob = out + (size_t)blk * nn;
    const T sc = (T)scale;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r)
            if (c < kn && r < jn) ob[(size_t)(k0 + c) * n + (j0 + r)] = (Tout)(sc * acc[r][c]);
}

// Chunked scan of zhat_n = qhat_n + g zhat_{n-1} over the N+1 blocks of each
// member, mode by mode, with an FP64 running value.
// pass 1: chunk-local recurrences from zero -> ends[member][chunk][mode]
template <class T>
__global__ void k_rec_local(const T *__restrict__ hat, double *__restrict__ ends,
                            const double *__restrict__ g, int nn, int nblk, int clen,
                            int nchunks, const MemberState *st) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y, member = blockIdx.z;
    if (mode >= nn || !runs(st, member)) return;
    const double gm = g[mode];
    const int k0 = chunk * clen, k1 = min(nblk, k0 + clen);
    const T *h = hat + (size_t)member * nblk * nn + mode;
    double z = 0.0;
    for (int k = k0; k < k1; ++k) z = fma(gm, z, (double)h[(size_t)k * nn]);
    ends[((size_t)member * nchunks + chunk) * nn + mode] = z;
}

// pass 2: carries into each chunk (sequential over chunks, in place)
__global__ void k_rec_carry(double *__restrict__ ends, const double *__restrict__ g, int nn,
                            int clen, int nchunks, const MemberState *st) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    const int member = blockIdx.y;
    if (mode >= nn || !runs(st, member)) return;
    double gl = 1.0;
    const double gm = g[mode];
    for (int k = 0; k < clen; ++k) gl *= gm;
    double carry = 0.0;
    double *e = ends + (size_t)member * nchunks * nn + mode;
    for (int c = 0; c < nchunks; ++c) {
        const double end = e[(size_t)c * nn];
        e[(size_t)c * nn] = carry;
        carry = fma(gl, carry, end);
    }
}

// pass 3: replay each chunk from its carry and write zhat
template <class T>
__global__ void k_rec_apply(T *__restrict__ hat, const double *__restrict__ ends,
                            const double *__restrict__ g, int nn, int nblk, int clen,
                            int nchunks, const MemberState *st) {
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y, member = blockIdx.z;
    if (mode >= nn || !runs(st, member)) return;
    const double gm = g[mode];
    const int k0 = chunk * clen, k1 = min(nblk, k0 + clen);
    T *h = hat + (size_t)member * nblk * nn + mode;
    double z = ends[((size_t)member * nchunks + chunk) * nn + mode];
    for (int k = k0; k < k1; ++k) {
        z = fma(gm, z, (double)h[(size_t)k * nn]);
        h[(size_t)k * nn] = (T)z;
    }
}

constexpr int REC_CHUNK = 16;   // blocks per scan chunk

template <class T>
size_t fine_smem(int TXp, int TYp, int n) {
    size_t s = 4 * (size_t)TYp * TXp * RX * sizeof(T);
    if (sizeof(T) == 8) s += (size_t)n * n * sizeof(T);
    return s;
}

void tile_shape(int n, int &TX, int &TXp, int &TY, int &TYp) {
    TX = (n + RX - 1) / RX;
    TXp = 1;
    while (TXp < TX) TXp <<= 1;
    TY = (n + RY - 1) / RY;
    const int threads = ((TXp * TY + 31) / 32) * 32;
    TYp = threads / TXp;
}

template <class T>
pit_status launch_fine(Problem *p, Heat2dArgs a, int nslices, cudaStream_t s) {
    int TX, TXp, TY, TYp;
    tile_shape(p->nx, TX, TXp, TY, TYp);
    a.TX = TX;
    a.TXp = TXp;
    a.TY = TY;
    const int threads = TXp * TYp;
    const size_t sm = fine_smem<T>(TXp, TYp, p->nx);
    PIT_CUDA(cudaFuncSetAttribute(k_heat2d_fine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    k_heat2d_fine<T><<<dim3(nslices, p->batch), threads, sm, s>>>(a);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

Heat2dArgs make_args(Problem *p, const double *x, double *y, int mode, const MemberState *st) {
    Heat2dArgs a{};
    a.x = x;
    a.y = y;
    a.y0 = p->y0.as<double>();
    a.n = p->nx;
    a.N = p->N;
    a.batch = p->batch;
    a.blen = p->blen;
    a.n_first = 1;
    a.mode = mode;
    a.steps = p->fine_steps;
    const double h = 1.0 / (p->nx + 1);
    const double dt = p->dT / p->fine_steps;
    const double k = p->nu / (h * h);
    a.c[0] = dt / 4.0 * k;
    a.c[1] = dt / 3.0 * k;
    a.c[2] = dt / 2.0 * k;
    a.c[3] = dt * k;
    a.st = st;
    return a;
}

template <class Tin, class T, class Tout>
pit_status launch_xS(Problem *p, const Tin *A, Tout *out, const T *S, double scale,
                     const MemberState *st, cudaStream_t s) {
    const int n = p->nx;
    const size_t sm = (size_t)n * (n + 4) * sizeof(T) * (sizeof(T) == 4 ? 2 : 1);
    PIT_CUDA(cudaFuncSetAttribute(k_block_xS_T<Tin, T, Tout>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int nblk = p->N + 1;
    k_block_xS_T<Tin, T, Tout><<<nblk * p->batch, PT, sm, s>>>(A, out, S, n, nblk, scale, st);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

template <class T>
pit_status sweep_t(Problem *p, const double *q, double *z, const T *S, const MemberState *st,
                   cudaStream_t s) {
    const int n = p->nx;
    const size_t nn = (size_t)n * n;
    const int nblk = p->N + 1;
    const size_t hat_elems = (size_t)p->batch * nblk * nn;
    const int nchunks = (nblk + REC_CHUNK - 1) / REC_CHUNK;
    const size_t ends_bytes = (size_t)p->batch * nchunks * nn * sizeof(double);
    PIT_TRY(p->hat.ensure(2 * hat_elems * sizeof(T) + ends_bytes));
    T *h1 = p->hat.as<T>();
    T *h2 = h1 + hat_elems;
    double *ends = reinterpret_cast<double *>(h2 + hat_elems);
    // qhat = S q S
    PIT_TRY((launch_xS<double, T, T>(p, q, h1, S, 1.0, st, s)));
    PIT_TRY((launch_xS<T, T, T>(p, h1, h2, S, 1.0, st, s)));
    // recurrence over slices, mode by mode
    const int RT = 256;
    dim3 g1((unsigned)((nn + RT - 1) / RT), nchunks, p->batch);
    k_rec_local<T><<<g1, RT, 0, s>>>(h2, ends, p->gmode.as<double>(), (int)nn, nblk, REC_CHUNK,
                                     nchunks, st);
    PIT_LAUNCH_CHECK();
    k_rec_carry<<<dim3((unsigned)((nn + RT - 1) / RT), p->batch), RT, 0, s>>>(
        ends, p->gmode.as<double>(), (int)nn, REC_CHUNK, nchunks, st);
    PIT_LAUNCH_CHECK();
    k_rec_apply<T><<<g1, RT, 0, s>>>(h2, ends, p->gmode.as<double>(), (int)nn, nblk, REC_CHUNK,
                                     nchunks, st);
    PIT_LAUNCH_CHECK();
    // z = (2/(n+1))^2 S zhat S
    const double sc = 2.0 / (n + 1);
    PIT_TRY((launch_xS<T, T, T>(p, h2, h1, S, sc, st, s)));
    PIT_TRY((launch_xS<T, T, double>(p, h1, z, S, sc, st, s)));
    return PIT_OK;
}

}  // namespace

pit_status heat2d_setup(Problem *p) {
    if (p->nx != p->ny) {
        set_error("heat2d: only square grids (nx == ny) are supported");
        return PIT_E_UNSUPPORTED;
    }
    if (p->fine_kind != PIT_STEP_RK4 || p->coarse_kind != PIT_STEP_IE) {
        set_error("heat2d: fine must be RK4 and coarse implicit Euler");
        return PIT_E_UNSUPPORTED;
    }
    if (p->nx > 128) {
        set_error("heat2d: n > 128 is not supported by the single-CTA slice kernel");
        return PIT_E_UNSUPPORTED;
    }
    const int n = p->nx;
    const double h = 1.0 / (n + 1);
    std::vector<double> S((size_t)n * n);
    std::vector<float> S32((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
            S[(size_t)j * n + k] = sin(M_PI * (double)(j + 1) * (double)(k + 1) / (n + 1));
            S32[(size_t)j * n + k] = (float)S[(size_t)j * n + k];
        }
    std::vector<double> mu(n), g((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        const double sk = sin(M_PI * (k + 1) * h / 2.0);
        mu[k] = -4.0 / (h * h) * sk * sk;
    }
    const double dtc = p->dT / p->coarse_steps;
    for (int l = 0; l < n; ++l)
        for (int k = 0; k < n; ++k)
            g[(size_t)l * n + k] = pow(1.0 - dtc * p->nu * (mu[l] + mu[k]), -(double)p->coarse_steps);
    PIT_TRY(p->S64.ensure(S.size() * sizeof(double)));
    PIT_TRY(p->S32.ensure(S32.size() * sizeof(float)));
    PIT_TRY(p->gmode.ensure(g.size() * sizeof(double)));
    PIT_CUDA(cudaMemcpy(p->S64.ptr, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice));
    PIT_CUDA(cudaMemcpy(p->S32.ptr, S32.data(), S32.size() * sizeof(float), cudaMemcpyHostToDevice));
    PIT_CUDA(cudaMemcpy(p->gmode.ptr, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice));
    return PIT_OK;
}

pit_status heat2d_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                          const MemberState *st, cudaStream_t s) {
    Heat2dArgs a = make_args(p, x, y, mode, st);
    if (prec == PIT_FP64) return launch_fine<double>(p, a, p->N, s);
    return launch_fine<float>(p, a, p->N, s);
}

pit_status heat2d_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s) {
    Heat2dArgs a = make_args(p, x, y - (size_t)p->M, 2, nullptr);
    if (prec == PIT_FP64) return launch_fine<double>(p, a, 1, s);
    return launch_fine<float>(p, a, 1, s);
}

pit_status heat2d_sweep(Problem *p, const double *q, double *z, int prec, const MemberState *st,
                        cudaStream_t s) {
    if (prec == PIT_FP64) return sweep_t<double>(p, q, z, p->S64.as<double>(), st, s);
    return sweep_t<float>(p, q, z, p->S32.as<float>(), st, s);
}

}  // namespace pit
