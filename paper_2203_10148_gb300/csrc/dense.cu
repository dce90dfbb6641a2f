// Dense-propagator mode: y' = A y with a dense M x M matrix A.
//
// Set-up: the fine propagator of one slice is the one-step matrix raised to
// the number of fine steps by binary powering, Phi = W^m, with W the RK4
// step matrix R(dt A), R(Z) = I + Z + Z^2/2 + Z^3/6 + Z^4/24 (nested form),
// or the implicit-Euler step (I - dt A)^{-1}; the coarse propagator is one
// implicit-Euler step, G = (I - dT A)^{-1}.  Inverses by Newton-Schulz
// iteration X <- X (2I - B X) on B = I - d A from the scaled start
// X = B^T/(|B|_1 |B|_inf).  All are FP64 matrix products (cuBLAS DGEMM, once
// per problem).
//
// Fine batch (the N independent slice problems of eq. (2)): all slices at
// once as one product C = Phi [x_0 ... x_{N-1}], then the shift-subtract of
// eq. (4).  Coarse sweep (eq. (7), right): z_n = q_n + G z_{n-1}, sequential in n.
#include <math.h>

#include <vector>

#include <cublas_v2.h>

#include "pit_internal.h"
#include "stencil_arith.cuh"

namespace pit {
namespace {

#define PIT_CUBLAS(call)                                                      \
    do {                                                                      \
        cublasStatus_t c_ = (call);                                           \
        if (c_ != CUBLAS_STATUS_SUCCESS) {                                    \
            set_error(std::string("cuBLAS error ") + std::to_string((int)c_) + \
                      " in " #call);                                          \
            return PIT_E_CUDA;                                                \
        }                                                                     \
    } while (0)

// Row-major M x M matrices: in cuBLAS' column-major view a buffer holds the
// transpose, so C = A B (row-major) is computed as C^T = B^T A^T.
pit_status mm(cublasHandle_t h, int M, const double *A, const double *B, double *C,
              double alpha = 1.0, double beta = 0.0) {
    PIT_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, M, M, M, &alpha, B, M, A, M, &beta, C, M));
    return PIT_OK;
}

__global__ void k_axpby_identity(double *Y, const double *X, double a, double b, double d, int M) {
    // Y = a X + b Y + d I
    const size_t n = (size_t)M * M;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / M, c = i % M;
        Y[i] = a * X[i] + b * Y[i] + ((r == c) ? d : 0.0);
    }
}

__global__ void k_copy_f32(const double *X, float *Y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        Y[i] = d2f_rn(X[i]);
}

// x = hi + lo, hi = RN32(x), lo = RN32(x - hi): the float-float form of x,
// for an rows_out x Mp array from the rows_src x M row-major X (zero where
// r >= rows_src or c >= M: the padding of the float-float product).
__global__ void k_split_ff(const double *X, float *hi, float *lo, int rows_src, int rows_out, int M,
                           int Mp) {
    const size_t n = (size_t)rows_out * Mp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / Mp, c = i % Mp;
        if (r < (size_t)rows_src && c < (size_t)M) {
            const double x = X[r * M + c];
            const float h = d2f_rn(x);
            hi[i] = h;
            lo[i] = d2f_rn(x - f2d(h));
        } else {
            hi[i] = 0.f;
            lo[i] = 0.f;
        }
    }
}

// ------------------------------------------------ float-float product
// C[g][c] = sum_k X[g][k] Phi[c][k] for the rows g = (member, slice < N) of
// the block vector, with X and Phi as float-float pairs (hi, lo) and the
// sum accumulated in the compensated form of Ogita, Rump and Oishi
// ("Accurate sum and dot product", 2005, Dot2) extended to two-word inputs:
// per term p = RN(ah bh) with its exact error e (FMA), the cross terms
// ah bl + al bh added to e, s <- TwoSum(s, p) with the rounding error of
// the sum and e collected in a second FP32 accumulator; the result is
// s + c in FP64.  Error about eps32 |sum| + (n eps32)^2 sum |x phi|.  The
// arithmetic runs two columns per packed f32x2 instruction.  One 64 x 64
// output tile per CTA of 256 threads (4 x 4 outputs each), K in steps of 16
// staged in shared memory, transposed so a thread's 4 rows / 4 columns are
// one 16-byte load.
constexpr int FG_B = 64, FG_K = 16, FG_T = 256;

// rows of the float-float operands, padded to the product's tile width
int pad_ff(int M) { return (M + FG_B - 1) / FG_B * FG_B; }

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// Xh, Xl: the block vector's rows (batch x (N+1) rows of Mp values, zero
// beyond M); Ph, Pl: Phi as Mp x Mp (zero beyond M); C: rows n < N of every
// member, M columns.  Mp is M rounded up to FG_B.
__global__ void __launch_bounds__(FG_T) k_gemm_ff(const float *__restrict__ Xh, const float *__restrict__ Xl,
                                                  const float *__restrict__ Ph, const float *__restrict__ Pl,
                                                  double *__restrict__ C, int M, int Mp, int N,
                                                  size_t cstride, int rows, const MemberState *st) {
    __shared__ __align__(16) float xs_h[FG_K][FG_B], xs_l[FG_K][FG_B];
    __shared__ __align__(16) float ps_h[FG_K][FG_B], ps_l[FG_K][FG_B];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int g0 = blockIdx.y * FG_B, c0 = blockIdx.x * FG_B;
    // staging: each thread moves 4 values of each operand tile per K step
    const int lr = tid >> 2, lk = (tid & 3) * 4;     // tile row 0..63, k 0..12 step 4
    const int gl = g0 + lr;
    const bool grow_ok = gl < rows;
    const int gmem = grow_ok ? gl / N : 0, gsl = grow_ok ? gl % N : 0;
    const bool live = grow_ok && (st == nullptr || (st[gmem].active && !st[gmem].skip && !st[gmem].half));
    const size_t xrow = ((size_t)gmem * (N + 1) + gsl) * Mp;
    const size_t prow = (size_t)(c0 + lr) * Mp;
    float2 s2[4][2], c2[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            s2[i][j] = make_float2(0.f, 0.f);
            c2[i][j] = make_float2(0.f, 0.f);
        }
    for (int k0 = 0; k0 < Mp; k0 += FG_K) {
        {
            float4 xh = make_float4(0.f, 0.f, 0.f, 0.f), xl = xh;
            if (live) {
                xh = *reinterpret_cast<const float4 *>(Xh + xrow + k0 + lk);
                xl = *reinterpret_cast<const float4 *>(Xl + xrow + k0 + lk);
            }
            const float4 ph = *reinterpret_cast<const float4 *>(Ph + prow + k0 + lk);
            const float4 pl = *reinterpret_cast<const float4 *>(Pl + prow + k0 + lk);
            xs_h[lk][lr] = xh.x; xs_h[lk + 1][lr] = xh.y; xs_h[lk + 2][lr] = xh.z; xs_h[lk + 3][lr] = xh.w;
            xs_l[lk][lr] = xl.x; xs_l[lk + 1][lr] = xl.y; xs_l[lk + 2][lr] = xl.z; xs_l[lk + 3][lr] = xl.w;
            ps_h[lk][lr] = ph.x; ps_h[lk + 1][lr] = ph.y; ps_h[lk + 2][lr] = ph.z; ps_h[lk + 3][lr] = ph.w;
            ps_l[lk][lr] = pl.x; ps_l[lk + 1][lr] = pl.y; ps_l[lk + 2][lr] = pl.z; ps_l[lk + 3][lr] = pl.w;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < FG_K; ++k) {
            const float4 ah = *reinterpret_cast<const float4 *>(&xs_h[k][ty * 4]);
            const float4 al = *reinterpret_cast<const float4 *>(&xs_l[k][ty * 4]);
            const float4 bh = *reinterpret_cast<const float4 *>(&ps_h[k][tx * 4]);
            const float4 bl = *reinterpret_cast<const float4 *>(&ps_l[k][tx * 4]);
            const float2 bh2[2] = {make_float2(bh.x, bh.y), make_float2(bh.z, bh.w)};
            const float2 bl2[2] = {make_float2(bl.x, bl.y), make_float2(bl.z, bl.w)};
            const float ahv[4] = {ah.x, ah.y, ah.z, ah.w};
            const float alv[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 a2 = make_float2(ahv[i], ahv[i]);
                const float2 na2 = make_float2(-ahv[i], -ahv[i]);
                const float2 l2 = make_float2(alv[i], alv[i]);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float2 p = __fmul2_rn(a2, bh2[j]);
                    const float2 ne = __ffma2_rn(na2, bh2[j], p);          // -(exact error of p)
                    const float2 s = __fadd2_rn(s2[i][j], p);               // TwoSum(s, p)
                    const float2 bb = f2sub(s, s2[i][j]);
                    const float2 sig = __fadd2_rn(f2sub(s2[i][j], f2sub(s, bb)), f2sub(p, bb));
                    s2[i][j] = s;
                    float2 c = __fadd2_rn(c2[i][j], sig);
                    c = f2sub(c, ne);
                    c = __ffma2_rn(a2, bl2[j], c);
                    c2[i][j] = __ffma2_rn(l2, bh2[j], c);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int g = g0 + ty * 4 + i;
        if (g >= rows) continue;
        const int mbr = g / N, sl = g % N;
        if (st && !(st[mbr].active && !st[mbr].skip && !st[mbr].half)) continue;
        const int cc = c0 + tx * 4;
        double *crow = C + (size_t)mbr * cstride + (size_t)sl * M + cc;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (cc + 2 * j < M) crow[2 * j] = f2d(s2[i][j].x) + f2d(c2[i][j].x);
            if (cc + 2 * j + 1 < M) crow[2 * j + 1] = f2d(s2[i][j].y) + f2d(c2[i][j].y);
        }
    }
}

// ----------------------------------------------------- FP64 product
// C[g][c] = sum_k X[g][k] Phi[c][k] in FP64 for the rows g = (member,
// slice < N) of the block vector (the FP64 path's fine batch).  One 64 x 64
// output tile per CTA of 256 threads (4 x 4 outputs each), K in steps of 16
// staged in shared memory; bound by GB300's FP64 pipe (2 FMA per clock per
// SM), so plain scalar loads with bounds checks serve any M.
constexpr int DG_B = 64, DG_K = 16, DG_T = 256;

__global__ void __launch_bounds__(DG_T) k_gemm_f64(const double *__restrict__ X,
                                                   const double *__restrict__ P,
                                                   double *__restrict__ C, int M, int N, size_t blen,
                                                   size_t cstride, int rows, const MemberState *st) {
    __shared__ __align__(16) double xs[DG_K][DG_B], ps[DG_K][DG_B];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int g0 = blockIdx.y * DG_B, c0 = blockIdx.x * DG_B;
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    const int gl = g0 + lr;
    const bool grow_ok = gl < rows;
    const int gmem = grow_ok ? gl / N : 0, gsl = grow_ok ? gl % N : 0;
    const bool live = grow_ok && (st == nullptr || (st[gmem].active && !st[gmem].skip && !st[gmem].half));
    const double *xr = X + (size_t)gmem * blen + (size_t)gsl * M;
    const int pc = c0 + lr;
    const double *pr = P + (size_t)(pc < M ? pc : 0) * M;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < M; k0 += DG_K) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + lk + e;
            xs[lk + e][lr] = (live && k < M) ? xr[k] : 0.0;
            ps[lk + e][lr] = (pc < M && k < M) ? pr[k] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < DG_K; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = xs[k][ty * 4 + i];
                b[i] = ps[k][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int g = g0 + ty * 4 + i;
        if (g >= rows) continue;
        const int mbr = g / N, sl = g % N;
        if (st && !(st[mbr].active && !st[mbr].skip && !st[mbr].half)) continue;
        double *crow = C + (size_t)mbr * cstride + (size_t)sl * M;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx * 4 + j;
            if (c < M) crow[c] = acc[i][j];
        }
    }
}

// out_b[i] = add_b[i] + sum_k Mat[i][k] in_b[k] for every member b (FP64, one
// warp per row i, the row's products summed lane-strided then by a fixed
// shuffle tree): one step of the sequential sweep z_n = q_n + G z_{n-1}
// (add = out, which holds q_n) or one slice of the serial fine trajectory
// (add = null).  Mat (M x M, row-major) stays in L2 across the steps.
__global__ void __launch_bounds__(256) k_gemv_f64(const double *__restrict__ Mat, const double *in,
                                                  double *out, const double *add, size_t stride,
                                                  int M, int batch) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= M) return;
    const double *row = Mat + (size_t)i * M;
    for (int b = 0; b < batch; ++b) {
        const double *v = in + (size_t)b * stride;
        double sum = 0.0;
        for (int k = lane; k < M; k += 32) sum = fma(row[k], v[k], sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            const size_t j = (size_t)b * stride + i;
            out[j] = (add ? add[j] : 0.0) + sum;
        }
    }
}

__global__ void k_transpose_scale(const double *X, double *Y, int M, double s) {
    const size_t n = (size_t)M * M;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / M, c = i % M;
        Y[c * M + r] = s * X[i];
    }
}

// |B|_1 and |B|_inf of a row-major matrix (one CTA, fixed order).
__global__ void k_norms_1_inf(const double *B, int M, double *out) {
    __shared__ double sh[2][256];
    double m1 = 0.0, mi = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        double cs = 0.0, rs = 0.0;
        for (int i = 0; i < M; ++i) {
            cs += fabs(B[(size_t)i * M + j]);
            rs += fabs(B[(size_t)j * M + i]);
        }
        m1 = fmax(m1, cs);
        mi = fmax(mi, rs);
    }
    sh[0][threadIdx.x] = m1;
    sh[1][threadIdx.x] = mi;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            a = fmax(a, sh[0][t]);
            b = fmax(b, sh[1][t]);
        }
        out[0] = a;
        out[1] = b;
    }
}

// max |(I - B X)_ij|
__global__ void k_max_abs_dev_identity(const double *P, int M, double *out) {
    __shared__ double sh[256];
    double m = 0.0;
    const size_t n = (size_t)M * M;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t r = i / M, c = i % M;
        m = fmax(m, fabs(((r == c) ? 1.0 : 0.0) - P[i]));
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) a = fmax(a, sh[t]);
        *out = a;
    }
}

// Block-operator rows from the product C (row n-1 of C = F x_{n-1}):
// mode FINE_APPLY: y_n = x_n - C_{n-1}, y_0 = x_0; FINE_RESIDUAL: y_n = C_{n-1} - x_n,
// y_0 = y0 - x_0; mode 2: y_n = C_{n-1} for n = n_first only.
template <class TC>
__global__ void k_dense_rows(const double *x, const TC *C, double *y, const double *y0, int M,
                             int N, size_t blen, size_t cstride, int mode,
                             const MemberState *st) {
    const int b = blockIdx.y;
    if (st && !(st[b].active && !st[b].skip && !st[b].half)) return;
    const size_t total = (size_t)(N + 1) * M;
    const size_t mb = (size_t)b * blen;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t n = i / M, k = i % M;
        double v;
        if (n == 0) v = (mode == FINE_APPLY) ? x[mb + k] : y0[(size_t)b * M + k] - x[mb + k];
        else {
            const double c = (double)C[(size_t)b * cstride + (n - 1) * M + k];
            v = (mode == FINE_APPLY) ? x[mb + i] - c : c - x[mb + i];
        }
        y[mb + i] = v;
    }
}

cublasHandle_t handle(Problem *p) { return reinterpret_cast<cublasHandle_t>(p->blas); }

pit_status grid_for(size_t n, int &blocks) {
    blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    return PIT_OK;
}


// --------------------------------------------------- persistent coarse sweep
// z_n = q_n + G z_{n-1} (eq. (7), right) as an exact chunked scan in one
// cooperative launch.  The N+1 blocks are cut into C chunks of L blocks.
//   phase 1: every chunk runs the recurrence from zero; only its last value
//            w_c is kept (L sequential steps, the C chunks side by side);
//   phase 2: carries e_c = w_{c-1} + G^L e_{c-1} into each chunk, a
//            recurrence of the same form scanned the same way: super-chunks
//            of L2 chunks from zero (L2 steps), their carries with G^(L L2)
//            (C2 - 1 steps), and the re-run from those (L2 steps);
//   phase 3: every chunk re-runs the recurrence from its carry and stores
//            each z_n (L steps).
// With L = round((N+1)^(1/3)) and L2 = round(sqrt(C)) a sweep of N + 1 =
// 4097 blocks takes 80 dependent steps (194 with one level).
// Every CTA keeps `rows` rows of G, G^L and G^(L L2) in shared memory and computes
// those rows of G v for all columns (chunks x members) each step; columns
// live in global memory (read through L2) between steps, separated by a
// grid barrier.  With C = 1 this is the plain sequential sweep.
constexpr int SW_THREADS = 256;
constexpr int SW_MAXROWS = 8;
constexpr long long SW_SPIN_LIMIT = 1LL << 24;   // bounded barrier wait

template <class T>
struct SweepArgs {
    const double *q;
    double *z;
    int M, N, batch;
    size_t blen;
    int L, C, rows;
    int L2, C2;           // carry scan: super-chunks of L2 chunks, C2 of them
    const T *G, *GL, *GLL;
    T *Za, *Zb, *E;
    T *F0, *F1, *Gc;      // carry scan: running super-chunk values (ping-pong), super-chunk carries
    unsigned *bar;        // [0] arrivals at the grid barrier, all barriers counted
    int *err;
    const MemberState *st;
};

// Grid-wide barrier with a bounded wait: every CTA adds one to a counter
// that only grows (a release reduction, no reply awaited) and polls it with
// acquire loads until it holds every CTA's arrivals so far (`target`, the
// barrier's number times the grid size); false when it gave up (error set).
__device__ bool grid_barrier(unsigned *bar, int *err, unsigned target) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long long spins = 0;
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if (++spins > SW_SPIN_LIMIT || ((spins & 63) == 0 && *(volatile int *)err)) {
                atomicExch(err, PIT_E_TIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

template <class T>
__device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

// Partial dot products of this CTA's rows of Gm with column v over
// k in [k0, k1), accumulated into acc (per lane; reduced by the caller).
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int W = 2;
};

__device__ __forceinline__ float4 ldcg16(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double2 ldcg16(const double *p) { return __ldcg(reinterpret_cast<const double2 *>(p)); }
__device__ __forceinline__ float vget(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2 &v, int i) { return i == 0 ? v.x : v.y; }

// Partial dot products of the CTA's SW_MAXROWS rows of Gm (zero-padded)
// with column v over k in [k0, k1), accumulated into acc (per lane; reduced
// by the caller).  16-byte loads when M and the range allow it.
template <class T>
__device__ __forceinline__ void rows_dot(const T *Gm, const T *v, int M, int rows, int k0, int k1,
                                         T (&acc)[SW_MAXROWS]) {
    (void)rows;
    constexpr int W = Vec16<T>::W;
    const int lane = threadIdx.x & 31;
    if ((M % W) == 0 && (k0 % W) == 0 && (k1 % W) == 0) {
        constexpr int U = 4;              // 16-byte column loads in flight per lane
        for (int kb = k0 + W * lane; kb < k1; kb += 32 * W * U) {
            typename Vec16<T>::V xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = kb + 32 * W * u;
                if (k < k1) xv[u] = ldcg16(v + k);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = kb + 32 * W * u;
                if (k < k1) {
#pragma unroll
                    for (int r = 0; r < SW_MAXROWS; ++r) {
                        const typename Vec16<T>::V g =
                            *reinterpret_cast<const typename Vec16<T>::V *>(Gm + (size_t)r * M + k);
#pragma unroll
                        for (int e = 0; e < W; ++e) acc[r] = fma(vget(g, e), vget(xv[u], e), acc[r]);
                    }
                }
            }
        }
        return;
    }
    for (int k = k0 + lane; k < k1; k += 32) {
        const T x = ld_cg(v + k);
#pragma unroll
        for (int r = 0; r < SW_MAXROWS; ++r) acc[r] = fma(Gm[(size_t)r * M + k], x, acc[r]);
    }
}

// out[col][row] = q_blk[row] + (Gm in[col])[row] for this CTA's rows and
// every column col = (member b, chunk c) with blk = c*L + i <= N; columns
// whose chunk has ended (or whose member is inactive) keep their value.
// Warps split the columns, and split k as well when there are fewer columns
// than warps; partial sums meet in shared memory.
// Warps own columns (at least as many columns as warps, M <= 32 x 8 x W,
// M % W == 0), SW_CP at a time: the lanes hold the SW_CP columns in
// registers (eight 16-byte loads per column each), every 16-byte vector of
// the CTA's G rows read from shared memory feeds all SW_CP columns, and lane
// r finishes row r0 + r of each column after a butterfly reduction, so a
// step has no CTA barrier.
constexpr int SW_CP = 4;

template <class T>
__device__ void sweep_step_warpcols(const SweepArgs<T> &a, const T *Gm, const T *in, T *out, int i,
                                    bool from_zero, bool store, int r0) {
    constexpr int NW = SW_THREADS / 32;
    constexpr int W = Vec16<T>::W;
    constexpr int U = 8;
    using V = typename Vec16<T>::V;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = a.batch * a.C;
    const int nvec = a.M / W;                      // 16-byte vectors per column
    const int row = r0 + lane;
    const bool row_ok = lane < a.rows && row < a.M;
    for (int base = warp * SW_CP; base < ncols; base += NW * SW_CP) {
        V x[SW_CP][U];
        double qv[SW_CP];
        bool live[SW_CP];
#pragma unroll
        for (int cp = 0; cp < SW_CP; ++cp) {
            const int col = base + cp;
            const bool ok = col < ncols;
            if (ok && !from_zero) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int vi = lane + 32 * u;
                    if (vi < nvec) x[cp][u] = ldcg16(in + (size_t)col * a.M + (size_t)vi * W);
                }
            }
            const int b = ok ? col / a.C : 0, c = ok ? col % a.C : 0;
            const int blk = c * a.L + i;
            live[cp] = ok && blk <= a.N &&
                       (a.st == nullptr || (a.st[b].active && !a.st[b].skip && !a.st[b].half));
            qv[cp] = (live[cp] && row_ok) ? __ldcg(a.q + (size_t)b * a.blen + (size_t)blk * a.M + row) : 0.0;
        }
        T acc[SW_CP][SW_MAXROWS];
#pragma unroll
        for (int cp = 0; cp < SW_CP; ++cp)
#pragma unroll
            for (int r = 0; r < SW_MAXROWS; ++r) acc[cp][r] = T(0);
        if (!from_zero) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int vi = lane + 32 * u;
                if (vi < nvec) {
#pragma unroll
                    for (int r = 0; r < SW_MAXROWS; ++r) {
                        const V g = *reinterpret_cast<const V *>(Gm + (size_t)r * a.M + (size_t)vi * W);
#pragma unroll
                        for (int cp = 0; cp < SW_CP; ++cp)
#pragma unroll
                            for (int e = 0; e < W; ++e)
                                acc[cp][r] = fma(vget(g, e), vget(x[cp][u], e), acc[cp][r]);
                    }
                }
            }
        }
#pragma unroll
        for (int cp = 0; cp < SW_CP; ++cp)
#pragma unroll
            for (int r = 0; r < SW_MAXROWS; ++r)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[cp][r] += __shfl_xor_sync(0xffffffffu, acc[cp][r], o);
        if (row_ok) {
#pragma unroll
            for (int cp = 0; cp < SW_CP; ++cp) {
                const int col = base + cp;
                if (col >= ncols) continue;
                T val = acc[cp][0];
#pragma unroll
                for (int rr = 1; rr < SW_MAXROWS; ++rr) val = (lane == rr) ? acc[cp][rr] : val;
                T res;
                if (live[cp]) {
                    res = (T)qv[cp] + val;
                    if (store) {
                        const int b = col / a.C, blk = (col % a.C) * a.L + i;
                        a.z[(size_t)b * a.blen + (size_t)blk * a.M + row] = (double)res;
                    }
                } else {
                    res = from_zero ? T(0) : ld_cg(in + (size_t)col * a.M + row);
                }
                __stcg(out + (size_t)col * a.M + row, res);
            }
        }
    }
}

template <class T>
__device__ void sweep_step(const SweepArgs<T> &a, const T *Gm, const T *in, T *out, int i,
                           bool from_zero, bool store, int r0, T *red) {
    constexpr int NW = SW_THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = a.batch * a.C;
    if (ncols >= NW && a.M % Vec16<T>::W == 0 && a.M <= 32 * 8 * Vec16<T>::W) {
        sweep_step_warpcols(a, Gm, in, out, i, from_zero, store, r0);
        return;
    }
    const int S = ncols >= NW ? 1 : NW / ncols;        // k segments per column
    const int per_round = NW / S;                        // columns per round
    const int seg_len = (((a.M + S - 1) / S) + 3) & ~3;
    for (int base = 0; base < ncols; base += per_round) {
        const int cl = warp / S, seg = warp % S;
        const int col = base + cl;
        T acc[SW_MAXROWS];
#pragma unroll
        for (int r = 0; r < SW_MAXROWS; ++r) acc[r] = T(0);
        if (col < ncols && !from_zero) {
            const int k0 = seg * seg_len, k1 = min(a.M, k0 + seg_len);
            rows_dot(Gm, in + (size_t)col * a.M, a.M, a.rows, k0, k1, acc);
        }
#pragma unroll
        for (int r = 0; r < SW_MAXROWS; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < SW_MAXROWS; ++r) red[(cl * NW + seg) * SW_MAXROWS + r] = acc[r];
        }
        __syncthreads();
        // finalize: thread t -> (column in round, row)
        const int t = threadIdx.x;
        if (t < per_round * SW_MAXROWS) {
            const int cl2 = t / SW_MAXROWS, r = t % SW_MAXROWS;
            const int col2 = base + cl2, row = r0 + r;
            if (col2 < ncols && r < a.rows && row < a.M) {
                const int b = col2 / a.C, c = col2 % a.C;
                const int blk = c * a.L + i;
                const bool live = blk <= a.N &&
                    (a.st == nullptr || (a.st[b].active && !a.st[b].skip && !a.st[b].half));
                T val = T(0);
                for (int sg = 0; sg < S; ++sg) val += red[(cl2 * NW + sg) * SW_MAXROWS + r];
                T res;
                if (live) {
                    const size_t at = (size_t)b * a.blen + (size_t)blk * a.M + row;
                    res = (T)a.q[at] + val;
                    if (store) a.z[at] = (double)res;
                } else {
                    res = from_zero ? T(0) : ld_cg(in + (size_t)col2 * a.M + row);
                }
                __stcg(out + (size_t)col2 * a.M + row, res);
            }
        }
        __syncthreads();
    }
}

// out(col, row) = add(col, row) + (Xm in(col))[row] for this CTA's rows and
// every live column col < ncols; in(col) == nullptr reads as zero.  Warps
// split the columns (and k, when there are fewer columns than warps);
// partial sums meet in shared memory.
template <class T, class InF, class AddF, class OutF, class LiveF>
__device__ void gen_step(const T *Xm, int M, int rows, int r0, int ncols, InF in_of, AddF add_of,
                         OutF out_of, LiveF live_of, T *red) {
    constexpr int NW = SW_THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = ncols >= NW ? 1 : NW / ncols;        // k segments per column
    const int per_round = NW / S;                        // columns per round
    const int seg_len = (((M + S - 1) / S) + 3) & ~3;
    for (int base = 0; base < ncols; base += per_round) {
        const int cl = warp / S, seg = warp % S;
        const int col = base + cl;
        T acc[SW_MAXROWS];
#pragma unroll
        for (int r = 0; r < SW_MAXROWS; ++r) acc[r] = T(0);
        if (col < ncols && live_of(col)) {
            const T *v = in_of(col);
            if (v != nullptr) {
                const int k0 = seg * seg_len, k1 = min(M, k0 + seg_len);
                rows_dot(Xm, v, M, rows, k0, k1, acc);
            }
        }
#pragma unroll
        for (int r = 0; r < SW_MAXROWS; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < SW_MAXROWS; ++r) red[(cl * NW + seg) * SW_MAXROWS + r] = acc[r];
        }
        __syncthreads();
        const int t = threadIdx.x;
        if (t < per_round * SW_MAXROWS) {
            const int cl2 = t / SW_MAXROWS, r = t % SW_MAXROWS;
            const int col2 = base + cl2, row = r0 + r;
            if (col2 < ncols && r < rows && row < M && live_of(col2)) {
                T val = T(0);
                for (int sg = 0; sg < S; ++sg) val += red[(cl2 * NW + sg) * SW_MAXROWS + r];
                out_of(col2, row, add_of(col2, row) + val);
            }
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(SW_THREADS, 1) k_dense_sweep(SweepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Gs = reinterpret_cast<T *>(smem_raw);
    T *GLs = Gs + (size_t)SW_MAXROWS * a.M;
    T *GLLs = GLs + (size_t)SW_MAXROWS * a.M;
    T *red = GLLs + (size_t)SW_MAXROWS * a.M;   // (SW_THREADS / 32)^2 * SW_MAXROWS partials
    const int r0 = blockIdx.x * a.rows;
    const unsigned nb = gridDim.x;
    unsigned nbar = 0;   // grid barriers passed
    for (size_t t = threadIdx.x; t < (size_t)SW_MAXROWS * a.M; t += SW_THREADS) {
        const int r = (int)(t / a.M), k = (int)(t % a.M);
        const bool ok = r < a.rows && r0 + r < a.M;     // rows beyond this CTA's share: zero
        Gs[t] = ok ? a.G[(size_t)(r0 + r) * a.M + k] : T(0);
        if (a.C > 1) {
            GLs[t] = ok ? a.GL[(size_t)(r0 + r) * a.M + k] : T(0);
            GLLs[t] = ok ? a.GLL[(size_t)(r0 + r) * a.M + k] : T(0);
        }
    }
    __syncthreads();
    T *in = a.Za, *out = a.Zb;
    if (a.C > 1) {
        // phase 1: chunk-local recurrences from zero
        for (int i = 0; i < a.L; ++i) {
            sweep_step(a, Gs, in, out, i, i == 0, false, r0, red);
            if (!grid_barrier(a.bar, a.err, ++nbar * nb)) return;
            T *t = in; in = out; out = t;
        }
        // phase 2: carries E[c] = u_c + A E[c-1] with A = G^L, u_c = W[c-1] (the
        // end of chunk c-1 from phase 1, columns of `in`), u_0 = 0, E[-1] = 0;
        // itself a chunked scan over super-chunks of L2 chunks:
        //   2a  F[s][k] = u_{s L2 + k} + A F[s][k-1] from F[s][-1] = 0 (L2 steps),
        //   2b  g_s = E[s L2 - 1]: g_0 = 0, g_s = F[s-1][L2-1] + A^L2 g_{s-1} (C2 - 1 steps),
        //   2c  E[s L2 + k] = u_{s L2 + k} + A E[s L2 + k - 1] from g_s (L2 steps).
        const T *W = in;
        const int C = a.C, L2 = a.L2, C2 = a.C2, M = a.M;
        auto member_live = [&](int b) {
            return a.st == nullptr || (a.st[b].active && !a.st[b].skip && !a.st[b].half);
        };
        auto u_of = [&](int b, int c, int row) -> T {
            return c == 0 ? T(0) : ld_cg(W + ((size_t)b * C + c - 1) * M + row);
        };
        T *Fi = a.F0, *Fo = a.F1;
        for (int k = 0; k < L2; ++k) {
            gen_step(GLs, M, a.rows, r0, a.batch * C2,
                     [&](int col) -> const T * { return k == 0 ? nullptr : Fi + (size_t)col * M; },
                     [&](int col, int row) -> T { return u_of(col / C2, (col % C2) * L2 + k, row); },
                     [&](int col, int row, T v) { __stcg(Fo + (size_t)col * M + row, v); },
                     [&](int col) { return (col % C2) * L2 + k < C && member_live(col / C2); }, red);
            if (!grid_barrier(a.bar, a.err, ++nbar * nb)) return;
            // columns whose super-chunk ended keep F[s][last] in Fi: copy forward
            // (only full super-chunks feed 2b, so the partial last one needs no copy)
            T *t = Fi; Fi = Fo; Fo = t;
        }
        // Fi: F[s][L2-1] for every full super-chunk s
        for (int sc = 1; sc < C2; ++sc) {
            gen_step(GLLs, M, a.rows, r0, a.batch,
                     [&](int b) -> const T * { return sc == 1 ? nullptr : a.Gc + ((size_t)b * C2 + sc - 1) * M; },
                     [&](int b, int row) -> T { return ld_cg(Fi + ((size_t)b * C2 + sc - 1) * M + row); },
                     [&](int b, int row, T v) { __stcg(a.Gc + ((size_t)b * C2 + sc) * M + row, v); },
                     [&](int b) { return member_live(b); }, red);
            if (!grid_barrier(a.bar, a.err, ++nbar * nb)) return;
        }
        for (int k = 0; k < L2; ++k) {
            gen_step(GLs, M, a.rows, r0, a.batch * C2,
                     [&](int col) -> const T * {
                         const int b = col / C2, sc = col % C2, c = sc * L2 + k;
                         if (k > 0) return a.E + ((size_t)b * C + c - 1) * M;
                         return sc == 0 ? nullptr : a.Gc + ((size_t)b * C2 + sc) * M;
                     },
                     [&](int col, int row) -> T { return u_of(col / C2, (col % C2) * L2 + k, row); },
                     [&](int col, int row, T v) {
                         const int b = col / C2, c = (col % C2) * L2 + k;
                         __stcg(a.E + ((size_t)b * C + c) * M + row, v);
                     },
                     [&](int col) { return (col % C2) * L2 + k < C && member_live(col / C2); }, red);
            if (!grid_barrier(a.bar, a.err, ++nbar * nb)) return;
        }
        // phase 3 starts from the carries
        in = a.E;
        out = a.Za;
    }
    // phase 3: re-run every chunk from its carry (zero when C = 1), storing z
    T *ping = a.Za, *pong = a.Zb;
    for (int i = 0; i < a.L; ++i) {
        sweep_step(a, Gs, in, out, i, a.C == 1 && i == 0, true, r0, red);
        if (!grid_barrier(a.bar, a.err, ++nbar * nb)) return;
        in = out;
        out = (out == ping) ? pong : ping;
    }
}

}  // namespace

pit_status dense_setup(Problem *p) {
    if ((p->fine_kind != PIT_STEP_RK4 && p->fine_kind != PIT_STEP_IE) || p->coarse_kind != PIT_STEP_IE) {
        set_error("dense: fine must be RK4 or implicit Euler (precomputed propagator), coarse implicit Euler");
        return PIT_E_UNSUPPORTED;
    }
    const int M = p->M;
    const size_t mm2 = (size_t)M * M;
    cublasHandle_t h = nullptr;
    PIT_CUBLAS(cublasCreate(&h));
    p->blas = h;
    PIT_CUBLAS(cublasSetStream(h, p->stream));
    PIT_CUBLAS(cublasSetMathMode(h, CUBLAS_DEFAULT_MATH));
    DevBuf work;
    PIT_TRY(work.ensure(5 * mm2 * sizeof(double) + 64));
    double *A = p->PhiF64.as<double>();      // staged by pit_problem_create
    PIT_TRY(p->A64.ensure(mm2 * sizeof(double)));
    PIT_CUDA(cudaMemcpyAsync(p->A64.ptr, A, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    double *T1 = work.as<double>(), *T2 = T1 + mm2, *T3 = T2 + mm2, *T4 = T3 + mm2;
    double *T5 = T4 + mm2;
    double *scal = T5 + mm2;
    int blocks;
    grid_for(mm2, blocks);
    cudaStream_t s = p->stream;
    // (I - d A)^{-1} by Newton-Schulz iteration into `out` (work: T1..T4)
    auto ns_inverse = [&](double d, double *out) -> pit_status {
        double *Bm = T1, *X = T2, *P = T3, *Xn = T4;
        PIT_CUDA(cudaMemsetAsync(Bm, 0, mm2 * sizeof(double), s));
        k_axpby_identity<<<blocks, 256, 0, s>>>(Bm, A, -d, 0.0, 1.0, M);   // B = I - d A
        PIT_LAUNCH_CHECK();
        k_norms_1_inf<<<1, 256, 0, s>>>(Bm, M, scal);
        PIT_LAUNCH_CHECK();
        double nrm[2];
        PIT_CUDA(cudaMemcpyAsync(nrm, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PIT_CUDA(cudaStreamSynchronize(s));
        k_transpose_scale<<<blocks, 256, 0, s>>>(Bm, X, M, 1.0 / (nrm[0] * nrm[1]));
        PIT_LAUNCH_CHECK();
        bool ok = false;
        double prev = 1e300;
        for (int it = 0; it < 200; ++it) {
            PIT_TRY(mm(h, M, Bm, X, P));                       // P = B X
            k_max_abs_dev_identity<<<1, 256, 0, s>>>(P, M, scal);
            PIT_LAUNCH_CHECK();
            double dev;
            PIT_CUDA(cudaMemcpyAsync(&dev, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
            PIT_CUDA(cudaStreamSynchronize(s));
            if (!(dev < 1e300)) break;
            // converged: at the rounding floor (no longer halving) or tiny
            if (dev < 1e-15 * M || (dev < 1e-10 && dev > 0.5 * prev)) {
                ok = true;
                break;
            }
            prev = dev;
            k_axpby_identity<<<blocks, 256, 0, s>>>(P, P, -1.0, 0.0, 2.0, M);   // P = 2I - B X
            PIT_LAUNCH_CHECK();
            PIT_TRY(mm(h, M, X, P, Xn));                       // X <- X (2I - B X)
            std::swap(X, Xn);
        }
        if (!ok) {
            set_error("dense: Newton-Schulz inverse of I - dt A did not converge");
            return PIT_E_INVALID;
        }
        PIT_CUDA(cudaMemcpyAsync(out, X, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return PIT_OK;
    };
    // G = (I - dTc A)^{-c}: the inverse, then its c-th power
    PIT_TRY(p->G64.ensure(mm2 * sizeof(double)));
    double *G = p->G64.as<double>();
    {
        PIT_TRY(ns_inverse(p->dT / p->coarse_steps, T5));
        double *X = T5, *P = T1;
        PIT_CUDA(cudaMemcpyAsync(G, X, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int c = 1; c < p->coarse_steps; ++c) {
            PIT_TRY(mm(h, M, G, X, P));
            PIT_CUDA(cudaMemcpyAsync(G, P, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
    }
    // Phi = W^m with the one-step matrix W: RK4, R(dt A) with
    // R(Z) = I + Z (I + Z/2 (I + Z/3 (I + Z/4))); implicit Euler, (I - dt A)^{-1}
    {
        const double dt = p->dT / p->fine_steps;
        double *R = T1, *W = T2, *Base = T3, *Res = T4;
        if (p->fine_kind == PIT_STEP_IE) {
            PIT_TRY(ns_inverse(dt, T5));
            W = T5;
        } else {
            // W = I + (dt/4) A
            PIT_CUDA(cudaMemsetAsync(W, 0, mm2 * sizeof(double), s));
            k_axpby_identity<<<blocks, 256, 0, s>>>(W, A, dt / 4.0, 0.0, 1.0, M);
            PIT_LAUNCH_CHECK();
            const double coef[3] = {dt / 3.0, dt / 2.0, dt};
            for (int k = 0; k < 3; ++k) {
                // W <- I + coef_k A W
                PIT_TRY(mm(h, M, A, W, R, coef[k], 0.0));
                PIT_CUDA(cudaMemsetAsync(W, 0, mm2 * sizeof(double), s));
                k_axpby_identity<<<blocks, 256, 0, s>>>(W, R, 1.0, 0.0, 1.0, M);
                PIT_LAUNCH_CHECK();
            }
        }
        // binary powering of W to the m-th power
        PIT_CUDA(cudaMemcpyAsync(Base, W, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PIT_CUDA(cudaMemsetAsync(Res, 0, mm2 * sizeof(double), s));
        k_axpby_identity<<<blocks, 256, 0, s>>>(Res, Res, 0.0, 0.0, 1.0, M);   // Res = I
        PIT_LAUNCH_CHECK();
        int m = p->fine_steps;
        while (m > 0) {
            if (m & 1) {
                PIT_TRY(mm(h, M, Res, Base, R));
                std::swap(Res, R);
            }
            m >>= 1;
            if (m) {
                PIT_TRY(mm(h, M, Base, Base, R));
                std::swap(Base, R);
            }
        }
        PIT_CUDA(cudaMemcpyAsync(p->PhiF64.ptr, Res, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    // G^L and G^(L L2) for the chunked sweep of the mixed path: chunks of
    // L = round((N + 1)^(1/3)) blocks, their carries scanned in super-chunks
    // of L2 = round(sqrt(C)) chunks (about 2L + 2 L2 + C / L2 dependent steps)
    {
        int L = std::max(1, (int)lround(cbrt((double)(p->N + 1))));
        const int C = (p->N + L) / L;
        const int L2 = std::max(1, (int)lround(sqrt((double)C)));
        p->sweep_L = L;
        p->sweep_L2 = L2;
        double *Res = T1, *Base = T2, *R = T3;
        PIT_CUDA(cudaMemcpyAsync(Base, G, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PIT_CUDA(cudaMemsetAsync(Res, 0, mm2 * sizeof(double), s));
        k_axpby_identity<<<blocks, 256, 0, s>>>(Res, Res, 0.0, 0.0, 1.0, M);
        PIT_LAUNCH_CHECK();
        while (L > 0) {
            if (L & 1) {
                PIT_TRY(mm(h, M, Res, Base, R));
                std::swap(Res, R);
            }
            L >>= 1;
            if (L) {
                PIT_TRY(mm(h, M, Base, Base, R));
                std::swap(Base, R);
            }
        }
        PIT_TRY(p->GL32.ensure(mm2 * sizeof(float)));
        k_copy_f32<<<blocks, 256, 0, s>>>(Res, p->GL32.as<float>(), mm2);
        PIT_LAUNCH_CHECK();
        // (G^L)^L2 by binary powering from Base2 = G^L (T4, T5 and the two of
        // T1..T3 that do not hold G^L are free here)
        double *Base2 = T4, *Res2 = T5, *R2 = (Res == T1) ? T2 : T1;
        PIT_CUDA(cudaMemcpyAsync(Base2, Res, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PIT_CUDA(cudaMemsetAsync(Res2, 0, mm2 * sizeof(double), s));
        k_axpby_identity<<<blocks, 256, 0, s>>>(Res2, Res2, 0.0, 0.0, 1.0, M);
        PIT_LAUNCH_CHECK();
        int e = L2;
        while (e > 0) {
            if (e & 1) {
                PIT_TRY(mm(h, M, Res2, Base2, R2));
                std::swap(Res2, R2);
            }
            e >>= 1;
            if (e) {
                PIT_TRY(mm(h, M, Base2, Base2, R2));
                std::swap(Base2, R2);
            }
        }
        PIT_TRY(p->GLL32.ensure(mm2 * sizeof(float)));
        k_copy_f32<<<blocks, 256, 0, s>>>(Res2, p->GLL32.as<float>(), mm2);
        PIT_LAUNCH_CHECK();
    }
    // The tensor-core sweep of the mixed path (one member, M <= 1024): G and
    // A_s = G^(L 2^s), s < S, as TF32 (hi, lo) parts, A_0 = G^L by binary
    // powering and A_s = A_{s-1}^2 (T1..T5 are free here).  PIT_DENSE_SWEEP_TC=0
    // keeps the CUDA-core sweep.
    p->dtc_on = false;
    if (!(getenv("PIT_DENSE_SWEEP_TC") && getenv("PIT_DENSE_SWEEP_TC")[0] == '0') &&
        dense_tc_sweep_fits(p)) {
        int L, C, S;
        dense_tc_sweep_shape(p->N, L, C, S);
        const int Mp = dense_tc_sweep_padded(M);
        const size_t mp2 = (size_t)Mp * Mp;
        if (S <= DTC_SMAX) {
            PIT_TRY(p->dtc_mats.ensure((size_t)(2 + 2 * S) * mp2 * sizeof(float)));
            float *mats = p->dtc_mats.as<float>();
            PIT_TRY(tc_split_tf32(G, mats, mats + mp2, M, Mp, M, Mp, s));
            double *Res = T1, *Base = T2, *R = T3;
            PIT_CUDA(cudaMemcpyAsync(Base, G, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
            PIT_CUDA(cudaMemsetAsync(Res, 0, mm2 * sizeof(double), s));
            k_axpby_identity<<<blocks, 256, 0, s>>>(Res, Res, 0.0, 0.0, 1.0, M);
            PIT_LAUNCH_CHECK();
            for (int e = L; e > 0;) {
                if (e & 1) {
                    PIT_TRY(mm(h, M, Res, Base, R));
                    std::swap(Res, R);
                }
                e >>= 1;
                if (e) {
                    PIT_TRY(mm(h, M, Base, Base, R));
                    std::swap(Base, R);
                }
            }
            for (int k = 0; k < S; ++k) {
                if (k > 0) {
                    PIT_TRY(mm(h, M, Res, Res, R));
                    std::swap(Res, R);
                }
                PIT_TRY(tc_split_tf32(Res, mats + (size_t)(2 + 2 * k) * mp2,
                                      mats + (size_t)(3 + 2 * k) * mp2, M, Mp, M, Mp, s));
            }
            const size_t bytes = 6 * (size_t)128 * Mp * sizeof(float) + 64;
            PIT_TRY(p->dtc_buf.ensure(bytes));
            PIT_CUDA(cudaMemsetAsync(p->dtc_buf.ptr, 0, bytes, s));
            p->dtc_on = true;
        }
    }
    // FP32 copies for the mixed path; Phi also as float-float (hi, lo) for
    // the residual product
    {
        const int Mp = pad_ff(M);
        const size_t mp2 = (size_t)Mp * Mp;
        PIT_TRY(p->PhiF_hi.ensure(mp2 * sizeof(float)));
        PIT_TRY(p->PhiF_lo.ensure(mp2 * sizeof(float)));
        k_split_ff<<<1024, 256, 0, s>>>(p->PhiF64.as<double>(), p->PhiF_hi.as<float>(),
                                        p->PhiF_lo.as<float>(), M, Mp, M, Mp);
        PIT_LAUNCH_CHECK();
    }
    PIT_TRY(p->G32.ensure(mm2 * sizeof(float)));
    k_copy_f32<<<blocks, 256, 0, s>>>(G, p->G32.as<float>(), mm2);
    PIT_LAUNCH_CHECK();
    // TF32 splits of Phi for the tensor-core product
    p->use_tc = dense_tc_supported(p);
    if (p->use_tc) PIT_TRY(dense_tc_split_phi(p));
    // digit slices of Phi for the true residual by error-free splitting
    // (PIT_DENSE_OZ=0: the float-float product instead)
    p->oz_on = dense_oz_supported(p) && !(getenv("PIT_DENSE_OZ") && getenv("PIT_DENSE_OZ")[0] == '0');
    if (p->oz_on) PIT_TRY(dense_oz_setup(p));
    PIT_CUDA(cudaStreamSynchronize(s));
    work.release();
    return PIT_OK;
}

// C (batch x N x M, row n = Phi x_n for n < N, FP64): the float-float
// compensated product (PIT_FF; PIT_MIXED too when the tensor-core product is
// unavailable) or the FP64 product, both hand-written kernels.
static pit_status dense_product(Problem *p, const double *x, int prec, const MemberState *st,
                                cudaStream_t s) {
    const int M = p->M, N = p->N;
    const size_t cstride = (size_t)N * M;
    const int rows = p->batch * N;
    PIT_TRY(p->dense_scratch.ensure((size_t)p->batch * cstride * sizeof(double)));
    if (prec != PIT_FP64) {
        // X split once into padded float-float rows, then the compensated GEMM
        const int Mp = pad_ff(M), R = p->batch * (N + 1);
        const size_t n = (size_t)R * Mp;
        PIT_TRY(p->q32.ensure(2 * n * sizeof(float)));
        float *xh = p->q32.as<float>(), *xl = xh + n;
        k_split_ff<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(x, xh, xl, R, R, M,
                                                                                     Mp);
        PIT_LAUNCH_CHECK();
        dim3 grid((unsigned)(Mp / FG_B), (unsigned)((rows + FG_B - 1) / FG_B));
        k_gemm_ff<<<grid, FG_T, 0, s>>>(xh, xl, p->PhiF_hi.as<float>(), p->PhiF_lo.as<float>(),
                                        p->dense_scratch.as<double>(), M, Mp, N, cstride, rows, st);
        PIT_LAUNCH_CHECK();
        return PIT_OK;
    }
    dim3 grid((unsigned)((M + DG_B - 1) / DG_B), (unsigned)((rows + DG_B - 1) / DG_B));
    k_gemm_f64<<<grid, DG_T, 0, s>>>(x, p->PhiF64.as<double>(), p->dense_scratch.as<double>(), M, N,
                                     p->blen, cstride, rows, st);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

pit_status dense_apply_F(Problem *p, const double *x, double *y, int mode, int prec,
                         const MemberState *st, cudaStream_t s) {
    if (prec == PIT_MIXED && p->use_tc) return dense_tc_apply(p, x, y, nullptr, mode, st, s);
    if (prec == PIT_SPLIT) {
        if (p->oz_on) return dense_oz_apply(p, x, y, mode, st, s);
        prec = PIT_FF;
    }
    // (the source rows of a residual are added by the caller)
    PIT_TRY(dense_product(p, x, prec, st, s));
    int blocks;
    grid_for(p->blen, blocks);
    const size_t cstride = (size_t)p->N * p->M;
    k_dense_rows<double><<<dim3(blocks, p->batch), 256, 0, s>>>(
        x, p->dense_scratch.as<double>(), y, p->y0.as<double>(), p->M, p->N, p->blen, cstride,
        mode, st);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

pit_status dense_fine_one(Problem *p, const double *x, double *y, int prec, cudaStream_t s) {
    // y (block n) = Phi x (block n-1) for every member; FP64
    (void)prec;
    const int M = p->M;
    k_gemv_f64<<<(M + 7) / 8, 256, 0, s>>>(p->PhiF64.as<double>(), x, y, nullptr, p->blen, M, p->batch);
    PIT_LAUNCH_CHECK();
    return PIT_OK;
}

// Steady states y* with A y* = -f for every member (f_host, ys_host: batch
// x M): LU factorisation of A with partial pivoting (cuBLAS, FP64) and two
// triangular solves per member.
pit_status dense_steady_state(Problem *p, const double *f_host, double *ys_host) {
    const int M = p->M, B = p->batch;
    const size_t mm2 = (size_t)M * M;
    cublasHandle_t h = handle(p);
    cudaStream_t s = p->stream;
    PIT_CUBLAS(cublasSetStream(h, s));
    DevBuf lu, rhs, piv, ptrs, info;
    PIT_TRY(lu.ensure(mm2 * sizeof(double)));
    PIT_TRY(rhs.ensure((size_t)B * M * sizeof(double)));
    PIT_TRY(piv.ensure((size_t)M * sizeof(int)));
    PIT_TRY(ptrs.ensure(2 * sizeof(double *)));
    PIT_TRY(info.ensure(sizeof(int)));
    // row-major A is the column-major A^T: factor A^T and solve A^T' y = b
    // with the transposed solve (op = T)
    PIT_CUDA(cudaMemcpyAsync(lu.ptr, p->A64.ptr, mm2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<double> negf((size_t)B * M);
    for (size_t i = 0; i < negf.size(); ++i) negf[i] = -f_host[i];
    PIT_CUDA(cudaMemcpyAsync(rhs.ptr, negf.data(), negf.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    double *hp[2] = {lu.as<double>(), rhs.as<double>()};
    PIT_CUDA(cudaMemcpyAsync(ptrs.ptr, hp, sizeof hp, cudaMemcpyHostToDevice, s));
    double **dA = reinterpret_cast<double **>(ptrs.ptr);
    PIT_CUBLAS(cublasDgetrfBatched(h, M, dA, M, piv.as<int>(), info.as<int>(), 1));
    int hinfo = 0;
    PIT_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    if (hinfo != 0) {
        set_error("dense: A is singular, the source has no steady state");
        return PIT_E_UNSUPPORTED;
    }
    int sinfo = 0;
    PIT_CUBLAS(cublasDgetrsBatched(h, CUBLAS_OP_T, M, B, dA, M, piv.as<int>(), dA + 1, M, &sinfo, 1));
    PIT_CUDA(cudaMemcpyAsync(ys_host, rhs.ptr, (size_t)B * M * sizeof(double), cudaMemcpyDeviceToHost, s));
    PIT_CUDA(cudaStreamSynchronize(s));
    if (sinfo != 0) {
        set_error("dense: steady-state solve failed");
        return PIT_E_CUDA;
    }
    return PIT_OK;
}

void dense_teardown(Problem *p) {
    if (p->blas) cublasDestroy(handle(p));
    p->blas = nullptr;
}

template <class T>
static pit_status persistent_sweep(Problem *p, const double *q, double *z, const T *G, const T *GL,
                                   const T *GLL, int L, int C, int L2, const MemberState *st,
                                   cudaStream_t s, bool *launched) {
    *launched = false;
    int dev = 0, sms = 0, coop = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PIT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const int M = p->M;
    const int rows = (M + sms - 1) / sms;
    if (!coop || rows > SW_MAXROWS) return PIT_OK;            // caller falls back
    const int grid = (M + rows - 1) / rows;
    const size_t smem = (3 * (size_t)SW_MAXROWS * M + (size_t)SW_MAXROWS * 64) * sizeof(T);
    if (smem > 200 * 1024) return PIT_OK;
    PIT_TRY(smem_limit(k_dense_sweep<T>, smem));
    int per_sm = 0;
    PIT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_sweep<T>, SW_THREADS,
                                                           smem));
    if (per_sm * sms < grid) return PIT_OK;
    const int C2 = (C + L2 - 1) / L2;
    const size_t ncols = (size_t)p->batch * C;
    const size_t ncols2 = (size_t)p->batch * C2;
    const size_t colbytes = ncols * M * sizeof(T);
    const size_t colbytes2 = ncols2 * M * sizeof(T);
    PIT_TRY(p->hat.ensure(3 * colbytes + 3 * colbytes2 + 64));
    T *Za = p->hat.as<T>();
    T *Zb = Za + ncols * M;
    T *E = Zb + ncols * M;
    T *F0 = E + ncols * M;
    T *F1 = F0 + ncols2 * M;
    T *Gc = F1 + ncols2 * M;
    unsigned *bar = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(p->hat.ptr) + 3 * colbytes +
                                                 3 * colbytes2);
    PIT_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    SweepArgs<T> a{q, z, M, p->N, p->batch, p->blen, L, C, rows, L2, C2, G, GL, GLL, Za, Zb, E,
                   F0, F1, Gc, bar, p->errword.as<int>(), st};
    void *args[] = {&a};
    PIT_CUDA(cudaLaunchCooperativeKernel((const void *)k_dense_sweep<T>, dim3(grid), dim3(SW_THREADS),
                                         args, smem, s));
    PIT_LAUNCH_CHECK();
    *launched = true;
    return PIT_OK;
}

pit_status dense_sweep(Problem *p, const double *q, double *z, int prec, const MemberState *st,
                       cudaStream_t s) {
    bool done = false;
    if (prec == PIT_MIXED && p->dtc_on) {
        PIT_TRY(dense_tc_sweep(p, q, z, st, s, &done));
        if (done) return PIT_OK;
    }
    if (prec == PIT_MIXED) {
        const int L = p->sweep_L, C = (p->N + L) / L;   // ceil((N + 1) / L)
        PIT_TRY(persistent_sweep<float>(p, q, z, p->G32.as<float>(), p->GL32.as<float>(),
                                        p->GLL32.as<float>(), L, C, p->sweep_L2, st, s, &done));
    } else {
        PIT_TRY(persistent_sweep<double>(p, q, z, p->G64.as<double>(), nullptr, nullptr, p->N + 1, 1,
                                         1, st, s, &done));
    }
    if (done) return PIT_OK;
    // grids too large for the persistent sweep (M above about 1000 in FP64):
    // one FP64 matrix-vector step per slice, z_n = q_n + G z_{n-1}
    const int M = p->M;
    if (q != z)
        PIT_CUDA(cudaMemcpyAsync(z, q, p->vlen * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int n = 1; n <= p->N; ++n) {
        double *zn = z + (size_t)n * M;
        k_gemv_f64<<<(M + 7) / 8, 256, 0, s>>>(p->G64.as<double>(), z + (size_t)(n - 1) * M, zn, zn,
                                               p->blen, M, p->batch);
        PIT_LAUNCH_CHECK();
    }
    return PIT_OK;
}

}  // namespace pit
