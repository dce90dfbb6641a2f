// Self-tests of device helpers that replace hardware operations.
#include "pit_internal.h"
#include "stencil_arith.cuh"

namespace pit {
namespace {
__global__ void k_convert_check(const double *in, int n, float *f32, double *back) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float f = d2f_rn(in[i]);
    f32[i] = f;
    back[i] = f2d(f);
}
}  // namespace
}  // namespace pit

extern "C" pit_status pit_selftest_convert(const double *in, int n, float *f32, double *back) {
    using namespace pit;
    if (!in || !f32 || !back || n < 0) {
        set_error("pit_selftest_convert: bad argument");
        return PIT_E_INVALID;
    }
    if (n == 0) return PIT_OK;
    k_convert_check<<<(n + 255) / 256, 256>>>(in, n, f32, back);
    PIT_LAUNCH_CHECK();
    PIT_CUDA(cudaDeviceSynchronize());
    return PIT_OK;
}
