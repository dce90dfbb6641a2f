// Placeholder for the dense operator family; replaced by the real kernels.
#include "pit_internal.h"

namespace pit {
pit_status dense_setup(Problem *) {
    set_error("dense: not implemented yet");
    return PIT_E_UNSUPPORTED;
}
pit_status dense_apply_F(Problem *, const double *, double *, int, int, const MemberState *,
                          cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
pit_status dense_sweep(Problem *, const double *, double *, int, const MemberState *,
                        cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
pit_status dense_fine_one(Problem *, const double *, double *, int, cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
}  // namespace pit
