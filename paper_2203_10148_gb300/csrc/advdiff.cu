// Placeholder for the advdiff operator family; replaced by the real kernels.
#include "pit_internal.h"

namespace pit {
pit_status advdiff_setup(Problem *) {
    set_error("advdiff: not implemented yet");
    return PIT_E_UNSUPPORTED;
}
pit_status advdiff_apply_F(Problem *, const double *, double *, int, int, const MemberState *,
                          cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
pit_status advdiff_sweep(Problem *, const double *, double *, int, const MemberState *,
                        cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
pit_status advdiff_fine_one(Problem *, const double *, double *, int, cudaStream_t) {
    return PIT_E_UNSUPPORTED;
}
}  // namespace pit
