// Mixed-precision instantiation of the wide trajectory kernel (mc_wide.cuh),
// a translation unit of its own so that it compiles in parallel with the
// FP64 one.
#include "mc_wide.cuh"

namespace qtl {

cudaError_t mw_occupancy_mixed(size_t smem, int xsmem, int* per_sm) {
    return mw_occupancy<true, int32_t>(smem, xsmem, per_sm);
}
void mw_launch_mixed(const McJob& J, const McWidePlan& p, const SellConst& C, cudaStream_t st) {
    mw_launch<true, int32_t>(J, p, C, st);
}

}  // namespace qtl
