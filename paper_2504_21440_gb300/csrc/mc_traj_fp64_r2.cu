// FP64 launcher of the trajectory kernel (mc_traj.cuh) for
// two rows per thread (256 < n <= 512), instantiated in a translation unit of its
// own so that it compiles in parallel with the other shapes.
#include "mc_traj.cuh"

namespace qtl {

template cudaError_t mc_launch_t<false, 2, 256, 2>(const McJob&, int, cudaStream_t);

}  // namespace qtl
