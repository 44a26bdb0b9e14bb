// FP64 launcher of the trajectory kernel (mc_traj.cuh) for
// four rows per thread (512 < n <= 1024), instantiated in a translation unit of its
// own so that it compiles in parallel with the other shapes.
#include "mc_traj.cuh"

namespace qtl {

template cudaError_t mc_launch_t<false, 4, 256, 1>(const McJob&, int, cudaStream_t);

}  // namespace qtl
