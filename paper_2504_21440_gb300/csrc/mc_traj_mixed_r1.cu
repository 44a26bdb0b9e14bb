// Mixed-precision launchers of the trajectory kernel (mc_traj.cuh) for
// one row per thread (n <= 256), instantiated in a translation unit of
// their own so that they compile in parallel with the other shapes.
#include "mc_traj.cuh"

namespace qtl {

template cudaError_t mc_launch_t<true, 1, 128, 6>(const McJob&, int, cudaStream_t);
template cudaError_t mc_launch_t<true, 1, 256, 3>(const McJob&, int, cudaStream_t);

}  // namespace qtl
