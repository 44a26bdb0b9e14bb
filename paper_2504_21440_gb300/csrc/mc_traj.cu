// mcsolve (paper Sec. 3.3): the launch shape for a dimension, the dispatch
// to the trajectory kernel's launchers (defined in mc_traj.cuh and
// instantiated in mc_traj_fp64_*.cu and mc_traj_mixed_*.cu), and the
// fixed-order mean over trajectories.
#include "internal.h"
#include "mc_common.cuh"

namespace qtl {

constexpr int MC_TMAX = 256;

// defined in mc_traj.cuh, instantiated in mc_traj_fp64_*.cu and mc_traj_mixed_*.cu
template <bool MIXED, int RPT, int MAXT, int MINB>
cudaError_t mc_launch_t(const McJob& J, int T, cudaStream_t st);

// Mean over trajectories in a fixed order: one CTA per (e_op, time) pair.
__global__ void mc_reduce_kernel(const double2* __restrict__ traj_expect, double2* __restrict__ expect,
                                 int nrows, int ntraj) {
    __shared__ double sx[32], sy[32];
    for (int rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
        const double2* src = traj_expect + (size_t)rr * ntraj;
        double ax = 0.0, ay = 0.0;
        for (int j = threadIdx.x; j < ntraj; j += blockDim.x) {
            double2 v = src[j];
            ax += v.x;
            ay += v.y;
        }
        ax = mc_warp_sum(ax);
        ay = mc_warp_sum(ay);
        if ((threadIdx.x & 31) == 0) {
            sx[threadIdx.x >> 5] = ax;
            sy[threadIdx.x >> 5] = ay;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tx = 0.0, ty = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                tx += sx[w];
                ty += sy[w];
            }
            expect[rr] = make_double2(tx / ntraj, ty / ntraj);
        }
        __syncthreads();
    }
}

int mc_traj_capacity() { return MC_TMAX * 4; }


// Launch shape: one row per thread up to 256 rows (so a trajectory spreads
// over all four SM sub-partitions), then 2 or 4 rows per thread.  Each shape
// has its own launch bounds so that the register budget keeps 6-8 CTAs of
// 96-128 threads resident per SM.
struct McShape {
    int T, rpt;
};
static McShape mc_shape(int n) {
    if (n <= 256) {
        int T = (n + 31) / 32 * 32;
        return {T < 32 ? 32 : T, 1};
    }
    if (n <= 512) return {256, 2};
    if (n <= 1024) return {256, 4};
    return {0, 0};
}

template <bool MIXED>
static cudaError_t mc_dispatch(const McJob& J, McShape sh, cudaStream_t st) {
    if (sh.rpt == 1 && sh.T <= 128) return mc_launch_t<MIXED, 1, 128, 6>(J, sh.T, st);
    if (sh.rpt == 1) return mc_launch_t<MIXED, 1, 256, 3>(J, sh.T, st);
    if (sh.rpt == 2) return mc_launch_t<MIXED, 2, 256, 2>(J, sh.T, st);
    return mc_launch_t<MIXED, 4, 256, 1>(J, sh.T, st);
}

cudaError_t launch_mc_traj(const McJob& J0, int precision, cudaStream_t st) {
    const McShape sh = mc_shape(J0.n);
    if (sh.T == 0) return cudaErrorInvalidValue;
    // Copy A into shared memory when it fits next to the state buffers.
    McJob J = J0;
    const size_t tv = precision == QTL_MIXED ? sizeof(float2) : sizeof(double2);
    const size_t base = (size_t)J.n * (sizeof(double2) + 2 * tv) + 64 +
                        (size_t)(sh.T / 32 + 1) * mc_red_stride(J.n_e, J.n_c) * sizeof(double);
    // (not with per-trajectory operators: the copy is made once per CTA)
    J.a_smem = !J.tops && base + 16 + (size_t)J.n * sizeof(int4) + (size_t)J.a_nnz * (tv + 4) <= 200 * 1024;
    return precision == QTL_MIXED ? mc_dispatch<true>(J, sh, st) : mc_dispatch<false>(J, sh, st);
}

cudaError_t launch_traj_mean(const double2* traj, double2* out, int nrows, int ntraj, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    count_launch();
    mc_reduce_kernel<<<nrows < 4096 ? nrows : 4096, 256, 0, st>>>(traj, out, nrows, ntraj);
    return cudaGetLastError();
}

cudaError_t launch_mc_reduce(const McJob& J, cudaStream_t st) {
    int nrows = J.n_e * J.nt;
    if (nrows == 0) return cudaSuccess;
    int grid = nrows < 4096 ? nrows : 4096;
    count_launch();
    mc_reduce_kernel<<<grid, 256, 0, st>>>(J.traj_expect, J.expect, nrows, J.ntraj);
    return cudaGetLastError();
}

}  // namespace qtl
