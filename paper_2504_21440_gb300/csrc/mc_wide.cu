// Host side of the wide trajectory kernel (mc_wide.cuh): launch planning,
// scratch layout and the FP64 instantiation.  The mixed-precision
// instantiation is in mc_wide_mixed.cu.
#include "mc_wide.cuh"

namespace qtl {

cudaError_t mw_occupancy_fp64(size_t smem, int xsmem, int* per_sm) {
    return mw_occupancy<false, int32_t>(smem, xsmem, per_sm);
}
void mw_launch_fp64(const McJob& J, const McWidePlan& p, const SellConst& C, cudaStream_t st) {
    mw_launch<false, int32_t>(J, p, C, st);
}

int mc_wide_capacity() { return 1 << 22; }

// Shared memory: the reduction area, then the stage inputs when they fit
// (two buffers if possible, one otherwise; above that they live in scratch).
static void mw_smem_plan(int n, int n_e, int n_c, int precision, int* xsmem, int* xbufs,
                         size_t* smem) {
    const size_t red = ((size_t)(MW_T / 32 + 1) * mc_red_stride(n_e, n_c) + 2) * sizeof(double) + 16;
    const size_t xb = (((size_t)n * (precision == QTL_MIXED ? sizeof(float2) : sizeof(double2))) + 15) &
                      ~(size_t)15;
    if (red + 2 * xb <= MW_SMEM_X_MAX) {
        *xsmem = 1;
        *xbufs = 2;
        *smem = red + 2 * xb;
    } else if (red + xb <= MW_SMEM_X_MAX) {
        *xsmem = 1;
        *xbufs = 1;
        *smem = red + xb;
    } else {
        *xsmem = 0;
        *xbufs = 2;
        *smem = red;
    }
}

cudaError_t mc_wide_plan(const McJob& J, int precision, McWidePlan* p) {
    mw_smem_plan(J.n, J.n_e, J.n_c, precision, &p->xsmem, &p->xbufs, &p->smem);
    int per_sm = 0;
    cudaError_t e = precision == QTL_MIXED ? mw_occupancy_mixed(p->smem, p->xsmem, &per_sm)
                                           : mw_occupancy_fp64(p->smem, p->xsmem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid = per_sm * nsm;
    // QTL_MC_WIDE_CTAS caps the resident trajectories (fewer CTAs keep more
    // of the per-CTA state in L2); unset = one per SM
    if (const char* env = std::getenv("QTL_MC_WIDE_CTAS")) {
        const int cap = std::atoi(env);
        if (cap > 0 && cap < grid) grid = cap;
    }
    if (grid > J.ntraj) grid = J.ntraj;
    p->grid = grid;
    p->stride = mw_vec_bytes(J.n) * (size_t)(MW_NV + (p->xsmem ? 0 : 2));
    p->scratch_bytes = p->stride * (size_t)grid + 256;  // + the trajectory counter
    return cudaSuccess;
}

cudaError_t launch_mc_wide(const McJob& J0, int precision, const McWidePlan& p, void* scratch,
                           const SellConst* cdesc, cudaStream_t st) {
    McJob J = J0;
    J.wscr = (unsigned char*)scratch;
    J.wstride = p.stride;
    J.xsmem = p.xsmem;
    J.xbufs = p.xbufs;
    // the trajectory counter sits after the CTAs' slices
    J.wnext = (int*)((unsigned char*)scratch + p.stride * (size_t)p.grid);
    cudaError_t e = cudaMemsetAsync(J.wnext, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    count_launch();
    // explicit columns are 32-bit (the 16-bit form cut bytes only in
    // explicit groups and doubled the instantiations)
    if (precision == QTL_MIXED)
        mw_launch_mixed(J, p, *cdesc, st);
    else
        mw_launch_fp64(J, p, *cdesc, st);
    return cudaGetLastError();
}

}  // namespace qtl
