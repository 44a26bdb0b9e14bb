// mcsolve without any device allocation (qtl_mcsolve_noalloc).
//
// Some callers cannot allocate device memory at solve time: code running
// while a CUDA stream is being captured into a graph (cudaMalloc is not
// allowed there), a process whose device memory is handed out entirely by
// another allocator (a framework's caching allocator, a fixed memory
// budget), or a latency-critical loop that may not wait on the driver's
// allocator.  For them this entry point runs the trajectory kernel with every
// operator passed in as caller-owned device CSR arrays and with its scratch
// (per-trajectory expectation values, the row-segment table and the FP32
// operator copy) placed in one file-scope device array of fixed size instead
// of memory from cudaMalloc / cudaMallocAsync.
//
// The array costs QTL_NOALLOC_SCRATCH_BYTES of device memory on every GPU
// that loads the library, for as long as the process lives.  Every call uses
// the same array and leaves its contents behind, so two calls that overlap on
// the GPU (on different streams, or from different host threads) race on it;
// callers must order them.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace qtl {

// The scratch.  In host code this name is only a host-side stand-in: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QTL_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
static qtl_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    if (dev < 0 || dev >= 64) return QTL_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_cuda_error(e);
            return QTL_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return QTL_OK;
}

// Row segments for plain CSR rows (every entry in the complex group) and,
// for the mixed precision, the complex64 copy of A.  Block 0 also checks A's
// structure (row pointers from 0 to a_nnz, non-decreasing, columns in
// [0, n)); a malformed A sets info->status = QTL_EINVAL and gets empty row
// segments, so the trajectory kernel that follows reads nothing outside the
// caller's arrays.  n <= 1024, so one block holds a thread per row.
__global__ void noalloc_prep_kernel(int n, const int32_t* __restrict__ rp,
                                    const int32_t* __restrict__ ci, int4* __restrict__ seg,
                                    int64_t nnz, const double2* __restrict__ a64,
                                    float2* __restrict__ a32, qtl_device_info* info) {
    if (blockIdx.x == 0) {
        bool bad = false;
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const int b = rp[r], e = rp[r + 1];
            if (b < 0 || e < b || e > nnz || (r == 0 && b != 0) || (r == n - 1 && e != nnz)) {
                bad = true;
                continue;
            }
            for (int p = b; p < e; ++p)
                if (ci[p] < 0 || ci[p] >= n) bad = true;
        }
        bad = __syncthreads_or(bad);
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const int b = bad ? 0 : rp[r];
            seg[r] = make_int4(b, b, b, bad ? 0 : rp[r + 1]);
        }
        if (bad && threadIdx.x == 0) atomicCAS((int*)&info->status, 0, (int)QTL_EINVAL);
    }
    if (a32) {
        const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t p = i0; p < nnz; p += stride) a32[p] = make_float2((float)a64[p].x, (float)a64[p].y);
    }
}

}  // namespace qtl

using namespace qtl;

extern "C" qtl_status qtl_mcsolve_noalloc(
    int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx, const qtl_c128* a_vals,
    int64_t a_nnz, int32_t n_c, const int32_t* c_row_ptr, const int32_t* c_col_idx,
    const qtl_c128* c_vals, int32_t n_e, const int32_t* o_row_ptr, const int32_t* o_col_idx,
    const qtl_c128* o_vals, const qtl_c128* psi0, const double* tlist, int32_t nt, int32_t ntraj,
    uint64_t seed, int64_t traj_offset, const qtl_opts* opts, qtl_c128* expect,
    qtl_device_info* info) {
    if (n > mc_traj_capacity()) return QTL_ETOOBIG;
    if (n < 1 || !a_row_ptr || a_nnz < 0 || a_nnz >= INT32_MAX ||
        (a_nnz > 0 && (!a_col_idx || !a_vals)) || n_c < 0 || n_c > 64 || n_e < 0 || n_e > 64 ||
        (n_c > 0 && (!c_row_ptr || !c_col_idx || !c_vals)) ||
        (n_e > 0 && (!o_row_ptr || !o_col_idx || !o_vals || !expect)) || !psi0 || !tlist ||
        nt < 1 || ntraj < 1 || traj_offset < 0 || !info)
        return QTL_EINVAL;
    qtl_status st = validate_opts(opts);
    if (st != QTL_OK) return st;
    // scratch layout: [segments n x 16 B][complex64 A (mixed)][expectations]
    const bool mixed = opts->precision == QTL_MIXED;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t seg_b = up((size_t)n * sizeof(int4));
    const size_t a32_b = mixed ? up((size_t)a_nnz * sizeof(float2)) : 0;
    const size_t ex_b = (size_t)n_e * nt * ntraj * sizeof(double2);
    if (seg_b + a32_b + ex_b > (size_t)QTL_NOALLOC_SCRATCH_BYTES) return QTL_ETOOBIG;
    void* base = nullptr;
    if ((st = noalloc_scratch(&base)) != QTL_OK) return st;
    unsigned char* sc = (unsigned char*)base;
    int4* seg = (int4*)sc;
    float2* a32 = mixed ? (float2*)(sc + seg_b) : nullptr;
    double2* traj_expect = (double2*)(sc + seg_b + a32_b);
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;

    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(qtl_device_info), stream);
    if (e == cudaSuccess) {
        int grid = a32 ? (int)((a_nnz + 1023) / 1024) : 1;
        if (grid > 1024) grid = 1024;
        if (grid < 1) grid = 1;
        count_launch();
        noalloc_prep_kernel<<<grid, 1024, 0, stream>>>(n, a_row_ptr, a_col_idx, seg, a_nnz,
                                                        (const double2*)a_vals, a32, info);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    McJob J;
    memset(&J, 0, sizeof(J));
    J.n = n;
    J.a_nnz = (int)a_nnz;
    J.aseg = seg;
    J.arp = a_row_ptr;
    J.aci = a_col_idx;
    J.av64 = (const double2*)a_vals;
    J.av32 = a32;
    J.n_c = n_c;
    J.crp = c_row_ptr;
    J.cci = c_col_idx;
    J.cv = (const double2*)c_vals;
    J.n_e = n_e;
    J.orp = o_row_ptr;
    J.oci = o_col_idx;
    J.ov = (const double2*)o_vals;
    J.tlist = tlist;
    J.nt = nt;
    J.psi0 = (const double2*)psi0;
    J.ntraj = ntraj;
    J.seed = seed;
    J.traj_offset = traj_offset;
    J.traj_expect = traj_expect;
    J.expect = (double2*)expect;
    J.info = info;
    J.rtol = opts->rtol;
    J.atol = opts->atol;
    J.dt0 = opts->dt0;
    J.dt_min = opts->dt_min;
    J.dt_fixed = opts->dt_fixed;
    J.max_steps = opts->max_steps;
    J.fixed = opts->fixed_step ? 1 : 0;
    J.method = opts->method;
    e = launch_mc_traj(J, opts->precision, stream);
    if (e == cudaSuccess) e = launch_mc_reduce(J, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    return QTL_OK;
}
