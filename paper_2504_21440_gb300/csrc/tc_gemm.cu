// Dense complex matrix products on the tensor cores (tcgen05, sm_103a), in a
// split-BF16 form: each FP64 operand entry is split into x_hi + x_lo (two
// BF16 numbers, about 16 significant bits together), and the product is
// accumulated in FP32 as A_hi B_hi + A_hi B_lo + A_lo B_hi.  The complex
// product C = op(A) op(B) of n x n matrices becomes one real GEMM
//     [C_r; C_i] = [A_r, -A_i; A_i, A_r] [B_r; B_i],
// with the three split products laid side by side along K (K = 6n).  Its
// relative accuracy is about 2^-16 of sum |a||b|: used where that suffices,
// as in the stationary-state preconditioner (an approximate inverse inside
// flexible GMRES, whose residuals stay FP64).
//
// The real GEMM C = A B^T (A: M x K, B: N x K, both K-contiguous BF16, C FP32
// row-major) runs one 128 x 128 output tile per CTA:
//   - a producer thread streams 128 x 64 tiles of A and B into a 4-stage
//     shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte swizzle),
//     each stage guarded by a "full" mbarrier (transaction bytes);
//   - one thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulator in tensor memory, M = 128, N = 128, K = 16 per
//     instruction) and releases each stage with tcgen05.commit on its
//     "empty" mbarrier;
//   - after a final commit the four warps read the accumulator with
//     tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e. rows) and store it.
// Every mbarrier wait is bounded: on timeout the kernel records an error
// flag, waits (bounded) for the copies it issued, frees its tensor memory
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"

namespace qtl {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_ST = 4;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;            // 16 KB per operand tile
constexpr int TC_SMEM = 1024 + TC_ST * 2 * TC_TILE_BYTES + 256;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;              // polls of a non-blocking test_wait

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes)
                 : "memory");
}
// true once the phase of the given parity has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit) {
    const uint32_t a = s_addr(b);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(s_addr(dst)),
        "l"((unsigned long long)map), "r"(s_addr(bar)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle
// (rows of 128 bytes, 8-row groups 1024 bytes apart): start address >> 4,
// leading offset 16 B (unused by this layout), stride offset 1024 B,
// descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sdesc_k128(const void* tile) {
    const uint32_t a = s_addr(tile);
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap ma,
                                                         const __grid_constant__ CUtensorMap mb, float* __restrict__ C,
                                                         int ldc, int K, int* __restrict__ err) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;
    unsigned char* sB = sm + TC_ST * TC_TILE_BYTES;
    uint64_t* full = (uint64_t*)(sB + TC_ST * TC_TILE_BYTES);
    uint64_t* empty = full + TC_ST;
    uint64_t* done = empty + TC_ST;
    uint32_t* tslot = (uint32_t*)(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
    const int nk = K / TC_BK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    if (threadIdx.x == 0) {
        // producer: stage s of k-block kb is reused once the MMAs of kb - TC_ST released it
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TC_ST, r = kb / TC_ST;
            if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1, TC_WAIT_LIMIT)) {
                ok = false;
                break;
            }
            mbar_expect_tx(&full[s], 2 * TC_TILE_BYTES);
            tma_load_2d(&ma, &full[s], sA + s * TC_TILE_BYTES, kb * TC_BK, m0);
            tma_load_2d(&mb, &full[s], sB + s * TC_TILE_BYTES, kb * TC_BK, n0);
            issued = kb + 1;
        }
        if (!ok) {
            atomicExch(err, 1);
            // the copies already issued complete into their full barriers
            for (int kb = (issued > TC_ST ? issued - TC_ST : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % TC_ST], (kb / TC_ST) & 1, TC_WAIT_LIMIT);
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(TC_BM, TC_BN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TC_ST;
            if (!mbar_wait(&full[s], (kb / TC_ST) & 1, TC_WAIT_LIMIT)) {
                ok = false;
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint64_t ad = sdesc_k128(sA + s * TC_TILE_BYTES), bd = sdesc_k128(sB + s * TC_TILE_BYTES);
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
                // K step of 16 BF16 = 32 bytes inside the swizzled rows: start address + 2 (units of 16 B)
                const uint32_t acc = (kb | k) != 0;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad + 2 * k), "l"(bd + 2 * k), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             s_addr(&empty[s]))
                         : "memory");
        }
        // arrives once every MMA issued above has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s_addr(done))
                     : "memory");
    }
    __syncwarp();
    const bool ready = mbar_wait(done, 0, TC_WAIT_LIMIT);
    tc_fence_after();
    // tcgen05.ld is warp-collective (.sync.aligned): the decision must be warp-uniform
    if (__all_sync(0xffffffffu, ready && ok)) {
        // warp w reads TMEM lanes 32w..32w+31: rows m0 + 32w + lane
        const int row = m0 + warp * 32 + lane;
        float* crow = C + (size_t)row * ldc + n0;
#pragma unroll 1
        for (int c = 0; c < TC_BN; c += 8) {
            uint32_t r[8];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4 v0 = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                                    __uint_as_float(r[3]));
            float4 v1 = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]),
                                    __uint_as_float(r[7]));
            *(float4*)(crow + c) = v0;
            *(float4*)(crow + c + 4) = v1;
        }
    } else if (!(ready && ok)) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
}

// ------------------------------------------------------------- packing --
// A side (M x K row-major BF16, M = 2n padded, K = 6n padded):
//   row i < 2n, column l < 2n of Ahat = [Ar, -Ai; Ai, Ar] (Ahat of op(A)):
//   [hi(Ahat) | hi(Ahat) | lo(Ahat)] along K.
// B side (N x K row-major, N = n padded): row j = column j of
//   Bhat = [Br; Bi] (of op(B)) as [hi | lo | hi] along K.
// op: 0 identity, 1 conjugate transpose.  Padding entries are zero.
__device__ __forceinline__ double2 op_at(const double2* X, int n, int op, int i, int j) {
    if (!op) return X[(size_t)i + (size_t)n * j];
    const double2 t = X[(size_t)j + (size_t)n * i];
    return make_double2(t.x, -t.y);
}
__device__ __forceinline__ void split_bf16(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn((float)x);
    lo = __float2bfloat16_rn((float)(x - (double)__bfloat162float(hi)));
}

__global__ void tc_pack_a_kernel(int n, const double2* __restrict__ A, int op, __nv_bfloat16* __restrict__ out,
                                 int Mp, int Kp) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)Mp * Kp) return;
    const int i = (int)(e / Kp), k = (int)(e % Kp);
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    const int n2 = 2 * n;
    if (i < n2 && k < 3 * n2) {
        const int part = k / n2, l = k % n2;
        // Ahat[i][l]
        const int bi = i / n, bl = l / n, ii = i % n, ll = l % n;
        const double2 a = op_at(A, n, op, ii, ll);
        const double x = (bi == bl) ? a.x : (bi == 0 ? -a.y : a.y);
        __nv_bfloat16 hi, lo;
        split_bf16(x, hi, lo);
        v = part < 2 ? hi : lo;
    }
    out[e] = v;
}

__global__ void tc_pack_b_kernel(int n, const double2* __restrict__ B, int op, __nv_bfloat16* __restrict__ out,
                                 int Np, int Kp) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)Np * Kp) return;
    const int j = (int)(e / Kp), k = (int)(e % Kp);
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    const int n2 = 2 * n;
    if (j < n && k < 3 * n2) {
        const int part = k / n2, l = k % n2;
        const double2 b = op_at(B, n, op, l % n, j);
        const double x = l < n ? b.x : b.y;
        __nv_bfloat16 hi, lo;
        split_bf16(x, hi, lo);
        v = part == 1 ? lo : hi;
    }
    out[e] = v;
}

// C (complex, n x n column-major) from the real product [Cr; Ci] (row-major, ldc)
__global__ void tc_unpack_kernel(int n, const float* __restrict__ Cr, int ldc, double2* __restrict__ C) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    C[e] = make_double2((double)Cr[(size_t)i * ldc + j], (double)Cr[(size_t)(i + n) * ldc + j]);
}

// --------------------------------------------------------------- host --
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2D BF16 tensor map of a rows x cols row-major matrix, box 64 x 128, 128 B swizzle
static bool tc_map(CUtensorMap* m, const void* base, int rows, int cols) {
    auto enc = tc_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_zgemm_scratch_bytes(int n) {
    const size_t Mp = ((size_t)2 * n + TC_BM - 1) / TC_BM * TC_BM, Np = ((size_t)n + TC_BN - 1) / TC_BN * TC_BN,
                 Kp = ((size_t)6 * n + TC_BK - 1) / TC_BK * TC_BK;
    return (Mp * Kp * 2 + 255) / 256 * 256 + (Np * Kp * 2 + 255) / 256 * 256 + Mp * Np * 4 + 256;
}

// C = op(A) op(B) (n x n complex FP64, column-major, device) by the split-BF16
// tensor-core product; scratch of tc_zgemm_scratch_bytes(n); err: device int
// set to 1 if a wait of the GEMM kernel timed out.
cudaError_t launch_tc_zgemm(int n, const double2* A, int opa, const double2* B, int opb, double2* C, void* scratch,
                            int* err, cudaStream_t st) {
    const int Mp = (2 * n + TC_BM - 1) / TC_BM * TC_BM, Np = (n + TC_BN - 1) / TC_BN * TC_BN,
              Kp = (6 * n + TC_BK - 1) / TC_BK * TC_BK;
    unsigned char* p = (unsigned char*)scratch;
    __nv_bfloat16* pa = (__nv_bfloat16*)p;
    p += ((size_t)Mp * Kp * 2 + 255) / 256 * 256;
    __nv_bfloat16* pb = (__nv_bfloat16*)p;
    p += ((size_t)Np * Kp * 2 + 255) / 256 * 256;
    float* cr = (float*)p;
    CUtensorMap ma, mb;
    if (!tc_map(&ma, pa, Mp, Kp) || !tc_map(&mb, pb, Np, Kp)) return cudaErrorNotSupported;
    static std::once_flag attr;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr, [] {
        attr_err = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const long long ea = (long long)Mp * Kp, eb = (long long)Np * Kp;
    count_launch(4);
    tc_pack_a_kernel<<<(unsigned)((ea + 255) / 256), 256, 0, st>>>(n, A, opa, pa, Mp, Kp);
    tc_pack_b_kernel<<<(unsigned)((eb + 255) / 256), 256, 0, st>>>(n, B, opb, pb, Np, Kp);
    tc_gemm_kernel<<<dim3(Np / TC_BN, Mp / TC_BM), 128, TC_SMEM, st>>>(ma, mb, cr, Np, Kp, err);
    tc_unpack_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, st>>>(n, cr, Np, C);
    return cudaGetLastError();
}

}  // namespace qtl

using namespace qtl;

extern "C" qtl_status qtl_zgemm_async(int32_t n, const qtl_c128* A, int32_t op_a, const qtl_c128* B, int32_t op_b,
                                      qtl_c128* C, int32_t precision, void* cuda_stream, int32_t* err_dev) {
    if (n < 1 || n > 8192 || !A || !B || !C || (op_a != 0 && op_a != 1) || (op_b != 0 && op_b != 1) ||
        (precision != QTL_FP64 && precision != QTL_MIXED) || (precision == QTL_MIXED && !err_dev))
        return QTL_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (precision == QTL_FP64) {
        e = launch_zgemm(n, (const double2*)A, op_a, (const double2*)B, op_b, (double2*)C, st);
    } else {
        void* scr = nullptr;
        e = qtl_malloc_async(&scr, tc_zgemm_scratch_bytes(n), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return QTL_ENOMEM;
        }
        e = launch_tc_zgemm(n, (const double2*)A, op_a, (const double2*)B, op_b, (double2*)C, scr, err_dev, st);
        cudaFreeAsync(scr, st);
        if (e == cudaErrorNotSupported) return QTL_ECUDA;
    }
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    return QTL_OK;
}
