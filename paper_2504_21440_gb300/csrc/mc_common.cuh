// Device helpers shared by the trajectory kernels (mc_traj.cu: state in
// registers, n <= 1024; mc_wide.cu: state in global memory, larger n).
#pragma once
#include "internal.h"
#include "rk.cuh"
#include "td.cuh"

namespace qtl {

// most warps a trajectory CTA may have
constexpr int MC_MAXWARPS = 32;

template <bool MIXED>
struct MPrec;
template <>
struct MPrec<false> {
    using T = double;
    using T2 = double2;
};
template <>
struct MPrec<true> {
    using T = float;
    using T2 = float2;
};

__device__ __forceinline__ double2 to_d2_mc(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2_mc(float2 v) { return make_double2(v.x, v.y); }
template <class T2>
__device__ __forceinline__ T2 from_d2_mc(double2 v);
template <>
__device__ __forceinline__ double2 from_d2_mc<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 from_d2_mc<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}

// Values reduced at once: |psi|^2 and 2 per observable, or 1 per channel.
__host__ __device__ __forceinline__ int mc_red_stride(int n_e, int n_c) {
    int a = 2 + 2 * n_e;
    return a > n_c ? a : n_c;
}

__device__ __forceinline__ float mc_warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double mc_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct BlockReducer {
    double* wred;  // [nw][rs]
    double* out;   // [rs]
    int rs, lane, warp, tid, nw;
    __device__ void stage(int i, double v) {
        v = mc_warp_sum(v);
        if (lane == 0) wred[warp * rs + i] = v;
    }
    __device__ void finish(int nv) {
        __syncthreads();
        // strided: nv may exceed the CTA's thread count (a 32-thread CTA
        // with 64 channels, or 1 + 2 * 64 observable slots)
        for (int i = tid; i < nv; i += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += wred[w * rs + i];
            out[i] = s;
        }
        __syncthreads();
    }
};

// Philox4x32-10: ten rounds of the published round function; key bumped by
// the Weyl constants between rounds.
__device__ __forceinline__ double philox_uniform(unsigned long long seed, unsigned long long traj,
                                                 unsigned draw) {
    unsigned c0 = draw, c1 = (unsigned)traj, c2 = 0u, c3 = 0u;
    unsigned k0 = (unsigned)(seed & 0xffffffffull), k1 = (unsigned)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        unsigned lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        unsigned lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    unsigned long long x = ((unsigned long long)c1 << 20) | (unsigned long long)(c0 >> 12);
    return ((double)x + 0.5) * 0x1p-52;
}

// Row r of a segmented CSR (real-only | imaginary-only | complex entries)
// times x held in shared memory.
template <class T2, class TV>
__device__ __forceinline__ T2 mc_spmv_row(int r, const int4* __restrict__ seg,
                                          const int32_t* __restrict__ ci,
                                          const TV* __restrict__ v, const T2* x) {
    const int4 sg = __ldg(seg + r);
    decltype(T2::x) ax = 0, ay = 0, bx = 0, by = 0;
    int p = sg.x;
    for (; p < sg.y; ++p) {
        const decltype(T2::x) a = __ldg(&v[p].x);
        const T2 xv = x[__ldg(ci + p)];
        ax = fma(a, xv.x, ax);
        ay = fma(a, xv.y, ay);
    }
    for (; p < sg.z; ++p) {
        const decltype(T2::x) b = __ldg(&v[p].y);
        const T2 xv = x[__ldg(ci + p)];
        bx = fma(-b, xv.y, bx);
        by = fma(b, xv.x, by);
    }
    for (; p < sg.w; ++p) {
        const TV a = __ldg(v + p);
        const T2 xv = x[__ldg(ci + p)];
        ax = fma(a.x, xv.x, ax);
        ay = fma(a.x, xv.y, ay);
        bx = fma(-a.y, xv.y, bx);
        by = fma(a.y, xv.x, by);
    }
    T2 acc;
    acc.x = ax + bx;
    acc.y = ay + by;
    return acc;
}

// A's row from the CTA's shared-memory copy (rows packed in CTA order).
template <class T2, class TV>
__device__ __forceinline__ T2 mc_spmv_row_s(int r, const int4* __restrict__ s_seg,
                                            const int32_t* __restrict__ s_ci,
                                            const TV* __restrict__ s_v, const T2* x) {
    // two accumulators (real, imaginary part of the result): on GB300's 1/64
    // rate FP64 pipe the final additions of split accumulators cost as much
    // as a row's entries
    const int4 sg = s_seg[r];
    decltype(T2::x) ar = 0, ai = 0;
    int p = sg.x;
#pragma unroll 4
    for (; p < sg.y; ++p) {
        const decltype(T2::x) a = s_v[p].x;
        const T2 xv = x[s_ci[p]];
        ar = fma(a, xv.x, ar);
        ai = fma(a, xv.y, ai);
    }
#pragma unroll 4
    for (; p < sg.z; ++p) {
        const decltype(T2::x) b = s_v[p].y;
        const T2 xv = x[s_ci[p]];
        ar = fma(-b, xv.y, ar);
        ai = fma(b, xv.x, ai);
    }
#pragma unroll 2
    for (; p < sg.w; ++p) {
        const TV a = s_v[p];
        const T2 xv = x[s_ci[p]];
        ar = fma(a.x, xv.x, ar);
        ai = fma(a.x, xv.y, ai);
        ar = fma(-a.y, xv.y, ar);
        ai = fma(a.y, xv.x, ai);
    }
    T2 acc;
    acc.x = ar;
    acc.y = ai;
    return acc;
}

enum { MC_STEP = 0, MC_REPEAT = 1, MC_DONE = 2 };

// Control block broadcast by thread 0 (scalar control in one thread: GB300's
// FP64 pipe is 1/64 rate, so no FP64 scalar work is replicated per thread).
struct McCtl {
    double coef[28];  // htry * a_sj (21, packed by stage), htry * e_j (7)
    float coeff[28];  // the same, rounded to FP32 (mixed precision)
    double inv;       // 1 / |C_k psi*| of the chosen channel
    // save: output index of an accepted step that landed on tlist (or -1);
    // rsave: output index of a repeated tlist time (action MC_REPEAT).  They
    // are separate because a landing step is followed at once by the next
    // action, which may be a repeat of the same time.
    int action, land, accept, save, rsave, ch, rootgo, pub;
    // second-order increment form of the wide kernel's mixed precision:
    // htry (FP64 and FP32), htry^2 sum_j b_j c_j, htry^2 sum_j e_j c_j,
    // htry^2 e_7, and htry^2 W_s with W_s = sum_{l<s} a_sl c_l
    double hd, c2b;
    float hf, c2e, he7h;
    float c2w[7];
    float wf[MC_MAXWARPS];
    double wd[MC_MAXWARPS];
    // time-dependent terms: f_k at the stage times t + c_s htry (slots 1..6)
    // and at one other time (slot 7); tnow = the step's start
    double tnow;
    double2 tdf[8][QTL_MAX_TD];
    float2 tdf32[8][QTL_MAX_TD];
};

// index of h*a_sj in McCtl::coef (stages packed row by row)
__host__ __device__ constexpr int mc_coef_a(int s, int j) { return s * (s - 1) / 2 + j; }

}  // namespace qtl
