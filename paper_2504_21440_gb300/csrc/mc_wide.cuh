// mcsolve for Hilbert spaces above the register-resident limit (n > 1024):
// the Monte-Carlo wave-function method of Sec. 3.3 with the same steps,
// readings and random streams as mc_traj.cu (threshold on |psi|^2, Illinois
// root find of the crossing, channel by cumulative weight, Philox4x32-10
// with counter (draw, trajectory, 0, 0)).
//
// One CTA of 1024 threads integrates one trajectory at a time (persistent
// loop over trajectories).  psi, y_new and k_1..k_7 no longer fit in the
// registers of one SM (n = 16,384 needs 1.2 MB in complex64), so each CTA
// owns a slice of a global scratch buffer holding them; thread t handles rows
// r = t + 1024 m, so every pass over a vector is a coalesced stream.  The
// stage input that the sparse product A x gathers from sits in shared memory
// when it fits (complex64 up to n = 25,600), else in the CTA's scratch.
// Per step the kernel makes six passes of "form the stage input from
// y and k_1..k_{s-1}, then k_s = A x_s"; the embedded error estimate and
// |y_new|^2 are folded into the sixth pass, so no extra pass over the stage
// vectors is made.  FSAL and accept/reject swap buffer indices, never data.
//
// Scalar control (PI controller, landing on tlist, jump bookkeeping, Philox
// draws) runs in thread 0 and is broadcast through shared memory, exactly as
// in the register-resident kernel.  Reductions are fixed-order (warp shuffle
// tree, then warps in order), so a trajectory's result does not depend on the
// CTA that runs it.
#pragma once
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "mc_common.cuh"

namespace qtl {

// Threads per trajectory CTA (a compile-time tunable).
#ifndef QTL_MW_THREADS
#define QTL_MW_THREADS 1024
#endif
constexpr int MW_T = QTL_MW_THREADS;
constexpr int MW_NV = 14;                   // vectors in a CTA's scratch slice
constexpr size_t MW_SMEM_X_MAX = 200 * 1024;  // shared-memory budget for stage inputs

// Slots of a CTA's scratch slice, each mw_vec_bytes(n) bytes (256-aligned):
//   0,1    y / y_new, complex128 (the roles swap on accept)
//   2,3    mixed precision: f = A y and f_new = A y_new as FP32 pairs (the
//          hi parts, then the lo parts; the roles swap with y / y_new)
//   4..10  FP64: k_1..k_7 (complex128); k_1 and k_7 trade slots 4 and 10 on
//          accept (FSAL).  Mixed precision: slot 5 holds f2 = A f (stage 2)
//          and slots 6..9 the remainders r_3..r_6 (complex64)
//   11     partial error estimate of the sixth pass
//   12     its scale sc_i = atol + rtol max(|y_i|, |y_new,i|) (float)
//   13     mixed precision: the FP32 remainder y_new - (float)y_new
//   14,15  the two stage inputs, when they do not fit in shared memory
//
// Mixed precision is a second-order increment form.  With f = A y and
// f2 = A f, every stage derivative is k_s = f + h c_s f2 + r_s, where
// r_s = A d_s, d_s = x_s - y - h c_s f = h^2 W_s f2 + h sum_{l<s} a_sl r_l
// (W_s = sum_l a_sl c_l, r_1 = r_2 = 0).  The FP32 operator then acts on f
// (stage 2, giving f2) and on the O(h^2) increments d_s (stages 3-6); the
// new state y_new = y + h f + h^2 (sum b c) f2 + h sum b_j r_j is formed in
// FP64, and the last stage evaluates f_new = A y_new with error-free FP32
// products and sums (sell_row_dd), which is the next step's f.  FP32
// rounding therefore enters only through terms of order h^2 |A|^2 |y|:
// with the plain FP32 right-hand side the 14-spin chain's trajectories
// differed from FP64 by 4e-6 on Sz; rounding the operator or the stage
// coefficients to FP32 shifts the method's frequencies, which accumulates
// over the span.  The error estimate is h^2 (sum e c) f2 + h sum e_j r_j
// (sum e_j = 0), with r_7 = f_new - f - h f2.
__host__ __device__ inline size_t mw_vec_bytes(int n) {
    return ((size_t)n * 16 + 255) & ~(size_t)255;
}

// Thread 0's control state, kept in shared memory so that the other 1023
// threads do not carry it in registers.
struct MwCtl0 {
    double t, h, htry, t_target, r, norm2;
    double lo, glo, hi, ghi, tau, log_r;  // jump-time root find
    long long attempts, acc_steps, rej_steps, rhs_evals, jumps;
    unsigned draw;
    int idx, side, it, status;
    CtlF ctl;
};

// Loads of A carry an L2 evict-last policy: A is read six times per step by
// every resident trajectory, while each CTA's state vectors stream through
// L2 once or twice a step with an evict-first hint (__ldcs / __stcs), so
// without the hints the state evicts A and each stage re-reads it from HBM.
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
#ifndef QTL_MW_L2HINT
#define QTL_MW_L2HINT 1
#endif
#if !QTL_MW_L2HINT
template <class V>
__device__ __forceinline__ auto lda(const V* p, unsigned long long) {
    if constexpr (sizeof(V) == 2)
        return (int)__ldg(p);
    else
        return __ldg(p);
}
#else
__device__ __forceinline__ int lda(const uint16_t* p, unsigned long long pol) {
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return (int)v;
}
__device__ __forceinline__ int lda(const int32_t* p, unsigned long long pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float lda(const float* p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double lda(const double* p, unsigned long long pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 lda(const float2* p, unsigned long long pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
        : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 lda(const double2* p, unsigned long long pol) {
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
        : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}
#endif

// Row q of A x from the pattern-compressed sliced ELLPACK copy (DevSell):
// all lanes of a warp are in the same slice, so the loops and the
// descriptor's column/value modes are warp-uniform, a uniform value is one
// broadcast load and an explicit one a coalesced load.  Same accumulation as
// mc_spmv_row: real parts into (ax, ay), imaginary parts into (bx, by), in
// entry order; padding entries are exact zeros.  x is read with 32-bit
// shared loads when it lives in shared memory (XS).  (Issuing a row's loads
// in explicit batches, out-of-line calls and 512- or 768-thread CTAs were
// all measured slower than this plain loop at 1024 threads.)
#ifndef QTL_MW_LDS_ASM
#define QTL_MW_LDS_ASM 1
#endif
__device__ __forceinline__ float2 lds2(unsigned a, float2) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ double2 lds2(unsigned a, double2) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}

// One group of a row: G = 0 real-only (into ax, ay), 1 imaginary-only (into
// bx, by), 2 complex.  The group type (warp-uniform) picks a loop without
// per-entry decoding where the host found a single pattern.
template <int G, bool MIXED, class T, class T2, class IT, class GX, class DG>
__device__ __forceinline__ void sell_group(int q, int lane, int w, int type, DG&& dg, int cbase,
                                           int vbase, const IT* __restrict__ ci,
                                           const T* __restrict__ vs, const T2* __restrict__ vc,
                                           GX&& gx, unsigned long long pol, T& ax, T& ay, T& bx,
                                           T& by) {
    using V = typename std::conditional<G == 2, T2, T>::type;
    auto acc = [&](const V& v, const T2& xv) {
        if constexpr (G == 0) {
            ax = fma(v, xv.x, ax);
            ay = fma(v, xv.y, ay);
        } else if constexpr (G == 1) {
            bx = fma(-v, xv.y, bx);
            by = fma(v, xv.x, by);
        } else {
            ax = fma(v.x, xv.x, ax);
            ay = fma(v.x, xv.y, ay);
            bx = fma(-v.y, xv.y, bx);
            by = fma(v.y, xv.x, by);
        }
    };
    const V* vp;
    if constexpr (G == 2)
        vp = vc;
    else
        vp = vs;
    if (w <= 0) return;
    if (type == SELL_G_XU) {
#pragma unroll 4
        for (int p = 0; p < w; ++p) {
            const int4 d = dg(p);
            V v;
            if constexpr (G < 2 && MIXED)
                v = __int_as_float(d.w);
            else
                v = __ldg(vp + d.z);
            acc(v, gx(q ^ d.y));
        }
    } else if (type == SELL_G_XE) {
        const int vb = vbase + dg(0).z + lane;
#pragma unroll 4
        for (int p = 0; p < w; ++p) {
            const int m = dg(p).y;
            acc(lda(vp + vb + 32 * p, pol), gx(q ^ m));
        }
    } else if (type == SELL_G_EE) {
        const int4 d0 = dg(0);  // .y column offset, .z value offset of the first block
        const int cb = cbase + d0.y + lane, vb = vbase + d0.z + lane;
#pragma unroll 4
        for (int p = 0; p < w; ++p) acc(lda(vp + vb + 32 * p, pol), gx(lda(ci + cb + 32 * p, pol)));
    } else {
#pragma unroll 2
        for (int p = 0; p < w; ++p) {
            const int4 d = dg(p);
            const int mode = d.x & 3;
            const int c = mode == SELL_COL_XOR      ? (q ^ d.y)
                          : mode == SELL_COL_OFFSET ? (q + d.y)
                                                    : (int)lda(ci + cbase + d.y + lane, pol);
            const V v = (d.x & SELL_VAL_UNIFORM) ? __ldg(vp + d.z) : lda(vp + vbase + d.z + lane, pol);
            acc(v, gx(c));
        }
    }
}

template <bool MIXED, class T, class T2, class IT, bool XS, bool DC>
__device__ __forceinline__ T2 sell_row(int q, const int4* __restrict__ sl,
                                       const int4* __restrict__ desc, const SellConst& C,
                                       const IT* __restrict__ ci, const T* __restrict__ vs,
                                       const T2* __restrict__ vc, const T2* x,
                                       unsigned long long pol) {
    unsigned xsa = 0;
    if constexpr (XS) xsa = (unsigned)__cvta_generic_to_shared(x);
    auto gx = [&](int c) -> T2 {
#if QTL_MW_LDS_ASM
        if constexpr (XS) return lds2(xsa + (unsigned)c * (unsigned)sizeof(T2), T2{});
#endif
        return x[c];
    };
    const int lane = q & 31;
    const int4 a = __ldg(sl + 2 * (q >> 5));      // {first descriptor, real, imaginary, complex widths}
    const int4 b = __ldg(sl + 2 * (q >> 5) + 1);  // {cbase, vsbase, vcbase, group types}
    // descriptor i of the slice's list: from the constant parameter (DC) or
    // through the read-only cache
    auto dgi = [&](int i) -> int4 {
        if constexpr (DC)
            return C.d[i];
        else
            return __ldg(desc + i);
    };
    const int g1 = a.x + a.y, g2 = g1 + a.z;
    T ax = 0, ay = 0, bx = 0, by = 0;
    sell_group<0, MIXED, T, T2, IT>(q, lane, a.y, b.w & 3, [&](int p) { return dgi(a.x + p); }, b.x,
                                    b.y, ci, vs, vc, gx, pol, ax, ay, bx, by);
    sell_group<1, MIXED, T, T2, IT>(q, lane, a.z, (b.w >> 2) & 3, [&](int p) { return dgi(g1 + p); },
                                    b.x, b.y, ci, vs, vc, gx, pol, ax, ay, bx, by);
    sell_group<2, MIXED, T, T2, IT>(q, lane, a.w, (b.w >> 4) & 3, [&](int p) { return dgi(g2 + p); },
                                    b.x, b.z, ci, vs, vc, gx, pol, ax, ay, bx, by);
    T2 acc;
    acc.x = ax + bx;
    acc.y = ay + by;
    return acc;
}

// ---- error-free row products (the base derivative of the mixed precision) ----
// s + c += (a + al) (x + xl) with the product a x exact (TwoProduct by FMA)
// and its addition to s exact (Knuth's TwoSum); the small cross terms a xl +
// al x and the rounding errors go to c.  The _rn intrinsics keep the
// compiler from contracting the multiply into the additions, which would
// break the error-free transformations.
__device__ __forceinline__ void dd_acc(float& s, float& c, float a, float x, float al, float xl) {
    const float p = __fmul_rn(a, x);
    const float e = __fmaf_rn(a, x, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fmaf_rn(al, x, __fmaf_rn(a, xl, __fadd_rn(__fadd_rn(c, err), e)));
}

// One group of a row, as sell_group, with the values (vh + vl) and the input
// (gx(c) + gl(c)) both given as FP32 pairs; accumulates into the pairs
// (rs, rc) (real part) and (is, ic) (imaginary part).
template <int G, class IT, class GX, class GL, class DG>
__device__ __forceinline__ void sell_group_dd(int q, int lane, int w, int type, DG&& dg, int cbase,
                                              int vbase, const IT* __restrict__ ci,
                                              const float* __restrict__ vs, const float2* __restrict__ vc,
                                              const float* __restrict__ vsl, const float2* __restrict__ vcl,
                                              GX&& gx, GL&& gl, unsigned long long pol, float& rs,
                                              float& rc, float& is, float& ic) {
    auto acc_s = [&](int c, float vh, float vl) {
        const float2 x = gx(c), xl = gl(c);
        if constexpr (G == 0) {
            dd_acc(rs, rc, vh, x.x, vl, xl.x);
            dd_acc(is, ic, vh, x.y, vl, xl.y);
        } else {
            dd_acc(rs, rc, -vh, x.y, -vl, xl.y);
            dd_acc(is, ic, vh, x.x, vl, xl.x);
        }
    };
    auto acc_c = [&](int c, float2 vh, float2 vl) {
        const float2 x = gx(c), xl = gl(c);
        dd_acc(rs, rc, vh.x, x.x, vl.x, xl.x);
        dd_acc(rs, rc, -vh.y, x.y, -vl.y, xl.y);
        dd_acc(is, ic, vh.x, x.y, vl.x, xl.y);
        dd_acc(is, ic, vh.y, x.x, vl.y, xl.x);
    };
    // value of entry position p: uniform (index d.z) or explicit (index i)
    auto val = [&](int4 d, bool uni, int i, auto&& use, int c) {
        if constexpr (G < 2) {
            const float vh = uni ? __int_as_float(d.w) : lda(vs + i, pol);
            const float vl = uni ? __ldg(vsl + d.z) : lda(vsl + i, pol);
            use(c, vh, vl);
        } else {
            const float2 vh = uni ? __ldg(vc + d.z) : lda(vc + i, pol);
            const float2 vl = uni ? __ldg(vcl + d.z) : lda(vcl + i, pol);
            use(c, vh, vl);
        }
    };
    auto use = [&](int c, auto vh, auto vl) {
        if constexpr (G < 2)
            acc_s(c, vh, vl);
        else
            acc_c(c, vh, vl);
    };
    if (w <= 0) return;
    if (type == SELL_G_XU) {
#pragma unroll 2
        for (int p = 0; p < w; ++p) {
            const int4 d = dg(p);
            val(d, true, 0, use, q ^ d.y);
        }
    } else if (type == SELL_G_XE) {
        const int vb = vbase + dg(0).z + lane;
#pragma unroll 2
        for (int p = 0; p < w; ++p) {
            const int4 d = dg(p);
            val(d, false, vb + 32 * p, use, q ^ d.y);
        }
    } else if (type == SELL_G_EE) {
        const int4 d0 = dg(0);
        const int cb = cbase + d0.y + lane, vb = vbase + d0.z + lane;
#pragma unroll 2
        for (int p = 0; p < w; ++p) val(d0, false, vb + 32 * p, use, (int)lda(ci + cb + 32 * p, pol));
    } else {
        for (int p = 0; p < w; ++p) {
            const int4 d = dg(p);
            const int mode = d.x & 3;
            const int c = mode == SELL_COL_XOR      ? (q ^ d.y)
                          : mode == SELL_COL_OFFSET ? (q + d.y)
                                                    : (int)lda(ci + cbase + d.y + lane, pol);
            const bool uni = (d.x & SELL_VAL_UNIFORM) != 0;
            val(d, uni, vbase + d.z + lane, use, c);
        }
    }
}

// Row q of A x to about FP64 accuracy in FP32 arithmetic: x = xh + xl (xh
// gathered like the stage inputs, xl from global memory), A = vh + vl.
// Returns {re hi, im hi, re lo, im lo} with |lo| <= ulp(hi) / 2.
template <class IT, bool XS, bool DC>
__device__ __forceinline__ float4 sell_row_dd(int q, const int4* __restrict__ sl,
                                              const int4* __restrict__ desc, const SellConst& C,
                                              const IT* __restrict__ ci, const float* __restrict__ vs,
                                              const float2* __restrict__ vc, const float* __restrict__ vsl,
                                              const float2* __restrict__ vcl, const float2* xh,
                                              const float2* xl, unsigned long long pol) {
    unsigned xsa = 0;
    if constexpr (XS) xsa = (unsigned)__cvta_generic_to_shared(xh);
    auto gx = [&](int c) -> float2 {
        if constexpr (XS) return lds2(xsa + (unsigned)c * (unsigned)sizeof(float2), float2{});
        return xh[c];
    };
    auto gl = [&](int c) -> float2 { return xl[c]; };
    const int lane = q & 31;
    const int4 a = __ldg(sl + 2 * (q >> 5));
    const int4 b = __ldg(sl + 2 * (q >> 5) + 1);
    auto dgi = [&](int i) -> int4 {
        if constexpr (DC)
            return C.d[i];
        else
            return __ldg(desc + i);
    };
    const int g1 = a.x + a.y, g2 = g1 + a.z;
    float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
    sell_group_dd<0, IT>(q, lane, a.y, b.w & 3, [&](int p) { return dgi(a.x + p); }, b.x, b.y, ci, vs, vc,
                         vsl, vcl, gx, gl, pol, rs, rc, is, ic);
    sell_group_dd<1, IT>(q, lane, a.z, (b.w >> 2) & 3, [&](int p) { return dgi(g1 + p); }, b.x, b.y, ci,
                         vs, vc, vsl, vcl, gx, gl, pol, rs, rc, is, ic);
    sell_group_dd<2, IT>(q, lane, a.w, (b.w >> 4) & 3, [&](int p) { return dgi(g2 + p); }, b.x, b.z, ci,
                         vs, vc, vsl, vcl, gx, gl, pol, rs, rc, is, ic);
    // renormalise: hi = fl(s + c), lo = the exact remainder (Fast2Sum, |s| >= |c|)
    const float hr = __fadd_rn(rs, rc), hi_ = __fadd_rn(is, ic);
    return make_float4(hr, hi_, __fsub_rn(rc, __fsub_rn(hr, rs)), __fsub_rn(ic, __fsub_rn(hi_, is)));
}

template <bool MIXED, class IT, bool XS, bool DC>
__global__ void __launch_bounds__(MW_T, 1) mc_wide_kernel(McJob J, const __grid_constant__ SellConst C) {
    using T = typename MPrec<MIXED>::T;
    using T2 = typename MPrec<MIXED>::T2;
    extern __shared__ __align__(16) unsigned char mw_smem[];
    __shared__ McCtl cb;
    __shared__ MwCtl0 z;
    const int n = J.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = MW_T / 32;
    const int rs = mc_red_stride(J.n_e, J.n_c);
    double* wred = (double*)mw_smem;
    double* bout = wred + nw * rs;
    BlockReducer red{wred, bout, rs, lane, warp, tid, nw};
    const RkTab& tab = RK_TABS[J.method];
    const T* svs = MIXED ? (const T*)J.svs32 : (const T*)J.svs64;
    const T2* svc = MIXED ? (const T2*)J.svc32 : (const T2*)J.svc64;

    const size_t vb = mw_vec_bytes(n);
    unsigned char* base = J.wscr + (size_t)blockIdx.x * J.wstride;
    // y / y_new (and their FP32 copies) by role index ys: no indexed arrays,
    // which would be placed in local memory
    auto Yp = [&](int i) -> double2* { return (double2*)(base + (size_t)i * vb); };
    auto YFp = [&](int i) -> float2* { return (float2*)(base + (size_t)(2 + i) * vb); };
    unsigned char* kbase = base + 4 * vb;
    T2* EP = (T2*)(base + 11 * vb);
    float* SC = (float*)(base + 12 * vb);
    // mixed precision: f (role i) hi and lo parts, and the stage-7 input's remainder
    auto FHp = [&](int i) -> float2* { return (float2*)(base + (size_t)(2 + i) * vb); };
    auto FLp = [&](int i) -> float2* { return (float2*)(base + (size_t)(2 + i) * vb) + n; };
    float2* XL = (float2*)(base + 13 * vb);
    // stage inputs: shared memory (XS; the compiler then addresses them with
    // 32-bit shared loads) or the CTA's scratch
    T2 *X0, *X1;
    if constexpr (XS) {
        unsigned char* xs = mw_smem + ((((size_t)nw + 1) * rs + 2) * sizeof(double) + 15) / 16 * 16;
        X0 = (T2*)xs;
        X1 = J.xbufs > 1 ? (T2*)(xs + (((size_t)n * sizeof(T2) + 15) & ~(size_t)15)) : X0;
    } else {
        X0 = (T2*)(base + 14 * vb);
        X1 = (T2*)(base + 15 * vb);
    }
    const bool xsingle = X1 == X0;
    const unsigned long long pol = l2_evict_last();
    auto rhs_row = [&](int r, const T2* x) -> T2 {
        return sell_row<MIXED, T, T2, IT, XS, DC>(r, J.sl, J.sdesc, C, (const IT*)J.sci, svs, svc, x, pol);
    };
    // FP64: A x plus sum_k f_k (-i H_k x) with the coefficients of slot `slot`
    // (1..6: the stages of the current step, 7: one other time); the
    // mixed-precision kernel takes no time-dependent terms
    auto rhs_td = [&](int r, const T2* x, int slot) -> T2 {
        T2 v = rhs_row(r, x);
        if constexpr (!MIXED) {
            for (int k = 0; k < J.n_td; ++k) {
                const SellRef R = J.tsl[k];
                const T2 w = sell_row<false, double, double2, int32_t, XS, false>(r, R.sl, R.desc, C, R.ci, R.vs64,
                                                                                 R.vc64, x, pol);
                const double2 f = cb.tdf[slot][k];
                v.x += f.x * w.x - f.y * w.y;
                v.y += f.x * w.y + f.y * w.x;
            }
        }
        return v;
    };
    // warp 0: f_k at time tp into slot 7
    auto publish_td_at = [&](double tp) {
        if (lane < J.n_td) cb.tdf[7][lane] = td_coef(J.tf[lane], tp);
    };
    // mixed precision: f = A (X + XL) for every row into slot `role` (pair)
    auto base_deriv = [&](int role, const T2* xh) {
        if constexpr (MIXED) {
            float2* fh = FHp(role);
            float2* fl = FLp(role);
            for (int q = tid; q < n; q += MW_T) {
                const float4 r = sell_row_dd<IT, XS, DC>(q, J.sl, J.sdesc, C, (const IT*)J.sci, J.svs32,
                                                         J.svc32, J.svs32lo, J.svc32lo, xh, XL, pol);
                fh[q] = make_float2(r.x, r.y);
                fl[q] = make_float2(r.z, r.w);
            }
        }
    };
    // the FP32 remainder of v after rounding to hi
    auto lo_of = [](double2 v, float2 hi) {
        return make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
    };

    long long& acc_steps = z.acc_steps;  // thread 0 only, as all of z
    long long& rej_steps = z.rej_steps;
    long long& rhs_evals = z.rhs_evals;
    long long& jumps = z.jumps;
    int& status = z.status;
    double& t = z.t;
    double& h = z.h;
    double& htry = z.htry;
    double& t_target = z.t_target;
    double& r = z.r;
    double& norm2 = z.norm2;
    double& lo = z.lo;
    double& glo = z.glo;
    double& hi = z.hi;
    double& ghi = z.ghi;
    double& tau = z.tau;
    double& log_r = z.log_r;
    long long& attempts = z.attempts;
    unsigned& draw = z.draw;
    int& idx = z.idx;
    int& side = z.side;
    int& it = z.it;
    CtlF& ctl = z.ctl;
    if (tid == 0) {
        acc_steps = rej_steps = rhs_evals = jumps = 0;
        status = QTL_OK;
    }

    // trajectories: the first one per CTA by block index, then the next free
    // one from a device counter (trajectories differ in length: number of
    // jumps and steps), so no CTA idles while another still has two to go
    __shared__ int s_next;
    for (int jt = blockIdx.x; jt < J.ntraj; jt = s_next) {
        const unsigned long long traj = (unsigned long long)(J.traj_offset + jt);
        int ys = 0;   // Y[ys] = y, Y[ys ^ 1] = y_new (same for YF)
        int k0s = 0;  // slot of k_1: 0 or 6 (k_7 takes the other)
        auto Kp = [&](int j) -> T2* {
            const int slot = j == 0 ? k0s : (j == 6 ? 6 - k0s : j);
            return (T2*)(kbase + slot * vb);
        };
        auto coefT = [&](int i) -> T {
            if constexpr (MIXED)
                return cb.coeff[i];
            else
                return cb.coef[i];
        };

        for (int q = tid; q < n; q += MW_T) {
            const double2 v = J.psi0[q];
            Yp(0)[q] = v;
            const T2 o = from_d2_mc<T2>(v);
            X0[q] = o;
            if constexpr (MIXED) XL[q] = lo_of(v, o);
        }
        if constexpr (!MIXED)
            if (warp == 0 && J.n_td > 0) publish_td_at(J.tlist[0]);
        __syncthreads();
        if constexpr (MIXED)
            base_deriv(0, X0);
        else
            for (int q = tid; q < n; q += MW_T) Kp(0)[q] = rhs_td(q, X0, 7);
        __syncthreads();

        // <psi|O_e|psi>/<psi|psi> for psi = Y[ys] (written and synchronised by
        // the caller); returns |psi|^2 in every thread.
        auto save = [&](int idx) -> double {
            const double2* psi = Yp(ys);
            double s2 = 0.0;
            for (int q = tid; q < n; q += MW_T) {
                const double2 v = psi[q];
                s2 += v.x * v.x + v.y * v.y;
            }
            red.stage(0, s2);
            for (int e = 0; e < J.n_e; ++e) {
                double sr = 0.0, si = 0.0;
                for (int q = tid; q < n; q += MW_T) {
                    // (O psi)_q over the row's segments: purely real and
                    // purely imaginary entries (Pauli-type observables) take
                    // 2 FP64 FMAs instead of 4 -- FP64 runs at 1/64 rate here
                    const int4 sg = __ldg(J.oseg + e * n + q);
                    double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
                    int p = sg.x;
                    for (; p < sg.y; ++p) {
                        const double a = __ldg(&J.ov[p].x);
                        const double2 v = psi[__ldg(J.oci + p)];
                        ax = fma(a, v.x, ax);
                        ay = fma(a, v.y, ay);
                    }
                    for (; p < sg.z; ++p) {
                        const double b = __ldg(&J.ov[p].y);
                        const double2 v = psi[__ldg(J.oci + p)];
                        bx = fma(-b, v.y, bx);
                        by = fma(b, v.x, by);
                    }
                    for (; p < sg.w; ++p) {
                        const double2 o = __ldg(J.ov + p);
                        const double2 v = psi[__ldg(J.oci + p)];
                        ax = fma(o.x, v.x, ax);
                        ay = fma(o.x, v.y, ay);
                        bx = fma(-o.y, v.y, bx);
                        by = fma(o.y, v.x, by);
                    }
                    const double ox = ax + bx, oy = ay + by;
                    const double2 y = psi[q];
                    // conj(psi_q) * (O psi)_q
                    sr += y.x * ox + y.y * oy;
                    si += y.x * oy - y.y * ox;
                }
                red.stage(1 + 2 * e, sr);
                red.stage(2 + 2 * e, si);
            }
            red.finish(1 + 2 * J.n_e);
            for (int e = tid; e < J.n_e; e += blockDim.x) {
                const double nn = bout[0];
                J.traj_expect[((size_t)e * J.nt + idx) * J.ntraj + jt] =
                    make_double2(bout[1 + 2 * e] / nn, bout[2 + 2 * e] / nn);
            }
            return bout[0];
        };
        const double norm2_0 = save(0);
        if (tid == 0) {
            norm2 = norm2_0;
            t = J.tlist[0];
            h = htry = t_target = 0.0;
            draw = 0;
            idx = 1;
            attempts = 0;
            ctl.init();
            r = philox_uniform(J.seed, traj, draw++);
            if (J.n_c == 0) r = 0.0;   // no channel to jump to: never below the threshold
            rhs_evals += 1;
        }
        // k_1 = f of the current state
        auto k1_of = [&](int q) -> double2 {
            if constexpr (MIXED) {
                const float2 a = FHp(ys)[q], b = FLp(ys)[q];
                return make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
            } else {
                return Kp(0)[q];
            }
        };
        // ---- starting step ----
        if (J.fixed) {
            if (tid == 0) h = J.dt_fixed;
        } else if (J.dt0 > 0.0) {
            if (tid == 0) h = J.dt0;
        } else {
            double s0 = 0.0, s1 = 0.0;
            for (int q = tid; q < n; q += MW_T) {
                const double2 y = Yp(ys)[q];
                const double2 f0 = k1_of(q);
                const float a = sqrtf((float)(y.x * y.x + y.y * y.y));
                const float sc = (float)J.atol + (float)J.rtol * a;
                const float q0 = a / sc, q1 = sqrtf((float)(f0.x * f0.x + f0.y * f0.y)) / sc;
                s0 += (double)(q0 * q0);
                s1 += (double)(q1 * q1);
            }
            red.stage(0, s0);
            red.stage(1, s1);
            red.finish(2);
            const double d0 = sqrt(bout[0] / n), d1 = sqrt(bout[1] / n);
            const double h0 = start_h0(d0, d1);
            for (int q = tid; q < n; q += MW_T) {
                const double2 y = Yp(ys)[q];
                const double2 f0 = k1_of(q);
                X1[q] = from_d2_mc<T2>(make_double2(y.x + h0 * f0.x, y.y + h0 * f0.y));
            }
            if constexpr (!MIXED)
                if (warp == 0 && J.n_td > 0) publish_td_at(J.tlist[0] + h0);
            __syncthreads();
            double s2 = 0.0;
            for (int q = tid; q < n; q += MW_T) {
                const double2 y = Yp(ys)[q];
                const double2 f1 = to_d2_mc(rhs_td(q, X1, 7));
                const double2 f0 = k1_of(q);
                const float sc = (float)J.atol + (float)J.rtol * sqrtf((float)(y.x * y.x + y.y * y.y));
                const float dx = (float)(f1.x - f0.x), dy = (float)(f1.y - f0.y);
                const float qq = sqrtf(dx * dx + dy * dy) / sc;
                s2 += (double)(qq * qq);
            }
            red.stage(0, s2);
            red.finish(1);
            if (tid == 0) {
                rhs_evals += 1;
                h = start_h(h0, d1, sqrt(bout[0] / n) / h0);
            }
        }

        auto next_action = [&]() {
            cb.pub = 0;
            if constexpr (!MIXED) cb.tnow = t;
            for (;;) {
                if (status != QTL_OK || idx >= J.nt) {
                    cb.action = MC_DONE;
                    return;
                }
                t_target = J.tlist[idx];
                if (!(t_target >= J.tlist[idx - 1]) || !isfinite(t_target)) {
                    status = QTL_EINVAL;
                    continue;
                }
                if (!(t < t_target)) {
                    cb.action = MC_REPEAT;
                    cb.rsave = idx++;
                    return;
                }
                if (attempts >= J.max_steps) {
                    status = QTL_ESTEP;
                    continue;
                }
                ++attempts;
                bool land;
                htry = step_toward(h, t, t_target, J.fixed != 0, &land);
                cb.land = land;
                cb.action = MC_STEP;
                cb.coef[27] = htry;
                cb.pub = 1;
                return;
            }
        };
        // warp 0: htry * (a_sj, e_j) in FP64, one product per lane, when
        // thread 0 has set cb.pub (read after the warp barrier)
        auto publish_coefs = [&]() {
            __syncwarp();
            if (cb.pub) {
                const double hh = cb.coef[27];
                __syncwarp();
                double c = 0.0;
                if (lane < 21) {
                    int s = 1, j = lane;
                    while (j >= s) {
                        j -= s;
                        ++s;
                    }
                    c = hh * tab.a[s][j];
                } else if (lane < 28) {
                    c = hh * tab.e[lane - 21];
                }
                if (lane < 28) {
                    cb.coef[lane] = c;
                    cb.coeff[lane] = (float)c;
                }
                // time-dependent terms (FP64): f_k at the stage times t + c_s htry
                if constexpr (!MIXED) {
                    for (int i = lane; i < 6 * J.n_td; i += 32) {
                        const int st = 1 + i / J.n_td, qk = i % J.n_td;
                        cb.tdf[st][qk] = td_coef(J.tf[qk], cb.tnow + tab.c[st] * hh);
                    }
                }
                if constexpr (MIXED) {
                    if (lane >= 28) {
                        // htry^2 W_s for the stages s = 2..5 (0-based) of the increment form
                        const int st = lane - 26;
                        double w = 0.0;
                        for (int l = 0; l < st; ++l) w += tab.a[st][l] * tab.c[l];
                        cb.c2w[st] = (float)(hh * hh * w);
                        if (lane == 28) {
                            cb.hd = hh;
                            cb.hf = (float)hh;
                        } else if (lane == 29) {
                            double bc = 0.0;
                            for (int j = 0; j < 7; ++j) bc += tab.a[6][j] * tab.c[j];
                            cb.c2b = hh * hh * bc;
                        } else if (lane == 30) {
                            double ec = 0.0;
                            for (int j = 0; j < 7; ++j) ec += tab.e[j] * tab.c[j];
                            cb.c2e = (float)(hh * hh * ec);
                        } else {
                            cb.he7h = (float)(hh * tab.e[6] * hh);
                        }
                    }
                }
            }
            __syncwarp();
        };
        // One RK step of size htry (coefficients in cb.coef) from (y, k_1):
        // k_2..k_7 and y_new.  The sixth pass also forms the embedded error
        // (scaled, summed in FP32 as in the register-resident kernel) and
        // |y_new|^2 (FP64); both are left as thread partials in *se, *sn.
        auto rk_step = [&](float* se_out, double* sn_out) {
          if constexpr (MIXED) {
            float se = 0.f;
            double sn = 0.0;
            const double2* y = Yp(ys);
            double2* yn = Yp(ys ^ 1);
            const float2* fh = FHp(ys);
            const float2* fl = FLp(ys);
            float2* fnh = FHp(ys ^ 1);
            float2* fnl = FLp(ys ^ 1);
            const float2* f2 = (const float2*)Kp(1);
#pragma unroll 1
            for (int s = 1; s < 7; ++s) {
                float2* xb = (float2*)((s & 1) ? X0 : X1);
                if (s == 1) {
                    // stage 2 evaluates f2 = A f
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) xb[q] = __ldcs(fh + q);
                } else if (s < 6) {
                    // d_s = h^2 W_s f2 + sum_{2 <= l < s} h a_sl r_l
                    const int ca = mc_coef_a(s, 0);
                    const float w = cb.c2w[s];
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) {
                        const float2 g = __ldcs(f2 + q);
                        float ax = w * g.x, ay = w * g.y;
#pragma unroll
                        for (int j = 2; j < 5; ++j) {
                            if (j < s) {
                                const float2 kv = __ldcs((const float2*)Kp(j) + q);
                                const float a = cb.coeff[ca + j];
                                ax = fmaf(a, kv.x, ax);
                                ay = fmaf(a, kv.y, ay);
                            }
                        }
                        xb[q] = make_float2(ax, ay);
                    }
                } else {
                    // y_new = y + h f + h^2 (sum b c) f2 + sum_j h b_j r_j in FP64;
                    // the error partial h^2 (sum e c) f2 + sum_{j<7} h e_j r_j
                    // - h e_7 (f + h f2), completed by + h e_7 f_new below
                    const int ca = mc_coef_a(6, 0);
                    const double hd = cb.hd, c2b = cb.c2b;
                    const float hf = cb.hf, c2e = cb.c2e, he7 = cb.coeff[27], he7h = cb.he7h;
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) {
                        const float2 g = __ldcs(f2 + q);
                        const float2 fa = __ldcs(fh + q), fb = __ldcs(fl + q);
                        float rx = hf * fb.x, ry = hf * fb.y;
                        float ex = fmaf(c2e, g.x, fmaf(-he7h, g.x, -he7 * (fa.x + fb.x)));
                        float ey = fmaf(c2e, g.y, fmaf(-he7h, g.y, -he7 * (fa.y + fb.y)));
#pragma unroll
                        for (int j = 2; j < 6; ++j) {
                            const float2 kv = __ldcs((const float2*)Kp(j) + q);
                            const float b = cb.coeff[ca + j], e = cb.coeff[21 + j];
                            rx = fmaf(b, kv.x, rx);
                            ry = fmaf(b, kv.y, ry);
                            ex = fmaf(e, kv.x, ex);
                            ey = fmaf(e, kv.y, ey);
                        }
                        const double2 yv = __ldcs(y + q);
                        const double2 nv = make_double2(fma(c2b, (double)g.x, fma(hd, (double)fa.x, yv.x)) + (double)rx,
                                                        fma(c2b, (double)g.y, fma(hd, (double)fa.y, yv.y)) + (double)ry);
                        __stcs(yn + q, nv);
                        const float2 o = make_float2((float)nv.x, (float)nv.y);
                        XL[q] = lo_of(nv, o);
                        const float yx = (float)yv.x, yy = (float)yv.y;
                        const float a2 = fmaxf(yx * yx + yy * yy, o.x * o.x + o.y * o.y);
                        __stcs(SC + q, (float)J.atol + (float)J.rtol * sqrtf(a2));
                        __stcs((float2*)EP + q, make_float2(ex, ey));
                        sn += nv.x * nv.x + nv.y * nv.y;
                        xb[q] = o;
                    }
                }
                __syncthreads();
                if (s < 6) {
                    T2* ks = Kp(s);
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) __stcs(ks + q, rhs_row(q, (const T2*)xb));
                } else {
                    // f_new = A y_new, error free; completes the error estimate
                    const float he7 = cb.coeff[27];
                    for (int q = tid; q < n; q += MW_T) {
                        const float4 r = sell_row_dd<IT, XS, DC>(q, J.sl, J.sdesc, C, (const IT*)J.sci, J.svs32,
                                                                 J.svc32, J.svs32lo, J.svc32lo, xb, XL, pol);
                        __stcs(fnh + q, make_float2(r.x, r.y));
                        __stcs(fnl + q, make_float2(r.z, r.w));
                        const float2 ep = __ldcs((const float2*)EP + q);
                        const float fx = fmaf(he7, r.x, ep.x), fy = fmaf(he7, r.y, ep.y);
                        const float sc = __ldcs(SC + q);
                        se += (fx * fx + fy * fy) / (sc * sc);
                    }
                }
                if (xsingle) __syncthreads();
            }
            *se_out = se;
            *sn_out = sn;
          } else {
            float se = 0.f;
            double sn = 0.0;
            const double2* y = Yp(ys);
            double2* yn = Yp(ys ^ 1);
            const float2* yf = YFp(ys);
            float2* yfn = YFp(ys ^ 1);
#pragma unroll 1
            for (int s = 1; s < 7; ++s) {
                T2* xb = (s & 1) ? X0 : X1;
                // coefficients are read from shared memory inside the loops
                // (a broadcast load) rather than held in 12-24 registers
                const int ca = mc_coef_a(s, 0);
                if (s < 6) {
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) {
                        T ax = 0, ay = 0;
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            if (j < s) {
                                const T2 kv = __ldcs(Kp(j) + q);
                                const T a = coefT(ca + j);
                                ax = fma(a, kv.x, ax);
                                ay = fma(a, kv.y, ay);
                            }
                        }
                        T2 o;
                        if constexpr (MIXED) {
                            const float2 b = __ldcs(yf + q);
                            o.x = b.x + ax;
                            o.y = b.y + ay;
                        } else {
                            const double2 b = __ldcs(y + q);
                            o.x = b.x + ax;
                            o.y = b.y + ay;
                        }
                        xb[q] = o;
                    }
                } else {
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) {
                        T ax = 0, ay = 0, ex = 0, ey = 0;
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            const T2 kv = __ldcs(Kp(j) + q);
                            const T a = coefT(ca + j), b = coefT(21 + j);
                            ax = fma(a, kv.x, ax);
                            ay = fma(a, kv.y, ay);
                            ex = fma(b, kv.x, ex);
                            ey = fma(b, kv.y, ey);
                        }
                        const double2 yv = __ldcs(y + q);
                        const double2 nv = make_double2(yv.x + (double)ax, yv.y + (double)ay);
                        __stcs(yn + q, nv);
                        const T2 o = from_d2_mc<T2>(nv);
                        float yx, yy, nx, ny;
                        if constexpr (MIXED) {
                            __stcs(yfn + q, o);
                            const float2 b = __ldcs(yf + q);
                            yx = b.x;
                            yy = b.y;
                            nx = o.x;
                            ny = o.y;
                        } else {
                            yx = (float)yv.x;
                            yy = (float)yv.y;
                            nx = (float)nv.x;
                            ny = (float)nv.y;
                        }
                        const float a2 = fmaxf(yx * yx + yy * yy, nx * nx + ny * ny);
                        __stcs(SC + q, (float)J.atol + (float)J.rtol * sqrtf(a2));
                        T2 ep;
                        ep.x = ex;
                        ep.y = ey;
                        __stcs(EP + q, ep);
                        sn += nv.x * nv.x + nv.y * nv.y;
                        xb[q] = o;
                    }
                }
                __syncthreads();
                T2* ks = Kp(s);
                if (s < 6) {
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) __stcs(ks + q, rhs_td(q, xb, s));
                } else {
                    const T he6 = coefT(27);
#pragma unroll 2
                    for (int q = tid; q < n; q += MW_T) {
                        const T2 kv = rhs_td(q, xb, 6);
                        __stcs(ks + q, kv);
                        const T2 ep = __ldcs(EP + q);
                        const float fx = (float)fma(he6, kv.x, ep.x);
                        const float fy = (float)fma(he6, kv.y, ep.y);
                        const float sc = __ldcs(SC + q);
                        se += (fx * fx + fy * fy) / (sc * sc);
                    }
                }
                if (xsingle) __syncthreads();
            }
            *se_out = se;
            *sn_out = sn;
          }
        };
        // FP32 error sum and FP64 |y_new|^2, warps -> thread 0.
        auto reduce_step = [&](float se, double sn, float* S, double* N) {
            se = mc_warp_sum_f(se);
            sn = mc_warp_sum(sn);
            if (lane == 0) {
                cb.wf[warp] = se;
                cb.wd[warp] = sn;
            }
            __syncthreads();
            if (tid == 0) {
                float a = 0.f;
                double b = 0.0;
                for (int w = 0; w < nw; ++w) {
                    a += cb.wf[w];
                    b += cb.wd[w];
                }
                *S = a;
                *N = b;
            }
        };

        if (tid == 0) next_action();
        if (warp == 0) publish_coefs();
        __syncthreads();

        for (;;) {
            const int action = cb.action;
            if (action == MC_DONE) break;
            if (action == MC_REPEAT) {
                const double nn = save(cb.rsave);
                if (tid == 0) {
                    norm2 = nn;
                    next_action();
                }
                if (warp == 0) publish_coefs();
                __syncthreads();
                continue;
            }
            const bool land = cb.land;
            float se = 0.f;
            double sn = 0.0;
            rk_step(&se, &sn);
            float S = 0.f;
            double norm2_new = 0.0;
            reduce_step(se, sn, &S, &norm2_new);
            if (tid == 0) {
                rhs_evals += 6;
                const float err = sqrtf(S / (float)n);
                int accept = 1;
                float fac = 1.0f;
                if (!J.fixed) {
                    if (!(S <= (float)n)) {
                        accept = 0;
                        ++rej_steps;
                        h = htry * (double)ctl.on_reject(err);
                        if (h < J.dt_min || !isfinite(S)) status = QTL_ESTEP;
                    } else {
                        fac = ctl.on_accept(err);
                    }
                }
                cb.save = -1;
                cb.rootgo = 0;
                if (accept) {
                    ++acc_steps;
                    const double h_next = J.fixed ? J.dt_fixed : htry * (double)fac;
                    if (norm2_new >= r) {
                        t = land ? t_target : t + htry;
                        norm2 = norm2_new;
                        h = h_next;
                        if (land) cb.save = idx++;
                    } else {
                        // jump inside [t, t + htry]: Illinois on ln|psi|^2 - ln r
                        accept = 2;
                        h = h_next;
                        log_r = log(r);
                        lo = 0.0;
                        glo = log(norm2) - log_r;
                        hi = htry;
                        ghi = log(norm2_new) - log_r;
                        tau = hi;
                        side = 0;
                        it = 0;
                        cb.pub = 0;
                        if (!(hi - lo <= 1e-10 * fmax(1.0, fabs(t)))) {
                            tau = (lo * ghi - hi * glo) / (ghi - glo);
                            cb.rootgo = 1;
                            cb.coef[27] = tau;
                            cb.pub = 1;
                        }
                    }
                }
                cb.accept = accept;
                if (accept != 2) next_action();
            }
            if (warp == 0) publish_coefs();
            __syncthreads();
            const int accept = cb.accept;
            if (accept == 1) {
                ys ^= 1;
                k0s = 6 - k0s;
                const int sv = cb.save;
                if (sv >= 0) save(sv);
                continue;
            }
            if (accept == 0) continue;
            // ---- quantum jump: locate the crossing ----
            while (cb.rootgo) {
                rk_step(&se, &sn);
                float dummy = 0.f;
                double n2 = 0.0;
                reduce_step(0.f, sn, &dummy, &n2);
                if (tid == 0) {
                    rhs_evals += 6;
                    ++it;
                    const double gv = log(n2) - log_r;
                    int go = 1;
                    if (gv > 0) {
                        lo = tau;
                        glo = gv;
                        if (side == 1) ghi *= 0.5;
                        side = 1;
                    } else if (gv < 0) {
                        hi = tau;
                        ghi = gv;
                        if (side == -1) glo *= 0.5;
                        side = -1;
                    } else {
                        go = 0;
                    }
                    if (go && (it >= 30 || hi - lo <= 1e-10 * fmax(1.0, fabs(t)))) go = 0;
                    if (go) {
                        tau = (lo * ghi - hi * glo) / (ghi - glo);
                        cb.coef[27] = tau;
                    }
                    cb.rootgo = go;
                    cb.pub = go;
                }
                if (warp == 0) publish_coefs();
                __syncthreads();
            }
            // psi* = y_new (last evaluated point); channel weights |C_c psi*|^2
            const double2* ps = Yp(ys ^ 1);
            for (int c = 0; c < J.n_c; ++c) {
                double s = 0.0;
                for (int q = tid; q < n; q += MW_T) {
                    const int i = c * n + q;
                    double vx = 0.0, vy = 0.0;
                    for (int p = __ldg(J.crp + i); p < __ldg(J.crp + i + 1); ++p) {
                        const double2 cv = J.cv[p];
                        const double2 v = ps[__ldg(J.cci + p)];
                        vx += cv.x * v.x - cv.y * v.y;
                        vy += cv.x * v.y + cv.y * v.x;
                    }
                    s += vx * vx + vy * vy;
                }
                red.stage(c, s);
            }
            red.finish(J.n_c);
            if (tid == 0) {
                double total = 0.0;
                for (int c = 0; c < J.n_c; ++c) total += bout[c];
                const double u = philox_uniform(J.seed, traj, draw++);
                int ch = J.n_c - 1;
                double acc = 0.0;
                for (int c = 0; c < J.n_c; ++c) {
                    acc += bout[c];
                    if (acc >= u * total) {
                        ch = c;
                        break;
                    }
                }
                cb.ch = ch;
                cb.inv = 1.0 / sqrt(bout[ch]);
                r = philox_uniform(J.seed, traj, draw++);
                t = t + tau;
                ++jumps;
                rhs_evals += 1;
                next_action();
            }
            if (warp == 0) publish_coefs();
            __syncthreads();
            // psi <- C_ch psi* / |C_ch psi*| into Y[ys] (y's old value is no
            // longer needed), then k_1 = A psi
            double n2p = 0.0;
            {
                const int ch = cb.ch;
                const double inv = cb.inv;
                for (int q = tid; q < n; q += MW_T) {
                    const int i = ch * n + q;
                    double vx = 0.0, vy = 0.0;
                    for (int p = __ldg(J.crp + i); p < __ldg(J.crp + i + 1); ++p) {
                        const double2 cv = J.cv[p];
                        const double2 v = ps[__ldg(J.cci + p)];
                        vx += cv.x * v.x - cv.y * v.y;
                        vy += cv.x * v.y + cv.y * v.x;
                    }
                    const double2 nv = make_double2(vx * inv, vy * inv);
                    Yp(ys)[q] = nv;
                    const T2 o = from_d2_mc<T2>(nv);
                    if constexpr (MIXED) XL[q] = lo_of(nv, o);
                    X0[q] = o;
                    n2p += nv.x * nv.x + nv.y * nv.y;
                }
            }
            if constexpr (!MIXED)
                if (warp == 0 && J.n_td > 0) publish_td_at(cb.tnow);   // the time after the jump
            __syncthreads();
            if constexpr (MIXED) {
                base_deriv(ys, X0);
            } else {
                T2* k0 = Kp(0);
                for (int q = tid; q < n; q += MW_T) k0[q] = rhs_td(q, X0, 7);
            }
            {
                float dummy = 0.f;
                double n2 = 0.0;
                reduce_step(0.f, n2p, &dummy, &n2);  // |psi|^2 after the jump
                if (tid == 0) norm2 = n2;
            }
            __syncthreads();
        }
        if (tid == 0) s_next = J.wnext ? (int)gridDim.x + atomicAdd(J.wnext, 1) : jt + (int)gridDim.x;
        __syncthreads();
    }
    if (tid == 0) {
        if (status != QTL_OK) atomicCAS((int*)&J.info->status, 0, status);
        atomicAdd((unsigned long long*)&J.info->steps_acc, (unsigned long long)acc_steps);
        atomicAdd((unsigned long long*)&J.info->steps_rej, (unsigned long long)rej_steps);
        atomicAdd((unsigned long long*)&J.info->rhs_evals, (unsigned long long)rhs_evals);
        atomicAdd((unsigned long long*)&J.info->jumps, (unsigned long long)jumps);
    }
}

template <bool MIXED, class IT, bool XS>
static cudaError_t mw_occupancy1(size_t smem, int* per_sm) {
    auto kern = mc_wide_kernel<MIXED, IT, XS, true>;
    cudaError_t e0 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e0 != cudaSuccess) return e0;
    int p0 = 0;
    e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, kern, MW_T, smem);
    if (e0 != cudaSuccess) return e0;
    auto kern2 = mc_wide_kernel<MIXED, IT, XS, false>;
    cudaError_t e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern2, MW_T, smem);
    if (p0 < *per_sm) *per_sm = p0;
    return e;
}
template <bool MIXED, class IT>
static cudaError_t mw_occupancy(size_t smem, int xsmem, int* per_sm) {
    return xsmem ? mw_occupancy1<MIXED, IT, true>(smem, per_sm)
                 : mw_occupancy1<MIXED, IT, false>(smem, per_sm);
}

template <bool MIXED, class IT>
static void mw_launch(const McJob& J, const McWidePlan& p, const SellConst& C, cudaStream_t st) {
    if (J.sdesc_const) {
        if (p.xsmem)
            mc_wide_kernel<MIXED, IT, true, true><<<p.grid, MW_T, p.smem, st>>>(J, C);
        else
            mc_wide_kernel<MIXED, IT, false, true><<<p.grid, MW_T, p.smem, st>>>(J, C);
    } else {
        if (p.xsmem)
            mc_wide_kernel<MIXED, IT, true, false><<<p.grid, MW_T, p.smem, st>>>(J, C);
        else
            mc_wide_kernel<MIXED, IT, false, false><<<p.grid, MW_T, p.smem, st>>>(J, C);
    }
}

// Per-precision instantiations, compiled in separate translation units
// (mc_wide.cu: FP64, mc_wide_mixed.cu: mixed) so that they build in
// parallel.
cudaError_t mw_occupancy_fp64(size_t smem, int xsmem, int* per_sm);
cudaError_t mw_occupancy_mixed(size_t smem, int xsmem, int* per_sm);
void mw_launch_fp64(const McJob& J, const McWidePlan& p, const SellConst& C, cudaStream_t st);
void mw_launch_mixed(const McJob& J, const McWidePlan& p, const SellConst& C, cudaStream_t st);

}  // namespace qtl
