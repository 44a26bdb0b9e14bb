// mesolve for large density matrices (n*n beyond what one cluster holds):
// one cooperative, persistent grid per solve integrating the Lindblad
// equation (paper Sec. 3.2) in product form,
//     d rho / dt = A rho + rho B + sum_k C_k rho C_k^dag,
//     A = -i H - 1/2 sum_k C_k^dag C_k,   B = i H - 1/2 sum_k C_k^dag C_k,
// so that the n^2 x n^2 Liouvillian is never formed.  rho is stored column
// major.  A and B^T are read in pattern-compressed sliced ELLPACK (32-row
// slices whose entry positions carry an XOR or offset column rule and a
// uniform or per-row value), the collapse operators as per-row column maps.
//
// Work is split into warp units of 32 rows (one slice of A) x 4 columns (four
// rows of one slice of B^T).  A unit loads its own entries once; an XOR column
// of A below 32 is a warp shuffle, an XOR column of B^T below 4 a register of
// the same lane, and every other operand a gather through L2.
//
// Hermitian mode.  With H = H^dag (checked exactly on the host) a Hermitian
// rho stays Hermitian, so when rho0 is (to 1e-13 of its largest entry, or a
// ket) only the entries a >= b are integrated: the stage inputs and the
// state are written to both triangles (rho[b, a] = conj(rho[a, b])) and the
// error norms weight off-diagonal entries twice.  Otherwise every entry is
// integrated.
//
// A step is 7 grid-wide phases: the first stage input; then for each stage
// its right-hand side fused with the next stage's input (of the same entry);
// the last phase adds the error-norm partials.  Every block reduces the
// per-block partials in the same fixed order and takes the same decision
// (controller and tlist landing in thread 0 of each block, identical to the
// cluster kernel's).  Accepting a step swaps the roles of the y / y_new
// buffers and of the first and last stage slots; nothing is copied.
// Expectation values Tr(O rho) are summed in FP64 over the observables'
// stored entries into per-block partials, added in block order at the end.
//
// Precision.  FP64: everything in FP64.  MIXED: the state is an FP32 pair
// (~48 bits) and the integration is in increment form, k_s = f + L delta_s
// with f = L y kept as an FP32 pair: the FP32 operator only ever acts on the
// O(h) increments delta_s, and f is re-evaluated from y in FP64 every few
// accepted steps.  Expectation values are FP64.
#include <cooperative_groups.h>

#include <type_traits>

#include "internal.h"
#include "rk.cuh"
#include "td.cuh"

namespace cg = cooperative_groups;

namespace qtl {

constexpr int MG_T = 512;
constexpr int MG_NW = MG_T / 32;
constexpr int MG_EMAX = 64;

enum { MG_STEP = 0, MG_REPEAT = 1, MG_DONE = 2 };

template <bool MIXED>
struct GPrec;
template <>
struct GPrec<false> {
    using T = double;
    using T2 = double2;
};
template <>
struct GPrec<true> {
    using T = float;
    using T2 = float2;
};

struct MgCtl0 {
    double t, h, htry, t_target;
    long long attempts, steps_acc, steps_rej, rhs_evals;
    int idx, status;
    int since_refresh;    // accepted steps since the last FP64 base evaluation
    CtlF ctl;
};

struct MgShared {
    float wf[MG_NW], wf2[MG_NW];
    double wd[MG_NW][2 * MG_EMAX];
    double coef[34];      // h a_sj (21), h e_j (7), h c_s for s = 1..6 (6)
    float coeff[34];
    double h0, d1;
    float red_a, red_b;
    int action, land, accept, save_idx, repeat_idx, refresh_now;
    double tnow;                     // the step's start (time-dependent terms)
    double2 tdf[7][QTL_MAX_TD];      // f_k at t + c_s h (slots 1..6) and at one other time (slot 0)
};

__device__ __forceinline__ double2 g_to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 g_to_d2(float2 v) { return make_double2(v.x, v.y); }
template <class T2>
__device__ __forceinline__ T2 g_from_d2(double2 v);
template <>
__device__ __forceinline__ double2 g_from_d2<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 g_from_d2<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}

template <class V>
__device__ __forceinline__ V g_warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ RHS
// One warp work unit: rows a = 32 s + lane (one slice of A's sliced
// ELLPACK) and the MG_CB columns b0 .. b0 + MG_CB - 1 (b0 a multiple of
// MG_CB, so the columns are neighbouring rows of one slice of B^T).  The
// unit's own entries Y[a, b0 + k] are loaded once; an XOR column of A below
// 32 is then a shuffle within the warp and an XOR column of B^T below MG_CB
// a register of the same lane.  Every other entry is a gather through L2
// (Y is rewritten every stage).  Accumulation as in the trajectory kernel:
// real parts into (ax, ay), imaginary parts into (bx, by).
constexpr int MG_CB = 4;

template <int CB, class T2>
__device__ __forceinline__ T2 mg_sel(const T2 (&v)[CB], int i) {
    T2 r = v[0];
#pragma unroll
    for (int j = 1; j < CB; ++j) r = i == j ? v[j] : r;
    return r;
}
__device__ __forceinline__ float2 mg_shfl(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ double2 mg_shfl(double2 v, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

template <int G, class T, class T2, class V>
__device__ __forceinline__ void mg_acc(const V& v, const T2& x, T& ar, T& ai) {
    if constexpr (G == 0) {
        ar = fma(v, x.x, ar);
        ai = fma(v, x.y, ai);
    } else if constexpr (G == 1) {
        ar = fma(-v, x.y, ar);
        ai = fma(v, x.x, ai);
    } else {
        ar = fma(v.x, x.x, ar);
        ai = fma(v.x, x.y, ai);
        ar = fma(-v.y, x.y, ar);
        ai = fma(v.y, x.x, ai);
    }
}

template <bool MIXED>
struct MgVals {
    using T = typename GPrec<MIXED>::T;
    using T2 = typename GPrec<MIXED>::T2;
    const T* vs;
    const T2* vc;
    __device__ MgVals(const SellRef& r) {
        if constexpr (MIXED) {
            vs = r.vs32;
            vc = r.vc32;
        } else {
            vs = r.vs64;
            vc = r.vc64;
        }
    }
};

// (A Y)[a, b0 + k]: group G of row slice s.
template <int G, int CB, bool MIXED, class T, class T2>
__device__ __forceinline__ void mg_a_group(const SellRef& A, const MgVals<MIXED>& V, int d0, int w, int cbase,
                                           int vbase, const T2* __restrict__ Y, size_t n, int nn, int a, bool arow,
                                           int lane, int b0, const T2 (&yo)[CB],
                                           T (&ar)[CB], T (&ai)[CB]) {
    using VT = typename std::conditional<G == 2, T2, T>::type;
    const VT* vp;
    if constexpr (G == 2)
        vp = V.vc;
    else
        vp = V.vs;
#pragma unroll 2
    for (int p = 0; p < w; ++p) {
        const int4 d = __ldg(A.desc + d0 + p);
        VT v;
        if (d.x & SELL_VAL_UNIFORM) {
            if constexpr (G < 2 && MIXED)
                v = __int_as_float(d.w);
            else
                v = __ldg(vp + d.z);
        } else {
            v = __ldg(vp + vbase + d.z + lane);
        }
        const int mode = d.x & 3;
        if (mode == SELL_COL_XOR && d.y < 32) {
#pragma unroll
            for (int k = 0; k < CB; ++k) mg_acc<G>(v, mg_shfl(yo[k], d.y), ar[k], ai[k]);
        } else {
            const int c = mode == SELL_COL_XOR      ? (a ^ d.y)
                          : mode == SELL_COL_OFFSET ? (a + d.y)
                                                    : __ldg(A.ci + cbase + d.y + lane);
            T2 x[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                x[k].x = 0;
                x[k].y = 0;
                if (arow) x[k] = __ldcg(Y + (size_t)c + n * (size_t)min(b0 + k, nn - 1));
            }
#pragma unroll
            for (int k = 0; k < CB; ++k) mg_acc<G>(v, x[k], ar[k], ai[k]);
        }
    }
}

// (Y B)[a, b0 + k] = sum_c Y[a, c] B^T[b0 + k, c]: group G of column slice
// b0 >> 5 (warp-uniform columns and values).
template <int G, int CB, bool MIXED, class T, class T2>
__device__ __forceinline__ void mg_b_group(const SellRef& B, const MgVals<MIXED>& V, int d0, int w, int cbase,
                                           int vbase, const T2* __restrict__ Y, size_t n, int nn, int a,
                                           bool arow, int b0, const T2 (&yo)[CB], T (&ar)[CB],
                                           T (&ai)[CB]) {
    using VT = typename std::conditional<G == 2, T2, T>::type;
    const VT* vp;
    if constexpr (G == 2)
        vp = V.vc;
    else
        vp = V.vs;
    const int l0 = b0 & 31;
#pragma unroll 2
    for (int p = 0; p < w; ++p) {
        const int4 d = __ldg(B.desc + d0 + p);
        const bool uni = (d.x & SELL_VAL_UNIFORM) != 0;
        VT vu;
        if constexpr (G < 2 && MIXED)
            vu = __int_as_float(d.w);
        else
            vu = __ldg(vp + (uni ? d.z : vbase + d.z + l0));
        const int mode = d.x & 3;
        const bool reg = mode == SELL_COL_XOR && d.y < CB;
        T2 x[CB];
        VT v[CB];
#pragma unroll
        for (int k = 0; k < CB; ++k) {
            const int b = b0 + k;
            v[k] = uni ? vu : __ldg(vp + vbase + d.z + l0 + k);
            x[k].x = 0;
            x[k].y = 0;
            if (b < nn) {
                if (reg) {
                    x[k] = mg_sel<CB>(yo, k ^ d.y);
                } else {
                    const int c = mode == SELL_COL_XOR      ? (b ^ d.y)
                                  : mode == SELL_COL_OFFSET ? (b + d.y)
                                                            : __ldg(B.ci + cbase + d.y + l0 + k);
                    if (arow) x[k] = __ldcg(Y + (size_t)a + n * (size_t)c);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < CB; ++k) mg_acc<G>(v[k], x[k], ar[k], ai[k]);
    }
}

// The product-form right-hand side A Y + Y B + sum_c C_c Y C_c^dag on one
// unit; out[k] is entry (a, b0 + k) (garbage where a or b0 + k >= n).
template <bool MIXED, int CB, bool TD = !MIXED>
__device__ __forceinline__ void rhs_unit(const MgJob& J, const typename GPrec<MIXED>::T2* __restrict__ Y,
                                         int s, int b0, int lane, typename GPrec<MIXED>::T2 (&out)[CB],
                                         const double2* __restrict__ tdf = nullptr) {
    using T = typename GPrec<MIXED>::T;
    using T2 = typename GPrec<MIXED>::T2;
    const int nn = J.n;
    const size_t n = (size_t)nn;
    const int a = 32 * s + lane;
    const bool arow = a < nn;
    T2 yo[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        yo[k].x = 0;
        yo[k].y = 0;
        if (arow) yo[k] = __ldcg(Y + (size_t)a + n * (size_t)min(b0 + k, nn - 1));
    }
    T ar[CB], ai[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) ar[k] = ai[k] = 0;
    // A Y
    {
        const MgVals<MIXED> V(J.a);
        const int4 h0 = __ldg(J.a.sl + 2 * s), h1 = __ldg(J.a.sl + 2 * s + 1);
        mg_a_group<0, CB, MIXED, T, T2>(J.a, V, h0.x, h0.y, h1.x, h1.y, Y, n, nn, a, arow, lane, b0, yo, ar, ai);
        mg_a_group<1, CB, MIXED, T, T2>(J.a, V, h0.x + h0.y, h0.z, h1.x, h1.y, Y, n, nn, a, arow, lane, b0, yo, ar, ai);
        mg_a_group<2, CB, MIXED, T, T2>(J.a, V, h0.x + h0.y + h0.z, h0.w, h1.x, h1.z, Y, n, nn, a, arow, lane, b0, yo, ar, ai);
    }
    // Y B
    {
        const MgVals<MIXED> V(J.bt);
        const int sb = b0 >> 5;
        const int4 h0 = __ldg(J.bt.sl + 2 * sb), h1 = __ldg(J.bt.sl + 2 * sb + 1);
        mg_b_group<0, CB, MIXED, T, T2>(J.bt, V, h0.x, h0.y, h1.x, h1.y, Y, n, nn, a, arow, b0, yo, ar, ai);
        mg_b_group<1, CB, MIXED, T, T2>(J.bt, V, h0.x + h0.y, h0.z, h1.x, h1.y, Y, n, nn, a, arow, b0, yo, ar, ai);
        mg_b_group<2, CB, MIXED, T, T2>(J.bt, V, h0.x + h0.y + h0.z, h0.w, h1.x, h1.z, Y, n, nn, a, arow, b0, yo, ar, ai);
    }
    // time-dependent terms (FP64 solves): f_k(t) ((-i H_k) Y + Y (i H_k))
    if constexpr (TD) {
        for (int q = 0; q < J.n_td; ++q) {
            T tr[CB], ti[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) tr[k] = ti[k] = 0;
            {
                const SellRef R = J.tsl[q];
                const MgVals<MIXED> V(R);
                const int4 h0 = __ldg(R.sl + 2 * s), h1 = __ldg(R.sl + 2 * s + 1);
                mg_a_group<0, CB, MIXED, T, T2>(R, V, h0.x, h0.y, h1.x, h1.y, Y, n, nn, a, arow, lane, b0, yo, tr, ti);
                mg_a_group<1, CB, MIXED, T, T2>(R, V, h0.x + h0.y, h0.z, h1.x, h1.y, Y, n, nn, a, arow, lane, b0, yo,
                                                tr, ti);
                mg_a_group<2, CB, MIXED, T, T2>(R, V, h0.x + h0.y + h0.z, h0.w, h1.x, h1.z, Y, n, nn, a, arow, lane,
                                                b0, yo, tr, ti);
            }
            {
                const SellRef R = J.tsl[J.n_td + q];
                const MgVals<MIXED> V(R);
                const int sb = b0 >> 5;
                const int4 h0 = __ldg(R.sl + 2 * sb), h1 = __ldg(R.sl + 2 * sb + 1);
                mg_b_group<0, CB, MIXED, T, T2>(R, V, h0.x, h0.y, h1.x, h1.y, Y, n, nn, a, arow, b0, yo, tr, ti);
                mg_b_group<1, CB, MIXED, T, T2>(R, V, h0.x + h0.y, h0.z, h1.x, h1.y, Y, n, nn, a, arow, b0, yo, tr,
                                                ti);
                mg_b_group<2, CB, MIXED, T, T2>(R, V, h0.x + h0.y + h0.z, h0.w, h1.x, h1.z, Y, n, nn, a, arow, b0,
                                                yo, tr, ti);
            }
            const double2 f = tdf[q];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                ar[k] += f.x * tr[k] - f.y * ti[k];
                ai[k] += f.x * ti[k] + f.y * tr[k];
            }
        }
    }
    // sum_c C_c Y C_c^dag
    if (J.cmap) {
        // every C_c has at most one entry per row: (C Y C^dag)_ab =
        // c(a) conj(c(b)) Y[m(a), m(b)], m the column map
        const T2* cmv = MIXED ? (const T2*)J.cmv32 : (const T2*)J.cmv64;
        for (int c = 0; c < J.n_c; ++c) {
            const int* cm = J.cmap + (size_t)c * n;
            const T2* cw = cmv + (size_t)c * n;
            const int ma = arow ? __ldg(cm + a) : -1;
            T2 u;
            u.x = 0;
            u.y = 0;
            if (ma >= 0) u = __ldg(cw + a);
            int mb[CB];
            T2 w[CB], x[CB];
#pragma unroll
            for (int k = 0; k < CB; ++k) {
                const int bc = min(b0 + k, nn - 1);
                mb[k] = __ldg(cm + bc);
                w[k] = __ldg(cw + bc);
                x[k].x = 0;
                x[k].y = 0;
                if (b0 + k < nn && mb[k] >= 0 && ma >= 0) x[k] = __ldcg(Y + (size_t)ma + n * (size_t)mb[k]);
            }
            if (J.c_real) {
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const T g = u.x * w[k].x;
                    ar[k] = fma(g, x[k].x, ar[k]);
                    ai[k] = fma(g, x[k].y, ai[k]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    const T gx = u.x * w[k].x + u.y * w[k].y, gy = u.y * w[k].x - u.x * w[k].y;
                    ar[k] = fma(gx, x[k].x, ar[k]);
                    ai[k] = fma(gx, x[k].y, ai[k]);
                    ar[k] = fma(-gy, x[k].y, ar[k]);
                    ai[k] = fma(gy, x[k].x, ai[k]);
                }
            }
        }
    } else {
        const T2* cv = MIXED ? (const T2*)J.cv32 : (const T2*)J.cv64;
        for (int c = 0; c < J.n_c; ++c) {
            const int pa0 = arow ? __ldg(J.crp + c * nn + a) : 0;
            const int pa1 = arow ? __ldg(J.crp + c * nn + a + 1) : 0;
            for (int p = pa0; p < pa1; ++p) {
                const T2 u = __ldg(cv + p);
                const T2* col = Y + (size_t)__ldg(J.cci + p);
#pragma unroll
                for (int k = 0; k < CB; ++k) {
                    if (b0 + k >= nn) continue;
                    const int rb = c * nn + b0 + k;
                    for (int q = __ldg(J.crp + rb); q < __ldg(J.crp + rb + 1); ++q) {
                        const T2 w = __ldg(cv + q);
                        const T gx = u.x * w.x + u.y * w.y, gy = u.y * w.x - u.x * w.y;
                        const T2 x = __ldcg(col + n * (size_t)__ldg(J.cci + q));
                        ar[k] = fma(gx, x.x, ar[k]);
                        ai[k] = fma(gx, x.y, ai[k]);
                        ar[k] = fma(-gy, x.y, ar[k]);
                        ai[k] = fma(gy, x.x, ai[k]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CB; ++k) {
        out[k].x = ar[k];
        out[k].y = ai[k];
    }
}

// v + inc for an unevaluated FP32 pair v = {hi.x, hi.y, lo.x, lo.y}: TwoSum
// on hi, the rounding error and lo folded into the new lo (~48-bit sum).
__device__ __forceinline__ float4 pair_add(float4 v, float2 inc) {
    auto two = [](float a, float b, float lo) {
        const float s1 = a + b, bb = s1 - a;
        const float err = (a - (s1 - bb)) + (b - bb) + lo;
        const float hi = s1 + err;
        return make_float2(hi, err - (hi - s1));
    };
    const float2 rx = two(v.x, inc.x, v.z), ry = two(v.y, inc.y, v.w);
    return make_float4(rx.x, ry.x, rx.y, ry.y);
}
__device__ __forceinline__ float4 pair_of(double2 v) {
    const float hx = (float)v.x, hy = (float)v.y;
    return make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
}
__device__ __forceinline__ double2 pair_val(float4 v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// Sum of one float per block over the grid, in a fixed order, identical in
// every block: each block reads all blocks' partials.
__device__ __forceinline__ float grid_sum_f(const float* __restrict__ part, int nb, MgShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float v = 0.f;
    for (int i = tid; i < nb; i += MG_T) v += __ldcg(part + i);
    v = g_warp_sum(v);
    if (lane == 0) sh.wf[warp] = v;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < MG_NW; ++w) s += sh.wf[w];
        sh.red_a = s;
    }
    __syncthreads();
    return sh.red_a;
}

// Block sum of a float (thread 0 gets it).
__device__ __forceinline__ float block_sum_f(float v, MgShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    v = g_warp_sum(v);
    if (lane == 0) sh.wf2[warp] = v;
    __syncthreads();
    float s = 0.f;
    if (tid == 0) {
#pragma unroll
        for (int w = 0; w < MG_NW; ++w) s += sh.wf2[w];
    }
    __syncthreads();
    return s;
}

// Largest of one float per block over the grid (every block gets it).
__device__ __forceinline__ float grid_max_f(const float* __restrict__ part, int nb, MgShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float v = 0.f;
    for (int i = tid; i < nb; i += MG_T) v = fmaxf(v, __ldcg(part + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh.wf[warp] = v;
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
#pragma unroll
        for (int w = 0; w < MG_NW; ++w) m = fmaxf(m, sh.wf[w]);
        sh.red_a = m;
    }
    __syncthreads();
    return sh.red_a;
}

// Largest of a float over the block (thread 0 gets it).
__device__ __forceinline__ float block_max_f(float v, MgShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh.wf2[warp] = v;
    __syncthreads();
    float m = 0.f;
    if (tid == 0) {
#pragma unroll
        for (int w = 0; w < MG_NW; ++w) m = fmaxf(m, sh.wf2[w]);
    }
    __syncthreads();
    return m;
}

// MIXED keeps two blocks (32 warps) per SM to hide the gather latency; FP64
// needs the larger register budget of one block per SM.
template <bool MIXED>
__global__ void __launch_bounds__(MG_T, MIXED ? 2 : 1) me_grid_kernel(MgJob J) {
    using T = typename GPrec<MIXED>::T;
    using T2 = typename GPrec<MIXED>::T2;
    __shared__ MgShared sh;
    cg::grid_group grid = cg::this_grid();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = gridDim.x;
    const size_t g0 = (size_t)blockIdx.x * MG_T + tid, G = (size_t)nb * MG_T;
    const size_t L = (size_t)J.L;
    const int n = J.n, NE2 = 2 * J.n_e;
    const RkTab& tab = RK_TABS[J.method];
    T2* kbase = (T2*)J.k;
    T2* ysb[2] = {(T2*)J.ys, (T2*)J.ys + L};
    // State buffers (current / candidate, swapped on accept).  FP64: one
    // double2 per entry.  MIXED: an unevaluated FP32 pair hi + lo per entry
    // (float4 {hi.x, hi.y, lo.x, lo.y}), updated with an error-free TwoSum:
    // ~48-bit state at FP32 cost (GB300 runs FP64 at 1/64 rate).
    using S = typename std::conditional<MIXED, float4, double2>::type;
    S* yb = (S*)J.y0buf;
    S* yn = (S*)J.y1buf;
    auto st_set = [&](S* buf, size_t e, double2 v) {
        if constexpr (MIXED) {
            const float hx = (float)v.x, hy = (float)v.y;
            buf[e] = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
        } else {
            buf[e] = v;
        }
    };
    auto st_d2 = [&](const S* buf, size_t e) -> double2 {   // the state in FP64
        const S v = __ldcg(buf + e);
        if constexpr (MIXED)
            return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
        else
            return v;
    };
    auto st_t2 = [&](const S* buf, size_t e) -> T2 {        // the state rounded to T
        const S v = buf[e];
        if constexpr (MIXED)
            return make_float2(v.x, v.y);
        else
            return v;
    };
    auto st_conj = [](S v) -> S {
        if constexpr (MIXED)
            return make_float4(v.x, -v.y, v.z, -v.w);
        else
            return make_double2(v.x, -v.y);
    };
    auto t2_conj = [](T2 v) -> T2 {
        v.y = -v.y;
        return v;
    };
    // candidate = current + inc (MIXED: TwoSum on hi, lo carries the error);
    // returns the stored candidate
    auto st_add = [&](const S* cur, S* out, size_t e, T2 inc) -> S {
        const S v = cur[e];
        if constexpr (MIXED) {
            const float4 r = pair_add(v, inc);
            out[e] = r;
            return r;
        } else {
            const double2 r = make_double2(v.x + inc.x, v.y + inc.y);
            out[e] = r;
            return r;
        }
    };
    auto st_hi = [](S v) -> T2 {
        if constexpr (MIXED)
            return make_float2(v.x, v.y);
        else
            return v;
    };
    // MIXED, increment form: the derivative f = L y at the step's start (the
    // FSAL stage) is kept as an FP32 pair; the other stages evaluate the FP32
    // operator on the O(h) increments only, k_s = f + L delta_s.  The next
    // step's f is f + L delta_7 (delta_7 = y_new - y), and every J.refresh
    // accepted steps it is instead L y_new evaluated in FP64, which removes the
    // drift (L32 - L)(y - y_r) of the FP32 operator.
    float4* bb = J.base;
    float4* bn = J.base + L;
    // stage slots: derivative j lives in buffer (slots >> 3j) & 7 (FSAL swaps 0 and 6)
    unsigned slots = 0u | 1u << 3 | 2u << 6 | 3u << 9 | 4u << 12 | 5u << 15 | 6u << 18;
    auto K = [&](int j) -> T2* { return kbase + (size_t)((slots >> (3 * j)) & 7u) * L; };

    // ---- Hermitian mode ----
    // With H = H^dag the equation maps Hermitian rho to Hermitian d rho / dt,
    // so only the entries a >= b are integrated and the stage inputs and the
    // state are mirrored (rho[b, a] = conj(rho[a, b])).  rho0 qualifies when
    // its anti-Hermitian part is at rounding level (<= 1e-13 max |rho0|); a
    // ket always does.
    bool herm = J.herm_h != 0;
    if (herm && !J.is_ket) {
        float asym = 0.f, mag = 0.f;
        for (size_t e = g0; e < L; e += G) {
            const int i = (int)(e % (size_t)n), j = (int)(e / (size_t)n);
            const double2 v = J.state0[e];
            mag = fmaxf(mag, (float)fmax(fabs(v.x), fabs(v.y)));
            if (i > j) {
                const double2 w = J.state0[(size_t)j + (size_t)n * i];
                asym = fmaxf(asym, (float)fmax(fabs(v.x - w.x), fabs(v.y + w.y)));
            } else if (i == j) {
                asym = fmaxf(asym, (float)fabs(v.y));
            }
        }
        const float ba = block_max_f(asym, sh), bm = block_max_f(mag, sh);
        if (tid == 0) {
            J.errpart[blockIdx.x] = ba;
            J.errpart[nb + blockIdx.x] = bm;
        }
        grid.sync();
        const float A = grid_max_f(J.errpart, nb, sh), M = grid_max_f(J.errpart + nb, nb, sh);
        herm = A <= 1e-13f * M;
        grid.sync();   // the partials are reused below
    }
    // Work units: warp wg takes units wg, wg + W, ...; unit {s, c} holds rows
    // 32 s .. 32 s + 31 and columns MG_CB c .. MG_CB c + MG_CB - 1.  An entry
    // (a, b) is owned by the unit holding it (in Hermitian mode: if a >= b).
    const int wg = blockIdx.x * MG_NW + warp, W = nb * MG_NW;
    const int nu = herm ? J.nu_tri : J.nu_all;
    auto for_owned = [&](auto&& body) {   // body(e, eT, a, b, k)
        for (int u = wg; u < nu; u += W) {
            const int2 us = __ldg(J.units + u);
            const int a = 32 * us.x + lane, b0 = MG_CB * us.y;
#pragma unroll
            for (int k = 0; k < MG_CB; ++k) {
                const int b = b0 + k;
                if (a < n && b < n && (!herm || a >= b))
                    body((size_t)a + (size_t)n * b, (size_t)b + (size_t)n * a, a, b, k);
            }
        }
    };
    // right-hand side of stage input `in` on every owned entry:
    // post(e, eT, a, b, k_entry)
    auto rhs_pass = [&](const T2* in, int slot, auto&& post) {
        for (int u = wg; u < nu; u += W) {
            const int2 us = __ldg(J.units + u);
            T2 r[MG_CB];
            rhs_unit<MIXED, MG_CB>(J, in, us.x, MG_CB * us.y, lane, r, sh.tdf[slot]);
            const int a = 32 * us.x + lane, b0 = MG_CB * us.y;
#pragma unroll
            for (int k = 0; k < MG_CB; ++k) {
                const int b = b0 + k;
                if (a < n && b < n && (!herm || a >= b))
                    post((size_t)a + (size_t)n * b, (size_t)b + (size_t)n * a, a, b, r[k]);
            }
        }
    };
    // MIXED: the FP64 right-hand side of J.y64 (two columns at a time, which
    // keeps the FP64 operands within the register budget)
    auto rhs_pass64 = [&](auto&& post) {
        for (int u = wg; u < nu; u += W) {
            const int2 us = __ldg(J.units + u);
            const int a = 32 * us.x + lane;
#pragma unroll 1
            for (int hb = 0; hb < MG_CB; hb += 2) {
                double2 r[2];
                rhs_unit<false, 2, false>(J, J.y64, us.x, MG_CB * us.y + hb, lane, r);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int b = MG_CB * us.y + hb + k;
                    if (a < n && b < n && (!herm || a >= b))
                        post((size_t)a + (size_t)n * b, (size_t)b + (size_t)n * a, a, b, r[k]);
                }
            }
        }
    };
    // weight of an owned entry in the error norms (all n^2 entries count)
    auto wt = [&](int a, int b) -> float { return herm && a != b ? 2.f : 1.f; };

    // ---- initial state, k1 ----
    for_owned([&](size_t e, size_t eT, int i, int j, int) {
        double2 v;
        if (J.is_ket) {
            const double2 a = J.state0[i], b = J.state0[j];
            v = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
        } else {
            v = J.state0[e];
        }
        st_set(yb, e, v);
        if constexpr (MIXED)
            J.y64[e] = v;
        else
            ysb[0][e] = v;
        if (herm && i != j) {
            const double2 c = make_double2(v.x, -v.y);
            st_set(yb, eT, c);
            if constexpr (MIXED)
                J.y64[eT] = c;
            else
                ysb[0][eT] = c;
        }
    });
    // warp 0 of every block: f_k(tp) into slot 0 (time-dependent terms, FP64)
    auto publish_td0 = [&](double tp) {
        if (warp == 0 && lane < J.n_td) sh.tdf[0][lane] = td_coef(J.tf[lane], tp);
    };
    publish_td0(J.tlist[0]);
    grid.sync();
    if constexpr (MIXED)
        rhs_pass64([&](size_t e, size_t, int, int, double2 r) { bb[e] = pair_of(r); });
    else
        rhs_pass(ysb[0], 0, [&](size_t e, size_t, int, int, T2 r) { K(0)[e] = r; });

    // Tr(O_e rho) for rho = src, per-block FP64 partials -> epart[idx][block]
    auto expect_partials = [&](const S* src, int idx) {
        for (int oe = 0; oe < J.n_e; ++oe) {
            double sr = 0.0, si = 0.0;
            for (size_t i = g0; i < (size_t)n; i += G) {
                const int r = oe * n + (int)i;
                for (int p = __ldg(J.orp + r); p < __ldg(J.orp + r + 1); ++p) {
                    const double2 o = J.ov[p];
                    const double2 v = st_d2(src, (size_t)__ldg(J.oci + p) + (size_t)n * i);
                    sr += o.x * v.x - o.y * v.y;
                    si += o.x * v.y + o.y * v.x;
                }
            }
            sr = g_warp_sum(sr);
            si = g_warp_sum(si);
            if (lane == 0) {
                sh.wd[warp][2 * oe] = sr;
                sh.wd[warp][2 * oe + 1] = si;
            }
        }
        __syncthreads();
        if (tid < NE2) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < MG_NW; ++w) s += sh.wd[w][tid];
            J.epart[((size_t)idx * nb + blockIdx.x) * NE2 + tid] = s;
        }
        __syncthreads();
    };
    auto states_write = [&](const S* src, int idx) {
        if (J.states)
            for (size_t e = g0; e < L; e += G) J.states[(size_t)idx * L + e] = st_d2(src, e);
    };
    grid.sync();
    expect_partials(yb, 0);
    states_write(yb, 0);

    // thread-0 control state (identical in every block), in shared memory so
    // that it takes no registers in the other threads
    __shared__ MgCtl0 z;
    double& t = z.t;
    double& h = z.h;
    double& htry = z.htry;
    double& t_target = z.t_target;
    int& idx = z.idx;
    int& status = z.status;
    long long& attempts = z.attempts;
    long long& steps_acc = z.steps_acc;
    long long& steps_rej = z.steps_rej;
    long long& rhs_evals = z.rhs_evals;
    CtlF& ctl = z.ctl;
    if (tid == 0) {
        t = J.tlist[0];
        h = htry = t_target = 0.0;
        idx = 1;
        status = QTL_OK;
        attempts = steps_acc = steps_rej = 0;
        rhs_evals = 1;
        z.since_refresh = 0;
        ctl.init();
    }

    // ---- starting step ----
    if (J.fixed) {
        if (tid == 0) h = J.dt_fixed;
    } else if (J.dt0 > 0.0) {
        if (tid == 0) h = J.dt0;
    } else {
        float s0 = 0.f, s1 = 0.f;
        auto f0_at = [&](size_t e) -> double2 {
            if constexpr (MIXED)
                return pair_val(bb[e]);
            else
                return g_to_d2(K(0)[e]);
        };
        for_owned([&](size_t e, size_t, int i, int j, int) {
            const double2 y = st_d2(yb, e);
            const double2 f0 = f0_at(e);
            const float a = sqrtf((float)(y.x * y.x + y.y * y.y));
            const float sc = (float)J.atol + (float)J.rtol * a;
            const float q0 = a / sc, q1 = sqrtf((float)(f0.x * f0.x + f0.y * f0.y)) / sc;
            s0 += wt(i, j) * (q0 * q0);
            s1 += wt(i, j) * (q1 * q1);
        });
        float b0 = block_sum_f(s0, sh), b1 = block_sum_f(s1, sh);
        if (tid == 0) {
            J.errpart[blockIdx.x] = b0;
            J.errpart[nb + blockIdx.x] = b1;
        }
        grid.sync();
        const float S0 = grid_sum_f(J.errpart, nb, sh), S1 = grid_sum_f(J.errpart + nb, nb, sh);
        const double d0 = sqrt((double)S0 / (double)L), d1 = sqrt((double)S1 / (double)L);
        const double h0 = start_h0(d0, d1);
        for_owned([&](size_t e, size_t eT, int i, int j, int) {
            const double2 f0 = f0_at(e);
            // MIXED probes with the increment h0 f0 (its derivative is f1 - f0)
            double2 y = make_double2(0.0, 0.0);
            if constexpr (!MIXED) y = st_d2(yb, e);
            const T2 o = g_from_d2<T2>(make_double2(y.x + h0 * f0.x, y.y + h0 * f0.y));
            ysb[1][e] = o;
            if (herm && i != j) ysb[1][eT] = t2_conj(o);
        });
        publish_td0(J.tlist[0] + h0);
        grid.sync();
        float s2 = 0.f;
        rhs_pass(ysb[1], 0, [&](size_t e, size_t, int i, int j, T2 r) {
            double2 d = g_to_d2(r);
            if constexpr (!MIXED) {
                const double2 f0 = g_to_d2(K(0)[e]);
                d = make_double2(d.x - f0.x, d.y - f0.y);
            }
            const double2 y = st_d2(yb, e);
            const float sc = (float)J.atol + (float)J.rtol * sqrtf((float)(y.x * y.x + y.y * y.y));
            const float dx = (float)d.x, dy = (float)d.y;
            const float q = sqrtf(dx * dx + dy * dy) / sc;
            s2 += wt(i, j) * (q * q);
        });
        float b2 = block_sum_f(s2, sh);
        __syncthreads();
        if (tid == 0) J.errpart[2 * nb + blockIdx.x] = b2;
        grid.sync();
        const float S2 = grid_sum_f(J.errpart + 2 * nb, nb, sh);
        if (tid == 0) {
            rhs_evals += 1;
            h = start_h(h0, d1, sqrt((double)S2 / (double)L) / h0);
        }
    }
    grid.sync();

    auto next_action = [&]() {
        sh.tnow = t;
        for (;;) {
            if (status != QTL_OK || idx >= J.nt) {
                sh.action = MG_DONE;
                return;
            }
            t_target = J.tlist[idx];
            if (!(t_target >= J.tlist[idx - 1]) || !isfinite(t_target)) {
                status = QTL_EINVAL;
                continue;
            }
            if (!(t < t_target)) {
                sh.action = MG_REPEAT;
                sh.repeat_idx = idx++;
                return;
            }
            if (attempts >= J.max_steps) {
                status = QTL_ESTEP;
                continue;
            }
            ++attempts;
            bool land;
            htry = step_toward(h, t, t_target, J.fixed != 0, &land);
            sh.land = land;
            sh.refresh_now = MIXED && z.since_refresh + 1 >= J.refresh;
            sh.action = MG_STEP;
            sh.coef[27] = htry;
            return;
        }
    };
    auto publish_coefs = [&]() {
        __syncwarp();
        if (sh.action == MG_STEP) {
            const double hh = sh.coef[27];
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
            } else {
                c = hh * tab.c[lane - 27];   // lanes 28..31: h c_1 .. h c_4
            }
            sh.coef[lane] = c;
            sh.coeff[lane] = (float)c;
            if (lane < 2) {                  // entries 32, 33: h c_5, h c_6
                const double c2 = hh * tab.c[5 + lane];
                sh.coef[32 + lane] = c2;
                sh.coeff[32 + lane] = (float)c2;
            }
            // f_k at the stage times t + c_s h (slots 1..6)
            for (int i = lane; i < 6 * J.n_td; i += 32) {
                const int st = 1 + i / J.n_td, q = i % J.n_td;
                sh.tdf[st][q] = td_coef(J.tf[q], sh.tnow + tab.c[st] * hh);
            }
        }
        __syncwarp();
    };
    auto coefT = [&](int i) -> T {
        if constexpr (MIXED)
            return sh.coeff[i];
        else
            return sh.coef[i];
    };
    if (tid == 0) next_action();
    if (warp == 0) publish_coefs();
    __syncthreads();

    // ---- main loop: one iteration per step attempt ----
    for (;;) {
        const int action = sh.action;
        if (action == MG_DONE) break;
        if (action == MG_REPEAT) {
            const int ri = sh.repeat_idx;
            if (tid < NE2)
                J.epart[((size_t)ri * nb + blockIdx.x) * NE2 + tid] =
                    __ldcg(J.epart + ((size_t)(ri - 1) * nb + blockIdx.x) * NE2 + tid);
            states_write(yb, ri);
            __syncthreads();
            if (tid == 0) next_action();
            if (warp == 0) publish_coefs();
            __syncthreads();
            continue;
        }
        const bool land = sh.land;
        // stage-2 input y + h a_21 k_1 (MIXED: the increment h a_21 f)
        {
            const T c = coefT(0);
            for_owned([&](size_t e, size_t eT, int i, int j, int) {
                T2 o;
                if constexpr (MIXED) {
                    const float4 f = bb[e];
                    o.x = c * f.x;
                    o.y = c * f.y;
                } else {
                    const T2 y = st_t2(yb, e), k0 = K(0)[e];
                    o.x = fma(c, k0.x, y.x);
                    o.y = fma(c, k0.y, y.y);
                }
                ysb[1][e] = o;
                if (herm && i != j) ysb[1][eT] = t2_conj(o);
            });
        }
        grid.sync();
        float se = 0.f;
#pragma unroll
        for (int s = 1; s < 7; ++s) {
            const T2* in = ysb[s & 1];
            // h a_{s+1,j} and h e_j from shared memory inside the pass (no registers held)
            auto ha = [&](int j) -> T { return coefT((s + 1) * s / 2 + j); };
            auto he = [&](int j) -> T { return coefT(21 + j); };
            // MIXED error estimate h sum_j e_j k_j = h sum_{j>=1} e_j p_j (the
            // e_j sum to zero, so the base f drops out); p7 = L delta_7
            auto mixed_err = [&](size_t e, int i, int j2, float2 p7) {
                T ex = he(6) * p7.x, ey = he(6) * p7.y;
#pragma unroll
                for (int j = 1; j < 6; ++j) {
                    const T2 kj = K(j)[e];
                    ex = fma(he(j), kj.x, ex);
                    ey = fma(he(j), kj.y, ey);
                }
                const T2 y = st_t2(yb, e), yv = st_t2(yn, e);
                const float a2 = fmaxf((float)(y.x * y.x + y.y * y.y), (float)(yv.x * yv.x + yv.y * yv.y));
                const float sc = (float)J.atol + (float)J.rtol * sqrtf(a2);
                const float fx = (float)ex, fy = (float)ey;
                se += wt(i, j2) * ((fx * fx + fy * fy) / (sc * sc));
            };
            if constexpr (MIXED) {
                if (s == 6 && sh.refresh_now) {
                    // FP64 base at y_new; p7 = L y_new - f
                    rhs_pass64([&](size_t e, size_t, int i, int j2, double2 r) {
                        const double2 f = pair_val(bb[e]);
                        bn[e] = pair_of(r);
                        mixed_err(e, i, j2, make_float2((float)(r.x - f.x), (float)(r.y - f.y)));
                    });
                } else {
                    rhs_pass(in, s, [&](size_t e, size_t eT, int i, int j2, T2 ks) {
                        if (s == 6) {
                            bn[e] = pair_add(bb[e], ks);
                            mixed_err(e, i, j2, ks);
                            return;
                        }
                        K(s)[e] = ks;
                        // delta_{s+1} = h c_{s+1} f + sum_{1<=j<=s} h a_{s+1,j} p_j
                        const float4 f = bb[e];
                        T ax = fma(ha(s), ks.x, coefT(27 + s + 1) * f.x);
                        T ay = fma(ha(s), ks.y, coefT(27 + s + 1) * f.y);
#pragma unroll
                        for (int j = 1; j < 5; ++j) {
                            if (j < s) {
                                const T2 kj = K(j)[e];
                                ax = fma(ha(j), kj.x, ax);
                                ay = fma(ha(j), kj.y, ay);
                            }
                        }
                        T2 d;
                        d.x = ax;
                        d.y = ay;
                        const bool mirror = herm && i != j2;
                        if (s + 1 < 6) {
                            ysb[(s + 1) & 1][e] = d;
                            if (mirror) ysb[(s + 1) & 1][eT] = t2_conj(d);
                        } else {
                            // delta_7 = y_new - y: the state update, then the
                            // last stage's input (FP64 y_new when the base is
                            // re-evaluated)
                            const S r = st_add(yb, yn, e, d);
                            if (mirror) yn[eT] = st_conj(r);
                            if (sh.refresh_now) {
                                const double2 v = pair_val(r);
                                J.y64[e] = v;
                                if (mirror) J.y64[eT] = make_double2(v.x, -v.y);
                            } else {
                                ysb[0][e] = d;
                                if (mirror) ysb[0][eT] = t2_conj(d);
                            }
                        }
                    });
                }
            } else {
                rhs_pass(in, s, [&](size_t e, size_t eT, int i, int j2, T2 ks) {
                    K(s)[e] = ks;
                    if (s < 6) {
                        // input of stage s+1: y + h sum_{j<=s} a_{s+1,j} k_j
                        T ax = ha(s) * ks.x, ay = ha(s) * ks.y;
    #pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            if (j < s) {
                                const T2 kj = K(j)[e];
                                ax = fma(ha(j), kj.x, ax);
                                ay = fma(ha(j), kj.y, ay);
                            }
                        }
                        T2 inc;
                        inc.x = ax;
                        inc.y = ay;
                        const bool mirror = herm && i != j2;
                        if (s + 1 < 6) {
                            const T2 y = st_t2(yb, e);
                            T2 o;
                            o.x = y.x + ax;
                            o.y = y.y + ay;
                            ysb[(s + 1) & 1][e] = o;
                            if (mirror) ysb[(s + 1) & 1][eT] = t2_conj(o);
                        } else {
                            // the last stage is evaluated at the candidate y_new
                            const S r = st_add(yb, yn, e, inc);
                            const T2 o = st_hi(r);
                            ysb[0][e] = o;
                            if (mirror) {
                                yn[eT] = st_conj(r);
                                ysb[0][eT] = t2_conj(o);
                            }
                        }
                    } else {
                        // error estimate e = h sum_j e_j k_j against sc = atol + rtol max(|y|, |y_new|)
                        T ex = he(6) * ks.x, ey = he(6) * ks.y;
    #pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            const T2 kj = K(j)[e];
                            ex = fma(he(j), kj.x, ex);
                            ey = fma(he(j), kj.y, ey);
                        }
                        const T2 y = st_t2(yb, e), yv = st_t2(yn, e);
                        const float a2 = fmaxf((float)(y.x * y.x + y.y * y.y), (float)(yv.x * yv.x + yv.y * yv.y));
                        const float sc = (float)J.atol + (float)J.rtol * sqrtf(a2);
                        const float fx = (float)ex, fy = (float)ey;
                        se += wt(i, j2) * ((fx * fx + fy * fy) / (sc * sc));
                    }
                });
            }
            if (s < 6) grid.sync();
        }
        const float bse = block_sum_f(se, sh);
        if (tid == 0) J.errpart[blockIdx.x] = bse;
        grid.sync();
        const float Se = grid_sum_f(J.errpart, nb, sh);
        // ---- decision (thread 0 of every block, identical), next action ----
        if (tid == 0) {
            rhs_evals += 6;
            const float err = sqrtf(Se / (float)L);
            bool acc = true;
            float fac = 1.0f;
            if (!J.fixed) {
                if (!(Se <= (float)L)) {
                    acc = false;
                    ++steps_rej;
                    h = htry * (double)ctl.on_reject(err);
                    if (h < J.dt_min || !isfinite(Se)) status = QTL_ESTEP;
                } else {
                    fac = ctl.on_accept(err);
                }
            }
            sh.accept = acc;
            sh.save_idx = -1;
            if (acc) {
                z.since_refresh = sh.refresh_now ? 0 : z.since_refresh + 1;
                ++steps_acc;
                t = land ? t_target : t + htry;
                h = J.fixed ? J.dt_fixed : htry * (double)fac;
                if (land) sh.save_idx = idx++;
            }
            next_action();
        }
        if (warp == 0) publish_coefs();
        __syncthreads();
        if (sh.accept) {
            S* tmp = yb;
            yb = yn;
            yn = tmp;
            float4* tb = bb;
            bb = bn;
            bn = tb;
            const unsigned k0 = slots & 7u, k6 = (slots >> 18) & 7u;
            slots = (slots & ~(7u | 7u << 18)) | k6 | k0 << 18;
            const int sv = sh.save_idx;
            if (sv >= 0) {
                expect_partials(yb, sv);
                states_write(yb, sv);
            }
        }
    }

    // ---- expectation values: block partials added in block order ----
    grid.sync();
    if (blockIdx.x == 0) {
        for (int v = tid; v < J.nt * NE2; v += MG_T) {
            const int ti = v / NE2, c2 = v % NE2;
            double s = 0.0;
            for (int r = 0; r < nb; ++r) s += __ldcg(J.epart + ((size_t)ti * nb + r) * NE2 + c2);
            double* ex = (double*)(J.expect + (size_t)(c2 >> 1) * J.nt + ti);
            ex[c2 & 1] = s;
        }
        if (tid == 0) {
            J.info->status = status;
            J.info->steps_acc = steps_acc;
            J.info->steps_rej = steps_rej;
            J.info->rhs_evals = rhs_evals;
            J.info->jumps = 0;
        }
    }
}

int me_grid_blocks(int precision) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (precision == QTL_MIXED)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, me_grid_kernel<true>, MG_T, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, me_grid_kernel<false>, MG_T, 0);
    if (per < 1) per = 1;
    if (per > 2) per = 2;
    return per * nsm;
}

cudaError_t launch_me_grid(const MgJob& J0, int precision, cudaStream_t st, int* grid_out) {
    MgJob J = J0;
    const int grid = *grid_out > 0 ? *grid_out : me_grid_blocks(precision);
    *grid_out = grid;
    void* args[] = {&J};
    count_launch();
    if (precision == QTL_MIXED)
        return cudaLaunchCooperativeKernel((void*)me_grid_kernel<true>, dim3(grid), dim3(MG_T), args, 0, st);
    return cudaLaunchCooperativeKernel((void*)me_grid_kernel<false>, dim3(grid), dim3(MG_T), args, 0, st);
}

}  // namespace qtl
