// mesolve for large density matrices (n*n beyond what one cluster holds):
// one cooperative, persistent grid per solve integrating the Lindblad
// equation (paper Sec. 3.2) in product form,
//     d rho / dt = A rho + rho B + sum_k C_k rho C_k^dag,
//     A = -i H - 1/2 sum_k C_k^dag C_k,   B = i H - 1/2 sum_k C_k^dag C_k,
// so that the n^2 x n^2 Liouvillian is never formed.  Each thread owns the
// column-major entries e = a + n b, e = g, g + G, ... (g its grid index), so
// a warp's gathers of rho[col, b] (A rho), rho[a, col] (rho B) and
// rho[col_p, col_q] (C rho C^dag) touch neighbouring addresses.
//
// A step is 7 grid-wide phases: the first stage input; then for each stage
// its right-hand side fused with the next stage's input (y + h sum_j a_sj k_j
// of the same entry); the last phase adds the error-norm partials.  Every
// block reduces the per-block partials in the same fixed order and takes the
// same decision (controller and tlist landing in thread 0 of each block,
// identical to the cluster kernel's).  Accepting a step swaps the roles of
// the y / y_new buffers and of the first and last stage slots; nothing is
// copied.  Expectation values Tr(O rho) are summed in FP64 over the
// observables' stored entries into per-block partials, added in block order
// at the end.
//
// Precision.  FP64: everything in FP64.  MIXED: stage inputs, derivatives
// and the right-hand side in FP32 (complex64 operators); y, y_new and the
// expectation values in FP64.
#include <cooperative_groups.h>

#include <type_traits>

#include "internal.h"
#include "rk.cuh"

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

struct MgShared {
    float wf[MG_NW], wf2[MG_NW];
    double wd[MG_NW][2 * MG_EMAX];
    double coef[28];
    float coeff[28];
    double h0, d1;
    float red_a, red_b;
    int action, land, accept, save_idx, repeat_idx;
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

// Product-form right-hand side at entry (a, b) of the stage input Y
// (column-major, L2-resident; read through L2 because Y is rewritten every
// stage).
template <class T2, class TV>
__device__ __forceinline__ T2 rhs_entry(const MgJob& J, const T2* __restrict__ Y, int a, int b,
                                        const TV* __restrict__ av, const TV* __restrict__ bv,
                                        const TV* __restrict__ cv, const void* cmvp) {
    using T = decltype(T2::x);
    const size_t n = (size_t)J.n;
    T ax = 0, ay = 0, bx = 0, by = 0;
    // A rho: row a of A against column b of Y
    {
        const int4 sg = __ldg(J.aseg + a);
        const T2* col = Y + n * (size_t)b;
        int p = sg.x;
        for (; p < sg.y; ++p) {
            const T v = __ldg(&av[p].x);
            const T2 x = __ldcg(col + __ldg(J.aci + p));
            ax = fma(v, x.x, ax);
            ay = fma(v, x.y, ay);
        }
        for (; p < sg.z; ++p) {
            const T v = __ldg(&av[p].y);
            const T2 x = __ldcg(col + __ldg(J.aci + p));
            bx = fma(-v, x.y, bx);
            by = fma(v, x.x, by);
        }
        for (; p < sg.w; ++p) {
            const TV v = __ldg(av + p);
            const T2 x = __ldcg(col + __ldg(J.aci + p));
            ax = fma(v.x, x.x, ax);
            ay = fma(v.x, x.y, ay);
            bx = fma(-v.y, x.y, bx);
            by = fma(v.y, x.x, by);
        }
    }
    // rho B: row a of Y against column b of B = row b of B^T
    {
        const int4 sg = __ldg(J.bseg + b);
        const T2* rowa = Y + a;
        int p = sg.x;
        for (; p < sg.y; ++p) {
            const T v = __ldg(&bv[p].x);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            ax = fma(v, x.x, ax);
            ay = fma(v, x.y, ay);
        }
        for (; p < sg.z; ++p) {
            const T v = __ldg(&bv[p].y);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            bx = fma(-v, x.y, bx);
            by = fma(v, x.x, by);
        }
        for (; p < sg.w; ++p) {
            const TV v = __ldg(bv + p);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            ax = fma(v.x, x.x, ax);
            ay = fma(v.x, x.y, ay);
            bx = fma(-v.y, x.y, bx);
            by = fma(v.y, x.x, by);
        }
    }
    // C rho C^dag
    if (J.cmap) {
        // every C_k has at most one entry per row: (C Y C^dag)_ab =
        // c(a) conj(c(b)) Y[m(a), m(b)], m the column map
        const TV* cmv = (const TV*)cmvp;
        for (int c = 0; c < J.n_c; ++c) {
            const int ma = __ldg(J.cmap + (size_t)c * n + a);
            const int mb = __ldg(J.cmap + (size_t)c * n + b);
            if (ma >= 0 && mb >= 0) {
                const TV u = __ldg(cmv + (size_t)c * n + a), w = __ldg(cmv + (size_t)c * n + b);
                const T gx = u.x * w.x + u.y * w.y, gy = u.y * w.x - u.x * w.y;
                const T2 x = __ldcg(Y + (size_t)ma + n * (size_t)mb);
                ax = fma(gx, x.x, ax);
                ay = fma(gx, x.y, ay);
                bx = fma(-gy, x.y, bx);
                by = fma(gy, x.x, by);
            }
        }
    } else
    for (int c = 0; c < J.n_c; ++c) {
        const int ra = c * J.n + a, rb = c * J.n + b;
        const int pa0 = __ldg(J.crp + ra), pa1 = __ldg(J.crp + ra + 1);
        const int qb0 = __ldg(J.crp + rb), qb1 = __ldg(J.crp + rb + 1);
        for (int p = pa0; p < pa1; ++p) {
            const TV u = __ldg(cv + p);
            const T2* col = Y + (size_t)__ldg(J.cci + p);
            for (int q = qb0; q < qb1; ++q) {
                const TV w = __ldg(cv + q);
                // u * conj(w)
                const T gx = u.x * w.x + u.y * w.y, gy = u.y * w.x - u.x * w.y;
                const T2 x = __ldcg(col + n * (size_t)__ldg(J.cci + q));
                ax = fma(gx, x.x, ax);
                ay = fma(gx, x.y, ay);
                bx = fma(-gy, x.y, bx);
                by = fma(gy, x.x, by);
            }
        }
    }
    T2 r;
    r.x = ax + bx;
    r.y = ay + by;
    return r;
}

// The same right-hand side for four entries (a, b[0..3]) of one row a: the
// row of A and the collapse maps of row a are loaded once and their gathers
// for the four columns are independent, so they overlap.
template <class T2, class TV>
__device__ __forceinline__ void rhs_row4(const MgJob& J, const T2* __restrict__ Y, int a,
                                         const int* b, T2* out, const TV* __restrict__ av,
                                         const TV* __restrict__ bv, const TV* __restrict__ cv,
                                         const void* cmvp) {
    using T = decltype(T2::x);
    const size_t n = (size_t)J.n;
    T ax[4], ay[4], bx[4], by[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ax[k] = ay[k] = bx[k] = by[k] = 0;
    // A rho: one pass over row a of A for all four columns
    {
        const int4 sg = __ldg(J.aseg + a);
        int p = sg.x;
        for (; p < sg.y; ++p) {
            const T v = __ldg(&av[p].x);
            const size_t c = (size_t)__ldg(J.aci + p);
            T2 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = __ldcg(Y + c + n * (size_t)b[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ax[k] = fma(v, x[k].x, ax[k]);
                ay[k] = fma(v, x[k].y, ay[k]);
            }
        }
        for (; p < sg.z; ++p) {
            const T v = __ldg(&av[p].y);
            const size_t c = (size_t)__ldg(J.aci + p);
            T2 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = __ldcg(Y + c + n * (size_t)b[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bx[k] = fma(-v, x[k].y, bx[k]);
                by[k] = fma(v, x[k].x, by[k]);
            }
        }
        for (; p < sg.w; ++p) {
            const TV v = __ldg(av + p);
            const size_t c = (size_t)__ldg(J.aci + p);
            T2 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = __ldcg(Y + c + n * (size_t)b[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ax[k] = fma(v.x, x[k].x, ax[k]);
                ay[k] = fma(v.x, x[k].y, ay[k]);
                bx[k] = fma(-v.y, x[k].y, bx[k]);
                by[k] = fma(v.y, x[k].x, by[k]);
            }
        }
    }
    // rho B: row b of B^T for each column (the same for a whole warp)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int4 sg = __ldg(J.bseg + b[k]);
        const T2* rowa = Y + a;
        int p = sg.x;
        for (; p < sg.y; ++p) {
            const T v = __ldg(&bv[p].x);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            ax[k] = fma(v, x.x, ax[k]);
            ay[k] = fma(v, x.y, ay[k]);
        }
        for (; p < sg.z; ++p) {
            const T v = __ldg(&bv[p].y);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            bx[k] = fma(-v, x.y, bx[k]);
            by[k] = fma(v, x.x, by[k]);
        }
        for (; p < sg.w; ++p) {
            const TV v = __ldg(bv + p);
            const T2 x = __ldcg(rowa + n * (size_t)__ldg(J.bci + p));
            ax[k] = fma(v.x, x.x, ax[k]);
            ay[k] = fma(v.x, x.y, ay[k]);
            bx[k] = fma(-v.y, x.y, bx[k]);
            by[k] = fma(v.y, x.x, by[k]);
        }
    }
    // C rho C^dag
    if (J.cmap) {
        const TV* cmv = (const TV*)cmvp;
        for (int c = 0; c < J.n_c; ++c) {
            const int ma = __ldg(J.cmap + (size_t)c * n + a);
            if (ma < 0) continue;
            const TV u = __ldg(cmv + (size_t)c * n + a);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int mb = __ldg(J.cmap + (size_t)c * n + b[k]);
                if (mb < 0) continue;
                const TV w = __ldg(cmv + (size_t)c * n + b[k]);
                const T gx = u.x * w.x + u.y * w.y, gy = u.y * w.x - u.x * w.y;
                const T2 x = __ldcg(Y + (size_t)ma + n * (size_t)mb);
                ax[k] = fma(gx, x.x, ax[k]);
                ay[k] = fma(gx, x.y, ay[k]);
                bx[k] = fma(-gy, x.y, bx[k]);
                by[k] = fma(gy, x.x, by[k]);
            }
        }
    } else {
        for (int c = 0; c < J.n_c; ++c) {
            const int ra = c * J.n + a;
            const int pa0 = __ldg(J.crp + ra), pa1 = __ldg(J.crp + ra + 1);
            for (int p = pa0; p < pa1; ++p) {
                const TV u = __ldg(cv + p);
                const T2* col = Y + (size_t)__ldg(J.cci + p);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int rb = c * J.n + b[k];
                    for (int q = __ldg(J.crp + rb); q < __ldg(J.crp + rb + 1); ++q) {
                        const TV w = __ldg(cv + q);
                        const T gx = u.x * w.x + u.y * w.y, gy = u.y * w.x - u.x * w.y;
                        const T2 x = __ldcg(col + n * (size_t)__ldg(J.cci + q));
                        ax[k] = fma(gx, x.x, ax[k]);
                        ay[k] = fma(gx, x.y, ay[k]);
                        bx[k] = fma(-gy, x.y, bx[k]);
                        by[k] = fma(gy, x.x, by[k]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        out[k].x = ax[k] + bx[k];
        out[k].y = ay[k] + by[k];
    }
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

// MIXED keeps two blocks (32 warps) per SM to hide the gather latency; FP64
// needs the larger register budget of one block per SM.
template <bool MIXED>
__global__ void __launch_bounds__(MG_T, MIXED ? 2 : 1) me_grid_kernel(MgJob J) {
    using T = typename GPrec<MIXED>::T;
    using T2 = typename GPrec<MIXED>::T2;
    using TV = T2;
    __shared__ MgShared sh;
    cg::grid_group grid = cg::this_grid();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = gridDim.x;
    const size_t g0 = (size_t)blockIdx.x * MG_T + tid, G = (size_t)nb * MG_T;
    const size_t L = (size_t)J.L;
    const int n = J.n, NE2 = 2 * J.n_e;
    const RkTab& tab = RK_TABS[J.method];
    const TV* av = MIXED ? (const TV*)J.av32 : (const TV*)J.av64;
    const TV* bv = MIXED ? (const TV*)J.bv32 : (const TV*)J.bv64;
    const TV* cv = MIXED ? (const TV*)J.cv32 : (const TV*)J.cv64;
    const void* cmv = MIXED ? (const void*)J.cmv32 : (const void*)J.cmv64;
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
    // candidate = current + inc (MIXED: TwoSum on hi, lo carries the error)
    auto st_add = [&](const S* cur, S* out, size_t e, T2 inc) -> T2 {
        const S v = cur[e];
        if constexpr (MIXED) {
            auto two = [](float a, float b, float lo) {
                const float s1 = a + b, bb = s1 - a;
                const float err = (a - (s1 - bb)) + (b - bb) + lo;
                const float hi = s1 + err;
                return make_float2(hi, err - (hi - s1));
            };
            const float2 rx = two(v.x, inc.x, v.z), ry = two(v.y, inc.y, v.w);
            out[e] = make_float4(rx.x, ry.x, rx.y, ry.y);
            return make_float2(rx.x, ry.x);
        } else {
            const double2 r = make_double2(v.x + inc.x, v.y + inc.y);
            out[e] = r;
            return r;
        }
    };
    int slot[7] = {0, 1, 2, 3, 4, 5, 6};
    // right-hand-side phases: thread (ra, jg) owns row ra and the columns
    // b = jg, jg + mcols, ... (n <= grid threads is required), processed four
    // at a time
    const int gtid = (int)g0;
    const int mcols = (int)(G / (size_t)n);
    const int ra = gtid % n, jg = gtid / n;
    const bool ractive = jg < mcols;
    auto K = [&](int j) -> T2* { return kbase + (size_t)slot[j] * L; };

    // ---- initial state, k1 ----
    for (size_t e = g0; e < L; e += G) {
        double2 v;
        if (J.is_ket) {
            const int i = (int)(e % n), j = (int)(e / n);
            const double2 a = J.state0[i], b = J.state0[j];
            v = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
        } else {
            v = J.state0[e];
        }
        st_set(yb, e, v);
        ysb[0][e] = g_from_d2<T2>(v);
    }
    grid.sync();
    for (int b0 = jg; ractive && b0 < n; b0 += 4 * mcols) {
        int bk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) bk[q] = b0 + q * mcols < n ? b0 + q * mcols : b0;
        T2 r[4];
        rhs_row4<T2, TV>(J, ysb[0], ra, bk, r, av, bv, cv, cmv);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (b0 + q * mcols < n) K(0)[(size_t)ra + (size_t)n * bk[q]] = r[q];
    }

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

    // thread-0 control state (identical in every block)
    double t = J.tlist[0], h = 0.0, htry = 0.0, t_target = 0.0;
    int idx = 1, status = QTL_OK;
    long long attempts = 0, steps_acc = 0, steps_rej = 0, rhs_evals = 1;
    CtlF ctl;
    ctl.init();

    // ---- starting step ----
    if (J.fixed) {
        h = J.dt_fixed;
    } else if (J.dt0 > 0.0) {
        h = J.dt0;
    } else {
        float s0 = 0.f, s1 = 0.f;
        for (size_t e = g0; e < L; e += G) {
            const double2 y = st_d2(yb, e);
            const double2 f0 = g_to_d2(K(0)[e]);
            const float a = sqrtf((float)(y.x * y.x + y.y * y.y));
            const float sc = (float)J.atol + (float)J.rtol * a;
            const float q0 = a / sc, q1 = sqrtf((float)(f0.x * f0.x + f0.y * f0.y)) / sc;
            s0 += q0 * q0;
            s1 += q1 * q1;
        }
        float b0 = block_sum_f(s0, sh), b1 = block_sum_f(s1, sh);
        if (tid == 0) {
            J.errpart[blockIdx.x] = b0;
            J.errpart[nb + blockIdx.x] = b1;
        }
        grid.sync();
        const float S0 = grid_sum_f(J.errpart, nb, sh), S1 = grid_sum_f(J.errpart + nb, nb, sh);
        const double d0 = sqrt((double)S0 / (double)L), d1 = sqrt((double)S1 / (double)L);
        const double h0 = start_h0(d0, d1);
        for (size_t e = g0; e < L; e += G) {
            const double2 y = st_d2(yb, e);
            const double2 f0 = g_to_d2(K(0)[e]);
            ysb[1][e] = g_from_d2<T2>(make_double2(y.x + h0 * f0.x, y.y + h0 * f0.y));
        }
        grid.sync();
        float s2 = 0.f;
        for (int b0 = jg; ractive && b0 < n; b0 += 4 * mcols) {
            int bk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) bk[q] = b0 + q * mcols < n ? b0 + q * mcols : b0;
            T2 r[4];
            rhs_row4<T2, TV>(J, ysb[1], ra, bk, r, av, bv, cv, cmv);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                if (b0 + q4 * mcols >= n) continue;
                const size_t e = (size_t)ra + (size_t)n * bk[q4];
                const double2 f1 = g_to_d2(r[q4]);
                const double2 f0 = g_to_d2(K(0)[e]);
                const double2 y = st_d2(yb, e);
                const float sc = (float)J.atol + (float)J.rtol * sqrtf((float)(y.x * y.x + y.y * y.y));
                const float dx = (float)(f1.x - f0.x), dy = (float)(f1.y - f0.y);
                const float q = sqrtf(dx * dx + dy * dy) / sc;
                s2 += q * q;
            }
        }
        float b2 = block_sum_f(s2, sh);
        __syncthreads();
        if (tid == 0) J.errpart[2 * nb + blockIdx.x] = b2;
        grid.sync();
        const float S2 = grid_sum_f(J.errpart + 2 * nb, nb, sh);
        rhs_evals += 1;
        h = start_h(h0, d1, sqrt((double)S2 / (double)L) / h0);
    }
    grid.sync();

    auto next_action = [&]() {
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
            const bool land = lands(h, t, t_target);
            htry = land ? (t_target - t) : h;
            sh.land = land;
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
            }
            if (lane < 28) {
                sh.coef[lane] = c;
                sh.coeff[lane] = (float)c;
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
        // stage-2 input y + h a_21 k_1
        {
            const T c = coefT(0);
            for (size_t e = g0; e < L; e += G) {
                const T2 y = st_t2(yb, e), k0 = K(0)[e];
                T2 o;
                o.x = fma(c, k0.x, y.x);
                o.y = fma(c, k0.y, y.y);
                ysb[1][e] = o;
            }
        }
        grid.sync();
        float se = 0.f;
#pragma unroll
        for (int s = 1; s < 7; ++s) {
            const T2* in = ysb[s & 1];
            T ha[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) ha[j] = (s < 6 && j <= s) ? coefT((s + 1) * s / 2 + j) : (T)0;
            T he[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) he[j] = s == 6 ? coefT(21 + j) : (T)0;
            for (int b0 = jg; ractive && b0 < n; b0 += 4 * mcols) {
              int bk[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) bk[q] = b0 + q * mcols < n ? b0 + q * mcols : b0;
              T2 r[4];
              rhs_row4<T2, TV>(J, in, ra, bk, r, av, bv, cv, cmv);
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                if (b0 + q4 * mcols >= n) continue;
                const size_t e = (size_t)ra + (size_t)n * bk[q4];
                const T2 ks = r[q4];
                K(s)[e] = ks;
                if (s < 6) {
                    // input of stage s+1: y + h sum_{j<=s} a_{s+1,j} k_j
                    T ax = ha[s] * ks.x, ay = ha[s] * ks.y;
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        if (j < s) {
                            const T2 kj = K(j)[e];
                            ax = fma(ha[j], kj.x, ax);
                            ay = fma(ha[j], kj.y, ay);
                        }
                    }
                    T2 inc;
                    inc.x = ax;
                    inc.y = ay;
                    if (s + 1 < 6) {
                        const T2 y = st_t2(yb, e);
                        T2 o;
                        o.x = y.x + ax;
                        o.y = y.y + ay;
                        ysb[(s + 1) & 1][e] = o;
                    } else {
                        // the last stage is evaluated at the candidate y_new
                        ysb[0][e] = st_add(yb, yn, e, inc);
                    }
                } else {
                    // error estimate e = h sum_j e_j k_j against sc = atol + rtol max(|y|, |y_new|)
                    T ex = he[6] * ks.x, ey = he[6] * ks.y;
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        const T2 kj = K(j)[e];
                        ex = fma(he[j], kj.x, ex);
                        ey = fma(he[j], kj.y, ey);
                    }
                    const T2 y = st_t2(yb, e), yv = st_t2(yn, e);
                    const float a2 = fmaxf((float)(y.x * y.x + y.y * y.y), (float)(yv.x * yv.x + yv.y * yv.y));
                    const float sc = (float)J.atol + (float)J.rtol * sqrtf(a2);
                    const float fx = (float)ex, fy = (float)ey;
                    se += (fx * fx + fy * fy) / (sc * sc);
                }
              }
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
            const int s0 = slot[0];
            slot[0] = slot[6];
            slot[6] = s0;
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
