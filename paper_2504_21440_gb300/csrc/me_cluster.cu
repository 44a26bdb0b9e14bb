// mesolve on a thread-block cluster: one solve of the Lindblad master
// equation (paper Sec. 3.2) integrated entirely on the device by one cluster
// of up to 16 CTAs: adaptive RK 5(4) steps, error norm, PI controller, exact
// landing on tlist and Tr(O_k rho) inside one launch.
//
// Layout.  vec(rho) (column stacking, L = n^2 complex entries) is split over
// the cluster: CTA c owns rows r = c + C*q, and its thread t holds the rows
// q = t + 256*m (m < RPT).  The owned rows of y, y_new and k_1..k_7 live in
// registers.  The stage input y_s = y + h sum_j a_sj k_j of a CTA's rows is
// written to that CTA's shared memory (two alternating buffers), and the
// Liouvillian SpMV gathers it from the owning CTAs over distributed shared
// memory.  Each CTA keeps its rows of the (constant) Liouvillian in shared
// memory too, every column stored as its DSMEM address.  One cluster barrier
// per stage and one per step for the error norm.
//
// Control.  GB300 runs FP64 at 1/64 of the FP32 rate and a warp-wide FP64
// instruction holds a sub-partition's FP64 pipe for ~64 cycles, so the scalar
// control (controller, tlist landing, step bookkeeping) runs in thread 0 of
// each CTA only, from bitwise identical inputs in every CTA, and is broadcast
// through shared memory.  The controller's factor is evaluated in FP32 and
// the error norm's per-entry ratios and their reduction are FP32 (the norm
// only steers the step size).  y, its update and the expectation values are
// FP64.
//
// Expectation values.  At a landing step every CTA sums w_e(r) * rho_r over
// its own rows in FP64 and stores the CTA partial; the partials are added in
// rank order at the end of the solve, so they cost no cluster barrier.
//
// Precision.  FP64: Liouvillian, stage sums and SpMV in FP64.  MIXED uses the
// increment form k_s = L y + L delta_s: the base L y is one FP64 product per
// step (the last stage, reused as the next step's first), the O(h) stage
// increments delta_s and their products L delta_s are FP32 (complex64
// operator), and y_new = y + h L y + sum_j h b_j L delta_j is formed in FP64.
// FP32 rounding then scales with |delta| ~ h|L y| instead of |L| |y|.
#include <cooperative_groups.h>

#include "internal.h"
#include "rk.cuh"
#include "td.cuh"

namespace cg = cooperative_groups;

namespace qtl {

constexpr int ME_T = 256;
constexpr int ME_NW = ME_T / 32;
constexpr int ME_CMAX = 16;
constexpr int ME_EMAX = 64;

enum { ACT_STEP = 0, ACT_REPEAT = 1, ACT_DONE = 2 };

template <bool MIXED>
struct Prec;
template <>
struct Prec<false> {
    using T = double;
    using T2 = double2;
};
template <>
struct Prec<true> {
    using T = float;
    using T2 = float2;
};

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
template <class T2>
__device__ __forceinline__ T2 from_d2(double2 v);
template <>
__device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 from_d2<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t dsmem_map(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ double2 ld_dsmem(uint32_t a, double2*) {
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 ld_dsmem(uint32_t a, float2*) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float ld_dsmem_f(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct MeShared {
    float wf[ME_NW];               // warp partials of the error / start-step sums
    float wf2[ME_NW];
    float pf[2][2];                // CTA partials, double-buffered across reductions
    double we[ME_NW][2 * ME_EMAX]; // warp partials of the expectation values
    double coef[34];               // htry * a_sj (21, by stage), htry * e_j (7), htry * c_s (6)
    float coeff[34];               // the same rounded to FP32 (mixed precision)
    double hcur;                   // htry of the current attempt
    double h0, d1;
    int action, land, accept, save_idx, repeat_idx;
    int scan[ME_NW];
    double tnow;                   // the step's start (time-dependent terms)
    double2 tdf[7][QTL_MAX_TD];    // f_k at t + c_s h (slots 1..6) and at one other time (slot 0)
    // mixed precision with time-dependent terms: f_k at the step's start, and
    // phi[s][k] = h sum_{j<s} a_sj f_k(t_j) (s = 1..6; the stage inputs and
    // y_new), phi[0][k] = h sum_j e_j f_k(t_j) (the error estimate)
    double2 tdfs[QTL_MAX_TD];
    double2 tdphi[7][QTL_MAX_TD];
    float2 tdphif[7][QTL_MAX_TD];
};

// Row q of this CTA's cached Liouvillian times the stage input held in the
// cluster's shared memory (buffer offset bufoff): real-only entries,
// imaginary-only entries, then complex entries.
template <class T2, class TV>
__device__ __forceinline__ T2 spmv_dsm(int q, const int4* __restrict__ s_seg,
                                       const uint32_t* __restrict__ s_addr,
                                       const TV* __restrict__ s_v, uint32_t bufoff) {
    // two accumulators (real and imaginary part): no final additions, which
    // on the 1/64-rate FP64 pipe cost as much as a short row's entries
    const int4 sg = s_seg[q];
    decltype(T2::x) ar = 0, ai = 0;
    int p = sg.x;
#pragma unroll 4
    for (; p < sg.y; ++p) {
        const decltype(T2::x) v = s_v[p].x;
        const T2 xv = ld_dsmem(s_addr[p] + bufoff, (T2*)nullptr);
        ar = fma(v, xv.x, ar);
        ai = fma(v, xv.y, ai);
    }
#pragma unroll 4
    for (; p < sg.z; ++p) {
        const decltype(T2::x) v = s_v[p].y;
        const T2 xv = ld_dsmem(s_addr[p] + bufoff, (T2*)nullptr);
        ar = fma(-v, xv.y, ar);
        ai = fma(v, xv.x, ai);
    }
#pragma unroll 2
    for (; p < sg.w; ++p) {
        const TV v = s_v[p];
        const T2 xv = ld_dsmem(s_addr[p] + bufoff, (T2*)nullptr);
        ar = fma(v.x, xv.x, ar);
        ai = fma(v.x, xv.y, ai);
        ar = fma(-v.y, xv.y, ar);
        ai = fma(v.y, xv.x, ai);
    }
    T2 acc;
    acc.x = ar;
    acc.y = ai;
    return acc;
}

// FP64 product of row q with FP64 stage inputs (the base derivative of the
// mixed-precision increment form): structure and DSMEM addresses from the
// shared-memory copy, FP64 values from global memory (gstart: the row's
// first entry in the global arrays).
__device__ __forceinline__ double2 spmv_dsm64(int q, const int4* __restrict__ s_seg,
                                              const uint32_t* __restrict__ s_addr,
                                              const double2* __restrict__ lv64, int gstart,
                                              uint32_t bufoff) {
    const int4 sg = s_seg[q];
    const double2* v = lv64 + (gstart - sg.x);
    double ax = 0, ay = 0, bx = 0, by = 0;
    int p = sg.x;
#pragma unroll 4
    for (; p < sg.y; ++p) {
        const double a = __ldg(&v[p].x);
        const double2 xv = ld_dsmem(s_addr[p] + bufoff, (double2*)nullptr);
        ax = fma(a, xv.x, ax);
        ay = fma(a, xv.y, ay);
    }
#pragma unroll 4
    for (; p < sg.z; ++p) {
        const double b = __ldg(&v[p].y);
        const double2 xv = ld_dsmem(s_addr[p] + bufoff, (double2*)nullptr);
        bx = fma(-b, xv.y, bx);
        by = fma(b, xv.x, by);
    }
#pragma unroll 2
    for (; p < sg.w; ++p) {
        const double2 a = __ldg(v + p);
        const double2 xv = ld_dsmem(s_addr[p] + bufoff, (double2*)nullptr);
        ax = fma(a.x, xv.x, ax);
        ay = fma(a.x, xv.y, ay);
        bx = fma(-a.y, xv.y, bx);
        by = fma(a.y, xv.x, by);
    }
    return make_double2(ax + bx, ay + by);
}

// Exclusive prefix sum of v over the CTA; *total gets the sum.
__device__ __forceinline__ int cta_exclusive_scan(int v, int* scratch, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    int base = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < ME_NW; ++w) {
        if (w < warp) base += scratch[w];
        tot += scratch[w];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// Index of h*a_sj in MeShared::coef (stages s = 1..6, j < s).
__host__ __device__ constexpr int coef_a(int s, int j) { return s * (s - 1) / 2 + j; }

template <bool MIXED, int RPT>
__device__ void me_solve(const MeJob& J, MeShared& sh, cg::cluster_group& cl, unsigned char* dsm) {
    using T = typename Prec<MIXED>::T;
    using T2 = typename Prec<MIXED>::T2;
    using TV = T2;
    const int C = (int)cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cl.block_rank();
    const int L = J.L, n = J.n, NE2 = 2 * J.n_e;
    const RkTab& tab = RK_TABS[J.method];
    const TV* lv = MIXED ? (const TV*)J.lv32 : (const TV*)J.lv64;

    // dynamic shared memory: ys[2][RPT*256] (16-byte slots: an FP64 value, or
    // an FP32 value in the slot's first half), seg[RPT*256], addr[cap], v[cap]
    double2* s_ys = (double2*)dsm;
    const uint32_t bufoff = (uint32_t)(RPT * ME_T * sizeof(double2));
    int4* s_seg = (int4*)(s_ys + 2 * RPT * ME_T);
    uint32_t* s_addr = (uint32_t*)(s_seg + RPT * ME_T);
    TV* s_v = (TV*)(((uintptr_t)(s_addr + J.smem_nnz) + 15) & ~(uintptr_t)15);
    const uint32_t ys_base = smem_addr(s_ys);
    // sum_k f_k (L_k y)_r for the stage input in buffer offset boff (FP64),
    // coefficients from slot `slot`; L_k from global memory, its columns
    // mapped to the owning CTA's stage-input slot on the fly
    // (a power-of-two cluster, the usual case, maps a column with shifts)
    const bool c_pow2 = (C & (C - 1)) == 0;
    const int c_lg = __ffs(C) - 1;
    auto td_row = [&](int r, uint32_t boff, int slot) -> double2 {
        double rx = 0.0, ry = 0.0;
        for (int q = 0; q < J.n_td; ++q) {
            double ax = 0.0, ay = 0.0;
            const int rr = q * L + r;
            for (int p = __ldg(J.trp + rr); p < __ldg(J.trp + rr + 1); ++p) {
                const int c = __ldg(J.tci + p);
                const double2 v = __ldg(J.tv + p);
                const uint32_t slot_c = c_pow2 ? (uint32_t)(c >> c_lg) : (uint32_t)(c / C);
                const uint32_t rank_c = c_pow2 ? (uint32_t)(c & (C - 1)) : (uint32_t)(c % C);
                const double2 x = ld_dsmem(
                    dsmem_map(ys_base + slot_c * (uint32_t)sizeof(double2), rank_c) + boff, (double2*)nullptr);
                ax += v.x * x.x - v.y * x.y;
                ay += v.x * x.y + v.y * x.x;
            }
            const double2 f = sh.tdf[slot][q];
            rx += f.x * ax - f.y * ay;
            ry += f.x * ay + f.y * ax;
        }
        return make_double2(rx, ry);
    };
    // mixed precision: (L_k x)_r of one term k, x in the stage-input slots at
    // boff as FP64 values or (f32) as FP32 values in the slots' first
    // halves; FP64 sums
    auto td_one = [&](int r, uint32_t boff, int q, bool f32) -> double2 {
        double ax = 0.0, ay = 0.0;
        const int rr = q * L + r;
        for (int p = __ldg(J.trp + rr); p < __ldg(J.trp + rr + 1); ++p) {
            const int c = __ldg(J.tci + p);
            const double2 v = __ldg(J.tv + p);
            const uint32_t slot_c = c_pow2 ? (uint32_t)(c >> c_lg) : (uint32_t)(c / C);
            const uint32_t rank_c = c_pow2 ? (uint32_t)(c & (C - 1)) : (uint32_t)(c % C);
            const uint32_t a = dsmem_map(ys_base + slot_c * (uint32_t)sizeof(double2), rank_c) + boff;
            double2 x;
            if (f32) {
                const float2 xf = ld_dsmem(a, (float2*)nullptr);
                x = make_double2((double)xf.x, (double)xf.y);
            } else {
                x = ld_dsmem(a, (double2*)nullptr);
            }
            ax += v.x * x.x - v.y * x.y;
            ay += v.x * x.y + v.y * x.x;
        }
        return make_double2(ax, ay);
    };
    // mixed precision: g_k = L_k y of the current state y (FP64, buffer gb
    // of J.tdg), row r
    int gb = 0;
    auto tdg_at = [&](int buf, int q, int r) -> double2* { return J.tdg + ((size_t)buf * J.n_td + q) * L + r; };

    double2 y[RPT], ynew[RPT];
    float2 yf[RPT], yfn[RPT];  // MIXED: FP32 copies, so the stage loop converts nothing
    // MIXED increment form: k1d = L y in FP64 (base), k[j] (j >= 1) hold the
    // FP32 corrections c_j = L delta_j with k_j = k1d + c_j.
    double2 k1d[RPT], k7d[RPT];
    float2 k1f[RPT];
    int gstart[RPT];
    T2 k[7][RPT];
    bool own[RPT];
    int row[RPT];
    auto slot_f = [&](double2* buf, int q) -> float2* { return (float2*)(buf + q); };
    auto coefT = [&](int i) -> T {
        if constexpr (MIXED)
            return sh.coeff[i];
        else
            return sh.coef[i];
    };
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        row[m] = rank + C * (tid + ME_T * m);
        own[m] = row[m] < L;
        y[m] = make_double2(0.0, 0.0);
        if (own[m]) {
            if (J.is_ket) {  // rho0 = |psi0><psi0| (ket2dm)
                const int i = row[m] % n, j = row[m] / n;
                const double2 a = J.state0[i], b = J.state0[j];
                y[m] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
            } else {
                y[m] = J.state0[row[m]];
            }
        }
        ynew[m] = y[m];
        yf[m] = make_float2((float)y[m].x, (float)y[m].y);
        yfn[m] = yf[m];
        s_ys[tid + ME_T * m] = y[m];
        gstart[m] = own[m] ? __ldg(J.seg + row[m]).x : 0;
    }

    // ---- this CTA's rows of the Liouvillian into shared memory ----
    {
        int cnt = 0;
#pragma unroll
        for (int m = 0; m < RPT; ++m)
            if (own[m]) {
                const int4 sg = __ldg(J.seg + row[m]);
                cnt += sg.w - sg.x;
            }
        int total = 0;
        int off = cta_exclusive_scan(cnt, sh.scan, &total);
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int q = tid + ME_T * m;
            if (!own[m]) {
                s_seg[q] = make_int4(0, 0, 0, 0);
                continue;
            }
            const int4 sg = __ldg(J.seg + row[m]);
            for (int p = sg.x; p < sg.w; ++p) {
                const int c = __ldg(J.ci + p);
                s_addr[off + p - sg.x] =
                    dsmem_map(ys_base + (uint32_t)((c / C) * sizeof(double2)), (uint32_t)(c % C));
                s_v[off + p - sg.x] = __ldg(lv + p);
            }
            s_seg[q] = make_int4(off, off + sg.y - sg.x, off + sg.z - sg.x, off + sg.w - sg.x);
            off += sg.w - sg.x;
        }
    }
    // time-dependent terms: f_k(tlist[0]) for k1 (slot 0)
    if (warp == 0 && lane < J.n_td) {
        sh.tdf[0][lane] = td_coef(J.tf[lane], J.tlist[0]);
        sh.tdfs[lane] = sh.tdf[0][lane];
    }
    cl.sync();

    // Per-CTA FP64 partials of Tr(O_e rho) over own rows -> J.epart[idx][rank][*].
    auto expect_partials = [&](const double2* v, int idx) {
        for (int e = 0; e < J.n_e; ++e) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!own[m]) continue;
                const double2 w = __ldg(J.ew + (size_t)row[m] * J.n_e + e);
                sr += w.x * v[m].x - w.y * v[m].y;
                si += w.x * v[m].y + w.y * v[m].x;
            }
            sr = warp_sum(sr);
            si = warp_sum(si);
            if (lane == 0) {
                sh.we[warp][2 * e] = sr;
                sh.we[warp][2 * e + 1] = si;
            }
        }
        __syncthreads();
        if (tid < NE2) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < ME_NW; ++w) s += sh.we[w][tid];
            J.epart[((size_t)idx * C + rank) * NE2 + tid] = s;
        }
    };
    auto states_write = [&](int idx) {
        if (J.states) {
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) J.states[(size_t)idx * L + row[m]] = y[m];
        }
    };
    // Cluster-wide FP32 sums of (a, b): warp -> CTA (thread 0) -> cluster
    // (thread 0 of every CTA reads all CTAs' partials in rank order).
    int par = 0;
    auto reduce2 = [&](float a, float b, float* out_a, float* out_b) {
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            sh.wf[warp] = a;
            sh.wf2[warp] = b;
        }
        __syncthreads();
        if (tid == 0) {
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int w = 0; w < ME_NW; ++w) {
                sa += sh.wf[w];
                sb += sh.wf2[w];
            }
            sh.pf[par][0] = sa;
            sh.pf[par][1] = sb;
        }
        cl.sync();
        if (tid == 0) {
            const uint32_t base = smem_addr(&sh.pf[par][0]);
            float va[ME_CMAX], vb[ME_CMAX];
#pragma unroll
            for (int r = 0; r < ME_CMAX; ++r) {
                if (r < C) {
                    const uint32_t a_r = dsmem_map(base, (uint32_t)r);
                    va[r] = ld_dsmem_f(a_r);
                    vb[r] = ld_dsmem_f(a_r + 4);
                } else {
                    va[r] = 0.f;
                    vb[r] = 0.f;
                }
            }
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int r = 0; r < ME_CMAX; ++r) {
                sa += va[r];
                sb += vb[r];
            }
            *out_a = sa;
            *out_b = sb;
        }
        par ^= 1;
    };

    // k1 = L y0 (FP64 in both precisions), expectation values at tlist[0]
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        if (!own[m]) continue;
        if constexpr (MIXED) {
            k1d[m] = spmv_dsm64(tid + ME_T * m, s_seg, s_addr, J.lv64, gstart[m], 0u);
            k1f[m] = make_float2((float)k1d[m].x, (float)k1d[m].y);
            k[0][m] = k1f[m];
            if (J.n_td > 0) {
                // g_k = L_k y0 (FP64), and k[0] = L(t0) y0 for the starting step
                double fx = k1d[m].x, fy = k1d[m].y;
                for (int q = 0; q < J.n_td; ++q) {
                    const double2 g = td_one(row[m], 0u, q, false);
                    *tdg_at(0, q, row[m]) = g;
                    const double2 f = sh.tdf[0][q];
                    fx += f.x * g.x - f.y * g.y;
                    fy += f.x * g.y + f.y * g.x;
                }
                k[0][m] = make_float2((float)fx, (float)fy);
            }
        } else {
            k[0][m] = spmv_dsm<T2, TV>(tid + ME_T * m, s_seg, s_addr, s_v, 0u);
            if (J.n_td > 0) {
                const double2 d = td_row(row[m], 0u, 0);
                k[0][m].x += d.x;
                k[0][m].y += d.y;
            }
        }
    }
    expect_partials(y, 0);
    states_write(0);

    // thread-0 control state (identical in every CTA)
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
        // Hairer-Norsett-Wanner: d0 = |y0|, d1 = |f0| (RMS, scaled by
        // atol + rtol |y0|), h0 = 0.01 d0/d1, d2 = |f(y0 + h0 f0) - f0| / h0.
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            if (!own[m]) continue;
            const double2 f0 = to_d2(k[0][m]);
            const float a = sqrtf((float)(y[m].x * y[m].x + y[m].y * y[m].y));
            const float sc = (float)J.atol + (float)J.rtol * a;
            const float q0 = a / sc;
            const float q1 = sqrtf((float)(f0.x * f0.x + f0.y * f0.y)) / sc;
            s0 += q0 * q0;
            s1 += q1 * q1;
        }
        float S0 = 0.f, S1 = 0.f;
        reduce2(s0, s1, &S0, &S1);
        if (tid == 0) {
            const double d0 = sqrt((double)S0 / L), d1 = sqrt((double)S1 / L);
            sh.h0 = start_h0(d0, d1);
            sh.d1 = d1;
        }
        __syncthreads();
        const double h0 = sh.h0;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            if constexpr (MIXED) {
                // increment form: f(y0 + h0 f0) - f0 = L (h0 f0) (plus, with
                // time-dependent terms, (f_k(t0 + h0) - f_k(t0)) L_k y0)
                *slot_f(s_ys + RPT * ME_T, tid + ME_T * m) =
                    make_float2((float)h0 * k[0][m].x, (float)h0 * k[0][m].y);
            } else {
                const double2 f0 = to_d2(k[0][m]);
                s_ys[RPT * ME_T + tid + ME_T * m] =
                    make_double2(y[m].x + h0 * f0.x, y[m].y + h0 * f0.y);
            }
        }
        if (warp == 0 && lane < J.n_td) sh.tdf[0][lane] = td_coef(J.tf[lane], J.tlist[0] + h0);
        cl.sync();
        float s2 = 0.f;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            if (!own[m]) continue;
            float dx, dy;
            if constexpr (MIXED) {
                const T2 c = spmv_dsm<T2, TV>(tid + ME_T * m, s_seg, s_addr, s_v, bufoff);
                dx = (float)c.x;
                dy = (float)c.y;
                if (J.n_td > 0) {
                    double ex = 0.0, ey = 0.0;
                    for (int q = 0; q < J.n_td; ++q) {
                        const double2 f1 = sh.tdf[0][q], f0 = sh.tdfs[q];
                        const double2 u = td_one(row[m], bufoff, q, true);
                        const double2 g = *tdg_at(0, q, row[m]);
                        const double dfx = f1.x - f0.x, dfy = f1.y - f0.y;
                        ex += f1.x * u.x - f1.y * u.y + dfx * g.x - dfy * g.y;
                        ey += f1.x * u.y + f1.y * u.x + dfx * g.y + dfy * g.x;
                    }
                    dx += (float)ex;
                    dy += (float)ey;
                }
            } else {
                double2 f1 = to_d2(spmv_dsm<T2, TV>(tid + ME_T * m, s_seg, s_addr, s_v, bufoff));
                if (J.n_td > 0) {
                    const double2 d = td_row(row[m], bufoff, 0);
                    f1.x += d.x;
                    f1.y += d.y;
                }
                const double2 f0 = to_d2(k[0][m]);
                dx = (float)(f1.x - f0.x);
                dy = (float)(f1.y - f0.y);
            }
            const float a = sqrtf((float)(y[m].x * y[m].x + y[m].y * y[m].y));
            const float sc = (float)J.atol + (float)J.rtol * a;
            const float q = sqrtf(dx * dx + dy * dy) / sc;
            s2 += q * q;
        }
        float S2 = 0.f, dummy = 0.f;
        reduce2(s2, 0.f, &S2, &dummy);
        if (tid == 0) {
            rhs_evals += 1;
            h = start_h(h0, sh.d1, sqrt((double)S2 / L) / h0);
        }
    }
    // every CTA has finished gathering from buffers 0/1 before they are rewritten
    cl.sync();

    // thread 0: choose the next action (step / repeated output time / done)
    auto next_action = [&]() {
        sh.tnow = t;
        for (;;) {
            if (status != QTL_OK || idx >= J.nt) {
                sh.action = ACT_DONE;
                return;
            }
            t_target = J.tlist[idx];
            if (!(t_target >= J.tlist[idx - 1]) || !isfinite(t_target)) {
                status = QTL_EINVAL;
                continue;
            }
            if (!(t < t_target)) {
                sh.action = ACT_REPEAT;
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
            sh.action = ACT_STEP;
            sh.coef[27] = htry;  // handed to warp 0 for the coefficient products
            sh.hcur = htry;
            return;
        }
    };
    // warp 0: the 28 products htry * (a_sj, e_j) in FP64, one per lane
    auto publish_coefs = [&]() {
        __syncwarp();
        if (sh.action == ACT_STEP) {
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
            } else {
                // htry * c_s for stages s = 1..6 (lanes 28..31 and 0..1 again)
                const double cs = hh * tab.c[lane - 27];
                sh.coef[lane] = cs;
                sh.coeff[lane] = (float)cs;
            }
            if (lane < 2) {
                const double cs = hh * tab.c[lane + 5];
                sh.coef[32 + lane] = cs;
                sh.coeff[32 + lane] = (float)cs;
            }
            // f_k at the stage times t + c_s htry (slots 1..6)
            for (int i = lane; i < 6 * J.n_td; i += 32) {
                const int st = 1 + i / J.n_td, q = i % J.n_td;
                sh.tdf[st][q] = td_coef(J.tf[q], sh.tnow + tab.c[st] * hh);
            }
            if constexpr (MIXED) {
                if (J.n_td > 0) {
                    // f_k at the step's start, then the sums over the stages
                    if (lane < J.n_td) sh.tdfs[lane] = td_coef(J.tf[lane], sh.tnow);
                    __syncwarp();
                    for (int i = lane; i < 7 * J.n_td; i += 32) {
                        const int st = i / J.n_td, q = i % J.n_td;
                        double px = 0.0, py = 0.0;
                        const int jn = st == 0 ? 7 : st;
                        for (int j = 0; j < jn; ++j) {
                            const double2 f = j == 0 ? sh.tdfs[q] : sh.tdf[j][q];
                            const double w = st == 0 ? tab.e[j] : tab.a[st][j];
                            px += w * f.x;
                            py += w * f.y;
                        }
                        sh.tdphi[st][q] = make_double2(hh * px, hh * py);
                        sh.tdphif[st][q] = make_float2((float)(hh * px), (float)(hh * py));
                    }
                }
            }
        }
    };
    if (tid == 0) next_action();
    if (warp == 0) publish_coefs();
    __syncthreads();

    // ---- main loop: one iteration per step attempt ----
    for (;;) {
        const int action = sh.action;
        if (action == ACT_DONE) break;
        if (action == ACT_REPEAT) {
            const int ri = sh.repeat_idx;
            if (tid < NE2)
                J.epart[((size_t)ri * C + rank) * NE2 + tid] =
                    __ldcg(J.epart + ((size_t)(ri - 1) * C + rank) * NE2 + tid);
            states_write(ri);
            __syncthreads();
            if (tid == 0) next_action();
            if (warp == 0) publish_coefs();
            __syncthreads();
            continue;
        }
        const bool land = sh.land;
        // stages 2..7: combine own rows -> own shared memory -> barrier -> SpMV
#pragma unroll
        for (int s = 1; s < 7; ++s) {
            const uint32_t off = (s & 1) ? 0u : bufoff;
            double2* ysb = s_ys + ((s & 1) ? 0 : RPT * ME_T);
            T ha[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) ha[j] = j < s ? coefT(coef_a(s, j)) : (T)0;
            if constexpr (MIXED) {
                // increment form: stage input delta_s = h c_s k1 + sum_{j>=1} h a_sj c_j
                // (FP32, O(h) small); its product c_s = L delta_s in FP32; the
                // last stage forms y_new = y + h k1 + sum_j h b_j c_j in FP64 and
                // evaluates k7 = L y_new in FP64 (the next step's base).
                const float hc = sh.coeff[27 + s];
                const double hcur = sh.hcur;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    float ax = 0.f, ay = 0.f;
#pragma unroll
                    for (int j = 1; j < 6; ++j) {
                        if (j < s) {
                            ax = fmaf(ha[j], k[j][m].x, ax);
                            ay = fmaf(ha[j], k[j][m].y, ay);
                        }
                    }
                    if (s < 6) {
                        ax = fmaf(hc, k1f[m].x, ax);
                        ay = fmaf(hc, k1f[m].y, ay);
                        if (J.n_td > 0 && own[m]) {
                            // + sum_k phi[s][k] g_k (the stage times' f_k on L_k y)
                            for (int q = 0; q < J.n_td; ++q) {
                                const double2 gd = *tdg_at(gb, q, row[m]);
                                const float2 g = make_float2((float)gd.x, (float)gd.y), ph = sh.tdphif[s][q];
                                ax = fmaf(ph.x, g.x, fmaf(-ph.y, g.y, ax));
                                ay = fmaf(ph.x, g.y, fmaf(ph.y, g.x, ay));
                            }
                        }
                        *slot_f(ysb, tid + ME_T * m) = make_float2(ax, ay);
                    } else {
                        ynew[m] = make_double2(fma(hcur, k1d[m].x, y[m].x) + (double)ax,
                                               fma(hcur, k1d[m].y, y[m].y) + (double)ay);
                        if (J.n_td > 0 && own[m]) {
                            double tx = 0.0, ty = 0.0;
                            for (int q = 0; q < J.n_td; ++q) {
                                const double2 g = *tdg_at(gb, q, row[m]), ph = sh.tdphi[6][q];
                                tx += ph.x * g.x - ph.y * g.y;
                                ty += ph.x * g.y + ph.y * g.x;
                            }
                            ynew[m].x += tx;
                            ynew[m].y += ty;
                        }
                        yfn[m] = make_float2((float)ynew[m].x, (float)ynew[m].y);
                        ysb[tid + ME_T * m] = ynew[m];
                    }
                }
                cl.sync();
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    if (s < 6) {
                        k[s][m] = spmv_dsm<T2, TV>(tid + ME_T * m, s_seg, s_addr, s_v, off);
                        if (J.n_td > 0) {
                            // + sum_k f_k(t_s) L_k delta_s
                            double ex = 0.0, ey = 0.0;
                            for (int q = 0; q < J.n_td; ++q) {
                                const double2 u = td_one(row[m], off, q, true), f = sh.tdf[s][q];
                                ex += f.x * u.x - f.y * u.y;
                                ey += f.x * u.y + f.y * u.x;
                            }
                            k[s][m].x += (float)ex;
                            k[s][m].y += (float)ey;
                        }
                    } else {
                        k7d[m] = spmv_dsm64(tid + ME_T * m, s_seg, s_addr, J.lv64, gstart[m], off);
                        double cx = k7d[m].x - k1d[m].x, cy = k7d[m].y - k1d[m].y;
                        if (J.n_td > 0) {
                            // g_k of y_new into the other buffer; the correction
                            // k_7 - L(t + h) y = (L0 y_new - L0 y) + sum_k f_k(t + h) (g_k' - g_k)
                            for (int q = 0; q < J.n_td; ++q) {
                                const double2 g1 = td_one(row[m], off, q, false), g0 = *tdg_at(gb, q, row[m]);
                                *tdg_at(gb ^ 1, q, row[m]) = g1;
                                const double2 f = sh.tdf[6][q];
                                const double dx = g1.x - g0.x, dy = g1.y - g0.y;
                                cx += f.x * dx - f.y * dy;
                                cy += f.x * dy + f.y * dx;
                            }
                        }
                        k[6][m] = make_float2((float)cx, (float)cy);
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    // the sum starts from y: no separate FP64 addition
                    double ax = y[m].x, ay = y[m].y;
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        if (j < s) {
                            ax = fma((double)ha[j], (double)k[j][m].x, ax);
                            ay = fma((double)ha[j], (double)k[j][m].y, ay);
                        }
                    }
                    const double2 o = make_double2(ax, ay);
                    if (s == 6) ynew[m] = o;
                    ysb[tid + ME_T * m] = o;
                }
                cl.sync();
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    k[s][m] = spmv_dsm<T2, TV>(tid + ME_T * m, s_seg, s_addr, s_v, off);
                    if (J.n_td > 0) {
                        const double2 d = td_row(row[m], off, s);
                        k[s][m].x += d.x;
                        k[s][m].y += d.y;
                    }
                }
            }
        }
        // error norm: sum over own rows of (|e| / sc)^2, e = h sum_j e_j k_j
        float se = 0.f;
        {
            T he[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) he[j] = coefT(21 + j);
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!own[m]) continue;
                T ex = 0, ey = 0;
                // (MIXED: k[j] are the corrections c_j; sum_j e_j = 0, so
                // e = h sum_{j>=1} e_j c_j and the base k1 drops out)
#pragma unroll
                for (int j = MIXED ? 1 : 0; j < 7; ++j) {
                    ex = fma(he[j], k[j][m].x, ex);
                    ey = fma(he[j], k[j][m].y, ey);
                }
                if constexpr (MIXED) {
                    // the stage bases differ by sum_k f_k(t_j) g_k: + sum_k psi_k g_k
                    for (int q = 0; q < J.n_td; ++q) {
                        const double2 gd = *tdg_at(gb, q, row[m]);
                        const float2 g = make_float2((float)gd.x, (float)gd.y), ps = sh.tdphif[0][q];
                        ex = fmaf(ps.x, g.x, fmaf(-ps.y, g.y, ex));
                        ey = fmaf(ps.x, g.y, fmaf(ps.y, g.x, ey));
                    }
                }
                float yx, yy, nx, ny;
                if constexpr (MIXED) {
                    yx = yf[m].x;
                    yy = yf[m].y;
                    nx = yfn[m].x;
                    ny = yfn[m].y;
                } else {
                    yx = (float)y[m].x;
                    yy = (float)y[m].y;
                    nx = (float)ynew[m].x;
                    ny = (float)ynew[m].y;
                }
                const float a2 = fmaxf(yx * yx + yy * yy, nx * nx + ny * ny);
                const float sc = (float)J.atol + (float)J.rtol * sqrtf(a2);
                const float fx = (float)ex, fy = (float)ey;
                se += (fx * fx + fy * fy) / (sc * sc);
            }
        }
        if (land) {
            // expectation values of the candidate state (kept only if accepted)
            if (tid == 0) sh.save_idx = idx;
            __syncthreads();
            expect_partials(ynew, sh.save_idx);
        }
        float S = 0.f, dummy = 0.f;
        reduce2(se, 0.f, &S, &dummy);
        // ---- decision (thread 0), then the next action ----
        if (tid == 0) {
            rhs_evals += 6;
            const float err = sqrtf(S / (float)L);
            bool acc = true;
            float fac = 1.0f;
            if (!J.fixed) {
                if (!(S <= (float)L)) {
                    acc = false;
                    ++steps_rej;
                    h = htry * (double)ctl.on_reject(err);
                    if (h < J.dt_min || !isfinite(S)) status = QTL_ESTEP;
                } else {
                    fac = ctl.on_accept(err);
                }
            }
            sh.accept = acc;
            if (acc) {
                ++steps_acc;
                t = land ? t_target : t + htry;
                h = J.fixed ? J.dt_fixed : htry * (double)fac;
                if (land) ++idx;
            }
            next_action();
        }
        if (warp == 0) publish_coefs();
        __syncthreads();
        if (sh.accept) {
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                y[m] = ynew[m];
                yf[m] = yfn[m];
                if constexpr (MIXED) {
                    k1d[m] = k7d[m];
                    k1f[m] = make_float2((float)k7d[m].x, (float)k7d[m].y);
                    k[0][m] = k1f[m];
                } else {
                    k[0][m] = k[6][m];
                }
            }
            if constexpr (MIXED) gb ^= (J.n_td > 0);   // g_k of y_new
            if (land) states_write(sh.save_idx);
        }
    }

    // ---- expectation values: CTA partials added in rank order ----
    cl.sync();
    if (rank == 0) {
        for (int v = tid; v < J.nt * NE2; v += ME_T) {
            const int ti = v / NE2, c2 = v % NE2;
            double s = 0.0;
            for (int r = 0; r < C; ++r) s += __ldcg(J.epart + ((size_t)ti * C + r) * NE2 + c2);
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

// One cluster per solve at a time.  With `next` (a zeroed device counter) the
// clusters take jobs dynamically: rank 0 draws the next index and hands it
// to the other CTAs over DSMEM; without it, job jb goes to cluster jb mod
// (number of clusters).
template <bool MIXED, int RPT>
__global__ void __launch_bounds__(ME_T, 1) me_cluster_kernel(const MeJob* __restrict__ jobs,
                                                              int njobs, int* next) {
    __shared__ MeShared sh;
    __shared__ int job_slot;
    extern __shared__ __align__(16) unsigned char me_dsm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    int jb = cid;
    for (;;) {
        if (next) {
            if (cl.block_rank() == 0 && threadIdx.x == 0) job_slot = atomicAdd(next, 1);
            cl.sync();
            jb = *cl.map_shared_rank(&job_slot, 0);
            cl.sync();
        }
        if (jb >= njobs) break;
        const MeJob J = jobs[jb];
        me_solve<MIXED, RPT>(J, sh, cl, me_dsm);
        cl.sync();
        if (!next) jb += ncl;
    }
}

int me_cluster_capacity() { return ME_CMAX * ME_T * 4; }

bool me_plan(int L_max, int cluster_size, int* C_out, int* rpt_out) {
    // Default: 16 CTAs (one per SM), the most SMs a cluster can bring to one
    // solve; rows per thread the smallest of 1, 2, 4 that covers L.
    int C = cluster_size > 0 ? cluster_size : ME_CMAX;
    int rpt = 1;
    while (rpt < 4 && (long long)C * ME_T * rpt < L_max) rpt *= 2;
    *C_out = C;
    *rpt_out = rpt;
    return C <= ME_CMAX && (long long)C * ME_T * rpt >= L_max;
}

static size_t me_dyn_smem(int precision, int rpt, int nnz) {
    const size_t t2 = precision == QTL_MIXED ? sizeof(float2) : sizeof(double2);
    return 2 * (size_t)rpt * ME_T * sizeof(double2) + (size_t)rpt * ME_T * sizeof(int4) +
           (size_t)nnz * 4 + 16 + (size_t)nnz * t2;
}

int me_smem_nnz_budget(int precision, int rpt) {
    const size_t limit = 200 * 1024;
    const size_t t2 = precision == QTL_MIXED ? sizeof(float2) : sizeof(double2);
    const size_t fixed = me_dyn_smem(precision, rpt, 0);
    return fixed >= limit ? 0 : (int)((limit - fixed) / (4 + t2));
}

template <bool MIXED, int RPT>
static cudaError_t launch_t(const MeJob* jobs, int njobs, int C, int nclusters, int smem_nnz,
                            int* next, cudaStream_t st) {
    auto kern = me_cluster_kernel<MIXED, RPT>;
    const size_t dsm = me_dyn_smem(MIXED ? QTL_MIXED : QTL_FP64, RPT, smem_nnz);
    cudaError_t e;
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * nclusters);
    cfg.blockDim = dim3(ME_T);
    cfg.dynamicSmemBytes = dsm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, kern, jobs, njobs, next);
}

cudaError_t launch_me_cluster(const MeJob* jobs_dev, int njobs, int L_max, int smem_nnz,
                              int precision, int cluster_size, int* next, cudaStream_t st) {
    int C, rpt;
    if (!me_plan(L_max, cluster_size, &C, &rpt)) return cudaErrorInvalidValue;
    if (smem_nnz > me_smem_nnz_budget(precision, rpt)) return cudaErrorInvalidValue;
    // clusters that can be resident at once (one CTA per SM at most, as the
    // shared-memory footprint allows)
    int nclusters = njobs;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t dsm = me_dyn_smem(precision, rpt, smem_nnz) + sizeof(MeShared) + 1024;
    int per_sm = (int)((228 * 1024) / dsm);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2) per_sm = 2;
    const int cap = (nsm * per_sm) / C > 0 ? (nsm * per_sm) / C : 1;
    if (nclusters > cap) nclusters = cap;
    if (nclusters < 1) nclusters = 1;
    const bool mixed = precision == QTL_MIXED;
    if (mixed) {
        if (rpt == 1) return launch_t<true, 1>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
        if (rpt == 2) return launch_t<true, 2>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
        return launch_t<true, 4>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
    }
    if (rpt == 1) return launch_t<false, 1>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
    if (rpt == 2) return launch_t<false, 2>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
    return launch_t<false, 4>(jobs_dev, njobs, C, nclusters, smem_nnz, next, st);
}

}  // namespace qtl
