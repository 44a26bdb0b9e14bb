// mcsolve: Monte-Carlo wave-function trajectories (paper Sec. 3.3).
//
// One CTA integrates one trajectory at a time (persistent loop over
// trajectories): d psi/dt = A psi with A = -i H_eff = -i H - 1/2 sum C^dag C,
// adaptive RK 5(4) with the PI controller, exact landing on tlist, a jump
// when |psi|^2 drops below the trajectory's threshold r:
//   * the crossing time inside the accepted step is located by the Illinois
//     method on ln|psi(t+tau)|^2 - ln r, psi(t+tau) being one RK step of size
//     tau from the step's start (stop at bracket < 1e-10 max(1,|t|) or after
//     30 evaluations; the jump is taken at the last evaluated point);
//   * channel k is the smallest with sum_{j<=k} |C_j psi|^2 >= u sum_j |C_j psi|^2;
//   * psi <- C_k psi / |C_k psi| and a new threshold is drawn.
// Uniforms come from Philox4x32-10 (Salmon et al., SC'11) with counter
// (draw, trajectory, 0, 0) and key (seed lo, seed hi), converted with 52 bits.
//
// Thread t of the CTA owns rows i = t + m*T (m < RPT) of psi, y_new and
// k_1..k_7 in registers; the stage input is staged in shared memory (two
// alternating buffers) for the sparse A*psi product, and an FP64 copy of psi
// is staged there for expectation values and jumps.  Sums are fixed-order
// (warp shuffle tree, then warps in order), so a trajectory's result does not
// depend on which CTA or batch it runs in.
//
// This header holds the kernel template and its launcher.  mc_traj.cu picks
// the launch shape; mc_traj_fp64_*.cu and mc_traj_mixed_*.cu instantiate the
// eight (precision, rows per thread, launch bounds) variants in six
// translation units, so that they compile in parallel.
#pragma once
#include "internal.h"
#include "mc_common.cuh"

namespace qtl {

template <bool MIXED, int RPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) mc_traj_kernel(McJob J) {
    using T = typename MPrec<MIXED>::T;
    using T2 = typename MPrec<MIXED>::T2;
    using TV = T2;
    extern __shared__ __align__(16) unsigned char mc_smem[];
    __shared__ McCtl cb;
    const int n = J.n;
    const int tid = threadIdx.x, T_ = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (T_ + 31) >> 5;
    const int rs = mc_red_stride(J.n_e, J.n_c);
    double2* yd = (double2*)mc_smem;
    T2* ys0 = (T2*)(yd + n);
    T2* ys1 = ys0 + n;
    double* wred = (double*)(((uintptr_t)(ys1 + n) + 15) & ~(uintptr_t)15);
    double* bout = wred + nw * rs;
    BlockReducer red{wred, bout, rs, lane, warp, tid, nw};
    const RkTab& tab = RK_TABS[J.method];
    const TV* av = MIXED ? (const TV*)J.av32 : (const TV*)J.av64;
    // A (constant, shared by every trajectory of this CTA) into shared memory
    const bool cached = J.a_smem;
    int4* s_seg = (int4*)(((uintptr_t)(bout + rs + 2) + 15) & ~(uintptr_t)15);
    TV* s_v = (TV*)(s_seg + n);
    int32_t* s_ci = (int32_t*)(s_v + J.a_nnz);
    if (cached) {
        for (int r = tid; r < n; r += T_) s_seg[r] = __ldg(J.aseg + r);
        for (int p = tid; p < J.a_nnz; p += T_) {
            s_v[p] = __ldg(av + p);
            s_ci[p] = __ldg(J.aci + p);
        }
        __syncthreads();
    }
    // operators: the job's, or (J.tops) the current trajectory's own
    const int4* Aseg = J.aseg;
    const int32_t* Aci = J.aci;
    const TV* Av = av;
    const int32_t *Crp = J.crp, *Cci = J.cci, *Orp = J.orp, *Oci = J.oci;
    const double2 *Cv = J.cv, *Ov = J.ov;
    // A x, plus sum_k f_k(t) (-i H_k) x with the coefficients of slot `slot`
    // (1..6: the stages of the current step, 7: one other time)
    const TV* tv = MIXED ? (const TV*)J.tv32 : (const TV*)J.tv64;
    auto rhs_row = [&](int r, const T2* x, int slot) -> T2 {
        T2 v = cached ? mc_spmv_row_s<T2, TV>(r, s_seg, s_ci, s_v, x)
                      : mc_spmv_row<T2, TV>(r, Aseg, Aci, Av, x);
        for (int k = 0; k < J.n_td; ++k) {
            const T2 w = mc_spmv_row<T2, TV>(k * n + r, J.tseg, J.tci, tv, x);
            T2 f;
            if constexpr (MIXED)
                f = cb.tdf32[slot][k];
            else
                f = cb.tdf[slot][k];
            v.x += f.x * w.x - f.y * w.y;
            v.y += f.x * w.y + f.y * w.x;
        }
        return v;
    };
    // warp 0: f_k at time tp into slot 7
    auto publish_td_at = [&](double tp) {
        if (lane < J.n_td) {
            const double2 f = td_coef(J.tf[lane], tp);
            cb.tdf[7][lane] = f;
            cb.tdf32[7][lane] = make_float2((float)f.x, (float)f.y);
        }
    };

    long long acc_steps = 0, rej_steps = 0, rhs_evals = 0, jumps = 0;  // thread 0
    int status = QTL_OK;                                                 // thread 0

    for (int jt = blockIdx.x; jt < J.ntraj; jt += gridDim.x) {
        const unsigned long long traj = (unsigned long long)(J.traj_offset + jt);
        if (J.tops) {
            const McTrajOps o = J.tops[jt];
            Aseg = o.aseg;
            Aci = o.aci;
            Av = MIXED ? (const TV*)o.av32 : (const TV*)o.av64;
            Crp = o.crp;
            Cci = o.cci;
            Cv = o.cv;
            Orp = o.orp;
            Oci = o.oci;
            Ov = o.ov;
        }
        double2 y[RPT], ynew[RPT];
        float2 yf[RPT], yfn[RPT];
        T2 k[7][RPT];
        bool own[RPT];
        int row[RPT];
        auto coefT = [&](int i) -> T {
            if constexpr (MIXED)
                return cb.coeff[i];
            else
                return cb.coef[i];
        };
        auto sync_yf = [&]() {
            if constexpr (MIXED) {
#pragma unroll
                for (int m = 0; m < RPT; ++m) yf[m] = make_float2((float)y[m].x, (float)y[m].y);
            }
        };
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            row[m] = tid + m * T_;
            own[m] = row[m] < n;
            y[m] = own[m] ? J.psi0[(size_t)jt * J.psi0_stride + row[m]] : make_double2(0.0, 0.0);
            ynew[m] = y[m];
            yfn[m] = make_float2(0.f, 0.f);
            if (own[m]) {
                yd[row[m]] = y[m];
                ys0[row[m]] = from_d2_mc<T2>(y[m]);
            }
        }
        sync_yf();
        if (warp == 0 && J.n_td > 0) publish_td_at(J.tlist[0]);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < RPT; ++m)
            if (own[m]) k[0][m] = rhs_row(row[m], ys0, 7);

        // <psi|O_e|psi>/<psi|psi> from the FP64 copy in yd (all rows written and
        // synchronised by the caller); returns |psi|^2 in thread 0.
        auto save = [&](int idx) -> double {
            if (J.odiag) {
                // real diagonal observables: <psi|O|psi> = sum_i O_ii |psi_i|^2,
                // imaginary part exactly 0 (one FMA per observable and row)
                double p[RPT];
                double s2 = 0.0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    p[m] = own[m] ? y[m].x * y[m].x + y[m].y * y[m].y : 0.0;
                    s2 += p[m];
                }
                red.stage(0, s2);
                for (int e = 0; e < J.n_e; ++e) {
                    double sr = 0.0;
#pragma unroll
                    for (int m = 0; m < RPT; ++m)
                        if (own[m]) sr = fma(__ldg(J.odiag + (size_t)e * n + row[m]), p[m], sr);
                    red.stage(1 + e, sr);
                }
                red.finish(1 + J.n_e);
                for (int e = tid; e < J.n_e; e += blockDim.x)
                    J.traj_expect[((size_t)e * J.nt + idx) * J.ntraj + jt] = make_double2(bout[1 + e] / bout[0], 0.0);
                return bout[0];
            }
            double s2 = 0.0;
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) s2 += y[m].x * y[m].x + y[m].y * y[m].y;
            red.stage(0, s2);
            for (int e = 0; e < J.n_e; ++e) {
                double sr = 0.0, si = 0.0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    const int i = e * n + row[m];
                    double ox = 0.0, oy = 0.0;
                    for (int p = __ldg(Orp + i); p < __ldg(Orp + i + 1); ++p) {
                        const double2 o = Ov[p];
                        const double2 v = yd[__ldg(Oci + p)];
                        ox += o.x * v.x - o.y * v.y;
                        oy += o.x * v.y + o.y * v.x;
                    }
                    // conj(psi_i) * (O psi)_i
                    sr += y[m].x * ox + y[m].y * oy;
                    si += y[m].x * oy - y[m].y * ox;
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
        double norm2 = save(0);  // meaningful in thread 0

        // thread-0 control state
        double t = J.tlist[0], h = 0.0, htry = 0.0, t_target = 0.0, r = 0.0;
        unsigned draw = 0;
        int idx = 1;
        long long attempts = 0;
        CtlF ctl;
        ctl.init();
        if (tid == 0) {
            if (J.rng_draw && J.rng_draw[jt] > 0) {
                // resumed trajectory: its stream and threshold carry over
                draw = J.rng_draw[jt];
                r = J.rng_r[jt];
            } else {
                r = philox_uniform(J.seed, traj, draw++);
                if (J.n_c == 0) r = 0.0;   // no channel to jump to: never below the threshold
            }
            rhs_evals += 1;
        }
        // ---- starting step ----
        if (J.fixed) {
            h = J.dt_fixed;
        } else if (J.dt0 > 0.0) {
            h = J.dt0;
        } else {
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!own[m]) continue;
                const double2 f0 = to_d2_mc(k[0][m]);
                const float a = sqrtf((float)(y[m].x * y[m].x + y[m].y * y[m].y));
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
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!own[m]) continue;
                const double2 f0 = to_d2_mc(k[0][m]);
                ys1[row[m]] = from_d2_mc<T2>(make_double2(y[m].x + h0 * f0.x, y[m].y + h0 * f0.y));
            }
            if (warp == 0 && J.n_td > 0) publish_td_at(J.tlist[0] + h0);
            __syncthreads();
            double s2 = 0.0;
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!own[m]) continue;
                const double2 f1 = to_d2_mc(rhs_row(row[m], ys1, 7));
                const double2 f0 = to_d2_mc(k[0][m]);
                const float sc = (float)J.atol + (float)J.rtol * sqrtf((float)(y[m].x * y[m].x + y[m].y * y[m].y));
                const float dx = (float)(f1.x - f0.x), dy = (float)(f1.y - f0.y);
                const float q = sqrtf(dx * dx + dy * dy) / sc;
                s2 += (double)(q * q);
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
            cb.tnow = t;
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
                // f_k at the stage times t + c_s htry (slots 1..6)
                for (int i = lane; i < 6 * J.n_td; i += 32) {
                    const int s = 1 + i / J.n_td, kk = i % J.n_td;
                    const double2 f = td_coef(J.tf[kk], cb.tnow + tab.c[s] * hh);
                    cb.tdf[s][kk] = f;
                    cb.tdf32[s][kk] = make_float2((float)f.x, (float)f.y);
                }
            }
            __syncwarp();
        };
        // One RK step of size h (coefficients in cb.coef) from (y, k1): k[1..6], ynew.
        // MIXED keeps FP32 copies of y (yf) and y_new (yfn) so that the stage
        // loop performs no FP64<->FP32 conversions (they run on the FP64 pipe).
        auto rk_step = [&]() {
#pragma unroll
            for (int s = 1; s < 7; ++s) {
                T2* ysb = (s & 1) ? ys0 : ys1;
                T ha[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) ha[j] = j < s ? coefT(mc_coef_a(s, j)) : (T)0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    // FP64: the sum starts from y (no separate addition on the
                    // 1/64-rate FP64 pipe); MIXED: FP32 increments added to y after
                    T ax = 0, ay = 0;
                    if constexpr (!MIXED) {
                        ax = y[m].x;
                        ay = y[m].y;
                    }
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        if (j < s) {
                            ax = fma(ha[j], k[j][m].x, ax);
                            ay = fma(ha[j], k[j][m].y, ay);
                        }
                    }
                    T2 o;
                    if constexpr (MIXED) {
                        if (s == 6) {
                            ynew[m] = make_double2(y[m].x + (double)ax, y[m].y + (double)ay);
                            o = from_d2_mc<T2>(ynew[m]);
                            yfn[m] = o;
                        } else {
                            o.x = yf[m].x + ax;
                            o.y = yf[m].y + ay;
                        }
                    } else {
                        o.x = ax;
                        o.y = ay;
                        if (s == 6) ynew[m] = make_double2(ax, ay);
                    }
                    ysb[row[m]] = o;
                }
                __syncthreads();
#pragma unroll
                for (int m = 0; m < RPT; ++m)
                    if (own[m]) k[s][m] = rhs_row(row[m], ysb, s);
            }
        };
        // |ynew|^2 (FP64) and the FP32 error sum, warp -> thread 0.
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
        auto norm2_ynew = [&](double* N) {
            double sn = 0.0;
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) sn += ynew[m].x * ynew[m].x + ynew[m].y * ynew[m].y;
            float dummy;
            reduce_step(0.f, sn, &dummy, N);
        };

        if (tid == 0) next_action();
        if (warp == 0) publish_coefs();
        __syncthreads();

        // root-find state (thread 0)
        double lo = 0.0, glo = 0.0, hi = 0.0, ghi = 0.0, tau = 0.0, log_r = 0.0;
        int side = 0, it = 0;

        for (;;) {
            const int action = cb.action;
            if (action == MC_DONE) break;
            if (action == MC_REPEAT) {
#pragma unroll
                for (int m = 0; m < RPT; ++m)
                    if (own[m]) yd[row[m]] = y[m];
                __syncthreads();
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
            rk_step();
            float se = 0.f;
            double sn = 0.0;
            {
                T he[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) he[j] = coefT(21 + j);
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    T ex = 0, ey = 0;
#pragma unroll
                    for (int j = 0; j < 7; ++j) {
                        ex = fma(he[j], k[j][m].x, ex);
                        ey = fma(he[j], k[j][m].y, ey);
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
                    sn += ynew[m].x * ynew[m].x + ynew[m].y * ynew[m].y;
                }
            }
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
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    y[m] = ynew[m];
                    yf[m] = yfn[m];
                    k[0][m] = k[6][m];
                }
                const int sv = cb.save;
                if (sv >= 0) {
#pragma unroll
                    for (int m = 0; m < RPT; ++m)
                        if (own[m]) yd[row[m]] = y[m];
                    __syncthreads();
                    save(sv);
                }
                continue;
            }
            if (accept == 0) continue;
            // ---- quantum jump: locate the crossing ----
            while (cb.rootgo) {
                rk_step();
                double n2 = 0.0;
                norm2_ynew(&n2);
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
            // psi* = ynew (last evaluated point); channel weights |C_c psi*|^2
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) yd[row[m]] = ynew[m];
            __syncthreads();
            for (int c = 0; c < J.n_c; ++c) {
                double s = 0.0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    const int i = c * n + row[m];
                    double vx = 0.0, vy = 0.0;
                    for (int p = __ldg(Crp + i); p < __ldg(Crp + i + 1); ++p) {
                        const double2 cv = Cv[p];
                        const double2 v = yd[__ldg(Cci + p)];
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
            {
                const int ch = cb.ch;
                const double inv = cb.inv;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    const int i = ch * n + row[m];
                    double vx = 0.0, vy = 0.0;
                    for (int p = __ldg(Crp + i); p < __ldg(Crp + i + 1); ++p) {
                        const double2 cv = Cv[p];
                        const double2 v = yd[__ldg(Cci + p)];
                        vx += cv.x * v.x - cv.y * v.y;
                        vy += cv.x * v.y + cv.y * v.x;
                    }
                    y[m] = make_double2(vx * inv, vy * inv);
                    ys0[row[m]] = from_d2_mc<T2>(y[m]);
                    ynew[m] = y[m];
                }
            }
            sync_yf();
            if (warp == 0 && J.n_td > 0) publish_td_at(cb.tnow);
            __syncthreads();
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) k[0][m] = rhs_row(row[m], ys0, 7);
            double n2 = 0.0;
            norm2_ynew(&n2);  // ynew == y here: |psi|^2 after the jump
            if (tid == 0) norm2 = n2;
            __syncthreads();
        }
        // resumable trajectories: the ket at the last time and the stream
        if (J.psi_out) {
#pragma unroll
            for (int m = 0; m < RPT; ++m)
                if (own[m]) J.psi_out[(size_t)jt * n + row[m]] = y[m];
        }
        if (J.rng_draw && tid == 0) {
            J.rng_draw[jt] = draw;
            J.rng_r[jt] = r;
        }
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

template <bool MIXED, int RPT, int MAXT, int MINB>
cudaError_t mc_launch_t(const McJob& J, int T, cudaStream_t st) {
    using T2 = typename MPrec<MIXED>::T2;
    size_t smem = (size_t)J.n * (sizeof(double2) + 2 * sizeof(T2)) + 16 +
                  (size_t)(T / 32 + 1) * mc_red_stride(J.n_e, J.n_c) * sizeof(double) + 32;
    if (J.a_smem) smem += 16 + (size_t)J.n * sizeof(int4) + (size_t)J.a_nnz * (sizeof(T2) + 4);
    auto kern = mc_traj_kernel<MIXED, RPT, MAXT, MINB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int grid = per_sm * nsm;
    if (grid > J.ntraj) grid = J.ntraj;
    count_launch();
    kern<<<grid, T, smem, st>>>(J);
    return cudaGetLastError();
}

}  // namespace qtl
