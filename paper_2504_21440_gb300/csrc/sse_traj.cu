// ssesolve: the stochastic Schroedinger equation under homodyne detection
// (paper Sec. 3.5), in Ito form
//     d psi = -i K psi dt + sum_n M_n psi dW_n,
//     -i K psi = A psi + sum_n (e_n/2) S_n psi - sum_n (e_n^2/8) psi,
//     A = -i H - 1/2 sum_n S_n^dag S_n,   M_n = S_n - e_n/2,
//     e_n = <psi| S_n + S_n^dag |psi> = 2 Re <psi| S_n psi>,
// with the homodyne current J_n = e_n + dW_n/dt.  The system's collapse
// operators are the stochastic operators S_n.
//
// One CTA integrates one trajectory at a time (persistent over
// trajectories), thread t owning rows t + m*T as in the jump trajectories.
// A step of size h (fixed, clamped to land on tlist) is Euler-Maruyama from
// the step's start: e_n by a block reduction, then
//     psi <- psi + h (-i K psi) + sum_n dW_n M_n psi,
// and the state renormalised by a second reduction.  dW_n = sqrt(h) z with
// z standard normal from the trajectory's Philox stream by the Box-Muller
// transform (draws 2j, 2j + 1, j = step * n_sc + n; cosine branch).  The
// state is FP64; psi is staged in shared memory for the operator products.
#include "internal.h"
#include "mc_common.cuh"

namespace qtl {

// z = sqrt(-2 ln u1) cos(2 pi u2) (Box & Muller, 1958)
__device__ __forceinline__ double box_muller(unsigned long long seed, unsigned long long traj, unsigned j) {
    const double u1 = philox_uniform(seed, traj, 2u * j);
    const double u2 = philox_uniform(seed, traj, 2u * j + 1u);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

struct SseCtl {
    double h, sqh;
    double dW[SSE_MAXSC];
    double js[SSE_MAXSC];
    int go;
};

template <int RPT>
__global__ void __launch_bounds__(256) sse_traj_kernel(McJob J) {
    extern __shared__ __align__(16) unsigned char sse_smem[];
    __shared__ SseCtl cb;
    const int n = J.n, nsc = J.n_c;
    const int tid = threadIdx.x, T_ = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (T_ + 31) >> 5;
    const int rs = (1 + 2 * J.n_e > nsc ? 1 + 2 * J.n_e : nsc) + 1;
    double2* xs = (double2*)sse_smem;
    double* wred = (double*)(((uintptr_t)(xs + n) + 15) & ~(uintptr_t)15);
    double* bout = wred + nw * rs;
    BlockReducer red{wred, bout, rs, lane, warp, tid, nw};
    long long steps = 0;   // thread 0

    for (int jt = blockIdx.x; jt < J.ntraj; jt += gridDim.x) {
        const unsigned long long traj = (unsigned long long)(J.traj_offset + jt);
        double2 y[RPT];
        int row[RPT];
        bool own[RPT];
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            row[m] = tid + m * T_;
            own[m] = row[m] < n;
            y[m] = own[m] ? J.psi0[row[m]] : make_double2(0.0, 0.0);
            if (own[m]) xs[row[m]] = y[m];
        }
        __syncthreads();
        // (S_n psi)_r from the shared copy of psi
        auto s_row = [&](int c, int r) -> double2 {
            double vx = 0.0, vy = 0.0;
            const int i = c * n + r;
            for (int p = __ldg(J.crp + i); p < __ldg(J.crp + i + 1); ++p) {
                const double2 cv = J.cv[p];
                const double2 v = xs[__ldg(J.cci + p)];
                vx += cv.x * v.x - cv.y * v.y;
                vy += cv.x * v.y + cv.y * v.x;
            }
            return make_double2(vx, vy);
        };
        // e_n = 2 Re <psi|S_n psi> into bout[0..nsc)
        auto measure_e = [&]() {
            for (int c = 0; c < nsc; ++c) {
                double s = 0.0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    const double2 v = s_row(c, row[m]);
                    s += 2.0 * (y[m].x * v.x + y[m].y * v.y);
                }
                red.stage(c, s);
            }
            red.finish(nsc);
        };
        // <psi|O|psi>/<psi|psi> and the currents in cb.js at output idx
        auto save = [&](int idx) {
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
                    for (int p = __ldg(J.orp + i); p < __ldg(J.orp + i + 1); ++p) {
                        const double2 o = J.ov[p];
                        const double2 v = xs[__ldg(J.oci + p)];
                        ox += o.x * v.x - o.y * v.y;
                        oy += o.x * v.y + o.y * v.x;
                    }
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
            if (tid < nsc)
                J.traj_meas[((size_t)tid * J.nt + idx) * J.ntraj + jt] = make_double2(cb.js[tid], 0.0);
            __syncthreads();
        };

        measure_e();
        if (tid < nsc) cb.js[tid] = bout[tid];
        __syncthreads();
        save(0);
        double t = J.tlist[0];   // thread 0
        unsigned step = 0;       // thread 0
        for (int idx = 1; idx < J.nt; ++idx) {
            const double t_target = J.tlist[idx];
            for (;;) {
                if (tid == 0) {
                    cb.go = t < t_target;
                    if (cb.go) {
                        const bool land = lands(J.dt_fixed, t, t_target);
                        const double h = land ? (t_target - t) : J.dt_fixed;
                        cb.h = h;
                        cb.sqh = sqrt(h);
                        for (int c = 0; c < nsc; ++c) cb.dW[c] = cb.sqh * box_muller(J.seed, traj, step * nsc + c);
                        t = land ? t_target : t + h;
                        ++step;
                        ++steps;
                    }
                }
                __syncthreads();
                if (!cb.go) break;
                const double h = cb.h;
                measure_e();   // e_n at the step's start (bout[0..nsc))
                double e[SSE_MAXSC], dW[SSE_MAXSC];
                double e2 = 0.0;
#pragma unroll
                for (int c = 0; c < SSE_MAXSC; ++c) {
                    e[c] = c < nsc ? bout[c] : 0.0;
                    dW[c] = c < nsc ? cb.dW[c] : 0.0;
                    e2 += e[c] * e[c];
                }
                double2 yn[RPT];
                double s2 = 0.0;
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    yn[m] = make_double2(0.0, 0.0);
                    if (!own[m]) continue;
                    const double2 a = mc_spmv_row<double2, double2>(row[m], J.aseg, J.aci, J.av64, xs);
                    // drift  A psi + sum (e/2) S psi - sum (e^2/8) psi
                    double dx = a.x - 0.125 * e2 * y[m].x, dy = a.y - 0.125 * e2 * y[m].y;
                    // noise  sum dW (S psi - e/2 psi)
                    double nx = 0.0, ny = 0.0;
                    for (int c = 0; c < nsc; ++c) {
                        const double2 v = s_row(c, row[m]);
                        dx += 0.5 * e[c] * v.x;
                        dy += 0.5 * e[c] * v.y;
                        nx += dW[c] * (v.x - 0.5 * e[c] * y[m].x);
                        ny += dW[c] * (v.y - 0.5 * e[c] * y[m].y);
                    }
                    yn[m] = make_double2(y[m].x + h * dx + nx, y[m].y + h * dy + ny);
                    s2 += yn[m].x * yn[m].x + yn[m].y * yn[m].y;
                }
                red.stage(0, s2);
                red.finish(1);   // everyone is past its reads of xs
                const double inv = 1.0 / sqrt(bout[0]);
#pragma unroll
                for (int m = 0; m < RPT; ++m) {
                    if (!own[m]) continue;
                    y[m] = make_double2(yn[m].x * inv, yn[m].y * inv);
                    xs[row[m]] = y[m];
                }
                if (tid < nsc) cb.js[tid] = e[tid] + dW[tid] / h;
                __syncthreads();
            }
            save(idx);
        }
    }
    if (tid == 0) atomicAdd((unsigned long long*)&J.info->steps_acc, (unsigned long long)steps);
}

cudaError_t launch_sse_traj(const McJob& J, cudaStream_t st) {
    int T = 32, rpt = 1;
    if (J.n <= 256) {
        T = (J.n + 31) / 32 * 32;
    } else {
        T = 256;
        rpt = J.n <= 512 ? 2 : 4;
    }
    if (J.n > 1024 || J.n_c < 1 || J.n_c > SSE_MAXSC) return cudaErrorInvalidValue;
    const int nw = (T + 31) / 32;
    const int rs = (1 + 2 * J.n_e > J.n_c ? 1 + 2 * J.n_e : J.n_c) + 1;
    const size_t smem = (size_t)J.n * sizeof(double2) + 16 + (size_t)(nw + 1) * rs * sizeof(double);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (rpt == 1) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sse_traj_kernel<1>, T, smem);
    } else if (rpt == 2) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sse_traj_kernel<2>, T, smem);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sse_traj_kernel<4>, T, smem);
    }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * nsm;
    if (grid > J.ntraj) grid = J.ntraj;
    count_launch();
    if (rpt == 1)
        sse_traj_kernel<1><<<grid, T, smem, st>>>(J);
    else if (rpt == 2)
        sse_traj_kernel<2><<<grid, T, smem, st>>>(J);
    else
        sse_traj_kernel<4><<<grid, T, smem, st>>>(J);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // trajectory means of the expectation values and of the currents
    if ((e = launch_traj_mean(J.traj_expect, J.expect, J.n_e * J.nt, J.ntraj, st)) != cudaSuccess) return e;
    return launch_traj_mean(J.traj_meas, J.meas, J.n_c * J.nt, J.ntraj, st);
}

}  // namespace qtl
