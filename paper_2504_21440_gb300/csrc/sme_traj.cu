// smesolve: the stochastic master equation under homodyne detection (paper
// Sec. 3.5), in Ito form
//     d rho = L rho dt + sum_n H[S_n] rho dW_n,
//     H[S] rho = S rho + rho S^dag - Tr(S rho + rho S^dag) rho,
// where L is the Liouvillian of H and of every collapse operator (the
// unmeasured C_i and the measured S_n), and the homodyne current is
// J_n = Tr(S_n rho + rho S_n^dag) + dW_n/dt.
//
// One CTA integrates one trajectory's density matrix at a time (persistent
// over trajectories): vec(rho) (column stacking, n*n <= 4096 entries) lives
// in shared memory and thread t owns the entries t + m*T.  A step of size h
// (fixed, clamped to land on tlist) is Euler-Maruyama from the step's start:
// the traces of S_n rho + rho S_n^dag from the diagonal entries (one block
// reduction), then every entry's update
//     rho_e + h (L rho)_e + sum_n dW_n ((S_n rho + rho S_n^dag)_e - tr_n rho_e)
// is formed in registers and written back after a barrier.  Wiener
// increments as in ssesolve (Philox, Box-Muller, draw j = step * n_sc + n).
// No renormalisation: at unit trace Tr H[S] rho = 0 and Tr L rho = 0.  FP64.
#include "internal.h"
#include "mc_common.cuh"

namespace qtl {

__device__ __forceinline__ double sme_normal(unsigned long long seed, unsigned long long traj, unsigned j) {
    const double u1 = philox_uniform(seed, traj, 2u * j);
    const double u2 = philox_uniform(seed, traj, 2u * j + 1u);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

struct SmeCtl {
    double h;
    double dW[SSE_MAXSC];
    double js[SSE_MAXSC];
    int go;
};

template <int EPT>
__global__ void __launch_bounds__(1024) sme_traj_kernel(McJob J) {
    extern __shared__ __align__(16) unsigned char sme_smem[];
    __shared__ SmeCtl cb;
    const int n = J.n, L = n * n, nsc = J.n_c;
    const int tid = threadIdx.x, T_ = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (T_ + 31) >> 5;
    const int rs = (2 * J.n_e > nsc ? 2 * J.n_e : nsc) + 1;
    double2* rho = (double2*)sme_smem;
    double* wred = (double*)(((uintptr_t)(rho + L) + 15) & ~(uintptr_t)15);
    double* bout = wred + nw * rs;
    BlockReducer red{wred, bout, rs, lane, warp, tid, nw};
    long long steps = 0;   // thread 0

    // (S_n rho + rho S_n^dag) at entry (i, j): rows i and j of S_n against
    // column j and row i of rho
    auto hom = [&](int c, int i, int j) -> double2 {
        double vx = 0.0, vy = 0.0;
        const int ri = c * n + i, rj = c * n + j;
        for (int p = __ldg(J.crp + ri); p < __ldg(J.crp + ri + 1); ++p) {
            const double2 s = J.cv[p];
            const double2 r = rho[__ldg(J.cci + p) + n * j];
            vx += s.x * r.x - s.y * r.y;
            vy += s.x * r.y + s.y * r.x;
        }
        for (int p = __ldg(J.crp + rj); p < __ldg(J.crp + rj + 1); ++p) {
            const double2 s = J.cv[p];   // rho[i, k] conj(S[j, k])
            const double2 r = rho[i + n * __ldg(J.cci + p)];
            vx += r.x * s.x + r.y * s.y;
            vy += r.y * s.x - r.x * s.y;
        }
        return make_double2(vx, vy);
    };
    // tr_n = Re Tr(S_n rho + rho S_n^dag) into bout[0..nsc)
    auto traces = [&]() {
        for (int c = 0; c < nsc; ++c) {
            double s = 0.0;
            for (int i = tid; i < n; i += T_) s += hom(c, i, i).x;
            red.stage(c, s);
        }
        red.finish(nsc);
    };
    for (int jt = blockIdx.x; jt < J.ntraj; jt += gridDim.x) {
        const unsigned long long traj = (unsigned long long)(J.traj_offset + jt);
        // rho0 = |psi0><psi0|
#pragma unroll
        for (int m = 0; m < EPT; ++m) {
            const int e = tid + m * T_;
            if (e < L) {
                const double2 a = J.psi0[e % n], b = J.psi0[e / n];
                rho[e] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
            }
        }
        __syncthreads();
        auto record = [&](int idx) {
            for (int k = 0; k < J.n_e; ++k) {
                double sr = 0.0, si = 0.0;
#pragma unroll
                for (int m = 0; m < EPT; ++m) {
                    const int e = tid + m * T_;
                    if (e >= L) continue;
                    const double2 w = __ldg(J.ew + (size_t)e * J.n_e + k), r = rho[e];
                    sr += w.x * r.x - w.y * r.y;
                    si += w.x * r.y + w.y * r.x;
                }
                red.stage(2 * k, sr);
                red.stage(2 * k + 1, si);
            }
            red.finish(2 * J.n_e);
            for (int e = tid; e < J.n_e; e += blockDim.x)
                J.traj_expect[((size_t)e * J.nt + idx) * J.ntraj + jt] =
                    make_double2(bout[2 * e], bout[2 * e + 1]);
            if (tid < nsc)
                J.traj_meas[((size_t)tid * J.nt + idx) * J.ntraj + jt] = make_double2(cb.js[tid], 0.0);
            __syncthreads();
        };
        traces();
        if (tid < nsc) cb.js[tid] = bout[tid];
        __syncthreads();
        record(0);
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
                        const double sq = sqrt(h);
                        for (int c = 0; c < nsc; ++c) cb.dW[c] = sq * sme_normal(J.seed, traj, step * nsc + c);
                        t = land ? t_target : t + h;
                        ++step;
                        ++steps;
                    }
                }
                __syncthreads();
                if (!cb.go) break;
                const double h = cb.h;
                traces();   // tr_n at the step's start in bout[0..nsc)
                double tr[SSE_MAXSC], dW[SSE_MAXSC];
#pragma unroll
                for (int c = 0; c < SSE_MAXSC; ++c) {
                    tr[c] = c < nsc ? bout[c] : 0.0;
                    dW[c] = c < nsc ? cb.dW[c] : 0.0;
                }
                double2 nv[EPT];
#pragma unroll
                for (int m = 0; m < EPT; ++m) {
                    const int e = tid + m * T_;
                    nv[m] = make_double2(0.0, 0.0);
                    if (e >= L) continue;
                    const double2 r = rho[e];
                    const double2 lr = mc_spmv_row<double2, double2>(e, J.aseg, J.aci, J.av64, rho);
                    double x = r.x + h * lr.x, y = r.y + h * lr.y;
                    for (int c = 0; c < nsc; ++c) {
                        const double2 v = hom(c, e % n, e / n);
                        x += dW[c] * (v.x - tr[c] * r.x);
                        y += dW[c] * (v.y - tr[c] * r.y);
                    }
                    nv[m] = make_double2(x, y);
                }
                __syncthreads();   // every read of rho is done
#pragma unroll
                for (int m = 0; m < EPT; ++m) {
                    const int e = tid + m * T_;
                    if (e < L) rho[e] = nv[m];
                }
                if (tid < nsc) cb.js[tid] = tr[tid] + dW[tid] / h;
                __syncthreads();
            }
            record(idx);
        }
    }
    if (tid == 0) atomicAdd((unsigned long long*)&J.info->steps_acc, (unsigned long long)steps);
}

cudaError_t launch_sme_traj(const McJob& J, cudaStream_t st) {
    const int L = J.n * J.n;
    if (L > 4096 || J.n_c < 1 || J.n_c > SSE_MAXSC) return cudaErrorInvalidValue;
    const int ept = L <= 1024 ? 1 : (L <= 2048 ? 2 : 4);
    int T = (L + ept - 1) / ept;
    T = (T + 31) / 32 * 32;
    const int nw = T / 32;
    const int rs = (2 * J.n_e > J.n_c ? 2 * J.n_e : J.n_c) + 1;
    const size_t smem = (size_t)L * sizeof(double2) + 16 + (size_t)(nw + 1) * rs * sizeof(double);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem)) != cudaSuccess) return r;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        int grid = per_sm * nsm;
        if (grid > J.ntraj) grid = J.ntraj;
        count_launch();
        kern<<<grid, T, smem, st>>>(J);
        return cudaGetLastError();
    };
    if (ept == 1)
        e = run(sme_traj_kernel<1>);
    else if (ept == 2)
        e = run(sme_traj_kernel<2>);
    else
        e = run(sme_traj_kernel<4>);
    if (e != cudaSuccess) return e;
    if ((e = launch_traj_mean(J.traj_expect, J.expect, J.n_e * J.nt, J.ntraj, st)) != cudaSuccess) return e;
    return launch_traj_mean(J.traj_meas, J.meas, J.n_c * J.nt, J.ntraj, st);
}

}  // namespace qtl
