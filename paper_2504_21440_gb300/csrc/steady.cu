// Stationary states on the GPU: steadystate (Sec. 3.2) and
// steadystate_fourier (the periodic long-time state of Appendix A).
//
// steadystate solves L vec(rho) = 0 with Tr rho = 1.  As in the direct
// method, one equation of L vec(rho) = 0 is redundant (Tr(L rho) = 0 for
// every rho) and row 0 is replaced by the trace row: M x = e_0.
// steadystate_fourier solves the block-tridiagonal system of the Fourier
// components rho_k (k = -K..K) of the periodic state under
// H(t) = H0 + F cos(w t) X:
//     (L0 - i k w) rho_k + L1 (rho_{k-1} + rho_{k+1}) = 0,  L1 = -i[(F/2) X, .],
// with Tr rho_0 = 1 in place of the first equation of the k = 0 block.
//
// Method (the paper prescribes a direct solve; this is an iterative one that
// runs on the GPU): flexible GMRES(m) with classical Gram-Schmidt applied
// twice, right-preconditioned by the inverse of the no-jump part of each
// diagonal block, S_k X = A X + X A^H - i k w X with A = -i H_eff.
// Diagonalising A = V diag(lambda) V^-1 once (host, eig.cpp) gives
//     S_k^-1 R = V [(V^-1 R V^-H) ./ (lambda_i + conj(lambda_j) - i k w)] V^H,
// four dense complex GEMMs and an elementwise division per block, which run
// here as a batched FP64 GEMM with the division fused into the second
// GEMM's epilogue.  Denominators that vanish (an undamped mode of A paired
// with itself, e.g. the ground state of a decaying system) are replaced by
// the smallest nonzero decay rate.  All vectors, products, dot products and
// the residual are FP64; the small Hessenberg least-squares problem is
// solved on the host.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace qtl {

using cd = std::complex<double>;
bool eig_dense(int n, const std::vector<cd>& A, std::vector<cd>& lam, std::vector<cd>& V,
               std::vector<cd>& Vinv, double* cond);

struct SsCache {
    int n = 0;
    double cond = 0.0;
    double2* V = nullptr;     // eigenvectors of A (columns), n x n column-major
    double2* Vinv = nullptr;
    double2* lam = nullptr;   // eigenvalues
    double floor_den = 1.0;   // replacement for vanishing denominators (negative real)
    double tiny = 0.0;        // |denominator| below this counts as vanishing
};

void ss_cache_free(System& s) {
    if (!s.ss) return;
    cudaFree(s.ss->V);
    cudaFree(s.ss->Vinv);
    cudaFree(s.ss->lam);
    delete s.ss;
    s.ss = nullptr;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// y = M x over K blocks of N2 = n^2 rows (block a has k = a - kmid):
// y_a = L0 x_a - i k w x_a + L1 (x_{a-1} + x_{a+1}); row 0 of block kmid is
// the trace of x_kmid.  One thread per row.
__global__ void ss_matvec_kernel(int n, int K, int kmid, double w, const int32_t* __restrict__ rp0,
                                 const int32_t* __restrict__ ci0, const double2* __restrict__ v0,
                                 const int32_t* __restrict__ rp1, const int32_t* __restrict__ ci1,
                                 const double2* __restrict__ v1, const double2* __restrict__ x,
                                 double2* __restrict__ y) {
    const long long N2 = (long long)n * n;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N2 * K) return;
    const int a = (int)(i / N2);
    const int r = (int)(i - (long long)a * N2);
    const double2* xa = x + (long long)a * N2;
    double2 acc = make_double2(0.0, 0.0);
    if (a == kmid && r == 0) {
        for (int d = 0; d < n; ++d) {
            const double2 v = xa[(long long)d * (n + 1)];
            acc.x += v.x;
            acc.y += v.y;
        }
        y[i] = acc;
        return;
    }
    for (int p = rp0[r]; p < rp0[r + 1]; ++p) acc = cfma(v0[p], xa[ci0[p]], acc);
    const double kw = (double)(a - kmid) * w;
    const double2 xr = xa[r];
    acc.x += kw * xr.y;   // - i k w x
    acc.y -= kw * xr.x;
    if (rp1) {
        for (int b = a - 1; b <= a + 1; b += 2) {
            if (b < 0 || b >= K) continue;
            const double2* xb = x + (long long)b * N2;
            for (int p = rp1[r]; p < rp1[r + 1]; ++p) acc = cfma(v1[p], xb[ci1[p]], acc);
        }
    }
    y[i] = acc;
}

// Batched complex GEMM, C_z = op(A_z) op(B_z) for z = blockIdx.z, n x n,
// column-major, op = identity or conjugate transpose.  A stride of 0 shares
// the operand across the batch.  Epilogue (mode 1): divide element (i, j) of
// block z by lambda_i + conj(lambda_j) - i k_z w, k_z = z - kmid.
constexpr int SG_T = 32, SG_K = 16;
__global__ void __launch_bounds__(256) ss_gemm_kernel(int n, const double2* __restrict__ A, long long sa,
                                                      int ta, const double2* __restrict__ B, long long sb,
                                                      int tb, double2* __restrict__ C, long long sc,
                                                      int mode, const double2* __restrict__ lam, int kmid,
                                                      double w, double tiny, double floor_den) {
    __shared__ double2 As[SG_K][SG_T + 1];   // As[k][i] = op(A)[i][k]
    __shared__ double2 Bs[SG_K][SG_T + 1];   // Bs[k][j] = op(B)[k][j]
    const int z = blockIdx.z;
    A += sa * z;
    B += sb * z;
    C += sc * z;
    const int i0 = blockIdx.y * SG_T, j0 = blockIdx.x * SG_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 2 x 2 outputs each
    double2 acc[2][2];
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) acc[u][v] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < n; k0 += SG_K) {
        for (int e = threadIdx.x; e < SG_K * SG_T; e += 256) {
            const int kk = e / SG_T, ii = e % SG_T;
            const int gi = i0 + ii, gk = k0 + kk;
            double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
            if (gi < n && gk < n) {
                if (!ta) {
                    va = A[(long long)gi + (long long)n * gk];
                } else {
                    const double2 t = A[(long long)gk + (long long)n * gi];
                    va = make_double2(t.x, -t.y);
                }
            }
            const int gj = j0 + ii;
            if (gj < n && gk < n) {
                if (!tb) {
                    vb = B[(long long)gk + (long long)n * gj];
                } else {
                    const double2 t = B[(long long)gj + (long long)n * gk];
                    vb = make_double2(t.x, -t.y);
                }
            }
            As[kk][ii] = va;
            Bs[kk][ii] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < SG_K; ++kk) {
            const double2 a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = cfma(a0, b0, acc[0][0]);
            acc[0][1] = cfma(a0, b1, acc[0][1]);
            acc[1][0] = cfma(a1, b0, acc[1][0]);
            acc[1][1] = cfma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    const double kw = (double)(z - kmid) * w;
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int gi = i0 + ty + 16 * u, gj = j0 + tx + 16 * v;
            if (gi >= n || gj >= n) continue;
            double2 c = acc[u][v];
            if (mode == 1) {
                const double2 li = lam[gi], lj = lam[gj];
                double dr = li.x + lj.x, di = li.y - lj.y - kw;
                if (hypot(dr, di) <= tiny) {
                    dr = floor_den;
                    di = 0.0;
                }
                const double q = 1.0 / (dr * dr + di * di);
                c = make_double2((c.x * dr + c.y * di) * q, (c.y * dr - c.x * di) * q);
            }
            C[(long long)gi + (long long)n * gj] = c;
        }
}

// C = op(A) op(B) for one n x n complex FP64 pair (used by dsf.cu)
cudaError_t launch_zgemm(int n, const double2* A, int ta, const double2* B, int tb, double2* C, cudaStream_t st) {
    dim3 g((n + SG_T - 1) / SG_T, (n + SG_T - 1) / SG_T, 1);
    count_launch();
    ss_gemm_kernel<<<g, 256, 0, st>>>(n, A, 0, ta, B, 0, tb, C, 0, 0, nullptr, 0, 0.0, 0.0, 0.0);
    return cudaGetLastError();
}

// Y_z ./= lambda_i + conj(lambda_j) - i k_z w (the tensor-core path's division)
__global__ void ss_divide_kernel(int n, int K, int kmid, double w, const double2* __restrict__ lam, double tiny,
                                 double floor_den, double2* __restrict__ Y) {
    const long long n2 = (long long)n * n;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n2 * K) return;
    const int z = (int)(e / n2);
    const long long r = e - (long long)z * n2;
    const int i = (int)(r % n), j = (int)(r / n);
    const double2 li = lam[i], lj = lam[j];
    double dr = li.x + lj.x, di = li.y - lj.y - (double)(z - kmid) * w;
    if (hypot(dr, di) <= tiny) {
        dr = floor_den;
        di = 0.0;
    }
    const double q = 1.0 / (dr * dr + di * di);
    const double2 c = Y[e];
    Y[e] = make_double2((c.x * dr + c.y * di) * q, (c.y * dr - c.x * di) * q);
}

// partial[b][j] = sum over this block's rows of conj(V[r][j]) w[r], j < J
__global__ void ss_mdot_kernel(long long N, int J, const double2* __restrict__ V, long long ldv,
                               const double2* __restrict__ w, double2* __restrict__ partial) {
    __shared__ double2 red[256];
    for (int j = 0; j < J; ++j) {
        double2 s = make_double2(0.0, 0.0);
        for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
             r += (long long)gridDim.x * blockDim.x) {
            const double2 v = V[r + ldv * j], x = w[r];
            s.x += v.x * x.x + v.y * x.y;
            s.y += v.x * x.y - v.y * x.x;
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                red[threadIdx.x].x += red[threadIdx.x + o].x;
                red[threadIdx.x].y += red[threadIdx.x + o].y;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * J + j] = red[0];
        __syncthreads();
    }
}

// out[j] = sum_b partial[b][j] (fixed order)
__global__ void ss_sum_kernel(int nb, int J, const double2* __restrict__ partial, double2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; ++b) {
        s.x += partial[(long long)b * J + j].x;
        s.y += partial[(long long)b * J + j].y;
    }
    out[j] = s;
}

// w[r] += sign * sum_j V[r][j] h[j]  (sign = -1: Gram-Schmidt; +1: x += Z y)
__global__ void ss_update_kernel(long long N, int J, const double2* __restrict__ V, long long ldv,
                                 const double2* __restrict__ h, double sign, double2* __restrict__ w) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= N) return;
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < J; ++j) s = cfma(V[r + ldv * j], h[j], s);
    w[r] = make_double2(w[r].x + sign * s.x, w[r].y + sign * s.y);
}

// y = a * x (complex scalar a given on the host)
__global__ void ss_scale_kernel(long long N, double ar, double ai, const double2* __restrict__ x,
                                double2* __restrict__ y) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= N) return;
    y[r] = cmul(make_double2(ar, ai), x[r]);
}

// y = b - y
__global__ void ss_residual_kernel(long long N, const double2* __restrict__ b, double2* __restrict__ y) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= N) return;
    y[r] = make_double2(b[r].x - y[r].x, b[r].y - y[r].y);
}

namespace {

struct SsSolver {
    int n = 0, K = 1, kmid = 0;
    double w = 0.0;
    long long N = 0;          // unknowns: K n^2
    cudaStream_t st = nullptr;
    const DevCsr* L0 = nullptr;
    DevCsr L1;                // Fourier coupling, or empty
    const SsCache* pc = nullptr;
    double2 *Vk = nullptr, *Zk = nullptr, *x = nullptr, *b = nullptr, *wv = nullptr, *t1 = nullptr,
            *t2 = nullptr, *partial = nullptr, *hd = nullptr;
    int m = 60, nb = 128;
    int mixed = 0;            // preconditioner GEMMs on the tensor cores (split BF16)
    void* tcs = nullptr;      // their scratch
    int* tc_err = nullptr;    // device flag of a tensor-core wait that gave up
    cudaError_t err = cudaSuccess;

    void chk(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    unsigned grid(long long cnt) const { return (unsigned)((cnt + 255) / 256); }

    void matvec(const double2* in, double2* out) {
        count_launch();
        ss_matvec_kernel<<<grid(N), 256, 0, st>>>(n, K, kmid, w, L0->rp, L0->ci, L0->v64, L1.rp, L1.ci,
                                                   L1.v64, in, out);
        chk(cudaGetLastError());
    }
    void gemm(const double2* A, long long sa, int ta, const double2* B, long long sb, int tb, double2* C,
              int mode) {
        dim3 g((n + SG_T - 1) / SG_T, (n + SG_T - 1) / SG_T, K);
        count_launch();
        ss_gemm_kernel<<<g, 256, 0, st>>>(n, A, sa, ta, B, sb, tb, C, (long long)n * n, mode, pc->lam, kmid,
                                          w, pc->tiny, pc->floor_den);
        chk(cudaGetLastError());
    }
    // out = S^-1 in, block by block
    void precond(const double2* in, double2* out) {
        const long long n2 = (long long)n * n;
        if (mixed) {
            for (int z = 0; z < K; ++z) {
                const long long o = n2 * z;
                chk(launch_tc_zgemm(n, pc->Vinv, 0, in + o, 0, t1 + o, tcs, tc_err, st));
                chk(launch_tc_zgemm(n, t1 + o, 0, pc->Vinv, 1, t2 + o, tcs, tc_err, st));
            }
            count_launch();
            ss_divide_kernel<<<grid(N), 256, 0, st>>>(n, K, kmid, w, pc->lam, pc->tiny, pc->floor_den, t2);
            chk(cudaGetLastError());
            for (int z = 0; z < K; ++z) {
                const long long o = n2 * z;
                chk(launch_tc_zgemm(n, pc->V, 0, t2 + o, 0, t1 + o, tcs, tc_err, st));
                chk(launch_tc_zgemm(n, t1 + o, 0, pc->V, 1, out + o, tcs, tc_err, st));
            }
            return;
        }
        gemm(pc->Vinv, 0, 0, in, n2, 0, t1, 0);     // V^-1 R
        gemm(t1, n2, 0, pc->Vinv, 0, 1, t2, 1);     // (V^-1 R V^-H) ./ D
        gemm(pc->V, 0, 0, t2, n2, 0, t1, 0);        // V Y
        gemm(t1, n2, 0, pc->V, 0, 1, out, 0);       // V Y V^H
    }
    // h[0..J) = V^H w on the host (and on the device in hd)
    void mdot(const double2* V, int J, const double2* vec, std::vector<cd>& h) {
        count_launch(2);
        ss_mdot_kernel<<<nb, 256, 0, st>>>(N, J, V, N, vec, partial);
        ss_sum_kernel<<<(J + 63) / 64, 64, 0, st>>>(nb, J, partial, hd);
        chk(cudaGetLastError());
        h.resize(J);
        chk(cudaMemcpyAsync(h.data(), hd, (size_t)J * sizeof(double2), cudaMemcpyDeviceToHost, st));
        chk(cudaStreamSynchronize(st));
    }
    double norm(const double2* vec) {
        std::vector<cd> h;
        mdot(vec, 1, vec, h);
        return std::sqrt(std::max(h[0].real(), 0.0));
    }
    void update(const double2* V, int J, const std::vector<cd>& h, double sign, double2* vec) {
        chk(cudaMemcpyAsync(hd, h.data(), (size_t)J * sizeof(double2), cudaMemcpyHostToDevice, st));
        count_launch();
        ss_update_kernel<<<grid(N), 256, 0, st>>>(N, J, V, N, hd, sign, vec);
        chk(cudaGetLastError());
    }
    void scale(cd a, const double2* in, double2* out) {
        count_launch();
        ss_scale_kernel<<<grid(N), 256, 0, st>>>(N, a.real(), a.imag(), in, out);
        chk(cudaGetLastError());
    }

    // FGMRES(m); returns QTL_OK when |b - M x| <= tol |b|
    qtl_status solve(double tol, int max_iter, int* iters, double* rel) {
        const double bn = 1.0;   // b = e_0 of the trace row
        int it = 0;
        double res = 1.0;
        std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), h, h2, cs_s(m);
        std::vector<double> cs_c(m);
        chk(cudaMemsetAsync(x, 0, (size_t)N * sizeof(double2), st));
        while (err == cudaSuccess && it < max_iter) {
            // r = b - M x into the first Krylov vector
            matvec(x, wv);
            count_launch();
            ss_residual_kernel<<<grid(N), 256, 0, st>>>(N, b, wv);
            chk(cudaGetLastError());
            const double beta = norm(wv);
            res = beta / bn;
            if (!(beta > tol * bn)) break;
            scale(1.0 / beta, wv, Vk);
            std::fill(H.begin(), H.end(), cd(0.0));
            std::fill(g.begin(), g.end(), cd(0.0));
            g[0] = beta;
            int j = 0;
            for (; j < m && it < max_iter; ++j) {
                precond(Vk + (long long)j * N, Zk + (long long)j * N);
                matvec(Zk + (long long)j * N, wv);
                ++it;
                // classical Gram-Schmidt, twice
                mdot(Vk, j + 1, wv, h);
                update(Vk, j + 1, h, -1.0, wv);
                mdot(Vk, j + 1, wv, h2);
                update(Vk, j + 1, h2, -1.0, wv);
                for (int i = 0; i <= j; ++i) H[(size_t)i + (size_t)(m + 1) * j] = h[i] + h2[i];
                const double hn = norm(wv);
                H[(size_t)(j + 1) + (size_t)(m + 1) * j] = hn;
                // previous rotations, then a new one on rows j, j+1
                for (int i = 0; i < j; ++i) {
                    cd& a = H[(size_t)i + (size_t)(m + 1) * j];
                    cd& c = H[(size_t)(i + 1) + (size_t)(m + 1) * j];
                    const cd t = cs_c[i] * a + cs_s[i] * c;
                    c = -std::conj(cs_s[i]) * a + cs_c[i] * c;
                    a = t;
                }
                {
                    cd& a = H[(size_t)j + (size_t)(m + 1) * j];
                    cd& c = H[(size_t)(j + 1) + (size_t)(m + 1) * j];
                    const double aa = std::abs(a), ac = std::abs(c);
                    double cc;
                    cd ss;
                    if (ac == 0.0) {
                        cc = 1.0;
                        ss = 0.0;
                    } else if (aa == 0.0) {
                        cc = 0.0;
                        ss = std::conj(c) / ac;
                    } else {
                        const double r = std::hypot(aa, ac);
                        cc = aa / r;
                        ss = (a / aa) * std::conj(c) / r;
                    }
                    cs_c[j] = cc;
                    cs_s[j] = ss;
                    a = cc * a + ss * c;
                    c = 0.0;
                    g[j + 1] = -std::conj(ss) * g[j];
                    g[j] = cc * g[j];
                }
                res = std::abs(g[j + 1]) / bn;
                if (res <= tol || hn == 0.0) {
                    ++j;
                    break;
                }
                scale(1.0 / hn, wv, Vk + (long long)(j + 1) * N);
            }
            // y from the triangular system, x += Z y
            std::vector<cd> y(j);
            for (int i = j - 1; i >= 0; --i) {
                cd s = g[i];
                for (int l = i + 1; l < j; ++l) s -= H[(size_t)i + (size_t)(m + 1) * l] * y[l];
                y[i] = s / H[(size_t)i + (size_t)(m + 1) * i];
            }
            if (j > 0) update(Zk, j, y, 1.0, x);
            if (res <= tol) break;
        }
        chk(cudaStreamSynchronize(st));
        *iters = it;
        *rel = res;
        if (err != cudaSuccess) return QTL_ECUDA;
        return res <= tol ? QTL_OK : QTL_ESTEP;
    }
};

}  // namespace

// The eigendecomposition of A = -i H_eff and its device copies, built once per system.
static qtl_status ensure_ss_cache(System& s) {
    // built once per system; concurrent first solves on one system build it once
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (s.ss) return QTL_OK;
    const int n = s.n;
    std::vector<cd> A((size_t)n * n, 0.0), lam, V, Vi;
    for (int r = 0; r < n; ++r)
        for (int p = s.A.rp[r]; p < s.A.rp[r + 1]; ++p)
            A[(size_t)r + (size_t)n * s.A.ci[p]] += cd(s.A.re[p], s.A.im[p]);
    double cond = 0.0;
    if (!eig_dense(n, A, lam, V, Vi, &cond)) return QTL_ESTEP;
    SsCache* c = new SsCache();
    c->n = n;
    c->cond = cond;
    double lmax = 0.0, dmin = 0.0;
    for (const cd& l : lam) lmax = std::max(lmax, std::abs(l));
    c->tiny = 1e-10 * std::max(lmax, 1e-300);
    for (const cd& l : lam) {
        const double d = 2.0 * std::fabs(l.real());
        if (d > c->tiny && (dmin == 0.0 || d < dmin)) dmin = d;
    }
    c->floor_den = -(dmin > 0.0 ? dmin : std::max(lmax, 1.0));
    auto up = [&](double2** dst, const std::vector<cd>& v) -> cudaError_t {
        cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(double2));
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*dst, v.data(), v.size() * sizeof(double2), cudaMemcpyHostToDevice);
    };
    cudaError_t e;
    if ((e = up(&c->V, V)) != cudaSuccess || (e = up(&c->Vinv, Vi)) != cudaSuccess ||
        (e = up(&c->lam, lam)) != cudaSuccess) {
        set_cuda_error(e);
        cudaFree(c->V);
        cudaFree(c->Vinv);
        cudaFree(c->lam);
        delete c;
        return e == cudaErrorMemoryAllocation ? QTL_ENOMEM : QTL_ECUDA;
    }
    s.ss = c;
    return QTL_OK;
}

static qtl_status ss_run(System& s, int K, double w, const Csr* L1h, const qtl_ss_opts* o,
                         qtl_c128* rho_out, qtl_ss_stats* stats) {
    qtl_status st;
    if ((st = ensure_liouvillian(s, (int64_t)QTL_SS_MAX_N * QTL_SS_MAX_N)) != QTL_OK) return st;
    if ((st = ensure_ss_cache(s)) != QTL_OK) return st;
    SsSolver S;
    S.n = s.n;
    S.K = K;
    S.kmid = K / 2;
    S.w = w;
    S.N = (long long)K * s.n * s.n;
    S.st = (cudaStream_t)o->cuda_stream;
    S.L0 = &s.dL;
    S.pc = s.ss;
    S.m = o->restart;
    if (L1h && (st = csr_upload(*L1h, S.L1)) != QTL_OK) return st;
    const size_t vb = (size_t)S.N * sizeof(double2);
    char* buf = nullptr;
    S.mixed = o->precision == QTL_MIXED;
    const size_t tcb = S.mixed ? tc_zgemm_scratch_bytes(s.n) : 0;
    const size_t bytes = vb * ((size_t)2 * S.m + 6) + (size_t)S.nb * (S.m + 1) * sizeof(double2) +
                         (size_t)(S.m + 1) * sizeof(double2) + tcb + 20 * 256;
    cudaError_t e = qtl_malloc_async((void**)&buf, bytes, S.st);
    if (e != cudaSuccess) {
        csr_free(S.L1);
        cudaGetLastError();
        return QTL_ENOMEM;
    }
    size_t off = 0;
    auto carve = [&](size_t b) {
        char* p = buf + off;
        off = (off + b + 255) & ~(size_t)255;
        return (double2*)p;
    };
    S.Vk = carve(vb * (S.m + 1));
    S.Zk = carve(vb * S.m);
    S.x = carve(vb);
    S.b = carve(vb);
    S.wv = carve(vb);
    S.t1 = carve(vb);
    S.t2 = carve(vb);
    S.partial = carve((size_t)S.nb * (S.m + 1) * sizeof(double2));
    S.hd = carve((size_t)(S.m + 1) * sizeof(double2));
    if (S.mixed) {
        S.tcs = carve(tcb);
        S.tc_err = (int*)carve(sizeof(int));
        S.chk(cudaMemsetAsync(S.tc_err, 0, sizeof(int), S.st));
    }
    // b = e_0 of the k = 0 block
    S.chk(cudaMemsetAsync(S.b, 0, vb, S.st));
    const double2 one = make_double2(1.0, 0.0);
    S.chk(cudaMemcpyAsync(S.b + (long long)S.kmid * s.n * s.n, &one, sizeof(one), cudaMemcpyHostToDevice, S.st));
    int iters = 0;
    double rel = 0.0;
    st = S.solve(o->tol, o->max_iter, &iters, &rel);
    double resid = -1.0;
    if (S.err == cudaSuccess) {
        // |M x - b| / |x| of the returned vector
        S.matvec(S.x, S.wv);
        count_launch();
        ss_residual_kernel<<<S.grid(S.N), 256, 0, S.st>>>(S.N, S.b, S.wv);
        S.chk(cudaGetLastError());
        const double rn = S.norm(S.wv), xn = S.norm(S.x);
        resid = xn > 0.0 ? rn / xn : rn;
        S.chk(cudaMemcpyAsync(rho_out, S.x, vb, cudaMemcpyDeviceToHost, S.st));
    }
    int tc_fail = 0;
    if (S.mixed && S.err == cudaSuccess)
        S.chk(cudaMemcpyAsync(&tc_fail, S.tc_err, sizeof(int), cudaMemcpyDeviceToHost, S.st));
    S.chk(cudaFreeAsync(buf, S.st));
    S.chk(cudaStreamSynchronize(S.st));
    csr_free(S.L1);
    if (S.err != cudaSuccess) {
        set_cuda_error(S.err);
        return QTL_ECUDA;
    }
    if (tc_fail) return QTL_ECUDA;
    if (stats) {
        stats->iterations = iters;
        stats->pad = 0;
        stats->residual = resid;
        stats->cond_v = s.ss->cond;
        stats->gmres_residual = rel;
    }
    return st;
}

static qtl_status check_ss_opts(const qtl_ss_opts* o) {
    if (!o || !(o->tol > 0.0) || o->restart < 1 || o->restart > 512 || o->max_iter < 1) return QTL_EINVAL;
    if (o->precision != QTL_FP64 && o->precision != QTL_MIXED) return QTL_EINVAL;
    return QTL_OK;
}

}  // namespace qtl

using namespace qtl;

extern "C" {

void qtl_ss_opts_default(qtl_ss_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-12;
    o->restart = 60;
    o->max_iter = 20000;
    o->cuda_stream = nullptr;
    o->precision = QTL_FP64;
}

qtl_status qtl_steadystate(qtl_system* sys, const qtl_ss_opts* opts, qtl_c128* rho_out, qtl_ss_stats* stats) {
    if (!sys || !rho_out) return QTL_EINVAL;
    qtl_status st = check_ss_opts(opts);
    if (st != QTL_OK) return st;
    System& s = sys->s;
    if (s.n > QTL_SS_MAX_N || !s.Htd.empty()) return s.n > QTL_SS_MAX_N ? QTL_ETOOBIG : QTL_EINVAL;
    return ss_run(s, 1, 0.0, nullptr, opts, rho_out, stats);
}

qtl_status qtl_steadystate_fourier(qtl_system* sys, const qtl_op* X, double F, double omega, int32_t nmax,
                                   const qtl_ss_opts* opts, qtl_c128* rho_out, qtl_ss_stats* stats) {
    if (!sys || !rho_out || !X || nmax < 0 || nmax > 64 || !std::isfinite(F) || !std::isfinite(omega))
        return QTL_EINVAL;
    qtl_status st = check_ss_opts(opts);
    if (st != QTL_OK) return st;
    System& s = sys->s;
    if (s.n > QTL_SS_MAX_N) return QTL_ETOOBIG;
    if (!s.Htd.empty()) return QTL_EINVAL;
    Csr Xc;
    if ((st = op_to_csr(X, s.n, Xc)) != QTL_OK) return st;
    // L1 = -i (I kron X' - X'^T kron I), X' = (F/2) X, column stacking
    const int n = s.n;
    const long long N2 = (long long)n * n;
    if (N2 * (2 * nmax + 1) > (1ll << 31) - 1) return QTL_ETOOBIG;
    std::vector<std::vector<std::pair<int32_t, cd>>> rows((size_t)N2);
    const double h = 0.5 * F;
    for (int j = 0; j < n; ++j)          // I kron X': block (j, j) = X'
        for (int r = 0; r < n; ++r)
            for (int p = Xc.rp[r]; p < Xc.rp[r + 1]; ++p)
                rows[(size_t)r + (size_t)n * j].emplace_back(Xc.ci[p] + n * j,
                                                            cd(0.0, -1.0) * h * cd(Xc.re[p], Xc.im[p]));
    for (int r = 0; r < n; ++r)          // X'^T kron I: entry (c, r) of X'^T is X'(r, c)
        for (int p = Xc.rp[r]; p < Xc.rp[r + 1]; ++p) {
            const int c = Xc.ci[p];
            const cd v = cd(0.0, 1.0) * h * cd(Xc.re[p], Xc.im[p]);
            for (int i = 0; i < n; ++i) rows[(size_t)i + (size_t)n * c].emplace_back(i + n * r, v);
        }
    Csr L1;
    L1.n = (int)N2;
    L1.rp.assign((size_t)N2 + 1, 0);
    for (long long r = 0; r < N2; ++r) {
        auto& rw = rows[(size_t)r];
        std::sort(rw.begin(), rw.end(), [](const std::pair<int32_t, cd>& a, const std::pair<int32_t, cd>& b) {
            return a.first < b.first;
        });
        for (size_t q = 0; q < rw.size(); ++q) {
            if (q + 1 < rw.size() && rw[q + 1].first == rw[q].first) {
                rw[q + 1].second += rw[q].second;
                continue;
            }
            if (rw[q].second == cd(0.0)) continue;
            L1.ci.push_back(rw[q].first);
            L1.re.push_back(rw[q].second.real());
            L1.im.push_back(rw[q].second.imag());
        }
        L1.rp[(size_t)r + 1] = (int32_t)L1.ci.size();
    }
    return ss_run(s, 2 * nmax + 1, omega, &L1, opts, rho_out, stats);
}

}  // extern "C"
