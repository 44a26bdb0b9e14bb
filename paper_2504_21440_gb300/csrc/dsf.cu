// Dynamical shifted Fock master equation (Sec. 3.6; Appendix B, Algorithm 1)
// on the GPU: the density matrix is kept in a frame displaced by a tracked
// coherence alpha_k for each DSF mode, so that a small Fock cutoff describes
// the fluctuations around a large coherent amplitude.
//
// At every time of tlist (the check interval of Algorithm 1 is tlist's
// spacing):
//   1. the master equation is integrated from the previous time by the
//      mesolve kernels of this library, on the system built for the current
//      coherences (H, collapse operators and observables as functions of
//      a_k + alpha_k I, built by the caller's callback);
//   2. the observables are recorded (before this time's displacement);
//   3. for each mode, d_k = Tr(rho a_k) is taken on the device; when
//      |d_k| > threshold the state is displaced, rho <- D rho D^H with
//      D = exp(-d_k a_k^H + conj(d_k) a_k) (the truncated-space exponential,
//      formed on the device by scaling and squaring of its Taylor series with
//      dense complex GEMMs), alpha_k += d_k, and the system is rebuilt.
// The state stays on the device from start to end; only d_k (one complex
// number per mode and time) and the expectation values come back to the
// host, which orders the rare displacement and rebuild events.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace qtl {

using cd = std::complex<double>;

// out = Tr(A rho) = sum_i sum_j A_ij rho_ji for A in CSR (one block)
__global__ void dsf_trace_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double2* __restrict__ v, const double2* __restrict__ rho,
                                 double2* __restrict__ out) {
    __shared__ double2 red[256];
    double2 s = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            const double2 a = v[p], r = rho[(long long)ci[p] + (long long)n * i];
            s.x += a.x * r.x - a.y * r.y;
            s.y += a.x * r.y + a.y * r.x;
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
    if (threadIdx.x == 0) *out = red[0];
}

// rho = psi psi^H (column-major)
__global__ void dsf_outer_kernel(int n, const double2* __restrict__ psi, double2* __restrict__ rho) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    const double2 a = psi[i], b = psi[j];
    rho[e] = make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// E = id * I + c T (c, id real; T may alias E)
__global__ void dsf_id_axpy_kernel(int n, double id, double c, const double2* T, double2* E) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    const double2 t = T[e];
    E[e] = make_double2((i == j ? id : 0.0) + c * t.x, c * t.y);
}

// DSF on trajectories: out[j * stride] = <psi_j|A|psi_j> / <psi_j|psi_j>
// for every trajectory j (one block of 128 threads each), A in CSR
__global__ void dsf_traj_trace_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      const double2* __restrict__ v, const double2* __restrict__ psi,
                                      double2* __restrict__ out, int stride) {
    __shared__ double rr[128], ri[128], rn[128];
    const double2* p = psi + (size_t)blockIdx.x * n;
    double sr = 0.0, si = 0.0, sn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double ax = 0.0, ay = 0.0;
        for (int q = rp[i]; q < rp[i + 1]; ++q) {
            const double2 a = v[q], x = p[ci[q]];
            ax += a.x * x.x - a.y * x.y;
            ay += a.x * x.y + a.y * x.x;
        }
        const double2 y = p[i];
        sr += y.x * ax + y.y * ay;   // conj(psi_i) (A psi)_i
        si += y.x * ay - y.y * ax;
        sn += y.x * y.x + y.y * y.y;
    }
    rr[threadIdx.x] = sr;
    ri[threadIdx.x] = si;
    rn[threadIdx.x] = sn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            rr[threadIdx.x] += rr[threadIdx.x + o];
            ri[threadIdx.x] += ri[threadIdx.x + o];
            rn[threadIdx.x] += rn[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)blockIdx.x * stride] = make_double2(rr[0] / rn[0], ri[0] / rn[0]);
}

// DSF on trajectories: psi_j <- exp(X) psi_j with X = -d a^H + conj(d) a for
// the listed trajectories (block b: trajectory traj[b], shift dv[b]), by the
// Taylor series of degree 18 of X / s applied s = reps[b] times; the host
// picks s with ||X||_1 / s <= 1/2, which puts the truncation below 1e-19.
// a and a^H in CSR; n <= 4 * blockDim.x; dynamic shared memory 3 n complex.
constexpr int DSF_DT = 256;
__global__ void __launch_bounds__(DSF_DT) dsf_traj_displace_kernel(
    int n, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, const double2* __restrict__ av,
    const int32_t* __restrict__ hrp, const int32_t* __restrict__ hci, const double2* __restrict__ hv,
    const int* __restrict__ traj, const double2* __restrict__ dv, const int* __restrict__ reps,
    double2* __restrict__ psi) {
    extern __shared__ double2 dsf_sm[];
    double2* x = dsf_sm;
    double2* t = dsf_sm + n;
    double2* u = dsf_sm + 2 * n;
    double2* p = psi + (size_t)traj[blockIdx.x] * n;
    const double2 d = dv[blockIdx.x];
    const int s = reps[blockIdx.x];
    const double2 cm = make_double2(-d.x / s, -d.y / s);   // -d / s      (times a^H)
    const double2 cp = make_double2(d.x / s, -d.y / s);    // conj(d) / s (times a)
    for (int i = threadIdx.x; i < n; i += DSF_DT) x[i] = p[i];
    __syncthreads();
    for (int rep = 0; rep < s; ++rep) {
        double2 acc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int i = threadIdx.x + m * DSF_DT;
            if (i < n) {
                acc[m] = x[i];
                t[i] = x[i];
            }
        }
        __syncthreads();
        for (int k = 1; k <= 18; ++k) {
            const double inv = 1.0 / k;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int i = threadIdx.x + m * DSF_DT;
                if (i >= n) continue;
                double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
                for (int q = arp[i]; q < arp[i + 1]; ++q) {
                    const double2 a = av[q], w = t[aci[q]];
                    ax += a.x * w.x - a.y * w.y;
                    ay += a.x * w.y + a.y * w.x;
                }
                for (int q = hrp[i]; q < hrp[i + 1]; ++q) {
                    const double2 a = hv[q], w = t[hci[q]];
                    bx += a.x * w.x - a.y * w.y;
                    by += a.x * w.y + a.y * w.x;
                }
                // (X t)_i / k = (cp (a t)_i + cm (a^H t)_i) / k
                const double2 z = make_double2((cp.x * ax - cp.y * ay + cm.x * bx - cm.y * by) * inv,
                                               (cp.x * ay + cp.y * ax + cm.x * by + cm.y * bx) * inv);
                u[i] = z;
                acc[m].x += z.x;
                acc[m].y += z.y;
            }
            __syncthreads();
            double2* w = t;
            t = u;
            u = w;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int i = threadIdx.x + m * DSF_DT;
            if (i < n) x[i] = acc[m];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += DSF_DT) p[i] = x[i];
}

// DSF on trajectories, operators from the polynomial fit: for the listed
// trajectories (blockIdx.y), vals[traj][p] = sum_i mu[b][i] coef[i][p] over
// all w entries (A, then C and O stacked), and the FP32 copy of A's entries
__global__ void dsf_assemble_kernel(int M, long long w, long long nnzA, const int* __restrict__ traj,
                                    const double2* __restrict__ mu, const double2* __restrict__ coef,
                                    double2* __restrict__ vals, float2* __restrict__ vals32) {
    const int b = blockIdx.y;
    const size_t j = (size_t)traj[b];
    const double2* u = mu + (size_t)b * M;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < w;
         p += (long long)gridDim.x * blockDim.x) {
        double vx = 0.0, vy = 0.0;
        for (int i = 0; i < M; ++i) {
            const double2 c = coef[(size_t)i * w + p], m = u[i];
            vx += m.x * c.x - m.y * c.y;
            vy += m.x * c.y + m.y * c.x;
        }
        vals[j * w + p] = make_double2(vx, vy);
        if (p < nnzA) vals32[j * nnzA + p] = make_float2((float)vx, (float)vy);
    }
}

namespace {

struct Dsf {
    int n = 0;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaSuccess;
    void chk(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    unsigned grid(long long c) const { return (unsigned)((c + 255) / 256); }
    void id_axpy(double id, double c, const double2* T, double2* E) {
        count_launch();
        dsf_id_axpy_kernel<<<grid((long long)n * n), 256, 0, st>>>(n, id, c, T, E);
        chk(cudaGetLastError());
    }

    // D = exp(X) for the dense X (device; overwritten with X / 2^s): the
    // Taylor series of degree 18 of X / 2^s by Horner's rule, then s
    // squarings; ||X||_1 / 2^s <= 1/2 puts the truncation below 1e-19.
    // D, T scratch of n^2 each; the result is in *D on return.
    void expm(double2* X, double xnorm1, double2*& D, double2*& T) {
        int s = 0;
        while (xnorm1 > 0.5 * std::ldexp(1.0, s) && s < 60) ++s;
        id_axpy(0.0, std::ldexp(1.0, -s), X, X);   // Y = X / 2^s
        const int q = 18;
        id_axpy(1.0, 1.0 / q, X, D);               // E = I + Y / q
        for (int j = q - 1; j >= 1; --j) {
            chk(launch_zgemm(n, X, 0, D, 0, T, st));   // T = Y E
            id_axpy(1.0, 1.0 / j, T, D);               // E = I + T / j
        }
        for (int k = 0; k < s; ++k) {
            chk(launch_zgemm(n, D, 0, D, 0, T, st));   // E <- E E
            std::swap(D, T);
        }
    }
};

}  // namespace

}  // namespace qtl

using namespace qtl;

extern "C" qtl_status qtl_dsf_mesolve(qtl_dsf_build_fn build, void* user, int32_t n_modes,
                                      const qtl_op* modes, const qtl_c128* alpha0, const qtl_c128* state0,
                                      int32_t is_ket, const double* tlist, int32_t nt, double threshold,
                                      const qtl_opts* opts, int32_t n_e, qtl_c128* expect_out,
                                      qtl_c128* alpha_out, int32_t* shifts, qtl_stats* stats) {
    if (!build || n_modes < 1 || n_modes > 16 || !modes || !alpha0 || !state0 || !tlist || nt < 1 ||
        !(threshold > 0.0) || n_e < 0 || (n_e > 0 && !expect_out) || !opts)
        return QTL_EINVAL;
    qtl_status st = validate_opts(opts);
    if (st != QTL_OK) return st;
    for (int i = 1; i < nt; ++i)
        if (!(tlist[i] >= tlist[i - 1]) || !std::isfinite(tlist[i])) return QTL_EINVAL;
    const int n = modes[0].n;
    if (n < 1 || n > 46340) return QTL_EINVAL;
    std::vector<Csr> mh(n_modes);
    for (int k = 0; k < n_modes; ++k)
        if ((st = op_to_csr(&modes[k], n, mh[k])) != QTL_OK) return st;
    Dsf Z;
    Z.n = n;
    Z.st = (cudaStream_t)opts->cuda_stream;
    const size_t n2 = (size_t)n * n, mb = n2 * sizeof(double2);
    std::vector<DevCsr> md(n_modes);
    char* buf = nullptr;
    qtl_system* sys = nullptr;
    qtl_status out_st = QTL_OK;
    auto fail = [&](qtl_status s2) {
        if (out_st == QTL_OK) out_st = s2;
    };
    for (int k = 0; k < n_modes && out_st == QTL_OK; ++k)
        if ((st = csr_upload(mh[k], md[k])) != QTL_OK) fail(st);
    const size_t bytes = 7 * ((mb + 255) & ~(size_t)255) + 4096 + (size_t)(n_e + 1) * 2 * sizeof(double2) * 2;
    if (out_st == QTL_OK && qtl_malloc_async((void**)&buf, bytes, Z.st) != cudaSuccess) {
        cudaGetLastError();
        fail(QTL_ENOMEM);
    }
    std::vector<cd> alpha(n_modes);
    for (int k = 0; k < n_modes; ++k) alpha[k] = cd(alpha0[k].re, alpha0[k].im);
    int nshift = 0;
    qtl_stats acc{};
    if (out_st == QTL_OK) {
        size_t off = 0;
        auto carve = [&](size_t b) {
            char* p = buf + off;
            off = (off + b + 255) & ~(size_t)255;
            return p;
        };
        double2* rho = (double2*)carve(mb);
        double2* states = (double2*)carve(2 * mb);
        double2* Xd = (double2*)carve(mb);
        double2* Da = (double2*)carve(mb);
        double2* Ta = (double2*)carve(mb);
        double2* ex = (double2*)carve((size_t)(n_e + 1) * 2 * sizeof(double2));
        double2* tr = (double2*)carve(sizeof(double2));
        double* tl2 = (double*)carve(2 * sizeof(double));
        qtl_device_info* info = (qtl_device_info*)carve(sizeof(qtl_device_info));
        // rho0 on the device
        if (is_ket) {
            Z.chk(cudaMemcpyAsync(Ta, state0, (size_t)n * sizeof(double2), cudaMemcpyHostToDevice, Z.st));
            count_launch();
            dsf_outer_kernel<<<Z.grid((long long)n2), 256, 0, Z.st>>>(n, Ta, rho);
            Z.chk(cudaGetLastError());
        } else {
            Z.chk(cudaMemcpyAsync(rho, state0, mb, cudaMemcpyHostToDevice, Z.st));
        }
        std::vector<qtl_c128> exh((size_t)n_e * 2);
        // one solve on the current system: the state at t1 into rho, the
        // observables at t1 into column idx (nt1 = 1: only the observables at t0)
        auto solve = [&](double t0, double t1, int nt1, int idx) -> bool {
            double th[2] = {t0, t1};
            Z.chk(cudaMemcpyAsync(tl2, th, 2 * sizeof(double), cudaMemcpyHostToDevice, Z.st));
            qtl_opts o = *opts;
            o.shadow_fp64 = 0;
            qtl_status s2 = qtl_mesolve_async(sys, (const qtl_c128*)rho, 0, tl2, nt1, &o, (qtl_c128*)ex,
                                              nt1 == 2 ? (qtl_c128*)states : nullptr, info);
            if (s2 != QTL_OK) {
                fail(s2);
                return false;
            }
            qtl_device_info hi{};
            Z.chk(cudaMemcpyAsync(&hi, info, sizeof(hi), cudaMemcpyDeviceToHost, Z.st));
            if (n_e > 0)
                Z.chk(cudaMemcpyAsync(exh.data(), ex, (size_t)n_e * nt1 * sizeof(double2), cudaMemcpyDeviceToHost,
                                      Z.st));
            Z.chk(cudaStreamSynchronize(Z.st));
            if (Z.err != cudaSuccess) return false;
            if (hi.status != QTL_OK) {
                fail((qtl_status)hi.status);
                return false;
            }
            acc.steps_acc += hi.steps_acc;
            acc.steps_rej += hi.steps_rej;
            acc.rhs_evals += hi.rhs_evals;
            for (int k = 0; k < n_e; ++k) expect_out[(size_t)k * nt + idx] = exh[(size_t)k * nt1 + (nt1 - 1)];
            if (nt1 == 2) Z.chk(cudaMemcpyAsync(rho, states + n2, mb, cudaMemcpyDeviceToDevice, Z.st));
            return true;
        };
        auto rebuild = [&]() -> bool {
            if (sys) qtl_system_free(sys);
            sys = nullptr;
            std::vector<qtl_c128> a(n_modes);
            for (int k = 0; k < n_modes; ++k) a[k] = {alpha[k].real(), alpha[k].imag()};
            qtl_status s2 = build(a.data(), n_modes, user, &sys);
            if (s2 != QTL_OK || !sys) {
                fail(s2 != QTL_OK ? s2 : QTL_EINVAL);
                return false;
            }
            if (sys->s.n != n || sys->s.n_e != n_e || !sys->s.Htd.empty()) {
                fail(QTL_EINVAL);
                return false;
            }
            return true;
        };
        bool ok = rebuild() && solve(tlist[0], tlist[0], 1, 0);
        std::vector<double2> Xh(n2);
        for (int idx = 0; ok && idx < nt; ++idx) {
            if (idx > 0 && !solve(tlist[idx - 1], tlist[idx], 2, idx)) break;
            bool changed = false;
            for (int k = 0; k < n_modes; ++k) {
                const Csr& a = mh[k];
                count_launch();
                dsf_trace_kernel<<<1, 256, 0, Z.st>>>(n, md[k].rp, md[k].ci, md[k].v64, rho, tr);
                Z.chk(cudaGetLastError());
                double2 dh;
                Z.chk(cudaMemcpyAsync(&dh, tr, sizeof(dh), cudaMemcpyDeviceToHost, Z.st));
                Z.chk(cudaStreamSynchronize(Z.st));
                if (Z.err != cudaSuccess) break;
                const cd d(dh.x, dh.y);
                if (std::abs(d) > threshold) {
                    // X = -d a^H + conj(d) a, dense, and its 1-norm
                    std::fill(Xh.begin(), Xh.end(), make_double2(0.0, 0.0));
                    for (int r = 0; r < n; ++r)
                        for (int p = a.rp[r]; p < a.rp[r + 1]; ++p) {
                            const cd v(a.re[p], a.im[p]);
                            const int c = a.ci[p];
                            const cd u = std::conj(d) * v;             // conj(d) a at (r, c)
                            const cd w = -d * std::conj(v);            // -d a^H at (c, r)
                            double2& x1 = Xh[(size_t)r + (size_t)n * c];
                            x1.x += u.real();
                            x1.y += u.imag();
                            double2& x2 = Xh[(size_t)c + (size_t)n * r];
                            x2.x += w.real();
                            x2.y += w.imag();
                        }
                    double x1n = 0.0;
                    for (int c = 0; c < n; ++c) {
                        double col = 0.0;
                        for (int r = 0; r < n; ++r) col += std::hypot(Xh[(size_t)r + (size_t)n * c].x,
                                                                      Xh[(size_t)r + (size_t)n * c].y);
                        x1n = std::max(x1n, col);
                    }
                    Z.chk(cudaMemcpyAsync(Xd, Xh.data(), mb, cudaMemcpyHostToDevice, Z.st));
                    double2 *D = Da, *T = Ta;
                    Z.expm(Xd, x1n, D, T);
                    // rho <- D rho D^H
                    Z.chk(launch_zgemm(n, D, 0, rho, 0, T, Z.st));
                    Z.chk(launch_zgemm(n, T, 0, D, 1, rho, Z.st));
                    Z.chk(cudaStreamSynchronize(Z.st));   // Xh is reused next
                    alpha[k] += d;
                    ++nshift;
                    changed = true;
                }
            }
            if (Z.err != cudaSuccess) break;
            if (alpha_out)
                for (int k = 0; k < n_modes; ++k)
                    alpha_out[(size_t)k * nt + idx] = {alpha[k].real(), alpha[k].imag()};
            if (changed && !rebuild()) break;
        }
        Z.chk(cudaFreeAsync(buf, Z.st));
        Z.chk(cudaStreamSynchronize(Z.st));
    }
    if (sys) qtl_system_free(sys);
    for (auto& d : md) csr_free(d);
    if (Z.err != cudaSuccess) {
        set_cuda_error(Z.err);
        fail(QTL_ECUDA);
    }
    if (shifts) *shifts = nshift;
    if (stats) {
        *stats = acc;
        stats->jumps = 0;
        stats->err_vs_fp64 = opts->precision == QTL_FP64 ? 0.0 : -1.0;
    }
    return out_st;
}

// ---- DSF on quantum trajectories (Sec. 3.6 applies Algorithm 1 to both
// solvers) ---------------------------------------------------------------
// Every trajectory carries its own frame alpha^(j).  Per interval of tlist
// one launch of the trajectory kernel integrates all trajectories, each with
// the operators of its own frame (a table of device pointers into its
// system), from its own ket, Philox stream and jump threshold, which the
// kernel writes back at the interval's end.  At each time of tlist the
// observables are recorded, <a_k> is taken per trajectory on the device, and
// the trajectories whose |<a_k>| exceeds the threshold are displaced there
// (psi <- exp(-d a_k^H + conj(d) a_k) psi); the host then rebuilds their
// systems through the caller's callback.  Until its first displacement a
// trajectory uses the system built for alpha0, shared by all.
namespace {

double csr_norm1(const Csr& a, int n) {
    std::vector<double> col(n, 0.0);
    for (int r = 0; r < n; ++r)
        for (int p = a.rp[r]; p < a.rp[r + 1]; ++p) col[a.ci[p]] += std::hypot(a.re[p], a.im[p]);
    return n > 0 ? *std::max_element(col.begin(), col.end()) : 0.0;
}

// conjugate transpose of a (n x n CSR)
void csr_adjoint(const Csr& a, int n, Csr& h) {
    std::vector<std::vector<std::pair<int32_t, cd>>> rows(n);
    for (int r = 0; r < n; ++r)
        for (int p = a.rp[r]; p < a.rp[r + 1]; ++p) rows[a.ci[p]].emplace_back(r, std::conj(cd(a.re[p], a.im[p])));
    h.n = n;
    h.rp.assign(n + 1, 0);
    h.ci.clear();
    h.re.clear();
    h.im.clear();
    for (int r = 0; r < n; ++r) {
        std::sort(rows[r].begin(), rows[r].end(),
                  [](const std::pair<int32_t, cd>& x, const std::pair<int32_t, cd>& y) { return x.first < y.first; });
        for (const auto& e : rows[r]) {
            h.ci.push_back(e.first);
            h.re.push_back(e.second.real());
            h.im.push_back(e.second.imag());
        }
        h.rp[r + 1] = (int32_t)h.ci.size();
    }
}

// ---- the operators of a frame as polynomials of the frame ----
// The operators for the frame alpha are built from a_k + alpha_k I by sums
// and products, so every entry of A = -i H_eff, of each C_k and of each O_e
// is a polynomial in the alpha_k and their conjugates.  With z = alpha / R
// (R bounds the frames in use), the host samples the callback at M random
// frames (|z_k| in [1/2, 1]), M the number of monomials in (z, conj z) of
// total degree <= D, and solves one M x M complex system for the
// coefficients of all entries; D = 1, 2, ... 6 is accepted when the fit
// reproduces the callback at three further frames (|z| = 0.1, 0.5, 0.95) to
// 1e-10 of the largest entry.  A displacement then rebuilds a trajectory's
// operators on the device as sum_m mu_m(z) M_m.
struct Pattern {
    int rows = 0;
    std::vector<int32_t> rp, ci;
    int64_t nnz() const { return (int64_t)ci.size(); }
};

struct PolyFit {
    int m = 0, D = 0, M = 0;          // modes, degree, monomials
    double R = 1.0;
    std::vector<int> ex;              // [M][2m] exponents of z_1..z_m, conj z_1..conj z_m
    Pattern pA, pC, pO;               // union patterns: A (n rows), C and O stacked
    std::vector<cd> coef;             // [M][nnzA + nnzC + nnzO]
    int64_t nnz() const { return pA.nnz() + pC.nnz() + pO.nnz(); }
    void mu(const cd* alpha, cd* out) const {
        std::vector<cd> z(m), zc(m);
        for (int k = 0; k < m; ++k) {
            z[k] = alpha[k] / R;
            zc[k] = std::conj(z[k]);
        }
        for (int i = 0; i < M; ++i) {
            cd v(1.0, 0.0);
            for (int k = 0; k < m; ++k) {
                for (int e = 0; e < ex[(size_t)i * 2 * m + k]; ++e) v *= z[k];
                for (int e = 0; e < ex[(size_t)i * 2 * m + m + k]; ++e) v *= zc[k];
            }
            out[i] = v;
        }
    }
};

// exponent vectors of total degree <= D over v variables, graded order
void monomials(int v, int D, std::vector<int>& out, int& M) {
    out.clear();
    M = 0;
    std::vector<int> e(v, 0);
    for (int deg = 0; deg <= D; ++deg) {
        // all compositions of deg into v parts
        std::function<void(int, int)> rec = [&](int pos, int left) {
            if (pos == v - 1) {
                e[pos] = left;
                out.insert(out.end(), e.begin(), e.end());
                ++M;
                return;
            }
            for (int x = left; x >= 0; --x) {
                e[pos] = x;
                rec(pos + 1, left - x);
            }
        };
        rec(0, deg);
    }
}

// the union pattern of the operators of several systems
void union_pattern(const std::vector<const System*>& ss, int which, Pattern& P) {
    const int n = ss[0]->n;
    const int nops = which == 0 ? 1 : (which == 1 ? ss[0]->n_c : ss[0]->n_e);
    P.rows = nops * n;
    std::vector<std::vector<int32_t>> cols(P.rows);
    for (const System* s : ss)
        for (int k = 0; k < nops; ++k) {
            const Csr& c = which == 0 ? s->A : (which == 1 ? s->C[k] : s->O[k]);
            for (int r = 0; r < n; ++r)
                for (int p = c.rp[r]; p < c.rp[r + 1]; ++p) cols[(size_t)k * n + r].push_back(c.ci[p]);
        }
    P.rp.assign(P.rows + 1, 0);
    P.ci.clear();
    for (int r = 0; r < P.rows; ++r) {
        auto& c = cols[r];
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        P.ci.insert(P.ci.end(), c.begin(), c.end());
        P.rp[r + 1] = (int32_t)P.ci.size();
    }
}

// a system's entries on the pattern (zero where it has none); false if it
// has a nonzero entry outside the pattern
bool values_on(const System& s, int which, const Pattern& P, cd* out) {
    const int n = s.n;
    const int nops = which == 0 ? 1 : (which == 1 ? s.n_c : s.n_e);
    std::fill(out, out + P.nnz(), cd(0.0, 0.0));
    for (int k = 0; k < nops; ++k) {
        const Csr& c = which == 0 ? s.A : (which == 1 ? s.C[k] : s.O[k]);
        for (int r = 0; r < n; ++r) {
            const int row = k * n + r;
            const int32_t* b = P.ci.data() + P.rp[row];
            const int32_t* e = P.ci.data() + P.rp[row + 1];
            for (int p = c.rp[r]; p < c.rp[r + 1]; ++p) {
                const int32_t* f = std::lower_bound(b, e, c.ci[p]);
                const cd v(c.re[p], c.im[p]);
                if (f == e || *f != c.ci[p]) {
                    if (v != cd(0.0, 0.0)) return false;
                    continue;
                }
                out[P.rp[row] + (f - b)] += v;
            }
        }
    }
    return true;
}

// solve V X = B in place (V: M x M row-major, B: M x w row-major), LU with
// partial pivoting; false if singular
bool lu_solve(int M, std::vector<cd>& V, std::vector<cd>& B, size_t w) {
    for (int k = 0; k < M; ++k) {
        int p = k;
        for (int i = k + 1; i < M; ++i)
            if (std::abs(V[(size_t)i * M + k]) > std::abs(V[(size_t)p * M + k])) p = i;
        if (std::abs(V[(size_t)p * M + k]) == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < M; ++j) std::swap(V[(size_t)k * M + j], V[(size_t)p * M + j]);
            for (size_t j = 0; j < w; ++j) std::swap(B[(size_t)k * w + j], B[(size_t)p * w + j]);
        }
        const cd inv = 1.0 / V[(size_t)k * M + k];
        for (int i = k + 1; i < M; ++i) {
            const cd f = V[(size_t)i * M + k] * inv;
            if (f == cd(0.0, 0.0)) continue;
            for (int j = k; j < M; ++j) V[(size_t)i * M + j] -= f * V[(size_t)k * M + j];
            for (size_t j = 0; j < w; ++j) B[(size_t)i * w + j] -= f * B[(size_t)k * w + j];
        }
    }
    for (int i = M - 1; i >= 0; --i) {
        const cd inv = 1.0 / V[(size_t)i * M + i];
        for (size_t j = 0; j < w; ++j) {
            cd acc = B[(size_t)i * w + j];
            for (int l = i + 1; l < M; ++l) acc -= V[(size_t)i * M + l] * B[(size_t)l * w + j];
            B[(size_t)i * w + j] = acc * inv;
        }
    }
    return true;
}

McTrajOps ops_of(const System& s) {
    McTrajOps o;
    o.aseg = s.dA.seg;
    o.aci = s.dA.ci;
    o.av64 = s.dA.v64;
    o.av32 = s.dA.v32;
    o.crp = s.dC.rp;
    o.cci = s.dC.ci;
    o.cv = s.dC.v64;
    o.orp = s.dO.rp;
    o.oci = s.dO.ci;
    o.ov = s.dO.v64;
    return o;
}

}  // namespace

extern "C" qtl_status qtl_dsf_mcsolve(qtl_dsf_build_fn build, void* user, int32_t n_modes,
                                      const qtl_op* modes, const qtl_c128* alpha0, const qtl_c128* psi0,
                                      const double* tlist, int32_t nt, double threshold, int32_t ntraj,
                                      uint64_t seed, const qtl_opts* opts, int32_t n_e, qtl_c128* expect_out,
                                      qtl_c128* traj_expect_out, int64_t* shifts, qtl_stats* stats) {
    if (!build || n_modes < 1 || n_modes > 16 || !modes || !alpha0 || !psi0 || !tlist || nt < 1 ||
        !(threshold > 0.0) || ntraj < 1 || n_e < 0 || (n_e > 0 && !expect_out) || !opts)
        return QTL_EINVAL;
    qtl_status st = validate_opts(opts);
    if (st != QTL_OK) return st;
    if (opts->engine == QTL_ENGINE_GRID) return QTL_EINVAL;   // per-trajectory operators: trajectory kernel only
    for (int i = 0; i < nt; ++i)
        if (!std::isfinite(tlist[i]) || (i > 0 && !(tlist[i] >= tlist[i - 1]))) return QTL_EINVAL;
    const int n = modes[0].n;
    if (n < 1) return QTL_EINVAL;
    if (n > mc_traj_capacity() || n > 4 * DSF_DT) return QTL_ETOOBIG;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(psi0[i].re) || !std::isfinite(psi0[i].im)) return QTL_EINVAL;
    std::vector<Csr> mh(n_modes), mhH(n_modes);
    std::vector<double> mnorm(n_modes);
    for (int k = 0; k < n_modes; ++k) {
        if ((st = op_to_csr(&modes[k], n, mh[k])) != QTL_OK) return st;
        csr_adjoint(mh[k], n, mhH[k]);
        mnorm[k] = csr_norm1(mh[k], n) + csr_norm1(mhH[k], n);
    }
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    };
    qtl_status out_st = QTL_OK;
    auto fail = [&](qtl_status s2) {
        if (out_st == QTL_OK) out_st = s2;
    };
    std::vector<DevCsr> md(n_modes), mdH(n_modes);
    for (int k = 0; k < n_modes && out_st == QTL_OK; ++k) {
        if ((st = csr_upload(mh[k], md[k])) != QTL_OK) fail(st);
        if (out_st == QTL_OK && (st = csr_upload(mhH[k], mdH[k])) != QTL_OK) fail(st);
    }
    // frames and systems: sys0 for alpha0, own[j] after trajectory j's first displacement
    std::vector<cd> alpha((size_t)ntraj * n_modes);
    for (int j = 0; j < ntraj; ++j)
        for (int k = 0; k < n_modes; ++k) alpha[(size_t)j * n_modes + k] = cd(alpha0[k].re, alpha0[k].im);
    qtl_system* sys0 = nullptr;
    std::vector<qtl_system*> own(ntraj, nullptr);
    int n_c = 0;
    auto make = [&](const cd* al, qtl_system** out) -> bool {
        std::vector<qtl_c128> a(n_modes);
        for (int k = 0; k < n_modes; ++k) a[k] = {al[k].real(), al[k].imag()};
        qtl_system* sy = nullptr;
        qtl_status s2 = build(a.data(), n_modes, user, &sy);
        if (s2 != QTL_OK || !sy) {
            if (sy) qtl_system_free(sy);
            fail(s2 != QTL_OK ? s2 : QTL_EINVAL);
            return false;
        }
        const System& s = sy->s;
        if (s.n != n || s.n_e != n_e || !s.Htd.empty() || (sys0 && s.n_c != n_c)) {
            qtl_system_free(sy);
            fail(QTL_EINVAL);
            return false;
        }
        *out = sy;
        return true;
    };
    if (out_st == QTL_OK && make(alpha.data(), &sys0)) n_c = sys0->s.n_c;
    // device buffers
    const size_t nx = (size_t)ntraj * n;
    char* buf = nullptr;
    const size_t bytes = nx * sizeof(double2) + (size_t)ntraj * sizeof(McTrajOps) + (size_t)ntraj * 4 +
                         (size_t)ntraj * 8 + (size_t)(n_e > 0 ? n_e : 1) * 2 * ntraj * sizeof(double2) +
                         (size_t)ntraj * n_modes * sizeof(double2) + 64 + sizeof(qtl_device_info) +
                         (size_t)ntraj * (4 + 16 + 4) + 12 * 256;
    if (out_st == QTL_OK && qtl_malloc_async((void**)&buf, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        fail(QTL_ENOMEM);
    }
    int64_t nshift = 0;
    qtl_stats acc{};
    if (out_st == QTL_OK) {
        size_t off = 0;
        auto carve = [&](size_t b) {
            char* p = buf + off;
            off = (off + b + 255) & ~(size_t)255;
            return p;
        };
        double2* psi = (double2*)carve(nx * sizeof(double2));
        McTrajOps* dtops = (McTrajOps*)carve((size_t)ntraj * sizeof(McTrajOps));
        unsigned* draw = (unsigned*)carve((size_t)ntraj * 4);
        double* rthr = (double*)carve((size_t)ntraj * 8);
        double2* texp = (double2*)carve((size_t)(n_e > 0 ? n_e : 1) * 2 * ntraj * sizeof(double2));
        double2* tr = (double2*)carve((size_t)ntraj * n_modes * sizeof(double2));
        double* tl2 = (double*)carve(2 * sizeof(double));
        qtl_device_info* info = (qtl_device_info*)carve(sizeof(qtl_device_info));
        int* ltraj = (int*)carve((size_t)ntraj * 4);
        double2* ld = (double2*)carve((size_t)ntraj * 16);
        int* lrep = (int*)carve((size_t)ntraj * 4);
        {
            std::vector<double2> h(nx);
            for (int j = 0; j < ntraj; ++j)
                for (int i = 0; i < n; ++i) h[(size_t)j * n + i] = make_double2(psi0[i].re, psi0[i].im);
            chk(cudaMemcpyAsync(psi, h.data(), nx * sizeof(double2), cudaMemcpyHostToDevice, stream));
            chk(cudaMemsetAsync(draw, 0, (size_t)ntraj * 4, stream));
            chk(cudaStreamSynchronize(stream));
        }
        std::vector<McTrajOps> hops(ntraj, ops_of(sys0->s));
        // ---- rebuilds on the device from the polynomial fit (QTL_DSF_REBUILD
        // = "callback" keeps the callback at every displacement) ----
        PolyFit F;
        bool poly = false;
        char* pb = nullptr;
        double2 *pvals = nullptr, *pmu = nullptr, *pcoef = nullptr;
        float2* pvals32 = nullptr;
        int* pidx = nullptr;
        std::vector<double2> hmu;
        std::vector<int> hidx;
        uint64_t rs = 0x2545F4914F6CDD1Dull;   // splitmix64 state of the sample frames
        auto uni = [&]() {
            rs += 0x9E3779B97F4A7C15ull;
            uint64_t z = rs;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            return (double)(z >> 11) * (1.0 / 9007199254740992.0);
        };
        // F for frames |alpha_k| <= R: false if no degree <= 6 fits (or a
        // build fails, which also sets the status)
        auto fit = [&](double R) -> bool {
            F.m = n_modes;
            F.R = R;
            for (int D = 1; D <= 6; ++D) {
                int M = 0;
                monomials(2 * n_modes, D, F.ex, M);
                if (M > 400) return false;
                F.D = D;
                F.M = M;
                std::vector<cd> al((size_t)(M + 3) * n_modes);
                for (int i = 0; i < M + 3; ++i)
                    for (int k = 0; k < n_modes; ++k) {
                        const double rad = i < M ? 0.5 + 0.5 * uni() : (i == M ? 0.1 : (i == M + 1 ? 0.5 : 0.95));
                        const double th = 6.283185307179586 * uni();
                        al[(size_t)i * n_modes + k] = R * rad * cd(std::cos(th), std::sin(th));
                    }
                std::vector<qtl_system*> built;
                auto cleanup = [&]() {
                    for (auto* b : built) qtl_system_free(b);
                };
                for (int i = 0; i < M + 3; ++i) {
                    qtl_system* sy = nullptr;
                    if (!make(&al[(size_t)i * n_modes], &sy)) {
                        cleanup();
                        return false;
                    }
                    built.push_back(sy);
                }
                std::vector<const System*> ss;
                for (int i = 0; i < M; ++i) ss.push_back(&built[i]->s);
                union_pattern(ss, 0, F.pA);
                union_pattern(ss, 1, F.pC);
                union_pattern(ss, 2, F.pO);
                const size_t w = (size_t)F.nnz(), nA = (size_t)F.pA.nnz(), nC = (size_t)F.pC.nnz();
                // no entries, or a fit too large for the host (M x w complex
                // coefficients above 5e7): the callback path
                if (w == 0 || (size_t)M * w > (size_t)50000000) {
                    cleanup();
                    return false;
                }
                auto fill = [&](const System& sy, cd* row) {
                    return values_on(sy, 0, F.pA, row) && values_on(sy, 1, F.pC, row + nA) &&
                           values_on(sy, 2, F.pO, row + nA + nC);
                };
                std::vector<cd> V((size_t)M * M), B((size_t)M * w);
                bool ok = true;
                for (int i = 0; i < M && ok; ++i) {
                    F.mu(&al[(size_t)i * n_modes], &V[(size_t)i * M]);
                    ok = fill(built[i]->s, &B[(size_t)i * w]);
                }
                ok = ok && lu_solve(M, V, B, w);
                if (ok) {
                    F.coef.swap(B);
                    std::vector<cd> mu(M), act(w);
                    for (int i = M; i < M + 3 && ok; ++i) {
                        F.mu(&al[(size_t)i * n_modes], mu.data());
                        ok = fill(built[i]->s, act.data());
                        double big = 1.0;
                        for (size_t q = 0; q < w; ++q) big = std::max(big, std::abs(act[q]));
                        for (size_t q = 0; q < w && ok; ++q) {
                            cd pr(0.0, 0.0);
                            for (int l = 0; l < M; ++l) pr += mu[l] * F.coef[(size_t)l * w + q];
                            if (!(std::abs(pr - act[q]) <= 1e-10 * big)) ok = false;
                        }
                    }
                }
                cleanup();
                if (ok) return true;
                if (out_st != QTL_OK) return false;
            }
            return false;
        };
        // operators of the listed trajectories from their frames (device)
        auto assemble = [&](const std::vector<int>& list) {
            const int M = F.M;
            const long long w = F.nnz(), nA = F.pA.nnz();
            for (size_t b0 = 0; b0 < list.size() && err == cudaSuccess; b0 += 65535) {
                const size_t cnt = std::min<size_t>(65535, list.size() - b0);
                hmu.resize(cnt * M);
                hidx.assign(list.begin() + b0, list.begin() + b0 + cnt);
                std::vector<cd> mu(M);
                for (size_t b = 0; b < cnt; ++b) {
                    F.mu(&alpha[(size_t)hidx[b] * n_modes], mu.data());
                    for (int i = 0; i < M; ++i) hmu[b * M + i] = make_double2(mu[i].real(), mu[i].imag());
                }
                chk(cudaMemcpyAsync(pidx, hidx.data(), cnt * 4, cudaMemcpyHostToDevice, stream));
                chk(cudaMemcpyAsync(pmu, hmu.data(), cnt * M * 16, cudaMemcpyHostToDevice, stream));
                const unsigned gx = (unsigned)std::min<long long>((w + 255) / 256, 64);
                count_launch();
                dsf_assemble_kernel<<<dim3(gx, (unsigned)cnt), 256, 0, stream>>>(M, w, nA, pidx, pmu, pcoef, pvals,
                                                                               pvals32);
                chk(cudaGetLastError());
                chk(cudaStreamSynchronize(stream));   // host staging reused
            }
        };
        // device copy of F, and every trajectory's operators; false: no room
        auto poly_setup = [&]() -> bool {
            if (pb) chk(cudaFreeAsync(pb, stream));
            pb = nullptr;
            const size_t w = (size_t)F.nnz(), nA = (size_t)F.pA.nnz(), nC = (size_t)F.pC.nnz(), M = F.M;
            const size_t rA = F.pA.rows, rC = F.pC.rows, rO = F.pO.rows;
            auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
            const size_t bytes = up((rA + 1) * 4) + up(nA * 4) + up(rA * 16) + up((rC + 1) * 4) + up(nC * 4 + 4) +
                                 up((rO + 1) * 4) + up((w - nA - nC) * 4 + 4) + up(M * w * 16) +
                                 up((size_t)ntraj * w * 16) + up((size_t)ntraj * nA * 8) + up(65535 * M * 16) +
                                 up(65535 * 4);
            if (bytes > ((size_t)16 << 30) || qtl_malloc_async((void**)&pb, bytes, stream) != cudaSuccess) {
                cudaGetLastError();
                pb = nullptr;
                return false;
            }
            size_t o = 0;
            auto cv = [&](size_t b) {
                char* q = pb + o;
                o += up(b);
                return q;
            };
            int32_t* rpA = (int32_t*)cv((rA + 1) * 4);
            int32_t* ciA = (int32_t*)cv(nA * 4);
            int4* segA = (int4*)cv(rA * 16);
            int32_t* rpC = (int32_t*)cv((rC + 1) * 4);
            int32_t* ciC = (int32_t*)cv(nC * 4 + 4);
            int32_t* rpO = (int32_t*)cv((rO + 1) * 4);
            int32_t* ciO = (int32_t*)cv((w - nA - nC) * 4 + 4);
            pcoef = (double2*)cv(M * w * 16);
            pvals = (double2*)cv((size_t)ntraj * w * 16);
            pvals32 = (float2*)cv((size_t)ntraj * nA * 8);
            pmu = (double2*)cv(65535 * M * 16);
            pidx = (int*)cv(65535 * 4);
            std::vector<int4> seg(rA);
            for (size_t r = 0; r < rA; ++r) seg[r] = make_int4(F.pA.rp[r], F.pA.rp[r], F.pA.rp[r], F.pA.rp[r + 1]);
            std::vector<double2> hc(M * w);
            for (size_t q = 0; q < M * w; ++q) hc[q] = make_double2(F.coef[q].real(), F.coef[q].imag());
            chk(cudaMemcpyAsync(rpA, F.pA.rp.data(), (rA + 1) * 4, cudaMemcpyHostToDevice, stream));
            if (nA) chk(cudaMemcpyAsync(ciA, F.pA.ci.data(), nA * 4, cudaMemcpyHostToDevice, stream));
            chk(cudaMemcpyAsync(segA, seg.data(), rA * 16, cudaMemcpyHostToDevice, stream));
            chk(cudaMemcpyAsync(rpC, F.pC.rp.data(), (rC + 1) * 4, cudaMemcpyHostToDevice, stream));
            if (nC) chk(cudaMemcpyAsync(ciC, F.pC.ci.data(), nC * 4, cudaMemcpyHostToDevice, stream));
            chk(cudaMemcpyAsync(rpO, F.pO.rp.data(), (rO + 1) * 4, cudaMemcpyHostToDevice, stream));
            if (w - nA - nC)
                chk(cudaMemcpyAsync(ciO, F.pO.ci.data(), (w - nA - nC) * 4, cudaMemcpyHostToDevice, stream));
            chk(cudaMemcpyAsync(pcoef, hc.data(), M * w * 16, cudaMemcpyHostToDevice, stream));
            chk(cudaStreamSynchronize(stream));
            for (int j = 0; j < ntraj; ++j) {
                double2* vj = pvals + (size_t)j * w;
                hops[j] = McTrajOps{segA, ciA, vj, pvals32 + (size_t)j * nA, rpC, ciC, vj + nA, rpO, ciO, vj + nA + nC};
            }
            std::vector<int> all(ntraj);
            for (int j = 0; j < ntraj; ++j) all[j] = j;
            assemble(all);
            return err == cudaSuccess;
        };
        auto frame_max = [&]() {
            double a = 0.0;
            for (const cd& x : alpha) a = std::max(a, std::abs(x));
            return a;
        };
        {
            const char* env = std::getenv("QTL_DSF_REBUILD");
            if (!(env && !std::strcmp(env, "callback"))) {
                poly = fit(std::max(8.0, 2.0 * frame_max())) && poly_setup();
                if (out_st != QTL_OK) poly = false;
            }
        }
        std::vector<double2> hexp((size_t)(n_e > 0 ? n_e : 1) * 2 * ntraj), htr((size_t)ntraj * n_modes);
        // one launch over [t0, t1] (ntl = 2) or the observables at t0 (ntl = 1);
        // records the observables at the last time into column idx
        auto run = [&](double t0, double t1, int ntl, int idx) -> bool {
            const double th[2] = {t0, t1};
            chk(cudaMemcpyAsync(tl2, th, sizeof(th), cudaMemcpyHostToDevice, stream));
            chk(cudaMemcpyAsync(dtops, hops.data(), (size_t)ntraj * sizeof(McTrajOps), cudaMemcpyHostToDevice,
                                stream));
            chk(cudaMemsetAsync(info, 0, sizeof(qtl_device_info), stream));
            const System& s0 = sys0->s;
            McJob J;
            std::memset(&J, 0, sizeof(J));
            J.n = n;
            J.aseg = s0.dA.seg;
            J.arp = s0.dA.rp;
            J.aci = s0.dA.ci;
            J.av64 = s0.dA.v64;
            J.av32 = s0.dA.v32;
            J.a_nnz = (int)s0.dA.nnz;
            J.n_c = n_c;
            J.n_e = n_e;
            J.tops = dtops;
            J.psi0 = psi;
            J.psi0_stride = n;
            J.psi_out = psi;
            J.rng_draw = draw;
            J.rng_r = rthr;
            J.tlist = tl2;
            J.nt = ntl;
            J.ntraj = ntraj;
            J.seed = seed;
            J.traj_expect = texp;
            J.info = info;
            J.rtol = opts->rtol;
            J.atol = opts->atol;
            J.dt0 = opts->dt0;
            J.dt_min = opts->dt_min;
            J.dt_fixed = opts->dt_fixed;
            J.max_steps = opts->max_steps;
            J.fixed = opts->fixed_step ? 1 : 0;
            J.method = opts->method;
            if (err == cudaSuccess) chk(launch_mc_traj(J, opts->precision, stream));
            for (int k = 0; k < n_modes && err == cudaSuccess; ++k) {
                count_launch();
                dsf_traj_trace_kernel<<<ntraj, 128, 0, stream>>>(n, md[k].rp, md[k].ci, md[k].v64, psi, tr + k,
                                                                  n_modes);
                chk(cudaGetLastError());
            }
            qtl_device_info hi{};
            chk(cudaMemcpyAsync(&hi, info, sizeof(hi), cudaMemcpyDeviceToHost, stream));
            if (n_e > 0)
                chk(cudaMemcpyAsync(hexp.data(), texp, (size_t)n_e * ntl * ntraj * sizeof(double2),
                                    cudaMemcpyDeviceToHost, stream));
            chk(cudaMemcpyAsync(htr.data(), tr, (size_t)ntraj * n_modes * sizeof(double2), cudaMemcpyDeviceToHost,
                                stream));
            chk(cudaStreamSynchronize(stream));
            if (err != cudaSuccess) return false;
            if (hi.status != QTL_OK) {
                fail((qtl_status)hi.status);
                return false;
            }
            acc.steps_acc += hi.steps_acc;
            acc.steps_rej += hi.steps_rej;
            acc.rhs_evals += hi.rhs_evals;
            acc.jumps += hi.jumps;
            // traj_expect layout of the kernel: [(e * ntl + t) * ntraj + j]
            for (int e = 0; e < n_e; ++e) {
                double sx = 0.0, sy = 0.0;
                for (int j = 0; j < ntraj; ++j) {
                    const double2 v = hexp[((size_t)e * ntl + (ntl - 1)) * ntraj + j];
                    sx += v.x;
                    sy += v.y;
                    if (traj_expect_out) traj_expect_out[((size_t)j * n_e + e) * nt + idx] = {v.x, v.y};
                }
                expect_out[(size_t)e * nt + idx] = {sx / ntraj, sy / ntraj};
            }
            return true;
        };
        // displace the trajectories whose |<a_k>| exceeds the threshold, mode
        // by mode (the modes commute, so <a_k> taken before any of this
        // time's displacements is the same), then rebuild their systems
        std::vector<int> hj;
        std::vector<double2> hd;
        std::vector<int> hr;
        auto displace = [&]() -> bool {
            std::vector<char> moved(ntraj, 0);
            for (int k = 0; k < n_modes; ++k) {
                hj.clear();
                hd.clear();
                hr.clear();
                for (int j = 0; j < ntraj; ++j) {
                    const double2 v = htr[(size_t)j * n_modes + k];
                    const cd d(v.x, v.y);
                    if (!(std::abs(d) > threshold)) continue;
                    hj.push_back(j);
                    hd.push_back(v);
                    hr.push_back(std::max(1, (int)std::ceil(2.0 * std::abs(d) * mnorm[k])));
                    alpha[(size_t)j * n_modes + k] += d;
                    moved[j] = 1;
                }
                if (hj.empty()) continue;
                nshift += (int64_t)hj.size();
                const size_t m = hj.size();
                chk(cudaMemcpyAsync(ltraj, hj.data(), m * 4, cudaMemcpyHostToDevice, stream));
                chk(cudaMemcpyAsync(ld, hd.data(), m * 16, cudaMemcpyHostToDevice, stream));
                chk(cudaMemcpyAsync(lrep, hr.data(), m * 4, cudaMemcpyHostToDevice, stream));
                count_launch();
                dsf_traj_displace_kernel<<<(unsigned)m, DSF_DT, 3 * (size_t)n * sizeof(double2), stream>>>(
                    n, md[k].rp, md[k].ci, md[k].v64, mdH[k].rp, mdH[k].ci, mdH[k].v64, ltraj, ld, lrep, psi);
                chk(cudaGetLastError());
                chk(cudaStreamSynchronize(stream));   // the host lists are reused
                if (err != cudaSuccess) return false;
            }
            if (poly) {
                std::vector<int> list;
                for (int j = 0; j < ntraj; ++j)
                    if (moved[j]) list.push_back(j);
                if (list.empty()) return true;
                const double amax = frame_max();
                if (amax <= F.R) {
                    assemble(list);
                    return err == cudaSuccess;
                }
                // a frame left the fitted range: fit again over twice the
                // largest frame and rebuild every trajectory's operators
                if (fit(2.0 * amax) && poly_setup()) return true;
                if (out_st != QTL_OK || err != cudaSuccess) return false;
                // no fit: every trajectory from the callback from here on
                poly = false;
                for (int j = 0; j < ntraj; ++j) moved[j] = 1;
            }
            for (int j = 0; j < ntraj; ++j) {
                if (!moved[j]) continue;
                qtl_system* sy = nullptr;
                if (!make(&alpha[(size_t)j * n_modes], &sy)) return false;
                if (own[j]) qtl_system_free(own[j]);
                own[j] = sy;
                hops[j] = ops_of(sy->s);
            }
            return true;
        };
        bool ok = out_st == QTL_OK && run(tlist[0], tlist[0], 1, 0) && displace();
        for (int idx = 1; ok && idx < nt; ++idx) ok = run(tlist[idx - 1], tlist[idx], 2, idx) && displace();
        if (pb) chk(cudaFreeAsync(pb, stream));
        chk(cudaFreeAsync(buf, stream));
        chk(cudaStreamSynchronize(stream));
    }
    for (auto* sy : own)
        if (sy) qtl_system_free(sy);
    if (sys0) qtl_system_free(sys0);
    for (auto& d : md) csr_free(d);
    for (auto& d : mdH) csr_free(d);
    if (err != cudaSuccess) {
        set_cuda_error(err);
        fail(QTL_ECUDA);
    }
    if (shifts) *shifts = nshift;
    if (stats) {
        *stats = acc;
        stats->err_vs_fp64 = opts->precision == QTL_FP64 ? 0.0 : -1.0;
    }
    return out_st;
}
