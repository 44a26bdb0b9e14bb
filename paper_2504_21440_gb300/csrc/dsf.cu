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
