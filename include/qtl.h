/*
 * qtl.h -- C ABI of the GB300 Lindblad / quantum-trajectory solver library.
 *
 * The library integrates
 *   - the Lindblad master equation (paper Sec. 3.2, the equation for d rho/dt
 *     and the Lindblad dissipator D[C] rho = C rho C^dag - 1/2 {C^dag C, rho}),
 *     with expectation values Tr(O_k rho(t)) at the times of tlist (Sec. 3.1,
 *     sol.expect), and
 *   - the Monte-Carlo wave-function method (Sec. 3.3: evolution under
 *     H_eff = H - i/2 sum_k C_k^dag C_k, a jump when the squared norm falls
 *     below a uniform threshold, channel k drawn with weight |C_k psi|^2),
 * with an adaptive embedded Runge-Kutta 5(4) pair (Dormand-Prince 1980 or
 * Tsitouras 2011) and a PI step-size controller.  The paper leaves the
 * integrator to DifferentialEquations.jl (Sec. 2); the readings fixed here,
 * implemented identically by the test oracle, are: the error norm
 * sqrt(mean_i |e_i|^2 / sc_i^2) over complex entries with
 * sc_i = atol + rtol max(|y_i|, |y_new,i|); a PI controller with factor
 * clamp(0.9 err^-0.14 err_prev^0.08, 0.2, 10) on accept (at most 1 right after
 * a reject, err_prev floored at 1e-4) and max(0.2, 0.9 err^-0.2) on reject;
 * the Hairer-Norsett-Wanner starting step; steps clamped to land exactly on
 * each time of tlist.
 *
 * Conventions for every entry point:
 *   - complex numbers are interleaved {re, im} FP64 (qtl_c128);
 *   - dense matrices are column-major; a density matrix is passed as its
 *     column-stacked vector vec(rho)[i + n*j] = rho[i][j];
 *   - the caller owns every buffer it passes; inputs are copied (system
 *     creation) or only read; outputs are caller-allocated;
 *   - errors are returned as qtl_status; nothing aborts the process.  A
 *     solve that cannot finish (step-size underflow, max_steps, a non-finite
 *     error estimate) returns QTL_ESTEP and leaves the outputs it had not
 *     reached untouched.
 *   - functions ending in _async take DEVICE pointers, enqueue the work on
 *     opts->cuda_stream and return at once; the status and counters of the
 *     solve are written to the caller's device-resident qtl_device_info when
 *     the work completes.  All other entry points take HOST pointers and
 *     return when the results are in the caller's buffers.
 */
#ifndef QTL_H
#define QTL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double re, im;
} qtl_c128;

typedef enum {
    QTL_OK = 0,
    QTL_EINVAL = 1,   /* malformed argument (CSR structure, sizes, NaN/Inf, tlist order) */
    QTL_ENOMEM = 2,   /* device allocation failed or an HBM budget would be exceeded */
    QTL_ESTEP = 3,    /* step size below dt_min, max_steps reached, or non-finite error */
    QTL_ECUDA = 4,    /* CUDA runtime error (message via qtl_last_cuda_error) */
    QTL_ECANCEL = 5,  /* request cancelled */
    QTL_EBUSY = 6,    /* result not ready yet */
    QTL_ETOOBIG = 7   /* problem size outside what the selected kernel supports */
} qtl_status;

/* One operator: CSR (is_csr = 1: row_ptr[n+1], col_idx[nnz], vals[nnz], rows
 * sorted or not, duplicates summed) or dense (is_csr = 0: vals[n*n]
 * column-major; row_ptr/col_idx ignored).  Exact zeros are dropped. */
typedef struct {
    int32_t n;
    int32_t is_csr;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const qtl_c128* vals;
} qtl_op;

enum { QTL_DP5 = 0, QTL_TSIT5 = 1 };
enum { QTL_FP64 = 0, QTL_MIXED = 1 };

/* Solver options.
 *   method    QTL_DP5 | QTL_TSIT5
 *   precision QTL_FP64: every operation in FP64.
 *             QTL_MIXED: right-hand side and stage sums in FP32 (complex64
 *             operator copies), state y and its update, error-norm
 *             reduction, controller, jump logic and renormalisation in FP64.
 *   rtol, atol    error-norm tolerances (rtol > 0, atol >= 0)
 *   dt0           starting step; 0 selects the Hairer-Norsett-Wanner heuristic
 *   dt_min        a rejected step that would shrink below dt_min fails (QTL_ESTEP)
 *   max_steps     attempted steps per solve (per trajectory for mcsolve)
 *   fixed_step    1: every step has size min(dt_fixed, time to the next
 *                 tlist point) and is accepted without error control
 *   cuda_stream   cudaStream_t to run on; NULL = the legacy default stream
 *   engine        mesolve kernel: QTL_ENGINE_AUTO (cluster kernel when n*n and
 *                 the Liouvillian fit one 16-CTA cluster, else the grid
 *                 kernel), QTL_ENGINE_CLUSTER (CSR Liouvillian in one thread-
 *                 block cluster; QTL_ETOOBIG if it does not fit) or
 *                 QTL_ENGINE_GRID (product form A rho + rho B + sum C rho C^dag
 *                 over a cooperative grid; no Liouvillian is formed).
 *                 mcsolve: AUTO (trajectory state in registers up to n = 1024,
 *                 else in global memory), CLUSTER (registers; QTL_ETOOBIG
 *                 above n = 1024) or GRID (global memory at any n)
 *   shadow_fp64   0 or 1.  With QTL_MIXED, 1 makes the host-pointer calls
 *                 qtl_mesolve and qtl_mcsolve, and server requests, run the
 *                 same solve a second time with precision QTL_FP64 (all other
 *                 options equal, the same seed) and report the largest
 *                 |difference| of their expectation values in
 *                 qtl_stats.err_vs_fp64: the reduced-precision result's error
 *                 against FP64, per result.  It roughly doubles the call's
 *                 cost.  Ignored by the _async calls, batches and plans. */
enum { QTL_ENGINE_AUTO = 0, QTL_ENGINE_CLUSTER = 1, QTL_ENGINE_GRID = 2 };
typedef struct {
    int32_t method;
    int32_t precision;
    double rtol;
    double atol;
    double dt0;
    double dt_min;
    int64_t max_steps;
    int32_t fixed_step;
    int32_t cluster_size; /* mesolve: CTAs per solve (0 = automatic, 1..16) */
    double dt_fixed;
    void* cuda_stream;
    int32_t engine;
    int32_t shadow_fp64;
} qtl_opts;

/* Counters of one solve (summed over trajectories for mcsolve), and
 * err_vs_fp64: max over observables and times of |expect - expect_FP64| for
 * a QTL_MIXED solve run with opts.shadow_fp64 = 1 (for mcsolve the FP64
 * trajectories use the same random draws, so the difference also holds the
 * rare trajectories whose jump decisions the FP32 rounding moved); 0 for a
 * QTL_FP64 solve; -1 when not computed (QTL_MIXED without the shadow, or a
 * shadow solve that failed). */
typedef struct {
    int64_t steps_acc;
    int64_t steps_rej;
    int64_t rhs_evals;
    int64_t jumps;
    double err_vs_fp64;
} qtl_stats;

/* Device-resident status of an _async solve: status is a qtl_status. */
typedef struct {
    int32_t status;
    int32_t pad;
    int64_t steps_acc;
    int64_t steps_rej;
    int64_t rhs_evals;
    int64_t jumps;
} qtl_device_info;

typedef struct qtl_system qtl_system;

/* Fills opts with the defaults: Tsit5, FP64, rtol 1e-8, atol 1e-10, automatic
 * dt0, dt_min 0, max_steps 10^7, adaptive, automatic cluster size, default stream. */
void qtl_opts_default(qtl_opts* opts);

/* Builds a system (paper Sec. 3.2 / 3.3 inputs: H, c_ops, e_ops) on the
 * current CUDA device.  The operators are copied; the caller may free them on
 * return.  All operators must have the same dimension n: 1 <= n <= 4,194,304
 * for CSR operators, n <= 46340 for dense ones.  mesolve needs n <= 46340
 * (QTL_ETOOBIG above); mcsolve takes the full range.
 * The library forms, in FP64 on the host:
 *   A = -i H - 1/2 sum_k C_k^dag C_k   (so -i H_eff psi = A psi, Sec. 3.3),
 *   B =  i H - 1/2 sum_k C_k^dag C_k,
 *   L = I kron A + B^T kron I + sum_k conj(C_k) kron C_k  (column stacking,
 *       the Liouvillian of Sec. 3.2; built on first use by a mesolve),
 * and uploads FP64 and complex64 copies to device memory.
 * Errors: QTL_EINVAL (bad structure, mismatched n, NaN/Inf, n_c or n_e < 0 or
 * > 64), QTL_ENOMEM, QTL_ECUDA.  *out is NULL on error. */
qtl_status qtl_system_create(const qtl_op* H, const qtl_op* c_ops, int32_t n_c,
                             const qtl_op* e_ops, int32_t n_e, qtl_system** out);

/* Time-dependent Hamiltonians (Sec. 2, QobjEvo: H(t) = H0 + sum_k f_k(t) H_k;
 * the drive F cos(w_d t)(a + a^dag) of Sec. 3.4; the complex pair
 * A e^{i w t} a + conj(.) a^dag of Sec. 5).  A coefficient is
 *   f(t) = (amp_re + i amp_im) * env(t) * g(omega t + phi),
 *   g = cos for QTL_COEF_COS, exp(i .) for QTL_COEF_EXP,
 *   env(t) = exp(-(t - t0)^2 / (2 sigma^2)) if sigma > 0, else 1,
 * evaluated in FP64 at every stage time of the integrator. */
typedef enum { QTL_COEF_COS = 0, QTL_COEF_EXP = 1 } qtl_coef_kind;
typedef struct {
    int32_t kind;
    double amp_re, amp_im, omega, phi, t0, sigma;
} qtl_coef;

/* Adds the term f(t) Hk to the system's Hamiltonian (H of qtl_system_create
 * becomes H0).  Up to 8 terms; Hk has the system's dimension.
 * Terms must be added before the system's first solve (QTL_EINVAL after).
 * Which solvers take them: qtl_sesolve (n <= 1024) and qtl_mcsolve
 * (trajectories, A(t) = A - i sum_k f_k(t) H_k: FP64 or mixed precision up to
 * n = 1024, FP64 above, where mixed precision returns QTL_EINVAL), and
 * qtl_mesolve / qtl_mesolve_async in FP64 on either engine (the cluster
 * kernel adds f_k(t) L_k y with L_k = -i (I kron H_k - H_k^T kron I); the
 * grid kernel adds f_k(t) ((-i H_k) rho + rho (i H_k)) and integrates only
 * the lower triangle of rho when H0 and every H_k are exactly Hermitian and
 * every f_k is real, QTL_COEF_COS with amp_im = 0), and in mixed precision
 * on the cluster kernel (the products L_k y of each step's state in FP64,
 * the stage increments' products in FP32), also inside batches and batch
 * plans.  Mixed-precision mesolve on the grid kernel returns QTL_EINVAL for
 * such a system.
 * Errors: QTL_EINVAL (NULL, bad operator or coefficient, 8 terms already,
 * a solve already ran or a request on the system was submitted to a
 * server), QTL_ENOMEM (the system keeps its earlier terms), QTL_ECUDA. */
qtl_status qtl_system_add_td(qtl_system* sys, const qtl_op* Hk, const qtl_coef* f);

/* Releases the system and its device memory (NULL is a no-op).  Work enqueued
 * by _async calls on the system must have completed. */
void qtl_system_free(qtl_system* sys);

/* Hilbert dimension, and the number of stored entries of the Liouvillian
 * (0 before a mesolve has built it). */
int32_t qtl_system_dim(const qtl_system* sys);
int64_t qtl_system_liouvillian_nnz(const qtl_system* sys);

/* Stored entries of one of the system's operators: which = 0 for H, 1 for
 * A = -i H_eff (the trajectory right-hand side), 2 for the Liouvillian (0
 * before it is built); 3 and 4 count those of A and of the Liouvillian whose
 * real or imaginary part is zero (a product with such an entry takes 4 flops
 * instead of 8).  -1 for a NULL system or an unknown `which`. */
int64_t qtl_system_nnz(const qtl_system* sys, int32_t which);

/* mesolve (Sec. 3.2): integrates d rho/dt = L rho from tlist[0].
 *   state0    is_ket = 1: psi0[n] (rho0 = |psi0><psi0|, ket2dm);
 *             is_ket = 0: vec(rho0)[n*n] column-major.
 *   tlist[nt] non-decreasing, finite, nt >= 1; steps land exactly on each time.
 *   expect_out[n_e*nt] (row k = e_op k): Tr(O_k rho(tlist[t])); may be NULL if n_e = 0.
 *   states_out NULL, or [nt*n*n]: vec(rho(tlist[t])) for each t.
 *   stats      NULL or filled.
 * Host pointers; returns when done.  The cluster kernel takes n*n up to
 * 16384 (and a Liouvillian whose rows fit each CTA's shared memory); larger
 * problems run on the grid kernel (opts->engine). */
qtl_status qtl_mesolve(qtl_system* sys, const qtl_c128* state0, int32_t is_ket,
                       const double* tlist, int32_t nt, const qtl_opts* opts,
                       qtl_c128* expect_out, qtl_c128* states_out, qtl_stats* stats);

/* Same as qtl_mesolve with device pointers, enqueued on opts->cuda_stream.
 * Scratch is taken stream-ordered from a memory pool that the library owns
 * on each device (freed blocks stay cached in it, up to 16 GiB) and
 * returned on the same stream.  Argument errors found on the host are
 * returned directly; errors found by the kernel (tlist order, step failure)
 * land in info->status. */
qtl_status qtl_mesolve_async(qtl_system* sys, const qtl_c128* state0_dev, int32_t is_ket,
                             const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                             qtl_c128* expect_dev, qtl_c128* states_dev,
                             qtl_device_info* info_dev);

/* Batched mesolve for parameter sweeps (Sec. 3.2 applied to nb independent
 * systems): nb solves sharing tlist and opts, each with its own system and
 * initial state.  Each system gets the launch plan its own size implies --
 * the smallest cluster C in {1, 2, 4, 8, 16} with C*1024 >= n^2, and the
 * fewest rows per thread that cover n^2 with that C -- so a solve's
 * arithmetic, and its result bit for bit, does not depend on what else is in
 * the batch; it equals qtl_mesolve with opts->cluster_size = that C.  Solves
 * with the same plan share one launch (clusters take solves dynamically,
 * largest first); different plans run concurrently on streams forked from
 * opts->cuda_stream and joined back into it.  opts->cluster_size is ignored.
 * Systems with time-dependent terms are taken, in FP64 and in mixed
 * precision (scratch for their FP64 products L_k y is allocated per solve).
 *   _async: state0_dev[b], expect_dev[b] are device pointers held in host
 *   arrays of nb entries; is_ket[b] host array; info_dev a device array of nb
 *   qtl_device_info.  Host form: the same with host pointers, stats[b] (or
 *   NULL), returning the first failing solve's status. */
qtl_status qtl_mesolve_batch_async(qtl_system* const* systems, int32_t nb,
                                   const qtl_c128* const* state0_dev, const int32_t* is_ket,
                                   const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                                   qtl_c128* const* expect_dev, qtl_device_info* info_dev);
qtl_status qtl_mesolve_batch(qtl_system* const* systems, int32_t nb, const qtl_c128* const* state0,
                             const int32_t* is_ket, const double* tlist, int32_t nt,
                             const qtl_opts* opts, qtl_c128* const* expect_out, qtl_stats* stats);

/* sesolve (Sec. 3.1): d psi/dt = -i H(t) psi from psi0[n] for a system
 * without collapse operators (QTL_EINVAL otherwise), n <= 1024: the
 * trajectory kernel with one trajectory, which never jumps.
 *   expect_out[n_e*nt]: <psi|O_k|psi>/<psi|psi> at each time of tlist.
 * Host pointers; returns when done; opts as for qtl_mcsolve. */
qtl_status qtl_sesolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt,
                       const qtl_opts* opts, qtl_c128* expect_out, qtl_stats* stats);

/* ssesolve (Sec. 3.5): the stochastic Schroedinger equation under homodyne
 * detection, in Ito form d psi = -i K psi dt + sum_n M_n psi dW_n with
 * K = H + i sum_n (e_n/2 S_n - 1/2 S_n^dag S_n - e_n^2/8), M_n = S_n - e_n/2,
 * e_n = <psi|S_n + S_n^dag|psi>; the homodyne current is J_n = e_n + dW_n/dt.
 * The system's collapse operators are the stochastic operators S_n (1 to 4);
 * time-dependent terms are not taken (QTL_EINVAL).  n <= 1024 (QTL_ETOOBIG).
 * Integration: Euler-Maruyama with the fixed step opts->dt_fixed
 * (opts->fixed_step must be 1, precision FP64; else QTL_EINVAL), each step
 * clamped to land on tlist, the state renormalised after every step.
 * dW_n = sqrt(h) z with z standard normal by the Box-Muller transform of
 * draws 2j and 2j + 1 (j = step * n_sc + n) of trajectory j's Philox stream
 * (counter (draw, trajectory, 0, 0), key from seed); trajectories 0..ntraj-1.
 *   expect_out[n_e*nt]: trajectory mean of <psi|O_k|psi>/<psi|psi>;
 *   meas_out[n_c*nt]:   trajectory mean of J_n of the last step ending at or
 *                       before each time (e_n(psi0) at tlist[0]).
 *   traj_expect_out, traj_meas_out: NULL, or the per-trajectory values,
 *                       [n_e*nt*ntraj] and [n_c*nt*ntraj] laid out
 *                       [(k*nt + t)*ntraj + j] as for qtl_mcsolve.
 * Host pointers; returns when done; stats->steps_acc = steps over all
 * trajectories.  QTL_ESTEP, before any work, when (tlist[nt-1] - tlist[0]) /
 * dt_fixed exceeds opts->max_steps (a trajectory's step count). */
qtl_status qtl_ssesolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt,
                        int32_t ntraj, uint64_t seed, const qtl_opts* opts, qtl_c128* expect_out,
                        double* meas_out, qtl_stats* stats, qtl_c128* traj_expect_out,
                        double* traj_meas_out);

/* smesolve (Sec. 3.5): the stochastic master equation under homodyne
 * detection, in Ito form
 *   d rho = -i[H, rho] dt + sum_i D[C_i] rho dt + sum_n D[S_n] rho dt
 *           + sum_n H[S_n] rho dW_n,
 *   H[S] rho = S rho + rho S^dag - Tr(S rho + rho S^dag) rho,
 * with homodyne currents J_n = Tr(S_n rho + rho S_n^dag) + dW_n/dt.  The
 * system's last n_sc collapse operators (1 to 4) are the measured S_n, the
 * others the unmeasured C_i.  rho0 = |psi0><psi0|; n*n <= 4096
 * (QTL_ETOOBIG); time-dependent terms are not taken (QTL_EINVAL).
 * Integration as qtl_ssesolve (Euler-Maruyama with the fixed step
 * opts->dt_fixed, FP64, the same Wiener increments and step budget), without
 * renormalisation (the scheme keeps Tr rho = 1 up to rounding).
 *   expect_out[n_e*nt]: trajectory mean of Tr(O_k rho);
 *   meas_out[n_sc*nt]:  trajectory mean of J_n, recorded as in qtl_ssesolve;
 *   traj_expect_out, traj_meas_out: NULL or per trajectory, as in qtl_ssesolve. */
qtl_status qtl_smesolve(qtl_system* sys, int32_t n_sc, const qtl_c128* psi0, const double* tlist, int32_t nt,
                        int32_t ntraj, uint64_t seed, const qtl_opts* opts, qtl_c128* expect_out,
                        double* meas_out, qtl_stats* stats, qtl_c128* traj_expect_out,
                        double* traj_meas_out);

/* Reusable batch plan (Sec. 3.2 over nb independent systems, as
 * qtl_mesolve_batch_async), built once and replayed.
 *   qtl_batch_create: the same arguments as qtl_mesolve_batch_async (device
 *     pointers, which the plan keeps: each launch reads state0_dev[b] and
 *     tlist_dev and writes expect_dev[b] and info_dev[b] as they are then)
 *     plus autotune.  Systems are grouped by the launch plan their size
 *     implies.  autotune = 1: for every group with more than one feasible
 *     cluster size among C/2, C, 2C, 4C, each candidate integrates the
 *     group's own solves over the first 5% of tlist's span (two output times,
 *     outputs into the plan's scratch) once to warm up and once timed with
 *     CUDA events on opts->cuda_stream, and the fastest is kept.  The job
 *     table is built on the device, and the launch sequence (status reset,
 *     one cluster launch per group on a stream of the plan's own, the join)
 *     is captured once in a CUDA graph.  Blocks until the plan is ready.
 *     The systems and device buffers must outlive the plan.  Returns
 *     QTL_ETOOBIG if a group does not fit the cluster kernel, QTL_ENOMEM if
 *     the plan's scratch cannot be allocated, QTL_ECUDA on a CUDA error.
 *   qtl_batch_launch: replays the graph on cuda_stream (a cudaStream_t of the
 *     device the plan was created on; else QTL_EINVAL).  Launches on one plan
 *     share its scratch, so they must not overlap: enqueue them on one
 *     stream.  A solve's result equals qtl_mesolve with opts->cluster_size =
 *     its group's cluster size.
 *   qtl_batch_groups / qtl_batch_group_info: number of groups; for group k
 *     its cluster size, number of solves, and the autotuner's candidates
 *     (ncand, cand_cluster[ncand], cand_ms[ncand]: probe time in ms; ncand =
 *     0 when not tuned).  Output pointers may be NULL.
 *   qtl_batch_group_of: the group of system index sys (-1 if out of range).
 *   qtl_batch_free: releases the plan (NULL is a no-op). */
typedef struct qtl_batch qtl_batch;
qtl_status qtl_batch_create(qtl_system* const* systems, int32_t nb, const qtl_c128* const* state0_dev,
                            const int32_t* is_ket, const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                            qtl_c128* const* expect_dev, qtl_device_info* info_dev, int32_t autotune,
                            qtl_batch** out);
qtl_status qtl_batch_launch(qtl_batch* b, void* cuda_stream);
int32_t qtl_batch_groups(const qtl_batch* b);
qtl_status qtl_batch_group_info(const qtl_batch* b, int32_t k, int32_t* cluster_size, int32_t* nsolves,
                                int32_t* ncand, int32_t* cand_cluster, double* cand_ms);
int32_t qtl_batch_group_of(const qtl_batch* b, int32_t sys);
void qtl_batch_free(qtl_batch* b);

/* mcsolve (Sec. 3.3): ntraj trajectories from the ket psi0[n].
 *   seed      64-bit key of the per-trajectory Philox4x32-10 streams: draw d
 *             of trajectory j uses counter (d, traj_offset + j, 0, 0) and key
 *             (seed & 0xffffffff, seed >> 32); draws alternate threshold,
 *             channel, threshold, ...
 *   expect_out[n_e*nt]: the trajectory mean of <psi|O_k|psi>/<psi|psi>.
 *   traj_expect_out NULL, or [n_e*nt*ntraj] laid out [(k*nt + t)*ntraj + j].
 * Host pointers; returns when done.  Up to n = 1024 a trajectory's state
 * stays in the registers of one CTA; larger n (up to 4,194,304) runs one
 * 1024-thread CTA per trajectory with its state in a stream-ordered scratch
 * buffer of about 13 * 16 * n bytes per resident CTA (one per SM), returning
 * QTL_ENOMEM if that cannot be allocated.  Both give the same trajectories
 * up to rounding order. */
qtl_status qtl_mcsolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt,
                       int32_t ntraj, uint64_t seed, int64_t traj_offset, const qtl_opts* opts,
                       qtl_c128* expect_out, qtl_c128* traj_expect_out, qtl_stats* stats);

/* Same with device pointers, enqueued on opts->cuda_stream (see
 * qtl_mesolve_async).  traj_expect_dev may be NULL (scratch is used). */
qtl_status qtl_mcsolve_async(qtl_system* sys, const qtl_c128* psi0_dev, const double* tlist_dev,
                             int32_t nt, int32_t ntraj, uint64_t seed, int64_t traj_offset,
                             const qtl_opts* opts, qtl_c128* expect_dev,
                             qtl_c128* traj_expect_dev, qtl_device_info* info_dev);

/* ------------------------------------------------------ stationary states ---
 * steadystate (Sec. 3.2): the density matrix with L vec(rho) = 0 and
 * Tr rho = 1.  steadystate_fourier (Appendix A): the Fourier components
 * rho_k, k = -nmax..nmax, of the periodic long-time state under
 * H(t) = H0 + F cos(omega t) X (H0 and the collapse operators are the
 * system's), from the block-tridiagonal system
 *   (L0 - i k omega) rho_k + L1 (rho_{k-1} + rho_{k+1}) = 0,
 *   L1 = -i [(F/2) X, .],  components beyond nmax taken as zero,
 * with Tr rho_0 = 1 in place of the first equation of the k = 0 block.
 * The paper solves these directly; here they are solved on the GPU by
 * flexible GMRES(restart) with classical Gram-Schmidt applied twice, right-
 * preconditioned by the inverse of the no-jump part of each diagonal block,
 * X -> A X + X A^H - i k omega X with A = -i H_eff, applied through the
 * eigendecomposition A = V diag(lambda) V^-1 (computed once per system on
 * the host in FP64, O(n^3): about a minute at n = 1024) as four dense
 * complex GEMMs per block.  Everything is FP64.
 *   rho_out: steadystate: vec(rho)[n*n] column-major; steadystate_fourier:
 *            [(2 nmax + 1) * n * n], block a = vec(rho_{a - nmax}).
 *   X: an operator of the system's dimension (CSR or dense); nmax <= 64.
 * n <= QTL_SS_MAX_N (QTL_ETOOBIG above); systems with time-dependent terms
 * are refused (QTL_EINVAL).  Host pointers; returns when done, on
 * opts->cuda_stream.  QTL_ESTEP when the GMRES residual |b - M x| / |b| has
 * not reached opts->tol within opts->max_iter preconditioned products (the
 * last iterate is still written), QTL_ESTEP too if the eigendecomposition
 * does not converge. */
#define QTL_SS_MAX_N 1024
typedef struct {
    double tol;          /* relative GMRES residual (default 1e-12) */
    int32_t restart;     /* Krylov vectors per cycle, 1..512 (default 60) */
    int32_t max_iter;    /* preconditioned matrix-vector products at most (default 20000) */
    void* cuda_stream;   /* cudaStream_t, NULL = the legacy default stream */
    int32_t precision;   /* QTL_FP64 (default): FP64 preconditioner GEMMs; QTL_MIXED: on the
                            tensor cores in split BF16 (qtl_zgemm_async), the Krylov
                            vectors, products with L and residuals staying FP64 */
    int32_t pad;
} qtl_ss_opts;
typedef struct {
    int32_t iterations;      /* preconditioned matrix-vector products */
    int32_t pad;
    double residual;         /* |M x - b|_2 / |x|_2 of the returned vector (M: the system with the trace row) */
    double cond_v;           /* ||V||_F ||V^-1||_F / n for the eigenvectors of A (1 for orthonormal V) */
    double gmres_residual;   /* |b - M x| / |b| at the last iteration */
} qtl_ss_stats;
void qtl_ss_opts_default(qtl_ss_opts* opts);
qtl_status qtl_steadystate(qtl_system* sys, const qtl_ss_opts* opts, qtl_c128* rho_out, qtl_ss_stats* stats);
qtl_status qtl_steadystate_fourier(qtl_system* sys, const qtl_op* X, double F, double omega, int32_t nmax,
                                   const qtl_ss_opts* opts, qtl_c128* rho_out, qtl_ss_stats* stats);

/* Dense complex matrix product C = op(A) op(B) of n x n matrices (device
 * pointers, column-major qtl_c128; op 0 = identity, 1 = conjugate
 * transpose), the building block of the stationary-state preconditioner
 * (no counterpart in the paper).  precision QTL_FP64: FP64 arithmetic.
 * QTL_MIXED: on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation)
 * with each entry split into two BF16 numbers and the three products
 * hi*hi + hi*lo + lo*hi, about 2^-16 of sum_k |a_ik||b_kj| per entry.
 * n <= 8192.  Enqueued on cuda_stream; scratch comes from the library's
 * pool.  err_dev (device int, QTL_MIXED only, not cleared here) is set to 1
 * if a wait inside the tensor-core kernel gave up (the result is then not
 * valid).  QTL_ECUDA also when the driver offers no tensor-map encoder. */
qtl_status qtl_zgemm_async(int32_t n, const qtl_c128* A, int32_t op_a, const qtl_c128* B, int32_t op_b,
                           qtl_c128* C, int32_t precision, void* cuda_stream, int32_t* err_dev);

/* ------------------------------------------- dynamical shifted Fock ---
 * dsf_mesolve (Sec. 3.6; Appendix B, Algorithm 1): the master equation in a
 * frame displaced by a tracked coherence alpha_k of each DSF mode, so that a
 * small Fock cutoff holds the fluctuations around a large coherent state.
 * The operators are functions of the shifted mode operators a_k + alpha_k I
 * (as in the paper, where H, c_ops and e_ops are functions of op_list): the
 * library calls build(alpha, n_modes, user, &sys) whenever alpha changes and
 * frees the system it returns; build creates it with qtl_system_create from
 * operators in which every a_k is replaced by a_k + alpha_k I, and returns
 * QTL_OK.
 * At every time of tlist (the check interval of Algorithm 1 is tlist's
 * spacing): the state is integrated from the previous time by qtl_mesolve's
 * kernels (opts as for qtl_mesolve; adaptive steps between checks), the
 * observables are recorded, then for each mode d_k = Tr(rho a_k) is
 * computed and, when |d_k| > threshold, rho <- D rho D^H with
 * D = exp(-d_k a_k^H + conj(d_k) a_k) exponentiated in the truncated space,
 * alpha_k += d_k, and the system is rebuilt.  The state stays on the device.
 *   modes[n_modes]   a_k on the full space (n x n), 1 <= n_modes <= 16
 *   alpha0[n_modes]  initial coherences; state0: ket (is_ket = 1, n entries)
 *                    or vec(rho0) (n*n), in the frame displaced by alpha0
 *   n_e              observables of the systems build returns (checked)
 *   expect_out[n_e*nt]   observables at each time (before that time's shift)
 *   alpha_out[n_modes*nt] (or NULL): alpha_k after each time's shift
 *   shifts (or NULL): number of displacements applied
 * Host pointers; returns when done.  Errors: QTL_EINVAL (arguments, a built
 * system of another dimension, observable count or with time-dependent
 * terms), build's own status, the solve's status (QTL_ESTEP), QTL_ENOMEM,
 * QTL_ECUDA. */
typedef qtl_status (*qtl_dsf_build_fn)(const qtl_c128* alpha, int32_t n_modes, void* user, qtl_system** out);
qtl_status qtl_dsf_mesolve(qtl_dsf_build_fn build, void* user, int32_t n_modes, const qtl_op* modes,
                           const qtl_c128* alpha0, const qtl_c128* state0, int32_t is_ket, const double* tlist,
                           int32_t nt, double threshold, const qtl_opts* opts, int32_t n_e, qtl_c128* expect_out,
                           qtl_c128* alpha_out, int32_t* shifts, qtl_stats* stats);

/* dsf_mcsolve (Sec. 3.6 applies Algorithm 1 of Appendix B to quantum
 * trajectories as well): the trajectories of qtl_mcsolve, each in its own
 * displaced frame alpha^(j).  Between the times of tlist every trajectory is
 * integrated (one launch of the trajectory kernel for all of them) with the
 * operators built for its own frame, its Philox stream (seed, trajectory
 * index j) and jump threshold carrying over from interval to interval, and
 * each interval starting with the starting-step heuristic.  At every time of
 * tlist the normalised observables are recorded, then for each mode
 * d_k = <psi|a_k|psi>/<psi|psi> of each trajectory and, when |d_k| >
 * threshold, psi <- exp(-d_k a_k^H + conj(d_k) a_k) psi (in the truncated
 * space, on the device), alpha_k^(j) += d_k, and the trajectory's system is
 * rebuilt (as for qtl_dsf_mesolve; until its first displacement a
 * trajectory uses the system built for alpha0).  Rebuilds run on the device:
 * at set-up the library calls build at sample frames and fits every entry of
 * the operators as a polynomial of degree <= 6 in alpha_k and conj(alpha_k),
 * accepted when it reproduces build at further frames to 1e-10 of the
 * largest entry (refitted over a wider range when a frame outgrows it).
 * Without such a fit, or with the environment variable
 * QTL_DSF_REBUILD=callback, build is called at every displacement.
 *   modes[n_modes]   a_k on the full space (n x n, n <= 1024), 1 <= n_modes <= 16
 *   alpha0, psi0     initial coherences and ket (n entries, in the frame of alpha0)
 *   ntraj, seed      trajectories 0..ntraj-1 of the Philox streams of seed
 *   opts             as for qtl_mcsolve; the grid engine is refused
 *   n_e              observables of the systems build returns (checked)
 *   expect_out[n_e*nt]             trajectory means (before each time's shift)
 *   traj_expect_out[ntraj*n_e*nt]  (or NULL) per trajectory, [j][e][t]
 *   shifts (or NULL): displacements applied, over all trajectories and modes
 * Host pointers; returns when done.  Errors: QTL_EINVAL (arguments, a built
 * system of another dimension, observable or collapse-operator count, or
 * with time-dependent terms), QTL_ETOOBIG (n > 1024), build's own status,
 * the solve's status (QTL_ESTEP), QTL_ENOMEM, QTL_ECUDA. */
qtl_status qtl_dsf_mcsolve(qtl_dsf_build_fn build, void* user, int32_t n_modes, const qtl_op* modes,
                           const qtl_c128* alpha0, const qtl_c128* psi0, const double* tlist, int32_t nt,
                           double threshold, int32_t ntraj, uint64_t seed, const qtl_opts* opts, int32_t n_e,
                           qtl_c128* expect_out, qtl_c128* traj_expect_out, int64_t* shifts, qtl_stats* stats);

/* ------------------------------------------------------------- serving ---
 * A request server (no counterpart in the paper; it serves the mesolve and
 * mcsolve calls above).  Requests are queued on submit and admitted in
 * arrival order while their estimated device memory fits the HBM budget;
 * each admitted request runs on its own CUDA stream, so requests that arrive
 * while others are on the GPU are admitted as memory frees up and their
 * kernels overlap.  A request whose kernel occupies every SM (mesolve on the
 * grid kernel, mcsolve above n = 1024) runs alone.  Continuous batching:
 * a mesolve request on the cluster kernel (automatic engine and cluster size,
 * no FP64 shadow) runs through qtl_mesolve_batch_async, and queued requests
 * with the same output times and options join its launch (up to 64).  Submit
 * builds the system's device structures for the request (on the caller's
 * thread) before queueing it.  Results are bit for bit those of the
 * corresponding call alone: qtl_mcsolve, qtl_mesolve, or for a batched
 * mesolve qtl_mesolve with opts->cluster_size set to its batch plan's
 * cluster size (each solve's arithmetic depends only on its own inputs).
 * The caller's host buffers (state0, tlist, expect_out) must stay valid
 * until the request is done; the system must outlive it. */
typedef struct qtl_server qtl_server;

enum { QTL_REQ_MESOLVE = 0, QTL_REQ_MCSOLVE = 1 };

typedef struct {
    int32_t kind;            /* QTL_REQ_MESOLVE | QTL_REQ_MCSOLVE */
    qtl_system* sys;
    const qtl_c128* state0;  /* host: ket (n) or, for mesolve with is_ket = 0, vec(rho0) */
    int32_t is_ket;
    const double* tlist;     /* host, nt entries */
    int32_t nt;
    int32_t ntraj;           /* mcsolve */
    uint64_t seed;           /* mcsolve */
    qtl_opts opts;           /* cuda_stream is ignored: the server owns its streams */
} qtl_request;

typedef struct {
    int32_t status;          /* qtl_status of the solve (QTL_EBUSY while running) */
    int32_t pad;
    qtl_stats stats;
    double t_submit;         /* seconds on a monotonic clock */
    double t_start;          /* admitted and enqueued */
    double t_end;            /* results in the caller's buffer */
} qtl_result;

/* hbm_budget_bytes: device memory the server may hold for requests at once
 * (0 = 90% of the device's free memory); max_inflight: streams (1..64). */
qtl_status qtl_server_create(size_t hbm_budget_bytes, int32_t max_inflight, qtl_server** out);
/* Queues a request; expect_out (host, n_e*nt) receives the expectation values.
 * QTL_ENOMEM if the request alone exceeds the budget, QTL_EINVAL on bad input. */
qtl_status qtl_server_submit(qtl_server* srv, const qtl_request* req, qtl_c128* expect_out,
                             uint64_t* ticket);
/* QTL_EBUSY while the request is queued or running, else QTL_OK with *out filled. */
qtl_status qtl_server_poll(qtl_server* srv, uint64_t ticket, qtl_result* out);
/* Blocks until the request is done. */
qtl_status qtl_server_wait(qtl_server* srv, uint64_t ticket, qtl_result* out);
/* Removes a request that has not been admitted yet (its result becomes
 * QTL_ECANCEL); QTL_EBUSY if it is already running. */
qtl_status qtl_server_cancel(qtl_server* srv, uint64_t ticket);
/* Device bytes currently held for admitted requests, and requests waiting. */
qtl_status qtl_server_usage(qtl_server* srv, size_t* bytes_in_use, int32_t* queued, int32_t* running);
/* Waits for running requests, cancels queued ones, releases everything. */
void qtl_server_free(qtl_server* srv);

/* No counterpart in the paper: an mcsolve entry point for callers that cannot
 * allocate device memory while they solve -- code running during CUDA stream
 * capture (cudaMalloc is not allowed there), processes whose device memory is
 * owned by another allocator or a fixed budget, and latency-critical loops
 * that must not wait on the driver's allocator.  It runs the register-
 * resident trajectory kernel of qtl_mcsolve_async (n <= 1024), with plain
 * CSR rows and general observables in place of that call's segmented rows and
 * diagonal-observable path, so the two agree to rounding (the library's tests
 * check 1e-8 in FP64, 1e-6 in mixed precision), and it allocates nothing:
 *   - every input is a caller-owned DEVICE array: A = -i H_eff as an n x n
 *     CSR (row pointers a_row_ptr[n+1], column indices and complex values of
 *     a_nnz entries), the n_c collapse operators stacked row-wise in one CSR
 *     of n_c*n rows (operator k in rows k*n .. k*n+n-1), the n_e observables
 *     stacked the same way, psi0[n] and tlist[nt];
 *   - expect[n_e*nt] (trajectory means, row k = observable k) and info are
 *     caller-owned device outputs;
 *   - scratch (row segments, the complex64 copy of A for QTL_MIXED and the
 *     n_e*nt*ntraj per-trajectory expectation values) lives in one
 *     file-scope device array of QTL_NOALLOC_SCRATCH_BYTES (32 MiB) that the
 *     library holds on every GPU that loads it until the process exits.
 * Requests whose scratch would exceed that size return QTL_ETOOBIG; n is
 * limited to 1024 (QTL_ETOOBIG above).  A's structure is checked on the
 * device (row pointers from 0 to a_nnz, non-decreasing, columns in [0, n)):
 * a malformed A sets info->status = QTL_EINVAL and the trajectories run on
 * empty rows.  The collapse and observable CSR arrays are not checked and
 * must be well formed.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array, which keeps the previous call's contents: calls that overlap
 * on the GPU race on it and must be ordered by the caller.  Enqueued on
 * opts->cuda_stream; status in info->status as for the _async calls. */
#define QTL_NOALLOC_SCRATCH_BYTES (32u << 20)
qtl_status qtl_mcsolve_noalloc(int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx,
                               const qtl_c128* a_vals, int64_t a_nnz, int32_t n_c,
                               const int32_t* c_row_ptr, const int32_t* c_col_idx,
                               const qtl_c128* c_vals, int32_t n_e, const int32_t* o_row_ptr,
                               const int32_t* o_col_idx, const qtl_c128* o_vals,
                               const qtl_c128* psi0, const double* tlist, int32_t nt,
                               int32_t ntraj, uint64_t seed, int64_t traj_offset,
                               const qtl_opts* opts, qtl_c128* expect, qtl_device_info* info);

/* Human-readable text of a status, and the last CUDA error seen by this
 * thread (empty string if none). */
const char* qtl_strerror(qtl_status s);
const char* qtl_last_cuda_error(void);

/* Number of kernel launches the library has issued in this process
 * (a monotone counter, for accounting in benchmarks). */
int64_t qtl_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* QTL_H */
