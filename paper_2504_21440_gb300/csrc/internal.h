// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qtl.h"

namespace qtl {

// ---------------------------------------------------------------- host CSR
struct Csr {
    int n = 0;
    std::vector<int32_t> rp;   // n+1
    std::vector<int32_t> ci;   // nnz
    std::vector<double> re, im;
    int64_t nnz() const { return (int64_t)ci.size(); }
};

// ------------------------------------------------------ device CSR copies
// Rows are stored with their entries grouped as [real-only | imaginary-only |
// complex]; seg[r] = {start, start of imaginary-only, start of complex, end},
// so a product spends 2 FMAs on an entry that is purely real or imaginary.
struct DevCsr {
    int n = 0;
    int64_t nnz = 0;
    int4* seg = nullptr;
    int32_t* rp = nullptr;
    int32_t* ci = nullptr;
    double2* v64 = nullptr;
    float2* v32 = nullptr;
    int64_t nnz_half = 0;   // entries with a zero real or zero imaginary part (4 flops in a product, not 8)
};

// Sliced ELLPACK copy of A for the wide trajectory kernel, with the
// structure of tensor-product operators factored out.  Rows come in slices of
// 32 (one warp's rows); each row's entries are grouped real-only |
// imaginary-only | complex as in DevCsr and ordered by col XOR row, and each
// group is padded to the slice's longest row.  Entry position p of a slice
// is described by {mode, column parameter, value index, 0}:
//   column: explicit (ci[cbase + param + lane]), XOR (row ^ param: Pauli-type
//           flips) or offset (row + param: ladder-type shifts), whichever
//           holds for all 32 rows (padding rows only need an in-range column);
//   value:  uniform (vs[param'] / vc[param'], one value shared by the 32
//           rows, stored once for the whole operator) or explicit
//           (vs[vsbase + param' + lane] / vc[vcbase + param' + lane]);
//           padding entries are zeros.
// Explicit parts are addressed relative to the slice's bases, so slices with
// the same pattern share one descriptor list: for the Ising chain all 512
// slices of the 14-spin operator use the same 15 descriptors (L1-resident),
// and the only per-row data left is the diagonal.
// Descriptor .w holds the FP32 bits of a uniform real or imaginary value.
// sl[2s] = {first descriptor, real, imaginary, complex widths},
// sl[2s+1] = {cbase, vsbase, vcbase, group types}.
enum { SELL_COL_EXPLICIT = 0, SELL_COL_XOR = 1, SELL_COL_OFFSET = 2, SELL_VAL_UNIFORM = 4 };
// Per-slice group types (sl[2s+1].w, 2 bits per group, real | imaginary |
// complex), each run by its own loop in the kernel.
enum { SELL_G_GENERAL = 0, SELL_G_XU = 1, SELL_G_XE = 2, SELL_G_EE = 3 };
struct DevSell {
    int n = 0, nslices = 0;
    int idx16 = 0;           // explicit columns stored as uint16 (n <= 65536)
    int64_t ndesc = 0, nci = 0, nvs = 0, nvc = 0;
    int4* sl = nullptr;      // [2 nslices]
    int4* desc = nullptr;    // [ndesc] shared descriptor lists
    void* ci = nullptr;      // [nci] explicit columns, 32 per explicit descriptor
    double* vs64 = nullptr;  // [nvs] real part (real-only group) or imaginary part
    float* vs32 = nullptr;
    double2* vc64 = nullptr; // [nvc] complex values
    float2* vc32 = nullptr;
    float* vs32lo = nullptr; // v - (double)(float)v: the FP32 remainder of each value
    float2* vc32lo = nullptr;
    std::vector<int4> hdesc; // host copy of the descriptors when there are few
};

// Descriptors passed to the wide kernel as a __grid_constant__ parameter
// when they fit: the loads then go through the constant cache and leave the
// L1 data pipe to the stage-input gathers.
constexpr int SELL_CDESC = 256;
struct SellConst {
    int4 d[SELL_CDESC];
};

// One operator in pattern-compressed sliced ELLPACK, as the kernels read it.
struct SellRef {
    const int4* sl;       // [2 nslices]
    const int4* desc;
    const int32_t* ci;
    const double* vs64;
    const float* vs32;
    const double2* vc64;
    const float2* vc32;
};

// ---------------------------------------------------------------- system
struct System {
    int n = 0, n_c = 0, n_e = 0;
    Csr H;
    std::vector<Csr> C;   // collapse operators
    std::vector<Csr> O;   // observables
    Csr A;                // -i H - 1/2 sum C^dag C
    Csr Bt;               // (i H - 1/2 sum C^dag C)^T
    // device
    DevCsr dA;            // mcsolve RHS; left factor of the product-form RHS
    DevCsr dBt;           // B^T (B = i H - 1/2 sum C^dag C): right factor of the product form
    DevCsr dC;            // all collapse operators stacked: rows k*n .. k*n+n-1
    DevCsr dO;            // all observables stacked: rows k*n .. k*n+n-1
    DevCsr dL;            // Liouvillian (built lazily)
    DevSell sA;           // A in sliced ELLPACK (built lazily: wide trajectories, grid mesolve)
    DevSell sBt;          // B^T in sliced ELLPACK (built lazily: grid mesolve)
    int2* units = nullptr;      // grid-mesolve work units (built with sBt)
    int nu_tri = 0, nu_all = 0;
    int herm_h = 0;             // H == H^dag exactly (and every time-dependent term real and Hermitian)
    int c_real = 0;             // every collapse-operator value is real
    std::vector<Csr> Htd;       // time-dependent terms f_k(t) H_k
    std::vector<qtl_coef> ftd;
    DevCsr dT;                  // -i H_k stacked row-wise, segmented (trajectory kernel)
    DevCsr dTL;                 // their Liouvillians -i (I kron H_k - H_k^T kron I), stacked (cluster kernel)
    std::vector<DevSell> sTa;   // -i H_k in sliced ELLPACK (grid kernel)
    std::vector<DevSell> sTb;   // (i H_k)^T in sliced ELLPACK (grid kernel)
    qtl_coef* d_tf = nullptr;   // device copy of ftd
    SellRef* d_tsl = nullptr;   // device [2 n_td] references to sTa, sTb (grid kernel)
    bool solved = false;        // a solve has run: no more terms
    std::vector<int32_t> L_rp;  // host copy of its row pointers (shared-memory sizing)
    double2* ew = nullptr;      // [n*n][n_e] trace weights (built with the Liouvillian)
    double* odiag = nullptr;    // [n_e][n] diagonals when every observable is real and diagonal
    int32_t* cmap = nullptr;    // [n_c][n] column of C_c's entry in row i, -1 if none
    double2* cval64 = nullptr;  // [n_c][n] its value (only when every row has <= 1 entry)
    float2* cval32 = nullptr;
    int device = 0;
    struct SsCache* ss = nullptr;   // stationary-state preconditioner (steady.cu), built on first use
};

// -------------------------------------------- device-side solve descriptors
struct MeJob {
    int n, L;
    int n_td;             // time-dependent terms f_k(t) L_k (single solves)
    const int32_t* trp;   // L_k = -i (I kron H_k - H_k^T kron I) stacked (rows k*L + r)
    const int32_t* tci;
    const double2* tv;
    const qtl_coef* tf;
    const int4* seg;      // Liouvillian, segmented rows
    const int32_t* ci;
    const double2* lv64;
    const float2* lv32;
    int n_e;
    const double2* ew;    // [L][n_e]: Tr(O_e rho) = sum_r ew[r][e] * vec(rho)[r]
    const double* tlist;
    int nt;
    const double2* state0;
    int is_ket;
    double* epart;        // scratch [nt][C][2 n_e]: per-CTA partial expectation values
    double2* expect;      // [n_e*nt]
    double2* states;      // [nt*L] or null
    qtl_device_info* info;
    double rtol, atol, dt0, dt_min, dt_fixed;
    long long max_steps;
    int fixed;
    int method;
    int smem_nnz;         // per-CTA shared-memory capacity for Liouvillian entries
    double2* tdg;         // mixed precision with n_td > 0: scratch [2][n_td][L], L_k y in FP64
};

// Time-dependent Hamiltonian terms f_k(t) H_k per system (qtl_system_add_td).
constexpr int QTL_MAX_TD = 8;


// Large-rho mesolve (one cooperative grid per solve, product-form RHS).
struct MgJob {
    int n;
    long long L;
    SellRef a;            // A = -i H - 1/2 sum C^dag C
    SellRef bt;           // B^T, B = i H - 1/2 sum C^dag C
    const int2* units;    // warp work units {row slice, column group}; the
                          // units meeting the lower triangle come first
    int nu_tri, nu_all;
    int herm_h;           // H(t) is exactly Hermitian at every t
    int c_real;           // every collapse-operator value is real (cmap path)
    int n_td;             // time-dependent terms (FP64 kernel only)
    const SellRef* tsl;   // device [2 n_td]: -i H_k for k < n_td, then (i H_k)^T
    const qtl_coef* tf;   // device [n_td] coefficients
    int n_c;
    const int32_t* crp;   // collapse operators stacked row-wise (plain CSR)
    const int32_t* cci;
    const double2* cv64;
    const float2* cv32;
    const int32_t* cmap;  // monomial collapse operators: [n_c][n] column map (or null)
    const double2* cmv64;
    const float2* cmv32;
    int n_e;
    const int32_t* orp;   // observables stacked row-wise (plain CSR)
    const int32_t* oci;
    const double2* ov;
    const double* tlist;
    int nt;
    const double2* state0;
    int is_ket;
    double2* y0buf;       // scratch [L] FP64 state (two alternating buffers: y, y_new)
    double2* y1buf;
    void* k;              // scratch [7][L] stage derivatives (FP64 or FP32)
    void* ys;             // scratch [2][L] stage inputs (FP64 or FP32)
    float4* base;         // MIXED: scratch [2][L] derivative at y as an FP32 pair (current, candidate)
    double2* y64;         // MIXED: scratch [L] FP64 stage input of the FP64 base evaluation
    int refresh;          // MIXED: accepted steps between FP64 evaluations of the base
    float* errpart;       // scratch [grid] error partials
    double* epart;        // scratch [nt][grid][2 n_e] expectation partials
    double2* expect;      // [n_e*nt]
    double2* states;      // [nt*L] or null
    qtl_device_info* info;
    double rtol, atol, dt0, dt_min, dt_fixed;
    long long max_steps;
    int fixed;
    int method;
};

// Operators of one trajectory (DSF on trajectories: each trajectory carries
// its own frame, so its own A = -i H_eff, collapse operators and
// observables); device pointers into that trajectory's system.
struct McTrajOps {
    const int4* aseg;
    const int32_t* aci;
    const double2* av64;
    const float2* av32;
    const int32_t* crp;
    const int32_t* cci;
    const double2* cv;
    const int32_t* orp;
    const int32_t* oci;
    const double2* ov;
};

struct McJob {
    int n;
    int a_nnz;            // entries of A
    int a_smem;           // 1: the kernel keeps A in shared memory
    const int4* aseg;     // A = -i H_eff, segmented rows
    const int32_t* arp;
    const int32_t* aci;
    const double2* av64;
    const float2* av32;
    int n_c;
    const int32_t* crp;   // stacked collapse ops
    const int32_t* cci;
    const double2* cv;
    int n_e;
    const int32_t* orp;   // stacked observables
    const int32_t* oci;
    const double2* ov;
    const int4* oseg;     // their row segments (real-only | imaginary-only | complex), or null
    const double* odiag;  // [n_e][n]: every observable real and diagonal (else null)
    double2* traj_meas;   // ssesolve: [(n*nt + t)*ntraj + j] homodyne currents (re; im = 0)
    double2* meas;        // ssesolve: [n_c*nt] their trajectory means
    const double2* ew;    // smesolve: [n*n][n_e] trace weights, Tr(O rho) = sum_r ew[r] vec(rho)[r]
    int n_td;             // time-dependent terms f_k(t) (-i H_k), trajectory kernel n <= 1024
    const int4* tseg;     // -i H_k stacked row-wise (rows k*n + r), segmented
    const int32_t* tci;
    const double2* tv64;
    const float2* tv32;
    const qtl_coef* tf;   // device [n_td] coefficients
    const SellRef* tsl;   // wide trajectory kernel (FP64): -i H_k in sliced ELLPACK, [n_td]
    const double* tlist;
    int nt;
    const double2* psi0;
    int ntraj;
    unsigned long long seed;
    long long traj_offset;
    double2* traj_expect;  // [(k*nt + t)*ntraj + j]
    double2* expect;       // [n_e*nt] (mean)
    qtl_device_info* info;
    double rtol, atol, dt0, dt_min, dt_fixed;
    long long max_steps;
    int fixed;
    int method;
    // trajectories above the register-resident size (mc_wide.cu)
    const int4* sl;        // A in pattern-compressed sliced ELLPACK (DevSell)
    const int4* sdesc;
    int sdesc_const;       // 1: the descriptors are in the kernel's SellConst parameter
    int sidx16;
    const void* sci;
    const double* svs64;
    const float* svs32;
    const double2* svc64;
    const float2* svc32;
    const float* svs32lo;  // FP32 remainders of the values (error-free products, mixed precision)
    const float2* svc32lo;
    unsigned char* wscr;   // [grid][wstride] bytes of per-CTA state
    size_t wstride;
    int xsmem;             // stage inputs in shared memory (1) or in wscr (0)
    int xbufs;             // stage-input buffers in shared memory (1 or 2)
    int* wnext;            // trajectory counter (zero at launch), or null: static assignment
    // trajectory kernel, resumable trajectories (null / 0: off)
    const McTrajOps* tops;  // [ntraj]: trajectory jt's own operators instead of the job's
    long long psi0_stride;  // elements between the trajectories' initial kets (0: one shared ket)
    double2* psi_out;       // [ntraj][n]: the unnormalised ket at the last time of tlist
    unsigned* rng_draw;     // [ntraj] in/out: Philox draw counter; 0 = start the stream
    double* rng_r;          // [ntraj] in/out: the current jump threshold (when rng_draw > 0)
};

// Launch plan of the wide trajectory kernel: grid, shared memory and the
// per-CTA scratch it needs (allocated by the caller).
struct McWidePlan {
    int grid;
    int xsmem, xbufs;
    size_t smem;
    size_t stride;         // bytes of scratch per CTA
    size_t scratch_bytes;  // grid * stride
};

// kernels (launchers return cudaError_t of the launch)
bool me_plan(int L_max, int cluster_size, int* C, int* rpt);
int me_smem_nnz_budget(int precision, int rpt);
cudaError_t launch_me_cluster(const MeJob* jobs_dev, int njobs, int L_max, int smem_nnz,
                              int precision, int cluster_size, int* next, cudaStream_t st);
cudaError_t launch_mc_traj(const McJob& job, int precision, cudaStream_t st);
cudaError_t launch_mc_reduce(const McJob& job, cudaStream_t st);
cudaError_t launch_sse_traj(const McJob& job, cudaStream_t st);   // ssesolve (FP64, n <= 1024)
cudaError_t launch_sme_traj(const McJob& job, cudaStream_t st);   // smesolve (FP64, n*n <= 4096)
// means over trajectories of traj[(row)*ntraj + j] into out[row] (fixed order)
cudaError_t launch_traj_mean(const double2* traj, double2* out, int nrows, int ntraj, cudaStream_t st);
constexpr int SSE_MAXSC = 4;      // stochastic operators per ssesolve
cudaError_t launch_info_init(qtl_device_info* info, cudaStream_t st);

qtl_status validate_opts(const qtl_opts* o);

int me_cluster_capacity();
cudaError_t launch_me_grid(const MgJob& J, int precision, cudaStream_t st, int* grid_out);
int me_grid_blocks(int precision);        // max L handled by the cluster kernel
int mc_traj_capacity();           // max n handled by the trajectory kernel
int mc_wide_capacity();           // max n handled by the wide trajectory kernel
cudaError_t mc_wide_plan(const McJob& job, int precision, McWidePlan* plan);
cudaError_t launch_mc_wide(const McJob& job, int precision, const McWidePlan& plan, void* scratch,
                           const SellConst* cdesc, cudaStream_t st);

// host helpers shared by the solve entry points (runtime.cpp)
// CSR Liouvillian (FP64, column stacking) on the device, built once per
// system; ETOOBIG when n^2 exceeds max_rows (default: the cluster kernel's
// capacity).
qtl_status ensure_liouvillian(System& s, int64_t max_rows = -1);
// kind: QTL_REQ_MESOLVE | QTL_REQ_MCSOLVE; *fills_gpu (if non-null): the
// solve's kernel occupies every SM (the cooperative grid mesolve, the
// one-CTA-per-SM wide trajectory kernel)
qtl_status prepare_solve(System& s, int kind, const qtl_opts* o, int* fills_gpu = nullptr);
void batch_plan(int L, int* C, int* rpt);
int64_t cta_nnz_max(const System& s, int C);
// one cluster-kernel job; tdg: scratch of 2 n_td n^2 complex (mixed
// precision with time-dependent terms), else null
void me_job_fill(MeJob& J, const System& s, const double* tlist_dev, int nt, const qtl_c128* state0_dev,
                 int is_ket, double* epart, qtl_c128* expect_dev, qtl_device_info* info_dev,
                 const qtl_opts* opts, int smem_nnz, double2* tdg = nullptr);
// bytes of that scratch for a solve of s in the given precision (0 if none)
size_t me_tdg_bytes(const System& s, int precision);
// the Liouvillians of the time-dependent terms on the device (built once)
qtl_status ensure_td_liouvillian(System& s);
// the time-dependent terms in sliced ELLPACK (s.sTa, s.sTb, s.d_tsl; built once)
qtl_status ensure_td_sell(System& s);

// Stream-ordered allocation from the library's own pool on the current
// device.  The pool keeps up to 16 GiB of freed memory for reuse instead
// of returning it to the driver at every synchronisation,
// which the default pool does: repeated solves then map no new memory.
cudaError_t qtl_malloc_async(void** p, size_t bytes, cudaStream_t st);

void count_launch(int k = 1);
void set_cuda_error(cudaError_t e);

// runtime.cpp helpers for the other translation units
qtl_status op_to_csr(const qtl_op* op, int n_expect, Csr& out);
qtl_status csr_upload(const Csr& m, DevCsr& d);
void csr_free(DevCsr& d);
void ss_cache_free(System& s);   // steady.cu
// C = op(A) op(B), n x n complex FP64, column-major, op: 0 identity, 1 conjugate transpose (steady.cu)
cudaError_t launch_zgemm(int n, const double2* A, int ta, const double2* B, int tb, double2* C, cudaStream_t st);
// the same product on the tensor cores, split BF16 (tc_gemm.cu)
size_t tc_zgemm_scratch_bytes(int n);
cudaError_t launch_tc_zgemm(int n, const double2* A, int opa, const double2* B, int opb, double2* C, void* scratch,
                            int* err, cudaStream_t st);

}  // namespace qtl

struct qtl_system {
    qtl::System s;
};
