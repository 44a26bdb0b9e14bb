// Host runtime behind the C ABI (include/qtl.h): operator validation and
// conversion to CSR, the FP64 host build of A = -i H - 1/2 sum C^dag C,
// B^T and the column-stacking Liouvillian (paper Sec. 3.2 / 3.3), device
// uploads, and the mesolve / mcsolve drivers that enqueue the kernels.
#include <algorithm>
#include <map>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace qtl {

using cplx = std::complex<double>;

static std::atomic<long long> g_launches{0};
static thread_local std::string g_cuda_err;

void count_launch(int k) { g_launches += k; }

cudaError_t qtl_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            if ((e = cudaMemPoolCreate(&np, &props)) != cudaSuccess) return e;
            unsigned long long thr = 16ull << 30;
            cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &thr);
            pools[dev] = np;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}
void set_cuda_error(cudaError_t e) {
    g_cuda_err = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
}

#define QTL_CUDA(call)                         \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) {               \
            set_cuda_error(e_);                \
            return e_ == cudaErrorMemoryAllocation ? QTL_ENOMEM : QTL_ECUDA; \
        }                                      \
    } while (0)

// ------------------------------------------------------------ CSR helpers
static bool finite_c(const qtl_c128& v) { return std::isfinite(v.re) && std::isfinite(v.im); }

// Converts a qtl_op to a canonical CSR: columns sorted, duplicates summed,
// exact zeros dropped.
static qtl_status to_csr(const qtl_op* op, int n_expect, Csr& out) {
    // CSR operators up to the trajectory kernel's limit; dense ones (n*n
    // values) and any mesolve up to n = 46340 (n*n < 2^31)
    if (!op || op->n <= 0 || op->n > mc_wide_capacity() || (n_expect > 0 && op->n != n_expect))
        return QTL_EINVAL;
    if (!op->is_csr && op->n > 46340) return QTL_EINVAL;
    if (!op->vals) return QTL_EINVAL;
    const int n = op->n;
    out = Csr();
    out.n = n;
    out.rp.assign(n + 1, 0);
    std::vector<std::pair<int32_t, cplx>> rowbuf;
    if (op->is_csr) {
        if (!op->row_ptr || (op->nnz > 0 && !op->col_idx) || op->nnz < 0) return QTL_EINVAL;
        if (op->row_ptr[0] != 0 || op->row_ptr[n] != op->nnz) return QTL_EINVAL;
        for (int i = 0; i < n; ++i)
            if (op->row_ptr[i + 1] < op->row_ptr[i]) return QTL_EINVAL;
        for (int i = 0; i < n; ++i) {
            rowbuf.clear();
            for (int64_t p = op->row_ptr[i]; p < op->row_ptr[i + 1]; ++p) {
                int32_t c = op->col_idx[p];
                if (c < 0 || c >= n || !finite_c(op->vals[p])) return QTL_EINVAL;
                rowbuf.emplace_back(c, cplx(op->vals[p].re, op->vals[p].im));
            }
            std::sort(rowbuf.begin(), rowbuf.end(),
                      [](const auto& a, const auto& b) { return a.first < b.first; });
            for (size_t q = 0; q < rowbuf.size();) {
                int32_t c = rowbuf[q].first;
                cplx s = 0;
                while (q < rowbuf.size() && rowbuf[q].first == c) s += rowbuf[q++].second;
                if (s != cplx(0)) {
                    out.ci.push_back(c);
                    out.re.push_back(s.real());
                    out.im.push_back(s.imag());
                }
            }
            out.rp[i + 1] = (int32_t)out.ci.size();
        }
    } else {
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                const qtl_c128& v = op->vals[(size_t)j * n + i];
                if (!finite_c(v)) return QTL_EINVAL;
                if (v.re != 0.0 || v.im != 0.0) {
                    out.ci.push_back(j);
                    out.re.push_back(v.re);
                    out.im.push_back(v.im);
                }
            }
            out.rp[i + 1] = (int32_t)out.ci.size();
        }
    }
    return QTL_OK;
}

static cplx at(const Csr& m, int64_t p) { return cplx(m.re[p], m.im[p]); }

// Builds a CSR from per-row (col, value) lists.
static void rows_to_csr(int n, std::vector<std::vector<std::pair<int32_t, cplx>>>& rows, Csr& out) {
    out = Csr();
    out.n = n;
    out.rp.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        auto& r = rows[i];
        std::sort(r.begin(), r.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t q = 0; q < r.size();) {
            int32_t c = r[q].first;
            cplx s = 0;
            while (q < r.size() && r[q].first == c) s += r[q++].second;
            if (s != cplx(0)) {
                out.ci.push_back(c);
                out.re.push_back(s.real());
                out.im.push_back(s.imag());
            }
        }
        out.rp[i + 1] = (int32_t)out.ci.size();
        r.clear();
        r.shrink_to_fit();
    }
}

// G = sum_k C_k^dag C_k:  G_ij = sum_k sum_l conj(C_k[l,i]) C_k[l,j].
static void sum_cdagc(int n, const std::vector<Csr>& C, Csr& G) {
    std::vector<std::vector<std::pair<int32_t, cplx>>> rows(n);
    for (const Csr& c : C)
        for (int l = 0; l < n; ++l)
            for (int64_t p = c.rp[l]; p < c.rp[l + 1]; ++p)
                for (int64_t q = c.rp[l]; q < c.rp[l + 1]; ++q)
                    rows[c.ci[p]].emplace_back(c.ci[q], std::conj(at(c, p)) * at(c, q));
    rows_to_csr(n, rows, G);
}

// A = -i H - G/2 and B^T with B = i H - G/2 (rows of B^T are columns of B).
static void build_a_bt(const Csr& H, const Csr& G, Csr& A, Csr& Bt) {
    const int n = H.n;
    std::vector<std::vector<std::pair<int32_t, cplx>>> ra(n), rb(n);
    const cplx I(0, 1);
    for (int i = 0; i < n; ++i) {
        for (int64_t p = H.rp[i]; p < H.rp[i + 1]; ++p) {
            ra[i].emplace_back(H.ci[p], -I * at(H, p));
            rb[H.ci[p]].emplace_back(i, I * at(H, p));
        }
        for (int64_t p = G.rp[i]; p < G.rp[i + 1]; ++p) {
            ra[i].emplace_back(G.ci[p], -0.5 * at(G, p));
            rb[G.ci[p]].emplace_back(i, -0.5 * at(G, p));
        }
    }
    rows_to_csr(n, ra, A);
    rows_to_csr(n, rb, Bt);
}

// Liouvillian for column stacking, row r = i + n j (the entry rho_ij):
//   (I kron A)        -> A_ik          at column k + n j
//   (B^T kron I)      -> (B^T)_jl      at column i + n l
//   (conj(C) kron C)  -> C_ik conj(C_jl) at column k + n l
static void build_liouvillian(const System& s, Csr& L) {
    const int n = s.n;
    const int64_t NL = (int64_t)n * n;
    L = Csr();
    L.n = (int)NL;
    L.rp.assign(NL + 1, 0);
    std::vector<std::pair<int32_t, cplx>> row;
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            row.clear();
            for (int64_t p = s.A.rp[i]; p < s.A.rp[i + 1]; ++p)
                row.emplace_back(s.A.ci[p] + n * j, at(s.A, p));
            for (int64_t p = s.Bt.rp[j]; p < s.Bt.rp[j + 1]; ++p)
                row.emplace_back(i + n * s.Bt.ci[p], at(s.Bt, p));
            for (const Csr& c : s.C)
                for (int64_t p = c.rp[i]; p < c.rp[i + 1]; ++p)
                    for (int64_t q = c.rp[j]; q < c.rp[j + 1]; ++q)
                        row.emplace_back(c.ci[p] + n * c.ci[q], at(c, p) * std::conj(at(c, q)));
            std::sort(row.begin(), row.end(),
                      [](const auto& a, const auto& b) { return a.first < b.first; });
            for (size_t q = 0; q < row.size();) {
                int32_t col = row[q].first;
                cplx v = 0;
                while (q < row.size() && row[q].first == col) v += row[q++].second;
                if (v != cplx(0)) {
                    L.ci.push_back(col);
                    L.re.push_back(v.real());
                    L.im.push_back(v.imag());
                }
            }
            L.rp[(int64_t)i + (int64_t)n * j + 1] = (int32_t)L.ci.size();
        }
    }
}

// Stacks operators row-wise (operator k occupies rows k*n .. k*n+n-1).
static void stack(const std::vector<Csr>& ops, int n, Csr& out) {
    out = Csr();
    out.n = n * (int)ops.size();
    out.rp.assign((size_t)out.n + 1, 0);
    int r = 0;
    for (const Csr& o : ops) {
        for (int i = 0; i < n; ++i, ++r) {
            for (int64_t p = o.rp[i]; p < o.rp[i + 1]; ++p) {
                out.ci.push_back(o.ci[p]);
                out.re.push_back(o.re[p]);
                out.im.push_back(o.im[p]);
            }
            out.rp[r + 1] = (int32_t)out.ci.size();
        }
    }
}

template <class T>
static qtl_status upload(T** dst, const T* src, size_t count) {
    *dst = nullptr;
    if (count == 0) return QTL_OK;
    QTL_CUDA(cudaMalloc((void**)dst, count * sizeof(T)));
    QTL_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return QTL_OK;
}

static void free_csr(DevCsr& d) {
    cudaFree(d.seg);
    cudaFree(d.rp);
    cudaFree(d.ci);
    cudaFree(d.v64);
    cudaFree(d.v32);
    d = DevCsr();
}

// All or nothing: on failure nothing stays allocated and d is empty, so a
// non-null d.rp always means a complete upload.
static qtl_status upload_csr(const Csr& m, DevCsr& d) {
    d.n = m.n;
    d.nnz = m.nnz();
    d.nnz_half = 0;
    std::vector<double2> v64(m.nnz());
    std::vector<float2> v32(m.nnz());
    std::vector<int32_t> ci(m.nnz());
    std::vector<int4> seg(m.n);
    std::vector<std::pair<int32_t, int64_t>> order;
    for (int r = 0; r < m.n; ++r) {
        // group the row's entries: real-only, imaginary-only, complex; inside
        // a group order them by col XOR row, so that in tensor-product
        // operators the p-th entry of neighbouring rows is the same term and
        // a warp's gathers stay in aligned blocks
        int32_t q = m.rp[r];
        int b[3];
        for (int grp = 0; grp < 3; ++grp) {
            b[grp] = q;
            order.clear();
            for (int64_t p = m.rp[r]; p < m.rp[r + 1]; ++p) {
                const bool re0 = m.re[p] == 0.0, im0 = m.im[p] == 0.0;
                const int gp = im0 ? 0 : (re0 ? 1 : 2);
                if (gp == grp) order.emplace_back(m.ci[p] ^ r, p);
            }
            std::sort(order.begin(), order.end());
            for (const auto& kp : order) {
                const int64_t p = kp.second;
                ci[q] = m.ci[p];
                v64[q] = make_double2(m.re[p], m.im[p]);
                v32[q] = make_float2((float)m.re[p], (float)m.im[p]);
                ++q;
            }
        }
        seg[r] = make_int4(b[0], b[1], b[2], m.rp[r + 1]);
        d.nnz_half += b[2] - b[0];
    }
    qtl_status st;
    if ((st = upload(&d.seg, seg.data(), seg.size())) != QTL_OK ||
        (st = upload(&d.rp, m.rp.data(), m.rp.size())) != QTL_OK ||
        (st = upload(&d.ci, ci.data(), ci.size())) != QTL_OK ||
        (st = upload(&d.v64, v64.data(), v64.size())) != QTL_OK ||
        (st = upload(&d.v32, v32.data(), v32.size())) != QTL_OK)
        free_csr(d);
    return st;
}

qtl_status op_to_csr(const qtl_op* op, int n_expect, Csr& out) { return to_csr(op, n_expect, out); }
qtl_status csr_upload(const Csr& m, DevCsr& d) { return upload_csr(m, d); }
void csr_free(DevCsr& d) { free_csr(d); }

// A in pattern-compressed sliced ELLPACK (see DevSell); entries grouped and
// ordered as in upload_csr.  Descriptor lists and uniform values are
// deduplicated across slices.
static qtl_status upload_sell(const Csr& m, DevSell& d) {
    const int n = m.n, ns_ = (n + 31) / 32;
    std::vector<int4> sl(2 * (size_t)ns_), desc, list;
    std::vector<int32_t> ci;
    std::vector<double> vs;
    std::vector<double2> vc;
    std::map<std::vector<int64_t>, int> lists;         // descriptor list -> first descriptor
    std::map<std::pair<double, double>, int> uni_s, uni_c;  // uniform value -> index
    std::vector<std::pair<int32_t, int64_t>> order;
    std::vector<std::vector<int64_t>> grp[3];
    for (int g = 0; g < 3; ++g) grp[g].resize(32);
    for (int s = 0; s < ns_; ++s) {
        int w[3] = {0, 0, 0};
        const int r0 = s * 32, nl = std::min(32, n - r0);  // valid rows of the slice
        for (int l = 0; l < 32; ++l) {
            for (int g = 0; g < 3; ++g) grp[g][l].clear();
            if (l >= nl) continue;
            const int r = r0 + l;
            for (int g = 0; g < 3; ++g) {
                order.clear();
                for (int64_t p = m.rp[r]; p < m.rp[r + 1]; ++p) {
                    const bool re0 = m.re[p] == 0.0, im0 = m.im[p] == 0.0;
                    if ((im0 ? 0 : (re0 ? 1 : 2)) == g) order.emplace_back(m.ci[p] ^ r, p);
                }
                std::sort(order.begin(), order.end());
                for (const auto& kp : order) grp[g][l].push_back(kp.second);
                w[g] = std::max(w[g], (int)grp[g][l].size());
            }
        }
        const int cbase = (int)ci.size(), vsbase = (int)vs.size(), vcbase = (int)vc.size();
        list.clear();
        for (int g = 0; g < 3; ++g)
            for (int p = 0; p < w[g]; ++p) {
                // entry of lane l at position p, or -1 (padding)
                auto ent = [&](int l) -> int64_t {
                    return p < (int)grp[g][l].size() ? grp[g][l][p] : -1;
                };
                // column pattern: XOR, then offset, else explicit; a padding
                // lane accepts any pattern whose column is in range
                int mode = SELL_COL_EXPLICIT, param = 0;
                for (int cand = SELL_COL_XOR; cand <= SELL_COL_OFFSET && mode == SELL_COL_EXPLICIT; ++cand) {
                    bool have = false, ok = true;
                    int64_t pv = 0;
                    for (int l = 0; l < nl && ok; ++l) {
                        const int64_t e = ent(l);
                        if (e < 0) continue;
                        const int r = r0 + l, c = m.ci[e];
                        const int64_t v = cand == SELL_COL_XOR ? (int64_t)(c ^ r) : (int64_t)c - r;
                        if (!have) {
                            pv = v;
                            have = true;
                        } else if (v != pv) {
                            ok = false;
                        }
                    }
                    if (!have || !ok) continue;
                    for (int l = 0; l < nl && ok; ++l) {
                        if (ent(l) >= 0) continue;
                        const int64_t r = r0 + l;
                        const int64_t c = cand == SELL_COL_XOR ? (r ^ pv) : r + pv;
                        ok = c >= 0 && c < n;
                    }
                    if (ok) {
                        mode = cand;
                        param = (int)pv;
                    }
                }
                if (mode == SELL_COL_EXPLICIT) {
                    param = (int)ci.size() - cbase;
                    for (int l = 0; l < 32; ++l) {
                        const int64_t e = l < nl ? ent(l) : -1;
                        ci.push_back(e >= 0 ? m.ci[e] : std::min(r0 + l, n - 1));
                    }
                }
                // values: uniform when every valid lane holds the same entry value
                bool uni = true;
                const int64_t e0 = ent(0);
                for (int l = 0; l < nl && uni; ++l) {
                    const int64_t e = ent(l);
                    if (e < 0 || e0 < 0 || m.re[e] != m.re[e0] || m.im[e] != m.im[e0]) uni = false;
                }
                int vix;
                if (uni) {
                    const std::pair<double, double> key(m.re[e0], m.im[e0]);
                    auto& tab = g < 2 ? uni_s : uni_c;
                    auto it = tab.find(key);
                    if (it != tab.end()) {
                        vix = it->second;
                    } else {
                        if (g < 2) {
                            vix = (int)vs.size();
                            vs.push_back(g == 0 ? m.re[e0] : m.im[e0]);
                        } else {
                            vix = (int)vc.size();
                            vc.push_back(make_double2(m.re[e0], m.im[e0]));
                        }
                        tab.emplace(key, vix);
                    }
                } else if (g < 2) {
                    vix = (int)vs.size() - vsbase;
                    for (int l = 0; l < 32; ++l) {
                        const int64_t e = l < nl ? ent(l) : -1;
                        vs.push_back(e < 0 ? 0.0 : (g == 0 ? m.re[e] : m.im[e]));
                    }
                } else {
                    vix = (int)vc.size() - vcbase;
                    for (int l = 0; l < 32; ++l) {
                        const int64_t e = l < nl ? ent(l) : -1;
                        vc.push_back(e < 0 ? make_double2(0.0, 0.0) : make_double2(m.re[e], m.im[e]));
                    }
                }
                // .w: the FP32 bits of a uniform real or imaginary value
                int f32 = 0;
                if (uni && g < 2) {
                    const float f = (float)(g == 0 ? m.re[e0] : m.im[e0]);
                    std::memcpy(&f32, &f, 4);
                }
                list.push_back(make_int4(mode | (uni ? SELL_VAL_UNIFORM : 0), param, vix, f32));
            }
        // group types (2 bits each): XOR columns with uniform values, XOR
        // columns with explicit values, explicit columns and values, or
        // mixed modes; explicit blocks of a typed group are contiguous
        // (32 entries apart), so the kernel needs only the group's first
        // descriptor for them
        int types = 0;
        {
            int off = 0;
            for (int g = 0; g < 3; ++g) {
                int ty = SELL_G_GENERAL;
                if (w[g] > 0) {
                    bool xu = true, xe = true, ee = true;
                    for (int p = 0; p < w[g]; ++p) {
                        const int4& q = list[off + p];
                        const int cm = q.x & 3;
                        const bool un = (q.x & SELL_VAL_UNIFORM) != 0;
                        const int4& q0 = list[off];
                        xu = xu && cm == SELL_COL_XOR && un;
                        xe = xe && cm == SELL_COL_XOR && !un && q.z == q0.z + 32 * p;
                        ee = ee && cm == SELL_COL_EXPLICIT && !un && q.z == q0.z + 32 * p &&
                             q.y == q0.y + 32 * p;
                    }
                    ty = xu ? SELL_G_XU : (xe ? SELL_G_XE : (ee ? SELL_G_EE : SELL_G_GENERAL));
                }
                types |= ty << (2 * g);
                off += w[g];
            }
        }
        // Explicit offsets are relative to the slice's bases; a uniform value
        // first seen inside a slice shifts them, so that slice's list is
        // stored separately, and from then on equal patterns share a list.
        std::vector<int64_t> key;
        key.reserve(list.size() * 3 + 3);
        key.push_back(w[0]);
        key.push_back(w[1]);
        key.push_back(w[2]);
        for (const int4& q : list) {
            key.push_back(q.x);
            key.push_back(q.y);
            key.push_back(q.z);
        }
        auto it = lists.find(key);
        int first;
        if (it != lists.end()) {
            first = it->second;
        } else {
            first = (int)desc.size();
            desc.insert(desc.end(), list.begin(), list.end());
            lists.emplace(std::move(key), first);
        }
        sl[2 * (size_t)s] = make_int4(first, w[0], w[1], w[2]);
        sl[2 * (size_t)s + 1] = make_int4(cbase, vsbase, vcbase, types);
        if (desc.size() >= (size_t)INT32_MAX || ci.size() >= (size_t)INT32_MAX ||
            vs.size() >= (size_t)INT32_MAX || vc.size() >= (size_t)INT32_MAX)
            return QTL_ETOOBIG;
    }
    // keep every array non-empty so that the device pointers are valid
    if (ci.empty()) ci.push_back(0);
    if (vs.empty()) vs.push_back(0.0);
    if (vc.empty()) vc.push_back(make_double2(0.0, 0.0));
    if (desc.empty()) desc.push_back(make_int4(0, 0, 0, 0));
    std::vector<float> vs32(vs.size());
    std::vector<float2> vc32(vc.size());
    for (size_t i = 0; i < vs.size(); ++i) vs32[i] = (float)vs[i];
    for (size_t i = 0; i < vc.size(); ++i) vc32[i] = make_float2((float)vc[i].x, (float)vc[i].y);
    std::vector<float> vs32lo(vs.size());
    std::vector<float2> vc32lo(vc.size());
    for (size_t i = 0; i < vs.size(); ++i) vs32lo[i] = (float)(vs[i] - (double)vs32[i]);
    for (size_t i = 0; i < vc.size(); ++i)
        vc32lo[i] = make_float2((float)(vc[i].x - (double)vc32[i].x), (float)(vc[i].y - (double)vc32[i].y));
    d.n = n;
    d.nslices = ns_;
    d.ndesc = (int64_t)desc.size();
    d.nci = (int64_t)ci.size();
    d.nvs = (int64_t)vs.size();
    d.nvc = (int64_t)vc.size();
    d.idx16 = 0;
    qtl_status st;
    if (desc.size() <= (size_t)SELL_CDESC) d.hdesc = desc;
    if ((st = upload(&d.sl, sl.data(), sl.size())) != QTL_OK) return st;
    if ((st = upload(&d.desc, desc.data(), desc.size())) != QTL_OK) return st;
    if (d.idx16) {
        // half the index traffic: columns fit in 16 bits
        std::vector<uint16_t> c16(ci.begin(), ci.end());
        uint16_t* dc = nullptr;
        if ((st = upload(&dc, c16.data(), c16.size())) != QTL_OK) return st;
        d.ci = dc;
    } else {
        int32_t* dc = nullptr;
        if ((st = upload(&dc, ci.data(), ci.size())) != QTL_OK) return st;
        d.ci = dc;
    }
    if ((st = upload(&d.vs64, vs.data(), vs.size())) != QTL_OK) return st;
    if ((st = upload(&d.vs32, vs32.data(), vs32.size())) != QTL_OK) return st;
    if ((st = upload(&d.vc64, vc.data(), vc.size())) != QTL_OK) return st;
    if ((st = upload(&d.vc32, vc32.data(), vc32.size())) != QTL_OK) return st;
    if ((st = upload(&d.vs32lo, vs32lo.data(), vs32lo.size())) != QTL_OK) return st;
    if ((st = upload(&d.vc32lo, vc32lo.data(), vc32lo.size())) != QTL_OK) return st;
    return QTL_OK;
}

static void free_sell(DevSell& d) {
    cudaFree(d.sl);
    cudaFree(d.desc);
    cudaFree(d.ci);
    cudaFree(d.vs64);
    cudaFree(d.vs32);
    cudaFree(d.vc64);
    cudaFree(d.vc32);
    cudaFree(d.vs32lo);
    cudaFree(d.vc32lo);
    d = DevSell();
}

static std::mutex g_build_mu;

static qtl_status ensure_sell(System& s) {
    std::lock_guard<std::mutex> lk(g_build_mu);
    if (s.sA.sl) return QTL_OK;
    qtl_status st = upload_sell(s.A, s.sA);
    if (st != QTL_OK) free_sell(s.sA);
    return st;
}

// H == H^dag, entry by entry and exactly.
static bool exactly_hermitian(const Csr& m) {
    std::map<std::pair<int32_t, int32_t>, std::pair<double, double>> ent;
    for (int i = 0; i < m.n; ++i)
        for (int64_t p = m.rp[i]; p < m.rp[i + 1]; ++p)
            if (m.re[p] != 0.0 || m.im[p] != 0.0) ent[{i, m.ci[p]}] = {m.re[p], m.im[p]};
    for (const auto& kv : ent) {
        auto it = ent.find({kv.first.second, kv.first.first});
        if (it == ent.end() || it->second.first != kv.second.first || it->second.second != -kv.second.second)
            return false;
    }
    return true;
}

// The time-dependent terms in sliced ELLPACK: -i H_k (the grid mesolve's
// left factors and the wide trajectory kernel's products) and (i H_k)^T (the
// grid's right factors), with their references on the device; built once.
// The caller holds g_build_mu.
static qtl_status ensure_td_sell_locked(System& s) {
    if (s.Htd.empty() || s.d_tsl) return QTL_OK;
    const int ntd = (int)s.Htd.size();
    s.sTa.resize(ntd);
    s.sTb.resize(ntd);
    qtl_status st = QTL_OK;
    for (int k = 0; k < ntd && st == QTL_OK; ++k) {
        const Csr& h = s.Htd[k];
        Csr ta = h, tb;
        for (int64_t p = 0; p < ta.nnz(); ++p) {   // -i (re + i im) = im - i re
            const double re = h.re[p], im = h.im[p];
            ta.re[p] = im;
            ta.im[p] = -re;
        }
        // (i H)^T: row j holds i H[i][j] at column i
        std::vector<std::vector<std::pair<int32_t, cplx>>> rows(s.n);
        for (int i = 0; i < s.n; ++i)
            for (int64_t p = h.rp[i]; p < h.rp[i + 1]; ++p)
                rows[h.ci[p]].emplace_back(i, cplx(-h.im[p], h.re[p]));
        rows_to_csr(s.n, rows, tb);
        if ((st = upload_sell(ta, s.sTa[k])) == QTL_OK) st = upload_sell(tb, s.sTb[k]);
    }
    if (st == QTL_OK) {
        auto ref = [](const DevSell& d) {
            SellRef r;
            r.sl = d.sl;
            r.desc = d.desc;
            r.ci = (const int32_t*)d.ci;
            r.vs64 = d.vs64;
            r.vs32 = d.vs32;
            r.vc64 = d.vc64;
            r.vc32 = d.vc32;
            return r;
        };
        std::vector<SellRef> refs(2 * ntd);
        for (int k = 0; k < ntd; ++k) {
            refs[k] = ref(s.sTa[k]);
            refs[ntd + k] = ref(s.sTb[k]);
        }
        st = upload(&s.d_tsl, refs.data(), refs.size());
    }
    if (st != QTL_OK) {
        // all or nothing: a later call starts again from empty tables
        for (DevSell& d : s.sTa) free_sell(d);
        for (DevSell& d : s.sTb) free_sell(d);
        s.sTa.clear();
        s.sTb.clear();
        cudaFree(s.d_tsl);
        s.d_tsl = nullptr;
    }
    return st;
}

qtl_status ensure_td_sell(System& s) {
    std::lock_guard<std::mutex> lk(g_build_mu);
    return ensure_td_sell_locked(s);
}

// Everything the grid mesolve kernel reads besides the CSR operators: A and
// B^T in sliced ELLPACK, the warp work units and the two structure flags.
// Units {row slice s, column group c} (32 rows x 4 columns) are ordered by
// column group, then slice; those that meet the lower triangle (some row >=
// some column) come first, so the Hermitian mode runs the first nu_tri.
static qtl_status ensure_grid(System& s) {
    qtl_status st = ensure_sell(s);
    if (st != QTL_OK) return st;
    std::lock_guard<std::mutex> lk(g_build_mu);
    if (s.units) return QTL_OK;   // the work units are uploaded last: present means complete
    if (!s.sBt.sl && (st = upload_sell(s.Bt, s.sBt)) != QTL_OK) {
        free_sell(s.sBt);
        return st;
    }
    if ((st = ensure_td_sell_locked(s)) != QTL_OK) return st;
    bool herm = exactly_hermitian(s.H);
    for (size_t k = 0; k < s.Htd.size(); ++k)
        herm = herm && s.ftd[k].kind == QTL_COEF_COS && s.ftd[k].amp_im == 0.0 && exactly_hermitian(s.Htd[k]);
    s.herm_h = herm ? 1 : 0;
    bool real = true;
    for (const Csr& c : s.C)
        for (double v : c.im) real = real && v == 0.0;
    s.c_real = real ? 1 : 0;
    const int n = s.n, ns = (n + 31) / 32, ncg = (n + 3) / 4;
    std::vector<int2> lower, upper;
    for (int c = 0; c < ncg; ++c)
        for (int sl = 0; sl < ns; ++sl) {
            const int amax = std::min(32 * sl + 31, n - 1);
            (amax >= 4 * c ? lower : upper).push_back(make_int2(sl, c));
        }
    s.nu_tri = (int)lower.size();
    s.nu_all = (int)(lower.size() + upper.size());
    lower.insert(lower.end(), upper.begin(), upper.end());
    return upload(&s.units, lower.data(), lower.size());
}

// The Liouvillians of the time-dependent terms alone, L_k = -i (I kron H_k -
// H_k^T kron I) (column stacking: row i + n j holds -i H_k[i][l] at column
// l + n j and +i H_k[l][j] at column i + n l), stacked row-wise.
qtl_status ensure_td_liouvillian(System& s) {
    std::lock_guard<std::mutex> lk(g_build_mu);
    if (s.Htd.empty() || s.dTL.rp) return QTL_OK;
    const int n = s.n;
    const int64_t L = (int64_t)n * n;
    if (L * (int64_t)s.Htd.size() >= (int64_t)INT32_MAX) return QTL_ETOOBIG;
    std::vector<Csr> parts(s.Htd.size());
    for (size_t k = 0; k < s.Htd.size(); ++k) {
        const Csr& h = s.Htd[k];
        std::vector<std::vector<std::pair<int32_t, cplx>>> ht(n);   // columns of H_k
        for (int i = 0; i < n; ++i)
            for (int64_t p = h.rp[i]; p < h.rp[i + 1]; ++p) ht[h.ci[p]].emplace_back(i, at(h, p));
        std::vector<std::vector<std::pair<int32_t, cplx>>> rows((size_t)L);
        const cplx mi(0.0, -1.0);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                auto& r = rows[(size_t)i + (size_t)n * j];
                for (int64_t p = h.rp[i]; p < h.rp[i + 1]; ++p)
                    r.emplace_back(h.ci[p] + n * j, mi * at(h, p));
                for (const auto& lv : ht[j]) r.emplace_back(i + n * lv.first, -mi * lv.second);
            }
        rows_to_csr((int)L, rows, parts[k]);
    }
    Csr stacked;
    stack(parts, (int)L, stacked);
    return upload_csr(stacked, s.dTL);
}

qtl_status ensure_liouvillian(System& s, int64_t max_rows) {
    // The size bound is checked before the cache: a Liouvillian built for a
    // larger caller (the stationary-state solver) is not handed to the
    // cluster kernels, whose bound is the default.
    if ((int64_t)s.n * s.n > (max_rows < 0 ? (int64_t)me_cluster_capacity() : max_rows)) return QTL_ETOOBIG;
    std::lock_guard<std::mutex> lk(g_build_mu);
    if (s.dL.rp) return QTL_OK;
    Csr L;
    build_liouvillian(s, L);
    if (L.nnz() >= (int64_t)INT32_MAX) return QTL_ETOOBIG;
    s.L_rp = L.rp;
    // Tr(O_e rho) = sum_{i,k} O_ik rho_ki: weight O_ik at vec row k + n i.
    const size_t NL = (size_t)s.n * s.n;
    if (s.n_e > 0) {
        std::vector<double2> ew(NL * s.n_e, make_double2(0.0, 0.0));
        for (int e = 0; e < s.n_e; ++e) {
            const Csr& o = s.O[e];
            for (int i = 0; i < s.n; ++i)
                for (int64_t p = o.rp[i]; p < o.rp[i + 1]; ++p)
                    ew[((size_t)o.ci[p] + (size_t)s.n * i) * s.n_e + e] = make_double2(o.re[p], o.im[p]);
        }
        cudaFree(s.ew);   // left by an earlier attempt whose Liouvillian upload failed
        qtl_status st = upload(&s.ew, ew.data(), ew.size());
        if (st != QTL_OK) return st;
    }
    return upload_csr(L, s.dL);
}

static qtl_status check_opts(const qtl_opts* o) {
    if (!o) return QTL_EINVAL;
    if (o->method != QTL_DP5 && o->method != QTL_TSIT5) return QTL_EINVAL;
    if (o->precision != QTL_FP64 && o->precision != QTL_MIXED) return QTL_EINVAL;
    if (o->fixed_step) {
        if (!(o->dt_fixed > 0.0) || !std::isfinite(o->dt_fixed)) return QTL_EINVAL;
    } else {
        if (!(o->rtol > 0.0) || !(o->atol >= 0.0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
            return QTL_EINVAL;
    }
    if (!(o->dt0 >= 0.0) || !(o->dt_min >= 0.0) || o->max_steps <= 0) return QTL_EINVAL;
    if (o->cluster_size < 0 || o->cluster_size > 16) return QTL_EINVAL;
    if (o->engine < QTL_ENGINE_AUTO || o->engine > QTL_ENGINE_GRID) return QTL_EINVAL;
    if (o->shadow_fp64 != 0 && o->shadow_fp64 != 1) return QTL_EINVAL;
    return QTL_OK;
}

// max |a_i - b_i| over m complex values
static double max_abs_diff(const qtl_c128* a, const qtl_c128* b, size_t m) {
    double e = 0.0;
    for (size_t i = 0; i < m; ++i) e = std::max(e, std::hypot(a[i].re - b[i].re, a[i].im - b[i].im));
    return e;
}

qtl_status validate_opts(const qtl_opts* o) { return check_opts(o); }

static qtl_status check_tlist_host(const double* tl, int nt) {
    if (!tl || nt < 1) return QTL_EINVAL;
    for (int i = 0; i < nt; ++i) {
        if (!std::isfinite(tl[i])) return QTL_EINVAL;
        if (i > 0 && tl[i] < tl[i - 1]) return QTL_EINVAL;
    }
    return QTL_OK;
}

// Fixed-step solvers: a trajectory takes about span / dt steps (plus at most
// one short landing step per output time); more than max_steps is refused on
// the host, since those kernels have no step budget of their own.
static qtl_status check_fixed_steps(const double* tl, int nt, const qtl_opts* o) {
    const double steps = (tl[nt - 1] - tl[0]) / o->dt_fixed;
    if (!(steps <= (double)o->max_steps)) return QTL_ESTEP;
    return QTL_OK;
}

int64_t cta_nnz_max_of(const System& s, int C) {
    const int L = s.n * s.n;
    std::vector<int64_t> per(C, 0);
    for (int r = 0; r < L; ++r) per[r % C] += s.L_rp[r + 1] - s.L_rp[r];
    return *std::max_element(per.begin(), per.end());
}

// mesolve on the cooperative grid kernel (product form, no Liouvillian).
// Builds, ahead of a solve, the device structures that solve will use
// (Liouvillian, grid-kernel operators, sliced ELLPACK of A), so that a caller
// such as the request server can do this host work outside its dispatcher.
// The choice of engine repeats the one the solve makes.
qtl_status prepare_solve(System& s, int kind, const qtl_opts* o, int* fills_gpu) {
    if (fills_gpu) *fills_gpu = 0;
    s.solved = true;   // the structures built here hold the terms as they are now
    if (kind == QTL_REQ_MCSOLVE) {
        const bool wide = s.n > mc_traj_capacity() || o->engine == QTL_ENGINE_GRID;
        if (fills_gpu) *fills_gpu = wide;
        if (!wide) return QTL_OK;
        qtl_status st = ensure_sell(s);
        return st == QTL_OK ? ensure_td_sell(s) : st;
    }
    if (s.n > 46340) return QTL_ETOOBIG;
    qtl_status st;
    const int64_t L64 = (int64_t)s.n * s.n;
    bool grid = o->engine == QTL_ENGINE_GRID || (o->engine == QTL_ENGINE_AUTO && L64 > me_cluster_capacity());
    if (!grid) {
        if ((st = ensure_liouvillian(s)) != QTL_OK) return st;
        if (o->engine == QTL_ENGINE_AUTO) {
            int C = 0, rpt = 0;
            me_plan((int)L64, o->cluster_size, &C, &rpt);
            grid = cta_nnz_max_of(s, C) > me_smem_nnz_budget(o->precision, rpt);
        }
    }
    if (fills_gpu) *fills_gpu = grid;
    // time-dependent terms: their Liouvillians only for the cluster kernel
    if (!grid && !s.Htd.empty() && (st = ensure_td_liouvillian(s)) != QTL_OK) return st;
    return grid ? ensure_grid(s) : QTL_OK;
}

qtl_status mesolve_grid(System& s, const qtl_c128* state0_dev, int32_t is_ket, const double* tlist_dev,
                        int32_t nt, const qtl_opts* opts, qtl_c128* expect_dev, qtl_c128* states_dev,
                        qtl_device_info* info_dev) {
    const size_t L = (size_t)s.n * s.n;
    if (L > (size_t)INT32_MAX) return QTL_ETOOBIG;
    qtl_status st = ensure_grid(s);
    if (st != QTL_OK) return st;
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    const int grid = me_grid_blocks(opts->precision);
    const size_t t2 = opts->precision == QTL_MIXED ? sizeof(float2) : sizeof(double2);
    const int ne = s.n_e > 0 ? s.n_e : 1;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_y = up(L * 16), b_k = up(7 * L * t2), b_ys = up(2 * L * t2);
    const size_t b_err = up(3 * (size_t)grid * sizeof(float));
    const size_t b_ep = up((size_t)nt * grid * 2 * ne * sizeof(double));
    const bool mixed = opts->precision == QTL_MIXED;
    const size_t b_base = mixed ? up(2 * L * sizeof(float4)) : 0, b_y64 = mixed ? up(L * sizeof(double2)) : 0;
    char* scratch = nullptr;
    QTL_CUDA(qtl_malloc_async((void**)&scratch, 2 * b_y + b_k + b_ys + b_err + b_ep + b_base + b_y64, stream));
    MgJob J;
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.L = (long long)L;
    auto ref = [](const DevSell& d) {
        SellRef r;
        r.sl = d.sl;
        r.desc = d.desc;
        r.ci = (const int32_t*)d.ci;
        r.vs64 = d.vs64;
        r.vs32 = d.vs32;
        r.vc64 = d.vc64;
        r.vc32 = d.vc32;
        return r;
    };
    J.a = ref(s.sA);
    J.bt = ref(s.sBt);
    J.units = s.units;
    J.nu_tri = s.nu_tri;
    J.nu_all = s.nu_all;
    J.herm_h = s.herm_h;
    J.c_real = s.c_real;
    J.n_td = (int)s.Htd.size();
    J.tsl = s.d_tsl;
    J.tf = s.d_tf;
    J.n_c = s.n_c;
    J.crp = s.dC.rp;
    J.cci = s.dC.ci;
    J.cv64 = s.dC.v64;
    J.cv32 = s.dC.v32;
    J.cmap = s.cmap;
    J.cmv64 = s.cval64;
    J.cmv32 = s.cval32;
    J.n_e = s.n_e;
    J.orp = s.dO.rp;
    J.oci = s.dO.ci;
    J.ov = s.dO.v64;
    J.tlist = tlist_dev;
    J.nt = nt;
    J.state0 = (const double2*)state0_dev;
    J.is_ket = is_ket ? 1 : 0;
    size_t off = 0;
    J.y0buf = (double2*)(scratch + off);
    off += b_y;
    J.y1buf = (double2*)(scratch + off);
    off += b_y;
    J.k = scratch + off;
    off += b_k;
    J.ys = scratch + off;
    off += b_ys;
    J.errpart = (float*)(scratch + off);
    off += b_err;
    J.epart = (double*)(scratch + off);
    off += b_ep;
    J.base = mixed ? (float4*)(scratch + off) : nullptr;
    off += b_base;
    J.y64 = mixed ? (double2*)(scratch + off) : nullptr;
    // FP64 re-evaluation of the base derivative every 8 accepted steps: on a
    // driven Kerr cavity (N = 30, t in [0, 20]) the error against the FP64
    // solution is 5e-8 at every step, 8e-8 at 8 and 1.2e-7 at 32, and the
    // 10-spin chain takes 114, 90 and 90 ms.
    J.refresh = 8;
    J.expect = (double2*)expect_dev;
    J.states = (double2*)states_dev;
    J.info = info_dev;
    J.rtol = opts->rtol;
    J.atol = opts->atol;
    J.dt0 = opts->dt0;
    J.dt_min = opts->dt_min;
    J.dt_fixed = opts->dt_fixed;
    J.max_steps = opts->max_steps;
    J.fixed = opts->fixed_step ? 1 : 0;
    J.method = opts->method;
    QTL_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(qtl_device_info), stream));
    int g = grid;
    cudaError_t e = launch_me_grid(J, opts->precision, stream, &g);
    cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    return QTL_OK;
}


// Launch plan of one system in a batch: cluster size from its own size.
void batch_plan(int L, int* C, int* rpt) {
    int c = 1;
    while (c < 16 && (int64_t)c * 1024 < L) c *= 2;
    me_plan(L, c, C, rpt);
}

int64_t cta_nnz_max(const System& s, int C) {
    const int L = s.n * s.n;
    std::vector<int64_t> per(C, 0);
    for (int r = 0; r < L; ++r) per[r % C] += s.L_rp[r + 1] - s.L_rp[r];
    return *std::max_element(per.begin(), per.end());
}

// One cluster-kernel job: system s from state0 over tlist with opts.
size_t me_tdg_bytes(const System& s, int precision) {
    return precision == QTL_MIXED ? (size_t)2 * s.Htd.size() * (size_t)s.n * s.n * sizeof(double2) : 0;
}

void me_job_fill(MeJob& J, const System& s, const double* tlist_dev, int nt, const qtl_c128* state0_dev,
                 int is_ket, double* epart, qtl_c128* expect_dev, qtl_device_info* info_dev,
                 const qtl_opts* opts, int smem_nnz, double2* tdg) {
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.L = s.n * s.n;
    J.seg = s.dL.seg;
    J.ci = s.dL.ci;
    J.lv64 = s.dL.v64;
    J.lv32 = s.dL.v32;
    J.n_e = s.n_e;
    J.ew = s.ew;
    J.tlist = tlist_dev;
    J.nt = nt;
    J.state0 = (const double2*)state0_dev;
    J.is_ket = is_ket ? 1 : 0;
    J.epart = epart;
    J.expect = (double2*)expect_dev;
    J.states = nullptr;
    J.info = info_dev;
    J.rtol = opts->rtol;
    J.atol = opts->atol;
    J.dt0 = opts->dt0;
    J.dt_min = opts->dt_min;
    J.dt_fixed = opts->dt_fixed;
    J.max_steps = opts->max_steps;
    J.fixed = opts->fixed_step ? 1 : 0;
    J.method = opts->method;
    J.smem_nnz = smem_nnz;
    J.n_td = (int)s.Htd.size();
    J.trp = s.dTL.rp;
    J.tci = s.dTL.ci;
    J.tv = s.dTL.v64;
    J.tf = s.d_tf;
    J.tdg = tdg;
}

}  // namespace qtl

using namespace qtl;

extern "C" {

void qtl_opts_default(qtl_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->method = QTL_TSIT5;
    o->precision = QTL_FP64;
    o->rtol = 1e-8;
    o->atol = 1e-10;
    o->dt0 = 0.0;
    o->dt_min = 0.0;
    o->max_steps = 10000000;
    o->fixed_step = 0;
    o->cluster_size = 0;
    o->dt_fixed = 0.0;
    o->cuda_stream = nullptr;
    o->engine = QTL_ENGINE_AUTO;
    o->shadow_fp64 = 0;
}

const char* qtl_strerror(qtl_status s) {
    switch (s) {
        case QTL_OK: return "ok";
        case QTL_EINVAL: return "invalid argument";
        case QTL_ENOMEM: return "out of device memory";
        case QTL_ESTEP: return "step size underflow, max_steps reached or non-finite error";
        case QTL_ECUDA: return "CUDA error";
        case QTL_ECANCEL: return "cancelled";
        case QTL_EBUSY: return "busy";
        case QTL_ETOOBIG: return "problem too large for the selected kernel";
    }
    return "unknown status";
}

const char* qtl_last_cuda_error(void) { return g_cuda_err.c_str(); }

int64_t qtl_launch_count(void) { return g_launches.load(); }

void qtl_system_free(qtl_system* sys) {
    if (!sys) return;
    System& s = sys->s;
    free_csr(s.dA);
    free_csr(s.dBt);
    cudaFree(s.cmap);
    cudaFree(s.cval64);
    cudaFree(s.cval32);
    free_csr(s.dC);
    free_csr(s.dO);
    free_csr(s.dL);
    free_sell(s.sA);
    free_sell(s.sBt);
    cudaFree(s.units);
    cudaFree(s.odiag);
    cudaFree(s.ew);
    // time-dependent terms: the trajectory kernel's stacked -i H_k, the
    // cluster kernel's Liouvillians, the grid kernel's copies, coefficients
    for (DevSell& d : s.sTa) free_sell(d);
    for (DevSell& d : s.sTb) free_sell(d);
    free_csr(s.dT);
    free_csr(s.dTL);
    cudaFree(s.d_tf);
    cudaFree(s.d_tsl);
    ss_cache_free(s);
    delete sys;
}

qtl_status qtl_system_create(const qtl_op* H, const qtl_op* c_ops, int32_t n_c, const qtl_op* e_ops,
                             int32_t n_e, qtl_system** out) {
    if (!out) return QTL_EINVAL;
    *out = nullptr;
    if (!H || n_c < 0 || n_e < 0 || n_c > 64 || n_e > 64) return QTL_EINVAL;
    if ((n_c > 0 && !c_ops) || (n_e > 0 && !e_ops)) return QTL_EINVAL;
    qtl_system* sys = new qtl_system();
    System& s = sys->s;
    qtl_status st = to_csr(H, 0, s.H);
    if (st != QTL_OK) {
        delete sys;
        return st;
    }
    s.n = s.H.n;
    s.n_c = n_c;
    s.n_e = n_e;
    s.C.resize(n_c);
    s.O.resize(n_e);
    for (int k = 0; k < n_c && st == QTL_OK; ++k) st = to_csr(&c_ops[k], s.n, s.C[k]);
    for (int k = 0; k < n_e && st == QTL_OK; ++k) st = to_csr(&e_ops[k], s.n, s.O[k]);
    if (st != QTL_OK) {
        delete sys;
        return st;
    }
    cudaGetDevice(&s.device);
    Csr G;
    sum_cdagc(s.n, s.C, G);
    build_a_bt(s.H, G, s.A, s.Bt);
    Csr Cs, Os;
    stack(s.C, s.n, Cs);
    stack(s.O, s.n, Os);
    // Collapse operators with at most one entry per row (sigma-, a, projectors,
    // ...): dense per-row column maps for the grid kernel's C rho C^dag.
    bool monomial = s.n_c > 0;
    for (const Csr& c : s.C)
        for (int i = 0; i < s.n && monomial; ++i)
            if (c.rp[i + 1] - c.rp[i] > 1) monomial = false;
    if (monomial) {
        std::vector<int32_t> cmap((size_t)s.n_c * s.n, -1);
        std::vector<double2> cval64((size_t)s.n_c * s.n, make_double2(0.0, 0.0));
        std::vector<float2> cval32((size_t)s.n_c * s.n, make_float2(0.f, 0.f));
        for (int c = 0; c < s.n_c; ++c)
            for (int i = 0; i < s.n; ++i)
                for (int64_t p = s.C[c].rp[i]; p < s.C[c].rp[i + 1]; ++p) {
                    cmap[(size_t)c * s.n + i] = s.C[c].ci[p];
                    cval64[(size_t)c * s.n + i] = make_double2(s.C[c].re[p], s.C[c].im[p]);
                    cval32[(size_t)c * s.n + i] = make_float2((float)s.C[c].re[p], (float)s.C[c].im[p]);
                }
        if ((st = upload(&s.cmap, cmap.data(), cmap.size())) != QTL_OK ||
            (st = upload(&s.cval64, cval64.data(), cval64.size())) != QTL_OK ||
            (st = upload(&s.cval32, cval32.data(), cval32.size())) != QTL_OK) {
            qtl_system_free(sys);
            return st;
        }
    }
    // observables that are real and diagonal (number operators, sigma_z,
    // projectors): their diagonals, for the trajectory kernel's saves
    bool rdiag = s.n_e > 0;
    for (const Csr& o : s.O)
        for (int i = 0; i < s.n && rdiag; ++i)
            for (int64_t p = o.rp[i]; p < o.rp[i + 1] && rdiag; ++p)
                if (o.ci[p] != i || o.im[p] != 0.0) rdiag = false;
    if (rdiag) {
        std::vector<double> d((size_t)s.n_e * s.n, 0.0);
        for (int e = 0; e < s.n_e; ++e)
            for (int i = 0; i < s.n; ++i)
                for (int64_t p = s.O[e].rp[i]; p < s.O[e].rp[i + 1]; ++p) d[(size_t)e * s.n + i] += s.O[e].re[p];
        if ((st = upload(&s.odiag, d.data(), d.size())) != QTL_OK) {
            qtl_system_free(sys);
            return st;
        }
    }
    if ((st = upload_csr(s.A, s.dA)) != QTL_OK || (st = upload_csr(s.Bt, s.dBt)) != QTL_OK ||
        (st = upload_csr(Cs, s.dC)) != QTL_OK ||
        (st = upload_csr(Os, s.dO)) != QTL_OK) {
        qtl_system_free(sys);
        return st;
    }
    *out = sys;
    return QTL_OK;
}

qtl_status qtl_system_add_td(qtl_system* sys, const qtl_op* Hk, const qtl_coef* f) {
    if (!sys || !Hk || !f) return QTL_EINVAL;
    System& s = sys->s;
    if (s.solved || (int)s.Htd.size() >= QTL_MAX_TD) return QTL_EINVAL;
    if (f->kind != QTL_COEF_COS && f->kind != QTL_COEF_EXP) return QTL_EINVAL;
    for (double v : {f->amp_re, f->amp_im, f->omega, f->phi, f->t0, f->sigma})
        if (!std::isfinite(v)) return QTL_EINVAL;
    if (f->sigma < 0.0) return QTL_EINVAL;
    Csr h;
    qtl_status st = to_csr(Hk, s.n, h);
    if (st != QTL_OK) return st;
    s.Htd.push_back(h);
    s.ftd.push_back(*f);
    // -i H_k stacked row-wise for the trajectory kernel, and the coefficients
    std::vector<Csr> scaled(s.Htd.size());
    for (size_t k = 0; k < s.Htd.size(); ++k) {
        scaled[k] = s.Htd[k];
        for (int64_t p = 0; p < scaled[k].nnz(); ++p) {
            const double re = s.Htd[k].re[p], im = s.Htd[k].im[p];
            scaled[k].re[p] = im;
            scaled[k].im[p] = -re;
        }
    }
    Csr stacked;
    stack(scaled, s.n, stacked);
    // the earlier terms keep their device copies unless the new ones are complete
    DevCsr nT;
    decltype(s.d_tf) ntf = nullptr;
    if ((st = upload_csr(stacked, nT)) != QTL_OK || (st = upload(&ntf, s.ftd.data(), s.ftd.size())) != QTL_OK) {
        free_csr(nT);
        s.Htd.pop_back();
        s.ftd.pop_back();
        return st;
    }
    free_csr(s.dT);
    cudaFree(s.d_tf);
    s.dT = nT;
    s.d_tf = ntf;
    return QTL_OK;
}

qtl_status qtl_sesolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt,
                       const qtl_opts* opts, qtl_c128* expect_out, qtl_stats* stats) {
    if (!sys || !opts) return QTL_EINVAL;
    if (sys->s.n_c != 0) return QTL_EINVAL;
    if (sys->s.n > mc_traj_capacity()) return QTL_ETOOBIG;
    qtl_opts o = *opts;
    o.engine = QTL_ENGINE_AUTO;
    return qtl_mcsolve(sys, psi0, tlist, nt, 1, 0, 0, &o, expect_out, nullptr, stats);
}

qtl_status qtl_ssesolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt, int32_t ntraj,
                        uint64_t seed, const qtl_opts* opts, qtl_c128* expect_out, double* meas_out,
                        qtl_stats* stats, qtl_c128* traj_expect_out, double* traj_meas_out) {
    if (!sys || !psi0 || !tlist || nt < 1 || ntraj < 1 || !meas_out) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    if (!opts->fixed_step || opts->precision != QTL_FP64) return QTL_EINVAL;
    System& s = sys->s;
    if (s.n_c < 1 || s.n_c > SSE_MAXSC || !s.Htd.empty()) return QTL_EINVAL;
    if (s.n_e > 0 && !expect_out) return QTL_EINVAL;
    if (s.n > 1024) return QTL_ETOOBIG;
    if ((st = check_tlist_host(tlist, nt)) != QTL_OK) return st;
    if ((st = check_fixed_steps(tlist, nt, opts)) != QTL_OK) return st;
    for (int i = 0; i < s.n; ++i)
        if (!finite_c(psi0[i])) return QTL_EINVAL;
    s.solved = true;
    const size_t n = (size_t)s.n, ne = (size_t)s.n_e * nt, nm = (size_t)s.n_c * nt;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = (off + b + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_psi = take(n * 16), o_tl = take((size_t)nt * 8), o_te = take(ne * ntraj * 16),
                 o_tm = take(nm * ntraj * 16), o_ex = take(ne * 16), o_ms = take(nm * 16),
                 o_inf = take(sizeof(qtl_device_info));
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    char* buf = nullptr;
    QTL_CUDA(qtl_malloc_async((void**)&buf, off, stream));
    McJob J;
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.aseg = s.dA.seg;
    J.aci = s.dA.ci;
    J.av64 = s.dA.v64;
    J.n_c = s.n_c;
    J.crp = s.dC.rp;
    J.cci = s.dC.ci;
    J.cv = s.dC.v64;
    J.n_e = s.n_e;
    J.orp = s.dO.rp;
    J.oci = s.dO.ci;
    J.ov = s.dO.v64;
    J.tlist = (const double*)(buf + o_tl);
    J.nt = nt;
    J.psi0 = (const double2*)(buf + o_psi);
    J.ntraj = ntraj;
    J.seed = seed;
    J.traj_expect = (double2*)(buf + o_te);
    J.expect = (double2*)(buf + o_ex);
    J.traj_meas = (double2*)(buf + o_tm);
    J.meas = (double2*)(buf + o_ms);
    J.info = (qtl_device_info*)(buf + o_inf);
    J.dt_fixed = opts->dt_fixed;
    cudaError_t e;
    std::vector<qtl_c128> mh(nm);
    qtl_device_info info;
    std::memset(&info, 0, sizeof(info));
    if ((e = cudaMemcpyAsync(buf + o_psi, psi0, n * 16, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_tl, tlist, (size_t)nt * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(buf + o_inf, 0, sizeof(qtl_device_info), stream)) != cudaSuccess ||
        (e = launch_sse_traj(J, stream)) != cudaSuccess ||
        (ne > 0 && (e = cudaMemcpyAsync(expect_out, buf + o_ex, ne * 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(mh.data(), buf + o_ms, nm * 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&info, buf + o_inf, sizeof(info), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) {
        set_cuda_error(e);
        cudaFreeAsync(buf, stream);
        cudaStreamSynchronize(stream);
        return QTL_ECUDA;
    }
    // per-trajectory values, [(k * nt + t) * ntraj + j]
    std::vector<qtl_c128> tmh(traj_meas_out ? nm * ntraj : 0);
    if (traj_expect_out && ne > 0)
        QTL_CUDA(cudaMemcpyAsync(traj_expect_out, buf + o_te, ne * ntraj * 16, cudaMemcpyDeviceToHost, stream));
    if (traj_meas_out)
        QTL_CUDA(cudaMemcpyAsync(tmh.data(), buf + o_tm, nm * ntraj * 16, cudaMemcpyDeviceToHost, stream));
    cudaFreeAsync(buf, stream);
    QTL_CUDA(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < nm; ++i) meas_out[i] = mh[i].re;
    for (size_t i = 0; i < tmh.size(); ++i) traj_meas_out[i] = tmh[i].re;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->steps_acc = info.steps_acc;
    }
    return QTL_OK;
}

qtl_status qtl_smesolve(qtl_system* sys, int32_t n_sc, const qtl_c128* psi0, const double* tlist, int32_t nt,
                        int32_t ntraj, uint64_t seed, const qtl_opts* opts, qtl_c128* expect_out, double* meas_out,
                        qtl_stats* stats, qtl_c128* traj_expect_out, double* traj_meas_out) {
    if (!sys || !psi0 || !tlist || nt < 1 || ntraj < 1 || !meas_out) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    if (!opts->fixed_step || opts->precision != QTL_FP64) return QTL_EINVAL;
    System& s = sys->s;
    if (n_sc < 1 || n_sc > SSE_MAXSC || n_sc > s.n_c || !s.Htd.empty()) return QTL_EINVAL;
    if (s.n_e > 0 && !expect_out) return QTL_EINVAL;
    if ((int64_t)s.n * s.n > 4096) return QTL_ETOOBIG;
    if ((st = check_tlist_host(tlist, nt)) != QTL_OK) return st;
    if ((st = check_fixed_steps(tlist, nt, opts)) != QTL_OK) return st;
    for (int i = 0; i < s.n; ++i)
        if (!finite_c(psi0[i])) return QTL_EINVAL;
    s.solved = true;
    if ((st = ensure_liouvillian(s)) != QTL_OK) return st;
    const size_t n = (size_t)s.n, ne = (size_t)s.n_e * nt, nm = (size_t)n_sc * nt;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = (off + b + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_psi = take(n * 16), o_tl = take((size_t)nt * 8), o_te = take(ne * ntraj * 16),
                 o_tm = take(nm * ntraj * 16), o_ex = take(ne * 16), o_ms = take(nm * 16),
                 o_inf = take(sizeof(qtl_device_info));
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    char* buf = nullptr;
    QTL_CUDA(qtl_malloc_async((void**)&buf, off, stream));
    McJob J;
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.aseg = s.dL.seg;   // the Liouvillian of H and of every collapse operator
    J.aci = s.dL.ci;
    J.av64 = s.dL.v64;
    J.n_c = n_sc;        // the measured operators: the last n_sc collapse operators
    J.crp = s.dC.rp + (size_t)(s.n_c - n_sc) * s.n;
    J.cci = s.dC.ci;
    J.cv = s.dC.v64;
    J.n_e = s.n_e;
    J.ew = s.ew;
    J.tlist = (const double*)(buf + o_tl);
    J.nt = nt;
    J.psi0 = (const double2*)(buf + o_psi);
    J.ntraj = ntraj;
    J.seed = seed;
    J.traj_expect = (double2*)(buf + o_te);
    J.expect = (double2*)(buf + o_ex);
    J.traj_meas = (double2*)(buf + o_tm);
    J.meas = (double2*)(buf + o_ms);
    J.info = (qtl_device_info*)(buf + o_inf);
    J.dt_fixed = opts->dt_fixed;
    cudaError_t e;
    std::vector<qtl_c128> mh(nm);
    qtl_device_info info;
    std::memset(&info, 0, sizeof(info));
    if ((e = cudaMemcpyAsync(buf + o_psi, psi0, n * 16, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(buf + o_tl, tlist, (size_t)nt * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(buf + o_inf, 0, sizeof(qtl_device_info), stream)) != cudaSuccess ||
        (e = launch_sme_traj(J, stream)) != cudaSuccess ||
        (ne > 0 && (e = cudaMemcpyAsync(expect_out, buf + o_ex, ne * 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(mh.data(), buf + o_ms, nm * 16, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&info, buf + o_inf, sizeof(info), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) {
        set_cuda_error(e);
        cudaFreeAsync(buf, stream);
        cudaStreamSynchronize(stream);
        return QTL_ECUDA;
    }
    // per-trajectory values, [(k * nt + t) * ntraj + j]
    std::vector<qtl_c128> tmh(traj_meas_out ? nm * ntraj : 0);
    if (traj_expect_out && ne > 0)
        QTL_CUDA(cudaMemcpyAsync(traj_expect_out, buf + o_te, ne * ntraj * 16, cudaMemcpyDeviceToHost, stream));
    if (traj_meas_out)
        QTL_CUDA(cudaMemcpyAsync(tmh.data(), buf + o_tm, nm * ntraj * 16, cudaMemcpyDeviceToHost, stream));
    cudaFreeAsync(buf, stream);
    QTL_CUDA(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < nm; ++i) meas_out[i] = mh[i].re;
    for (size_t i = 0; i < tmh.size(); ++i) traj_meas_out[i] = tmh[i].re;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->steps_acc = info.steps_acc;
    }
    return QTL_OK;
}

int32_t qtl_system_dim(const qtl_system* sys) { return sys ? sys->s.n : 0; }

int64_t qtl_system_liouvillian_nnz(const qtl_system* sys) { return sys ? sys->s.dL.nnz : 0; }

int64_t qtl_system_nnz(const qtl_system* sys, int32_t which) {
    if (!sys) return -1;
    switch (which) {
        case 0: return sys->s.H.nnz();
        case 1: return sys->s.A.nnz();
        case 2: return sys->s.dL.nnz;
        case 3: return sys->s.dA.nnz_half;
        case 4: return sys->s.dL.nnz_half;
    }
    return -1;
}

qtl_status qtl_mesolve_async(qtl_system* sys, const qtl_c128* state0_dev, int32_t is_ket,
                             const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                             qtl_c128* expect_dev, qtl_c128* states_dev, qtl_device_info* info_dev) {
    if (!sys || !state0_dev || !tlist_dev || nt < 1 || !info_dev) return QTL_EINVAL;
    if (sys->s.n_e > 0 && !expect_dev) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    System& s = sys->s;
    if (s.n > 46340) return QTL_ETOOBIG;
    s.solved = true;
    {
        // time-dependent H: the cluster kernel (FP64 or mixed) when it fits,
        // else the grid kernel (FP64)
        // engine: the cluster kernel when the problem fits one cluster
        const int64_t L64 = (int64_t)s.n * s.n;
        bool grid = opts->engine == QTL_ENGINE_GRID ||
                    (opts->engine == QTL_ENGINE_AUTO && L64 > me_cluster_capacity());
        if (!grid && opts->engine == QTL_ENGINE_AUTO) {
            if ((st = ensure_liouvillian(s)) != QTL_OK) return st;
            int C = 0, rpt = 0;
            me_plan((int)L64, opts->cluster_size, &C, &rpt);
            grid = cta_nnz_max_of(s, C) > me_smem_nnz_budget(opts->precision, rpt);
        }
        if (grid) {
            if (!s.Htd.empty() && opts->precision != QTL_FP64) return QTL_EINVAL;
            return mesolve_grid(s, state0_dev, is_ket, tlist_dev, nt, opts, expect_dev, states_dev, info_dev);
        }
    }
    if ((st = ensure_liouvillian(s)) != QTL_OK) return st;
    if (!s.Htd.empty() && (st = ensure_td_liouvillian(s)) != QTL_OK) return st;
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    const int L = s.n * s.n;
    // Largest number of Liouvillian entries in one CTA's rows (CTA c owns the
    // rows r = c mod C): sizes the shared-memory copy of the operator.
    int C = 0, rpt = 0;
    if (!me_plan(L, opts->cluster_size, &C, &rpt)) return QTL_ETOOBIG;
    std::vector<int64_t> per(C, 0);
    for (int r = 0; r < L; ++r) per[r % C] += s.L_rp[r + 1] - s.L_rp[r];
    const int64_t need = *std::max_element(per.begin(), per.end());
    if (need > me_smem_nnz_budget(opts->precision, rpt)) return QTL_ETOOBIG;
    char* scratch = nullptr;
    const size_t epart_bytes = (size_t)nt * C * 2 * (s.n_e > 0 ? s.n_e : 1) * sizeof(double);
    // mixed precision with time-dependent terms: L_k y of y and y_new (FP64)
    const size_t tdg_bytes =
        opts->precision == QTL_MIXED ? (size_t)2 * s.Htd.size() * (size_t)L * sizeof(double2) : 0;
    const size_t bytes = epart_bytes + sizeof(MeJob) + 512 + tdg_bytes + 256;
    QTL_CUDA(qtl_malloc_async((void**)&scratch, bytes, stream));
    MeJob J;
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.L = L;
    J.seg = s.dL.seg;
    J.ci = s.dL.ci;
    J.lv64 = s.dL.v64;
    J.lv32 = s.dL.v32;
    J.n_e = s.n_e;
    J.ew = s.ew;
    J.tlist = tlist_dev;
    J.nt = nt;
    J.state0 = (const double2*)state0_dev;
    J.is_ket = is_ket ? 1 : 0;
    J.epart = (double*)scratch;
    MeJob* jd = (MeJob*)(scratch + ((epart_bytes + 255) & ~(size_t)255));
    J.expect = (double2*)expect_dev;
    J.states = (double2*)states_dev;
    J.info = info_dev;
    J.rtol = opts->rtol;
    J.atol = opts->atol;
    J.dt0 = opts->dt0;
    J.dt_min = opts->dt_min;
    J.dt_fixed = opts->dt_fixed;
    J.max_steps = opts->max_steps;
    J.fixed = opts->fixed_step ? 1 : 0;
    J.method = opts->method;
    J.smem_nnz = (int)need;
    J.n_td = (int)s.Htd.size();
    J.trp = s.dTL.rp;
    J.tci = s.dTL.ci;
    J.tv = s.dTL.v64;
    J.tf = s.d_tf;
    if (tdg_bytes)
        J.tdg = (double2*)(scratch + ((((epart_bytes + 255) & ~(size_t)255) + sizeof(MeJob) + 255) & ~(size_t)255));
    QTL_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(qtl_device_info), stream));
    QTL_CUDA(cudaMemcpyAsync(jd, &J, sizeof(J), cudaMemcpyHostToDevice, stream));
    cudaError_t e = launch_me_cluster(jd, 1, L, J.smem_nnz, opts->precision, opts->cluster_size, nullptr, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        cudaFreeAsync(scratch, stream);
        return e == cudaErrorInvalidValue ? QTL_ETOOBIG : QTL_ECUDA;
    }
    QTL_CUDA(cudaFreeAsync(scratch, stream));
    return QTL_OK;
}

// ---------------------------------------------------------------- batches
namespace {

// Streams forked from the caller's stream for concurrent launch plans
// (created once per device).
std::mutex g_fork_mu;
std::vector<cudaStream_t> g_fork[64];

qtl_status fork_streams(int k, cudaStream_t** out) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return QTL_EINVAL;
    std::lock_guard<std::mutex> lk(g_fork_mu);
    while ((int)g_fork[dev].size() < k) {
        cudaStream_t s;
        QTL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        g_fork[dev].push_back(s);
    }
    *out = g_fork[dev].data();
    return QTL_OK;
}

}  // namespace


extern "C" qtl_status qtl_mesolve_batch_async(qtl_system* const* systems, int32_t nb,
                                              const qtl_c128* const* state0_dev, const int32_t* is_ket,
                                              const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                                              qtl_c128* const* expect_dev, qtl_device_info* info_dev) {
    if (!systems || nb < 1 || !state0_dev || !is_ket || !tlist_dev || nt < 1 || !expect_dev || !info_dev)
        return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    struct Plan {
        int C, rpt;
        int64_t need;
    };
    std::vector<Plan> plan(nb);
    for (int b = 0; b < nb; ++b) {
        if (!systems[b] || !state0_dev[b] || (systems[b]->s.n_e > 0 && !expect_dev[b])) return QTL_EINVAL;
        System& s = systems[b]->s;
        s.solved = true;
        if ((st = ensure_liouvillian(s)) != QTL_OK) return st;
        if (!s.Htd.empty() && (st = ensure_td_liouvillian(s)) != QTL_OK) return st;
        const int L = s.n * s.n;
        batch_plan(L, &plan[b].C, &plan[b].rpt);
        plan[b].need = cta_nnz_max(s, plan[b].C);
        if (plan[b].need > me_smem_nnz_budget(opts->precision, plan[b].rpt)) return QTL_ETOOBIG;
    }
    // buckets of equal plans, jobs ordered by decreasing Liouvillian size
    std::vector<std::pair<int, int>> keys;
    for (int b = 0; b < nb; ++b) {
        std::pair<int, int> k(plan[b].C, plan[b].rpt);
        if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
    const int nk = (int)keys.size();
    std::vector<std::vector<int>> bucket(nk);
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < nk; ++k)
            if (keys[k] == std::make_pair(plan[b].C, plan[b].rpt)) bucket[k].push_back(b);
    for (auto& v : bucket)
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
            return systems[x]->s.dL.nnz > systems[y]->s.dL.nnz;
        });
    // scratch: jobs (bucket order), per-job expectation partials, counters
    std::vector<size_t> ep_off(nb), tdg_off(nb);
    size_t off = ((size_t)nb * sizeof(MeJob) + 255) & ~(size_t)255;
    const size_t cnt_off = off;
    off += ((size_t)nk * sizeof(int) + 255) & ~(size_t)255;
    for (int b = 0; b < nb; ++b) {
        ep_off[b] = off;
        const int ne = systems[b]->s.n_e > 0 ? systems[b]->s.n_e : 1;
        off += (((size_t)nt * plan[b].C * 2 * ne * sizeof(double)) + 255) & ~(size_t)255;
        tdg_off[b] = off;
        off += (me_tdg_bytes(systems[b]->s, opts->precision) + 255) & ~(size_t)255;
    }
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    char* scratch = nullptr;
    QTL_CUDA(qtl_malloc_async((void**)&scratch, off, stream));
    std::vector<MeJob> jobs(nb);
    std::vector<int> first(nk + 1, 0);
    int q = 0;
    for (int k = 0; k < nk; ++k) {
        first[k] = q;
        for (int b : bucket[k])
            me_job_fill(jobs[q++], systems[b]->s, tlist_dev, nt, state0_dev[b], is_ket[b],
                        (double*)(scratch + ep_off[b]), expect_dev[b], info_dev + b, opts, 0,
                        me_tdg_bytes(systems[b]->s, opts->precision) ? (double2*)(scratch + tdg_off[b]) : nullptr);
    }
    first[nk] = q;
    for (int k = 0; k < nk; ++k) {
        int64_t need = 0;
        for (int b : bucket[k]) need = std::max(need, plan[b].need);
        for (int j = first[k]; j < first[k + 1]; ++j) jobs[j].smem_nnz = (int)need;
    }
    MeJob* jd = (MeJob*)scratch;
    int* counters = (int*)(scratch + cnt_off);
    cudaError_t e;
    if ((e = cudaMemsetAsync(info_dev, 0, (size_t)nb * sizeof(qtl_device_info), stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(counters, 0, (size_t)nk * sizeof(int), stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(jd, jobs.data(), (size_t)nb * sizeof(MeJob), cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess) {
        set_cuda_error(e);
        cudaFreeAsync(scratch, stream);
        return QTL_ECUDA;
    }
    cudaStream_t* fs = nullptr;
    if (nk > 1 && (st = fork_streams(nk, &fs)) != QTL_OK) {
        cudaFreeAsync(scratch, stream);
        return st;
    }
    cudaEvent_t fork_ev = nullptr;
    if (nk > 1) {
        cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
        cudaEventRecord(fork_ev, stream);
    }
    e = cudaSuccess;
    for (int k = 0; k < nk && e == cudaSuccess; ++k) {
        cudaStream_t sk = nk > 1 ? fs[k] : stream;
        if (nk > 1) cudaStreamWaitEvent(sk, fork_ev, 0);
        int Lmax = 0;
        for (int b : bucket[k]) Lmax = std::max(Lmax, systems[b]->s.n * systems[b]->s.n);
        e = launch_me_cluster(jd + first[k], first[k + 1] - first[k], Lmax, jobs[first[k]].smem_nnz,
                              opts->precision, keys[k].first, counters + k, sk);
        if (nk > 1) {
            cudaEvent_t done;
            cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
            cudaEventRecord(done, sk);
            cudaStreamWaitEvent(stream, done, 0);
            cudaEventDestroy(done);
        }
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    return QTL_OK;
}

extern "C" qtl_status qtl_mesolve_batch(qtl_system* const* systems, int32_t nb,
                                        const qtl_c128* const* state0, const int32_t* is_ket,
                                        const double* tlist, int32_t nt, const qtl_opts* opts,
                                        qtl_c128* const* expect_out, qtl_stats* stats) {
    if (!systems || nb < 1 || !state0 || !is_ket || !expect_out) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    if ((st = check_tlist_host(tlist, nt)) != QTL_OK) return st;
    std::vector<size_t> s_off(nb), e_off(nb), s_len(nb), e_len(nb);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = (off + b + 255) & ~(size_t)255;
        return o;
    };
    const size_t tl_off = take((size_t)nt * 8);
    const size_t info_off = take((size_t)nb * sizeof(qtl_device_info));
    for (int b = 0; b < nb; ++b) {
        if (!systems[b] || !state0[b]) return QTL_EINVAL;
        const System& s = systems[b]->s;
        s_len[b] = (is_ket[b] ? (size_t)s.n : (size_t)s.n * s.n) * 16;
        for (size_t i = 0; i < s_len[b] / 16; ++i)
            if (!finite_c(state0[b][i])) return QTL_EINVAL;
        e_len[b] = (size_t)s.n_e * nt * 16;
        s_off[b] = take(s_len[b]);
        e_off[b] = take(e_len[b]);
    }
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    char* buf = nullptr;
    QTL_CUDA(qtl_malloc_async((void**)&buf, off, stream));
    std::vector<const qtl_c128*> sd(nb);
    std::vector<qtl_c128*> ed(nb);
    QTL_CUDA(cudaMemcpyAsync(buf + tl_off, tlist, (size_t)nt * 8, cudaMemcpyHostToDevice, stream));
    for (int b = 0; b < nb; ++b) {
        sd[b] = (const qtl_c128*)(buf + s_off[b]);
        ed[b] = (qtl_c128*)(buf + e_off[b]);
        QTL_CUDA(cudaMemcpyAsync(buf + s_off[b], state0[b], s_len[b], cudaMemcpyHostToDevice, stream));
    }
    st = qtl_mesolve_batch_async(systems, nb, sd.data(), is_ket, (const double*)(buf + tl_off), nt, opts,
                                 ed.data(), (qtl_device_info*)(buf + info_off));
    if (st != QTL_OK) {
        cudaFreeAsync(buf, stream);
        return st;
    }
    std::vector<qtl_device_info> info(nb);
    for (int b = 0; b < nb; ++b)
        if (e_len[b]) QTL_CUDA(cudaMemcpyAsync(expect_out[b], buf + e_off[b], e_len[b], cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaMemcpyAsync(info.data(), buf + info_off, (size_t)nb * sizeof(qtl_device_info),
                             cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaFreeAsync(buf, stream));
    QTL_CUDA(cudaStreamSynchronize(stream));
    qtl_status first_bad = QTL_OK;
    for (int b = 0; b < nb; ++b) {
        if (stats) {
            stats[b].steps_acc = info[b].steps_acc;
            stats[b].steps_rej = info[b].steps_rej;
            stats[b].rhs_evals = info[b].rhs_evals;
            stats[b].jumps = info[b].jumps;
            stats[b].err_vs_fp64 = opts->precision == QTL_FP64 ? 0.0 : -1.0;
        }
        if (first_bad == QTL_OK && info[b].status != QTL_OK) first_bad = (qtl_status)info[b].status;
    }
    return first_bad;
}

qtl_status qtl_mesolve(qtl_system* sys, const qtl_c128* state0, int32_t is_ket, const double* tlist,
                       int32_t nt, const qtl_opts* opts, qtl_c128* expect_out, qtl_c128* states_out,
                       qtl_stats* stats) {
    if (!sys || !state0) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    if ((st = check_tlist_host(tlist, nt)) != QTL_OK) return st;
    System& s = sys->s;
    if (s.n_e > 0 && !expect_out) return QTL_EINVAL;
    const size_t n0 = is_ket ? (size_t)s.n : (size_t)s.n * s.n;
    for (size_t i = 0; i < n0; ++i)
        if (!finite_c(state0[i])) return QTL_EINVAL;
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    const size_t L = (size_t)s.n * s.n;
    const size_t ne = (size_t)s.n_e * nt;
    char* buf = nullptr;
    const size_t bytes = n0 * 16 + (size_t)nt * 8 + ne * 16 + (states_out ? (size_t)nt * L * 16 : 0) +
                         sizeof(qtl_device_info) + 5 * 256;
    QTL_CUDA(qtl_malloc_async((void**)&buf, bytes, stream));
    size_t off = 0;
    auto carve = [&](size_t b) {
        char* p = buf + off;
        off = (off + b + 255) & ~(size_t)255;
        return p;
    };
    qtl_c128* d_state = (qtl_c128*)carve(n0 * 16);
    double* d_tl = (double*)carve((size_t)nt * 8);
    qtl_c128* d_ex = (qtl_c128*)carve(ne * 16);
    qtl_c128* d_states = states_out ? (qtl_c128*)carve((size_t)nt * L * 16) : nullptr;
    qtl_device_info* d_info = (qtl_device_info*)carve(sizeof(qtl_device_info));
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_state, state0, n0 * 16, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_tl, tlist, (size_t)nt * 8, cudaMemcpyHostToDevice, stream)) != cudaSuccess) {
        set_cuda_error(e);
        cudaFreeAsync(buf, stream);
        return QTL_ECUDA;
    }
    if (ne) cudaMemsetAsync(d_ex, 0, ne * 16, stream);
    st = qtl_mesolve_async(sys, d_state, is_ket, d_tl, nt, opts, d_ex, d_states, d_info);
    if (st != QTL_OK) {
        cudaFreeAsync(buf, stream);
        return st;
    }
    qtl_device_info info;
    if (ne) QTL_CUDA(cudaMemcpyAsync(expect_out, d_ex, ne * 16, cudaMemcpyDeviceToHost, stream));
    if (states_out)
        QTL_CUDA(cudaMemcpyAsync(states_out, d_states, (size_t)nt * L * 16, cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(info), cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaFreeAsync(buf, stream));
    QTL_CUDA(cudaStreamSynchronize(stream));
    if (stats) {
        stats->steps_acc = info.steps_acc;
        stats->steps_rej = info.steps_rej;
        stats->rhs_evals = info.rhs_evals;
        stats->jumps = info.jumps;
        stats->err_vs_fp64 = opts->precision == QTL_FP64 ? 0.0 : -1.0;
    }
    if (info.status == QTL_OK && opts->precision == QTL_MIXED && opts->shadow_fp64 && stats) {
        // the same solve in FP64, compared on the host
        qtl_opts o = *opts;
        o.precision = QTL_FP64;
        o.shadow_fp64 = 0;
        std::vector<qtl_c128> ref(ne > 0 ? ne : 1);
        qtl_stats rs{};
        if (qtl_mesolve(sys, state0, is_ket, tlist, nt, &o, ref.data(), nullptr, &rs) == QTL_OK)
            stats->err_vs_fp64 = max_abs_diff(expect_out, ref.data(), ne);
    }
    return (qtl_status)info.status;
}

qtl_status qtl_mcsolve_async(qtl_system* sys, const qtl_c128* psi0_dev, const double* tlist_dev,
                             int32_t nt, int32_t ntraj, uint64_t seed, int64_t traj_offset,
                             const qtl_opts* opts, qtl_c128* expect_dev, qtl_c128* traj_expect_dev,
                             qtl_device_info* info_dev) {
    if (!sys || !psi0_dev || !tlist_dev || nt < 1 || ntraj < 1 || !info_dev || traj_offset < 0)
        return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    System& s = sys->s;
    if (s.n_e > 0 && !expect_dev) return QTL_EINVAL;
    if (s.n > mc_wide_capacity()) return QTL_ETOOBIG;
    if (opts->engine == QTL_ENGINE_CLUSTER && s.n > mc_traj_capacity()) return QTL_ETOOBIG;
    const bool wide = s.n > mc_traj_capacity() || opts->engine == QTL_ENGINE_GRID;
    // time-dependent terms above the register-resident size: FP64 only
    if (wide && !s.Htd.empty() && opts->precision != QTL_FP64) return QTL_EINVAL;
    s.solved = true;
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    const size_t ne = (size_t)s.n_e * nt;
    double2* scratch = nullptr;
    if (!traj_expect_dev && ne > 0) {
        QTL_CUDA(qtl_malloc_async((void**)&scratch, ne * ntraj * sizeof(double2), stream));
    }
    McJob J;
    std::memset(&J, 0, sizeof(J));
    J.n = s.n;
    J.a_nnz = (int)s.dA.nnz;
    J.aseg = s.dA.seg;
    J.arp = s.dA.rp;
    J.aci = s.dA.ci;
    J.av64 = s.dA.v64;
    J.av32 = s.dA.v32;
    J.n_c = s.n_c;
    J.crp = s.dC.rp;
    J.cci = s.dC.ci;
    J.cv = s.dC.v64;
    J.n_e = s.n_e;
    J.orp = s.dO.rp;
    J.oci = s.dO.ci;
    J.ov = s.dO.v64;
    J.oseg = s.dO.seg;
    J.odiag = s.odiag;
    J.tlist = tlist_dev;
    J.nt = nt;
    J.psi0 = (const double2*)psi0_dev;
    J.n_td = (int)s.Htd.size();
    J.tseg = s.dT.seg;
    J.tci = s.dT.ci;
    J.tv64 = s.dT.v64;
    J.tv32 = s.dT.v32;
    J.tf = s.d_tf;
    J.ntraj = ntraj;
    J.seed = seed;
    J.traj_offset = traj_offset;
    J.traj_expect = traj_expect_dev ? (double2*)traj_expect_dev : scratch;
    J.expect = (double2*)expect_dev;
    J.info = info_dev;
    J.rtol = opts->rtol;
    J.atol = opts->atol;
    J.dt0 = opts->dt0;
    J.dt_min = opts->dt_min;
    J.dt_fixed = opts->dt_fixed;
    J.max_steps = opts->max_steps;
    J.fixed = opts->fixed_step ? 1 : 0;
    J.method = opts->method;
    QTL_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(qtl_device_info), stream));
    cudaError_t e = cudaSuccess;
    if (wide) {
        // per-CTA integrator state in global memory (psi does not fit on chip)
        if ((st = ensure_sell(s)) != QTL_OK || (st = ensure_td_sell(s)) != QTL_OK) {
            if (scratch) cudaFreeAsync(scratch, stream);
            return st;
        }
        J.tsl = s.d_tsl;
        J.sl = s.sA.sl;
        J.sdesc = s.sA.desc;
        SellConst cdesc;
        std::memset(&cdesc, 0, sizeof(cdesc));
        J.sdesc_const = !s.sA.hdesc.empty();
        if (J.sdesc_const) std::memcpy(cdesc.d, s.sA.hdesc.data(), s.sA.hdesc.size() * sizeof(int4));
        J.sidx16 = s.sA.idx16;
        J.sci = s.sA.ci;
        J.svs64 = s.sA.vs64;
        J.svs32 = s.sA.vs32;
        J.svc64 = s.sA.vc64;
        J.svc32 = s.sA.vc32;
        J.svs32lo = s.sA.vs32lo;
        J.svc32lo = s.sA.vc32lo;
        McWidePlan plan;
        void* wscr = nullptr;
        e = mc_wide_plan(J, opts->precision, &plan);
        if (e == cudaSuccess && qtl_malloc_async(&wscr, plan.scratch_bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            if (scratch) cudaFreeAsync(scratch, stream);
            return QTL_ENOMEM;
        }
        if (e == cudaSuccess) e = launch_mc_wide(J, opts->precision, plan, wscr, &cdesc, stream);
        if (wscr) cudaFreeAsync(wscr, stream);
    } else {
        e = launch_mc_traj(J, opts->precision, stream);
    }
    if (e == cudaSuccess) e = launch_mc_reduce(J, stream);
    if (scratch) cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    return QTL_OK;
}

qtl_status qtl_mcsolve(qtl_system* sys, const qtl_c128* psi0, const double* tlist, int32_t nt,
                       int32_t ntraj, uint64_t seed, int64_t traj_offset, const qtl_opts* opts,
                       qtl_c128* expect_out, qtl_c128* traj_expect_out, qtl_stats* stats) {
    if (!sys || !psi0) return QTL_EINVAL;
    qtl_status st = check_opts(opts);
    if (st != QTL_OK) return st;
    if ((st = check_tlist_host(tlist, nt)) != QTL_OK) return st;
    System& s = sys->s;
    if (ntraj < 1 || (s.n_e > 0 && !expect_out)) return QTL_EINVAL;
    for (int i = 0; i < s.n; ++i)
        if (!finite_c(psi0[i])) return QTL_EINVAL;
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    const size_t ne = (size_t)s.n_e * nt;
    char* buf = nullptr;
    const size_t bytes = (size_t)s.n * 16 + (size_t)nt * 8 + ne * 16 + ne * ntraj * 16 +
                         sizeof(qtl_device_info) + 5 * 256;
    QTL_CUDA(qtl_malloc_async((void**)&buf, bytes, stream));
    size_t off = 0;
    auto carve = [&](size_t b) {
        char* p = buf + off;
        off = (off + b + 255) & ~(size_t)255;
        return p;
    };
    qtl_c128* d_psi = (qtl_c128*)carve((size_t)s.n * 16);
    double* d_tl = (double*)carve((size_t)nt * 8);
    qtl_c128* d_ex = (qtl_c128*)carve(ne * 16);
    qtl_c128* d_tex = (qtl_c128*)carve(ne * ntraj * 16);
    qtl_device_info* d_info = (qtl_device_info*)carve(sizeof(qtl_device_info));
    QTL_CUDA(cudaMemcpyAsync(d_psi, psi0, (size_t)s.n * 16, cudaMemcpyHostToDevice, stream));
    QTL_CUDA(cudaMemcpyAsync(d_tl, tlist, (size_t)nt * 8, cudaMemcpyHostToDevice, stream));
    st = qtl_mcsolve_async(sys, d_psi, d_tl, nt, ntraj, seed, traj_offset, opts, d_ex, d_tex, d_info);
    if (st != QTL_OK) {
        cudaFreeAsync(buf, stream);
        return st;
    }
    qtl_device_info info;
    if (ne) QTL_CUDA(cudaMemcpyAsync(expect_out, d_ex, ne * 16, cudaMemcpyDeviceToHost, stream));
    if (traj_expect_out && ne)
        QTL_CUDA(cudaMemcpyAsync(traj_expect_out, d_tex, ne * ntraj * 16, cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(info), cudaMemcpyDeviceToHost, stream));
    QTL_CUDA(cudaFreeAsync(buf, stream));
    QTL_CUDA(cudaStreamSynchronize(stream));
    if (stats) {
        stats->steps_acc = info.steps_acc;
        stats->steps_rej = info.steps_rej;
        stats->rhs_evals = info.rhs_evals;
        stats->jumps = info.jumps;
        stats->err_vs_fp64 = opts->precision == QTL_FP64 ? 0.0 : -1.0;
    }
    if (info.status == QTL_OK && opts->precision == QTL_MIXED && opts->shadow_fp64 && stats) {
        // the same trajectories (same seed and offset) in FP64
        qtl_opts o = *opts;
        o.precision = QTL_FP64;
        o.shadow_fp64 = 0;
        std::vector<qtl_c128> ref(ne > 0 ? ne : 1);
        qtl_stats rs{};
        if (qtl_mcsolve(sys, psi0, tlist, nt, ntraj, seed, traj_offset, &o, ref.data(), nullptr, &rs) == QTL_OK)
            stats->err_vs_fp64 = max_abs_diff(expect_out, ref.data(), ne);
    }
    return (qtl_status)info.status;
}

}  // extern "C"
