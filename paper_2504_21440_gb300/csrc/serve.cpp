// Request server (qtl_server_*): a queue of mesolve / mcsolve requests
// admitted in arrival order while their estimated device memory fits an HBM
// budget, each admitted request running on its own CUDA stream so that work
// from requests that arrived at different times overlaps on the GPU.  A
// request whose kernel occupies every SM (the cooperative grid mesolve, the
// one-CTA-per-SM wide trajectory kernel) runs alone: overlap gains it
// nothing, and other streams' kernels can hold back a cooperative launch.
// The device structures of a request's system are built by submit, on the
// caller's thread.
//
// One dispatcher thread owns the CUDA work: it admits requests (device
// buffers from the stream-ordered pool, host->device copies, the _async
// solve, device->host copies into a pinned per-slot staging buffer, the
// stream-ordered free, a completion event), and retires them when their
// event has completed (copy from staging to the caller's buffer, release of
// the budget and the slot).  Submit / poll / wait / cancel only touch the
// queue under a mutex.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace qtl {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
    uint64_t ticket = 0;
    qtl_request r{};
    qtl_c128* expect_out = nullptr;
    size_t bytes = 0;
    size_t ex_bytes = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int fills_gpu = 0;  // runs alone: its kernel occupies every SM
    int batch = 0;      // a cluster-kernel mesolve: runs through the batched launch
    int slot = -1;
    size_t stage_off = 0;  // its [info | expect] in the slot's pinned staging
    qtl_result res{};
};

struct SrvSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* pinned = nullptr;   // staging: device info, then the expectation values
    size_t pinned_bytes = 0;
    SrvReq* req = nullptr;            // a request run alone, or
    std::vector<SrvReq*> group;       // requests sharing one batched launch
    bool busy() const { return req || !group.empty(); }
};

}  // namespace qtl

struct qtl_server {
    int device = 0;
    size_t budget = 0, in_use = 0;
    std::vector<qtl::SrvSlot> slots;
    std::deque<uint64_t> queue;
    std::map<uint64_t, qtl::SrvReq*> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    int running = 0;
    int exclusive = 0;   // a request whose kernel fills the GPU is running
};

namespace qtl {

// Device bytes a request will hold while it runs (inputs, outputs and the
// solver's scratch), used for admission.
static size_t request_bytes_one(const qtl_request& r);
static bool wants_shadow(const qtl_request& r) {
    return r.opts.precision == QTL_MIXED && r.opts.shadow_fp64;
}
// With the FP64 shadow both solves' buffers are counted: the shadow runs
// after the reduced-precision solve on the same stream.
static size_t request_bytes(const qtl_request& r) {
    size_t b = request_bytes_one(r);
    if (wants_shadow(r)) {
        qtl_request f = r;
        f.opts.precision = QTL_FP64;
        b += request_bytes_one(f);
    }
    return b;
}

static size_t request_bytes_one(const qtl_request& r) {
    const System& s = r.sys->s;
    const size_t n = (size_t)s.n, L = n * n, nt = (size_t)r.nt, ne = (size_t)(s.n_e > 0 ? s.n_e : 1);
    const size_t t2 = r.opts.precision == QTL_MIXED ? 8 : 16;
    size_t b = (r.is_ket || r.kind == QTL_REQ_MCSOLVE ? n : L) * 16 + nt * 8 + ne * nt * 16 + 4096;
    if (r.kind == QTL_REQ_MCSOLVE) {
        b += ne * nt * (size_t)r.ntraj * 16;
        if (s.n > mc_traj_capacity()) {
            McJob J{};
            J.n = s.n;
            J.n_e = s.n_e;
            J.n_c = s.n_c;
            J.ntraj = r.ntraj;
            McWidePlan p{};
            if (mc_wide_plan(J, r.opts.precision, &p) == cudaSuccess) b += p.scratch_bytes;
            else b += (size_t)r.ntraj * 15 * n * 16;
        }
    } else if (L <= (size_t)me_cluster_capacity() && r.opts.engine != QTL_ENGINE_GRID) {
        b += nt * 16 * 2 * ne * 8 + L * 40;  // expectation partials; Liouvillian if built here
    } else {
        b += 2 * L * 16 + 9 * L * t2 + nt * 2 * 304 * ne * 8;
    }
    return b;
}

static void srv_admit(qtl_server* S, SrvReq* q, int slot) {
    SrvSlot& sl = S->slots[slot];
    const System& s = q->r.sys->s;
    cudaStream_t st = sl.stream;
    const size_t n = (size_t)s.n, nt = (size_t)q->r.nt;
    const size_t n0 = (q->r.kind == QTL_REQ_MCSOLVE || q->r.is_ket) ? n : n * n;
    q->ex_bytes = (size_t)s.n_e * nt * 16;
    const bool shadow = wants_shadow(q->r);
    // pinned staging: [info | expect] and, with the shadow, [info | expect] of the FP64 solve
    const size_t stage_b = 64 + ((q->ex_bytes + 63) & ~(size_t)63);
    const size_t need_pinned = shadow ? 2 * stage_b : stage_b;
    q->slot = slot;
    q->state = 1;
    q->res.t_start = now_s();
    sl.req = q;
    qtl_status stt = QTL_OK;
    if (sl.pinned_bytes < need_pinned) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.pinned_bytes = 0;
        if (cudaMallocHost(&sl.pinned, need_pinned) == cudaSuccess) sl.pinned_bytes = need_pinned;
        else stt = QTL_ENOMEM;
    }
    char* dbuf = nullptr;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_st = 0, o_tl = up(n0 * 16), o_ex = o_tl + up(nt * 8), o_inf = o_ex + up(q->ex_bytes + 16);
    const size_t o_ex2 = o_inf + 256, o_inf2 = o_ex2 + up(q->ex_bytes + 16);
    const size_t total = shadow ? o_inf2 + 256 : o_inf + 256;
    if (stt == QTL_OK && qtl_malloc_async((void**)&dbuf, total, st) != cudaSuccess) stt = QTL_ENOMEM;
    if (stt == QTL_OK) {
        cudaMemcpyAsync(dbuf + o_st, q->r.state0, n0 * 16, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dbuf + o_tl, q->r.tlist, nt * 8, cudaMemcpyHostToDevice, st);
        qtl_opts o = q->r.opts;
        o.cuda_stream = st;
        qtl_device_info* dinfo = (qtl_device_info*)(dbuf + o_inf);
        if (q->r.kind == QTL_REQ_MESOLVE)
            stt = qtl_mesolve_async(q->r.sys, (const qtl_c128*)(dbuf + o_st), q->r.is_ket,
                                    (const double*)(dbuf + o_tl), q->r.nt, &o,
                                    (qtl_c128*)(dbuf + o_ex), nullptr, dinfo);
        else
            stt = qtl_mcsolve_async(q->r.sys, (const qtl_c128*)(dbuf + o_st),
                                    (const double*)(dbuf + o_tl), q->r.nt, q->r.ntraj, q->r.seed, 0, &o,
                                    (qtl_c128*)(dbuf + o_ex), nullptr, dinfo);
        if (stt == QTL_OK) {
            cudaMemcpyAsync(sl.pinned, dinfo, sizeof(qtl_device_info), cudaMemcpyDeviceToHost, st);
            if (q->ex_bytes)
                cudaMemcpyAsync((char*)sl.pinned + 64, dbuf + o_ex, q->ex_bytes, cudaMemcpyDeviceToHost, st);
        }
        if (stt == QTL_OK && shadow) {
            // the same request in FP64, after the reduced-precision solve
            qtl_opts f = o;
            f.precision = QTL_FP64;
            f.shadow_fp64 = 0;
            qtl_device_info* dinfo2 = (qtl_device_info*)(dbuf + o_inf2);
            qtl_status s2;
            if (q->r.kind == QTL_REQ_MESOLVE)
                s2 = qtl_mesolve_async(q->r.sys, (const qtl_c128*)(dbuf + o_st), q->r.is_ket,
                                       (const double*)(dbuf + o_tl), q->r.nt, &f,
                                       (qtl_c128*)(dbuf + o_ex2), nullptr, dinfo2);
            else
                s2 = qtl_mcsolve_async(q->r.sys, (const qtl_c128*)(dbuf + o_st),
                                       (const double*)(dbuf + o_tl), q->r.nt, q->r.ntraj, q->r.seed, 0,
                                       &f, (qtl_c128*)(dbuf + o_ex2), nullptr, dinfo2);
            char* p2 = (char*)sl.pinned + stage_b;
            if (s2 == QTL_OK) {
                cudaMemcpyAsync(p2, dinfo2, sizeof(qtl_device_info), cudaMemcpyDeviceToHost, st);
                if (q->ex_bytes)
                    cudaMemcpyAsync(p2 + 64, dbuf + o_ex2, q->ex_bytes, cudaMemcpyDeviceToHost, st);
            } else {
                qtl_device_info fail{};
                fail.status = s2;
                std::memcpy(p2, &fail, sizeof(fail));
            }
        }
        cudaFreeAsync(dbuf, st);
    }
    if (stt != QTL_OK) {
        // nothing to wait for beyond what is already enqueued on the stream
        qtl_device_info fail{};
        fail.status = stt;
        if (sl.pinned) std::memcpy(sl.pinned, &fail, sizeof(fail));
        q->res.status = stt;
    }
    cudaEventRecord(sl.done, st);
}

// Requests that may share one batched launch: mesolve on the cluster kernel
// with the same output times and options.  The batched launch gives each
// solve the plan its own size implies (qtl_mesolve_batch), so a request's
// result is the same bit for bit whether it runs in a group or alone.
static bool batch_compatible(const qtl_request& a, const qtl_request& b) {
    const qtl_opts &x = a.opts, &y = b.opts;
    if (a.nt != b.nt || x.method != y.method || x.precision != y.precision || x.rtol != y.rtol ||
        x.atol != y.atol || x.dt0 != y.dt0 || x.dt_min != y.dt_min || x.max_steps != y.max_steps ||
        x.fixed_step != y.fixed_step || (x.fixed_step && x.dt_fixed != y.dt_fixed))
        return false;
    return std::memcmp(a.tlist, b.tlist, (size_t)a.nt * sizeof(double)) == 0;
}

constexpr int SRV_MAX_GROUP = 64;

static void srv_admit_group(qtl_server* S, const std::vector<SrvReq*>& g, int slot) {
    SrvSlot& sl = S->slots[slot];
    cudaStream_t st = sl.stream;
    const int nb = (int)g.size();
    const SrvReq* q0 = g[0];
    const size_t nt = (size_t)q0->r.nt;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // pinned staging: [info | expect] per request; device: tlist, states, expects, infos
    size_t pin = 0, dev = up(nt * 8);
    std::vector<size_t> o_st(nb), o_ex(nb);
    for (int i = 0; i < nb; ++i) {
        SrvReq* q = g[i];
        const System& s = q->r.sys->s;
        const size_t n0 = q->r.is_ket ? (size_t)s.n : (size_t)s.n * s.n;
        q->ex_bytes = (size_t)s.n_e * nt * 16;
        q->slot = slot;
        q->state = 1;
        q->res.t_start = now_s();
        q->stage_off = pin;
        pin += 64 + ((q->ex_bytes + 63) & ~(size_t)63);
        o_st[i] = dev;
        dev += up(n0 * 16);
        o_ex[i] = dev;
        dev += up(q->ex_bytes + 16);
    }
    const size_t o_inf = dev;
    dev += up((size_t)nb * sizeof(qtl_device_info));
    sl.group = g;
    qtl_status stt = QTL_OK;
    if (sl.pinned_bytes < pin) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.pinned_bytes = 0;
        if (cudaMallocHost(&sl.pinned, pin) == cudaSuccess) sl.pinned_bytes = pin;
        else stt = QTL_ENOMEM;
    }
    char* dbuf = nullptr;
    if (stt == QTL_OK && qtl_malloc_async((void**)&dbuf, dev, st) != cudaSuccess) stt = QTL_ENOMEM;
    if (stt == QTL_OK) {
        cudaMemcpyAsync(dbuf, q0->r.tlist, nt * 8, cudaMemcpyHostToDevice, st);
        std::vector<qtl_system*> sys(nb);
        std::vector<const qtl_c128*> s0(nb);
        std::vector<qtl_c128*> ex(nb);
        std::vector<int32_t> ket(nb);
        for (int i = 0; i < nb; ++i) {
            const SrvReq* q = g[i];
            const System& s = q->r.sys->s;
            const size_t n0 = q->r.is_ket ? (size_t)s.n : (size_t)s.n * s.n;
            cudaMemcpyAsync(dbuf + o_st[i], q->r.state0, n0 * 16, cudaMemcpyHostToDevice, st);
            sys[i] = q->r.sys;
            s0[i] = (const qtl_c128*)(dbuf + o_st[i]);
            ex[i] = (qtl_c128*)(dbuf + o_ex[i]);
            ket[i] = q->r.is_ket;
        }
        qtl_opts o = q0->r.opts;
        o.cuda_stream = st;
        qtl_device_info* dinfo = (qtl_device_info*)(dbuf + o_inf);
        stt = qtl_mesolve_batch_async(sys.data(), nb, s0.data(), ket.data(), (const double*)dbuf, (int32_t)nt,
                                      &o, ex.data(), dinfo);
        if (stt == QTL_OK)
            for (int i = 0; i < nb; ++i) {
                char* p = (char*)sl.pinned + g[i]->stage_off;
                cudaMemcpyAsync(p, dinfo + i, sizeof(qtl_device_info), cudaMemcpyDeviceToHost, st);
                if (g[i]->ex_bytes)
                    cudaMemcpyAsync(p + 64, dbuf + o_ex[i], g[i]->ex_bytes, cudaMemcpyDeviceToHost, st);
            }
        cudaFreeAsync(dbuf, st);
    }
    if (stt != QTL_OK)
        for (SrvReq* q : g) {
            qtl_device_info fail{};
            fail.status = stt;
            if (sl.pinned) std::memcpy((char*)sl.pinned + q->stage_off, &fail, sizeof(fail));
            q->res.status = stt;
        }
    cudaEventRecord(sl.done, st);
}

// one request's results from its staging area
static void srv_finish(qtl_server* S, SrvReq* q, const char* stage) {
    qtl_device_info info{};
    if (stage) std::memcpy(&info, stage, sizeof(info));
    if (q->res.status == QTL_OK || q->res.status == QTL_EBUSY) q->res.status = info.status;
    q->res.stats.steps_acc = info.steps_acc;
    q->res.stats.steps_rej = info.steps_rej;
    q->res.stats.rhs_evals = info.rhs_evals;
    q->res.stats.jumps = info.jumps;
    q->res.stats.err_vs_fp64 = q->r.opts.precision == QTL_FP64 ? 0.0 : -1.0;
    if (q->ex_bytes && q->res.status == QTL_OK && q->expect_out && stage)
        std::memcpy(q->expect_out, stage + 64, q->ex_bytes);
    q->res.t_end = now_s();
    q->state = 2;
    S->in_use -= q->bytes;
}

static void srv_retire(qtl_server* S, int slot) {
    SrvSlot& sl = S->slots[slot];
    if (!sl.group.empty()) {
        for (SrvReq* q : sl.group) srv_finish(S, q, sl.pinned ? (const char*)sl.pinned + q->stage_off : nullptr);
        S->running -= (int)sl.group.size();
        sl.group.clear();
        return;
    }
    SrvReq* q = sl.req;
    qtl_device_info info{};
    if (sl.pinned) std::memcpy(&info, sl.pinned, sizeof(info));
    if (q->res.status == QTL_OK || q->res.status == QTL_EBUSY) q->res.status = info.status;
    q->res.stats.steps_acc = info.steps_acc;
    q->res.stats.steps_rej = info.steps_rej;
    q->res.stats.rhs_evals = info.rhs_evals;
    q->res.stats.jumps = info.jumps;
    q->res.stats.err_vs_fp64 = q->r.opts.precision == QTL_FP64 ? 0.0 : -1.0;
    if (q->ex_bytes && q->res.status == QTL_OK && q->expect_out)
        std::memcpy(q->expect_out, (char*)sl.pinned + 64, q->ex_bytes);
    if (q->res.status == QTL_OK && wants_shadow(q->r) && sl.pinned) {
        const size_t stage_b = 64 + ((q->ex_bytes + 63) & ~(size_t)63);
        const char* p2 = (const char*)sl.pinned + stage_b;
        qtl_device_info info2{};
        std::memcpy(&info2, p2, sizeof(info2));
        if (info2.status == QTL_OK) {
            const qtl_c128* a = (const qtl_c128*)((const char*)sl.pinned + 64);
            const qtl_c128* b = (const qtl_c128*)(p2 + 64);
            double e = 0.0;
            for (size_t i = 0; i < q->ex_bytes / 16; ++i)
                e = std::max(e, std::hypot(a[i].re - b[i].re, a[i].im - b[i].im));
            q->res.stats.err_vs_fp64 = e;
        }
    }
    q->res.t_end = now_s();
    q->state = 2;
    sl.req = nullptr;
    S->in_use -= q->bytes;
    S->running -= 1;
    if (q->fills_gpu) S->exclusive = 0;
}

static void srv_loop(qtl_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        for (size_t i = 0; i < S->slots.size(); ++i) {
            if (S->slots[i].busy() && cudaEventQuery(S->slots[i].done) == cudaSuccess) {
                srv_retire(S, (int)i);
                progressed = true;
            }
        }
        if (progressed) S->cv_done.notify_all();
        // admit in arrival order while memory and a slot are free
        while (!S->queue.empty()) {
            SrvReq* q = S->reqs[S->queue.front()];
            if (S->in_use + q->bytes > S->budget) break;
            // a request whose kernel occupies every SM (a cooperative grid
            // that must be resident at once, or one persistent CTA per SM)
            // gains nothing from overlap and can be held back by it: it
            // runs alone, and nothing is admitted beside it
            if (S->exclusive || (q->fills_gpu && S->running > 0)) break;
            int slot = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].busy()) {
                    slot = (int)i;
                    break;
                }
            if (slot < 0) break;
            S->queue.pop_front();
            S->in_use += q->bytes;
            S->running += 1;
            if (q->batch) {
                // continuous batching: queued requests that can share the
                // launch join it, in queue order, while memory allows
                std::vector<SrvReq*> g{q};
                for (auto it = S->queue.begin(); it != S->queue.end() && (int)g.size() < SRV_MAX_GROUP;) {
                    SrvReq* o = S->reqs[*it];
                    if (o->batch && batch_compatible(q->r, o->r) && S->in_use + o->bytes <= S->budget) {
                        S->in_use += o->bytes;
                        S->running += 1;
                        g.push_back(o);
                        it = S->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                srv_admit_group(S, g, slot);
                continue;
            }
            if (q->fills_gpu) S->exclusive = 1;
            srv_admit(S, q, slot);
        }
        if (S->stop && S->running == 0) break;
        if (S->running > 0)
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    }
}

}  // namespace qtl

using namespace qtl;

extern "C" {

qtl_status qtl_server_create(size_t hbm_budget_bytes, int32_t max_inflight, qtl_server** out) {
    if (!out || max_inflight < 1 || max_inflight > 64) return QTL_EINVAL;
    *out = nullptr;
    qtl_server* S = new qtl_server();
    cudaGetDevice(&S->device);
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return QTL_ECUDA;
        }
        hbm_budget_bytes = fr / 10 * 9;
    }
    S->budget = hbm_budget_bytes;
    S->slots.resize(max_inflight);
    for (auto& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (auto& x : S->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
            }
            delete S;
            return QTL_ECUDA;
        }
    }
    S->worker = std::thread(srv_loop, S);
    *out = S;
    return QTL_OK;
}

qtl_status qtl_server_submit(qtl_server* S, const qtl_request* req, qtl_c128* expect_out,
                             uint64_t* ticket) {
    if (!S || !req || !ticket || !req->sys || !req->state0 || !req->tlist || req->nt < 1) return QTL_EINVAL;
    if (req->kind != QTL_REQ_MESOLVE && req->kind != QTL_REQ_MCSOLVE) return QTL_EINVAL;
    if (req->kind == QTL_REQ_MCSOLVE && req->ntraj < 1) return QTL_EINVAL;
    if (req->sys->s.n_e > 0 && !expect_out) return QTL_EINVAL;
    qtl_status st = validate_opts(&req->opts);
    if (st != QTL_OK) return st;
    for (int i = 1; i < req->nt; ++i)
        if (!(req->tlist[i] >= req->tlist[i - 1])) return QTL_EINVAL;
    // the system's device structures are built here, on the caller's thread,
    // not by the dispatcher while it holds the server
    int fills = 0;
    if ((st = prepare_solve(req->sys->s, req->kind, &req->opts, &fills)) != QTL_OK) return st;
    if (wants_shadow(*req)) {
        qtl_opts f = req->opts;
        f.precision = QTL_FP64;
        int f2 = 0;
        if ((st = prepare_solve(req->sys->s, req->kind, &f, &f2)) != QTL_OK) return st;
        fills |= f2;
    }
    SrvReq* q = new SrvReq();
    q->fills_gpu = fills;
    // a mesolve the batched cluster launch takes (automatic engine and
    // cluster size, no FP64 shadow, its batch plan within shared memory)
    if (req->kind == QTL_REQ_MESOLVE && !fills && !wants_shadow(*req) && req->opts.engine == QTL_ENGINE_AUTO &&
        req->opts.cluster_size == 0) {
        const System& s = req->sys->s;
        const int64_t L = (int64_t)s.n * s.n;
        if (L <= me_cluster_capacity()) {
            int C = 0, rpt = 0;
            batch_plan((int)L, &C, &rpt);
            q->batch = cta_nnz_max(s, C) <= me_smem_nnz_budget(req->opts.precision, rpt);
        }
    }
    q->r = *req;
    q->expect_out = expect_out;
    q->bytes = request_bytes(*req);
    q->res.status = QTL_EBUSY;
    q->res.t_submit = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->bytes > S->budget) {
        delete q;
        return QTL_ENOMEM;
    }
    q->ticket = S->next_ticket++;
    S->reqs[q->ticket] = q;
    S->queue.push_back(q->ticket);
    *ticket = q->ticket;
    S->cv_work.notify_one();
    return QTL_OK;
}

static qtl_status take_result(qtl_server* S, uint64_t ticket, qtl_result* out) {
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return QTL_EINVAL;
    SrvReq* q = it->second;
    if (q->state != 2) return QTL_EBUSY;
    if (out) *out = q->res;
    delete q;
    S->reqs.erase(it);
    return QTL_OK;
}

qtl_status qtl_server_poll(qtl_server* S, uint64_t ticket, qtl_result* out) {
    if (!S) return QTL_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    return take_result(S, ticket, out);
}

qtl_status qtl_server_wait(qtl_server* S, uint64_t ticket, qtl_result* out) {
    if (!S) return QTL_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        qtl_status st = take_result(S, ticket, out);
        if (st != QTL_EBUSY) return st;
        S->cv_done.wait(lk);
    }
}

qtl_status qtl_server_cancel(qtl_server* S, uint64_t ticket) {
    if (!S) return QTL_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return QTL_EINVAL;
    SrvReq* q = it->second;
    if (q->state != 0) return QTL_EBUSY;
    for (auto qi = S->queue.begin(); qi != S->queue.end(); ++qi)
        if (*qi == ticket) {
            S->queue.erase(qi);
            break;
        }
    q->state = 2;
    q->res.status = QTL_ECANCEL;
    q->res.t_end = now_s();
    S->cv_done.notify_all();
    return QTL_OK;
}

qtl_status qtl_server_usage(qtl_server* S, size_t* bytes_in_use, int32_t* queued, int32_t* running) {
    if (!S) return QTL_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (bytes_in_use) *bytes_in_use = S->in_use;
    if (queued) *queued = (int32_t)S->queue.size();
    if (running) *running = S->running;
    return QTL_OK;
}

void qtl_server_free(qtl_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (uint64_t t : S->queue) {
            SrvReq* q = S->reqs[t];
            q->state = 2;
            q->res.status = QTL_ECANCEL;
        }
        S->queue.clear();
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->reqs) delete kv.second;
    for (auto& sl : S->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    delete S;
}

}  // extern "C"
