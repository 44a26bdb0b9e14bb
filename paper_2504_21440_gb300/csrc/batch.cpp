// Reusable batch plans: mesolve over many independent systems of uneven size
// (parameter sweeps), planned once and replayed.
//
// qtl_batch_create groups the systems by launch plan (cluster size C and
// rows per thread, from each system's n^2 as in qtl_mesolve_batch), can time
// candidate cluster sizes per group on a short probe of that group's own
// solves and keep the fastest (the autotuner), builds the device job table
// once, and captures the whole launch sequence -- status reset, one cluster
// launch per group on its own stream, the join -- in a CUDA graph.
// qtl_batch_launch replays that graph on the caller's stream: one call, no
// host-side planning, the same kernels and the same job table every time.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace qtl;

struct qtl_batch {
    int device = 0;
    int nb = 0, precision = 0;
    std::vector<std::vector<int>> group;   // system indices per launch plan, largest first
    std::vector<int> C, Lmax, smem;        // per group: cluster size, largest n^2, shared entries
    std::vector<std::vector<int>> cand_c;  // per group: autotuner candidates and probe times
    std::vector<std::vector<double>> cand_ms;
    char* scratch = nullptr;               // job table | counters | expectation partials
    MeJob* jobs = nullptr;
    int* counters = nullptr;
    qtl_device_info* info = nullptr;       // the caller's
    std::vector<cudaStream_t> streams;     // one per group (owned)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Status reset, then one cluster launch per group (groups > 1: on the plan's
// own streams, forked from and joined back into st).
cudaError_t enqueue(const qtl_batch& b, const MeJob* jobs, int* counters, qtl_device_info* info,
                    cudaStream_t st) {
    const int ng = (int)b.group.size();
    cudaError_t e;
    if ((e = cudaMemsetAsync(info, 0, (size_t)b.nb * sizeof(qtl_device_info), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counters, 0, (size_t)ng * sizeof(int), st)) != cudaSuccess) return e;
    std::vector<cudaEvent_t> evs;
    auto event = [&]() {
        cudaEvent_t ev = nullptr;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        evs.push_back(ev);
        return ev;
    };
    cudaEvent_t fork = nullptr;
    if (ng > 1) {
        fork = event();
        e = cudaEventRecord(fork, st);
    }
    int first = 0;
    for (int k = 0; k < ng && e == cudaSuccess; ++k) {
        cudaStream_t sk = ng > 1 ? b.streams[k] : st;
        if (ng > 1 && (e = cudaStreamWaitEvent(sk, fork, 0)) != cudaSuccess) break;
        const int cnt = (int)b.group[k].size();
        e = launch_me_cluster(jobs + first, cnt, b.Lmax[k], b.smem[k], b.precision, b.C[k], counters + k, sk);
        first += cnt;
        if (ng > 1 && e == cudaSuccess) {
            cudaEvent_t done = event();
            if ((e = cudaEventRecord(done, sk)) == cudaSuccess) e = cudaStreamWaitEvent(st, done, 0);
        }
    }
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    return e;
}

// Largest per-CTA Liouvillian entry count of a group at cluster size C, or -1
// when C cannot hold the group's largest solve.
int64_t group_need(qtl_system* const* systems, const std::vector<int>& g, int Lmax, int C, int precision) {
    int Cc = 0, rpt = 0;
    if (!me_plan(Lmax, C, &Cc, &rpt)) return -1;
    int64_t need = 0;
    for (int b : g) need = std::max(need, cta_nnz_max(systems[b]->s, C));
    return need > me_smem_nnz_budget(precision, rpt) ? -1 : need;
}

}  // namespace

extern "C" qtl_status qtl_batch_create(qtl_system* const* systems, int32_t nb,
                                       const qtl_c128* const* state0_dev, const int32_t* is_ket,
                                       const double* tlist_dev, int32_t nt, const qtl_opts* opts,
                                       qtl_c128* const* expect_dev, qtl_device_info* info_dev,
                                       int32_t autotune, qtl_batch** out) {
    if (!out) return QTL_EINVAL;
    *out = nullptr;
    if (!systems || nb < 1 || !state0_dev || !is_ket || !tlist_dev || nt < 1 || !expect_dev || !info_dev)
        return QTL_EINVAL;
    qtl_status st = validate_opts(opts);
    if (st != QTL_OK) return st;
    for (int b = 0; b < nb; ++b) {
        if (!systems[b] || !state0_dev[b] || (systems[b]->s.n_e > 0 && !expect_dev[b])) return QTL_EINVAL;
        systems[b]->s.solved = true;
        if ((st = ensure_liouvillian(systems[b]->s)) != QTL_OK) return st;
        if (!systems[b]->s.Htd.empty() && (st = ensure_td_liouvillian(systems[b]->s)) != QTL_OK) return st;
    }
    cudaStream_t stream = (cudaStream_t)opts->cuda_stream;
    qtl_batch* p = new qtl_batch();
    p->nb = nb;
    p->precision = opts->precision;
    p->info = info_dev;
    cudaGetDevice(&p->device);
    auto fail = [&](qtl_status s) {
        qtl_batch_free(p);
        return s;
    };
    // groups by default plan, largest Liouvillian first inside a group
    {
        std::vector<std::pair<int, int>> keys;
        std::vector<int> key_of(nb);
        for (int b = 0; b < nb; ++b) {
            const int L = systems[b]->s.n * systems[b]->s.n;
            int C = 0, rpt = 0;
            batch_plan(L, &C, &rpt);
            const std::pair<int, int> k(C, rpt);
            auto it = std::find(keys.begin(), keys.end(), k);
            key_of[b] = (int)(it - keys.begin());
            if (it == keys.end()) keys.push_back(k);
        }
        p->group.resize(keys.size());
        for (int b = 0; b < nb; ++b) p->group[key_of[b]].push_back(b);
        for (size_t k = 0; k < keys.size(); ++k) {
            auto& g = p->group[k];
            std::stable_sort(g.begin(), g.end(), [&](int x, int y) {
                return systems[x]->s.dL.nnz > systems[y]->s.dL.nnz;
            });
            int Lmax = 0;
            for (int b : g) Lmax = std::max(Lmax, systems[b]->s.n * systems[b]->s.n);
            p->C.push_back(keys[k].first);
            p->Lmax.push_back(Lmax);
            const int64_t need = group_need(systems, g, Lmax, keys[k].first, p->precision);
            if (need < 0) return fail(QTL_ETOOBIG);
            p->smem.push_back((int)need);
        }
    }
    const int ng = (int)p->group.size();
    p->cand_c.resize(ng);
    p->cand_ms.resize(ng);
    p->streams.resize(ng, nullptr);
    for (int k = 0; k < ng; ++k)
        if (cudaStreamCreateWithFlags(&p->streams[k], cudaStreamNonBlocking) != cudaSuccess)
            return fail(QTL_ECUDA);
    auto ne_of = [&](int b) { return systems[b]->s.n_e > 0 ? systems[b]->s.n_e : 1; };

    // ---- autotuner: per group, candidate cluster sizes C/2, C, 2C, 4C timed
    // on a probe (the group's own solves over the first 5% of tlist's span,
    // two output times, outputs into plan scratch), fastest kept ----
    if (autotune) {
        std::vector<double> tl(nt);
        if (cudaMemcpy(tl.data(), tlist_dev, (size_t)nt * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(QTL_ECUDA);
        const double probe_t[2] = {tl[0], tl[0] + 0.05 * (tl[nt - 1] - tl[0])};
        for (int k = 0; k < ng; ++k) {
            const auto& g = p->group[k];
            const int cnt = (int)g.size();
            std::vector<int> cands;
            for (int c : {p->C[k] / 2, p->C[k], 2 * p->C[k], 4 * p->C[k]})
                if (c >= 1 && c <= 16 && group_need(systems, g, p->Lmax[k], c, p->precision) >= 0 &&
                    std::find(cands.begin(), cands.end(), c) == cands.end())
                    cands.push_back(c);
            if (cands.size() < 2 || probe_t[1] <= probe_t[0]) continue;
            // probe scratch: tlist, jobs, counter, info, expect, partials (at C = 16)
            size_t off = 0;
            auto take = [&](size_t bytes) {
                const size_t o = off;
                off += (bytes + 255) & ~(size_t)255;
                return o;
            };
            const size_t o_tl = take(16), o_jobs = take((size_t)cnt * sizeof(MeJob)), o_cnt = take(sizeof(int)),
                         o_info = take((size_t)cnt * sizeof(qtl_device_info));
            std::vector<size_t> o_ex(cnt), o_ep(cnt), o_td(cnt);
            for (int q = 0; q < cnt; ++q) {
                o_ex[q] = take((size_t)ne_of(g[q]) * 2 * 16);
                o_ep[q] = take((size_t)2 * 16 * 2 * ne_of(g[q]) * sizeof(double));
                o_td[q] = take(me_tdg_bytes(systems[g[q]]->s, p->precision));
            }
            char* ps = nullptr;
            if (cudaMalloc((void**)&ps, off) != cudaSuccess) return fail(QTL_ENOMEM);
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            cudaEventCreate(&t0);
            cudaEventCreate(&t1);
            bool ok = cudaMemcpy(ps + o_tl, probe_t, 16, cudaMemcpyHostToDevice) == cudaSuccess;
            double best = 1e300;
            int best_c = p->C[k];
            for (int c : cands) {
                if (!ok) break;
                const int need = (int)group_need(systems, g, p->Lmax[k], c, p->precision);
                std::vector<MeJob> jobs(cnt);
                for (int q = 0; q < cnt; ++q)
                    me_job_fill(jobs[q], systems[g[q]]->s, (const double*)(ps + o_tl), 2, state0_dev[g[q]],
                                is_ket[g[q]], (double*)(ps + o_ep[q]), (qtl_c128*)(ps + o_ex[q]),
                                (qtl_device_info*)(ps + o_info) + q, opts, need,
                                me_tdg_bytes(systems[g[q]]->s, p->precision) ? (double2*)(ps + o_td[q]) : nullptr);
                ok = cudaMemcpy(ps + o_jobs, jobs.data(), (size_t)cnt * sizeof(MeJob), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
                float ms = 0.f;
                for (int rep = 0; rep < 2 && ok; ++rep) {   // first run warms, second is timed
                    ok = cudaMemsetAsync(ps + o_cnt, 0, sizeof(int), stream) == cudaSuccess &&
                         cudaEventRecord(t0, stream) == cudaSuccess &&
                         launch_me_cluster((const MeJob*)(ps + o_jobs), cnt, p->Lmax[k], need, p->precision, c,
                                           (int*)(ps + o_cnt), stream) == cudaSuccess &&
                         cudaEventRecord(t1, stream) == cudaSuccess &&
                         cudaEventSynchronize(t1) == cudaSuccess &&
                         cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess;
                }
                if (!ok) break;
                p->cand_c[k].push_back(c);
                p->cand_ms[k].push_back(ms);
                if (ms < best) {
                    best = ms;
                    best_c = c;
                }
            }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            cudaFree(ps);
            if (!ok) {
                set_cuda_error(cudaGetLastError());
                return fail(QTL_ECUDA);
            }
            p->C[k] = best_c;
            p->smem[k] = (int)group_need(systems, g, p->Lmax[k], best_c, p->precision);
        }
    }

    // ---- job table and scratch ----
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_jobs = take((size_t)nb * sizeof(MeJob)), o_cnt = take((size_t)ng * sizeof(int));
    std::vector<size_t> o_ep(nb), o_td(nb);
    for (int k = 0; k < ng; ++k)
        for (int b : p->group[k]) {
            o_ep[b] = take((size_t)nt * p->C[k] * 2 * ne_of(b) * sizeof(double));
            o_td[b] = take(me_tdg_bytes(systems[b]->s, p->precision));
        }
    if (cudaMalloc((void**)&p->scratch, off) != cudaSuccess) return fail(QTL_ENOMEM);
    p->jobs = (MeJob*)(p->scratch + o_jobs);
    p->counters = (int*)(p->scratch + o_cnt);
    std::vector<MeJob> jobs(nb);
    int q = 0;
    for (int k = 0; k < ng; ++k)
        for (int b : p->group[k])
            me_job_fill(jobs[q++], systems[b]->s, tlist_dev, nt, state0_dev[b], is_ket[b],
                        (double*)(p->scratch + o_ep[b]), expect_dev[b], info_dev + b, opts, p->smem[k],
                        me_tdg_bytes(systems[b]->s, p->precision) ? (double2*)(p->scratch + o_td[b]) : nullptr);
    if (cudaMemcpy(p->jobs, jobs.data(), (size_t)nb * sizeof(MeJob), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(QTL_ECUDA);

    // ---- capture the launch sequence once ----
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return fail(QTL_ECUDA);
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = enqueue(*p, p->jobs, p->counters, p->info, cap);
        e = cudaStreamEndCapture(cap, &p->graph);
        if (e1 != cudaSuccess) e = e1;
        count_launch(-ng);   // captured, not launched: replays count them
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return fail(QTL_ECUDA);
    }
    *out = p;
    return QTL_OK;
}

extern "C" qtl_status qtl_batch_launch(qtl_batch* b, void* cuda_stream) {
    if (!b || !b->exec) return QTL_EINVAL;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return QTL_EINVAL;
    const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return QTL_ECUDA;
    }
    count_launch((int)b->group.size());
    return QTL_OK;
}

extern "C" int32_t qtl_batch_groups(const qtl_batch* b) { return b ? (int32_t)b->group.size() : 0; }

extern "C" qtl_status qtl_batch_group_info(const qtl_batch* b, int32_t k, int32_t* cluster_size, int32_t* nsolves,
                                           int32_t* ncand, int32_t* cand_cluster, double* cand_ms) {
    if (!b || k < 0 || k >= (int32_t)b->group.size()) return QTL_EINVAL;
    if (cluster_size) *cluster_size = b->C[k];
    if (nsolves) *nsolves = (int32_t)b->group[k].size();
    const int nc = (int)b->cand_c[k].size();
    if (ncand) *ncand = nc;
    for (int i = 0; i < nc; ++i) {
        if (cand_cluster) cand_cluster[i] = b->cand_c[k][i];
        if (cand_ms) cand_ms[i] = b->cand_ms[k][i];
    }
    return QTL_OK;
}

extern "C" int32_t qtl_batch_group_of(const qtl_batch* b, int32_t sys) {
    if (!b || sys < 0 || sys >= b->nb) return -1;
    for (size_t k = 0; k < b->group.size(); ++k)
        for (int x : b->group[k])
            if (x == sys) return (int32_t)k;
    return -1;
}

extern "C" void qtl_batch_free(qtl_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    cudaFree(b->scratch);
    delete b;
}
