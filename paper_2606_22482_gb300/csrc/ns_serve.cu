// ns_serve.cu -- continuous batching of SpMM requests on one GPU.
//
// Two host threads share the server state under one mutex.
//   planner: builds the plan of each new key on its own stream and keeps a host copy of the
//            plan's work list and cost classes.  The key is (graph, K, dtype); when the tune
//            keeps every nonzero on the CUDA cores and asks for no hot-row bitmap, the plan does
//            not depend on K or on the dtype of B, so one plan per graph serves them all.
//            A request waits in the queue for its plan while requests behind it whose plans are
//            built go ahead.
//   worker : admit  : queued requests with a built plan enter in arrival order while slots are
//                     free and their footprint (B + C + the plan's own partial-row slots) fits
//                     the HBM budget beside the resident plans; idle plans are evicted, least
//                     recently used first, to make room;
//            prepare: B is copied to the device on the copy stream;
//            launch : every request admitted since the last launch joins ONE persistent launch
//                     per (K, dtype, kernel) group: their work lists are merged by cost class and
//                     each item carries its request's descriptor (staged through pinned host
//                     memory, so the upload never waits for running launches); launches
//                     alternate between two streams so a new batch overlaps the running ones;
//            retire : when a launch's event completes, its requests are done (C was copied back
//                     on the launch's stream) and their memory returns to the budget.
// Requests never share execution scratch (each owns its partial-row slots and their counters),
// so two requests on the same plan may run in the same or in overlapping launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ns_internal.cuh"

namespace ns {

static double serve_clock()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct SGraph {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rowptr, colidx;
    std::vector<float> vals;
};

struct SPlan {
    uint64_t key = 0;
    int32_t graph = 0, K = 0;
    ns_dtype_t dt = NS_F32;
    int state = 0;  // 0 waiting for the planner, 1 built, 2 failed
    ns_status_t err = NS_OK;
    Plan* plan = nullptr;
    int64_t bytes = 0;  // device bytes (an estimate until built)
    int users = 0;      // requests queued or in flight on this plan
    double last_used = 0, t_ready = 0;
    std::vector<int32_t> hq;   // the plan's work list (host copy)
    std::vector<int8_t> hcls;  // cost class (floor log2 of the Eq. 1 cost) of each entry of hq
};

struct SReq {
    uint64_t ticket = 0;
    ns_request_t r{};
    ns_req_stats_t st{};
    int state = 0;  // 0 queued, 1 admitted, 2 launched, 3 done
    double t_submit = 0;
    int64_t bytes = 0;
    SPlan* sp = nullptr;
    void* block = nullptr;  // B, C, the partial-row slots and their counters on the device
    void* dB = nullptr;
    float* dC = nullptr;
    float* slots = nullptr;
    int32_t* cnt = nullptr;
};

struct Pinned {
    void* p = nullptr;
    size_t bytes = 0;
};

struct SLaunch {
    std::vector<SReq*> reqs;
    void* block = nullptr;  // descriptors, work list, ctrl (device)
    Pinned staging;         // the same, host side
    cudaEvent_t ev = nullptr;
    cudaStream_t stream = nullptr;
};

struct Server {
    ns_serve_cfg_t cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv, plan_cv;
    bool stop = false;
    bool kick = false;  // something for the worker: a request, a built plan, freed memory
    std::thread worker, planner;
    std::deque<SGraph> graphs;  // a deque: references stay valid while graphs are added
    std::list<SReq*> queue;
    std::deque<SPlan*> plan_jobs;
    std::unordered_map<uint64_t, SReq*> reqs;
    std::map<uint64_t, SPlan> plans;
    uint64_t next_ticket = 1;
    int inflight = 0;
    int64_t used = 0;
    cudaStream_t s_plan = nullptr, s_copy = nullptr, s_exec[2] = {nullptr, nullptr};
    int flip = 0;
    std::list<SLaunch> launches;
    std::vector<Pinned> pinned_free;  // staging buffers ready for reuse (worker thread only)
};

static bool plan_per_graph(const ns_tune_t& t) { return t.tau_tile == kTauInf && t.l2_hints != 2; }

static uint64_t plan_key(const ns_tune_t& t, int32_t g, int32_t K, ns_dtype_t dt)
{
    if (plan_per_graph(t)) return ((uint64_t)(uint32_t)g << 32) | 0xFFFFFFFFull;
    return ((uint64_t)(uint32_t)g << 32) | ((uint64_t)(uint32_t)K << 1) | (uint64_t)(dt == NS_BF16);
}

// accounted for a plan until the planner has built it: a few bytes per row and per nonzero
static int64_t est_plan_bytes(const SGraph& g)
{
    return (int64_t)g.m * 24 + g.nnz * 8 + 4096;
}

// a request's own device memory: B, C, the partial-row slots of its plan and their counters
static int64_t req_bytes(const SGraph& g, int32_t K, ns_dtype_t dt, int64_t n_slots, int64_t n_split)
{
    const size_t eb = dt == NS_BF16 ? 2 : 4;
    return (int64_t)(al256((size_t)g.n * K * eb) + al256((size_t)g.m * K * 4) + al256((size_t)n_slots * K * 4) +
                     al256((size_t)(n_split > 0 ? n_split : 1) * 4));
}

static void drop_plan(Server* S, SPlan* sp)  // lock held
{
    S->used -= sp->bytes;
    delete sp->plan;
    S->plans.erase(sp->key);
}

// least recently used idle built plan, or nullptr
static SPlan* idle_lru(Server* S)
{
    SPlan* v = nullptr;
    for (auto& kv : S->plans) {
        SPlan& sp = kv.second;
        if (sp.state == 1 && sp.users == 0 && (!v || sp.last_used < v->last_used)) v = &sp;
    }
    return v;
}

// evict idle plans until `need` more bytes fit the budget; lock held
static bool make_room(Server* S, int64_t need)
{
    while (S->used + need > S->cfg.hbm_budget_bytes) {
        SPlan* v = idle_lru(S);
        if (!v) return false;
        drop_plan(S, v);
    }
    return true;
}

// keep at most max_graphs plans resident (idle ones go first); lock held
static void trim_plans(Server* S)
{
    while ((int64_t)S->plans.size() > (int64_t)S->cfg.max_graphs) {
        SPlan* v = idle_lru(S);
        if (!v) return;
        drop_plan(S, v);
    }
}

static void release_plan(Server* S, SPlan* sp)  // lock held
{
    sp->users--;
    sp->last_used = serve_clock();
    if (sp->state == 2 && sp->users == 0) drop_plan(S, sp);  // a later request retries
}

// a request leaves the server (done or failed); lock held
static void finish_req(Server* S, SReq* q, ns_status_t code)
{
    q->st.status = code;
    q->st.t_done = serve_clock();
    if (q->state >= 1) {
        S->inflight--;
        S->used -= q->bytes;
    }
    q->state = 3;
    release_plan(S, q->sp);
    S->kick = true;
}

// the plan's work list and the cost class of each entry, copied to the host once
static ns_status_t host_work_list(const Plan* P, cudaStream_t s, std::vector<int32_t>* hq,
                                  std::vector<int8_t>* hcls)
{
    const int64_t n = P->st.n_items;
    hq->assign(n, 0);
    hcls->assign(n, 0);
    if (n == 0) return NS_OK;
    std::vector<int64_t> cost(n);
    NS_CUDA_TRY(cudaMemcpyAsync(cost.data(), P->item_cost, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NS_CUDA_TRY(cudaMemcpyAsync(hq->data(), P->queue, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    NS_CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t j = 0; j < n; ++j) {
        const int64_t c = cost[(*hq)[j]];
        int b = 0;
        while (b < 62 && (c >> (b + 1)) > 0) ++b;
        (*hcls)[j] = (int8_t)b;
    }
    return NS_OK;
}

static void planner_loop(Server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        SPlan* sp = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->plan_cv.wait(lk, [&] { return S->stop || !S->plan_jobs.empty(); });
            if (S->stop) return;
            sp = S->plan_jobs.front();
            S->plan_jobs.pop_front();
        }
        const SGraph& g = S->graphs[sp->graph];
        ns_csr_t A{g.m, g.n, g.nnz, g.rowptr.data(), g.colidx.data(), g.vals.data(), 0};
        Plan* P = nullptr;
        std::vector<int32_t> hq;
        std::vector<int8_t> hcls;
        ns_status_t r = plan_create(&A, sp->K, sp->dt, &S->cfg.tune, S->s_plan, &P);
        if (r == NS_OK) r = host_work_list(P, S->s_plan, &hq, &hcls);
        std::lock_guard<std::mutex> lk(S->mu);
        if (r != NS_OK) {
            delete P;
            sp->state = 2;
            sp->err = r;
        } else {
            const int64_t real = P->st.device_bytes;
            S->used += real - sp->bytes;
            sp->bytes = real;
            sp->plan = P;
            sp->hq = std::move(hq);
            sp->hcls = std::move(hcls);
            sp->t_ready = serve_clock();
            sp->last_used = sp->t_ready;
            sp->state = 1;
            trim_plans(S);
        }
        S->kick = true;
        S->cv.notify_one();
    }
}

// admission, in arrival order; lock held
static void admit(Server* S, std::vector<SReq*>& fresh)
{
    for (auto it = S->queue.begin(); it != S->queue.end() && S->inflight < S->cfg.max_inflight;) {
        SReq* q = *it;
        SPlan* sp = q->sp;
        if (sp->state == 0) {  // its plan is being built: requests behind it may go ahead
            ++it;
            continue;
        }
        if (sp->state == 2) {
            it = S->queue.erase(it);
            finish_req(S, q, sp->err);
            continue;
        }
        const SGraph& g = S->graphs[q->r.graph_id];
        const int64_t need = req_bytes(g, q->r.K, q->r.b_dtype, sp->plan->st.n_slots, sp->plan->st.n_split);
        if (need + sp->bytes > S->cfg.hbm_budget_bytes) {
            it = S->queue.erase(it);
            finish_req(S, q, NS_ERR_TOO_LARGE);
            continue;
        }
        // Memory: wait for running requests to return theirs, keeping the arrival order.  With
        // nothing running, only plans of queued requests can hold the budget; the oldest request
        // is admitted anyway so the queue keeps moving (over the budget until it retires).
        if (!make_room(S, need) && S->inflight > 0) break;
        it = S->queue.erase(it);
        const double now = serve_clock();
        q->bytes = need;
        S->used += need;
        sp->last_used = now;
        q->state = 1;
        q->st.t_admit = now;
        q->st.t_planned = sp->t_ready > q->t_submit ? sp->t_ready : 0.0;
        S->inflight++;
        fresh.push_back(q);
    }
}

static Pinned get_pinned(Server* S, size_t bytes)
{
    for (size_t i = 0; i < S->pinned_free.size(); ++i)
        if (S->pinned_free[i].bytes >= bytes) {
            Pinned p = S->pinned_free[i];
            S->pinned_free.erase(S->pinned_free.begin() + i);
            return p;
        }
    Pinned p;
    size_t sz = 64 << 10;
    while (sz < bytes) sz <<= 1;
    if (cudaHostAlloc(&p.p, sz, cudaHostAllocDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        return Pinned{};
    }
    p.bytes = sz;
    return p;
}

// device memory of the fresh requests and the upload of their B
static void prepare(Server* S, std::vector<SReq*>& fresh, std::vector<SReq*>& ready)
{
    for (SReq* q : fresh) {
        const SGraph& g = S->graphs[q->r.graph_id];
        const Plan* P = q->sp->plan;
        const size_t eb = q->r.b_dtype == NS_BF16 ? 2 : 4;
        const size_t bB = al256((size_t)g.n * q->r.K * eb);
        const size_t bC = al256((size_t)g.m * q->r.K * 4);
        const size_t bS = al256((size_t)P->st.n_slots * q->r.K * 4);
        const size_t bN = al256((size_t)(P->st.n_split > 0 ? P->st.n_split : 1) * 4);
        void* blk = nullptr;
        if (pool_alloc(&blk, bB + bC + bS + bN, S->s_copy) != cudaSuccess) {
            (void)cudaGetLastError();
            std::lock_guard<std::mutex> lk(S->mu);
            finish_req(S, q, NS_ERR_OOM);
            continue;
        }
        q->block = blk;
        q->dB = blk;
        q->dC = reinterpret_cast<float*>(static_cast<char*>(blk) + bB);
        q->slots = reinterpret_cast<float*>(static_cast<char*>(blk) + bB + bC);
        q->cnt = reinterpret_cast<int32_t*>(static_cast<char*>(blk) + bB + bC + bS);
        cudaMemsetAsync(q->cnt, 0, bN, S->s_copy);  // split-row arrival counters start at zero
        if (g.n > 0) cudaMemcpyAsync(q->dB, q->r.B, (size_t)g.n * q->r.K * eb, cudaMemcpyHostToDevice, S->s_copy);
        ready.push_back(q);
    }
}

// one persistent launch for a group of requests sharing K, dtype and kernel
static void launch_group(Server* S, std::vector<SReq*>& rs, int K, bool bf16, bool dense, int TM, int TK,
                         cudaEvent_t copied)
{
    struct It {
        int cls;
        int32_t slot, item, rank;
    };
    std::vector<It> items;
    std::vector<ExecDesc> descs(rs.size());
    for (size_t k = 0; k < rs.size(); ++k) {
        SPlan* sp = rs[k]->sp;
        Plan* P = sp->plan;
        fill_desc(P, rs[k]->dB, K, rs[k]->dC, K, &descs[k]);
        descs[k].K = K;  // a plan shared across K and dtype takes the request's
        descs[k].b_bf16 = bf16 ? 1 : 0;
        descs[k].slots = rs[k]->slots;
        descs[k].split_cnt = rs[k]->cnt;
        for (size_t j = 0; j < sp->hq.size(); ++j)
            items.push_back({sp->hcls[j], (int32_t)k, sp->hq[j], (int32_t)j});
    }
    std::stable_sort(items.begin(), items.end(), [](const It& a, const It& b) {
        if (a.cls != b.cls) return a.cls > b.cls;
        if (a.slot != b.slot) return a.slot < b.slot;
        return a.rank < b.rank;
    });
    const int64_t ni = (int64_t)items.size();
    SLaunch L;
    L.reqs = rs;
    L.stream = S->s_exec[S->flip];
    S->flip ^= 1;
    const size_t bD = al256(descs.size() * sizeof(ExecDesc));
    const size_t bQ = al256((size_t)(ni > 0 ? ni : 1) * 4);
    const size_t total = bD + 2 * bQ + 256;
    L.staging = get_pinned(S, total);
    if (!L.staging.p || pool_alloc(&L.block, total, L.stream) != cudaSuccess) {
        (void)cudaGetLastError();
        if (L.staging.p) S->pinned_free.push_back(L.staging);
        std::lock_guard<std::mutex> lk(S->mu);
        for (SReq* q : rs) {
            cudaFreeAsync(q->block, S->s_copy);
            q->block = nullptr;
            finish_req(S, q, NS_ERR_OOM);
        }
        return;
    }
    char* h = static_cast<char*>(L.staging.p);
    std::memcpy(h, descs.data(), descs.size() * sizeof(ExecDesc));
    int32_t* hq = reinterpret_cast<int32_t*>(h + bD);
    int32_t* hd = reinterpret_cast<int32_t*>(h + bD + bQ);
    for (int64_t j = 0; j < ni; ++j) {
        hq[j] = items[j].item;
        hd[j] = items[j].slot;
    }
    std::memset(h + bD + 2 * bQ, 0, 256);  // ctrl: work ticket and status
    char* base = static_cast<char*>(L.block);
    cudaStreamWaitEvent(L.stream, copied, 0);
    cudaMemcpyAsync(base, h, total, cudaMemcpyHostToDevice, L.stream);
    int grid = 0;
    ns_status_t r = exec_launch(reinterpret_cast<ExecDesc*>(base), reinterpret_cast<int32_t*>(base + bD),
                                reinterpret_cast<int32_t*>(base + bD + bQ), ni,
                                reinterpret_cast<int32_t*>(base + bD + 2 * bQ), K, TM, TK, bf16,
                                S->cfg.tune.l2_hints != 0, dense, &grid, L.stream, nullptr,
                                S->cfg.tune.chunk_nnz);
    const double t_start = serve_clock();
    for (SReq* q : rs) {
        const SGraph& g = S->graphs[q->r.graph_id];
        q->st.t_start = t_start;
        if (g.m > 0) cudaMemcpyAsync(q->r.C, q->dC, (size_t)g.m * q->r.K * 4, cudaMemcpyDeviceToHost, L.stream);
    }
    cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
    cudaEventRecord(L.ev, L.stream);
    std::lock_guard<std::mutex> lk(S->mu);
    if (r != NS_OK) {
        cudaEventSynchronize(L.ev);
        cudaEventDestroy(L.ev);
        for (SReq* q : rs) {
            cudaFreeAsync(q->block, L.stream);
            q->block = nullptr;
            finish_req(S, q, r);
        }
        cudaFreeAsync(L.block, L.stream);
        S->pinned_free.push_back(L.staging);
        return;
    }
    for (SReq* q : rs) q->state = 2;
    S->launches.push_back(L);
}

static void worker_loop(Server* S)
{
    cudaSetDevice(S->device);
    std::vector<SReq*> fresh, ready;
    for (;;) {
        fresh.clear();
        ready.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (!S->kick) {
                // nothing new: sleep until a submit or a built plan; while launches run, wake
                // often enough to retire them promptly
                const auto wait = std::chrono::microseconds(S->launches.empty() ? 2000 : 20);
                S->cv.wait_for(lk, wait, [&] { return S->stop || S->kick; });
            }
            S->kick = false;
            if (S->stop && S->launches.empty()) break;  // destroy dropped the queue
            if (!S->stop) admit(S, fresh);
        }
        prepare(S, fresh, ready);
        if (!ready.empty()) {
            cudaEvent_t copied;
            cudaEventCreateWithFlags(&copied, cudaEventDisableTiming);
            cudaEventRecord(copied, S->s_copy);
            std::map<std::tuple<int, int, int, int, int>, std::vector<SReq*>> groups;
            for (SReq* q : ready) {
                const Plan* P = q->sp->plan;
                groups[{q->r.K, (int)q->r.b_dtype, P->st.n_dwin > 0 ? 1 : 0, P->tune.TM, P->tune.TK}].push_back(q);
            }
            for (auto& kv : groups)
                launch_group(S, kv.second, std::get<0>(kv.first), std::get<1>(kv.first) == NS_BF16,
                             std::get<2>(kv.first) != 0, std::get<3>(kv.first), std::get<4>(kv.first), copied);
            cudaEventDestroy(copied);
        }
        // ---- retire finished launches ----
        for (auto it = S->launches.begin(); it != S->launches.end();) {
            if (cudaEventQuery(it->ev) != cudaSuccess) {
                (void)cudaGetLastError();
                ++it;
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            for (SReq* q : it->reqs) {
                cudaFreeAsync(q->block, it->stream);
                q->block = nullptr;
                finish_req(S, q, NS_OK);
            }
            cudaEventDestroy(it->ev);
            cudaFreeAsync(it->block, it->stream);
            S->pinned_free.push_back(it->staging);
            it = S->launches.erase(it);
        }
    }
}

}  // namespace ns

using namespace ns;

extern "C" {

double ns_serve_now(void) { return serve_clock(); }

ns_status_t ns_serve_create(const ns_serve_cfg_t* cfg, ns_server_t* out)
{
    if (!cfg || !out) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->max_inflight < 1 || cfg->max_queue < 1 || cfg->max_graphs < 1) {
        set_error("budget, max_inflight, max_queue and max_graphs must be positive");
        return NS_ERR_INVALID;
    }
    if (plan_check_tune(cfg->tune) != NS_OK) {
        set_error("invalid tune");
        return NS_ERR_INVALID;
    }
    Server* S = new (std::nothrow) Server();
    if (!S) {
        set_error("host allocation failed");
        return NS_ERR_OOM;
    }
    S->cfg = *cfg;
    NS_CUDA_TRY(cudaGetDevice(&S->device));
    NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_plan, cudaStreamNonBlocking));
    NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_copy, cudaStreamNonBlocking));
    NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_exec[0], cudaStreamNonBlocking));
    NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_exec[1], cudaStreamNonBlocking));
    S->worker = std::thread(worker_loop, S);
    S->planner = std::thread(planner_loop, S);
    *out = reinterpret_cast<ns_server_t>(S);
    return NS_OK;
}

ns_status_t ns_serve_register_graph(ns_server_t sv, const ns_csr_t* A, int32_t* graph_id)
{
    Server* S = reinterpret_cast<Server*>(sv);
    if (!S || !A || !graph_id) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    if (A->on_device) {
        set_error("register a host CSR");
        return NS_ERR_INVALID;
    }
    if (A->m < 0 || A->n < 0 || A->nnz < 0 || !A->rowptr || (A->nnz && (!A->colidx || !A->vals))) {
        set_error("bad CSR");
        return NS_ERR_INVALID;
    }
    SGraph g;
    g.m = A->m;
    g.n = A->n;
    g.nnz = A->nnz;
    g.rowptr.assign(A->rowptr, A->rowptr + A->m + 1);
    g.colidx.assign(A->colidx, A->colidx + A->nnz);
    g.vals.assign(A->vals, A->vals + A->nnz);
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(std::move(g));
    *graph_id = (int32_t)S->graphs.size() - 1;
    return NS_OK;
}

ns_status_t ns_serve_submit(ns_server_t sv, const ns_request_t* r, uint64_t* ticket)
{
    Server* S = reinterpret_cast<Server*>(sv);
    if (!S || !r || !ticket) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->graph_id < 0 || r->graph_id >= (int32_t)S->graphs.size()) {
        set_error("unknown graph id %d", r->graph_id);
        return NS_ERR_NOT_FOUND;
    }
    if (r->K < 8 || r->K > 1024 || r->K % 8 || (r->b_dtype != NS_F32 && r->b_dtype != NS_BF16)) {
        set_error("unsupported K or dtype");
        return NS_ERR_UNSUPPORTED;
    }
    const SGraph& g = S->graphs[r->graph_id];
    if ((g.n > 0 && !r->B) || (g.m > 0 && !r->C)) {
        set_error("B or C is NULL");
        return NS_ERR_INVALID;
    }
    if (req_bytes(g, r->K, r->b_dtype, 0, 0) + est_plan_bytes(g) > S->cfg.hbm_budget_bytes) {
        set_error("request footprint exceeds the HBM budget");
        return NS_ERR_TOO_LARGE;
    }
    if ((int)S->queue.size() >= S->cfg.max_queue) {
        set_error("admission queue full");
        return NS_ERR_AGAIN;
    }
    SReq* q = new (std::nothrow) SReq();
    if (!q) {
        set_error("host allocation failed");
        return NS_ERR_OOM;
    }
    q->ticket = S->next_ticket++;
    q->r = *r;
    q->st.status = NS_OK;
    q->t_submit = serve_clock();
    const uint64_t key = plan_key(S->cfg.tune, r->graph_id, r->K, r->b_dtype);
    auto pit = S->plans.find(key);
    if (pit == S->plans.end()) {  // first request on this key: the planner builds its plan
        SPlan sp;
        sp.key = key;
        sp.graph = r->graph_id;
        sp.K = r->K;
        sp.dt = r->b_dtype;
        sp.bytes = est_plan_bytes(g);
        pit = S->plans.emplace(key, std::move(sp)).first;
        S->used += pit->second.bytes;
        S->plan_jobs.push_back(&pit->second);
        q->st.plan_built = 1;
        S->plan_cv.notify_one();
    }
    pit->second.users++;
    q->sp = &pit->second;
    S->queue.push_back(q);
    S->reqs[q->ticket] = q;
    *ticket = q->ticket;
    S->kick = true;
    S->cv.notify_one();
    return NS_OK;
}

ns_status_t ns_serve_poll(ns_server_t sv, uint64_t ticket, int* done, ns_req_stats_t* st)
{
    Server* S = reinterpret_cast<Server*>(sv);
    if (!S || !done) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_error("unknown ticket");
        return NS_ERR_NOT_FOUND;
    }
    SReq* q = it->second;
    *done = q->state == 3;
    if (st) *st = q->st;
    if (q->state == 3) {  // reported once: forget the request
        ns_status_t code = (ns_status_t)q->st.status;
        S->reqs.erase(it);
        delete q;
        if (code != NS_OK) {
            set_error("request failed");
            return code;
        }
    }
    return NS_OK;
}

ns_status_t ns_serve_destroy(ns_server_t sv)
{
    Server* S = reinterpret_cast<Server*>(sv);
    if (!S) return NS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // requests still queued are dropped
        for (SReq* q : S->queue) {
            S->reqs.erase(q->ticket);
            delete q;
        }
        S->queue.clear();
    }
    S->cv.notify_all();
    S->plan_cv.notify_all();
    if (S->planner.joinable()) S->planner.join();
    if (S->worker.joinable()) S->worker.join();  // retires the launches in flight first
    cudaDeviceSynchronize();
    for (auto& kv : S->plans) delete kv.second.plan;
    for (auto& kv : S->reqs) delete kv.second;
    for (auto& p : S->pinned_free) cudaFreeHost(p.p);
    cudaStreamDestroy(S->s_plan);
    cudaStreamDestroy(S->s_copy);
    cudaStreamDestroy(S->s_exec[0]);
    cudaStreamDestroy(S->s_exec[1]);
    delete S;
    return NS_OK;
}

}  // extern "C"
