// ns_serve.cu -- continuous batching of SpMM requests on one GPU.
//
// A worker thread runs the loop
//   admit  : FIFO requests enter while slots are free and their HBM footprint (resident plan +
//            B + C + partial-row scratch) fits the budget; least-recently-used idle plans are
//            evicted to make room;
//   prepare: plan on first use of (graph, K, dtype) -- plans stay resident for later requests --
//            and copy B to the device on the copy stream;
//   launch : every request admitted since the last launch joins ONE persistent launch per
//            (K, dtype) group: their work lists are merged by cost class and each item carries
//            its request's descriptor; launches alternate between two streams so a new batch
//            overlaps the batches still running;
//   retire : when a launch's event completes, C is copied back, the request is marked done and
//            its memory returns to the budget.
// Requests never share execution scratch (each owns its split counters and slots), so two
// requests on the same graph may run in the same or in overlapping launches.
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

struct SGraph {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rowptr, colidx;
    std::vector<float> vals;
};

struct SPlan {
    Plan* plan = nullptr;
    int64_t bytes = 0;
    int users = 0;
    double last_used = 0;
};

struct SReq {
    uint64_t ticket = 0;
    ns_request_t r{};
    ns_req_stats_t st{};
    int state = 0;  // 0 queued, 1 admitted, 2 launched, 3 done
    int64_t bytes = 0;
    SPlan* sp = nullptr;
    uint64_t plan_key = 0;
    void* dB = nullptr;
    float* dC = nullptr;
    float* slots = nullptr;
    int32_t* cnt = nullptr;
    void* block = nullptr;
    cudaEvent_t done_ev = nullptr;
    int launch_id = -1;
};

struct SLaunch {
    std::vector<SReq*> reqs;
    void* block = nullptr;  // descriptors, queue, ctrl
    cudaEvent_t ev = nullptr;
    cudaStream_t stream = nullptr;
};

struct Server {
    ns_serve_cfg_t cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::thread worker;
    std::vector<SGraph> graphs;
    std::deque<SReq*> queue;
    std::unordered_map<uint64_t, SReq*> reqs;
    std::map<uint64_t, SPlan> plans;
    uint64_t next_ticket = 1;
    int inflight = 0;
    int64_t used = 0;
    cudaStream_t s_plan = nullptr, s_copy = nullptr, s_exec[2] = {nullptr, nullptr};
    int flip = 0;
    std::list<SLaunch> launches;
    std::atomic<int> error{0};
};

static uint64_t plan_key(int32_t g, int32_t K, ns_dtype_t dt)
{
    return ((uint64_t)(uint32_t)g << 32) | ((uint64_t)(uint32_t)K << 1) | (uint64_t)(dt == NS_BF16);
}

static int64_t plan_bytes(const Plan* P)
{
    int64_t b = 0;
    for (auto& blk : P->blocks) b += (int64_t)blk.bytes;
    return b;
}

// footprint estimate before planning: the plan arrays of a residual-only plan are a few bytes per
// row and per chunk on top of the graph copy
static int64_t est_plan_bytes(const SGraph& g)
{
    return (int64_t)g.m * 24 + g.nnz * 8 + 4096;
}

static int64_t req_bytes(const SGraph& g, int32_t K, ns_dtype_t dt)
{
    const int64_t eb = dt == NS_BF16 ? 2 : 4;
    const int64_t slots = ((g.m + g.nnz) / 64 + 64) * (int64_t)K * 4;  // generous bound of split slots
    return (int64_t)g.n * K * eb + (int64_t)g.m * K * 4 + slots + 4096;
}

// evict idle plans (least recently used first) until `need` more bytes fit; lock held
static bool make_room(Server* S, int64_t need)
{
    while (S->used + need > S->cfg.hbm_budget_bytes) {
        auto victim = S->plans.end();
        for (auto it = S->plans.begin(); it != S->plans.end(); ++it)
            if (it->second.users == 0 && (victim == S->plans.end() || it->second.last_used < victim->second.last_used))
                victim = it;
        if (victim == S->plans.end()) return false;
        S->used -= victim->second.bytes;
        delete victim->second.plan;
        S->plans.erase(victim);
    }
    return true;
}

static void fail_req(Server* S, SReq* q, ns_status_t code)
{
    q->st.status = code;
    q->st.t_done = serve_clock();
    q->state = 3;
    S->inflight--;
    S->used -= q->bytes;
    if (q->sp) q->sp->users--;
}

static void worker_loop(Server* S)
{
    cudaSetDevice(S->device);
    std::vector<SReq*> fresh;
    while (true) {
        fresh.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->queue.empty() && S->launches.empty())
                S->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && S->queue.empty() && S->launches.empty()) break;
            // ---- admit (FIFO, by slots and HBM footprint) ----
            while (!S->queue.empty() && S->inflight < S->cfg.max_inflight) {
                SReq* q = S->queue.front();
                const SGraph& g = S->graphs[q->r.graph_id];
                q->plan_key = plan_key(q->r.graph_id, q->r.K, q->r.b_dtype);
                auto pit = S->plans.find(q->plan_key);
                int64_t need = req_bytes(g, q->r.K, q->r.b_dtype) + (pit == S->plans.end() ? est_plan_bytes(g) : 0);
                if (!make_room(S, need)) break;  // head of line waits for memory
                S->queue.pop_front();
                q->bytes = req_bytes(g, q->r.K, q->r.b_dtype);
                S->used += need;
                if (pit == S->plans.end()) {
                    SPlan sp;
                    sp.bytes = est_plan_bytes(g);
                    pit = S->plans.emplace(q->plan_key, sp).first;
                }
                pit->second.users++;
                pit->second.last_used = serve_clock();
                q->sp = &pit->second;
                q->state = 1;
                q->st.t_admit = serve_clock();
                S->inflight++;
                fresh.push_back(q);
            }
        }
        // ---- prepare: plans (resident), operands ----
        std::vector<SReq*> ready;
        for (SReq* q : fresh) {
            const SGraph& g = S->graphs[q->r.graph_id];
            if (!q->sp->plan) {
                ns_csr_t A{g.m, g.n, g.nnz, g.rowptr.data(), g.colidx.data(), g.vals.data(), 0};
                Plan* P = nullptr;
                ns_status_t r = plan_create(&A, q->r.K, q->r.b_dtype, &S->cfg.tune, S->s_plan, &P);
                std::lock_guard<std::mutex> lk(S->mu);
                if (r != NS_OK) {
                    fail_req(S, q, r);
                    continue;
                }
                q->sp->plan = P;
                int64_t real = plan_bytes(P);
                S->used += real - q->sp->bytes;
                q->sp->bytes = real;
            }
            Plan* P = q->sp->plan;
            const size_t eb = q->r.b_dtype == NS_BF16 ? 2 : 4;
            const size_t bB = ((size_t)g.n * q->r.K * eb + 255) & ~size_t(255);
            const size_t bC = ((size_t)g.m * q->r.K * 4 + 255) & ~size_t(255);
            const size_t bS = ((size_t)P->st.n_slots * q->r.K * 4 + 255) & ~size_t(255);
            const size_t bN = ((size_t)(P->st.n_split > 0 ? P->st.n_split : 1) * 4 + 255) & ~size_t(255);
            void* blk = nullptr;
            if (pool_alloc(&blk, bB + bC + bS + bN, S->s_copy) != cudaSuccess) {
                (void)cudaGetLastError();
                std::lock_guard<std::mutex> lk(S->mu);
                fail_req(S, q, NS_ERR_OOM);
                continue;
            }
            q->block = blk;
            q->dB = blk;
            q->dC = reinterpret_cast<float*>(static_cast<char*>(blk) + bB);
            q->slots = reinterpret_cast<float*>(static_cast<char*>(blk) + bB + bC);
            q->cnt = reinterpret_cast<int32_t*>(static_cast<char*>(blk) + bB + bC + bS);
            cudaMemsetAsync(q->cnt, 0, bN, S->s_copy);
            if (g.n > 0) cudaMemcpyAsync(q->dB, q->r.B, (size_t)g.n * q->r.K * eb, cudaMemcpyHostToDevice, S->s_copy);
            ready.push_back(q);
        }
        // ---- launch: one persistent launch per (K, dtype, dense) group of fresh requests ----
        if (!ready.empty()) {
            cudaEvent_t copied;
            cudaEventCreateWithFlags(&copied, cudaEventDisableTiming);
            cudaEventRecord(copied, S->s_copy);
            std::map<std::tuple<int, int, int, int, int>, std::vector<SReq*>> groups;
            for (SReq* q : ready) {
                Plan* P = q->sp->plan;
                groups[{q->r.K, (int)q->r.b_dtype, P->st.n_dwin > 0 ? 1 : 0, P->tune.TM, P->tune.TK}].push_back(q);
            }
            for (auto& kv : groups) {
                auto& rs = kv.second;
                const int K = std::get<0>(kv.first);
                const bool bf16 = std::get<1>(kv.first) == NS_BF16;
                const bool dense = std::get<2>(kv.first) != 0;
                const int TM = std::get<3>(kv.first), TK = std::get<4>(kv.first);
                // merged work list: (cost class desc, request, item order)
                struct It {
                    int cls;
                    int32_t slot, item, rank;
                };
                std::vector<It> items;
                std::vector<ExecDesc> descs(rs.size());
                for (size_t k = 0; k < rs.size(); ++k) {
                    Plan* P = rs[k]->sp->plan;
                    fill_desc(P, rs[k]->dB, K, rs[k]->dC, K, &descs[k]);
                    descs[k].slots = rs[k]->slots;
                    descs[k].split_cnt = rs[k]->cnt;
                    const int64_t n = P->st.n_items;
                    std::vector<int64_t> cost(n);
                    std::vector<int32_t> qq(n);
                    if (n) {
                        cudaMemcpy(cost.data(), P->item_cost, n * 8, cudaMemcpyDeviceToHost);
                        cudaMemcpy(qq.data(), P->queue, n * 4, cudaMemcpyDeviceToHost);
                    }
                    for (int64_t j = 0; j < n; ++j) {
                        int64_t c = cost[qq[j]];
                        int b = 0;
                        while (b < 62 && (c >> (b + 1)) > 0) ++b;
                        items.push_back({b, (int32_t)k, qq[j], (int32_t)j});
                    }
                }
                std::stable_sort(items.begin(), items.end(), [](const It& a, const It& b) {
                    if (a.cls != b.cls) return a.cls > b.cls;
                    if (a.slot != b.slot) return a.slot < b.slot;
                    return a.rank < b.rank;
                });
                const int64_t ni = (int64_t)items.size();
                std::vector<int32_t> hq(ni), hd(ni);
                for (int64_t j = 0; j < ni; ++j) {
                    hq[j] = items[j].item;
                    hd[j] = items[j].slot;
                }
                SLaunch L;
                L.reqs = rs;
                L.stream = S->s_exec[S->flip];
                S->flip ^= 1;
                const size_t bD = (descs.size() * sizeof(ExecDesc) + 255) & ~size_t(255);
                const size_t bQ = ((size_t)(ni > 0 ? ni : 1) * 4 + 255) & ~size_t(255);
                if (pool_alloc(&L.block, bD + 2 * bQ + 256, L.stream) != cudaSuccess) {
                    (void)cudaGetLastError();
                    std::lock_guard<std::mutex> lk(S->mu);
                    for (SReq* q : rs) fail_req(S, q, NS_ERR_OOM);
                    continue;
                }
                char* base = static_cast<char*>(L.block);
                ExecDesc* dd = reinterpret_cast<ExecDesc*>(base);
                int32_t* dq = reinterpret_cast<int32_t*>(base + bD);
                int32_t* dqd = reinterpret_cast<int32_t*>(base + bD + bQ);
                int32_t* ctrl = reinterpret_cast<int32_t*>(base + bD + 2 * bQ);
                cudaStreamWaitEvent(L.stream, copied, 0);
                cudaMemcpyAsync(dd, descs.data(), descs.size() * sizeof(ExecDesc), cudaMemcpyHostToDevice, L.stream);
                if (ni) {
                    cudaMemcpyAsync(dq, hq.data(), ni * 4, cudaMemcpyHostToDevice, L.stream);
                    cudaMemcpyAsync(dqd, hd.data(), ni * 4, cudaMemcpyHostToDevice, L.stream);
                }
                cudaMemsetAsync(ctrl, 0, 256, L.stream);
                int grid = 0;
                ns_status_t r = exec_launch(dd, dq, dqd, ni, ctrl, K, TM, TK, bf16, S->cfg.tune.l2_hints != 0,
                                            dense, &grid, L.stream, nullptr, S->cfg.tune.chunk_nnz);
                const double t_start = serve_clock();
                for (SReq* q : rs) {
                    const SGraph& g = S->graphs[q->r.graph_id];
                    q->st.t_start = t_start;
                    if (g.m > 0)
                        cudaMemcpyAsync(q->r.C, q->dC, (size_t)g.m * q->r.K * 4, cudaMemcpyDeviceToHost, L.stream);
                }
                cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
                cudaEventRecord(L.ev, L.stream);
                std::lock_guard<std::mutex> lk(S->mu);
                if (r != NS_OK) {
                    for (SReq* q : rs) fail_req(S, q, r);
                    cudaEventSynchronize(L.ev);
                    cudaEventDestroy(L.ev);
                    cudaFreeAsync(L.block, L.stream);
                    continue;
                }
                for (SReq* q : rs) q->state = 2;
                S->launches.push_back(L);
            }
            cudaEventDestroy(copied);
        }
        // ---- retire finished launches ----
        for (auto it = S->launches.begin(); it != S->launches.end();) {
            if (cudaEventQuery(it->ev) != cudaSuccess) {
                (void)cudaGetLastError();
                ++it;
                continue;
            }
            const double t = serve_clock();
            std::lock_guard<std::mutex> lk(S->mu);
            for (SReq* q : it->reqs) {
                q->st.status = NS_OK;
                q->st.t_done = t;
                q->state = 3;
                cudaFreeAsync(q->block, it->stream);
                q->block = nullptr;
                S->inflight--;
                S->used -= q->bytes;
                q->sp->users--;
                q->sp->last_used = t;
            }
            cudaEventDestroy(it->ev);
            cudaFreeAsync(it->block, it->stream);
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
    if (cfg->hbm_budget_bytes <= 0 || cfg->max_inflight < 1 || cfg->max_queue < 1) {
        set_error("budget, max_inflight and max_queue must be positive");
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
    if (req_bytes(g, r->K, r->b_dtype) + est_plan_bytes(g) > S->cfg.hbm_budget_bytes) {
        set_error("request footprint exceeds the HBM budget");
        return NS_ERR_TOO_LARGE;
    }
    if ((int)S->queue.size() >= S->cfg.max_queue) {
        set_error("admission queue full");
        return NS_ERR_AGAIN;
    }
    SReq* q = new SReq();
    q->ticket = S->next_ticket++;
    q->r = *r;
    q->st.status = NS_OK;
    S->queue.push_back(q);
    S->reqs[q->ticket] = q;
    *ticket = q->ticket;
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
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    for (auto& kv : S->plans) delete kv.second.plan;
    for (auto& kv : S->reqs) delete kv.second;
    cudaStreamDestroy(S->s_plan);
    cudaStreamDestroy(S->s_copy);
    cudaStreamDestroy(S->s_exec[0]);
    cudaStreamDestroy(S->s_exec[1]);
    delete S;
    return NS_OK;
}

}  // extern "C"
