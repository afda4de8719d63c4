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
//            launch : every request admitted since the last launch joins ONE persistent launch
//                     per (size class, K, dtype, kernel) group: their B go up on the class's copy
//                     stream, their work lists are merged by cost class and each item carries its
//                     request's descriptor (staged through pinned host memory, so the upload never
//                     waits for running launches); the C copies follow the kernel, smallest
//                     first, each with its own event.  Requests whose B + C exceed 32 MB form the
//                     bulk class, with its own copy and execute streams, so small requests never
//                     queue behind a bulk request's copies; within a class launches alternate
//                     between two streams so a new batch overlaps the running ones;
//            retire : a request is done when its C copy's event completes; its memory returns
//                     to the budget and its device block to the server's block cache.
// Device blocks (a request's B, C and scratch; a launch's descriptors and work list) come from a
// cache of blocks whose last use the worker has seen complete, in power-of-two sizes, so reusing
// one never makes a stream wait for another's work and the steady state allocates nothing.
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
    size_t block_bytes = 0; // its size class
    void* dB = nullptr;
    float* dC = nullptr;
    float* slots = nullptr;
    int32_t* cnt = nullptr;
    int cls = 0;                    // size class: 1 = bulk
    cudaEvent_t done_ev = nullptr;  // recorded after the copy of C to the host
    const void* hB = nullptr;       // small requests with page-locked B and C: their device
    float* hC = nullptr;            // mappings, copied by SM loads (NULL: copy engines)
};

struct Pinned {
    void* p = nullptr;
    size_t bytes = 0;
};

struct SLaunch {
    std::vector<SReq*> reqs;      // requests not retired yet
    cudaEvent_t h2d_ev = nullptr;   // the group's B uploads done (timing)
    cudaEvent_t exec_ev = nullptr;  // its kernel done (timing)
    Pinned staging;               // descriptors, work list and ctrl, host side
    cudaEvent_t up_ev = nullptr;  // their upload has finished: the staging may be reused
    void* block = nullptr;        // the same on the device (back to the cache with the last request)
    size_t block_bytes = 0;
};

constexpr int64_t kBulkBytes = 32ll << 20;  // B + C above this: the bulk size class
// Bulk requests admitted at once (small ones pass waiting bulk ones).  The copy engines take
// copies in arrival order whatever their stream, so bulk transfers queued ahead of another copy
// delay it by their whole length; small requests with mapped host buffers use no copy engine at
// all (SM copies for B, C, counters and the launch's staging), so this cap only bounds how long
// a bulk request's own copies wait behind earlier bulk transfers.
constexpr int kBulkInflight = 8;

// Host<->device copies go in pieces of at most 4 MB: a copy engine switches between streams at
// copy boundaries, so a small request's copy waits at most one piece behind a bulk transfer.
constexpr size_t kCopyPiece = 4u << 20;

// Small requests' copies by SM loads and stores over the host link, when the host buffer is
// page-locked and mapped: they never queue behind a bulk request's transfer in a copy engine.
// 16-byte vectors, four in flight per thread, a few CTAs (the bulk launches leave SMs free).
__global__ void __launch_bounds__(256) k_copy16(uint4* __restrict__ dst, const uint4* __restrict__ src, int64_t n16)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}

static void copy_sm(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    const int64_t n16 = (int64_t)(bytes / 16);
    if (n16 == 0) return;
    int64_t blocks = (n16 + 4 * 256 - 1) / (4 * 256);
    if (blocks > 32) blocks = 32;
    k_copy16<<<(unsigned)blocks, 256, 0, s>>>(static_cast<uint4*>(dst), static_cast<const uint4*>(src), n16);
    count_launch();
    (void)cudaGetLastError();
}

// the device address of a page-locked, mapped host buffer (16-byte aligned), else NULL
static void* mapped(const void* h)
{
    if (!h || (reinterpret_cast<uintptr_t>(h) & 15u)) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    if (reinterpret_cast<uintptr_t>(at.devicePointer) & 15u) return nullptr;
    return at.devicePointer;
}

static void copy_pieces(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s)
{
    for (size_t off = 0; off < bytes; off += kCopyPiece) {
        const size_t len = bytes - off < kCopyPiece ? bytes - off : kCopyPiece;
        cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, len, kind, s);
    }
}

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
    int bulk_inflight = 0;
    int64_t used = 0;
    cudaStream_t s_plan = nullptr, s_copy[2] = {nullptr, nullptr};
    cudaStream_t s_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [size class][alternate]
    int flip[2] = {0, 0};
    std::list<SLaunch> launches;
    std::vector<Pinned> pinned_free;  // staging buffers ready for reuse (worker thread only)
    std::multimap<size_t, void*> dev_free;  // device blocks whose last use has completed (worker)
    cudaEvent_t ref_ev = nullptr;  // GPU time origin: completed at server clock t_ref
    void* zeros = nullptr;         // pinned zeros: split counters are cleared by a copy, not a kernel
    const void* zeros_dev = nullptr;  // their device address when mapped (SM copies), else NULL
    size_t zeros_bytes = 0;
    double t_ref = 0;
    size_t dev_cached = 0;
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
        if (q->cls) S->bulk_inflight--;
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
        const size_t eb = q->r.b_dtype == NS_BF16 ? 2 : 4;
        const int cls = (int64_t)(al256((size_t)g.n * q->r.K * eb) + al256((size_t)g.m * q->r.K * 4)) > kBulkBytes;
        if (cls && S->bulk_inflight >= kBulkInflight) {  // small requests behind it may pass
            ++it;
            continue;
        }
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
        q->cls = cls;
        S->bulk_inflight += cls;
        S->used += need;
        sp->last_used = now;
        q->state = 1;
        q->st.t_admit = now;
        q->st.t_planned = sp->t_ready > q->t_submit ? sp->t_ready : 0.0;
        S->inflight++;
        fresh.push_back(q);
    }
}

static size_t block_class(size_t bytes)
{
    size_t c = 64 << 10;
    while (c < bytes) c <<= 1;
    return c;
}

// a device block of at least `bytes` (its size class in *cls): the smallest cached block of that
// class or up to three classes larger, else a new one from the pool.  Growing the pool maps new
// memory, which holds the worker for milliseconds, so a larger idle block is the better choice.
static void* get_block(Server* S, size_t bytes, size_t* cls, cudaStream_t s)
{
    *cls = block_class(bytes);
    auto it = S->dev_free.lower_bound(*cls);
    if (it != S->dev_free.end() && it->first <= 8 * *cls) {
        void* p = it->second;
        *cls = it->first;
        S->dev_free.erase(it);
        S->dev_cached -= *cls;
        return p;
    }
    void* p = nullptr;
    if (pool_alloc(&p, *cls, s) != cudaSuccess) {
        (void)cudaGetLastError();
        // make room from the cache and try once more
        for (auto& kv : S->dev_free) cudaFreeAsync(kv.second, s);
        S->dev_free.clear();
        S->dev_cached = 0;
        if (pool_alloc(&p, *cls, s) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
    }
    return p;
}

// a block whose last use has completed goes back to the cache (at most half the budget is kept)
static void put_block(Server* S, void* p, size_t cls)
{
    if (!p) return;
    if ((int64_t)(S->dev_cached + cls) > S->cfg.hbm_budget_bytes / 2) {
        cudaFreeAsync(p, S->s_copy[0]);
        return;
    }
    S->dev_free.emplace(cls, p);
    S->dev_cached += cls;
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

// device memory of the fresh requests
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
        void* blk = get_block(S, bB + bC + bS + bN, &q->block_bytes, S->s_copy[q->cls]);
        if (!blk) {
            std::lock_guard<std::mutex> lk(S->mu);
            finish_req(S, q, NS_ERR_OOM);
            continue;
        }
        q->block = blk;
        q->dB = blk;
        q->hB = nullptr;
        q->hC = nullptr;
        if (q->cls == 0 && bB % 16 == 0 && bC % 16 == 0) {  // both mapped, or neither is used
            const void* mb = g.n > 0 ? mapped(q->r.B) : nullptr;
            void* mc = g.m > 0 ? mapped(q->r.C) : nullptr;
            if (mb && mc) {
                q->hB = mb;
                q->hC = static_cast<float*>(mc);
            }
        }
        q->dC = reinterpret_cast<float*>(static_cast<char*>(blk) + bB);
        q->slots = reinterpret_cast<float*>(static_cast<char*>(blk) + bB + bC);
        q->cnt = reinterpret_cast<int32_t*>(static_cast<char*>(blk) + bB + bC + bS);
        // split-row arrival counters start at zero: a copy from pinned zeros keeps the copy stream
        // off the SMs (a memset is a kernel, which would wait behind running SpMM launches).  A
        // request whose B and C move by SM copies clears them by an SM copy too: the copy engines
        // take copies in arrival order, so even this small copy would wait behind every piece of
        // a bulk transfer queued before it.
        if (q->hB && S->zeros_dev && bN <= S->zeros_bytes) copy_sm(q->cnt, S->zeros_dev, bN, S->s_copy[q->cls]);
        else if (bN <= S->zeros_bytes) cudaMemcpyAsync(q->cnt, S->zeros, bN, cudaMemcpyHostToDevice, S->s_copy[q->cls]);
        else cudaMemsetAsync(q->cnt, 0, bN, S->s_copy[q->cls]);
        ready.push_back(q);
    }
}

// one persistent launch for a group of requests sharing size class, K, dtype and kernel
static void launch_group(Server* S, std::vector<SReq*>& rs, int cls, int K, bool bf16, bool dense, int TM, int TK)
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
    cudaStream_t cs = S->s_copy[cls];
    cudaStream_t es = S->s_exec[cls][S->flip[cls]];
    S->flip[cls] ^= 1;
    const size_t bD = al256(descs.size() * sizeof(ExecDesc));
    const size_t bQ = al256((size_t)(ni > 0 ? ni : 1) * 4);
    const size_t total = bD + 2 * bQ + 256;
    SLaunch L;
    L.staging = get_pinned(S, total);
    void* block = L.staging.p ? get_block(S, total, &L.block_bytes, es) : nullptr;
    if (!block) {
        if (L.staging.p) S->pinned_free.push_back(L.staging);
        cudaStreamSynchronize(cs);  // the counters' memsets: then the blocks are idle
        std::lock_guard<std::mutex> lk(S->mu);
        for (SReq* q : rs) {
            put_block(S, q->block, q->block_bytes);
            q->block = nullptr;
            finish_req(S, q, NS_ERR_OOM);
        }
        return;
    }
    L.block = block;
    // B of every request on the class's copy stream
    for (SReq* q : rs) {
        const SGraph& g = S->graphs[q->r.graph_id];
        const size_t eb = q->r.b_dtype == NS_BF16 ? 2 : 4;
        if (g.n > 0) {
            if (q->hB) copy_sm(q->dB, q->hB, (size_t)g.n * q->r.K * eb, cs);
            else copy_pieces(q->dB, q->r.B, (size_t)g.n * q->r.K * eb, cudaMemcpyHostToDevice, cs);
        }
    }
    cudaEventCreate(&L.h2d_ev);
    cudaEventRecord(L.h2d_ev, cs);
    char* h = static_cast<char*>(L.staging.p);
    std::memcpy(h, descs.data(), descs.size() * sizeof(ExecDesc));
    int32_t* hq = reinterpret_cast<int32_t*>(h + bD);
    int32_t* hd = reinterpret_cast<int32_t*>(h + bD + bQ);
    for (int64_t j = 0; j < ni; ++j) {
        hq[j] = items[j].item;
        hd[j] = items[j].slot;
    }
    std::memset(h + bD + 2 * bQ, 0, 256);  // ctrl: work ticket and status
    char* base = static_cast<char*>(block);
    // the launch's descriptors and work list: by an SM copy when the staging is mapped (a copy
    // engine would queue it behind every bulk piece issued before it), else by a copy engine
    if (const void* hm = mapped(h)) copy_sm(base, hm, total, es);
    else cudaMemcpyAsync(base, h, total, cudaMemcpyHostToDevice, es);
    cudaEventCreateWithFlags(&L.up_ev, cudaEventDisableTiming);
    cudaEventRecord(L.up_ev, es);
    cudaStreamWaitEvent(es, L.h2d_ev, 0);
    // a bulk launch leaves a quarter of the GPU free, so small requests' launches start at once
    int grid = 0;
    if (cls) {
        const int contig = 0;
        if (exec_prepare(ni, K, TM, TK, bf16, S->cfg.tune.l2_hints != 0, dense, &grid, S->cfg.tune.chunk_nnz,
                         contig) != NS_OK)
            grid = 0;
        grid = grid > 4 ? grid * 3 / 4 : grid;
    }
    ns_status_t r = exec_launch(reinterpret_cast<ExecDesc*>(base), reinterpret_cast<int32_t*>(base + bD),
                                reinterpret_cast<int32_t*>(base + bD + bQ), ni,
                                reinterpret_cast<int32_t*>(base + bD + 2 * bQ), K, TM, TK, bf16,
                                S->cfg.tune.l2_hints != 0, dense, &grid, es, nullptr, S->cfg.tune.chunk_nnz);
    cudaEventCreate(&L.exec_ev);
    cudaEventRecord(L.exec_ev, es);
    const double t_start = serve_clock();
    // C back to the host, smallest first; each request's event follows its copy
    std::vector<SReq*> order(rs);
    std::stable_sort(order.begin(), order.end(), [&](const SReq* a, const SReq* b) {
        return (int64_t)S->graphs[a->r.graph_id].m * a->r.K < (int64_t)S->graphs[b->r.graph_id].m * b->r.K;
    });
    for (SReq* q : order) {
        const SGraph& g = S->graphs[q->r.graph_id];
        q->st.t_start = t_start;
        if (r == NS_OK && g.m > 0) {
            if (q->hC) copy_sm(q->hC, q->dC, (size_t)g.m * q->r.K * 4, es);
            else copy_pieces(q->r.C, q->dC, (size_t)g.m * q->r.K * 4, cudaMemcpyDeviceToHost, es);
        }
        cudaEventCreate(&q->done_ev);
        cudaEventRecord(q->done_ev, es);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (r != NS_OK) {
        cudaStreamSynchronize(es);
        for (SReq* q : rs) {
            cudaEventDestroy(q->done_ev);
            q->done_ev = nullptr;
            put_block(S, q->block, q->block_bytes);
            q->block = nullptr;
            finish_req(S, q, r);
        }
        cudaEventDestroy(L.up_ev);
        cudaEventDestroy(L.h2d_ev);
        cudaEventDestroy(L.exec_ev);
        S->pinned_free.push_back(L.staging);
        put_block(S, L.block, L.block_bytes);
        return;
    }
    for (SReq* q : rs) q->state = 2;
    L.reqs = order;
    S->launches.push_back(L);
}

// requests whose C has arrived are done; launches whose upload has finished give their staging
// back; lock not held
static void retire(Server* S)
{
    for (auto it = S->launches.begin(); it != S->launches.end();) {
        SLaunch& L = *it;
        if (L.up_ev && cudaEventQuery(L.up_ev) == cudaSuccess) {
            cudaEventDestroy(L.up_ev);
            L.up_ev = nullptr;
            S->pinned_free.push_back(L.staging);
            L.staging = Pinned{};
        }
        (void)cudaGetLastError();
        size_t keep = 0;
        for (size_t k = 0; k < L.reqs.size(); ++k) {
            SReq* q = L.reqs[k];
            if (cudaEventQuery(q->done_ev) != cudaSuccess) {
                (void)cudaGetLastError();
                L.reqs[keep++] = q;
                continue;
            }
            // GPU completion times on the server clock
            auto at = [&](cudaEvent_t e) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, S->ref_ev, e) != cudaSuccess) {
                    (void)cudaGetLastError();
                    return 0.0;
                }
                return S->t_ref + 1e-3 * ms;
            };
            q->st.t_h2d = at(L.h2d_ev);
            q->st.t_exec = at(L.exec_ev);
            q->st.t_d2h = at(q->done_ev);
            cudaEventDestroy(q->done_ev);
            q->done_ev = nullptr;
            put_block(S, q->block, q->block_bytes);  // its C copy, hence the kernel, has completed
            q->block = nullptr;
            std::lock_guard<std::mutex> lk(S->mu);
            finish_req(S, q, NS_OK);
        }
        L.reqs.resize(keep);
        if (L.reqs.empty() && !L.up_ev) {
            put_block(S, L.block, L.block_bytes);
            cudaEventDestroy(L.h2d_ev);
            cudaEventDestroy(L.exec_ev);
            it = S->launches.erase(it);
        } else {
            ++it;
        }
    }
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
            std::map<std::tuple<int, int, int, int, int, int>, std::vector<SReq*>> groups;
            for (SReq* q : ready) {
                const Plan* P = q->sp->plan;
                groups[{q->cls, q->r.K, (int)q->r.b_dtype, P->st.n_dwin > 0 ? 1 : 0, P->tune.TM, P->tune.TK}]
                    .push_back(q);
            }
            for (auto& kv : groups)  // small class first
                launch_group(S, kv.second, std::get<0>(kv.first), std::get<1>(kv.first),
                             std::get<2>(kv.first) == NS_BF16, std::get<3>(kv.first) != 0, std::get<4>(kv.first),
                             std::get<5>(kv.first));
        }
        retire(S);
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
    for (int c = 0; c < 2; ++c) {
        NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_copy[c], cudaStreamNonBlocking));
        NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_exec[c][0], cudaStreamNonBlocking));
        NS_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_exec[c][1], cudaStreamNonBlocking));
    }
    // the origin of GPU times: an event that completed just before t_ref
    S->zeros_bytes = 1 << 20;
    NS_CUDA_TRY(cudaHostAlloc(&S->zeros, S->zeros_bytes, cudaHostAllocDefault));
    std::memset(S->zeros, 0, S->zeros_bytes);
    S->zeros_dev = mapped(S->zeros);
    NS_CUDA_TRY(cudaEventCreate(&S->ref_ev));
    NS_CUDA_TRY(cudaEventRecord(S->ref_ev, S->s_exec[0][0]));
    NS_CUDA_TRY(cudaEventSynchronize(S->ref_ev));
    S->t_ref = serve_clock();
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
    for (auto& kv : S->dev_free) cudaFree(kv.second);
    cudaEventDestroy(S->ref_ev);
    if (S->zeros) cudaFreeHost(S->zeros);
    cudaStreamDestroy(S->s_plan);
    for (int c = 0; c < 2; ++c) {
        cudaStreamDestroy(S->s_copy[c]);
        cudaStreamDestroy(S->s_exec[c][0]);
        cudaStreamDestroy(S->s_exec[c][1]);
    }
    delete S;
    return NS_OK;
}

}  // extern "C"
