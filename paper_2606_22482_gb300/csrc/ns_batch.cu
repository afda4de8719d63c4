// ns_batch.cu -- the batched form and the autotuner.
//
// Batched form: many independent SpMMs (uneven graphs) share ONE persistent launch.  Each graph
// keeps its own plan; their work items are merged into one list ordered by Eq. 1 cost class
// (heaviest first across all graphs, Section 7 balanced lists), and every item carries the index
// of its graph's descriptor.  The launch is captured into a CUDA graph on the first execute and
// replayed afterwards; new operand pointers only refresh the descriptor table.
//
// Autotuner (Section 5.2.1 dry run, Section 8 threshold and tile-size sweeps): times the
// residual-only and dense-only extremes on the matrix to get P_res and P_tc, derives
// alpha0 = P_res / P_tc (Eq. 3 with r = 1: both classes share the SMs) and tau0 =
// ceil(alpha0 * TM * TK), then times tau in {1/2, 3/4, 1, 3/2, 2} * tau0 for each window height
// and keeps the fastest (execution time plus the plan time amortised over 200 runs, the
// paper's GCN setting).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ns_internal.cuh"

namespace ns {

struct Batch {
    struct Group {              // graphs sharing K (one persistent launch each)
        int K = 0;
        bool dense = false;
        bool contig = false;  // every plan of the group has a contiguous residual stream
        std::vector<int> graphs;
        ExecDesc* descs_dev = nullptr;
        int32_t* queue = nullptr;
        int32_t* queue_desc = nullptr;
        int32_t* ctrl = nullptr;
        int64_t n_items = 0;
        int grid = 0;
        int TM = 16, TK = 16, W = 256;
    };
    std::vector<Plan*> plans;
    std::vector<Group> groups;
    std::vector<ExecDesc> descs_host;   // per graph, in group order
    std::vector<const void*> lastB;
    std::vector<float*> lastC;
    ns_dtype_t dtype = NS_F32;
    bool hint = true;
    std::vector<DevBlock> blocks;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream for the one-time capture
    int64_t n_items = 0;
    ~Batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (Plan* p : plans) delete p;
        cudaStreamSynchronize(graph_stream);
        for (auto& b : blocks)
            if (b.ptr) cudaFree(b.ptr);
    }
};

static int cost_class_host(int64_t c)
{
    int b = 0;
    while (b < 62 && (c >> (b + 1)) > 0) ++b;
    return b;
}

}  // namespace ns

using namespace ns;

extern "C" {

ns_status_t ns_batch_plan(const ns_csr_t* As, int32_t count, const int32_t* Ks, ns_dtype_t b_dtype,
                          const ns_tune_t* tune, ns_stream_t s, ns_batch_t* out)
{
    if (!out || !As || !Ks || count < 0) {
        set_error("NULL argument or negative count");
        return NS_ERR_INVALID;
    }
    *out = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(s);
    Batch* Bt = new (std::nothrow) Batch();
    if (!Bt) {
        set_error("host allocation failed");
        return NS_ERR_OOM;
    }
    Bt->dtype = b_dtype;
    Bt->graph_stream = st;
    ns_tune_t t;
    if (tune) t = *tune;
    else ns_tune_default(&t);
    Bt->hint = t.l2_hints != 0;
    for (int32_t g = 0; g < count; ++g) {
        Plan* P = nullptr;
        ns_status_t r = plan_create(&As[g], Ks[g], b_dtype, &t, st, &P);
        if (r != NS_OK) {
            std::string msg = ns_last_error();
            delete Bt;
            set_error("graph %d: %s", g, msg.c_str());
            return r;
        }
        Bt->plans.push_back(P);
    }
    // group graphs by K
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Ks[a] < Ks[b]; });
    Bt->descs_host.resize(count);
    Bt->lastB.assign(count, nullptr);
    Bt->lastC.assign(count, nullptr);
    for (int q = 0; q < count;) {
        Batch::Group G;
        G.K = Ks[order[q]];
        G.TM = t.TM;
        G.TK = t.TK;
        G.W = t.chunk_nnz;
        while (q < count && Ks[order[q]] == G.K) G.graphs.push_back(order[q++]);
        Bt->groups.push_back(G);
    }
    // merged work lists: (cost class desc, graph asc, item order within the graph's own list)
    for (auto& G : Bt->groups) {
        struct It {
            int cls;
            int32_t graph_slot, item, rank;
        };
        std::vector<It> items;
        for (int gi = 0; gi < (int)G.graphs.size(); ++gi) {
            Plan* P = Bt->plans[G.graphs[gi]];
            G.dense = G.dense || P->st.n_dwin > 0;
            G.contig = (gi == 0 || G.contig) && plan_contig(P);
            int64_t n = P->st.n_items;
            std::vector<int64_t> cost(n);
            std::vector<int32_t> q(n);
            if (n) {
                if (cudaMemcpy(cost.data(), P->item_cost, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(q.data(), P->queue, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    delete Bt;
                    set_error("reading plan work lists failed");
                    return NS_ERR_CUDA;
                }
            }
            for (int64_t k = 0; k < n; ++k)
                items.push_back({cost_class_host(cost[q[k]]), gi, q[k], (int32_t)k});
        }
        std::stable_sort(items.begin(), items.end(), [](const It& a, const It& b) {
            if (a.cls != b.cls) return a.cls > b.cls;
            if (a.graph_slot != b.graph_slot) return a.graph_slot < b.graph_slot;
            return a.rank < b.rank;
        });
        G.n_items = (int64_t)items.size();
        Bt->n_items += G.n_items;
        Arena a;
        a.reserve(&G.descs_dev, (int64_t)G.graphs.size());
        a.reserve(&G.queue, G.n_items);
        a.reserve(&G.queue_desc, G.n_items);
        a.reserve(&G.ctrl, 8);
        ns_status_t r = a.commit(st);
        if (r != NS_OK) {
            delete Bt;
            return r;
        }
        Bt->blocks.push_back(a.take());
        std::vector<int32_t> hq(G.n_items), hd(G.n_items);
        for (int64_t k = 0; k < G.n_items; ++k) {
            hq[k] = items[k].item;
            hd[k] = items[k].graph_slot;
        }
        if (G.n_items &&
            (cudaMemcpyAsync(G.queue, hq.data(), G.n_items * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
             cudaMemcpyAsync(G.queue_desc, hd.data(), G.n_items * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
            delete Bt;
            set_error("uploading the merged work list failed");
            return NS_ERR_CUDA;
        }
        cudaMemsetAsync(G.ctrl, 0, sizeof(int32_t) * 8, st);
        cudaStreamSynchronize(st);
    }
    *out = reinterpret_cast<ns_batch_t>(Bt);
    return NS_OK;
}

ns_status_t ns_batch_execute(ns_batch_t b, const void* const* Bs, float* const* Cs, ns_stream_t s)
{
    Batch* Bt = reinterpret_cast<Batch*>(b);
    if (!Bt || !Bs || !Cs) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    const int count = (int)Bt->plans.size();
    bool changed = false;
    for (int g = 0; g < count; ++g) {
        const Plan* P = Bt->plans[g];
        if ((P->st.n > 0 && !Bs[g]) || (P->st.m > 0 && !Cs[g])) {
            set_error("graph %d: B or C is NULL", g);
            return NS_ERR_INVALID;
        }
        if ((reinterpret_cast<uintptr_t>(Bs[g]) & 15u) || (reinterpret_cast<uintptr_t>(Cs[g]) & 15u)) {
            set_error("graph %d: B and C must be 16-byte aligned", g);
            return NS_ERR_UNSUPPORTED;
        }
        if (Bs[g] != Bt->lastB[g] || Cs[g] != Bt->lastC[g]) changed = true;
    }
    if (changed) {
        for (auto& G : Bt->groups) {
            std::vector<ExecDesc> d(G.graphs.size());
            for (size_t k = 0; k < G.graphs.size(); ++k) {
                int g = G.graphs[k];
                fill_desc(Bt->plans[g], Bs[g], G.K, Cs[g], G.K, &d[k]);
                Bt->lastB[g] = Bs[g];
                Bt->lastC[g] = Cs[g];
            }
            NS_CUDA_TRY(cudaMemcpyAsync(G.descs_dev, d.data(), d.size() * sizeof(ExecDesc),
                                        cudaMemcpyHostToDevice, st));
            NS_CUDA_TRY(cudaStreamSynchronize(st));  // d is a local buffer
        }
    }
    if (!Bt->exec) {
        // capture every group's persistent launch once; later calls replay the graph
        for (auto& G : Bt->groups)  // occupancy queries and attributes outside the capture
            NS_TRY(exec_prepare(G.n_items, G.K, G.TM, G.TK, Bt->dtype == NS_BF16, Bt->hint, G.dense, &G.grid, G.W,
                                G.contig));
        // the caller's stream may be the legacy default stream, which cannot be captured: record
        // the launches on a private stream once; the graph then replays on the caller's stream
        if (!Bt->cap_stream) NS_CUDA_TRY(cudaStreamCreateWithFlags(&Bt->cap_stream, cudaStreamNonBlocking));
        NS_CUDA_TRY(cudaStreamBeginCapture(Bt->cap_stream, cudaStreamCaptureModeThreadLocal));
        ns_status_t r = NS_OK;
        for (auto& G : Bt->groups) {
            r = exec_launch(G.descs_dev, G.queue, G.queue_desc, G.n_items, G.ctrl, G.K, G.TM, G.TK,
                            Bt->dtype == NS_BF16, Bt->hint, G.dense, &G.grid, Bt->cap_stream, nullptr, G.W,
                            G.contig);
            if (r != NS_OK) break;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(Bt->cap_stream, &graph);
        if (r != NS_OK) return r;
        if (e != cudaSuccess) {
            set_error("stream capture failed: %s", cudaGetErrorString(e));
            return NS_ERR_CUDA;
        }
        Bt->graph = graph;
        count_launch(-(int64_t)Bt->groups.size());  // recorded, not launched: counted at replay
        NS_CUDA_TRY(cudaGraphInstantiate(&Bt->exec, graph, 0));
    }
    NS_CUDA_TRY(cudaGraphLaunch(Bt->exec, st));
    count_launch((int64_t)Bt->groups.size());
    Bt->graph_stream = st;
    return NS_OK;
}

ns_status_t ns_batch_stats(ns_batch_t b, int64_t* n_items, int64_t* n_graphs)
{
    Batch* Bt = reinterpret_cast<Batch*>(b);
    if (!Bt) {
        set_error("NULL batch");
        return NS_ERR_INVALID;
    }
    if (n_items) *n_items = Bt->n_items;
    if (n_graphs) *n_graphs = (int64_t)Bt->plans.size();
    return NS_OK;
}

ns_status_t ns_batch_destroy(ns_batch_t b)
{
    delete reinterpret_cast<Batch*>(b);
    return NS_OK;
}

// The residual chunk size W of the whole batch: every candidate is planned as a batch and its
// launch timed (best of three replays after a warm one), the rest of the tune kept.
ns_status_t ns_batch_autotune(const ns_csr_t* As, int32_t count, const int32_t* Ks, ns_dtype_t b_dtype,
                              const ns_tune_t* start, const void* const* Bs, float* const* Cs,
                              ns_stream_t s, ns_tune_t* out, double* best_ms)
{
    if (!As || count <= 0 || !Ks || !Bs || !Cs || !out) {
        set_error("NULL argument or empty batch");
        return NS_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    ns_tune_t base;
    if (start) base = *start;
    else ns_tune_default(&base);
    const int32_t Ws[4] = {128, 256, 512, 1024};
    ns_tune_t best = base;
    double best_t = 1e300;
    cudaEvent_t e0, e1;
    NS_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return NS_ERR_CUDA;
    }
    ns_status_t r = NS_OK;
    for (int32_t w : Ws) {
        ns_tune_t t = base;
        t.chunk_nnz = w;
        t.absorb_cap = w;
        ns_batch_t b = nullptr;
        r = ns_batch_plan(As, count, Ks, b_dtype, &t, s, &b);
        if (r == NS_ERR_UNSUPPORTED || r == NS_ERR_INVALID) {  // this W does not apply; try the next
            r = NS_OK;
            continue;
        }
        if (r != NS_OK) break;
        double t_best = 1e300;
        for (int rep = 0; rep < 4 && r == NS_OK; ++rep) {
            cudaEventRecord(e0, st);
            r = ns_batch_execute(b, Bs, Cs, s);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) r = NS_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < t_best) t_best = ms;  // the first replay captures the graph
        }
        ns_batch_destroy(b);
        if (r != NS_OK) break;
        if (t_best < best_t) {
            best_t = t_best;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != NS_OK) return r;
    if (best_t >= 1e300) {
        set_error("no chunk size applies to this batch");
        return NS_ERR_UNSUPPORTED;
    }
    *out = best;
    if (best_ms) *best_ms = best_t;
    return NS_OK;
}

// ---------------------------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------------------------
static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// best of two plans + best-of-3 execute of one tune; returns execute ms and plan ms.  The first
// plan of a configuration also pays one-time costs (kernels loaded on first use), which would
// count against whichever candidate happens to be tried first.
static ns_status_t time_tune(const ns_csr_t* A, int32_t K, ns_dtype_t dt, const ns_tune_t& t,
                             const void* Bd, float* Cd, cudaStream_t st, double* exec_ms,
                             double* plan_ms, Plan** keep)
{
    Plan* P = nullptr;
    double t0 = now_s();
    NS_TRY(plan_create(A, K, dt, &t, st, &P));
    *plan_ms = (now_s() - t0) * 1e3;
    delete P;
    P = nullptr;
    t0 = now_s();
    NS_TRY(plan_create(A, K, dt, &t, st, &P));
    const double again = (now_s() - t0) * 1e3;
    if (again < *plan_ms) *plan_ms = again;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    ns_status_t r = NS_OK;
    for (int rep = 0; rep < 4 && r == NS_OK; ++rep) {
        cudaEventRecord(e0, st);
        r = ns_spmm_execute(reinterpret_cast<ns_plan_t>(P), Bd, K, Cd, K, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) r = NS_ERR_CUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first run warms caches and the grid size
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *exec_ms = best;
    if (keep) *keep = P;
    else delete P;
    return r;
}

// A fresh plan for every execute: the whole cycle (plan, execute, release), best of two, which is
// what a caller that re-plans every step pays (launch gaps and the release included).
static ns_status_t time_cycle(const ns_csr_t* A, int32_t K, ns_dtype_t dt, const ns_tune_t& t,
                              const void* Bd, float* Cd, cudaStream_t st, double* cycle_ms, int reps = 2)
{
    double best = 1e30;
    for (int rep = 0; rep < reps; ++rep) {
        const double t0 = now_s();
        Plan* P = nullptr;
        NS_TRY(plan_create(A, K, dt, &t, st, &P));
        ns_status_t r = ns_spmm_execute(reinterpret_cast<ns_plan_t>(P), Bd, K, Cd, K, st);
        delete P;
        if (r != NS_OK) return r;
        NS_CUDA_TRY(cudaStreamSynchronize(st));
        const double ms = (now_s() - t0) * 1e3;
        if (ms < best) best = ms;
    }
    *cycle_ms = best;
    return NS_OK;
}

int32_t ns_rebalance_next(int32_t lo, int32_t hi, int32_t tau, double dt_tc, double dt_res, double eps,
                          int32_t* lo_out, int32_t* hi_out, int32_t* tau_out)
{
    const double mx = dt_tc > dt_res ? dt_tc : dt_res, mn = dt_tc > dt_res ? dt_res : dt_tc;
    if (mn > 0 && mx / mn <= 1.0 + eps) {  // balanced (Eq. 6)
        *lo_out = lo;
        *hi_out = hi;
        *tau_out = tau;
        return 1;
    }
    if (dt_tc > dt_res) lo = tau;  // the tensor side finishes last: fewer dense tiles
    else hi = tau;                 // the CUDA-core side finishes last: more dense tiles
    *lo_out = lo;
    *hi_out = hi;
    if (hi - lo <= 1) {
        *tau_out = tau;
        return 1;
    }
    *tau_out = lo + (hi - lo) / 2;
    return 0;
}

ns_status_t ns_rebalance(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, const void* B, int64_t ldb,
                         float* C, int64_t ldc, ns_stream_t s, const ns_tune_t* start, double eps,
                         int32_t max_iter, ns_tune_t* out, ns_rebalance_report_t* report)
{
    if (!A || !out || !B || !C) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    if (!A->on_device) {
        set_error("ns_rebalance needs a device CSR");
        return NS_ERR_INVALID;
    }
    if (max_iter < 1 || max_iter > 16 || !(eps >= 0)) {
        set_error("max_iter must be in 1..16 and eps >= 0");
        return NS_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    ns_tune_t t;
    if (start) t = *start;
    else ns_tune_default(&t);
    NS_TRY(plan_check_tune(t));
    int32_t lo = 0, hi = t.TM * t.TK + 1;
    int32_t tau = (t.tau_tile >= 1 && t.tau_tile <= t.TM * t.TK) ? t.tau_tile : lo + (hi - lo) / 2;
    ns_rebalance_report_t rep{};
    unsigned long long* clk = nullptr;
    NS_CUDA_TRY(pool_alloc(reinterpret_cast<void**>(&clk), 3 * sizeof(unsigned long long), st));
    static const unsigned long long kReset[3] = {~0ull, 0ull, 0ull};
    int32_t best_tau = tau;
    double best_span = 1e300;
    ns_status_t r = NS_OK;
    for (int it = 0; it < max_iter; ++it) {
        t.tau_tile = tau;
        Plan* P = nullptr;
        r = plan_create(A, K, b_dtype, &t, st, &P);
        if (r != NS_OK) break;
        // one untimed epoch (caches, grid size), then the stamped one
        r = ns_spmm_execute(reinterpret_cast<ns_plan_t>(P), B, ldb, C, ldc, st);
        unsigned long long h[3] = {0, 0, 0};
        if (r == NS_OK) {
            P->class_clock = clk;
            if (cudaMemcpyAsync(clk, kReset, sizeof kReset, cudaMemcpyHostToDevice, st) != cudaSuccess)
                r = NS_ERR_CUDA;
            if (r == NS_OK) r = ns_spmm_execute(reinterpret_cast<ns_plan_t>(P), B, ldb, C, ldc, st);
            if (r == NS_OK && (cudaMemcpyAsync(h, clk, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                               cudaStreamSynchronize(st) != cudaSuccess))
                r = NS_ERR_CUDA;
            P->class_clock = nullptr;
        }
        delete P;
        if (r != NS_OK) break;
        const double dt_tc = h[1] > h[0] ? (double)(h[1] - h[0]) * 1e-6 : 0.0;
        const double dt_res = h[2] > h[0] ? (double)(h[2] - h[0]) * 1e-6 : 0.0;
        rep.tau[it] = tau;
        rep.dt_tc_ms[it] = dt_tc;
        rep.dt_res_ms[it] = dt_res;
        rep.skew[it] = ns_skew(dt_tc, dt_res);
        rep.iterations = it + 1;
        const double span = dt_tc > dt_res ? dt_tc : dt_res;
        if (span < best_span) {
            best_span = span;
            best_tau = tau;
        }
        const double mn = dt_tc > dt_res ? dt_res : dt_tc;
        if (mn > 0 && span / mn <= 1.0 + eps) rep.converged = 1;
        if (ns_rebalance_next(lo, hi, tau, dt_tc, dt_res, eps, &lo, &hi, &tau)) break;
    }
    cudaFreeAsync(clk, st);
    cudaStreamSynchronize(st);
    if (r != NS_OK) return r;
    *out = t;
    out->tau_tile = best_tau;
    if (report) *report = rep;
    return NS_OK;
}

ns_status_t ns_autotune(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, ns_stream_t s,
                        ns_tune_t* out, ns_tune_report_t* report)
{
    if (!A || !out) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    if (!A->on_device) {
        set_error("ns_autotune needs a device CSR");
        return NS_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    const size_t eb = b_dtype == NS_BF16 ? 2 : 4;
    void* Bd = nullptr;
    float* Cd = nullptr;
    NS_CUDA_TRY(pool_alloc(&Bd, (size_t)(A->n > 0 ? A->n : 1) * K * eb, st));
    NS_CUDA_TRY(pool_alloc(reinterpret_cast<void**>(&Cd), (size_t)(A->m > 0 ? A->m : 1) * K * 4, st));
    NS_CUDA_TRY(cudaMemsetAsync(Bd, 0, (size_t)(A->n > 0 ? A->n : 1) * K * eb, st));
    auto release = [&]() {
        cudaFreeAsync(Bd, st);
        cudaFreeAsync(Cd, st);
        cudaStreamSynchronize(st);
    };

    ns_tune_t base;
    ns_tune_default(&base);
    // plan cost amortised over the executions of one plan (default: a 200-epoch workload)
    const double amort = (report && report->plan_runs > 0) ? report->plan_runs : 200.0;
    int trials = 0;
    ns_tune_t best = base;
    double best_cost = 1e300, best_exec = 0;
    struct Seen {
        double cost, exec;
        ns_tune_t t;
    };
    std::vector<Seen> seen;  // every candidate with its cost
    auto consider = [&](const ns_tune_t& t, double ex, double pl) {
        double c = ex + pl / amort;
        if (amort <= 1.0) {  // re-planned every execute: time the whole cycle as the caller runs it
            double cyc = 0;
            if (time_cycle(A, K, b_dtype, t, Bd, Cd, st, &cyc) == NS_OK) c = cyc;
        }
        seen.push_back({c, ex, t});
        ++trials;
        if (c < best_cost) {
            best_cost = c;
            best = t;
            best_exec = ex;
        }
    };

    // dry run 1: the vector-engine extreme (every nonzero on the CUDA cores)
    ns_tune_t tr = base;
    tr.tau_tile = NS_TAU_INF;
    double ex_res = 0, pl_res = 0;
    ns_status_t r = time_tune(A, K, b_dtype, tr, Bd, Cd, st, &ex_res, &pl_res, nullptr);
    if (r != NS_OK) {
        release();
        return r;
    }
    consider(tr, ex_res, pl_res);
    const double p_res = ex_res > 0 ? (double)A->nnz * K / (ex_res * 1e-3) : 0.0;

    // dry run 2: the matrix-engine extreme (every compacted tile dense) at TM = 16
    double p_tc = 0.0;
    {
        ns_tune_t td = base;
        td.tau_tile = 1;
        Plan* P = nullptr;
        double ex = 0, pl = 0;
        r = time_tune(A, K, b_dtype, td, Bd, Cd, st, &ex, &pl, &P);
        if (r == NS_OK) {
            consider(td, ex, pl);
            double elems = (double)P->st.n_dtiles * td.TM * td.TK;
            p_tc = ex > 0 ? elems * K / (ex * 1e-3) : 0.0;
        }
        delete P;
        if (r != NS_OK && r != NS_ERR_UNSUPPORTED) {
            release();
            return r;
        }
    }
    const double alpha0 = p_tc > 0 ? p_res / p_tc : 1.0;

    // sweeps: tile shape (window height x compacted width) x tau around tau0 (Section 8
    // threshold and tile-size studies)
    const int TMs[3] = {16, 32, 64};
    const int TKs[2] = {16, 32};
    const double mult[5] = {0.5, 0.75, 1.0, 1.5, 2.0};
    for (int TK : TKs)
    for (int TM : TMs) {
        if ((int64_t)TM * K > 16384) continue;
        int32_t tau0 = ns_cost_tau(alpha0, TM, TK);
        int32_t last = -1;
        for (double mu : mult) {
            int32_t tau = (int32_t)std::ceil(mu * tau0);
            if (tau < 2) tau = 2;
            if (tau > TM * TK) tau = TM * TK;
            if (tau == last) continue;
            last = tau;
            ns_tune_t t = base;
            t.TM = TM;
            t.TK = TK;
            t.tau_tile = tau;
            double ex = 0, pl = 0;
            r = time_tune(A, K, b_dtype, t, Bd, Cd, st, &ex, &pl, nullptr);
            if (r == NS_OK) consider(t, ex, pl);
            else if (r != NS_ERR_UNSUPPORTED) {
                release();
                return r;
            }
        }
    }
    // residual chunk size W and the L2 policy of the best configuration so far
    {
        const ns_tune_t base_best = best;
        const int32_t Ws[3] = {128, 512, 1024};
        for (int32_t w : Ws) {
            if (w == base_best.chunk_nnz) continue;
            ns_tune_t t = base_best;
            t.chunk_nnz = w;
            t.absorb_cap = w;
            double ex = 0, pl = 0;
            r = time_tune(A, K, b_dtype, t, Bd, Cd, st, &ex, &pl, nullptr);
            if (r == NS_OK) consider(t, ex, pl);
            else if (r != NS_ERR_UNSUPPORTED) {
                release();
                return r;
            }
        }
        ns_tune_t t = best;
        t.l2_hints = 2;
        double ex = 0, pl = 0;
        r = time_tune(A, K, b_dtype, t, Bd, Cd, st, &ex, &pl, nullptr);
        if (r == NS_OK) consider(t, ex, pl);
        else if (r != NS_ERR_UNSUPPORTED) {
            release();
            return r;
        }
    }
    // column slices (Section 6.2.2 N shaping): narrower passes keep the gathered B rows in L2
    {
        const ns_tune_t base_best = best;
        for (int div = 2; div <= 4; div *= 2) {
            const int32_t tn = (K / div) & ~7;
            if (tn < 32 || tn >= K) continue;
            ns_tune_t t = base_best;
            t.TN = tn;
            double ex = 0, pl = 0;
            r = time_tune(A, K, b_dtype, t, Bd, Cd, st, &ex, &pl, nullptr);
            if (r == NS_OK) consider(t, ex, pl);
            else if (r != NS_ERR_UNSUPPORTED) {
                release();
                return r;
            }
        }
    }
    // Re-planned every execute, the whole-cycle times of the leading candidates are close and
    // noisy: time the three best again, longer, and keep the fastest.
    if (amort <= 1.0 && seen.size() > 1) {
        std::stable_sort(seen.begin(), seen.end(), [](const Seen& x, const Seen& y) { return x.cost < y.cost; });
        double best_c = 1e30;
        for (size_t k = 0; k < seen.size() && k < 3; ++k) {
            double cyc = 0;
            if (time_cycle(A, K, b_dtype, seen[k].t, Bd, Cd, st, &cyc, 6) != NS_OK) continue;
            if (cyc < best_c) {
                best_c = cyc;
                best = seen[k].t;
                best_exec = seen[k].exec;
            }
        }
    }
    release();
    *out = best;
    if (report) {
        report->p_res = p_res;
        report->p_tc = p_tc;
        report->alpha0 = alpha0;
        report->best_ms = best_exec;
        report->trials = trials;
    }
    return NS_OK;
}

}  // extern "C"
