// ns_api.cu -- the C ABI (include/ns_spmm.h): argument checks, plan lifetime, export, execute.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "ns_internal.cuh"

namespace ns {

static thread_local std::string t_err;
std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {nullptr};

static cudaMemPool_t pool_for(int dev)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pl = nullptr;
        if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool[dev] = pl;
    }
    return g_pool[dev];
}

static std::mutex g_inject_mu;
static int32_t g_alloc_countdown = -1;  // injection: allocations to pass before one fails

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s)
{
    {
        std::lock_guard<std::mutex> lk(g_inject_mu);
        if (g_alloc_countdown == 0) {
            g_alloc_countdown = -1;
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_countdown > 0) --g_alloc_countdown;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pl = pool_for(dev);
    if (!pl) return cudaMallocAsync(p, bytes, s);
    return cudaMallocFromPoolAsync(p, bytes, pl, s);
}

void pool_trim()
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& pl : g_pool)
        if (pl) cudaMemPoolTrimTo(pl, 0);
}

ns_status_t Arena::commit(cudaStream_t s)
{
    size_t total = 0;
    for (auto& r : reqs) total += (r.bytes + 255) & ~size_t(255);
    if (total == 0) total = 256;
    void* p = nullptr;
    cudaError_t e = pool_alloc(&p, total, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", total, cudaGetErrorString(e));
        return NS_ERR_OOM;
    }
    block.ptr = p;
    block.bytes = total;
    stream = s;
    size_t off = 0;
    for (auto& r : reqs) {
        *r.slot = static_cast<char*>(p) + off;
        off += (r.bytes + 255) & ~size_t(255);
    }
    return NS_OK;
}

void Arena::release(cudaStream_t s)
{
    if (block.ptr) {
        cudaFreeAsync(block.ptr, s ? s : stream);
        block = DevBlock{};
    }
    reqs.clear();
}

// Stream-ordered release: the blocks go back to the pool after everything already enqueued on
// the stream of the last plan/execute call, so a destroy right after an asynchronous execute
// never frees memory a running kernel still reads.
Plan::~Plan()
{
    if (status_ev) cudaEventDestroy(status_ev);
    bool failed = false;
    for (auto& b : blocks) {
        if (!b.ptr) continue;
        if (!failed && cudaFreeAsync(b.ptr, last_stream) != cudaSuccess) {
            (void)cudaGetLastError();
            failed = true;
            cudaDeviceSynchronize();
        }
        if (failed) cudaFree(b.ptr);
        b.ptr = nullptr;
    }
}

// pinned host slots for the status words of plans (one slab for the process)
static std::mutex g_slab_mu;
static int32_t* g_slab = nullptr;
static uint32_t g_slab_next = 0;
constexpr uint32_t kSlabSlots = 65536;

static int32_t* status_slot()
{
    std::lock_guard<std::mutex> lk(g_slab_mu);
    if (!g_slab) {
        if (cudaHostAlloc(reinterpret_cast<void**>(&g_slab), kSlabSlots * sizeof(int32_t), 0) != cudaSuccess) {
            (void)cudaGetLastError();
            g_slab = nullptr;
            return nullptr;
        }
        memset(g_slab, 0, kSlabSlots * sizeof(int32_t));
    }
    int32_t* p = g_slab + (g_slab_next++ % kSlabSlots);
    *p = 0;
    return p;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static ns_status_t check_csr_args(const ns_csr_t* A)
{
    if (!A) {
        set_error("A is NULL");
        return NS_ERR_INVALID;
    }
    if (A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz > 2147483647LL) {
        set_error("bad CSR shape m=%d n=%d nnz=%lld", A->m, A->n, (long long)A->nnz);
        return NS_ERR_INVALID;
    }
    if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->vals))) {
        set_error("CSR arrays missing");
        return NS_ERR_INVALID;
    }
    // merge items (nnz + m) are counted in int32
    if ((int64_t)A->m + A->nnz > 2147483647LL) {
        set_error("m + nnz must be < 2^31");
        return NS_ERR_UNSUPPORTED;
    }
    return NS_OK;
}

static ns_status_t check_K(int32_t K)
{
    if (K < 8 || K > 1024 || (K % 8) != 0) {
        set_error("K=%d unsupported: need 8 <= K <= 1024 and K %% 8 == 0", K);
        return NS_ERR_UNSUPPORTED;
    }
    return NS_OK;
}

ns_status_t plan_create(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, const ns_tune_t* tune,
                        cudaStream_t st, Plan** out)
{
    *out = nullptr;
    NS_TRY(check_csr_args(A));
    NS_TRY(check_K(K));
    if (b_dtype != NS_F32 && b_dtype != NS_BF16) {
        set_error("unknown dtype");
        return NS_ERR_INVALID;
    }
    ns_tune_t t;
    if (tune) t = *tune;
    else ns_tune_default(&t);
    if (plan_check_tune(t) != NS_OK) {
        set_error("invalid tune (TM in {16,32,64}, TK in {16,32}, group=%d, chunk_nnz >= 2)", kExecWarps);
        return NS_ERR_INVALID;
    }
    Plan* P = new (std::nothrow) Plan();
    if (!P) {
        set_error("host allocation failed");
        return NS_ERR_OOM;
    }
    cudaGetDevice(&P->device);
    P->last_stream = st;
    ns_status_t r = plan_build(P, A, K, b_dtype, &t, st);
    if (r != NS_OK) {
        cudaStreamSynchronize(st);
        (void)cudaGetLastError();
        delete P;
        return r;
    }
    P->st.device_bytes = 0;
    for (auto& b : P->blocks) P->st.device_bytes += (int64_t)b.bytes;
    *out = P;
    return NS_OK;
}

}  // namespace ns

using namespace ns;

extern "C" {

void ns_tune_default(ns_tune_t* t)
{
    if (!t) return;
    t->TM = 16;
    t->TK = 16;
    t->tau_tile = NS_TAU_INF;
    t->tau_row = 0;
    t->tau_col = 0;
    t->col_order = 0;
    t->chunk_nnz = 256;
    t->absorb_cap = 256;
    t->group = kExecWarps;
    t->cost_tc = 1;
    t->cost_res = 8;
    t->l2_hints = 1;
    t->TN = 0;
    t->reorder = 0;
}

const char* ns_last_error(void) { return t_err.c_str(); }

int64_t ns_launch_count(void) { return g_launches.load(); }

ns_status_t ns_inject_alloc_failure(int32_t after)
{
    if (after < -1) {
        set_error("after must be >= -1");
        return NS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_alloc_countdown = after;
    return NS_OK;
}

ns_status_t ns_plan_inject_status(ns_plan_t p, int32_t bits)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    if (!P || bits == 0 || (bits & ~(kStatusTimeout | kStatusInternal))) {
        set_error("NULL plan or status bits outside 2 | 4");
        return NS_ERR_INVALID;
    }
    int32_t cur = 0;
    NS_CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    NS_CUDA_TRY(cudaMemcpy(&cur, P->ctrl + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
    cur |= bits;
    NS_CUDA_TRY(cudaMemcpy(P->ctrl + 2, &cur, sizeof(int32_t), cudaMemcpyHostToDevice));
    return NS_OK;
}

int32_t ns_device_ok(void)
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return (prop.major == 10 && prop.minor == 3) ? 1 : 0;
}

ns_status_t ns_spmm_plan(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, const ns_tune_t* tune,
                         ns_stream_t s, ns_plan_t* out)
{
    if (!out) {
        set_error("out is NULL");
        return NS_ERR_INVALID;
    }
    *out = nullptr;
    Plan* P = nullptr;
    NS_TRY(plan_create(A, K, b_dtype, tune, static_cast<cudaStream_t>(s), &P));
    *out = reinterpret_cast<ns_plan_t>(P);
    return NS_OK;
}

ns_status_t ns_spmm_execute(ns_plan_t p, const void* B, int64_t ldb, float* C, int64_t ldc,
                            ns_stream_t s)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    if (!P) {
        set_error("plan is NULL");
        return NS_ERR_INVALID;
    }
    if ((P->st.n > 0 && !B) || (P->st.m > 0 && !C)) {
        set_error("B or C is NULL");
        return NS_ERR_INVALID;
    }
    if (ldb < P->K || ldc < P->K) {
        set_error("ldb/ldc smaller than K");
        return NS_ERR_INVALID;
    }
    if (!aligned16(B) || !aligned16(C) || (ldb % 8) || (ldc % 8)) {
        set_error("B and C must be 16-byte aligned with ldb, ldc multiples of 8");
        return NS_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    if (st != P->last_stream) {
        // later frees are ordered on the new stream; make it wait for the old one first
        cudaEvent_t ev;
        NS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, P->last_stream);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        P->last_stream = st;
    }
    // the device status word of an earlier launch, if its pinned copy has already landed
    // (never waits: a launch still running is checked by a later call)
    if (P->status_ev && cudaEventQuery(P->status_ev) == cudaSuccess) {
        const int32_t status = *P->status_host;
        if (status & kStatusTimeout) {
            set_error("an earlier launch gave up a bounded wait");
            return NS_ERR_TIMEOUT;
        }
        if (status) {
            set_error("an earlier launch found an out-of-range plan index (status %d); results of "
                      "that launch are invalid", status);
            return NS_ERR_CUDA;
        }
    }
    (void)cudaGetLastError();
    const int32_t TN = (P->tune.TN > 0 && P->tune.TN < P->K) ? P->tune.TN : P->K;
    const size_t es = P->dtype == NS_BF16 ? 2 : 4;
    for (int32_t c0 = 0; c0 < P->K; c0 += TN) {
        // column slice [c0, c0 + w): B and C shifted by c0 columns, same leading dimensions
        const int32_t w = P->K - c0 < TN ? P->K - c0 : TN;
        fill_desc(P, static_cast<const char*>(B) + (size_t)c0 * es, ldb, C + c0, ldc, &P->desc_host);
        P->desc_host.K = w;
        P->desc_valid = true;
        NS_TRY(exec_launch_plan(P, st));
    }
    if (!P->status_host) {
        P->status_host = status_slot();
        if (P->status_host) cudaEventCreateWithFlags(&P->status_ev, cudaEventDisableTiming);
    }
    if (P->status_host && P->status_ev) {
        cudaMemcpyAsync(P->status_host, P->ctrl + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaEventRecord(P->status_ev, st);
    }
    return NS_OK;
}

ns_status_t ns_plan_stats(ns_plan_t p, ns_plan_stats_t* st)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    if (!P || !st) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    *st = P->st;
    return NS_OK;
}

struct ArrayRef {
    const void* ptr;
    int64_t count;
    int32_t esize;
};

static bool find_array(Plan* P, const char* name, ArrayRef* a)
{
    const int64_t TM = P->st.TM, TK = P->st.TK, BW = TM * TK / 32;
    const ns_plan_stats_t& s = P->st;
#define A(x, ptr_, cnt, es)                                                                    \
    if (!strcmp(name, #x)) {                                                                   \
        *a = ArrayRef{ptr_, (cnt), (es)};                                                      \
        return true;                                                                           \
    }
    A(aic_rows, P->aic_rows, s.m_aic, 4)
    A(win_rows, P->win_rows, s.n_win * TM, 4)
    A(win_dptr, P->win_dptr, s.n_win + 1, 4)
    A(dwin, P->dwin, s.n_dwin, 4)
    A(dwin_absorb, P->dwin_absorb, s.n_dwin, 4)
    A(dtile_cols, P->dtile_cols, s.n_dtiles * TK, 4)
    A(dtile_bits, P->dtile_bits, s.n_dtiles * BW, 4)
    A(dtile_voff, P->dtile_voff, s.n_dtiles + 1, 4)
    A(dtile_vals, P->dtile_vals, s.n_dvals, s.b_bf16 ? 2 : 4)
    A(dtile_x, P->dtile_x, s.b_bf16 ? s.n_dtiles * TM * TK : 0, 2)
    A(res_rowptr, P->res_rowptr, s.m + 1, 4)
    A(res_col, P->res_col, s.n_res, 4)
    A(res_val, P->res_val, s.n_res, 4)
    A(rl_rows, P->rl_rows, s.n_rl, 4)
    A(rl_start, P->rl_start, s.n_rl + 1, 4)
    A(chunk_b, P->chunk_b, s.n_chunks + 1, 4)
    A(chunk_k0, P->chunk_k0, s.n_chunks, 4)
    A(row_split, P->row_split, s.m, 4)
    A(split_row, P->split_row, s.n_split, 4)
    A(split_np, P->split_np, s.n_split, 4)
    A(split_slot, P->split_slot, s.n_split, 4)
    A(split_base, P->split_base, s.n_split, 4)
    A(queue, P->queue, s.n_items, 4)
    A(item_cost, P->item_cost, s.n_items, 8)
#undef A
    return false;
}

ns_status_t ns_plan_array_info(ns_plan_t p, const char* name, int64_t* count, int32_t* esize)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    ArrayRef a;
    if (!P || !name || !count || !esize) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    if (!find_array(P, name, &a)) {
        set_error("unknown plan array '%s'", name);
        return NS_ERR_NOT_FOUND;
    }
    // arrays a plan does not materialise (no windows) export as zeros of the reference length
    *count = a.count;
    *esize = a.esize;
    return NS_OK;
}

ns_status_t ns_plan_export(ns_plan_t p, const char* name, void* host_dst, int64_t bytes)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    ArrayRef a;
    if (!P || !name) {
        set_error("NULL argument");
        return NS_ERR_INVALID;
    }
    if (!find_array(P, name, &a)) {
        set_error("unknown plan array '%s'", name);
        return NS_ERR_NOT_FOUND;
    }
    int64_t need = a.count * a.esize;
    if (need == 0) return NS_OK;
    if (!host_dst || bytes < need) {
        set_error("destination too small: need %lld bytes", (long long)need);
        return NS_ERR_INVALID;
    }
    if (!a.ptr) {
        memset(host_dst, 0, (size_t)need);
        return NS_OK;
    }
    NS_CUDA_TRY(cudaMemcpy(host_dst, a.ptr, (size_t)need, cudaMemcpyDeviceToHost));
    return NS_OK;
}

ns_status_t ns_plan_destroy(ns_plan_t p)
{
    Plan* P = reinterpret_cast<Plan*>(p);
    if (!P) return NS_OK;
    delete P;
    return NS_OK;
}

double ns_cost_alpha(double p_res, double p_tc, double r) { return p_tc > 0 ? r * p_res / p_tc : 0.0; }

int32_t ns_cost_tau(double alpha, int32_t TM, int32_t TK)
{
    double t = alpha * (double)TM * (double)TK;
    if (!(t < 2147483646.0)) return NS_TAU_INF;
    double c = (double)(int64_t)t;
    if (c < t) c += 1.0;
    return (int32_t)c;
}

double ns_skew(double dt_tc, double dt_res)
{
    double hi = dt_tc > dt_res ? dt_tc : dt_res;
    double lo = dt_tc > dt_res ? dt_res : dt_tc;
    return lo > 0 ? hi / lo : 0.0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// one-shot host-memory entry: H2D copies, plan, execute, D2H copy, all on one stream
// ---------------------------------------------------------------------------------------------
namespace ns {
struct HostCache {
    std::mutex mu;
    void* buf = nullptr;
    size_t bytes = 0;
    int device = -1;
};
static HostCache g_host_cache;
}  // namespace ns

extern "C" ns_status_t ns_spmm_host(const ns_csr_t* A, const void* B, int32_t K, ns_dtype_t b_dtype,
                                    float* C, const ns_tune_t* tune, ns_stream_t s)
{
    NS_TRY(check_csr_args(A));
    NS_TRY(check_K(K));
    if (A->on_device) {
        set_error("ns_spmm_host takes a host CSR");
        return NS_ERR_INVALID;
    }
    if ((A->n > 0 && !B) || (A->m > 0 && !C)) {
        set_error("B or C is NULL");
        return NS_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(s);
    const size_t eb = b_dtype == NS_BF16 ? 2 : 4;
    const size_t bB = ((size_t)A->n * K * eb + 255) & ~size_t(255);
    const size_t bC = (size_t)A->m * K * 4;
    std::lock_guard<std::mutex> lk(g_host_cache.mu);
    int dev = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
    if (g_host_cache.buf && (g_host_cache.bytes < bB + bC || g_host_cache.device != dev)) {
        cudaFree(g_host_cache.buf);
        g_host_cache.buf = nullptr;
        g_host_cache.bytes = 0;
    }
    if (!g_host_cache.buf) {
        NS_CUDA_TRY(cudaMalloc(&g_host_cache.buf, bB + bC + 256));
        g_host_cache.bytes = bB + bC + 256;
        g_host_cache.device = dev;
    }
    void* dB = g_host_cache.buf;
    float* dC = reinterpret_cast<float*>(static_cast<char*>(g_host_cache.buf) + bB);
    if (A->n > 0) NS_CUDA_TRY(cudaMemcpyAsync(dB, B, (size_t)A->n * K * eb, cudaMemcpyHostToDevice, st));
    ns_plan_t p = nullptr;
    NS_TRY(ns_spmm_plan(A, K, b_dtype, tune, s, &p));
    ns_status_t r = ns_spmm_execute(p, dB, K, dC, K, s);
    if (r == NS_OK && bC > 0) {
        cudaError_t e = cudaMemcpyAsync(C, dC, bC, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) {
            set_error("cudaMemcpyAsync(C) failed: %s", cudaGetErrorString(e));
            r = NS_ERR_CUDA;
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (r == NS_OK && e != cudaSuccess) {
        set_error("stream synchronize failed: %s", cudaGetErrorString(e));
        r = NS_ERR_CUDA;
    }
    ns_plan_destroy(p);
    return r;
}

extern "C" ns_status_t ns_release_cache(void)
{
    {
        std::lock_guard<std::mutex> lk(g_host_cache.mu);
        if (g_host_cache.buf) cudaFree(g_host_cache.buf);
        g_host_cache.buf = nullptr;
        g_host_cache.bytes = 0;
    }
    cudaDeviceSynchronize();
    pool_trim();
    return NS_OK;
}
