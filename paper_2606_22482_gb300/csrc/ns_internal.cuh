// ns_internal.cuh -- shared internals of libns_spmm (plan object, errors, device utilities).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "ns_spmm.h"

namespace ns {

// ---------------------------------------------------------------------------------------------
// errors and bookkeeping
// ---------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

#define NS_CUDA_TRY(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ::ns::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                            __LINE__);                                                         \
            return (e_ == cudaErrorMemoryAllocation) ? NS_ERR_OOM : NS_ERR_CUDA;               \
        }                                                                                      \
    } while (0)

#define NS_TRY(expr)                                                                           \
    do {                                                                                       \
        ns_status_t s_ = (expr);                                                               \
        if (s_ != NS_OK) return s_;                                                            \
    } while (0)

// after a kernel launch: report launch-configuration errors
#define NS_LAUNCH_CHECK()                                                                      \
    do {                                                                                       \
        ::ns::count_launch();                                                                  \
        NS_CUDA_TRY(cudaGetLastError());                                                       \
    } while (0)

constexpr int32_t kTauInf = NS_TAU_INF;
constexpr int kReorderMaxRows = 1024;  // rows of one local-reordering cluster (Section 6.1)
constexpr int kExecWarps = 4;            // warps per execute CTA (== residual chunks per item)
constexpr int kExecThreads = kExecWarps * 32;

// device status word bits (written by kernels, read by the host on the next call)
enum : int32_t {
    kStatusOk = 0,
    kStatusInvalidCsr = 1,
    kStatusTimeout = 2,
    kStatusInternal = 4,
};

// ---------------------------------------------------------------------------------------------
// stream-ordered device allocations from the library's own memory pool
// ---------------------------------------------------------------------------------------------
// The pool keeps freed blocks mapped (release threshold = max) so that planning again does not
// re-map physical memory at every synchronisation; ns_release_cache trims it.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_trim();
struct DevBlock {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// A bump allocator: reserve() sizes first, then commit() makes one allocation.
struct Arena {
    struct Req {
        void** slot;
        size_t bytes;
    };
    std::vector<Req> reqs;
    DevBlock block;
    cudaStream_t stream = nullptr;
    template <class T>
    void reserve(T** slot, int64_t count)
    {
        reqs.push_back({reinterpret_cast<void**>(slot), (size_t)(count > 0 ? count : 1) * sizeof(T)});
    }
    void reserve_bytes(void** slot, size_t bytes) { reqs.push_back({slot, bytes > 0 ? bytes : 1}); }
    ns_status_t commit(cudaStream_t s);   // one cudaMallocAsync for every reserved array
    DevBlock take()                         // hand the block to a new owner
    {
        DevBlock b = block;
        block = DevBlock{};
        reqs.clear();
        return b;
    }
    void release(cudaStream_t s);           // free the block (stream-ordered)
    ~Arena() { release(nullptr); }
};

// ---------------------------------------------------------------------------------------------
// the device-side description of one plan's execution (read by the persistent kernel)
// ---------------------------------------------------------------------------------------------
// Execution-side summary of one merge-path chunk (derived from the plan's chunk boundaries, not
// part of the canonical plan): merge range [b0, b1), residual-list rows k0 .. kL with an item in
// the range, the residual index of the chunk's first nonzero (the whole chunk's nonzeros are
// z0 .. z0 + total - 1 when the residual list is every row in order) and its nonzero count.
struct alignas(32) ChunkRec {
    int32_t b0, b1, k0, kL, z0, total, pad0, pad1;
};

struct ExecDesc {
    // residual CSR and its chunks
    const int32_t* res_rowptr;
    const int32_t* res_col;
    const float* res_val;
    const int32_t* rl_rows;
    const int32_t* rl_start;
    const int32_t* chunk_b;
    const int32_t* chunk_k0;
    const ChunkRec* chunk_rec;
    int32_t n_chunks;
    int32_t n_dwin;
    // dense windows and tiles
    const int32_t* win_rows;
    const int32_t* win_dptr;
    const int32_t* dwin;
    const int32_t* dwin_absorb;
    const int32_t* dtile_cols;
    const uint32_t* dtile_bits;
    const int32_t* dtile_voff;
    const void* dtile_vals;
    const uint16_t* dtile_x;  // BF16 plans: every dense tile expanded, in the tensor-core layout
    // split rows
    const int32_t* row_split;
    const int32_t* split_np;
    const int32_t* split_slot;
    const int32_t* split_base;
    float* slots;        // n_slots * K floats
    int32_t* split_cnt;  // n_split arrival counters (zero between launches)
    // operands
    const void* B;
    float* C;
    int64_t ldb, ldc;
    int32_t K, b_bf16, TM, TK, group, l2_hints;
    int32_t m, n;          // shape of A (bounds guards)
    int32_t n_rl, n_res;   // residual list rows, residual nonzeros (bounds guards)
    int32_t rl_all;        // 1: the residual list is every row in order (contiguous stream)
    const uint32_t* hot;   // bit j set: B row j is among the most gathered (evict-last); null: all
    int32_t chunk_nnz;     // W of the plan (sizes the staged chunk buffers)
    int32_t* status;       // device status word (kStatus* bits)
    // per-class progress clock (Section 5.3 epoch monitoring), null when off: [0] earliest CTA
    // start, [1] latest end of a dense item, [2] latest end of a residual chunk (globaltimer ns)
    unsigned long long* class_clock;
};

// ---------------------------------------------------------------------------------------------
// the plan object
// ---------------------------------------------------------------------------------------------
struct Plan {
    ns_plan_stats_t st{};
    ns_tune_t tune{};
    ns_dtype_t dtype = NS_F32;
    int32_t K = 0;
    int device = 0;

    // input copy (host CSR) or alias (device CSR)
    const int32_t* rowptr = nullptr;
    const int32_t* colidx = nullptr;
    const float* vals = nullptr;

    // plan arrays (device)
    int32_t* aic_rows = nullptr;
    int32_t* win_rows = nullptr;
    int32_t* win_dptr = nullptr;
    int32_t* dwin = nullptr;
    int32_t* dwin_absorb = nullptr;
    int32_t* dtile_cols = nullptr;
    uint32_t* dtile_bits = nullptr;
    int32_t* dtile_voff = nullptr;
    void* dtile_vals = nullptr;
    uint16_t* dtile_x = nullptr;  // BF16 plans: dense tiles expanded (execution format, see k_emit_tiles)
    const int32_t* res_rowptr = nullptr;  // aliases rowptr when nothing is dense
    const int32_t* res_col = nullptr;
    const float* res_val = nullptr;
    int32_t* res_rowptr_own = nullptr;
    int32_t* res_col_own = nullptr;
    float* res_val_own = nullptr;
    int32_t* rl_rows = nullptr;
    int32_t* rl_start = nullptr;
    int32_t* chunk_b = nullptr;
    int32_t* chunk_k0 = nullptr;
    ChunkRec* chunk_rec = nullptr;  // per chunk, for the execute kernel
    int32_t* row_split = nullptr;
    int32_t* split_row = nullptr;
    int32_t* split_np = nullptr;
    int32_t* split_slot = nullptr;
    int32_t* split_base = nullptr;
    int32_t* queue = nullptr;
    int64_t* item_cost = nullptr;
    uint32_t* hot_bits = nullptr;    // execution hint (l2_hints == 2): hot B rows, n bits
    // execution scratch
    float* slots = nullptr;
    int32_t* split_cnt = nullptr;
    int32_t* ctrl = nullptr;       // [0] ticket, [1] CTAs done, [2] status, [3..] scalars
    unsigned long long* class_clock = nullptr;  // set while the rebalance loop times the launch
    ExecDesc desc_host{};           // the single-plan descriptor (a kernel parameter)
    bool desc_valid = false;
    std::vector<DevBlock> blocks;  // every device allocation the plan owns
    int exec_grid = 0;
    int exec_grid_slice = 0, exec_grid_slice_K = 0;  // grid of the column-slice launches
    cudaStream_t last_stream = nullptr;  // stream of the last plan/execute call: frees go there
    int32_t* status_host = nullptr;      // pinned copy of the device status word after a launch
    cudaEvent_t status_ev = nullptr;     // completes when that copy has landed
    ~Plan();
};

// Result of the window pass (a2-a7) that later planner stages need.
struct WindowResult {
    int8_t* row_state = nullptr;  // per row: 0 free, 1 dense window (absorbing), 2 dense window
    int64_t* dcost = nullptr;     // per dense window: Eq. 1 cost
    DevBlock temp;                // temporaries freed after planning
};
ns_status_t window_pass(Plan* P, WindowResult* W, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int num_sms(int device);
int64_t l2_bytes(int device);

// residual-only launch modes of exec_launch / exec_prepare (`contig`)
constexpr int kContig = 1;       // contiguous residual stream
constexpr int kContigBInL2 = 2;  // the same, with B small enough to stay in L2
constexpr int kContigHot = 3;    // kContig, single plan with a hot-row map (l2_hints = 2)

// planner entry (ns_plan.cu)
ns_status_t plan_build(Plan* P, const ns_csr_t* A, int32_t K, ns_dtype_t dt, const ns_tune_t* tune,
                       cudaStream_t s);
ns_status_t plan_check_tune(const ns_tune_t& t);

// execute entry (ns_exec.cu)
void fill_desc(const Plan* P, const void* B, int64_t ldb, float* C, int64_t ldc, ExecDesc* d);
ns_status_t exec_launch(const ExecDesc* descs, const int32_t* queue, const int32_t* queue_desc,
                        int64_t n_items, int32_t* ctrl, int K, int TM, int TK, bool bf16, bool hint,
                        bool dense, int* grid_cache, cudaStream_t s, const ExecDesc* d0 = nullptr,
                        int W = 256, int contig = 0);
ns_status_t exec_launch_plan(Plan* P, cudaStream_t s);
ns_status_t exec_prepare(int64_t n_items, int K, int TM, int TK, bool bf16, bool hint, bool dense,
                         int* grid_out, int W = 256, int contig = 0);
bool plan_contig(const Plan* P);  // contiguous residual stream (tau_tile = inf)
ns_status_t plan_create(const ns_csr_t* A, int32_t K, ns_dtype_t dt, const ns_tune_t* tune,
                        cudaStream_t s, Plan** out);  // checks + build; on error nothing is kept

}  // namespace ns
