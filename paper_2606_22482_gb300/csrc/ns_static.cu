// ns_static.cu -- an SpMM entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already handed to
// another allocator (a framework's caching allocator or a fixed per-tenant HBM budget leaves
// nothing for a second allocator), or a latency-critical path that cannot pay the implicit
// device synchronisation of cudaMalloc/cudaFree.  ns_spmm_csr_static serves them: it computes
// C = A * B straight from a device CSR on the CUDA cores, with its scratch (work ticket, split-row
// counters and partial-row slots) in one file-scope __device__ array of kStaticScratchBytes that
// every GPU loading the library holds until the process exits.  The caller passes A, B and C.
//
// The first call on a device looks up the array's device address with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any stream capture.  Every
// call shares the array and it keeps the last call's contents, so each call clears the counters
// it needs first; calls that overlap on the GPU (other streams, other threads) race on it.
#include <mutex>

#include "ns_internal.cuh"

namespace ns {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int64_t kStaticW = 256;                          // merge items per warp chunk

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[64] = {nullptr};
static int g_static_grid[64] = {0};

struct StaticArgs {
    const int32_t* rowptr;
    const int32_t* colidx;
    const float* vals;
    const void* B;
    float* C;
    int64_t ldb, ldc, nnz, T, nc;
    int32_t m, n, K;
    int32_t* ctrl;    // [0] chunk ticket
    int32_t* cnt;     // nc arrival counters (one per split row, indexed by its first chunk)
    float* slots;     // 2 * nc partial rows of K floats (head piece, tail piece of each chunk)
};

__device__ __forceinline__ int64_t st_ptr(const StaticArgs& a, int64_t i)
{
    int64_t r = __ldg(a.rowptr + i);
    return r < 0 ? 0 : (r > a.nnz ? a.nnz : r);
}

template <bool BF16>
__device__ __forceinline__ float4 st_ldb(const void* B, int64_t off)
{
    if (!BF16) return __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(B) + off));
    uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint16_t*>(B) + off));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

// slot of chunk c's piece of a row whose first chunk is fc (tail slot in fc, head slot after)
__device__ __forceinline__ int64_t st_slot(int64_t c, int64_t fc) { return c == fc ? 2 * c + 1 : 2 * c; }

template <int L, int VPL, bool BF16>
__global__ void __launch_bounds__(128) k_spmm_static(StaticArgs a)
{
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31, g = lane / L, li = lane % L;
    const int nv = a.K >> 2;
    for (;;) {
        int64_t c = 0;
        if (lane == 0) c = atomicAdd(a.ctrl, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= a.nc) break;
        const int64_t b0 = c * kStaticW;
        const int64_t b1 = b0 + kStaticW < a.T ? b0 + kStaticW : a.T;
        // row holding merge item b0: largest k with rowptr[k] + k <= b0
        int64_t lo = 0, hi = a.m;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (st_ptr(a, mid) + mid <= b0) lo = mid;
            else hi = mid;
        }
        int64_t k = lo, x = b0;
        while (x < b1 && k < a.m) {
            const int64_t zr = st_ptr(a, k), ze = st_ptr(a, k + 1);
            const int64_t s = zr + k, e = (ze > zr ? ze : zr) + k + 1;
            const int64_t xe = b1 < e - 1 ? b1 : e - 1;
            float4 acc[VPL];
#pragma unroll
            for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            int64_t z0 = zr + (x - s), z1 = zr + (xe - s);
            if (z0 < zr) z0 = zr;  // only reachable with malformed row pointers: stay in the row
            if (z1 > ze) z1 = ze;
            for (int64_t zb = z0; zb < z1; zb += 32) {
                const int cntb = (int)(z1 - zb < 32 ? z1 - zb : 32);
                int32_t mc = 0;
                float mv = 0.f;
                if (lane < cntb) {
                    mc = __ldg(a.colidx + zb + lane);
                    mv = __ldg(a.vals + zb + lane);
                    if ((unsigned)mc >= (unsigned)a.n) mc = -1, mv = 0.f;  // never gather outside B
                }
                for (int j0 = 0; j0 < cntb; j0 += G) {
                    const int j = j0 + g;
                    const int32_t col = __shfl_sync(0xffffffffu, mc, j & 31);
                    float val = __shfl_sync(0xffffffffu, mv, j & 31);
                    if (j >= cntb) val = 0.f;
#pragma unroll
                    for (int q = 0; q < VPL; ++q) {
                        const int v = li + L * q;
                        if (j < cntb && col >= 0 && v < nv) {  // an invalid column gathers nothing
                            float4 b = st_ldb<BF16>(a.B, (int64_t)col * a.ldb + 4 * v);
                            acc[q].x = fmaf(val, b.x, acc[q].x);
                            acc[q].y = fmaf(val, b.y, acc[q].y);
                            acc[q].z = fmaf(val, b.z, acc[q].z);
                            acc[q].w = fmaf(val, b.w, acc[q].w);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = L; o < 32; o <<= 1)
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                    acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
                    acc[q].z += __shfl_xor_sync(0xffffffffu, acc[q].z, o);
                    acc[q].w += __shfl_xor_sync(0xffffffffu, acc[q].w, o);
                }
            // deliver: whole row, or one piece of a row cut by chunk boundaries
            const int64_t fc = s / kStaticW, lc = (e - 1) / kStaticW;
            float* crow = a.C + k * a.ldc;
            if (fc == lc) {
                if (lane < L)
#pragma unroll
                    for (int q = 0; q < VPL; ++q) {
                        const int v = lane + L * q;
                        if (v < nv) *reinterpret_cast<float4*>(crow + 4 * v) = acc[q];
                    }
            } else {
                float* my = a.slots + st_slot(c, fc) * a.K;
                if (lane < L)
#pragma unroll
                    for (int q = 0; q < VPL; ++q) {
                        const int v = lane + L * q;
                        if (v < nv) __stcg(reinterpret_cast<float4*>(my + 4 * v), acc[q]);
                    }
                __threadfence();
                __syncwarp();
                int old = 0;
                if (lane == 0) old = atomicAdd(a.cnt + fc, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                if (old == (int)(lc - fc)) {  // last of the row's lc - fc + 1 pieces
                    __threadfence();
                    if (lane < L)
#pragma unroll
                        for (int q = 0; q < VPL; ++q) {
                            const int v = lane + L * q;
                            if (v < nv) {
                                float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                                for (int64_t p = fc; p <= lc; ++p) {
                                    float4 t = __ldcg(reinterpret_cast<const float4*>(a.slots + st_slot(p, fc) * a.K + 4 * v));
                                    sum.x += t.x;
                                    sum.y += t.y;
                                    sum.z += t.z;
                                    sum.w += t.w;
                                }
                                *reinterpret_cast<float4*>(crow + 4 * v) = sum;
                            }
                        }
                }
            }
            if (e - 1 < b1) {
                x = e;
                ++k;
            } else {
                x = b1;
            }
        }
    }
}

typedef void (*StaticKernel)(StaticArgs);

template <bool BF16>
static StaticKernel static_pick(int K)
{
    const int nv = K / 4;
    if (nv <= 2) return k_spmm_static<2, 1, BF16>;
    if (nv <= 4) return k_spmm_static<4, 1, BF16>;
    if (nv <= 8) return k_spmm_static<8, 1, BF16>;
    if (nv <= 16) return k_spmm_static<16, 1, BF16>;
    if (nv <= 32) return k_spmm_static<32, 1, BF16>;
    if (nv <= 64) return k_spmm_static<32, 2, BF16>;
    if (nv <= 128) return k_spmm_static<32, 4, BF16>;
    return k_spmm_static<32, 8, BF16>;
}

// bytes of the static array one call needs
static int64_t static_need(int64_t nc, int32_t K)
{
    return 256 + ((4 * nc + 255) / 256) * 256 + 2 * nc * (int64_t)K * 4;
}

}  // namespace ns

using namespace ns;

extern "C" ns_status_t ns_spmm_csr_static(const ns_csr_t* A, const void* B, int64_t ldb, float* C,
                                          int64_t ldc, int32_t K, ns_dtype_t b_dtype, ns_stream_t s)
{
    if (!A || !A->on_device) {
        set_error("ns_spmm_csr_static takes a device CSR (on_device = 1)");
        return NS_ERR_INVALID;
    }
    if (A->m < 0 || A->n < 0 || A->nnz < 0 || (int64_t)A->m + A->nnz > 2147483647LL) {
        set_error("bad CSR shape");
        return NS_ERR_INVALID;
    }
    if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->vals)) || (A->n > 0 && !B) || (A->m > 0 && !C)) {
        set_error("NULL array");
        return NS_ERR_INVALID;
    }
    if (A->nnz > 0 && A->n == 0) {  // no column index can be valid, and B has no rows
        set_error("CSR with n = 0 columns cannot hold %lld nonzeros", (long long)A->nnz);
        return NS_ERR_INVALID;
    }
    if (K < 8 || K > 1024 || K % 8) {
        set_error("K=%d unsupported: need 8 <= K <= 1024 and K %% 8 == 0", K);
        return NS_ERR_UNSUPPORTED;
    }
    if (b_dtype != NS_F32 && b_dtype != NS_BF16) {
        set_error("unknown dtype");
        return NS_ERR_INVALID;
    }
    if ((reinterpret_cast<uintptr_t>(B) & 15u) || (reinterpret_cast<uintptr_t>(C) & 15u) || ldb < K ||
        ldc < K || (ldb % 8) || (ldc % 8)) {
        set_error("B and C must be 16-byte aligned with ldb, ldc >= K and multiples of 8");
        return NS_ERR_UNSUPPORTED;
    }
    const int64_t T = (int64_t)A->m + A->nnz;
    const int64_t nc = (T + kStaticW - 1) / kStaticW;
    const int64_t need = static_need(nc, K);
    if (need > (int64_t)kStaticScratchBytes) {
        set_error("A too large for the %zu-byte static scratch: needs %lld bytes (2 partial rows "
                  "of K floats per %lld merge items of m + nnz); use ns_spmm_plan instead",
                  kStaticScratchBytes, (long long)need, (long long)kStaticW);
        return NS_ERR_TOO_LARGE;
    }
    int dev = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return NS_ERR_UNSUPPORTED;
    }
    StaticKernel kern = b_dtype == NS_BF16 ? static_pick<true>(K) : static_pick<false>(K);
    void* base = nullptr;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            // host code cannot use the array's name as a device address: look it up once
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) {
                set_error("cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
                return NS_ERR_CUDA;
            }
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_static<32, 1, false>, 128, 0);
            if (e != cudaSuccess) {
                set_error("occupancy query failed: %s", cudaGetErrorString(e));
                return NS_ERR_CUDA;
            }
            g_static_grid[dev] = (per_sm > 0 ? per_sm : 1) * num_sms(dev);
            g_static_ptr[dev] = p;
        }
        base = g_static_ptr[dev];
        grid = g_static_grid[dev];
    }
    if (T == 0) return NS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(s);
    StaticArgs a;
    a.rowptr = A->rowptr;
    a.colidx = A->colidx;
    a.vals = A->vals;
    a.B = B;
    a.C = C;
    a.ldb = ldb;
    a.ldc = ldc;
    a.nnz = A->nnz;
    a.T = T;
    a.nc = nc;
    a.m = A->m;
    a.n = A->n;
    a.K = K;
    unsigned char* bp = static_cast<unsigned char*>(base);
    a.ctrl = reinterpret_cast<int32_t*>(bp);
    a.cnt = reinterpret_cast<int32_t*>(bp + 256);
    a.slots = reinterpret_cast<float*>(bp + 256 + ((4 * nc + 255) / 256) * 256);
    // the ticket and the arrival counters must start at zero; the slots are written before read
    NS_CUDA_TRY(cudaMemsetAsync(bp, 0, (size_t)(256 + 4 * nc), st));
    const int64_t warps = nc < (int64_t)grid * 4 ? nc : (int64_t)grid * 4;
    kern<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(a);
    NS_LAUNCH_CHECK();
    return NS_OK;
}
