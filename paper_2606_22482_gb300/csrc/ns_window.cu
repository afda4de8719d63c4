// ns_window.cu -- the window pass of the device planner (arXiv 2606.22482 Sections 5.2.2, 6.1).
//
//   W1  row extraction (Eq. 4-5, integer threshold): rows with Len > tau_row are kept
//   W2  column extraction inside the kept rows: columns with count <= tau_col leave
//   W3  windows = TM consecutive kept rows; window element ranges by a scan of kept lengths
//   W4  gather every window's kept columns (rows' sorted segments, concatenated)
//   W5  per window (one CTA): merge the sorted row segments, run-length encode to the unique
//       columns with counts (column compaction, Section 6.1), order them canonically (count
//       descending then column, or column ascending), cut TK-wide tiles, bin them by density
//       (nnz >= tau_tile), map every element to its compacted position, count dense elements
//       per row
//   W6  scans: dense tiles / values per window, residual row pointers, dense windows
//   W7  dense windows: absorb decision, Eq. 1 cost, row ownership
//   W8  residual row list with merge starts
//   W9  emit dense tiles (columns, bitmap, packed values in bitmap order, BF16 RNE if asked)
//   W10 residual CSR: every element outside a dense tile, original rows and column order
// All of it is integer work with fixed orders, matching the CPU reference partition exactly.
#include "ns_internal.cuh"
#include "ns_scan.cuh"

#include <cuda_bf16.h>

namespace ns {

constexpr int kWinThreads = 512;
constexpr int kWinSmemKeys = 4096;  // windows up to this many elements sort in shared memory
constexpr int kMaxTM = 64;
// Windows with more elements than kWinSmemKeys, of a matrix with at most kDenseCols columns, count
// their columns in a per-CTA array instead of sorting: byte counters (TM <= 64 < 256) packed four
// to a word, then a presence bit per column and an ascending index per 32 columns (1.25 bytes a
// column in all).
constexpr int kDenseCols = 49152;
// counting path's shared memory: a byte counter per column (4 a word), a presence bit per column
// and an index per 32 columns
// and, for windows of up to kCanonSmem distinct columns, each column's canonical position (16 bits)
constexpr int kCanonSmem = 16384;
constexpr size_t count_table_bytes(int64_t n)
{
    return (size_t)4 * ((n + 3) / 4) + (size_t)8 * ((n + 31) / 32) + (size_t)2 * kCanonSmem;
}
// emission assembles a window's dense-tile bitmaps (4 bytes a word), their per-tile prefix counts
// (2 bytes a word) and its tiles' dense ranks (2 bytes a tile) in dynamic shared memory sized
// from the plan's largest window, up to this limit (larger windows use global memory)
constexpr int kEmitSmemMax = 192 * 1024;

// ---------------------------------------------------------------------------------------------
// W1: kept rows
// ---------------------------------------------------------------------------------------------
struct KeepLoad {
    const int32_t* rowptr;
    int32_t tau_row;
    __device__ __forceinline__ int64_t operator()(int64_t i) const
    {
        return (__ldg(rowptr + i + 1) - __ldg(rowptr + i)) > tau_row ? 1 : 0;
    }
};
struct KeepStore {
    int32_t* aic_rows;
    __device__ __forceinline__ void operator()(int64_t i, int64_t pre, int64_t v) const
    {
        if (v) aic_rows[pre] = (int32_t)i;
    }
};

// W2: column counts over kept rows (warp per kept row)
__global__ void k_colcount(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                           const int32_t* __restrict__ aic_rows, int64_t m_aic, int32_t* colcount)
{
    const int lane = threadIdx.x & 31;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m_aic;
         k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t i = __ldg(aic_rows + k);
        for (int64_t p = __ldg(rowptr + i) + lane; p < __ldg(rowptr + i + 1); p += 32)
            atomicAdd(colcount + __ldg(colidx + p), 1);
    }
}

// W3: kept length of kept row k (all of it when no column extraction)
struct KeptLenLoad {
    const int32_t* rowptr;
    const int32_t* colidx;
    const int32_t* aic_rows;
    const int32_t* colcount;  // nullptr: keep every column
    int32_t tau_col;
    __device__ __forceinline__ int64_t operator()(int64_t k) const
    {
        int32_t i = __ldg(aic_rows + k);
        int64_t b = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
        if (!colcount) return e - b;
        int64_t c = 0;
        for (int64_t p = b; p < e; ++p) c += __ldg(colcount + __ldg(colidx + p)) > tau_col;
        return c;
    }
};
struct KeptLenStore {
    int64_t* row_kbase;
    __device__ __forceinline__ void operator()(int64_t k, int64_t pre, int64_t) const { row_kbase[k] = pre; }
};

// W4: gather kept columns and their original indices (warp per kept row)
__global__ void k_gather_window_elems(const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ colidx,
                                      const int32_t* __restrict__ aic_rows, int64_t m_aic,
                                      const int64_t* __restrict__ row_kbase,
                                      const int32_t* __restrict__ colcount, int32_t tau_col,
                                      int32_t* ekey, int32_t* eidx)
{
    const int lane = threadIdx.x & 31;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m_aic;
         k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int32_t i = __ldg(aic_rows + k);
        int64_t b = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
        int64_t out = row_kbase[k];
        for (int64_t p0 = b; p0 < e; p0 += 128) {  // four batches of 32 loads in flight
            int32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                c[u] = p < e ? __ldg(colidx + p) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                const bool keep = p < e && (!colcount || __ldg(colcount + c[u]) > tau_col);
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int64_t o = out + __popc(bal & ((1u << lane) - 1u));
                    ekey[o] = c[u];
                    eidx[o] = (int32_t)p;
                }
                out += __popc(bal);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// W5: per-window compaction (one CTA per window)
// ---------------------------------------------------------------------------------------------
// stable merge path: elements taken from A among the first d outputs (ties go to A)
__device__ __forceinline__ int64_t merge_corank(const int32_t* A, int64_t na, const int32_t* B,
                                                int64_t nb, int64_t d)
{
    int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        int64_t i = (lo + hi) >> 1;
        if (A[i] <= B[d - i - 1]) lo = i + 1;
        else hi = i;
    }
    return lo;
}

// sort N keys made of R sorted runs (boundaries rb[0..R]) by pairwise merge rounds.
// Returns the buffer holding the result (in or tmp).  rb is modified (shared memory).
__device__ int32_t* cta_merge_runs(int32_t* in, int32_t* tmp, int64_t N, int64_t* rb, int R)
{
    int32_t* src = in;
    int32_t* dst = tmp;
    const int nt = blockDim.x;
    while (R > 1) {
        const int64_t S = (N + nt - 1) / nt;
        int64_t o0 = (int64_t)threadIdx.x * S;
        const int64_t o1 = o0 + S < N ? o0 + S : N;
        while (o0 < o1) {
            // pair j containing o0: largest j with rb[2j] <= o0
            int j = 0;
            for (int q = 0; 2 * q < R; ++q)
                if (rb[2 * q] <= o0) j = q;
            const int64_t ps = rb[2 * j];
            const int64_t mid = rb[2 * j + 1 < R ? 2 * j + 1 : R];
            const int64_t pe = rb[2 * j + 2 < R ? 2 * j + 2 : R];
            const int64_t seg_end = o1 < pe ? o1 : pe;
            const int32_t* A = src + ps;
            const int32_t* B = src + mid;
            const int64_t na = mid - ps, nb = pe - mid;
            int64_t d = o0 - ps;
            int64_t ia = merge_corank(A, na, B, nb, d);
            int64_t ib = d - ia;
            for (int64_t o = o0; o < seg_end; ++o) {
                bool take_a = ib >= nb || (ia < na && A[ia] <= B[ib]);
                dst[o] = take_a ? A[ia++] : B[ib++];
            }
            o0 = seg_end;
        }
        __syncthreads();
        // next round's runs: every other boundary
        int64_t nrb[kMaxTM / 2 + 2];
        int nR = (R + 1) / 2;
        if (threadIdx.x == 0) {
            for (int q = 0; q < nR; ++q) nrb[q] = rb[2 * q];
            nrb[nR] = rb[R];
            for (int q = 0; q <= nR; ++q) rb[q] = nrb[q];
        }
        __syncthreads();
        R = nR;
        int32_t* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

struct WinArgs {
    // inputs
    const int32_t* rowptr;
    const int32_t* aic_rows;
    const int64_t* row_kbase;  // m_aic + 1
    const int32_t* ekey;
    int64_t m_aic;
    int32_t TM, TK, tau_tile, col_order;
    // temporaries in window-element space (offset wbase)
    int32_t* sortbuf0;
    int32_t* sortbuf1;
    int32_t* uasc;
    int32_t* ucnt;  // counts of uasc entries
    int32_t* upos;  // canonical position of uasc entries
    int32_t* ucan;  // column at canonical position
    int32_t* ccnt;  // count at canonical position
    int32_t* trank; // dense rank of tile t (or -1)
    int32_t* tvoff; // value offset of dense tile t inside the window
    int32_t* epos;  // canonical position of each element
    // per-window outputs
    int32_t* win_U;
    int32_t* win_ndt;
    int32_t* win_ndv;
    int64_t* win_res;   // residual nonzeros of the window's rows
    int32_t* res_len;   // per row (m)
    int32_t n;          // columns of A
    int32_t count_cols; // 1: launched with count_table_bytes(n) bytes of dynamic shared memory (n <= kDenseCols)
};

// row slot of window element e: the largest r < nrows with rb[r] <= e (empty rows share their
// start with the next row, so the largest such r is the row that holds e)
__device__ __forceinline__ int row_slot_of(const int64_t* rb, int nrows, int64_t e)
{
    int lo = 0, hi = nrows;  // answer in [lo, hi)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (rb[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kWinThreads) k_window_compact(WinArgs a)
{
    __shared__ int64_t rb[kMaxTM + 1];   // run boundaries (relative to wbase)
    __shared__ int64_t rb0[kMaxTM + 1];  // original row boundaries
    __shared__ int64_t sscan[kWinThreads / 32 + 1];
    __shared__ int32_t wc[kWinThreads / 32][kMaxTM + 1];
    __shared__ int32_t binoff[kMaxTM + 1];
    __shared__ int32_t dcnt[kMaxTM];
    __shared__ int64_t s_carry[2];
    __shared__ uint32_t tdense[kDenseCols / 16 / 32 + 1];  // counting path: dense flag per tile (TK >= 16)

    const int w = blockIdx.x;
    const int TM = a.TM, TK = a.TK;
    const int64_t r0 = (int64_t)w * TM;
    const int nrows = (int)(a.m_aic - r0 < TM ? a.m_aic - r0 : TM);
    const int64_t wbase = a.row_kbase[r0];
    const int64_t N = a.row_kbase[r0 + nrows] - wbase;
    for (int q = threadIdx.x; q <= nrows; q += blockDim.x) {
        rb[q] = a.row_kbase[r0 + q] - wbase;
        rb0[q] = rb[q];
    }
    for (int q = threadIdx.x; q < TM; q += blockDim.x) dcnt[q] = 0;
    __syncthreads();

    int32_t* uasc = a.uasc + wbase;
    int32_t* ucnt = a.ucnt + wbase;
    int32_t* upos = a.upos + wbase;
    // ---- unique columns of the window in ascending order, with their counts ----
    // Dynamic shared memory: the column counters and positions of the counting path, or (the
    // other path) the two key buffers of an in-shared-memory sort; a CTA takes one of the two.
    extern __shared__ uint32_t dyn_cols[];
    const bool count_cols = a.count_cols && N > kWinSmemKeys;  // window-uniform
    const int nwords = (a.n + 3) >> 2;
    // after the counters: a presence bit per column and, per 32 columns, the ascending index of
    // the first present one; a column's ascending index is then one lookup and a popcount
    const int ngroups = (a.n + 31) >> 5;
    uint32_t* const cbits = dyn_cols + nwords;
    int32_t* const gpre = reinterpret_cast<int32_t*>(cbits + ngroups);
    uint16_t* const scan = reinterpret_cast<uint16_t*>(gpre + ngroups);  // canonical position by ascending index
    if (count_cols) {
        // byte counters, four per word (a count is at most TM <= 64)
        for (int q = threadIdx.x; q < nwords; q += blockDim.x) dyn_cols[q] = 0u;
        __syncthreads();
        for (int64_t e0 = threadIdx.x; e0 < N; e0 += 8 * blockDim.x) {
            int32_t cv[8];  // eight column ids per thread in flight
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t e = e0 + (int64_t)u * blockDim.x;
                cv[u] = e < N ? a.ekey[wbase + e] : -1;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (cv[u] >= 0) atomicAdd(&dyn_cols[cv[u] >> 2], 1u << (8 * (cv[u] & 3)));
        }
        if (threadIdx.x == 0) s_carry[0] = 0;
        __syncthreads();
        // compaction in ascending column order: warp w owns a segment of the words, counts its
        // columns, the segments' counts are scanned once, and each warp then emits its segment
        // 32 words at a time with a warp scan (no block barrier per step)
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            const int seg = (((nwords + nw - 1) / nw) + 31) & ~31;
            const int wlo = warp * seg, whi = wlo + seg < nwords ? wlo + seg : nwords;
            auto present = [](uint32_t wv) {
                return (int)((wv & 0xffu) != 0) + (int)((wv & 0xff00u) != 0) + (int)((wv & 0xff0000u) != 0) +
                       (int)((wv & 0xff000000u) != 0);
            };
            int cnt = 0;
            for (int q = wlo + lane; q < whi; q += 32) cnt += present(dyn_cols[q]);
            cnt = warp_sum(cnt);
            if (lane == 0) sscan[warp] = cnt;
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t acc = 0;
                for (int q = 0; q < nw; ++q) {
                    const int64_t c = sscan[q];
                    sscan[q] = acc;
                    acc += c;
                }
                s_carry[0] = acc;
            }
            __syncthreads();
            int64_t base = sscan[warp];
            for (int q0 = wlo; q0 < whi; q0 += 32) {
                const int q = q0 + lane;
                const uint32_t wv = q < whi ? dyn_cols[q] : 0u;
                const int f = present(wv);
                const int inc = warp_incl_scan(f);
                int64_t pre = base + inc - f;
                // presence bits of the 32 columns of 8 consecutive words (q0 is a multiple of 32)
                uint32_t bw = ((uint32_t)((wv & 0xffu) != 0) | ((uint32_t)((wv & 0xff00u) != 0) << 1) |
                               ((uint32_t)((wv & 0xff0000u) != 0) << 2) | ((uint32_t)((wv & 0xff000000u) != 0) << 3))
                              << (4 * (lane & 7));
                bw |= __shfl_xor_sync(0xffffffffu, bw, 1);
                bw |= __shfl_xor_sync(0xffffffffu, bw, 2);
                bw |= __shfl_xor_sync(0xffffffffu, bw, 4);
                if ((lane & 7) == 0 && q < whi) {
                    cbits[q >> 3] = bw;
                    gpre[q >> 3] = (int32_t)pre;
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t c = (wv >> (8 * b)) & 0xffu;
                    if (c) {
                        uasc[pre] = 4 * q + b;
                        ucnt[pre] = (int32_t)c;
                        ++pre;
                    }
                }
                base += __shfl_sync(0xffffffffu, inc, 31);
            }
            __syncthreads();
        }
    } else {
        // sort the window's columns (merge of sorted row segments), then run-length encode;
        // start positions go to upos (temporary)
        const bool in_smem = N <= kWinSmemKeys;
        int32_t* const skeys = reinterpret_cast<int32_t*>(dyn_cols);
        int32_t* b0 = in_smem ? skeys : a.sortbuf0 + wbase;
        int32_t* b1 = in_smem ? skeys + kWinSmemKeys : a.sortbuf1 + wbase;
        for (int64_t e = threadIdx.x; e < N; e += blockDim.x) b0[e] = a.ekey[wbase + e];
        __syncthreads();
        const int32_t* sorted = cta_merge_runs(b0, b1, N, rb, nrows);
        if (threadIdx.x == 0) s_carry[0] = 0;
        __syncthreads();
        for (int64_t c0 = 0; c0 < N; c0 += blockDim.x) {
            int64_t e = c0 + threadIdx.x;
            int64_t f = (e < N && (e == 0 || sorted[e] != sorted[e - 1])) ? 1 : 0;
            int64_t tot;
            int64_t pre = block_excl_scan<int64_t, kWinThreads>(f, &tot, sscan) + s_carry[0];
            if (f) {
                uasc[pre] = sorted[e];
                upos[pre] = (int32_t)e;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_carry[0] += tot;
            __syncthreads();
        }
    }
    const int64_t U = s_carry[0];
    if (!count_cols) {
        for (int64_t u = threadIdx.x; u < U; u += blockDim.x) {
            int64_t nxt = u + 1 < U ? upos[u + 1] : N;
            ucnt[u] = (int32_t)(nxt - upos[u]);
        }
    }
    __syncthreads();

    // ---- canonical order ----
    int32_t* ucan = a.ucan + wbase;
    int32_t* ccnt = a.ccnt + wbase;
    if (a.col_order == 1) {
        for (int64_t u = threadIdx.x; u < U; u += blockDim.x) {
            upos[u] = (int32_t)u;
            if (count_cols && U <= kCanonSmem) scan[u] = (uint16_t)u;
            ucan[u] = uasc[u];
            ccnt[u] = ucnt[u];
        }
    } else {
        // stable counting sort by count, descending (counts are 1..TM)
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (threadIdx.x <= TM) binoff[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t u = threadIdx.x; u < U; u += blockDim.x) atomicAdd(&binoff[ucnt[u]], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t acc = 0;
            for (int c = TM; c >= 0; --c) {
                int32_t h = binoff[c];
                binoff[c] = acc;
                acc += h;
            }
        }
        __syncthreads();
        for (int64_t c0 = 0; c0 < U; c0 += blockDim.x) {
            for (int q = threadIdx.x; q < (kWinThreads / 32) * (kMaxTM + 1); q += blockDim.x)
                (&wc[0][0])[q] = 0;
            __syncthreads();
            int64_t u = c0 + threadIdx.x;
            int c = u < U ? ucnt[u] : -1;
            unsigned peers = __match_any_sync(0xffffffffu, c);
            int rk = __popc(peers & ((1u << lane) - 1u));
            if (c >= 0 && rk == 0) wc[warp][c] = __popc(peers);
            __syncthreads();
            if (c >= 0) {
                int before = 0;
                for (int q = 0; q < warp; ++q) before += wc[q][c];
                int32_t dest = binoff[c] + before + rk;
                upos[u] = dest;
                if (count_cols && U <= kCanonSmem) scan[u] = (uint16_t)dest;
                ucan[dest] = uasc[u];
                ccnt[dest] = c;
            }
            __syncthreads();
            if (threadIdx.x <= TM) {
                int add = 0;
                for (int q = 0; q < kWinThreads / 32; ++q) add += wc[q][threadIdx.x];
                binoff[threadIdx.x] += add;
            }
            __syncthreads();
        }
    }
    __syncthreads();

    // counting path: the column table now maps a column to its canonical position
    if (count_cols) {
        for (int q = threadIdx.x; q < kDenseCols / 16 / 32 + 1; q += blockDim.x) tdense[q] = 0u;
        __syncthreads();
    }

    // ---- tiles: nnz, density, dense rank and value offset inside the window ----
    const int64_t ntile = (U + TK - 1) / TK;
    int32_t* trank = a.trank + wbase;
    int32_t* tvoff = a.tvoff + wbase;
    if (threadIdx.x == 0) s_carry[0] = s_carry[1] = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < ntile; c0 += blockDim.x) {
        int64_t t = c0 + threadIdx.x;
        int64_t v = 0;
        int32_t tn = 0;
        if (t < ntile) {
            for (int64_t p = t * TK; p < (t + 1) * TK && p < U; ++p) tn += ccnt[p];
            if (tn >= a.tau_tile) v = ((int64_t)1 << 32) | (int64_t)(((tn + 7) / 8) * 8);
        }
        int64_t tot;
        int64_t pre = block_excl_scan<int64_t, kWinThreads>(v, &tot, sscan);
        if (t < ntile) {
            trank[t] = v ? (int32_t)(s_carry[0] + (pre >> 32)) : -1;
            tvoff[t] = (int32_t)(s_carry[1] + (pre & 0xffffffffLL));
            if (count_cols && v) atomicOr(&tdense[t >> 5], 1u << (t & 31));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry[0] += tot >> 32;
            s_carry[1] += tot & 0xffffffffLL;
        }
        __syncthreads();
    }

    // ---- elements: compacted position, dense counts per row ----
    int32_t* epos = a.epos + wbase;
    if (count_cols) {
        // table lookups only, one warp per row: the row's dense elements counted by ballots
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int r = warp; r < nrows; r += nwarps) {
            int cnt = 0;
            const int64_t rend = rb0[r + 1];
            for (int64_t eb = rb0[r]; eb < rend; eb += 128) {  // four column ids per lane in flight
                int32_t cv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t e = eb + 32 * u + lane;
                    cv[u] = e < rend ? a.ekey[wbase + e] : -1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    bool dense = false;
                    if (cv[u] >= 0) {
                        const int32_t c = cv[u];
                        const int32_t ai = gpre[c >> 5] + __popc(cbits[c >> 5] & ((1u << (c & 31)) - 1u));
                        const int32_t pos = U <= kCanonSmem ? (int32_t)scan[ai] : upos[ai];
                        epos[eb + 32 * u + lane] = pos;
                        const int t = pos >> (TK == 32 ? 5 : 4);  // TK is 16 or 32
                        dense = (tdense[t >> 5] >> (t & 31)) & 1u;
                    }
                    cnt += __popc(__ballot_sync(0xffffffffu, dense));
                }
            }
            if (lane == 0) dcnt[r] += cnt;
        }
    }
    for (int64_t e = count_cols ? N : threadIdx.x; e < N; e += blockDim.x) {
        const int32_t col = a.ekey[wbase + e];
        int64_t lo = 0, hi = U;  // ascending index of col: the counters' table, or a lower bound in uasc
        if (count_cols) {
            lo = gpre[col >> 5] + __popc(cbits[col >> 5] & ((1u << (col & 31)) - 1u));
        } else {
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (uasc[mid] < col) lo = mid + 1;
                else hi = mid;
            }
        }
        const int32_t pos = upos[lo];
        epos[e] = pos;
        // dense elements per row: one shared atomic per distinct row of the warp's 32 elements
        const int slot = trank[pos >> (TK == 32 ? 5 : 4)] >= 0 ? row_slot_of(rb0, nrows, e) : -1;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, slot);
        if (slot >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&dcnt[slot], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.win_U[w] = (int32_t)U;
        a.win_ndt[w] = (int32_t)s_carry[0];
        a.win_ndv[w] = (int32_t)s_carry[1];
    }
    if (threadIdx.x < 32) {
        int64_t rs = 0;
        for (int r = threadIdx.x; r < nrows; r += 32) {
            int32_t i = __ldg(a.aic_rows + r0 + r);
            int32_t len = __ldg(a.rowptr + i + 1) - __ldg(a.rowptr + i);
            int32_t rl = len - dcnt[r];
            a.res_len[i] = rl;
            rs += rl;
        }
        rs = warp_sum(rs);
        if (threadIdx.x == 0) a.win_res[w] = rs;
    }
}

// non-kept rows: the whole row is residual
__global__ void k_res_len_free_rows(const int32_t* __restrict__ rowptr, int64_t m, int32_t tau_row,
                                    int32_t* res_len)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t len = __ldg(rowptr + i + 1) - __ldg(rowptr + i);
        if (len <= tau_row) res_len[i] = len;
    }
}

// ---------------------------------------------------------------------------------------------
// W6/W7: scans over windows and rows, dense windows and ownership
// ---------------------------------------------------------------------------------------------
struct I32Load {
    const int32_t* p;
    __device__ __forceinline__ int64_t operator()(int64_t i) const { return p[i]; }
};
struct PtrStore32 {  // out[i] = prefix (int32)
    int32_t* out;
    __device__ __forceinline__ void operator()(int64_t i, int64_t pre, int64_t) const { out[i] = (int32_t)pre; }
};
struct PtrStore64 {
    int64_t* out;
    __device__ __forceinline__ void operator()(int64_t i, int64_t pre, int64_t) const { out[i] = pre; }
};
struct DenseWinLoad {
    const int32_t* win_ndt;
    __device__ __forceinline__ int64_t operator()(int64_t w) const { return win_ndt[w] > 0 ? 1 : 0; }
};
struct DenseWinStore {
    int32_t* dwin;
    __device__ __forceinline__ void operator()(int64_t w, int64_t pre, int64_t v) const
    {
        if (v) dwin[pre] = (int32_t)w;
    }
};

__global__ void k_dense_windows(const int32_t* __restrict__ dwin, int64_t n_dwin,
                                const int32_t* __restrict__ win_ndt,
                                const int64_t* __restrict__ win_res,
                                const int32_t* __restrict__ aic_rows, int64_t m_aic, int32_t TM,
                                int32_t TK, int32_t absorb_cap, int64_t cost_tc, int64_t cost_res,
                                int32_t* dwin_absorb, int64_t* dcost, int8_t* row_state)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_dwin;
         d += (int64_t)gridDim.x * blockDim.x) {
        int32_t w = dwin[d];
        int64_t r0 = (int64_t)w * TM;
        int64_t nvalid = m_aic - r0 < TM ? m_aic - r0 : TM;
        int64_t res = win_res[w];
        int absorb = res <= absorb_cap;
        dwin_absorb[d] = absorb;
        dcost[d] = (int64_t)win_ndt[w] * TM * TK * cost_tc + ((absorb ? res : 0) + nvalid) * cost_res;
        for (int64_t r = 0; r < nvalid; ++r) row_state[aic_rows[r0 + r]] = absorb ? 1 : 2;
    }
}

// W8: residual list rows: free rows, and rows of non-absorbing dense windows with residual
struct RlLoad {
    const int8_t* row_state;
    const int32_t* res_len;
    __device__ __forceinline__ int64_t operator()(int64_t i) const
    {
        int8_t st = row_state[i];
        int32_t rl = res_len[i];
        bool in = st == 0 || (st == 2 && rl > 0);
        return in ? (((int64_t)1 << 32) | (int64_t)(rl + 1)) : 0;
    }
};
struct RlStore {
    int32_t* rl_rows;
    int32_t* rl_start;
    __device__ __forceinline__ void operator()(int64_t i, int64_t pre, int64_t v) const
    {
        if (!v) return;
        int64_t k = pre >> 32;
        rl_rows[k] = (int32_t)i;
        rl_start[k] = (int32_t)(pre & 0xffffffffLL);
    }
};

// ---------------------------------------------------------------------------------------------
// W9: emit dense tiles (one CTA per window)
// ---------------------------------------------------------------------------------------------
struct EmitArgs {
    const int64_t* row_kbase;
    const int32_t* eidx;  // CSR position of each window element; NULL: element e is position e
    const int32_t* epos;
    const int32_t* ucan;
    const int32_t* trank;
    const int32_t* tvoff;
    const int32_t* win_U;
    const int32_t* win_ndt;
    const int32_t* win_dptr;
    const int64_t* win_vbase;
    const float* vals;
    int64_t m_aic;
    int32_t TM, TK, bf16;
    int32_t* dtile_cols;
    uint32_t* dtile_bits;
    int32_t* dtile_voff;
    void* dtile_vals;
    uint8_t* pdense;  // per original element: 1 if in a dense tile
    int32_t cap_words;  // bitmap words and tiles a window may have for the shared-memory path
    int32_t cap_tiles;
    int32_t tk_log;     // log2(TK)
    uint16_t* dtile_x;  // BF16 plans: the values go straight into the expanded tiles (zeroed
                        // beforehand) and k_pack_tiles packs them afterwards; NULL: packed here
};

// Position of element (row r, compacted column c) inside an expanded TM x TK tile: 8 x 8 blocks
// of 128 contiguous bytes (8 rows of 8 consecutive columns), the blocks of a row group side by
// side along the columns, row groups one after another.  This is the no-swizzle K-major operand
// layout of the tensor core's shared-memory descriptors (K = compacted columns, N = rows), so
// the execute kernel copies a tile into shared memory as one contiguous block.
__host__ __device__ __forceinline__ int tile_x_offset(int r, int c, int TK)
{
    return (r >> 3) * (TK >> 3) * 64 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7);
}

__global__ void __launch_bounds__(kWinThreads, 4) k_emit_tiles(EmitArgs a)
{
    __shared__ int64_t rb0[kMaxTM + 1];
    extern __shared__ __align__(16) unsigned char emit_smem[];
    uint32_t* const sbits = reinterpret_cast<uint32_t*>(emit_smem);
    int32_t* const stvoff = reinterpret_cast<int32_t*>(sbits + a.cap_words);
    uint16_t* const wpre = reinterpret_cast<uint16_t*>(stvoff + a.cap_tiles);
    int16_t* const srank = reinterpret_cast<int16_t*>(wpre + a.cap_words);
    const int tkl = a.tk_log;
    const int w = blockIdx.x;
    if (a.win_ndt[w] == 0) return;
    const int TM = a.TM, TK = a.TK, BW = TM * TK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t r0 = (int64_t)w * TM;
    const int nrows = (int)(a.m_aic - r0 < TM ? a.m_aic - r0 : TM);
    const int64_t wbase = a.row_kbase[r0];
    for (int q = threadIdx.x; q <= nrows; q += blockDim.x) rb0[q] = a.row_kbase[r0 + q] - wbase;
    const int64_t U = a.win_U[w];
    const int64_t ntile = (U + TK - 1) / TK;
    const int32_t dbase = a.win_dptr[w];
    const int32_t ndt = a.win_ndt[w];
    // the window's dense-tile bitmaps (and tile ranks) in shared memory when they fit, else the
    // plan's bitmaps with global atomics and the ranks from global memory
    const bool in_smem = (int64_t)ndt * BW <= a.cap_words && ntile <= a.cap_tiles;
    // ranks and value offsets of the tiles, value offsets of the dense tiles
    for (int64_t t = threadIdx.x; t < ntile; t += blockDim.x) {
        const int32_t k = a.trank[wbase + t];
        const int32_t tv = a.tvoff[wbase + t];
        if (in_smem) {
            srank[t] = (int16_t)k;
            stvoff[t] = tv;
        }
        if (k >= 0) a.dtile_voff[dbase + k] = (int32_t)(a.win_vbase[w] + tv);
    }
    // columns of the dense tiles: one thread per (tile, column), reads of ucan coalesced
    for (int64_t q = threadIdx.x; q < ntile * TK; q += blockDim.x) {
        const int32_t k = a.trank[wbase + (q >> tkl)];
        if (k < 0) continue;
        a.dtile_cols[(int64_t)(dbase + k) * TK + (q & (TK - 1))] = q < U ? a.ucan[wbase + q] : -1;
    }
    if (in_smem)
        for (int q = threadIdx.x; q < ndt * BW; q += blockDim.x) sbits[q] = 0u;
    __syncthreads();
    auto rank_of = [&](int32_t pos) -> int32_t {
        return in_smem ? (int32_t)srank[pos >> tkl] : a.trank[wbase + (pos >> tkl)];
    };
    // bitmap bits: one warp per row of the window (the row of an element is its warp's row)
    for (int r = warp; r < nrows; r += nwarps) {
        const int64_t rend = rb0[r + 1];
        for (int64_t eb = rb0[r]; eb < rend; eb += 128) {  // four positions per lane in flight
            int32_t pv[4], iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = eb + 32 * u + lane;
                pv[u] = e < rend ? a.epos[wbase + e] : -1;
                if (a.dtile_x) iv[u] = e < rend ? (a.eidx ? a.eidx[wbase + e] : (int32_t)(wbase + e)) : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // consecutive elements of a row mostly set bits of one word: OR the bits of lanes
                // with the same word together (segmented scan over runs of equal words), then one
                // atomic per run instead of up to 32 on one address
                int32_t key = -1;
                uint32_t mbit = 0u;
                if (pv[u] >= 0) {
                    const int32_t k = rank_of(pv[u]);
                    if (k >= 0) {
                        const int bit = (r << tkl) + (pv[u] & (TK - 1));
                        key = k * BW + (bit >> 5);
                        mbit = 1u << (bit & 31);
                        if (a.dtile_x) {  // BF16: the value into its expanded tile
                            const float v = __ldg(a.vals + iv[u]);
                            __nv_bfloat16 h = __float2bfloat16_rn(v);
                            a.dtile_x[(int64_t)(dbase + k) * TM * TK + tile_x_offset(r, pv[u] & (TK - 1), TK)] =
                                *reinterpret_cast<uint16_t*>(&h);
                            a.pdense[iv[u]] = 1;
                        }
                    }
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t ko = __shfl_up_sync(0xffffffffu, key, o);
                    const uint32_t mo = __shfl_up_sync(0xffffffffu, mbit, o);
                    if (lane >= o && ko == key) mbit |= mo;
                }
                const int32_t kn = __shfl_down_sync(0xffffffffu, key, 1);
                if (key >= 0 && (lane == 31 || kn != key)) {
                    if (in_smem) atomicOr(&sbits[key], mbit);
                    else atomicOr(a.dtile_bits + (int64_t)dbase * BW + key, mbit);
                }
            }
        }
    }
    __syncthreads();
    if (a.dtile_x) {  // BF16: values already placed; k_pack_tiles packs them from the tiles
        if (in_smem)
            for (int q = threadIdx.x; q < ndt * BW; q += blockDim.x) a.dtile_bits[(int64_t)dbase * BW + q] = sbits[q];
        return;
    }
    // per dense tile, the value index of each bitmap word's first bit
    if (in_smem) {
        for (int q = threadIdx.x; q < ndt * BW; q += blockDim.x) a.dtile_bits[(int64_t)dbase * BW + q] = sbits[q];
        for (int k = threadIdx.x; k < ndt; k += blockDim.x) {
            int acc = 0;  // at most TM * TK = 2048 values a tile
            for (int q = 0; q < BW; ++q) {
                wpre[k * BW + q] = (uint16_t)acc;
                acc += __popc(sbits[k * BW + q]);
            }
        }
        __syncthreads();
    }
    // packed values in bitmap order
    const int64_t vbase = a.win_vbase[w];
    for (int r = warp; r < nrows; r += nwarps) {
        const int64_t rend = rb0[r + 1];
        for (int64_t eb = rb0[r]; eb < rend; eb += 128) {
          int32_t pv[4], iv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
              const int64_t e = eb + 32 * u + lane;
              pv[u] = e < rend ? a.epos[wbase + e] : -1;
              iv[u] = e < rend ? (a.eidx ? a.eidx[wbase + e] : (int32_t)(wbase + e)) : -1;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int32_t pos = pv[u];
            const int32_t p = iv[u];
            if (pos < 0) continue;
            const int32_t k = rank_of(pos);
            if (k < 0) continue;
            const int32_t t = pos >> tkl;
            const int bit = (r << tkl) + (pos & (TK - 1));
            int idx = 0;
            int32_t tv;
            if (in_smem) {
                idx = wpre[k * BW + (bit >> 5)] + __popc(sbits[k * BW + (bit >> 5)] & ((1u << (bit & 31)) - 1u));
                tv = stvoff[t];
            } else {
                const uint32_t* bw = a.dtile_bits + (int64_t)(dbase + k) * BW;
                for (int q = 0; q < (bit >> 5); ++q) idx += __popc(__ldcg(bw + q));
                idx += __popc(__ldcg(bw + (bit >> 5)) & ((1u << (bit & 31)) - 1u));
                tv = a.tvoff[wbase + t];
            }
            const int64_t vi = vbase + tv + idx;
            const float v = __ldg(a.vals + p);
            if (a.bf16) {
                __nv_bfloat16 h = __float2bfloat16_rn(v);
                const uint16_t hb = *reinterpret_cast<uint16_t*>(&h);
                reinterpret_cast<uint16_t*>(a.dtile_vals)[vi] = hb;
            } else {
                reinterpret_cast<float*>(a.dtile_vals)[vi] = v;
            }
            a.pdense[p] = 1;
          }
        }
    }
}

// W9b: BF16 plans, packed values from the expanded tiles (emission wrote each value straight into
// its tile at tile_x_offset).  One warp per tile: the lanes take the bitmap's words in order, 32
// bits at a time; a set bit's value goes to its rank in bitmap order (the words' popcounts scanned
// across the lanes, plus the bits before it in its word).
__global__ void k_pack_tiles(const uint32_t* __restrict__ bits, const int32_t* __restrict__ voff,
                             const uint16_t* __restrict__ x, int64_t n_dtiles, int32_t TM, int32_t TK,
                             uint16_t* __restrict__ vals)
{
    const int lane = threadIdx.x & 31;
    const int BW = TM * TK / 32;
    const int WPL = (BW + 31) / 32;
    const int tkl = TK == 32 ? 5 : 4;
    for (int64_t d = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < n_dtiles;
         d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t* tb = bits + d * BW;
        uint32_t wv[2] = {0u, 0u};
        int own = 0;
        for (int j = 0; j < WPL; ++j) {
            const int q = lane * WPL + j;
            wv[j] = q < BW ? __ldg(tb + q) : 0u;
            own += __popc(wv[j]);
        }
        int incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - own;
        const int64_t v0 = __ldg(voff + d);
        const uint16_t* tx = x + d * (int64_t)TM * TK;
#pragma unroll 8
        for (int q = 0; q < BW; ++q) {
            const int src = WPL == 2 ? q >> 1 : q, j = WPL == 2 ? q & 1 : 0;
            const uint32_t word = __shfl_sync(0xffffffffu, j == 0 ? wv[0] : wv[1], src);
            int base = __shfl_sync(0xffffffffu, excl, src);
            if (j == 1) base += __popc(__shfl_sync(0xffffffffu, wv[0], src));
            if ((word >> lane) & 1u) {
                const int b = 32 * q + lane;
                vals[v0 + base + __popc(word & ((1u << lane) - 1u))] = tx[tile_x_offset(b >> tkl, b & (TK - 1), TK)];
            }
        }
    }
}

// the largest window's dense tiles and tiles (emission's shared-memory sizing)
__global__ void k_window_max(const int32_t* __restrict__ win_ndt, const int32_t* __restrict__ win_U, int64_t n_win,
                             int32_t TK, int64_t* out)
{
    int64_t mt = 0, mu = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_win; w += (int64_t)gridDim.x * blockDim.x) {
        mt = max(mt, (int64_t)win_ndt[w]);
        mu = max(mu, ((int64_t)win_U[w] + TK - 1) / TK);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mt = max(mt, __shfl_xor_sync(0xffffffffu, mt, o));
        mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)mt);
        atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)mu);
    }
}

// W10: residual CSR (warp per row)
__global__ void k_residual_scatter(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                   const float* __restrict__ vals, const uint8_t* __restrict__ pdense,
                                   const int32_t* __restrict__ res_rowptr, int64_t m,
                                   int32_t* res_col, float* res_val)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t b = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
        int64_t out = res_rowptr[i];
        for (int64_t p0 = b; p0 < e; p0 += 128) {  // four batches of 32 loads in flight
            uint8_t dn[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                dn[u] = p < e ? pdense[p] : 1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t p = p0 + 32 * u + lane;
                const bool keep = p < e && !dn[u];
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int64_t o = out + __popc(bal & ((1u << lane) - 1u));
                    res_col[o] = __ldg(colidx + p);
                    res_val[o] = __ldg(vals + p);
                }
                out += __popc(bal);
            }
        }
    }
}

__global__ void k_fill_win_rows(const int32_t* __restrict__ aic_rows, int64_t m_aic, int64_t total,
                                int32_t* win_rows)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < total;
         s += (int64_t)gridDim.x * blockDim.x)
        win_rows[s] = s < m_aic ? aic_rows[s] : -1;
}

static int32_t ilog2(int32_t v)
{
    int32_t l = 0;
    while ((2 << l) <= v) ++l;
    return l;
}

static unsigned wgrid(int64_t n, int threads = 256)
{
    int64_t g = ceil_div(n > 0 ? n : 1, threads);
    return (unsigned)(g < 8 * 152 * 8 ? g : 8 * 152 * 8);
}

// ---------------------------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------------
// Section 6.1 local reordering, one CTA per cluster of CR consecutive kept rows: the first
// unassigned row anchors a window and takes the TM - 1 unassigned rows with the largest Jaccard
// similarity of kept-column sets (earlier rows first on ties), best first.  Similarities are
// compared exactly as fractions (cross products in 64 bits).
//
// The intersections |cols(anchor) & cols(b)| come from an index of the cluster's kept entries
// by column: a hash table of chains in shared memory (heads) with the chain links and each
// entry's row in global scratch indexed by the entry's CSR position (clusters own disjoint
// rows, hence disjoint positions).  For an anchor, each of its kept columns walks its chain and
// counts one for every unassigned row holding that column, so the work per anchor is the number
// of entries sharing a column with it, not the cluster's size times the rows' lengths.
// ---------------------------------------------------------------------------------------------
constexpr int kReorderThreads = 256;
constexpr int kReorderHash = 4096;  // chain heads per cluster (power of two)

struct SimKey {
    int64_t num, den;  // Jaccard = num / den (0 / 1 for two empty sets)
    int32_t pos;       // position in the cluster; INT32_MAX: no candidate
};

__device__ __forceinline__ bool sim_better(const SimKey& x, const SimKey& y)
{
    if (x.pos == INT32_MAX) return false;
    if (y.pos == INT32_MAX) return true;
    const int64_t l = x.num * y.den, r = y.num * x.den;
    return l > r || (l == r && x.pos < y.pos);
}

__device__ __forceinline__ uint32_t col_hash(int32_t c)
{
    return ((uint32_t)c * 2654435761u) >> (32 - 12);  // 12 bits: kReorderHash buckets
}

__global__ void __launch_bounds__(kReorderThreads) k_local_reorder(
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
    const int32_t* __restrict__ colcount, int32_t tau_col, const int32_t* __restrict__ aic_in,
    int64_t m_aic, int TM, int CR, int32_t* __restrict__ aic_out, int32_t* __restrict__ link,
    int16_t* __restrict__ erow)
{
    static_assert(kReorderHash == 1 << 12, "col_hash yields 12 bits");
    __shared__ uint8_t used[kReorderMaxRows];
    __shared__ int32_t klen[kReorderMaxRows];
    __shared__ int32_t inter[kReorderMaxRows];
    __shared__ int32_t head[kReorderHash];
    __shared__ SimKey wbest[kReorderThreads / 32];
    __shared__ int32_t s_anchor, s_out, s_next, s_win;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * CR;
    if (c0 >= m_aic) return;
    const int R = (int)(m_aic - c0 < CR ? m_aic - c0 : CR);
    auto kept = [&](int32_t j) { return tau_col <= 0 || colcount[j] > tau_col; };
    for (int q = threadIdx.x; q < kReorderHash; q += blockDim.x) head[q] = -1;
    __syncthreads();
    // the index: one warp per row, its kept entries pushed on their columns' chains
    for (int b = warp; b < R; b += blockDim.x >> 5) {
        const int32_t i = aic_in[c0 + b];
        const int32_t p0 = rowptr[i], p1 = rowptr[i + 1];
        int32_t cnt = 0;
        for (int32_t p = p0 + lane; p < p1; p += 32) {
            const int32_t c = colidx[p];
            if (!kept(c)) continue;
            ++cnt;
            erow[p] = (int16_t)b;
            link[p] = atomicExch(&head[col_hash(c)], p);
        }
        cnt = warp_sum(cnt);
        if (lane == 0) {
            klen[b] = cnt;
            used[b] = 0;
        }
    }
    if (threadIdx.x == 0) {
        s_out = 0;
        s_next = 0;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {  // the first unassigned row anchors the next window
            int a = s_next;
            while (a < R && used[a]) ++a;
            s_next = a;
            s_anchor = a;
            if (a < R) {
                used[a] = 1;
                aic_out[c0 + s_out++] = aic_in[c0 + a];
            }
        }
        for (int b = threadIdx.x; b < R; b += blockDim.x) inter[b] = 0;
        __syncthreads();
        const int a = s_anchor;
        if (a >= R) break;
        const int32_t ia = aic_in[c0 + a];
        // intersections through the index: each kept column of the anchor walks its chain
        for (int32_t p = rowptr[ia] + threadIdx.x; p < rowptr[ia + 1]; p += blockDim.x) {
            const int32_t c = colidx[p];
            if (!kept(c)) continue;
            for (int32_t q = head[col_hash(c)]; q >= 0; q = link[q]) {
                if (colidx[q] != c) continue;  // another column in the same bucket
                const int b = erow[q];
                if (!used[b]) atomicAdd(&inter[b], 1);
            }
        }
        __syncthreads();
        for (int pick = 0; pick < TM - 1; ++pick) {
            SimKey best{0, 1, INT32_MAX};
            for (int b = threadIdx.x; b < R; b += blockDim.x) {
                if (used[b]) continue;
                const int64_t uni = (int64_t)klen[a] + klen[b] - inter[b];
                const SimKey k{uni > 0 ? (int64_t)inter[b] : 0, uni > 0 ? uni : 1, b};
                if (sim_better(k, best)) best = k;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                SimKey other;
                other.num = __shfl_xor_sync(0xffffffffu, best.num, o);
                other.den = __shfl_xor_sync(0xffffffffu, best.den, o);
                other.pos = __shfl_xor_sync(0xffffffffu, best.pos, o);
                if (sim_better(other, best)) best = other;
            }
            if (lane == 0) wbest[warp] = best;
            __syncthreads();
            if (threadIdx.x == 0) {
                SimKey w = wbest[0];
                for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
                    if (sim_better(wbest[q], w)) w = wbest[q];
                s_win = w.pos;
                if (w.pos != INT32_MAX) {
                    used[w.pos] = 1;
                    aic_out[c0 + s_out++] = aic_in[c0 + w.pos];
                }
            }
            __syncthreads();
            if (s_win == INT32_MAX) break;
        }
    }
}

ns_status_t window_pass(Plan* P, WindowResult* W, cudaStream_t s)
{
    const ns_tune_t& t = P->tune;
    const int64_t m = P->st.m, n = P->st.n, nnz = P->st.nnz;
    const int TM = t.TM, TK = t.TK, BW = TM * TK / 32;
    const bool bf16 = P->dtype == NS_BF16;

    // ---- stage 1 arrays: kept rows, column counts, kept lengths ----
    Arena a1;                          // temporaries of stage 1
    int64_t* partial = nullptr;
    int64_t* totals = nullptr;
    int32_t* aic_rows = nullptr;
    int32_t* colcount = nullptr;
    int64_t* row_kbase = nullptr;
    a1.reserve(&partial, scan_partials(m + 1));
    a1.reserve(&totals, 8);
    a1.reserve(&aic_rows, m);
    a1.reserve(&row_kbase, m + 1);
    if (t.tau_col > 0) a1.reserve(&colcount, n);
    NS_TRY(a1.commit(s));
    NS_CUDA_TRY(cudaMemsetAsync(totals, 0, sizeof(int64_t) * 8, s));
    NS_TRY(device_scan<int64_t>(KeepLoad{P->rowptr, t.tau_row}, KeepStore{aic_rows}, m, partial,
                                totals + 0, s));
    int64_t m_aic_h = 0;
    NS_CUDA_TRY(cudaMemcpyAsync(&m_aic_h, totals + 0, sizeof m_aic_h, cudaMemcpyDeviceToHost, s));
    NS_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t m_aic = m_aic_h;
    if (t.tau_col > 0) {
        NS_CUDA_TRY(cudaMemsetAsync(colcount, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
        if (m_aic > 0) {
            k_colcount<<<wgrid(m_aic * 32), 256, 0, s>>>(P->rowptr, P->colidx, aic_rows, m_aic, colcount);
            NS_LAUNCH_CHECK();
        }
    }
    if (t.reorder > 0 && m_aic > 0) {  // Section 6.1 local reordering of the kept rows
        int32_t* reordered = nullptr;
        int32_t* link = nullptr;  // the clusters' column indexes, by CSR position
        int16_t* erow = nullptr;
        Arena ar;
        ar.reserve(&reordered, m_aic);
        ar.reserve(&link, nnz > 0 ? nnz : 1);
        ar.reserve(&erow, nnz > 0 ? nnz : 1);
        NS_TRY(ar.commit(s));
        const int CR = t.reorder * TM;
        k_local_reorder<<<(unsigned)ceil_div(m_aic, CR), kReorderThreads, 0, s>>>(
            P->rowptr, P->colidx, colcount, t.tau_col, aic_rows, m_aic, TM, CR, reordered, link, erow);
        NS_LAUNCH_CHECK();
        NS_CUDA_TRY(cudaMemcpyAsync(aic_rows, reordered, sizeof(int32_t) * m_aic, cudaMemcpyDeviceToDevice, s));
        ar.release(s);
    }
    NS_TRY(device_scan<int64_t>(KeptLenLoad{P->rowptr, P->colidx, aic_rows, colcount, t.tau_col},
                                KeptLenStore{row_kbase}, m_aic, partial, row_kbase + m_aic, s));
    int64_t nnz_win = 0;
    if (m_aic > 0) {
        NS_CUDA_TRY(cudaMemcpyAsync(&nnz_win, row_kbase + m_aic, sizeof nnz_win, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        NS_CUDA_TRY(cudaMemsetAsync(row_kbase, 0, sizeof(int64_t), s));
    }
    const int64_t n_win = ceil_div(m_aic, TM);
    P->st.m_aic = m_aic;
    P->st.n_win = n_win;

    // ---- stage 2 arrays: plan arrays known by now + window temporaries ----
    Arena pa;  // plan-owned
    pa.reserve(&P->aic_rows, m_aic);
    pa.reserve(&P->win_rows, n_win * TM);
    pa.reserve(&P->win_dptr, n_win + 1);
    pa.reserve(&P->dwin, n_win);
    pa.reserve(&P->dwin_absorb, n_win);
    pa.reserve(&P->res_rowptr_own, m + 1);
    pa.reserve(&P->rl_rows, m);
    pa.reserve(&P->rl_start, m + 1);
    NS_TRY(pa.commit(s));
    P->blocks.push_back(pa.take());
    P->res_rowptr = P->res_rowptr_own;

    // Every row kept, in order, with all its columns: the window elements are A's own column
    // array in CSR order, so the element gather is skipped (element e is CSR position e).
    const bool ident = m_aic == m && t.reorder <= 0 && t.tau_col <= 0 && nnz_win == nnz;
    Arena tw;  // window temporaries (freed when planning ends)
    int32_t *ekey = nullptr, *eidx = nullptr;
    int32_t *sb0, *sb1, *uasc, *ucnt, *upos, *ucan, *ccnt, *trank, *tvoff, *epos;
    int32_t *win_U, *win_ndt, *win_ndv, *res_len;
    int64_t *win_res, *win_vbase, *part2;
    int8_t* row_state;
    int64_t* dcost;
    uint8_t* pdense;
    if (!ident) {
        tw.reserve(&ekey, nnz_win);
        tw.reserve(&eidx, nnz_win);
    }
    for (int32_t** q : {&sb0, &sb1, &uasc, &ucnt, &upos, &ucan, &ccnt, &trank, &tvoff, &epos})
        tw.reserve(q, nnz_win);
    tw.reserve(&win_U, n_win);
    tw.reserve(&win_ndt, n_win);
    tw.reserve(&win_ndv, n_win);
    tw.reserve(&win_res, n_win);
    tw.reserve(&win_vbase, n_win + 1);
    tw.reserve(&res_len, m);
    tw.reserve(&part2, scan_partials(m + 1));
    tw.reserve(&row_state, m);
    tw.reserve(&dcost, n_win);
    tw.reserve(&pdense, nnz);
    NS_TRY(tw.commit(s));
    W->temp = tw.take();
    W->row_state = row_state;
    W->dcost = dcost;

    if (m_aic > 0) {
        NS_CUDA_TRY(cudaMemcpyAsync(P->aic_rows, aic_rows, sizeof(int32_t) * m_aic, cudaMemcpyDeviceToDevice, s));
        k_fill_win_rows<<<wgrid(n_win * TM), 256, 0, s>>>(aic_rows, m_aic, n_win * TM, P->win_rows);
        NS_LAUNCH_CHECK();
        if (!ident) {
            k_gather_window_elems<<<wgrid(m_aic * 32), 256, 0, s>>>(P->rowptr, P->colidx, aic_rows, m_aic,
                                                                   row_kbase, colcount, t.tau_col, ekey, eidx);
            NS_LAUNCH_CHECK();
        }
    }
    k_res_len_free_rows<<<wgrid(m), 256, 0, s>>>(P->rowptr, m, t.tau_row, res_len);
    NS_LAUNCH_CHECK();
    if (n_win > 0) {
        const bool count_cols = n <= kDenseCols;
        WinArgs wa{P->rowptr, aic_rows, row_kbase, ident ? P->colidx : ekey, m_aic, TM, TK, t.tau_tile, t.col_order,
                   sb0, sb1, uasc, ucnt, upos, ucan, ccnt, trank, tvoff, epos,
                   win_U, win_ndt, win_ndv, win_res, res_len, (int32_t)n, count_cols ? 1 : 0};
        // the counting table (3 bytes a column) or the two sort buffers, whichever is larger
        const size_t tbl = count_cols ? count_table_bytes(n) : 0;
        const size_t keys = (size_t)2 * kWinSmemKeys * sizeof(int32_t);
        const size_t dyn = tbl > keys ? tbl : keys;
        // static + dynamic shared memory above 48 KB needs the opt-in; one fixed limit (the largest
        // counting table) keeps concurrent planners from lowering it under each other's launches
        static_assert(count_table_bytes(kDenseCols) >= 2 * kWinSmemKeys * 4, "sort buffers fit the opt-in limit");
        NS_CUDA_TRY(cudaFuncSetAttribute(k_window_compact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)count_table_bytes(kDenseCols)));
        k_window_compact<<<(unsigned)n_win, kWinThreads, dyn, s>>>(wa);
        NS_LAUNCH_CHECK();
    }

    // ---- W6: scans ----
    NS_CUDA_TRY(cudaMemsetAsync(totals, 0, sizeof(int64_t) * 8, s));
    NS_TRY(device_scan<int64_t>(I32Load{win_ndt}, PtrStore32{P->win_dptr}, n_win, partial, totals + 1, s));
    NS_TRY(device_scan<int64_t>(I32Load{win_ndv}, PtrStore64{win_vbase}, n_win, partial, totals + 2, s));
    NS_TRY(device_scan<int64_t>(DenseWinLoad{win_ndt}, DenseWinStore{P->dwin}, n_win, partial, totals + 3, s));
    NS_TRY(device_scan<int64_t>(I32Load{res_len}, PtrStore32{P->res_rowptr_own}, m, part2, totals + 4, s));
    if (n_win > 0) {
        k_window_max<<<wgrid(n_win), 256, 0, s>>>(win_ndt, win_U, n_win, TK, totals + 6);
        NS_LAUNCH_CHECK();
    }
    int64_t ht[8];
    NS_CUDA_TRY(cudaMemcpyAsync(ht, totals, sizeof ht, cudaMemcpyDeviceToHost, s));
    NS_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t n_dtiles = ht[1], n_dvals = ht[2], n_dwin = ht[3], n_res = ht[4];
    const int64_t max_ndt = ht[6], max_ntile = ht[7];
    P->st.n_dtiles = n_dtiles;
    P->st.n_dvals = n_dvals;
    P->st.n_dwin = n_dwin;
    P->st.n_res = n_res;
    // scan totals at the end of the pointer arrays
    {
        int32_t v32 = (int32_t)n_dtiles;
        NS_CUDA_TRY(cudaMemcpyAsync(P->win_dptr + n_win, &v32, sizeof v32, cudaMemcpyHostToDevice, s));
        int32_t r32 = (int32_t)n_res;
        NS_CUDA_TRY(cudaMemcpyAsync(P->res_rowptr_own + m, &r32, sizeof r32, cudaMemcpyHostToDevice, s));
    }

    // ---- W7: dense windows, ownership; W8: residual list ----
    NS_CUDA_TRY(cudaMemsetAsync(row_state, 0, (size_t)(m > 0 ? m : 1), s));
    if (n_dwin > 0) {
        k_dense_windows<<<wgrid(n_dwin), 256, 0, s>>>(P->dwin, n_dwin, win_ndt, win_res, aic_rows, m_aic,
                                                      TM, TK, t.absorb_cap, t.cost_tc, t.cost_res,
                                                      P->dwin_absorb, dcost, row_state);
        NS_LAUNCH_CHECK();
    }
    NS_TRY(device_scan<int64_t>(RlLoad{row_state, res_len}, RlStore{P->rl_rows, P->rl_start}, m, part2,
                                totals + 5, s));

    // ---- W9/W10: dense tiles and the residual CSR ----
    Arena pb;
    pb.reserve(&P->dtile_cols, n_dtiles * TK);
    pb.reserve(&P->dtile_bits, n_dtiles * BW);
    pb.reserve(&P->dtile_voff, n_dtiles + 1);
    pb.reserve_bytes(&P->dtile_vals, (size_t)(n_dvals > 0 ? n_dvals : 1) * (bf16 ? 2 : 4));
    pb.reserve(&P->res_col_own, n_res);
    pb.reserve(&P->res_val_own, n_res);
    if (bf16) pb.reserve(&P->dtile_x, n_dtiles * TM * TK);
    NS_TRY(pb.commit(s));
    P->blocks.push_back(pb.take());
    P->res_col = P->res_col_own;
    P->res_val = P->res_val_own;
    NS_CUDA_TRY(cudaMemsetAsync(P->dtile_bits, 0, sizeof(uint32_t) * (n_dtiles * BW > 0 ? n_dtiles * BW : 1), s));
    NS_CUDA_TRY(cudaMemsetAsync(P->dtile_vals, 0, (size_t)(n_dvals > 0 ? n_dvals : 1) * (bf16 ? 2 : 4), s));
    NS_CUDA_TRY(cudaMemsetAsync(pdense, 0, (size_t)(nnz > 0 ? nnz : 1), s));
    {
        int32_t v32 = (int32_t)n_dvals;
        NS_CUDA_TRY(cudaMemcpyAsync(P->dtile_voff + n_dtiles, &v32, sizeof v32, cudaMemcpyHostToDevice, s));
    }
    if (n_dtiles > 0) {
        // shared memory for the largest window, or for as much as fits the limit
        int64_t cap_tiles = max_ntile, cap_words = max_ndt * BW;
        if (cap_tiles * 6 + cap_words * 6 > kEmitSmemMax) {
            cap_tiles = cap_tiles * 6 <= kEmitSmemMax / 4 ? cap_tiles : kEmitSmemMax / 24;
            cap_words = (kEmitSmemMax - cap_tiles * 6) / 6;
        }
        cap_words &= ~int64_t(3);  // keeps the tiles' offsets 16-byte aligned
        const size_t dyn = (size_t)(cap_words * 6 + cap_tiles * 6 + 16);
        // one fixed opt-in limit, so concurrent planners never lower it under each other
        NS_CUDA_TRY(cudaFuncSetAttribute(k_emit_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kEmitSmemMax + 16));
        EmitArgs ea{row_kbase, eidx, epos, ucan, trank, tvoff, win_U, win_ndt, P->win_dptr, win_vbase,
                    P->vals, m_aic, TM, TK, bf16 ? 1 : 0, P->dtile_cols, P->dtile_bits, P->dtile_voff,
                    P->dtile_vals, pdense, (int32_t)cap_words, (int32_t)cap_tiles, ilog2(TK),
                    bf16 ? P->dtile_x : nullptr};
        if (bf16) NS_CUDA_TRY(cudaMemsetAsync(P->dtile_x, 0, sizeof(uint16_t) * n_dtiles * TM * TK, s));
        k_emit_tiles<<<(unsigned)n_win, kWinThreads, dyn, s>>>(ea);
        NS_LAUNCH_CHECK();
        if (bf16) {
            const int64_t warps = n_dtiles;
            const int64_t blocks = (warps * 32 + 255) / 256;
            k_pack_tiles<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(
                P->dtile_bits, P->dtile_voff, P->dtile_x, n_dtiles, TM, TK,
                reinterpret_cast<uint16_t*>(P->dtile_vals));
            NS_LAUNCH_CHECK();
        }
    }
    if (m > 0) {
        k_residual_scatter<<<wgrid(m * 32), 256, 0, s>>>(P->rowptr, P->colidx, P->vals, pdense,
                                                          P->res_rowptr_own, m, P->res_col_own,
                                                          P->res_val_own);
        NS_LAUNCH_CHECK();
    }
    int64_t rl_tot = 0;
    NS_CUDA_TRY(cudaMemcpyAsync(&rl_tot, totals + 5, sizeof rl_tot, cudaMemcpyDeviceToHost, s));
    NS_CUDA_TRY(cudaStreamSynchronize(s));
    P->st.n_rl = rl_tot >> 32;
    P->st.T = rl_tot & 0xffffffffLL;
    {
        int32_t T32 = (int32_t)P->st.T;
        NS_CUDA_TRY(cudaMemcpyAsync(P->rl_start + P->st.n_rl, &T32, sizeof T32, cudaMemcpyHostToDevice, s));
        NS_CUDA_TRY(cudaStreamSynchronize(s));  // the host values above must outlive the copies
    }
    a1.release(s);
    return NS_OK;
}

}  // namespace ns
