// ns_plan.cu -- the device-side planner (Sections 4, 5.2.2, 6.1 and 7 of arXiv 2606.22482).
//
// Turns a CSR matrix into the execution plan consumed by the persistent kernel:
//   a1  validate + row lengths Len (Eq. 4)
//   a2  row extraction: Len <= tau_row -> residual (Eq. 5 with an integer threshold)
//   a3  column extraction inside the kept rows: count <= tau_col -> residual
//   a4  row windows of TM consecutive kept rows (Section 6.1)
//   a5  column compaction per window, canonical column order, TK-wide tiles
//   a6  density binning: tile dense iff nnz >= tau_tile (alpha of Eq. 3 as an integer)
//   a7  residual CSR of everything not in a dense tile
//   a8  merge-path chunks of the residual with short rows never cut
//   a9  work items ordered by cost class (Eq. 1), heaviest first (Section 7 balanced lists)
// Every array is defined exactly like the CPU reference partition; the tests compare them bit
// for bit.  All arithmetic is integer; all reductions have a fixed order.
#include "ns_internal.cuh"
#include "ns_scan.cuh"

namespace ns {

// ---------------------------------------------------------------------------------------------
// a1: validation without per-row loops.  Inside a row columns must strictly increase, so every
// position p where colidx[p+1] <= colidx[p] ("descent") must be a row start.  Counting all
// descents (element-parallel) and the descents that sit at row starts (row-parallel) and
// comparing the two counts checks sortedness and uniqueness of every row.
// ---------------------------------------------------------------------------------------------
enum { kCtrTicket = 0, kCtrDone = 1, kCtrStatus = 2 };
// 64-bit counters used by the planner
enum { kCnBadRange = 0, kCnDescents = 1, kCnBadPtr = 2, kCnStartDescents = 3, kCnTotals = 4 };

// Adds two per-thread counts into cnt[ia] and cnt[ib] with one atomic each per block: every
// counter is a single address, so per-warp atomics would queue up at one L2 slice.  Called by all
// threads of the block.
__device__ __forceinline__ void block_add2(unsigned long long* cnt, int ia, unsigned long long a, int ib,
                                           unsigned long long b)
{
    __shared__ unsigned long long sa[32], sb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        a = warp_sum(lane < nw ? sa[lane] : 0ull);
        b = warp_sum(lane < nw ? sb[lane] : 0ull);
        if (lane == 0) {
            if (a) atomicAdd(cnt + ia, a);
            if (b) atomicAdd(cnt + ib, b);
        }
    }
}

__global__ void k_check_elems(const int32_t* __restrict__ colidx, int64_t nnz, int32_t n,
                              unsigned long long* cnt)
{
    unsigned long long bad = 0, desc = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = __ldg(colidx + p);
        bad += (c < 0 || c >= n);
        if (p + 1 < nnz) desc += (__ldg(colidx + p + 1) <= c);
    }
    block_add2(cnt, kCnBadRange, bad, kCnDescents, desc);
}

// the same counts from 16-byte loads (colidx 16-byte aligned): quad q holds positions 4q .. 4q+3,
// the descent at 4q+3 compares with the next quad's first entry; the last nnz mod 4 positions go
// to the first threads of the grid.  Each thread keeps four quads in flight.
__global__ void k_check_elems4(const int4* __restrict__ colidx4, const int32_t* __restrict__ colidx,
                               int64_t nnz, int32_t n, unsigned long long* cnt)
{
    constexpr int U = 4;
    unsigned long long bad = 0, desc = 0;
    const int64_t nq = nnz >> 2;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = t0; q0 < nq; q0 += U * stride) {
        int4 v[U];
        int32_t nx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = q0 + u * stride;
            if (q < nq) {
                v[u] = __ldg(colidx4 + q);
                nx[u] = 4 * q + 4 < nnz ? __ldg(colidx + 4 * q + 4) : INT32_MAX;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (q0 + u * stride < nq) {
                const int4 w = v[u];
                bad += (w.x < 0 || w.x >= n) + (w.y < 0 || w.y >= n) + (w.z < 0 || w.z >= n) +
                       (w.w < 0 || w.w >= n);
                desc += (w.y <= w.x) + (w.z <= w.y) + (w.w <= w.z) + (nx[u] <= w.w);
            }
        }
    }
    if (t0 < nnz - 4 * nq) {
        const int64_t p = 4 * nq + t0;
        const int32_t c = __ldg(colidx + p);
        bad += (c < 0 || c >= n);
        if (p + 1 < nnz) desc += (__ldg(colidx + p + 1) <= c);
    }
    block_add2(cnt, kCnBadRange, bad, kCnDescents, desc);
}

__global__ void k_check_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                             int32_t m, int64_t nnz, unsigned long long* cnt)
{
    unsigned long long bad = 0, sdesc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = __ldg(rowptr + i);
        bool ok = r >= 0 && r <= nnz;
        if (i == 0 && r != 0) ok = false;
        if (i == m && r != nnz) ok = false;
        if (i < m) {
            int64_t r1 = __ldg(rowptr + i + 1);
            if (r1 < r) ok = false;
            // a non-empty row starting after position 0: is its start a descent?
            if (ok && r1 > r && r > 0 && r < nnz) sdesc += (__ldg(colidx + r) <= __ldg(colidx + r - 1));
        }
        bad += !ok;
    }
    block_add2(cnt, kCnBadPtr, bad, kCnStartDescents, sdesc);
}

// ---------------------------------------------------------------------------------------------
// chunk rows: chunk_k0[c] = the residual-list row holding merge item c*W, c in [0, nc).  Row k
// holds items [rl_start[k], rl_start[k+1]), so it owns the multiples of W in that range: written
// row-parallel, without searches.  (rl_start strictly increases for valid inputs; the consumer
// clamps what an invalid one leaves unwritten.)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void own_chunk_rows(int64_t k, int64_t s, int64_t e, int64_t W, int64_t nc,
                                               int32_t* chunk_k0)
{
    int64_t c = s > 0 ? (s + W - 1) / W : 0;
    const int64_t ce = e > 0 ? (e + W - 1) / W : 0;
    for (; c < ce && c < nc; ++c) chunk_k0[c] = (int32_t)k;
}

__global__ void k_chunk_rows(const int32_t* __restrict__ rl_start, int64_t n_rl, int64_t W, int64_t nc,
                             int32_t* chunk_k0)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_rl;
         k += (int64_t)gridDim.x * blockDim.x)
        own_chunk_rows(k, __ldg(rl_start + k), __ldg(rl_start + k + 1), W, nc, chunk_k0);
}

// ---------------------------------------------------------------------------------------------
// the all-residual plan in one row-parallel pass: the row checks of a1, the residual row list
// (every row, merge start rowptr[i] + i), no split rows yet, and the chunk rows
// ---------------------------------------------------------------------------------------------
__global__ void k_rows_all_residual(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                    int32_t m, int64_t nnz, int64_t W, int64_t nc,
                                    unsigned long long* cnt, int32_t* rl_rows, int32_t* rl_start,
                                    int32_t* row_split, int32_t* chunk_k0)
{
    unsigned long long bad = 0, sdesc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = __ldg(rowptr + i);
        bool ok = r >= 0 && r <= nnz;
        if (i == 0 && r != 0) ok = false;
        if (i == m && r != nnz) ok = false;
        const int64_t rc = i == m ? nnz : (r < 0 ? 0 : (r > nnz ? nnz : r));
        rl_start[i] = (int32_t)(rc + i);
        if (i < m) {
            const int64_t r1 = __ldg(rowptr + i + 1);
            if (r1 < r) ok = false;
            if (ok && r1 > r && r > 0 && r < nnz) sdesc += (__ldg(colidx + r) <= __ldg(colidx + r - 1));
            rl_rows[i] = (int32_t)i;
            row_split[i] = -1;
            const int64_t r1c = i + 1 == m ? nnz : (r1 < 0 ? 0 : (r1 > nnz ? nnz : r1));
            own_chunk_rows(i, rc + i, r1c + i + 1, W, nc, chunk_k0);
        }
        bad += !ok;
    }
    block_add2(cnt, kCnBadPtr, bad, kCnStartDescents, sdesc);
}

// ---------------------------------------------------------------------------------------------
// a8: merge-path chunk boundaries with snapping.  Boundary c sits at merge item c*W unless that
// item falls in a residual row with 2*(len+1) <= W, in which case it moves to the row's start.
// rl_start must be non-decreasing (guaranteed for valid inputs; clamped otherwise).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t chunk_boundary(const int32_t* __restrict__ rl_start, int64_t T,
                                                  int64_t W, int64_t nc, int64_t c, int64_t k)
{
    if (c == 0) return 0;
    if (c >= nc) return T;
    const int64_t d = c * W;  // merge item c*W lies in row k
    const int64_t rlen = (int64_t)__ldg(rl_start + k + 1) - __ldg(rl_start + k) - 1;
    return (2 * (rlen + 1) <= W) ? (int64_t)__ldg(rl_start + k) : d;
}

// also the execution-side chunk records: rows k0 .. kL with an item in [b0, b1) (row kL + 1
// starts at or after b1), and the nonzero count = items - row ends inside the range (rows
// k0 .. kL - 1 end inside it, row kL when its end item precedes b1).  chunk_k0 (from the chunk
// rows pass) is the row of merge item c*W, which is also the row of the snapped boundary b0.
__global__ void k_chunks(const int32_t* __restrict__ rl_start, const int32_t* __restrict__ rl_rows,
                         const int32_t* __restrict__ res_rowptr, int64_t m, int64_t n_rl, int64_t T,
                         int64_t W, int64_t nc, int32_t* chunk_b, const int32_t* __restrict__ chunk_k0,
                         ChunkRec* rec)
{
    auto row_of = [&](int64_t c) -> int64_t {
        const int64_t k = __ldg(chunk_k0 + c);
        return k < 0 ? 0 : (k >= n_rl ? n_rl - 1 : k);
    };
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nc;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = c < nc ? row_of(c) : 0;
        const int64_t b = chunk_boundary(rl_start, T, W, nc, c, k0);
        chunk_b[c] = (int32_t)b;
        if (c < nc) {
            const int64_t k1 = (c + 1 < nc) ? row_of(c + 1) : n_rl - 1;
            const int64_t b1 = chunk_boundary(rl_start, T, W, nc, c + 1, k1);
            int64_t kL = k1;
            if (kL > k0 && (int64_t)__ldg(rl_start + kL) >= b1) --kL;
            ChunkRec r;
            r.b0 = (int32_t)b;
            r.b1 = (int32_t)b1;
            r.k0 = (int32_t)k0;
            r.kL = (int32_t)kL;
            r.total = -1;
            r.z0 = -1;
            if (kL >= k0) {
                r.total = (int32_t)((b1 - b) - (kL - k0) - ((int64_t)__ldg(rl_start + kL + 1) <= b1 ? 1 : 0));
                const int64_t i0 = __ldg(rl_rows + k0);
                if (i0 >= 0 && i0 < m) r.z0 = (int32_t)((int64_t)__ldg(res_rowptr + i0) + (b - __ldg(rl_start + k0)));
            }
            r.pad0 = r.pad1 = 0;
            rec[c] = r;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// pieces per residual-list row and split rows.  A row is assembled from several pieces when a
// chunk boundary cuts it or when a non-absorbing dense window also contributes to it.
// ---------------------------------------------------------------------------------------------
struct PieceInfo {
    const int32_t* rl_rows;
    const int32_t* rl_start;
    const int32_t* chunk_b;
    const int8_t* row_state;  // 2 = in a non-absorbing dense window; nullptr = none
    int64_t nc;
    int64_t W;
    __device__ __forceinline__ void pieces(int64_t k, int32_t* i_out, int32_t* np, int32_t* base) const
    {
        int32_t i = __ldg(rl_rows + k);
        int64_t s = __ldg(rl_start + k), e = __ldg(rl_start + k + 1);
        int hd = (row_state && row_state[i] == 2) ? 1 : 0;
        *i_out = i;
        if (2 * (e - s) <= W) {
            // short row: boundaries snap to its start, so it lies in one chunk; that chunk is only
            // needed when a dense window also contributes (the row is then split)
            *np = 1 + hd;
            *base = hd ? (int32_t)(upper_minus_one(chunk_b, nc, s) - 1) : 0;
            return;
        }
        int64_t fc = upper_minus_one(chunk_b, nc, s);
        int64_t lc = upper_minus_one(chunk_b, nc, e - 1);
        *np = (int32_t)(lc - fc + 1 + hd);
        *base = (int32_t)(fc - hd);
    }
};

// packed scan value: (is_split << 32) | (is_split ? pieces : 0)
struct PieceLoad {
    PieceInfo pi;
    __device__ __forceinline__ int64_t operator()(int64_t k) const
    {
        int32_t i, np, base;
        pi.pieces(k, &i, &np, &base);
        return np >= 2 ? ((int64_t)1 << 32) | (int64_t)np : 0;
    }
};

struct PieceStore {
    PieceInfo pi;
    int32_t* row_split;
    int32_t* split_row;
    int32_t* split_np;
    int32_t* split_slot;
    int32_t* split_base;
    __device__ __forceinline__ void operator()(int64_t k, int64_t pre, int64_t v) const
    {
        if (v == 0) return;
        int32_t i, np, base;
        pi.pieces(k, &i, &np, &base);
        int64_t s = pre >> 32;
        row_split[i] = (int32_t)s;
        split_row[s] = i;
        split_np[s] = np;
        split_slot[s] = (int32_t)(pre & 0xffffffffLL);
        split_base[s] = base;
    }
};

// All-residual plans have no dense windows, so a row is split only where chunk boundaries cut
// it, and only a long row (2 * (len + 1) > W) can be cut: the boundaries inside it are the
// unsnapped multiples of W.  Boundary c (1 <= c < nc) is the first cut of its row k when it lies
// strictly inside the row and boundary c - 1 does not; the row's pieces then run from chunk c - 1
// to the chunk of its end item, floor((e - 1) / W).  Scanning the nc - 1 boundaries instead of
// the rows finds the same split rows in the same (ascending) order.
struct CutInfo {
    const int32_t* rl_rows;
    const int32_t* rl_start;
    const int32_t* chunk_k0;
    int64_t n_rl;
    int64_t nc;
    int64_t W;
    // the row that boundary c cuts first, or -1; its piece count in *np
    __device__ __forceinline__ int64_t first_cut(int64_t c, int32_t* np) const
    {
        int64_t k = __ldg(chunk_k0 + c);
        k = k < 0 ? 0 : (k >= n_rl ? n_rl - 1 : k);
        const int64_t s = __ldg(rl_start + k), e = __ldg(rl_start + k + 1);
        if (2 * (e - s) <= W || c * W <= s || (c - 1) * W > s) return -1;
        int64_t lc = (e - 1) / W;
        if (lc > nc - 1) lc = nc - 1;
        *np = (int32_t)(lc - (c - 1) + 1);
        return k;
    }
};
struct CutLoad {  // item j is boundary j + 1
    CutInfo ci;
    __device__ __forceinline__ int64_t operator()(int64_t j) const
    {
        int32_t np = 0;
        return ci.first_cut(j + 1, &np) >= 0 ? ((int64_t)1 << 32) | (int64_t)np : 0;
    }
};
struct CutStore {
    CutInfo ci;
    int32_t* row_split;
    int32_t* split_row;
    int32_t* split_np;
    int32_t* split_slot;
    int32_t* split_base;
    __device__ __forceinline__ void operator()(int64_t j, int64_t pre, int64_t v) const
    {
        if (v == 0) return;
        int32_t np = 0;
        const int64_t k = ci.first_cut(j + 1, &np);
        const int32_t i = __ldg(ci.rl_rows + k);
        const int64_t sp = pre >> 32;
        row_split[i] = (int32_t)sp;
        split_row[sp] = i;
        split_np[sp] = np;
        split_slot[sp] = (int32_t)(pre & 0xffffffffLL);
        split_base[sp] = (int32_t)j;  // chunk c - 1
    }
};

// ---------------------------------------------------------------------------------------------
// a9: work items and their cost classes (floor log2 of the Eq. 1 cost), heaviest class first
// ---------------------------------------------------------------------------------------------
__global__ void k_item_costs(const int32_t* __restrict__ chunk_b, int64_t nc, int64_t group,
                             int64_t n_dwin, const int64_t* __restrict__ dcost, int64_t n_items,
                             int64_t cost_res, int64_t* item_cost)
{
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n_items;
         it += (int64_t)gridDim.x * blockDim.x) {
        int64_t c;
        if (it < n_dwin) c = dcost[it];
        else {
            int64_t q = it - n_dwin;
            int64_t c0 = q * group, c1 = c0 + group < nc ? c0 + group : nc;
            c = ((int64_t)__ldg(chunk_b + c1) - __ldg(chunk_b + c0)) * cost_res;
        }
        item_cost[it] = c;
    }
}

__device__ __forceinline__ int cost_class(int64_t c) { return c <= 1 ? 0 : 63 - __clzll((unsigned long long)c); }

struct CostKey {
    const int64_t* cost;
    __device__ __forceinline__ int operator()(int64_t i) const { return cost_class(cost[i]); }
};
struct QueueEmit {
    int32_t* queue;
    __device__ __forceinline__ void operator()(int64_t i, int64_t pos) const { queue[pos] = (int32_t)i; }
};

__global__ void k_bucket_offsets(int32_t* hist, int64_t nblocks)
{
    __shared__ int64_t tot[kSortBuckets];
    __shared__ int64_t base[kSortBuckets];
    const int b = threadIdx.x;
    if (b < kSortBuckets) {
        int64_t t = 0;
        for (int64_t k = 0; k < nblocks; ++k) t += hist[k * kSortBuckets + b];
        tot[b] = t;
    }
    __syncthreads();
    if (b == 0) {
        int64_t acc = 0;
        for (int q = kSortBuckets - 1; q >= 0; --q) {
            base[q] = acc;
            acc += tot[q];
        }
    }
    __syncthreads();
    if (b < kSortBuckets) {
        int64_t acc = base[b];
        for (int64_t k = 0; k < nblocks; ++k) {
            int32_t h = hist[k * kSortBuckets + b];
            hist[k * kSortBuckets + b] = (int32_t)acc;
            acc += h;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// hot B rows (Section 6.2.1: the rows of B gathered most often are kept in L2, capped at about
// 80% of its capacity; the rest bypass).  Execution hint only, not part of the partition.
// ---------------------------------------------------------------------------------------------
__global__ void k_gather_counts(const int32_t* __restrict__ col, int64_t nres, int32_t n, int32_t* cnt)
{
    const int lane = threadIdx.x & 31;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p - lane < nres;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = p < nres ? __ldg(col + p) : -1;
        // one atomic per distinct column per warp (hub columns repeat inside a warp)
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && c < n && (__ffs(peers) - 1) == lane) atomicAdd(cnt + c, __popc(peers));
    }
}

// 64 bins of floor(log2(count)) over the columns
__global__ void k_count_bins(const int32_t* __restrict__ cnt, int32_t n, unsigned long long* bins)
{
    __shared__ unsigned long long sb[64];
    if (threadIdx.x < 64) sb[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cnt[j];
        if (c > 0) atomicAdd(&sb[31 - __clz(c)], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 64 && sb[threadIdx.x]) atomicAdd(bins + threadIdx.x, sb[threadIdx.x]);
}

// threshold: the smallest power of two h such that the columns with count >= h fit in `cap` rows
__global__ void k_hot_threshold(const unsigned long long* bins, int64_t cap, int32_t* h_out)
{
    if (threadIdx.x != 0) return;
    unsigned long long acc = 0;
    int b = 31;
    for (; b >= 0; --b) {
        if (acc + bins[b] > (unsigned long long)cap) break;
        acc += bins[b];
    }
    *h_out = b >= 31 ? 0x7fffffff : (1 << (b + 1));  // counts >= 2^(b+1) are hot
}

__global__ void k_hot_bits(const int32_t* __restrict__ cnt, int32_t n, const int32_t* h, uint32_t* bits)
{
    const int lane = threadIdx.x & 31;
    const int32_t th = *h;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j - lane < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const bool hot = j < n && cnt[j] >= th;
        const unsigned b = __ballot_sync(0xffffffffu, hot);
        if (lane == 0 && j < n) bits[j >> 5] = b;
    }
}

// fill with a 32-bit value
__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

static unsigned grid_for(int64_t n, int threads = 256)
{
    int64_t g = ceil_div(n > 0 ? n : 1, threads);
    return (unsigned)(g < 8 * 152 * 8 ? g : 8 * 152 * 8);
}

ns_status_t plan_check_tune(const ns_tune_t& t)
{
    if (!(t.TM == 16 || t.TM == 32 || t.TM == 64)) return NS_ERR_INVALID;
    if (!(t.TK == 16 || t.TK == 32)) return NS_ERR_INVALID;
    if (t.chunk_nnz < 2 || t.chunk_nnz > 1024) return NS_ERR_INVALID;  // chunk buffers fit a CTA
    if (t.group != kExecWarps) return NS_ERR_INVALID;
    if (t.cost_tc < 0 || t.cost_res < 0 || t.absorb_cap < 0) return NS_ERR_INVALID;
    if (t.col_order != 0 && t.col_order != 1) return NS_ERR_INVALID;
    if (t.TN < 0 || (t.TN % 8) != 0) return NS_ERR_INVALID;
    if (t.l2_hints < 0 || t.l2_hints > 2) return NS_ERR_INVALID;
    if (t.reorder < 0 || (int64_t)t.reorder * t.TM > kReorderMaxRows) return NS_ERR_INVALID;
    return NS_OK;
}

// ---------------------------------------------------------------------------------------------
// orchestration
// ---------------------------------------------------------------------------------------------
static ns_status_t chunks_and_splits(Plan* P, const WindowResult* W, cudaStream_t s, int64_t* totals)
{
    const int64_t m = P->st.m;
    const int64_t n_rl = P->st.n_rl;
    const int64_t nc = P->st.n_chunks;
    const int64_t T = P->st.T;
    const int64_t Wn = P->tune.chunk_nnz;

    if (nc > 0) {
        if (W) {  // plans with windows; the all-residual plan wrote the chunk rows in its rows pass
            k_chunk_rows<<<grid_for(n_rl), 256, 0, s>>>(P->rl_start, n_rl, Wn, nc, P->chunk_k0);
            NS_LAUNCH_CHECK();
        }
        k_chunks<<<grid_for(nc + 1), 256, 0, s>>>(P->rl_start, P->rl_rows, P->res_rowptr, m, n_rl, T, Wn, nc,
                                                   P->chunk_b, P->chunk_k0, P->chunk_rec);
        NS_LAUNCH_CHECK();
    } else {
        NS_CUDA_TRY(cudaMemsetAsync(P->chunk_b, 0, sizeof(int32_t), s));
    }
    if (W && m > 0) {  // no split rows yet (the all-residual rows pass did this itself)
        k_fill_i32<<<grid_for(m), 256, 0, s>>>(P->row_split, m, -1);
        NS_LAUNCH_CHECK();
    }
    Arena tmp;
    int64_t* partial = nullptr;
    tmp.reserve(&partial, scan_partials(W ? n_rl : nc));
    NS_TRY(tmp.commit(s));
    if (n_rl > 0 && nc > 0 && W) {
        PieceInfo pi{P->rl_rows, P->rl_start, P->chunk_b, W->row_state, nc, Wn};
        PieceStore st{pi, P->row_split, P->split_row, P->split_np, P->split_slot, P->split_base};
        NS_TRY(device_scan<int64_t>(PieceLoad{pi}, st, n_rl, partial, totals, s));
    } else if (n_rl > 0 && nc > 0) {
        CutInfo ci{P->rl_rows, P->rl_start, P->chunk_k0, n_rl, nc, Wn};
        CutStore st{ci, P->row_split, P->split_row, P->split_np, P->split_slot, P->split_base};
        NS_TRY((device_scan<int64_t, CutLoad, CutStore, 1>(CutLoad{ci}, st, nc - 1, partial, totals, s)));
    }
    tmp.release(s);
    return NS_OK;
}

static ns_status_t work_queue(Plan* P, const WindowResult* W, cudaStream_t s)
{
    if (P->st.n_items <= 0) return NS_OK;
    Arena tmp;
    int32_t* hist = nullptr;
    tmp.reserve(&hist, bucket_hist_size(P->st.n_items));
    NS_TRY(tmp.commit(s));
    k_item_costs<<<grid_for(P->st.n_items), 256, 0, s>>>(P->chunk_b, P->st.n_chunks, P->tune.group,
                                                          P->st.n_dwin, W ? W->dcost : nullptr,
                                                          P->st.n_items, P->tune.cost_res, P->item_cost);
    NS_LAUNCH_CHECK();
    NS_TRY(bucket_sort_desc(CostKey{P->item_cost}, QueueEmit{P->queue}, P->st.n_items, hist, s));
    tmp.release(s);
    return NS_OK;
}

// Pinned host words for the planner's readbacks, one buffer per host thread (plans may be built
// from several threads at once).  A device-to-host copy into pageable memory returns only after
// the stream has drained, so pinned words let the host wait on an event instead while the GPU
// goes on with the work queue.  nullptr when pinned memory is unavailable.
constexpr int kReadbackWords = 24;  // 8 validation counters + 16 totals
static unsigned long long* readback_words()
{
    thread_local unsigned long long* buf = nullptr;
    thread_local bool tried = false;
    if (!tried) {
        tried = true;
        if (cudaHostAlloc(reinterpret_cast<void**>(&buf), kReadbackWords * sizeof(unsigned long long), 0) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            buf = nullptr;
        }
    }
    return buf;
}

static ns_status_t report_invalid(const unsigned long long* hc)
{
    set_error("invalid CSR: %llu out-of-range columns, %llu bad row pointers, %llu "
              "unsorted/duplicate positions",
              hc[kCnBadRange], hc[kCnBadPtr], hc[kCnDescents] - hc[kCnStartDescents]);
    return NS_ERR_INVALID;
}

static bool csr_ok(const unsigned long long* hc)
{
    return !hc[kCnBadRange] && !hc[kCnBadPtr] && hc[kCnDescents] == hc[kCnStartDescents];
}

ns_status_t plan_build(Plan* P, const ns_csr_t* A, int32_t K, ns_dtype_t dt, const ns_tune_t* tune,
                       cudaStream_t s)
{
    const int64_t m = A->m, n = A->n, nnz = A->nnz;
    P->tune = *tune;
    P->dtype = dt;
    P->K = K;
    P->st.m = m;
    P->st.n = n;
    P->st.nnz = nnz;
    P->st.K = K;
    P->st.b_bf16 = dt == NS_BF16;
    P->st.TM = tune->TM;
    P->st.TK = tune->TK;

    // ---- inputs on the device (a host CSR is copied; a device CSR is referenced) ----
    if (A->on_device) {
        P->rowptr = A->rowptr;
        P->colidx = A->colidx;
        P->vals = A->vals;
    } else {
        Arena in;
        int32_t *rp = nullptr, *ci = nullptr;
        float* v = nullptr;
        in.reserve(&rp, m + 1);
        in.reserve(&ci, nnz);
        in.reserve(&v, nnz);
        NS_TRY(in.commit(s));
        P->blocks.push_back(in.take());
        NS_CUDA_TRY(cudaMemcpyAsync(rp, A->rowptr, sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice, s));
        if (nnz) {
            NS_CUDA_TRY(cudaMemcpyAsync(ci, A->colidx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
            NS_CUDA_TRY(cudaMemcpyAsync(v, A->vals, sizeof(float) * nnz, cudaMemcpyHostToDevice, s));
        }
        P->rowptr = rp;
        P->colidx = ci;
        P->vals = v;
    }

    // ---- control block ----
    unsigned long long* counters = nullptr;  // validation counters
    int64_t* totals = nullptr;               // [0] packed split total, [1..] window totals
    {
        Arena a;
        a.reserve(&P->ctrl, 8);
        a.reserve(&counters, 8);
        a.reserve(&totals, 16);
        NS_TRY(a.commit(s));
        P->blocks.push_back(a.take());
        NS_CUDA_TRY(cudaMemsetAsync(P->ctrl, 0, sizeof(int32_t) * 8, s));
        NS_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * 8, s));
        NS_CUDA_TRY(cudaMemsetAsync(totals, 0, sizeof(int64_t) * 16, s));
    }

    // ---- a1: validation (the row half runs in the all-residual rows pass when there are no windows) ----
    const bool windows_on = tune->tau_tile != kTauInf && m > 0;
    if (nnz > 0) {
        if (((uintptr_t)P->colidx & 15) == 0)
            k_check_elems4<<<grid_for(nnz / 16 + 1), 256, 0, s>>>((const int4*)P->colidx, P->colidx, nnz,
                                                                 (int32_t)n, counters);
        else
            k_check_elems<<<grid_for(nnz), 256, 0, s>>>(P->colidx, nnz, (int32_t)n, counters);
        NS_LAUNCH_CHECK();
    }
    if (windows_on) {
        k_check_rows<<<grid_for(m + 1), 256, 0, s>>>(P->rowptr, P->colidx, (int32_t)m, nnz, counters);
        NS_LAUNCH_CHECK();
    }
    if (tune->tau_tile != kTauInf && (int64_t)tune->TM * K > 16384) {
        set_error("dense tiles need TM * K <= 16384 (TM=%d, K=%d); lower TM", tune->TM, K);
        return NS_ERR_UNSUPPORTED;
    }
    WindowResult win{};
    if (!windows_on) {
        // everything is residual: the residual CSR is A itself, every row in the list
        P->st.n_res = nnz;
        P->st.n_rl = m;
        P->st.T = nnz + m;
        P->res_rowptr = P->rowptr;
        P->res_col = P->colidx;
        P->res_val = P->vals;
    } else {
        // the window kernels read row contents: validation must pass first
        unsigned long long hc_own[8];
        unsigned long long* rb = readback_words();
        unsigned long long* hc = rb ? rb : hc_own;
        NS_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaStreamSynchronize(s));
        if (!csr_ok(hc)) return report_invalid(hc);
        NS_TRY(window_pass(P, &win, s));  // sets m_aic .. T and the residual / window arrays
    }
    const int64_t n_rl = P->st.n_rl;
    const int64_t T = P->st.T;
    const int64_t nc = T > 0 ? ceil_div(T, tune->chunk_nnz) : 0;
    P->st.n_chunks = nc;
    P->st.n_items = P->st.n_dwin + ceil_div(nc, tune->group);
    {
        Arena a;
        if (!windows_on) {
            a.reserve(&P->rl_rows, n_rl);
            a.reserve(&P->rl_start, n_rl + 1);
        }
        a.reserve(&P->chunk_b, nc + 1);
        a.reserve(&P->chunk_k0, nc);
        a.reserve(&P->chunk_rec, nc);
        a.reserve(&P->row_split, m);
        a.reserve(&P->split_row, n_rl);  // split rows are residual-list rows
        a.reserve(&P->split_np, n_rl);
        a.reserve(&P->split_slot, n_rl);
        a.reserve(&P->split_base, n_rl);
        a.reserve(&P->queue, P->st.n_items);
        a.reserve(&P->item_cost, P->st.n_items);
        NS_TRY(a.commit(s));
        P->blocks.push_back(a.take());
    }
    if (!windows_on) {
        k_rows_all_residual<<<grid_for(m + 1), 256, 0, s>>>(P->rowptr, P->colidx, (int32_t)m, nnz,
                                                            tune->chunk_nnz, nc, counters, P->rl_rows,
                                                            P->rl_start, P->row_split, P->chunk_k0);
        NS_LAUNCH_CHECK();
    }
    const WindowResult* W = windows_on ? &win : nullptr;
    NS_TRY(chunks_and_splits(P, W, s, totals));

    // ---- one readback (validation counters and split totals), overlapped with the work queue ----
    unsigned long long hbuf[kReadbackWords];
    unsigned long long* rb = readback_words();
    unsigned long long* hc = rb ? rb : hbuf;
    int64_t* ht = reinterpret_cast<int64_t*>(hc + 8);
    struct EventGuard {
        cudaEvent_t e = nullptr;
        ~EventGuard()
        {
            if (e) cudaEventDestroy(e);
        }
    } ev;
    if (rb) {
        NS_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaMemcpyAsync(ht, totals, sizeof(int64_t) * 16, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaEventCreateWithFlags(&ev.e, cudaEventDisableTiming));
        NS_CUDA_TRY(cudaEventRecord(ev.e, s));
    }
    NS_TRY(work_queue(P, W, s));

    // ---- hot B rows for the L2 policy (l2_hints == 2) ----
    if (tune->l2_hints == 2 && n > 0) {
        Arena h;
        int32_t* cnt = nullptr;
        unsigned long long* bins = nullptr;
        int32_t* th = nullptr;
        h.reserve(&cnt, n);
        h.reserve(&bins, 64);
        h.reserve(&th, 1);
        NS_TRY(h.commit(s));
        Arena hb;
        hb.reserve(&P->hot_bits, ceil_div(n, 32));
        NS_TRY(hb.commit(s));
        P->blocks.push_back(hb.take());
        NS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));
        NS_CUDA_TRY(cudaMemsetAsync(bins, 0, sizeof(unsigned long long) * 64, s));
        if (P->st.n_res > 0) {
            k_gather_counts<<<grid_for(P->st.n_res), 256, 0, s>>>(P->res_col, P->st.n_res, (int32_t)n, cnt);
            NS_LAUNCH_CHECK();
        }
        k_count_bins<<<grid_for(n), 256, 0, s>>>(cnt, (int32_t)n, bins);
        NS_LAUNCH_CHECK();
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, P->device);
        const int64_t row_bytes = (int64_t)K * (dt == NS_BF16 ? 2 : 4);
        const int64_t cap = (int64_t)(0.8 * (double)(l2 > 0 ? l2 : (96 << 20))) / row_bytes;
        k_hot_threshold<<<1, 32, 0, s>>>(bins, cap, th);
        NS_LAUNCH_CHECK();
        k_hot_bits<<<grid_for(n), 256, 0, s>>>(cnt, (int32_t)n, th, P->hot_bits);
        NS_LAUNCH_CHECK();
        h.release(s);
    }

    if (ev.e) {
        NS_CUDA_TRY(cudaEventSynchronize(ev.e));
    } else {
        NS_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaMemcpyAsync(ht, totals, sizeof(int64_t) * 16, cudaMemcpyDeviceToHost, s));
        NS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (win.temp.ptr) {
        NS_CUDA_TRY(cudaFreeAsync(win.temp.ptr, s));
        win.temp = DevBlock{};
    }
    if (!csr_ok(hc)) return report_invalid(hc);
    P->st.n_split = ht[0] >> 32;
    P->st.n_slots = ht[0] & 0xffffffffLL;

    // ---- execution scratch, sized exactly ----
    {
        Arena a;
        a.reserve(&P->slots, P->st.n_slots * (int64_t)K);
        a.reserve(&P->split_cnt, P->st.n_split);
        NS_TRY(a.commit(s));
        P->blocks.push_back(a.take());
        NS_CUDA_TRY(cudaMemsetAsync(P->split_cnt, 0, sizeof(int32_t) * (P->st.n_split > 0 ? P->st.n_split : 1), s));
    }
    return NS_OK;
}

}  // namespace ns
