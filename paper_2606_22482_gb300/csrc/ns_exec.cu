// ns_exec.cu -- the persistent execute kernel (Sections 5.1 and 7 of arXiv 2606.22482).
//
// One launch, grid = resident CTAs on every SM.  CTAs pull work items from one atomic ticket in
// the plan's cost order (heaviest first, Section 7 "row window list migration" in GPU form):
//   * dense item    -- a row window: sum over its dense tiles of A_tile * B[cols, :] on the
//                      tensor cores (matrix-engine execution model, Section 5.1), then the rows'
//                      absorbed residual on the CUDA cores, then the rows are stored;
//   * residual item -- kExecWarps merge-path chunks of the residual CSR, one per warp: gather B
//                      rows by column index and accumulate into output rows (vector-engine
//                      execution model, Section 5.1), several B rows per warp step when K is
//                      narrow (Section 7 "vector tiles merging").
// A row assembled from several pieces (cut by a chunk boundary, or shared by a dense window and
// residual chunks) is combined without atomics on C: each piece writes a partial to its slot,
// the last piece to arrive sums the slots in piece order and stores the row.  The result is
// therefore deterministic.
//
// L2 policy (Section 6.2.1 hot-B staging in GPU form): A's arrays and C are streamed with an
// evict-first policy, B rows are loaded with evict-last so that reused B rows stay in L2.
#include <type_traits>

#include "ns_internal.cuh"
#include "ns_ptx.cuh"

namespace ns {

// ---------------------------------------------------------------------------------------------
// memory helpers with L2 cache policies
// ---------------------------------------------------------------------------------------------
struct Policies {
    uint64_t first, last;
};

__device__ __forceinline__ Policies make_policies()
{
    Policies p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p.first));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p.last));
    return p;
}

template <bool HINT>
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p, uint64_t pol)
{
    int32_t v;
    if (HINT)
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
                     : "=r"(v) : "l"(p), "l"(pol));
    else
        v = __ldg(p);
    return v;
}

template <bool HINT>
__device__ __forceinline__ float ld_stream_f32(const float* p, uint64_t pol)
{
    float v;
    if (HINT)
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
                     : "=f"(v) : "l"(p), "l"(pol));
    else
        v = __ldg(p);
    return v;
}

// Four consecutive B elements as loaded: 16 B of FP32 or 8 B of BF16.  Rings of gathers keep
// this raw form and widen a vector only where it is used: a conversion next to its load would
// wait for the load there and leave one gather in flight instead of the ring's depth.
template <bool BF16>
using BRaw = std::conditional_t<BF16, uint2, float4>;

template <bool BF16, bool HINT>
__device__ __forceinline__ BRaw<BF16> ld_braw(const void* p, uint64_t pol)
{
    BRaw<BF16> r;
    if constexpr (!BF16) {
        if (HINT)
            asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                         : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p), "l"(pol));
        else
            r = __ldg(reinterpret_cast<const float4*>(p));
    } else {
        if (HINT)
            asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
                         : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
        else
            r = __ldg(reinterpret_cast<const uint2*>(p));
    }
    return r;
}

// 16 raw bytes (eight BF16 columns)
template <bool HINT>
__device__ __forceinline__ uint4 ld_b16(const void* p, uint64_t pol)
{
    uint4 r;
    if (HINT)
        asm volatile("ld.global.nc.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p), "l"(pol));
    else
        r = __ldg(reinterpret_cast<const uint4*>(p));
    return r;
}

template <bool BF16>
__device__ __forceinline__ BRaw<BF16> braw_zero()
{
    if constexpr (BF16) return make_uint2(0u, 0u);
    else return make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float4 widen(const float4& v) { return v; }
__device__ __forceinline__ float4 widen(const uint2& v)  // BF16 is the high half of an FP32
{
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                       __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
}

template <bool HINT>
__device__ __forceinline__ void st_c4(float* p, float4 v, uint64_t pol)
{
    if (HINT)
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;"
                     :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
    else
        *reinterpret_cast<float4*>(p) = v;
}

__device__ __forceinline__ float4 f4_fma(float a, float4 b, float4 c)
{
    c.x = fmaf(a, b.x, c.x);
    c.y = fmaf(a, b.y, c.y);
    c.z = fmaf(a, b.z, c.z);
    c.w = fmaf(a, b.w, c.w);
    return c;
}
__device__ __forceinline__ float4 f4_add(float4 a, float4 b)
{
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// ---------------------------------------------------------------------------------------------
// delivering one piece of an output row
//   L lanes (lane < L) hold VPL float4 vectors each: vector v = lane + L*q covers columns 4v..4v+3
// ---------------------------------------------------------------------------------------------
// `split`: the row's split id when the caller has it (>= -1), else kSplitUnknown (loaded here)
constexpr int32_t kSplitUnknown = -2;
template <int L, int VPL, bool HINT>
__device__ __forceinline__ void deliver_row(const ExecDesc& D, int32_t row, int32_t piece_of_chunk,
                                            bool dense_piece, const float4 (&acc)[VPL], int lane,
                                            uint64_t pol_first, int32_t split = kSplitUnknown)
{
    const int nv = D.K >> 2;
    const int32_t s = split != kSplitUnknown ? split : __ldg(D.row_split + row);
    float* crow = D.C + (int64_t)row * D.ldc;
    if (s < 0) {
        if (lane < L) {
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                int v = lane + L * q;
                if (v < nv) st_c4<HINT>(crow + 4 * v, acc[q], pol_first);
            }
        }
        return;
    }
    const int32_t np = __ldg(D.split_np + s);
    const int32_t piece = dense_piece ? 0 : piece_of_chunk - __ldg(D.split_base + s);
    float* slot0 = D.slots + (int64_t)__ldg(D.split_slot + s) * D.K;
    if (lane < L) {
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            int v = lane + L * q;
            if (v < nv) __stcg(reinterpret_cast<float4*>(slot0 + (int64_t)piece * D.K + 4 * v), acc[q]);
        }
    }
    __threadfence();
    __syncwarp();
    int old = 0;
    if (lane == 0) old = atomicAdd(D.split_cnt + s, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != np - 1) return;  // not the last piece
    __threadfence();
    if (lane < L) {
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            int v = lane + L * q;
            if (v < nv) {
                float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int p = 0; p < np; ++p)
                    sum = f4_add(sum, __ldcg(reinterpret_cast<const float4*>(slot0 + (int64_t)p * D.K + 4 * v)));
                st_c4<HINT>(crow + 4 * v, sum, pol_first);
            }
        }
    }
    if (lane == 0) atomicExch(D.split_cnt + s, 0);  // ready for the next launch
}

// ---------------------------------------------------------------------------------------------
// residual: acc += sum_{z in [z0, z1)} val[z] * B[col[z], :]
//   the warp's 32 lanes form G = 32/L groups; group g handles nonzeros g, g+G, ... of each batch
//   of 32 (vector tiles merging when K < 128), then the groups are summed with shuffles.
// ---------------------------------------------------------------------------------------------
template <int L, int VPL, bool BF16, bool HINT>
__device__ __forceinline__ void gather_accumulate(const ExecDesc& D, int64_t z0, int64_t z1,
                                                  float4 (&acc)[VPL], int lane, const Policies& pol)
{
    constexpr int G = 32 / L;
    const int g = lane / L, li = lane % L;
    const int nv = D.K >> 2;
    for (int64_t zb = z0; zb < z1; zb += 32) {
        const int cnt = (int)(z1 - zb < 32 ? z1 - zb : 32);
        int32_t mc = 0;
        float mv = 0.f;
        if (lane < cnt) {
            mc = ld_stream_i32<HINT>(D.res_col + zb + lane, pol.first);
            mv = ld_stream_f32<HINT>(D.res_val + zb + lane, pol.first);
            if ((unsigned)mc >= (unsigned)D.n) {  // guard: never gather outside B
                atomicOr(D.status, kStatusInternal);
                mc = 0;
                mv = 0.f;
            }
        }
        // 4 independent B rows in flight per lane
        for (int j0 = 0; j0 < cnt; j0 += 4 * G) {
            int32_t col[4];
            float val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int j = j0 + u * G + g;
                col[u] = __shfl_sync(0xffffffffu, mc, j & 31);
                val[u] = __shfl_sync(0xffffffffu, mv, j & 31);
                if (j >= cnt) val[u] = 0.f, col[u] = -1;
            }
            BRaw<BF16> b[4][VPL];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int v = li + L * q;
                    const int64_t off = (int64_t)col[u] * D.ldb + 4 * v;
                    b[u][q] = (col[u] >= 0 && v < nv)
                                  ? ld_braw<BF16, HINT>(static_cast<const unsigned char*>(D.B) +
                                                            off * (BF16 ? 2 : 4), pol.last)
                                  : braw_zero<BF16>();
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(val[u], widen(b[u][q]), acc[q]);
        }
    }
}

template <int L, int VPL>
__device__ __forceinline__ void group_reduce(float4 (&acc)[VPL])
{
#pragma unroll
    for (int o = L; o < 32; o <<= 1)
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
            acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
            acc[q].z += __shfl_xor_sync(0xffffffffu, acc[q].z, o);
            acc[q].w += __shfl_xor_sync(0xffffffffu, acc[q].w, o);
        }
}

// split-row delivery out of line (rare): keeps the inlined row flush of the stream path small
// PAIR: the lane holds vectors 2 lane and 2 lane + 1 (adjacent), otherwise lane and lane + 32
template <int VPL, bool HINT, bool PAIR = false>
__device__ __noinline__ void deliver_split_row(const ExecDesc& D, int32_t row, int32_t s, int32_t c,
                                               float4 a0, float4 a1, int lane, uint64_t pol_first)
{
    const int nv = D.K >> 2;
    const int32_t np = __ldg(D.split_np + s);
    const int32_t piece = c - __ldg(D.split_base + s);
    float* slot0 = D.slots + (int64_t)__ldg(D.split_slot + s) * D.K;
    const int v0 = PAIR ? 2 * lane : lane, v1 = PAIR ? 2 * lane + 1 : lane + 32;
    if (v0 < nv) __stcg(reinterpret_cast<float4*>(slot0 + (int64_t)piece * D.K + 4 * v0), a0);
    if (VPL > 1 && v1 < nv) __stcg(reinterpret_cast<float4*>(slot0 + (int64_t)piece * D.K + 4 * v1), a1);
    __threadfence();
    __syncwarp();
    int old = 0;
    if (lane == 0) old = atomicAdd(D.split_cnt + s, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != np - 1) return;
    __threadfence();
    float* crow = D.C + (int64_t)row * D.ldc;
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
        const int v = PAIR ? 2 * lane + q : lane + 32 * q;
        if (v < nv) {
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int p = 0; p < np; ++p)
                sum = f4_add(sum, __ldcg(reinterpret_cast<const float4*>(slot0 + (int64_t)p * D.K + 4 * v)));
            st_c4<HINT>(crow + 4 * v, sum, pol_first);
        }
    }
    if (lane == 0) atomicExch(D.split_cnt + s, 0);
}

// ---------------------------------------------------------------------------------------------
// residual chunks with K <= 256: decoded chunk in shared memory, gathers through a register ring
// ---------------------------------------------------------------------------------------------
// A chunk holds at most 3W/2 merge items (boundaries snap by less than W/2), so its rows and its
// nonzero stream fit in `cap` entries.  Per warp, shared memory holds the decoded chunk: the
// nonzeros as (column, value) pairs (padded by the ring depth), and per row its id, split id,
// first and past-last stream positions and first residual index.
constexpr int kRing = 8;  // gathered rows in flight per warp (K <= 128; 4 for K <= 256)

struct StageGeom {
    int cap;         // capacity of the chunk's stream and of its row arrays
    int rows_off;    // byte offset of the row arrays (after cap + kRing (col, val) pairs)
    int warp_bytes;  // shared memory of one warp, a multiple of 128
};

__host__ __device__ inline StageGeom stage_geom(int K, bool bf16, int W)
{
    (void)K;
    (void)bf16;
    StageGeom g;
    g.cap = ((3 * W) / 2 + 32 + 31) & ~31;
    g.rows_off = 8 * (g.cap + kRing);
    g.warp_bytes = (g.rows_off + 16 * (g.cap + 1) + 8 * g.cap + 127) & ~127;
    return g;
}

// the staged stream path serves K <= 256 (at most two 4-column vectors per lane)
__host__ __device__ inline bool staged_path(int L, int VPL) { return VPL <= 2; }

__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Row metadata of up to 32 consecutive residual-list rows of a chunk, one row per lane, with the
// rows' positions in the chunk's stream of nonzeros (rows clipped to the chunk's merge range).
struct RowWin {
    int64_t kb;     // first row of the window
    int64_t base;   // stream position of the window's first row
    int64_t total;  // stream position after the window
    int32_t row;    // original row id (-1 past the chunk's last row)
    int32_t split;  // split id of the row or -1
    int64_t zoff;   // residual index of the row's first nonzero inside the chunk
    int32_t n;      // nonzeros of the row inside the chunk
    int64_t cum;    // stream position of the row's first nonzero
};

__device__ __forceinline__ void load_win(const ExecDesc& D, RowWin& w, int64_t kb, int64_t base,
                                         int64_t kL, int64_t b0, int64_t b1, int lane)
{
    w.kb = kb;
    w.base = base;
    const int64_t k = kb + lane;
    int32_t n = 0;
    w.row = -1;
    w.split = -1;
    w.zoff = 0;
    if (k <= kL) {
        const int32_t i = __ldg(D.rl_rows + k);
        const int64_t s = __ldg(D.rl_start + k), e = __ldg(D.rl_start + k + 1);
        const int64_t xs = b0 > s ? b0 : s;
        const int64_t xe = b1 < e - 1 ? b1 : e - 1;
        n = xe > xs ? (int32_t)(xe - xs) : 0;
        if (i >= 0 && i < D.m) {
            w.row = i;
            w.split = __ldg(D.row_split + i);
            w.zoff = (int64_t)__ldg(D.res_rowptr + i) + (xs - s);
            if (w.zoff < 0 || w.zoff + n > D.n_res) n = 0, w.row = -2;  // guard: corrupt plan
        } else {
            w.row = -2;
        }
    }
    w.n = n;
    int32_t inc = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    w.cum = base + inc - n;
    w.total = base + __shfl_sync(0xffffffffu, inc, 31);
}

// The streamed inner loop.  FULL: every lane holds VPL whole vectors (K == 128 * VPL), so no
// per-lane width test; HOT: the planner's hot-row map picks each gather's L2 policy.
template <int VPL, bool BF16, bool HINT, bool FULL, bool HOT>
__device__ __forceinline__ void stream_rows(const ExecDesc& D, int32_t c, int lane, const int2* ent,
                                            int tot_pad, int nr, const int32_t* rrow,
                                            const int32_t* rsplit, const int32_t* rend,
                                            const Policies& pol)
{
    const int nv = D.K >> 2;
    constexpr int VB = BF16 ? 8 : 16;  // bytes of one 4-column vector
    const unsigned char* const Bl = reinterpret_cast<const unsigned char*>(D.B) + VB * lane;
    const uint32_t ldb_bytes = (uint32_t)(D.ldb * (BF16 ? 2 : 4));
    float* const Cp = D.C;
    const int64_t ldc = D.ldc;

    float4 acc[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int r = 0;
    int next_end = rend[0];
    auto flush = [&]() {  // deliver row r, move to row r + 1
        const int32_t i = rrow[r];
        const int32_t sp = rsplit[r];
        if (i >= 0) {
            if (sp < 0) {
                float* crow = Cp + (int64_t)i * ldc;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int v = lane + 32 * q;
                    if (FULL || v < nv) st_c4<HINT>(crow + 4 * v, acc[q], pol.first);
                }
            } else {
                deliver_split_row<VPL, HINT>(D, i, sp, c, acc[0], acc[VPL > 1 ? VPL - 1 : 0], lane, pol.first);
            }
        } else if (i == -2 && lane == 0) {
            atomicOr(D.status, kStatusInternal);
        }
#pragma unroll
        for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        ++r;
        next_end = rend[r];
    };

    constexpr int U = VPL == 1 ? kRing : kRing / 2;
    BRaw<BF16> b[U][VPL];
    float w[U];
    auto gather = [&](int2 e, BRaw<BF16> (&dst)[VPL], float& wv) {
        // padding entries point at a real row with value 0: no test needed here.  With the hot
        // map, bit 31 of the column id marks a hot row (set when the chunk was decoded).
        const uint32_t col = HOT ? ((uint32_t)e.x & 0x7fffffffu) : (uint32_t)e.x;
        const unsigned char* row = Bl + (size_t)col * ldb_bytes;
        uint64_t pl = pol.last;
        if (HOT) pl = e.x < 0 ? pol.last : pol.first;
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            if (FULL || lane + 32 * q < nv) dst[q] = ld_braw<BF16, HINT>(row + 32 * VB * q, pl);
            else dst[q] = braw_zero<BF16>();
        }
        wv = __int_as_float(e.y);
    };
#pragma unroll
    for (int u = 0; u < U; ++u) gather(ent[u], b[u], w[u]);
    for (int j0 = 0; j0 < tot_pad; j0 += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int P = j0 + u;
            while (P >= next_end) flush();
            const int2 e = ent[P + U];
#pragma unroll
            for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(w[u], widen(b[u][q]), acc[q]);
            gather(e, b[u], w[u]);
        }
    }
    while (r < nr) flush();  // rows ending at or after the last item (and the last row)
}

template <int VPL, bool BF16, bool HINT>
__device__ void residual_chunk_staged(const ExecDesc& D, int32_t c, int lane, unsigned char* wbase,
                                      const Policies& pol)
{
    const StageGeom G = stage_geom(D.K, BF16, D.chunk_nnz);
    const int64_t b0 = __ldg(D.chunk_b + c), b1 = __ldg(D.chunk_b + c + 1);
    const int64_t k0 = __ldg(D.chunk_k0 + c);
    // last row with a merge item in [b0, b1): the row holding b1 - 1
    int64_t kL = (c + 1 < D.n_chunks) ? (int64_t)__ldg(D.chunk_k0 + c + 1) : (int64_t)D.n_rl - 1;
    if (kL > k0 && (int64_t)__ldg(D.rl_start + kL) >= b1) --kL;
    const int nr = (int)(kL - k0 + 1);
    if (k0 < 0 || kL >= D.n_rl || kL < k0 || b1 <= b0 || nr > G.cap) {
        if (lane == 0) atomicOr(D.status, kStatusInternal);
        return;
    }
    int2* const ent = reinterpret_cast<int2*>(wbase);  // (col, value bits), cap + kRing
    int32_t* const rrow = reinterpret_cast<int32_t*>(wbase + G.rows_off);
    int32_t* const rsplit = rrow + (G.cap + 1);
    int32_t* const rbeg = rsplit + (G.cap + 1);
    int32_t* const rend = rbeg + (G.cap + 1);
    int64_t* const rzoff = reinterpret_cast<int64_t*>(rend + (G.cap + 1));

    // ---- decode the chunk's rows: ids, split ids, stream positions, first residual index ----
    int total = 0;
    {
        RowWin w;
        int64_t kb = k0, base = 0;
        for (;;) {
            load_win(D, w, kb, base, kL, b0, b1, lane);
            const int r = (int)(kb - k0) + lane;
            if (kb + lane <= kL) {
                rrow[r] = w.row;
                rsplit[r] = w.split;
                rbeg[r] = (int32_t)w.cum;
                rend[r] = (int32_t)(w.cum + w.n);
                rzoff[r] = w.zoff;
            }
            base = w.total;
            if (kb + 32 > kL) break;
            kb += 32;
        }
        total = (int)base;
        if (lane == 0) rend[nr] = 0x7fffffff;  // sentinel after the last row
    }
    if (total < 0 || total > G.cap) {
        if (lane == 0) atomicOr(D.status, kStatusInternal);
        return;
    }
    __syncwarp();
    // ---- the nonzero stream as (col, value) entries; every load issued before any store ----
    const int tot_pad = (total + kRing - 1) / kRing * kRing;
    int32_t last_col = 0;
    for (int P0 = 0; P0 < total; P0 += 128) {
        int32_t cc[4];
        float vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int P = P0 + 32 * u + lane;
            cc[u] = 0;
            vv[u] = 0.f;
            if (P < total) {
                int64_t z;
                if (D.rl_all) {
                    z = rzoff[0] + P;  // one contiguous residual range
                } else {             // the row holding P: largest r with rbeg[r] <= P
                    int lo = 0, hi = nr;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (rbeg[mid] <= P) lo = mid;
                        else hi = mid;
                    }
                    z = rzoff[lo] + (P - rbeg[lo]);
                }
                if (z >= 0 && z < D.n_res) {
                    cc[u] = ld_stream_i32<HINT>(D.res_col + z, pol.first);
                    vv[u] = ld_stream_f32<HINT>(D.res_val + z, pol.first);
                } else {
                    atomicOr(D.status, kStatusInternal);
                }
            }
        }
        uint32_t hw[4];  // hot-map words of the columns (independent loads as well)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int P = P0 + 32 * u + lane;
            if ((unsigned)cc[u] >= (unsigned)D.n) {  // guard: never gather outside B
                if (P < total) atomicOr(D.status, kStatusInternal);
                cc[u] = 0;
                vv[u] = 0.f;
            }
            hw[u] = (D.hot && P < total) ? __ldg(D.hot + (cc[u] >> 5)) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int P = P0 + 32 * u + lane;
            if (P < total) {
                const int32_t hotbit = (D.hot && ((hw[u] >> (cc[u] & 31)) & 1u)) ? (int32_t)0x80000000 : 0;
                ent[P] = make_int2(cc[u] | hotbit, __float_as_int(vv[u]));
            }
        }
    }
    __syncwarp();
    if (total > 0) last_col = ent[total - 1].x;
    // padding: the last real row again with value 0 (a cached load, no branch in the loop)
    for (int P = total + lane; P < tot_pad + kRing; P += 32) ent[P] = make_int2(last_col, 0);
    __syncwarp();

    const bool full = D.K == 128 * VPL;
    if (D.hot) {
        if (full) stream_rows<VPL, BF16, HINT, true, true>(D, c, lane, ent, tot_pad, nr, rrow, rsplit, rend, pol);
        else stream_rows<VPL, BF16, HINT, false, true>(D, c, lane, ent, tot_pad, nr, rrow, rsplit, rend, pol);
    } else {
        if (full) stream_rows<VPL, BF16, HINT, true, false>(D, c, lane, ent, tot_pad, nr, rrow, rsplit, rend, pol);
        else stream_rows<VPL, BF16, HINT, false, false>(D, c, lane, ent, tot_pad, nr, rrow, rsplit, rend, pol);
    }
}

// one merge-path chunk c of the residual (one warp)
template <int L, int VPL, bool BF16, bool HINT>
__device__ void residual_chunk(const ExecDesc& D, int32_t c, int lane, const Policies& pol)
{
    const int64_t b0 = __ldg(D.chunk_b + c), b1 = __ldg(D.chunk_b + c + 1);
    int64_t k = __ldg(D.chunk_k0 + c);
    int64_t x = b0;
    while (x < b1) {
        // guards: a corrupt plan sets the status word and stops instead of faulting
        if (k < 0 || k >= D.n_rl) {
            if (lane == 0) atomicOr(D.status, kStatusInternal);
            return;
        }
        const int32_t i = __ldg(D.rl_rows + k);
        const int64_t s = __ldg(D.rl_start + k), e = __ldg(D.rl_start + k + 1);
        const int64_t zrow = (i >= 0 && i < D.m) ? __ldg(D.res_rowptr + i) : -1;
        const int64_t xe = b1 < e - 1 ? b1 : e - 1;  // nonzero merge items of this row in chunk
        if (zrow < 0 || x < s || e <= s || zrow + (xe - s) > D.n_res) {
            if (lane == 0) atomicOr(D.status, kStatusInternal);
            return;
        }
        float4 acc[VPL];
#pragma unroll
        for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        gather_accumulate<L, VPL, BF16, HINT>(D, zrow + (x - s), zrow + (xe - s), acc, lane, pol);
        group_reduce<L, VPL>(acc);
        deliver_row<L, VPL, HINT>(D, i, c, false, acc, lane, pol.first);
        if (e - 1 < b1) {  // the row's end item is in this chunk: move on
            x = e;
            ++k;
        } else {
            x = b1;
        }
    }
}

}  // namespace ns

#include "ns_dense.cuh"
#include "ns_dense_tc.cuh"

namespace ns {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------------------------
// residual-only kernels are held to 128 registers (4 CTAs = 16 warps per SM, each with an 8-deep
// gather ring); kernels with the tensor-core item keep their registers for the accumulators
template <int L, int VPL, bool BF16, bool HINT, bool DENSE>
__global__ void __launch_bounds__(kExecThreads, DENSE ? 1 : 4) k_exec(const ExecDesc* __restrict__ descs,
                                                       const int32_t* __restrict__ queue,
                                                       const int32_t* __restrict__ queue_desc,
                                                       int64_t n_items, int32_t* ctrl,
                                                       const __grid_constant__ ExecDesc d0)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int32_t s_ticket;
    __shared__ int4 s_rowmeta[DENSE ? 64 : 1];  // a dense window's rows (TM <= 64)
    // BF16 plans with K <= 256 run their dense tiles on the 5th-generation tensor cores (tcgen05,
    // accumulator in tensor memory); other dense plans use the warp-level mma.sync item
    constexpr bool TC = DENSE && BF16 && VPL <= 2;
    __shared__ __align__(8) uint64_t s_tc_bars[TC ? kTcBars : 1];
    __shared__ uint32_t s_tc_tmem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Policies pol{0, 0};
    if (HINT) pol = make_policies();
    unsigned long long* const clk = descs ? nullptr : d0.class_clock;  // single-plan launches only
    if (clk && threadIdx.x == 0) atomicMin(clk, global_ns());
    if (DENSE) {
        TcState tcs{};
        if constexpr (TC) tc_setup(tcs, s_tc_bars, &s_tc_tmem);
        // phase 1: dense windows, one CTA each, taken in work-list order
        for (;;) {
            if (threadIdx.x == 0) s_ticket = atomicAdd(ctrl + 0, 1);
            __syncthreads();
            const int64_t t = s_ticket;
            __syncthreads();
            if (t >= n_items) break;
            const int32_t it = __ldg(queue + t);
            const ExecDesc& D = descs ? descs[queue_desc ? __ldg(queue_desc + t) : 0] : d0;
            if (it < D.n_dwin) {
                if constexpr (TC) {
                    const TcGeom G = tc_geom(D.K, D.TM, D.TK);
                    if (!tcs.ok) {
                        // an earlier bounded wait of this CTA gave up (status already set)
                    } else if (dynamic_smem_bytes() >= (uint32_t)G.total && tc_supported(D.K) && D.dtile_x &&
                               D.TM % 16 == 0 && D.TM <= 64 && D.TK % 16 == 0) {
                        const int32_t w = __ldg(D.dwin + it);
                        if (tc_window_product<HINT>(D, w, smem_raw, G, tcs, pol))
                            dense_deliver_rows<L, VPL, BF16, HINT>(D, it, w, reinterpret_cast<float*>(smem_raw + G.off_c),
                                                                  G.cs_stride, s_rowmeta, pol);
                    } else if (threadIdx.x == 0) {
                        atomicOr(D.status, kStatusInternal);  // guard: launch without the tile buffers
                    }
                } else {
                    if (dynamic_smem_bytes() >= (uint32_t)dense_geom(D.K, D.TM, D.TK, BF16).total)
                        dense_item<L, VPL, BF16, HINT>(D, it, smem_raw, s_rowmeta, pol);
                    else if (threadIdx.x == 0)
                        atomicOr(D.status, kStatusInternal);  // guard: launch without the tile buffers
                }
                if (clk && threadIdx.x == 0) atomicMax(clk + 1, global_ns());
            }
        }
        if constexpr (TC) tc_teardown(tcs, descs ? descs[0].status : d0.status);
    }
    // phase 2: residual chunks, one warp each, in work-list order (no CTA barrier)
    for (;;) {
        int64_t u = 0;
        if (lane == 0) u = atomicAdd(ctrl + 3, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        const int64_t t = u / kExecWarps;
        if (t >= n_items) break;
        const int32_t it = __ldg(queue + t);
        const ExecDesc& D = descs ? descs[queue_desc ? __ldg(queue_desc + t) : 0] : d0;
        if (it < D.n_dwin) continue;
        const int64_t c = (int64_t)(it - D.n_dwin) * kExecWarps + (u % kExecWarps);
        if (c >= D.n_chunks) continue;
        // K <= 256: the streamed path, which needs the shared memory the host sized for it; this
        // warp's slice follows the descriptor's chunk geometry (plans of one batched launch may
        // differ in W; nothing in it outlives a chunk)
        if constexpr (VPL <= 2) {
            const StageGeom SG = stage_geom(D.K, BF16, D.chunk_nnz);
            if (dynamic_smem_bytes() < (uint32_t)(kExecWarps * SG.warp_bytes)) {
                if (lane == 0) atomicOr(D.status, kStatusInternal);  // guard: misconfigured launch
                continue;
            }
            residual_chunk_staged<(VPL <= 2 ? VPL : 2), BF16, HINT>(D, (int32_t)c, lane,
                                                                    smem_raw + warp * SG.warp_bytes, pol);
        } else {
            residual_chunk<L, VPL, BF16, HINT>(D, (int32_t)c, lane, pol);
        }
        if (clk && lane == 0) atomicMax(clk + 2, global_ns());
    }
    // the last CTA out resets the tickets for the next launch (stream order makes it visible)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int done = atomicAdd(ctrl + 1, 1);
        if (done == (int)gridDim.x - 1) {
            atomicExch(ctrl + 0, 0);
            atomicExch(ctrl + 3, 0);
            atomicExch(ctrl + 1, 0);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// residual-only plans whose list is every row in order (tau_tile = inf): a chunk's nonzeros are
// one contiguous range of A and its rows are k0 .. kL themselves.  The lanes read column ids and
// values 32 at a time, two batches ahead, into a 4-batch ring of (col, value) pairs in this warp's
// shared memory (1 KB), which every step reads with one broadcast load; row ends and split ids
// come 32 rows at a time; B rows are gathered through a 4-deep register ring.  At 64 registers
// 8 CTAs (32 warps) fit on an SM: the gathers of many independent warps hide the latency spread
// of a power-law column stream better than deeper rings in fewer warps.
// ---------------------------------------------------------------------------------------------
constexpr int kCRing = 4;

// EPS: nonzeros per warp step (Section 7 "vector tiles merging"): the warp splits into EPS lane
// groups of G = 32 / EPS lanes, group g takes entry P + g of the step, and a row's partial sums
// are added across the groups when the row ends (K <= 4 G, so VPL = 1 when EPS > 1).
// FULL: every lane of a group holds VPL whole vectors (K == 4 G VPL), so no per-lane width test.
// HOT: the planner's hot-row map picks each gather's L2 policy; the map is read when a batch is
// fetched and its bit travels as bit 31 of the column id.
template <int VPL, int EPS, bool BF16, bool HINT, bool FULL, bool HOT, bool ASYNC>
__device__ __forceinline__ void contig_chunk(const ExecDesc& D, int32_t c, int lane, const Policies& pol,
                                             float4* park, int2* bat, float4* aring)
{
    // ASYNC (FP32, one 4-column vector per lane, one nonzero per step): the gathered rows land in
    // an 8-deep ring in shared memory through cp.async (each lane copies and later reads its own
    // 16 bytes, so no warp barrier), which doubles the rows in flight without spending registers;
    // otherwise a kCRing-deep register ring.
    constexpr int kR = ASYNC ? 8 : kCRing;  // ring depth (steps in flight)
    // PAIR (BF16, K <= 128): each lane gathers 8 adjacent columns (16 bytes, vectors 2 li and
    // 2 li + 1), so 16 lanes cover a row and the warp takes two nonzeros per step
    constexpr bool PAIR = BF16 && VPL == 2 && EPS == 2;
    static_assert(EPS == 1 || VPL == 1 || PAIR, "several nonzeros per step only for K <= 128");
    constexpr int G = 32 / EPS;
    const int g = lane / G, li = lane % G;
    const int4 h0 = __ldg(reinterpret_cast<const int4*>(D.chunk_rec + c));
    const int4 h1 = __ldg(reinterpret_cast<const int4*>(D.chunk_rec + c) + 1);
    const int32_t b0 = h0.x, k0 = h0.z, kL = h0.w, z0 = h1.x, total = h1.y;
    const int nr = kL - k0 + 1;
    if (k0 < 0 || kL >= D.n_rl || kL < k0 || h0.y <= b0 || total < 0 || z0 < 0 ||
        (int64_t)z0 + total > D.n_res) {
        if (lane == 0) atomicOr(D.status, kStatusInternal);  // guard: corrupt plan
        return;
    }
    const int nv = D.K >> 2;
    constexpr int VB = BF16 ? 8 : 16;  // bytes of one 4-column vector
    const unsigned char* const Bl = reinterpret_cast<const unsigned char*>(D.B) + (PAIR ? 2 : 1) * VB * li;
    auto vidx = [&](int q) { return PAIR ? 2 * li + q : li + 32 * q; };  // vector q of this lane
    const uint32_t ldb_bytes = (uint32_t)(D.ldb * (BF16 ? 2 : 4));

    // ---- batches of 32 (col, value) pairs; past the end: the last column again with value 0 ----
    const int32_t clast = total > 0 ? ld_stream_i32<HINT>(D.res_col + z0 + total - 1, pol.first) : 0;
    auto fetch = [&](int P0, int32_t& cc, float& vv) {
        const int P = P0 + lane;
        cc = clast;
        vv = 0.f;
        if (P < total) {
            cc = ld_stream_i32<HINT>(D.res_col + z0 + P, pol.first);
            vv = ld_stream_f32<HINT>(D.res_val + z0 + P, pol.first);
        }
        if ((unsigned)cc >= (unsigned)D.n) {  // guard: never gather outside B
            atomicOr(D.status, kStatusInternal);
            cc = 0;
            vv = 0.f;
        }
        if (HOT) cc |= (int32_t)(((__ldg(D.hot + (cc >> 5)) >> (cc & 31)) & 1u) << 31);
    };
    auto put = [&](int P0, int32_t cc, float vv) { bat[(P0 & 127) + lane] = make_int2(cc, __float_as_int(vv)); };
    int32_t cr;
    float vr;
    fetch(0, cr, vr);
    put(0, cr, vr);
    fetch(32, cr, vr);
    put(32, cr, vr);
    fetch(64, cr, vr);  // stored when batch 32 starts

    // lane j: stream end of row k0 + base + j (merge position of its end item, less b0 and the
    // end items of the rows before it) and its split id
    int32_t wend = 0x7fffffff, wsplit = -1;
    auto rows = [&](int base) {
        const int32_t k = k0 + base + lane;
        wend = 0x7fffffff;
        wsplit = -1;
        if (k <= kL) {
            wend = __ldg(D.rl_start + k + 1) - 1 - b0 - (k - k0);
            wsplit = __ldg(D.row_split + k);
        }
    };
    rows(0);
    __syncwarp();

    float4 acc[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    using Raw = std::conditional_t<PAIR, uint4, BRaw<BF16>>;
    Raw b[ASYNC ? 1 : kR][PAIR ? 1 : VPL];
    float w[kR];
    auto gather = [&](int2 e, int u) {
        const uint32_t col = HOT ? ((uint32_t)e.x & 0x7fffffffu) : (uint32_t)e.x;
        const unsigned char* row = Bl + (size_t)col * ldb_bytes;
        const uint64_t pl = HOT ? (e.x < 0 ? pol.last : pol.first) : pol.last;
        if constexpr (ASYNC) {
            cp_async16<HINT>(aring + u * 32 + lane, row, FULL || li < nv, pl);
            cp_async_commit();
        } else if constexpr (PAIR) {  // K a multiple of 8: both vectors valid or neither
            if (FULL || 2 * li < nv) b[u][0] = ld_b16<HINT>(row, pl);
            else b[u][0] = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                if (FULL || li + 32 * q < nv) b[u][q] = ld_braw<BF16, HINT>(row + 32 * VB * q, pl);
                else b[u][q] = braw_zero<BF16>();
            }
        }
        w[u] = __int_as_float(e.y);
    };
    auto bvec = [&](int u, int q) -> float4 {
        if constexpr (ASYNC) return aring[u * 32 + lane];
        else if constexpr (PAIR) {
            const uint4 v = b[u][0];
            return q == 0 ? widen(make_uint2(v.x, v.y)) : widen(make_uint2(v.z, v.w));
        } else return widen(b[u][q]);
    };
    // step u of a group covers entries P + u EPS + g; the ring's first kR steps
#pragma unroll
    for (int u = 0; u < kR; ++u) gather(bat[u * EPS + g], u);

    // Row ends inside the stream.  Only the chunk's first and last rows can be split (a middle
    // row lies inside the chunk's merge range, so no other chunk touches it); the last one ends
    // after the loop.  A split first row parks its partial sum in shared memory and is delivered
    // after the loop, so the loop has no call in it and the ring keeps its registers.
    int r = 0;
    bool parked = false;
    int next_end = __shfl_sync(0xffffffffu, wend, 0);
    auto reduce_groups = [&]() {  // every group ends up with the row's full sum
#pragma unroll
        for (int o = G; o < 32; o <<= 1)
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
                acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
                acc[q].z += __shfl_xor_sync(0xffffffffu, acc[q].z, o);
                acc[q].w += __shfl_xor_sync(0xffffffffu, acc[q].w, o);
            }
    };
    auto store_row = [&]() {  // group 0 stores
        float* crow = D.C + (int64_t)(k0 + r) * D.ldc;
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            const int v = vidx(q);
            if (g == 0 && (FULL || v < nv)) st_c4<HINT>(crow + 4 * v, acc[q], pol.first);
        }
    };
    auto advance = [&]() {
#pragma unroll
        for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        ++r;
        if ((r & 31) == 0) rows(r);
        next_end = __shfl_sync(0xffffffffu, wend, r & 31);
    };
    auto flush = [&]() {  // inside the loop
        const int32_t sp = __shfl_sync(0xffffffffu, wsplit, r & 31);
        if (EPS > 1) reduce_groups();
        if (sp < 0) {
            store_row();
        } else if (r == 0) {
#pragma unroll
            for (int q = 0; q < VPL; ++q) park[32 * q + lane] = acc[q];
            parked = true;
        } else if (lane == 0) {
            atomicOr(D.status, kStatusInternal);  // guard: a middle row marked split
        }
        advance();
    };
    // One step: entries P .. P + EPS - 1 (ring slot u) accumulated, then the slot gathers the
    // entries kCRing steps ahead.  A row that ends inside the step takes the groups before its end;
    // rows ending at or after the chunk's last nonzero are left to the end.  TAIL: the step may
    // reach past the last nonzero (those groups add nothing).
    auto step = [&](int P, int u, const int2* e1, auto tail) {
        constexpr bool TAIL = decltype(tail)::value;
        const int mine = P + g;
        if constexpr (ASYNC) cp_async_wait<kR - 1>();  // this step's row has landed
        if (next_end >= P + EPS || next_end >= total) {
            if (!TAIL || mine < total) {
#pragma unroll
                for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(w[u], bvec(u, q), acc[q]);
            }
        } else {
            int from = P;
            while (next_end < P + EPS && next_end < total) {
                if (mine >= from && mine < next_end) {
#pragma unroll
                    for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(w[u], bvec(u, q), acc[q]);
                }
                if (next_end > from) from = next_end;
                flush();
            }
            if (mine >= from && (!TAIL || mine < total)) {
#pragma unroll
                for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(w[u], bvec(u, q), acc[q]);
            }
        }
        gather(e1[u * EPS + g], u);
    };

    constexpr int GS = kR * EPS;  // entries per group of steps (divides the batch of 32)
    int P = 0;
    for (; P + GS <= total; P += GS) {
        if ((P & 31) == 0 && P > 0) {  // batch P + 32 into the ring, batch P + 64 requested
            put(P + 32, cr, vr);
            __syncwarp();
            fetch(P + 64, cr, vr);
        }
        const int2* e1 = bat + ((P + GS) & 127);  // entries P + GS .. P + 2 GS - 1 (GS divides 128)
#pragma unroll
        for (int u = 0; u < kR; ++u) step(P + u * EPS, u, e1, std::false_type{});
    }
    if (P < total) {  // the last partial group (its entries are already in the ring)
        if ((P & 31) == 0 && P > 0) {
            put(P + 32, cr, vr);
            __syncwarp();
        }
        const int2* e1 = bat + ((P + GS) & 127);
#pragma unroll
        for (int u = 0; u < kR; ++u)
            if (P + u * EPS < total) step(P + u * EPS, u, e1, std::true_type{});
    }
    if (parked) {
        float4 p[VPL];
#pragma unroll
        for (int q = 0; q < VPL; ++q) p[q] = park[32 * q + lane];
        deliver_split_row<VPL, HINT, PAIR>(D, k0, __ldg(D.row_split + k0), c, p[0], p[VPL > 1 ? VPL - 1 : 0],
                                           lane, pol.first);
    }
    while (r < nr) {  // rows ending at or after the last nonzero (and the last row)
        const int32_t sp = __shfl_sync(0xffffffffu, wsplit, r & 31);
        if (EPS > 1) reduce_groups();
        if (sp < 0) store_row();
        else deliver_split_row<VPL, HINT, PAIR>(D, k0 + r, sp, c, acc[0], acc[VPL > 1 ? VPL - 1 : 0], lane,
                                                pol.first);
        advance();
    }
    if constexpr (ASYNC) cp_async_wait<0>();  // the look-ahead copies land before the ring is reused
    __syncwarp();  // the batch ring is reused by this warp's next chunk
}

// SMEM_RING: the FP32 one-vector form may stage its gathers in the shared-memory cp.async ring
// (pays off when the gathered rows come from DRAM; when B sits in L2 the register ring is faster).
// HOTMAP: that ring form is built twice, with and without the planner's hot-row map, so the common
// build carries no registers for the map (the map is a cache hint only: a build without it ignores
// it and computes the same C); the register-ring forms read the map whenever a plan has one.
template <int VPL, int EPS, bool BF16, bool HINT, bool SMEM_RING = true, bool HOTMAP = false>
__global__ void __launch_bounds__(kExecThreads, VPL == 1 ? 8 : (EPS == 2 ? 6 : 5)) k_exec_contig(
    const ExecDesc* __restrict__ descs, const int32_t* __restrict__ queue,
    const int32_t* __restrict__ queue_desc, int64_t n_items, int32_t* ctrl,
    const __grid_constant__ ExecDesc d0)
{
    constexpr bool ASYNC = SMEM_RING && VPL == 1 && EPS == 1 && !BF16;
    constexpr bool READ_HOT = HINT && (!ASYNC || HOTMAP);
    __shared__ float4 s_park[kExecWarps * 32 * VPL];  // one parked partial row per warp
    __shared__ float4 s_aring[ASYNC ? kExecWarps * 8 * 32 : 1];
    __shared__ int2 s_bat[kExecWarps * 128];          // per warp: 4 batches of 32 (col, value)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* const park = s_park + warp * 32 * VPL;
    int2* const bat = s_bat + warp * 128;
    Policies pol{0, 0};
    if (HINT) pol = make_policies();
    unsigned long long* const clk = descs ? nullptr : d0.class_clock;  // single-plan launches only
    if (clk && threadIdx.x == 0) atomicMin(clk, global_ns());
    for (;;) {
        int64_t u = 0;
        if (lane == 0) u = atomicAdd(ctrl + 3, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        const int64_t t = u / kExecWarps;
        if (t >= n_items) break;
        const int32_t it = __ldg(queue + t);
        const ExecDesc& D = descs ? descs[queue_desc ? __ldg(queue_desc + t) : 0] : d0;
        if (it < D.n_dwin) continue;
        const int64_t c = (int64_t)(it - D.n_dwin) * kExecWarps + (u % kExecWarps);
        if (c >= D.n_chunks) continue;
        if (!D.rl_all) {  // guard: launched for a plan without a contiguous residual stream
            if (lane == 0) atomicOr(D.status, kStatusInternal);
            continue;
        }
        const bool full = D.K == 128 / EPS * VPL;
        float4* const aring = s_aring + (ASYNC ? (threadIdx.x >> 5) * 8 * 32 : 0);
        if (READ_HOT && D.hot) {
            if (full) contig_chunk<VPL, EPS, BF16, HINT, true, HINT, ASYNC>(D, (int32_t)c, lane, pol, park, bat, aring);
            else contig_chunk<VPL, EPS, BF16, HINT, false, HINT, ASYNC>(D, (int32_t)c, lane, pol, park, bat, aring);
        } else {
            if (full) contig_chunk<VPL, EPS, BF16, HINT, true, false, ASYNC>(D, (int32_t)c, lane, pol, park, bat, aring);
            else contig_chunk<VPL, EPS, BF16, HINT, false, false, ASYNC>(D, (int32_t)c, lane, pol, park, bat, aring);
        }
        if (clk && lane == 0) atomicMax(clk + 2, global_ns());
    }
    // the last CTA out resets the tickets for the next launch (stream order makes it visible)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int done = atomicAdd(ctrl + 1, 1);
        if (done == (int)gridDim.x - 1) {
            atomicExch(ctrl + 0, 0);
            atomicExch(ctrl + 3, 0);
            atomicExch(ctrl + 1, 0);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
// the residual list is every row in order and A itself is the residual (no window pass ran):
// a chunk's nonzeros are one contiguous range of A and its rows are k0 .. kL
bool plan_contig(const Plan* P)
{
    return P->tune.tau_tile == kTauInf && P->st.n_dwin == 0 && P->st.n_rl == P->st.m;
}

void fill_desc(const Plan* P, const void* B, int64_t ldb, float* C, int64_t ldc, ExecDesc* d)
{
    *d = ExecDesc{};
    d->res_rowptr = P->res_rowptr;
    d->res_col = P->res_col;
    d->res_val = P->res_val;
    d->rl_rows = P->rl_rows;
    d->rl_start = P->rl_start;
    d->chunk_b = P->chunk_b;
    d->chunk_k0 = P->chunk_k0;
    d->chunk_rec = P->chunk_rec;
    d->n_chunks = (int32_t)P->st.n_chunks;
    d->n_dwin = (int32_t)P->st.n_dwin;
    d->win_rows = P->win_rows;
    d->win_dptr = P->win_dptr;
    d->dwin = P->dwin;
    d->dwin_absorb = P->dwin_absorb;
    d->dtile_cols = P->dtile_cols;
    d->dtile_bits = P->dtile_bits;
    d->dtile_voff = P->dtile_voff;
    d->dtile_vals = P->dtile_vals;
    d->dtile_x = P->dtile_x;
    d->row_split = P->row_split;
    d->split_np = P->split_np;
    d->split_slot = P->split_slot;
    d->split_base = P->split_base;
    d->slots = P->slots;
    d->split_cnt = P->split_cnt;
    d->B = B;
    d->C = C;
    d->ldb = ldb;
    d->ldc = ldc;
    d->K = P->K;
    d->b_bf16 = P->dtype == NS_BF16;
    d->TM = P->tune.TM;
    d->TK = P->tune.TK;
    d->group = P->tune.group;
    d->l2_hints = P->tune.l2_hints;
    d->m = (int32_t)P->st.m;
    d->n = (int32_t)P->st.n;
    d->n_rl = (int32_t)P->st.n_rl;
    d->n_res = (int32_t)P->st.n_res;
    d->rl_all = plan_contig(P) ? 1 : 0;
    d->hot = P->hot_bits;
    d->chunk_nnz = P->tune.chunk_nnz;
    d->status = P->ctrl + 2;
    d->class_clock = P->class_clock;
}

typedef void (*ExecKernel)(const ExecDesc*, const int32_t*, const int32_t*, int64_t, int32_t*, ExecDesc);

template <bool BF16, bool HINT, bool DENSE>
static ExecKernel pick_kernel(int K)
{
    const int nv = K / 4;
    if (nv <= 2) return k_exec<2, 1, BF16, HINT, DENSE>;
    if (nv <= 4) return k_exec<4, 1, BF16, HINT, DENSE>;
    if (nv <= 8) return k_exec<8, 1, BF16, HINT, DENSE>;
    if (nv <= 16) return k_exec<16, 1, BF16, HINT, DENSE>;
    if (nv <= 32) return k_exec<32, 1, BF16, HINT, DENSE>;
    if (nv <= 64) return k_exec<32, 2, BF16, HINT, DENSE>;
    if (nv <= 128) return k_exec<32, 4, BF16, HINT, DENSE>;
    return k_exec<32, 8, BF16, HINT, DENSE>;
}

// nonzeros per warp step: as many lane groups as the K/4 vectors of a row leave room for
template <bool BF16, bool HINT>
static ExecKernel pick_contig(int K, bool b_in_l2, bool hot)
{
    if (K <= 32) return k_exec_contig<1, 4, BF16, HINT>;
    if (K <= 64) return k_exec_contig<1, 2, BF16, HINT>;
    if constexpr (BF16) {
        if (K <= 128) return k_exec_contig<2, 2, BF16, HINT>;  // 8 columns a lane, 2 nonzeros a step
    } else {
        if (K <= 128 && b_in_l2) return k_exec_contig<1, 1, BF16, HINT, false>;
    }
    if (K <= 128) {
        if constexpr (!BF16 && HINT)
            if (hot) return k_exec_contig<1, 1, BF16, HINT, true, true>;
        return k_exec_contig<1, 1, BF16, HINT>;
    }
    return k_exec_contig<2, 1, BF16, HINT>;
}

// contig: 0, or a residual-only launch whose plans all have a contiguous residual stream
// (K <= 256): kContig, kContigBInL2 when B fits comfortably in L2, or kContigHot for a single
// plan with a hot-row map
static ExecKernel select_kernel(int K, bool bf16, bool hint, bool dense, int contig)
{
    if (contig && !dense && K <= 256) {
        const bool in_l2 = contig == kContigBInL2, hot = contig == kContigHot;
        if (bf16) return hint ? pick_contig<true, true>(K, in_l2, hot) : pick_contig<true, false>(K, in_l2, hot);
        return hint ? pick_contig<false, true>(K, in_l2, hot) : pick_contig<false, false>(K, in_l2, hot);
    }
    if (bf16) {
        if (hint) return dense ? pick_kernel<true, true, true>(K) : pick_kernel<true, true, false>(K);
        return dense ? pick_kernel<true, false, true>(K) : pick_kernel<true, false, false>(K);
    }
    if (hint) return dense ? pick_kernel<false, true, true>(K) : pick_kernel<false, true, false>(K);
    return dense ? pick_kernel<false, false, true>(K) : pick_kernel<false, false, false>(K);
}

int64_t l2_bytes(int device)
{
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 0;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device) != cudaSuccess || v <= 0) v = 1;
        cached[device] = v;
    }
    return cached[device];
}

int num_sms(int device)
{
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 148;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
        cached[device] = v;
    }
    return cached[device];
}

// dynamic shared memory of one execute CTA: the dense item's tiles (phase 1) or the residual
// warps' staging rings (phase 2), whichever is larger
static size_t exec_smem_bytes(int K, int TM, int TK, bool bf16, bool dense, int W, int contig)
{
    if (contig && !dense && K <= 256) return 0;  // the contiguous-stream kernel keeps no staging
    // (L, VPL) exactly as pick_kernel chooses the instantiation
    const int nv = K / 4;
    const int L = nv <= 2 ? 2 : (nv <= 4 ? 4 : (nv <= 8 ? 8 : (nv <= 16 ? 16 : 32)));
    const int VPL = nv <= 32 ? 1 : (nv <= 64 ? 2 : (nv <= 128 ? 4 : 8));
    size_t b = staged_path(L, VPL) ? (size_t)kExecWarps * stage_geom(K, bf16, W).warp_bytes : 0;
    // (chunk_nnz <= 1024 keeps this within the 227 KB a CTA may use)
    if (dense) {
        // BF16 with K <= 256: the tensor-core (tcgen05) item's ring; otherwise the mma.sync item
        size_t d = (bf16 && VPL <= 2) ? (size_t)tc_geom(K, TM, TK).total : dense_smem_bytes(K, TM, TK, bf16);
        if (d > b) b = d;
    }
    return b;
}

// Kernel attributes and the persistent grid (resident CTAs on every SM, at most n_items).
// Must run outside stream capture.
ns_status_t exec_prepare(int64_t n_items, int K, int TM, int TK, bool bf16, bool hint, bool dense,
                         int* grid_out, int W, int contig)
{
    ExecKernel kern = select_kernel(K, bf16, hint, dense, contig);
    const size_t smem = exec_smem_bytes(K, TM, TK, bf16, dense, W, contig);
    if (smem > 48 * 1024) NS_TRY(dense_prepare(reinterpret_cast<const void*>(kern), smem));
    int per_sm = 0;
    NS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kExecThreads, smem));
    int dev = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
    if (smem > 48 * 1024) {
        // The query may assume a smaller shared-memory carve-out than the SM has; the persistent
        // grid is sized from the SM's capacity (CTAs that do not fit simply start later).
        int sm_smem = 0, regs_sm = 0;
        cudaFuncAttributes fa{};
        NS_CUDA_TRY(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        NS_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
        NS_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        const int by_smem = sm_smem / (int)(smem + fa.sharedSizeBytes + 1024);
        const int by_regs = fa.numRegs > 0 ? regs_sm / (fa.numRegs * kExecThreads) : by_smem;
        const int fit = by_smem < by_regs ? by_smem : by_regs;
        if (fit > per_sm) per_sm = fit;
    }
    // the tensor-core item allocates tensor memory per CTA: no more CTAs per SM than it holds
    if (dense && bf16 && tc_supported(K) && per_sm > kTcCtasPerSm) per_sm = kTcCtasPerSm;
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)per_sm * num_sms(dev);
    if (g > n_items) g = n_items;
    *grid_out = (int)(g > 0 ? g : 1);
    return NS_OK;
}

// One persistent launch over `n_items` work items.  queue[t] is an item id of descriptor
// queue_desc[t] (descriptor 0 when queue_desc is NULL).  All descriptors share K, dtype and L2
// policy; `dense` selects the kernel with the tensor-core item compiled in.  *grid_cache keeps
// the occupancy-derived grid between launches (0 = compute).
ns_status_t exec_launch(const ExecDesc* descs, const int32_t* queue, const int32_t* queue_desc,
                        int64_t n_items, int32_t* ctrl, int K, int TM, int TK, bool bf16, bool hint,
                        bool dense, int* grid_cache, cudaStream_t s, const ExecDesc* d0, int W,
                        int contig)
{
    ExecKernel kern = select_kernel(K, bf16, hint, dense, contig);
    const size_t smem = exec_smem_bytes(K, TM, TK, bf16, dense, W, contig);
    int grid = grid_cache ? *grid_cache : 0;
    if (grid == 0) NS_TRY(exec_prepare(n_items, K, TM, TK, bf16, hint, dense, &grid, W, contig));
    if (grid_cache) *grid_cache = grid;
    if (n_items == 0) return NS_OK;
    ExecDesc dv{};
    if (d0) dv = *d0;
    kern<<<grid, kExecThreads, smem, s>>>(d0 ? nullptr : descs, queue, queue_desc, n_items, ctrl, dv);
    NS_LAUNCH_CHECK();
    return NS_OK;
}

// single plan: the descriptor travels as a kernel parameter (no upload per launch)
ns_status_t exec_launch_plan(Plan* P, cudaStream_t s)
{
    const int K = P->desc_host.K;  // the column slice of this launch
    int* gc = K == P->K ? &P->exec_grid : &P->exec_grid_slice;
    if (K != P->K && P->exec_grid_slice_K != K) {
        P->exec_grid_slice = 0;
        P->exec_grid_slice_K = K;
    }
    int contig = 0;
    if (plan_contig(P)) {
        // B (this slice of it) within half of L2: the gathers hit L2, keep them in registers
        const int64_t b_bytes = P->st.n * (int64_t)K * (P->dtype == NS_BF16 ? 2 : 4);
        contig = 2 * b_bytes <= l2_bytes(P->device) ? kContigBInL2 : (P->hot_bits ? kContigHot : kContig);
    }
    return exec_launch(nullptr, P->queue, nullptr, P->st.n_items, P->ctrl, K, P->tune.TM,
                       P->tune.TK, P->dtype == NS_BF16, P->tune.l2_hints != 0, P->st.n_dwin > 0,
                       gc, s, &P->desc_host, P->tune.chunk_nnz, contig);
}

}  // namespace ns
