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
#include "ns_internal.cuh"

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

// four consecutive B elements (16 B of FP32 or 8 B of BF16) widened to float
template <bool BF16, bool HINT>
__device__ __forceinline__ float4 ld_b4(const void* B, int64_t off, uint64_t pol)
{
    float4 r;
    if (!BF16) {
        const float* p = reinterpret_cast<const float*>(B) + off;
        if (HINT)
            asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                         : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p), "l"(pol));
        else
            r = __ldg(reinterpret_cast<const float4*>(p));
    } else {
        const uint16_t* p = reinterpret_cast<const uint16_t*>(B) + off;
        uint32_t a, b;
        if (HINT)
            asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
                         : "=r"(a), "=r"(b) : "l"(p), "l"(pol));
        else {
            uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
            a = u.x;
            b = u.y;
        }
        r.x = __uint_as_float(a << 16);
        r.y = __uint_as_float(a & 0xffff0000u);
        r.z = __uint_as_float(b << 16);
        r.w = __uint_as_float(b & 0xffff0000u);
    }
    return r;
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
template <int L, int VPL, bool HINT>
__device__ __forceinline__ void deliver_row(const ExecDesc& D, int32_t row, int32_t piece_of_chunk,
                                            bool dense_piece, const float4 (&acc)[VPL], int lane,
                                            uint64_t pol_first)
{
    const int nv = D.K >> 2;
    const int32_t s = __ldg(D.row_split + row);
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
            float4 b[4][VPL];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    int v = li + L * q;
                    b[u][q] = (col[u] >= 0 && v < nv)
                                  ? ld_b4<BF16, HINT>(D.B, (int64_t)col[u] * D.ldb + 4 * v, pol.last)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(val[u], b[u][q], acc[q]);
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
template <int VPL, bool HINT>
__device__ __noinline__ void deliver_split_row(const ExecDesc& D, int32_t row, int32_t s, int32_t c,
                                               float4 a0, float4 a1, int lane, uint64_t pol_first)
{
    const int nv = D.K >> 2;
    const int32_t np = __ldg(D.split_np + s);
    const int32_t piece = c - __ldg(D.split_base + s);
    float* slot0 = D.slots + (int64_t)__ldg(D.split_slot + s) * D.K;
    if (lane < nv) __stcg(reinterpret_cast<float4*>(slot0 + (int64_t)piece * D.K + 4 * lane), a0);
    if (VPL > 1 && lane + 32 < nv)
        __stcg(reinterpret_cast<float4*>(slot0 + (int64_t)piece * D.K + 4 * (lane + 32)), a1);
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
        const int v = lane + 32 * q;
        if (v < nv) {
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int p = 0; p < np; ++p)
                sum = f4_add(sum, __ldcg(reinterpret_cast<const float4*>(slot0 + (int64_t)p * D.K + 4 * v)));
            st_c4<HINT>(crow + 4 * v, sum, pol_first);
        }
    }
    if (lane == 0) atomicExch(D.split_cnt + s, 0);
}

// Residual chunk when the residual list is every row in order (no dense windows) and K >= 128
// (one nonzero per warp step, 32 lanes x 4 columns x VPL).  The chunk's nonzeros are then one
// contiguous stream: (col, val) batches of 32 are loaded one batch ahead, row ends and split ids
// of 32 rows at a time, and U gathered B rows stay in flight across row boundaries.  Removes the
// per-row chain of dependent loads (row pointer -> column ids -> B row).
template <int VPL, bool BF16, bool HINT>
__device__ void residual_chunk_stream(const ExecDesc& D, int32_t c, int lane, const Policies& pol)
{
    constexpr int U = VPL == 1 ? 8 : 4;
    const int nv = D.K >> 2;
    const int64_t b0 = __ldg(D.chunk_b + c), b1 = __ldg(D.chunk_b + c + 1);
    const int64_t k0 = __ldg(D.chunk_k0 + c);
    // last row with a merge item in [b0, b1): the row holding b1 - 1
    int64_t kL = (c + 1 < D.n_chunks) ? (int64_t)__ldg(D.chunk_k0 + c + 1) : (int64_t)D.n_rl - 1;
    if (kL > k0 && (int64_t)__ldg(D.res_rowptr + kL) + kL >= b1) --kL;
    const int64_t zA = b0 - k0;                              // first nonzero of the chunk
    const int64_t eL = __ldg(D.res_rowptr + kL + 1);
    const int64_t zZ = (eL + kL >= b1) ? b1 - kL : eL;       // end of the chunk's nonzeros
    if (k0 < 0 || kL >= D.n_rl || zA < 0 || zZ > D.n_res || zA > zZ + 1) {
        if (lane == 0) atomicOr(D.status, kStatusInternal);
        return;
    }
    int64_t kb = k0;  // first row of the lanes' metadata window
    int32_t my_end = kb + lane <= kL ? __ldg(D.res_rowptr + kb + lane + 1) : 0x7fffffff;
    int32_t my_split = kb + lane <= kL ? __ldg(D.row_split + kb + lane) : -1;
    int64_t k = k0;
    int64_t rend = __shfl_sync(0xffffffffu, my_end, 0);
    float4 acc[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    // deliver row k (its nonzeros in this chunk are summed in acc) and move to row k + 1
    auto flush = [&]() {
        const int32_t s = __shfl_sync(0xffffffffu, my_split, (int)(k - kb));
        if (s < 0) {
            float* crow = D.C + k * D.ldc;
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                const int v = lane + 32 * q;
                if (v < nv) st_c4<HINT>(crow + 4 * v, acc[q], pol.first);
            }
        } else {
            deliver_split_row<VPL, HINT>(D, (int32_t)k, s, c, acc[0], acc[VPL > 1 ? VPL - 1 : 0], lane,
                                         pol.first);
        }
#pragma unroll
        for (int q = 0; q < VPL; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        ++k;
        if (k - kb == 32) {
            kb = k;
            my_end = kb + lane <= kL ? __ldg(D.res_rowptr + kb + lane + 1) : 0x7fffffff;
            my_split = kb + lane <= kL ? __ldg(D.row_split + kb + lane) : -1;
        }
        rend = __shfl_sync(0xffffffffu, my_end, (int)(k - kb));
    };

    int32_t mc = 0, nc_ = 0;
    float mv = 0.f, nv_ = 0.f;
    if (zA + lane < zZ) {
        mc = ld_stream_i32<HINT>(D.res_col + zA + lane, pol.first);
        mv = ld_stream_f32<HINT>(D.res_val + zA + lane, pol.first);
    }
    for (int64_t zb = zA; zb < zZ; zb += 32) {
        const int cnt = (int)(zZ - zb < 32 ? zZ - zb : 32);
        // next batch of column ids and values, one batch ahead
        if (zb + 32 + lane < zZ) {
            nc_ = ld_stream_i32<HINT>(D.res_col + zb + 32 + lane, pol.first);
            nv_ = ld_stream_f32<HINT>(D.res_val + zb + 32 + lane, pol.first);
        }
        if (lane < cnt && (unsigned)mc >= (unsigned)D.n) {  // guard: never gather outside B
            atomicOr(D.status, kStatusInternal);
            mc = 0;
            mv = 0.f;
        }
        for (int j0 = 0; j0 < cnt; j0 += U) {
            float4 b[U][VPL];
            float val[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                const int32_t col = __shfl_sync(0xffffffffu, mc, j & 31);
                val[u] = __shfl_sync(0xffffffffu, mv, j & 31);
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int v = lane + 32 * q;
                    b[u][q] = (j < cnt && v < nv) ? ld_b4<BF16, HINT>(D.B, (int64_t)col * D.ldb + 4 * v, pol.last)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j0 + u < cnt) {
                    const int64_t z = zb + j0 + u;
                    while (z >= rend) flush();
#pragma unroll
                    for (int q = 0; q < VPL; ++q) acc[q] = f4_fma(val[u], b[u][q], acc[q]);
                }
            }
        }
        mc = nc_;
        mv = nv_;
    }
    while (k <= kL) flush();  // the last row (whole or a piece) and trailing empty rows
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

namespace ns {

// ---------------------------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------------------------
template <int L, int VPL, bool BF16, bool HINT, bool DENSE>
__global__ void __launch_bounds__(kExecThreads) k_exec(const ExecDesc* __restrict__ descs,
                                                       const int32_t* __restrict__ queue,
                                                       const int32_t* __restrict__ queue_desc,
                                                       int64_t n_items, int32_t* ctrl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t s_ticket;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Policies pol{0, 0};
    if (HINT) pol = make_policies();
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(ctrl + 0, 1);
        __syncthreads();
        const int64_t t = s_ticket;
        __syncthreads();
        if (t >= n_items) break;
        const int32_t it = __ldg(queue + t);
        const int32_t di = queue_desc ? __ldg(queue_desc + t) : 0;
        const ExecDesc& D = descs[di];
        if (DENSE && it < D.n_dwin) {
            dense_item<L, VPL, BF16, HINT>(D, it, smem_raw, pol);
        } else {
            const int32_t c = (it - D.n_dwin) * D.group + warp;
            if (c < D.n_chunks) {
                if (L == 32 && VPL <= 2 && D.rl_all)
                    residual_chunk_stream<(VPL <= 2 ? VPL : 2), BF16, HINT>(D, c, lane, pol);
                else
                    residual_chunk<L, VPL, BF16, HINT>(D, c, lane, pol);
            }
        }
    }
    // the last CTA out resets the ticket for the next launch (stream order makes it visible)
    if (threadIdx.x == 0) {
        __threadfence();
        int done = atomicAdd(ctrl + 1, 1);
        if (done == (int)gridDim.x - 1) {
            atomicExch(ctrl + 0, 0);
            atomicExch(ctrl + 1, 0);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
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
    d->rl_all = P->st.n_rl == P->st.m ? 1 : 0;
    d->status = P->ctrl + 2;
}

typedef void (*ExecKernel)(const ExecDesc*, const int32_t*, const int32_t*, int64_t, int32_t*);

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

static ExecKernel select_kernel(int K, bool bf16, bool hint, bool dense)
{
    if (bf16) {
        if (hint) return dense ? pick_kernel<true, true, true>(K) : pick_kernel<true, true, false>(K);
        return dense ? pick_kernel<true, false, true>(K) : pick_kernel<true, false, false>(K);
    }
    if (hint) return dense ? pick_kernel<false, true, true>(K) : pick_kernel<false, true, false>(K);
    return dense ? pick_kernel<false, false, true>(K) : pick_kernel<false, false, false>(K);
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

// Kernel attributes and the persistent grid (resident CTAs on every SM, at most n_items).
// Must run outside stream capture.
ns_status_t exec_prepare(int64_t n_items, int K, int TM, int TK, bool bf16, bool hint, bool dense,
                         int* grid_out)
{
    ExecKernel kern = select_kernel(K, bf16, hint, dense);
    const size_t smem = dense ? dense_smem_bytes(K, TM, TK, bf16) : 0;
    if (dense) NS_TRY(dense_prepare(reinterpret_cast<const void*>(kern), smem));
    int per_sm = 0;
    NS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kExecThreads, smem));
    if (per_sm < 1) per_sm = 1;
    int dev = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
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
                        bool dense, int* grid_cache, cudaStream_t s)
{
    ExecKernel kern = select_kernel(K, bf16, hint, dense);
    const size_t smem = dense ? dense_smem_bytes(K, TM, TK, bf16) : 0;
    int grid = grid_cache ? *grid_cache : 0;
    if (grid == 0) NS_TRY(exec_prepare(n_items, K, TM, TK, bf16, hint, dense, &grid));
    if (grid_cache) *grid_cache = grid;
    if (n_items == 0) return NS_OK;
    kern<<<grid, kExecThreads, smem, s>>>(descs, queue, queue_desc, n_items, ctrl);
    NS_LAUNCH_CHECK();
    return NS_OK;
}

ns_status_t exec_launch_plan(Plan* P, cudaStream_t s)
{
    return exec_launch(P->desc_dev, P->queue, nullptr, P->st.n_items, P->ctrl, P->K, P->tune.TM,
                       P->tune.TK, P->dtype == NS_BF16, P->tune.l2_hints != 0, P->st.n_dwin > 0,
                       &P->exec_grid, s);
}

}  // namespace ns
