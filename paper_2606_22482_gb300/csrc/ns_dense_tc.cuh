// ns_dense_tc.cuh -- the dense-tile work item on the 5th-generation tensor cores (tcgen05, BF16).
//
// Matrix-engine execution model of arXiv 2606.22482 Section 5.1 on GB300: for one row window
// (TM rows) the product of its dense tiles with the gathered B rows,
//     C[window rows, :] = sum over dense tiles t of  A_t (TM x TK) * B[cols_t, :] (TK x K),
// runs as tcgen05.mma with the accumulator in tensor memory.  The MMA is posed transposed,
//     D (K features x TM rows) += B[cols_t, :]^T (features x TK) * A_t^T (TK x TM),
// so that M = 128 features per MMA (one or two feature blocks for K <= 256), N = TM rows
// (16, 32 or 64) and the MMA's K is the tile's compacted columns, 16 per instruction.
//
// Operands come straight from memory into shared memory with cp.async, in the no-swizzle
// layouts of the tensor core's shared-memory descriptors (8 x 8 blocks of 128 contiguous bytes):
//   * the A tile was expanded at plan time (dtile_x) in the K-major layout of the MMA's second
//     operand, so it is one contiguous copy of TM * TK * 2 bytes;
//   * each B row (compacted column c) is cut into 16-byte pieces of 8 features; piece j lands in
//     block (feature group j, column group c / 8), row c % 8 -- the MN-major layout of the first
//     operand (features contiguous).
// Tiles stream through a ring of up to kTcMaxStages stages (Section 7 "double buffer pipelining",
// deeper): the producer warps (1..3) copy a tile into a stage, and once a thread's copies of a
// tile have landed (kTcLag tiles later, so several tiles stay in flight) it fences them for the
// async proxy and arrives on the stage's `full` barrier; the producers run ahead of the MMAs by
// as many tiles as the ring holds.  One lane of warp 0 waits for `full`, issues the tile's MMAs
// and commits them to the stage's `empty` barrier, which the copies of a later tile wait for
// before reusing the stage.  When the window's last MMA has completed the accumulator is read out
// of tensor memory (tcgen05.ld, one warp per 32 features) into a shared TM x K tile; the rows'
// absorbed residual is added on the CUDA cores and every row is delivered as in the other item.
//
// Every wait is bounded: a wait that gives up sets the plan's timeout status, lets the CTA's
// copies and MMAs drain (again bounded) and stops taking dense items; the tensor memory is freed
// before the kernel ends.
#pragma once
#include "ns_internal.cuh"
#include "ns_ptx.cuh"

namespace ns {

constexpr int kTcMaxStages = 16;
// ring budget: three CTAs per SM with the result tile (measured on the attention shape, TM 64,
// TK 32: 0.153 ms per execute at three CTAs with a 3-stage ring, 0.191 ms at two CTAs with a 6- or
// 4-stage ring; resident windows hide the gathers' latency better than deeper rings)
constexpr int kTcRingBytes = 36 * 1024;  // (the result tile shares it: four CTAs per SM)
constexpr int kTcTmemCols = 128;         // two feature blocks x TM <= 64 columns of FP32 accumulators
constexpr int kTcCtasPerSm = 512 / kTcTmemCols;  // CTAs whose tensor memory fits an SM's 512 columns
constexpr int kTcProducers = kExecThreads - 32;  // warps 1..3 copy; warp 0 issues the MMAs
constexpr int kTcLag = 2;  // tiles a producer thread keeps in flight before it signals the oldest

struct TcGeom {
    int FB;           // feature blocks of 128 (ceil(K / 128))
    int a_bytes;      // expanded A tile
    int b_bytes;      // gathered B rows of one tile, all feature blocks
    int stage_bytes;  // one ring stage (A, then B), 128-byte aligned
    int S;            // ring stages (as many as the ring budget holds, kTcLag + 1 .. kTcMaxStages)
    int off_c;        // TM x cs_stride FP32 result tile (shares the ring: written only once the
                      // window's MMAs have completed and its producers are done)
    int cs_stride;
    int total;
};

__host__ __device__ inline TcGeom tc_geom(int K, int TM, int TK)
{
    TcGeom g;
    g.FB = (K + 127) / 128;
    g.a_bytes = TM * TK * 2;
    g.b_bytes = g.FB * TK * 256;
    g.stage_bytes = (g.a_bytes + g.b_bytes + 127) & ~127;
    g.S = kTcRingBytes / g.stage_bytes;
    if (g.S > kTcMaxStages) g.S = kTcMaxStages;
    if (g.S < kTcLag + 1) g.S = kTcLag + 1;  // the ring holds every tile a producer has in flight
    g.cs_stride = K + 4;
    g.off_c = 0;
    const int ring = g.S * g.stage_bytes, cs = (TM * g.cs_stride * 4 + 127) & ~127;
    g.total = ring > cs ? ring : cs;
    return g;
}

// the tensor-core item serves BF16 plans with K <= 256 (one or two feature blocks)
__host__ __device__ inline bool tc_supported(int K) { return K >= 8 && K <= 256; }

// ---- tcgen05 wrappers ---------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets, no swizzle.
// With no swizzle the leading offset is the distance between adjacent 8-row x 16-byte blocks
// along the MMA's K dimension and the stride offset the distance along M (first operand) or N
// (second operand), for K-major and MN-major operands alike (measured on this GPU with a
// standalone check over both readings, every element exact).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version field of this architecture
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 operands, first operand MN-major
// (features contiguous), second K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(n >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

// arrive once on `bar` when every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Tensor memory of the CTA: one warp allocates kTcTmemCols columns at kernel start and frees them
// at the end; the address goes through shared memory.
__device__ __forceinline__ void tc_alloc(uint32_t* slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(slot)), "r"(kTcTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kTcTmemCols) : "memory");
}

// Per-CTA state of the tensor-core item across the dense windows it takes.  The barriers live in
// static shared memory: full[kTcMaxStages] (one arrival per producer thread: its copies landed),
// empty[kTcMaxStages] (one arrival: the stage's MMAs completed), drain (the CTA's last MMAs).
// The ring's stage count depends on the plan's geometry, so every window of a CTA must use the
// same geometry (one plan per launch, or plans of one batch, which share their tune and K).
struct TcState {
    uint64_t* bars;  // full, empty, drain
    uint32_t tmem;   // tensor-memory base address (lane 0, first column)
    uint32_t gi;     // tiles this CTA has put through the ring (stage = gi % S)
    int S;           // stage count the ring was used with (0 before the first window)
    bool ok;         // false once a bounded wait gave up: no further dense items
};
constexpr int kTcBars = 2 * kTcMaxStages + 1;

// set-up by the whole CTA: barriers, then one warp allocates the tensor memory
__device__ __forceinline__ void tc_setup(TcState& S, uint64_t* bars, uint32_t* tmem_slot)
{
    S.bars = bars;
    S.gi = 0;
    S.S = 0;
    S.ok = true;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcMaxStages; ++i) {
            mbar_init(bars + i, kTcProducers);
            mbar_init(bars + kTcMaxStages + i, 1);
        }
        mbar_init(bars + 2 * kTcMaxStages, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();  // warp 0 converged again before the warp-wide allocation
    if ((threadIdx.x >> 5) == 0) tc_alloc(tmem_slot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    S.tmem = *tmem_slot;
}

// tear-down by the whole CTA: the MMAs it issued have completed (bounded wait), then the warp
// that allocated the tensor memory frees it
__device__ __forceinline__ void tc_teardown(TcState& S, int32_t* status)
{
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && S.gi > 0) {
        tc_commit(S.bars + 2 * kTcMaxStages);
        if (!mbar_wait(S.bars + 2 * kTcMaxStages, 0) && status) atomicOr(status, kStatusTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tc_dealloc(S.tmem);
}

// Copy tile d of the window into ring stage `st`: the expanded A tile (contiguous) and the TK
// gathered B rows cut into 16-byte pieces of 8 features.  Producer thread pt copies pieces
// q = pt, pt + kTcProducers, ... of the B rows, q = (piece j) * TK + (column c); kTcProducers is
// a multiple of TK, so c = pt % TK throughout and the column id (`col`, loaded tiles ahead) is
// the only index the copies need.
static_assert(kTcProducers % 32 == 0, "every producer thread serves one column of a tile");
template <bool HINT>
__device__ __forceinline__ void tc_stage_tile(const ExecDesc& D, int32_t d, int32_t col, unsigned char* st,
                                              const TcGeom& G, const Policies& pol)
{
    const int TK = D.TK, K = D.K;
    const int pt = threadIdx.x - 32;  // producer thread 0 .. kTcProducers - 1
    const unsigned char* ax = reinterpret_cast<const unsigned char*>(D.dtile_x) + (int64_t)d * G.a_bytes;
    for (int q = pt; q < G.a_bytes / 16; q += kTcProducers)
        cp_async16<HINT>(st + 16 * q, ax + 16 * q, true, pol.first);
    unsigned char* sb = st + G.a_bytes;
    const int c = pt % TK;
    const bool ok = col >= 0 && col < D.n;  // -1 pads the window's last tile
    if (col >= D.n) atomicOr(D.status, kStatusInternal);  // guard: corrupt plan (no copy is made)
    const unsigned char* src0 = reinterpret_cast<const unsigned char*>(D.B) + (ok ? (int64_t)col * D.ldb * 2 : 0);
    unsigned char* dst0 = sb + (c >> 3) * 2048 + (c & 7) * 16;
    const int npieces = TK * (K >> 3);
    for (int q = pt; q < npieces; q += kTcProducers) {
        const int j = q / TK;  // 8-feature piece of the row
        const int fb = j >> 4, m8 = j & 15;
        cp_async16<HINT>(dst0 + fb * (TK * 256) + m8 * 128, src0 + (ok ? 16 * j : 0), ok, pol.last);
    }
}

// the column id producer thread pt serves in tile d (-1 past the window's columns); nothing here
// may use the value, or the load would stall the loop it was hoisted out of
__device__ __forceinline__ int32_t tc_tile_col(const ExecDesc& D, int32_t d)
{
    return __ldg(D.dtile_cols + (int64_t)d * D.TK + (threadIdx.x - 32) % D.TK);
}

// One dense window on the tensor cores; Cs receives the TM x K product (FP32).  Returns false
// when a bounded wait gave up (the CTA then stops taking dense items).
template <bool HINT>
__device__ bool tc_window_product(const ExecDesc& D, int32_t w, unsigned char* smem, const TcGeom& G,
                                  TcState& S, const Policies& pol)
{
    const int TM = D.TM, TK = D.TK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t t0 = __ldg(D.win_dptr + w), t1 = __ldg(D.win_dptr + w + 1);
    const int T = t1 - t0;
    uint64_t* full = S.bars;
    uint64_t* empty = S.bars + kTcMaxStages;
    float* Cs = reinterpret_cast<float*>(smem + G.off_c);
    const uint32_t g0 = S.gi;
    const uint32_t idesc = tc_idesc_bf16(TM);
    bool ok = true;
    if (T <= 0) {  // a dense window holds at least one tile; guard against a corrupt plan
        if (threadIdx.x == 0) atomicOr(D.status, kStatusInternal);
        for (int q = threadIdx.x; q < TM * G.cs_stride; q += kExecThreads) Cs[q] = 0.f;
        __syncthreads();
        return true;
    }
    const int NS = G.S;
    if (S.S != 0 && S.S != NS) {  // guard: the ring's stage count changed between windows
        if (threadIdx.x == 0) atomicOr(D.status, kStatusInternal);
        S.ok = false;
        return false;
    }
    S.S = NS;
    if (warp != 0) {
        // producers (warps 1..3): run up to NS tiles ahead of the MMAs; each thread's column id
        // is loaded four tiles ahead, so no copy waits for an index load
        int32_t cq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cq[u] = u < T ? tc_tile_col(D, t0 + u) : -1;
        for (int i = 0; i < T; ++i) {
            const uint32_t g = g0 + (uint32_t)i;
            const int st = (int)(g % (uint32_t)NS);
            const int32_t col = cq[0];
            cq[0] = cq[1];
            cq[1] = cq[2];
            cq[2] = cq[3];
            cq[3] = i + 4 < T ? tc_tile_col(D, t0 + i + 4) : -1;
            if (g >= (uint32_t)NS && ok && !mbar_wait(empty + st, ((g / NS) - 1) & 1u)) ok = false;
            if (ok) tc_stage_tile<HINT>(D, t0 + i, col, smem + st * G.stage_bytes, G, pol);
            cp_async_commit();  // one group per tile, empty or not
            // The tile kTcLag back has landed: its bytes were written through the generic proxy
            // and the MMA reads them through the async proxy, so this thread fences its own
            // writes before it signals the stage full.
            if (i >= kTcLag) {
                cp_async_wait<kTcLag>();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(full + (int)((g - kTcLag) % (uint32_t)NS));
            }
        }
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int i = (T > kTcLag ? T - kTcLag : 0); i < T; ++i)
            mbar_arrive(full + (int)((g0 + (uint32_t)i) % (uint32_t)NS));
    } else if (lane == 0) {
        // the MMA lane: as each stage lands, its MMAs accumulate into tensor memory
        for (int i = 0; i < T; ++i) {
            const uint32_t g = g0 + (uint32_t)i;
            const int st = (int)(g % (uint32_t)NS);
            if (ok && !mbar_wait(full + st, (g / NS) & 1u)) ok = false;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * G.stage_bytes);  // A tile (second operand)
            const uint32_t sb = sa + (uint32_t)G.a_bytes;             // B rows (first operand)
            if (ok) {
                for (int fb = 0; fb < G.FB; ++fb)
                    for (int ks = 0; ks < TK / 16; ++ks) {
                        // first operand: features x 16 columns, MN-major (8-feature blocks 128 B
                        // apart along M, 8-column groups 2048 B apart along K)
                        const uint64_t ad = tc_desc(sb + fb * (TK * 256) + ks * 4096, 2048, 128);
                        // second operand: TM rows x 16 columns, K-major (column groups 128 B
                        // apart along K, 8-row groups TK * 16 B apart along N)
                        const uint64_t bd = tc_desc(sa + ks * 256, 128, TK * 16);
                        tc_mma(S.tmem + (uint32_t)(fb * TM), ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    }
            }
            tc_commit(empty + st);  // the stage is free once these MMAs completed
        }
    }
    __syncwarp();  // warp 0 reconverges after its MMA-issuing lane (tcgen05.ld is warp-wide)
    // the window's product is complete when its last tile's MMAs are
    {
        const uint32_t g = g0 + (uint32_t)(T - 1);
        if (!mbar_wait(empty + (g % (uint32_t)NS), (g / NS) & 1u)) ok = false;
    }
    S.gi = g0 + (uint32_t)T;
    tc_fence_after();
    // the result tile overwrites the ring the MMAs read through the async proxy: order those
    // reads (complete, as the barrier wait above showed) before this thread's generic writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // accumulator -> shared result tile: warp w reads TMEM lanes 32w..32w+31 (features), 16
    // columns (rows) at a time
    for (int fb = 0; fb < G.FB; ++fb) {
        const int f = fb * 128 + 32 * warp + lane;
        for (int c0 = 0; c0 < TM; c0 += 16) {
            uint32_t r[16];
            tc_ld16(S.tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(fb * TM + c0), r);
            if (f < D.K)
#pragma unroll
                for (int j = 0; j < 16; ++j) Cs[(c0 + j) * G.cs_stride + f] = ok ? __uint_as_float(r[j]) : 0.f;
        }
    }
    tc_fence_before();
    // every thread's outcome: any failed wait stops the CTA's dense work
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    if (!all_ok) {
        if (threadIdx.x == 0) atomicOr(D.status, kStatusTimeout);
        cp_async_wait<0>();
        S.ok = false;
        return false;
    }
    return true;
}

}  // namespace ns
