// ns_dense.cuh -- the dense-tile (tensor-core) work item of the persistent kernel.
//
// Matrix-engine execution model of arXiv 2606.22482 Section 5.1: for one row window, every
// dense tile's column ids gather the matching B rows, the A tile is expanded from its bitmap
// (Section 5.2.2 stores the dense core as a bitmap) and the product runs on the tensor cores,
// zeros included.  Tiles are double-buffered (Section 7 "double buffer pipelining"): the B rows,
// packed values and bitmap of tile t+1 stream into shared memory with cp.async while tile t is
// multiplied.
//
//   BF16 form: mma.sync m16n8k16, BF16 operands, FP32 accumulation (ldmatrix fragments).
//   FP32 form: mma.sync m16n8k8 on TF32 with the 3-term split of Markidis et al. (2018):
//              x = hi + lo with hi = tf32(x), lo = tf32(x - hi); a*b ~ ahi*bhi + ahi*blo + alo*bhi,
//              which keeps the error near FP32 while running on the tensor pipe.
//
// The window's TM x K result is assembled in shared memory, the rows' absorbed residual is
// added on the CUDA cores and each row is delivered (stored, or written as piece 0 of a split
// row).  The CTA's four warps split the window as TM/16 row groups x 4/(TM/16) column groups.
#pragma once
#include "ns_internal.cuh"
#include "ns_ptx.cuh"

namespace ns {

constexpr int kDenseMaxNB = 16;      // n8 blocks per warp per column pass
constexpr int kDenseBufBytes = 16384;  // per B staging buffer

struct DenseGeom {
    int CG, RG, NBW, PW, es, BW;
    int b_stride;   // elements per staged B row
    int a_stride;   // elements per expanded A row
    int cs_stride;  // floats per C row
    int off_b[2], off_p[2], off_bits[2], off_a, off_wp, off_c, total;
};

__host__ __device__ inline DenseGeom dense_geom(int K, int TM, int TK, bool bf16)
{
    DenseGeom g;
    g.es = bf16 ? 2 : 4;
    g.RG = TM / 16;
    g.CG = 4 / g.RG;
    g.BW = TM * TK / 32;
    int cap_cols = kDenseBufBytes / (TK * g.es);
    int nb_need = (K + 8 * g.CG - 1) / (8 * g.CG);
    int nb_cap = cap_cols / (8 * g.CG);
    int nb = nb_need < nb_cap ? nb_need : nb_cap;
    if (nb > kDenseMaxNB) nb = kDenseMaxNB;
    if (nb < 1) nb = 1;
    g.NBW = nb;
    g.PW = nb * 8 * g.CG;
    g.b_stride = g.PW + 8;
    g.a_stride = TK + (bf16 ? 8 : 4);
    g.cs_stride = K + 4;
    int off = 0;
    auto take = [&](int bytes) {
        int o = off;
        off += (bytes + 127) & ~127;
        return o;
    };
    for (int b = 0; b < 2; ++b) g.off_b[b] = take(TK * g.b_stride * g.es);
    for (int b = 0; b < 2; ++b) g.off_p[b] = take(TM * TK * g.es);
    for (int b = 0; b < 2; ++b) g.off_bits[b] = take(g.BW * 4);
    g.off_a = take(TM * g.a_stride * g.es);
    g.off_wp = take((g.BW + 1) * 4);
    g.off_c = take(TM * g.cs_stride * 4);
    g.total = off;
    return g;
}

inline size_t dense_smem_bytes(int K, int TM, int TK, bool bf16)
{
    return (size_t)dense_geom(K, TM, TK, bf16).total;
}

// Opt the kernel in to the largest dynamic shared memory the device allows (never a per-plan
// value: a smaller plan must not lower the limit under a larger plan's cached launches).
inline ns_status_t dense_prepare(const void* kern, size_t smem)
{
    int dev = 0, optin = 0;
    NS_CUDA_TRY(cudaGetDevice(&dev));
    NS_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    NS_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((int64_t)smem > lim) {
        set_error("execute needs %zu bytes of shared memory per block, the device allows %d", smem, lim);
        return NS_ERR_UNSUPPORTED;
    }
    NS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    NS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    return NS_OK;
}

// ---- tensor-core PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// hi/lo split of the 3xTF32 product
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

template <int L, int VPL, bool BF16, bool HINT>
__device__ void dense_deliver_rows(const ExecDesc& D, int32_t di, int32_t w, float* Cs, int cs_stride,
                                   int4* meta, const Policies& pol);

// ---------------------------------------------------------------------------------------------
template <int L, int VPL, bool BF16, bool HINT>
__device__ void dense_item(const ExecDesc& D, int32_t di, unsigned char* smem, int4* meta, const Policies& pol)
{
    const int TM = D.TM, TK = D.TK, K = D.K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    const DenseGeom G = dense_geom(K, TM, TK, BF16);
    const int rg = warp / G.CG, cg = warp % G.CG;
    const int lg_tk = TK == 16 ? 4 : 5;
    const int32_t w = __ldg(D.dwin + di);
    const int32_t t0 = __ldg(D.win_dptr + w), t1 = __ldg(D.win_dptr + w + 1);
    float* Cs = reinterpret_cast<float*>(smem + G.off_c);
    int32_t* wp = reinterpret_cast<int32_t*>(smem + G.off_wp);

    for (int p0 = 0; p0 < K; p0 += G.PW) {
        float acc[kDenseMaxNB][4];
#pragma unroll
        for (int nb = 0; nb < kDenseMaxNB; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;

        // stage tile t into buffer b: gathered B rows of this column pass, packed values, bitmap
        auto stage = [&](int32_t t, int b) {
            const int cpr = G.PW * G.es / 16;  // 16-byte chunks per B row
            unsigned char* bs = smem + G.off_b[b];
            for (int q = threadIdx.x; q < TK * cpr; q += blockDim.x) {
                const int c = q / cpr, off = q % cpr;
                const int32_t col = __ldg(D.dtile_cols + (int64_t)t * TK + c);
                const int gcol = p0 + off * (16 / G.es);
                const bool ok = col >= 0 && col < D.n && gcol < K;
                if (col >= D.n) atomicOr(D.status, kStatusInternal);  // guard: corrupt plan
                const unsigned char* src = reinterpret_cast<const unsigned char*>(D.B) +
                                           ((ok ? (int64_t)col * D.ldb + gcol : 0) * G.es);
                cp_async16<HINT>(bs + (c * G.b_stride + off * (16 / G.es)) * G.es, src, ok, pol.last);
            }
            const int32_t v0 = __ldg(D.dtile_voff + t), v1 = __ldg(D.dtile_voff + t + 1);
            const int pchunks = (v1 - v0) * G.es / 16;
            const unsigned char* vsrc = reinterpret_cast<const unsigned char*>(D.dtile_vals) + (int64_t)v0 * G.es;
            for (int q = threadIdx.x; q < pchunks; q += blockDim.x)
                cp_async16<HINT>(smem + G.off_p[b] + q * 16, vsrc + q * 16, true, pol.first);
            const unsigned char* bsrc = reinterpret_cast<const unsigned char*>(D.dtile_bits + (int64_t)t * G.BW);
            for (int q = threadIdx.x; q < G.BW / 4; q += blockDim.x)
                cp_async16<HINT>(smem + G.off_bits[b] + q * 16, bsrc + q * 16, true, pol.first);
        };

        if (t0 < t1) stage(t0, 0);
        cp_async_commit();
        for (int32_t t = t0; t < t1; ++t) {
            const int cur = (t - t0) & 1;
            if (t + 1 < t1) stage(t + 1, cur ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            // bitmap word prefix counts (value index of the first bit of every word)
            const uint32_t* bits = reinterpret_cast<const uint32_t*>(smem + G.off_bits[cur]);
            if (warp == 0) {
                int carry = 0;
                for (int q0 = 0; q0 < G.BW; q0 += 32) {
                    int q = q0 + lane;
                    int c = q < G.BW ? __popc(bits[q]) : 0;
                    int inc = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (q < G.BW) wp[q] = carry + inc - c;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
            __syncthreads();
            // expand the bitmap tile into a dense TM x TK operand
            for (int e = threadIdx.x; e < TM * TK; e += blockDim.x) {
                const int r = e >> lg_tk, c = e & (TK - 1);  // TK is 16 or 32
                const uint32_t word = bits[e >> 5];
                const bool set = (word >> (e & 31)) & 1u;
                const int idx = wp[e >> 5] + __popc(word & ((1u << (e & 31)) - 1u));
                if (BF16) {
                    const uint16_t* P = reinterpret_cast<const uint16_t*>(smem + G.off_p[cur]);
                    reinterpret_cast<uint16_t*>(smem + G.off_a)[r * G.a_stride + c] = set ? P[idx] : (uint16_t)0;
                } else {
                    const float* P = reinterpret_cast<const float*>(smem + G.off_p[cur]);
                    reinterpret_cast<float*>(smem + G.off_a)[r * G.a_stride + c] = set ? P[idx] : 0.f;
                }
            }
            __syncthreads();
            // tensor-core products for this warp's 16 rows and NBW n8 blocks
            const int cb0 = cg * G.NBW * 8;  // first column of this warp inside the pass
            if (BF16) {
                const uint16_t* As = reinterpret_cast<const uint16_t*>(smem + G.off_a);
                const uint16_t* Bs = reinterpret_cast<const uint16_t*>(smem + G.off_b[cur]);
                for (int kk = 0; kk < TK; kk += 16) {
                    uint32_t a[4];
                    ldsm_x4(a, As + (16 * rg + (lane & 15)) * G.a_stride + kk + (lane >> 4) * 8);
#pragma unroll
                    for (int nb = 0; nb < kDenseMaxNB; nb += 2) {
                        if (nb + 1 < G.NBW) {
                            uint32_t b[4];
                            ldsm_x4_t(b, Bs + (kk + (lane & 15)) * G.b_stride + cb0 + nb * 8 + (lane >> 4) * 8);
                            mma_bf16(acc[nb], a, b[0], b[1]);
                            mma_bf16(acc[nb + 1], a, b[2], b[3]);
                        } else if (nb < G.NBW) {
                            uint32_t b[2];
                            ldsm_x2_t(b, Bs + (kk + (lane & 15)) * G.b_stride + cb0 + nb * 8);
                            mma_bf16(acc[nb], a, b[0], b[1]);
                        }
                    }
                }
            } else {
                // The tensor pipe's FP32 accumulation is not round-to-nearest; a long chain of
                // tiles into one accumulator drifts.  Each tile's products go to a fresh
                // accumulator that is then added to the window's sum with an ordinary FP32 add.
                float part[kDenseMaxNB][4];
#pragma unroll
                for (int nb = 0; nb < kDenseMaxNB; ++nb) part[nb][0] = part[nb][1] = part[nb][2] = part[nb][3] = 0.f;
                const float* As = reinterpret_cast<const float*>(smem + G.off_a);
                const float* Bs = reinterpret_cast<const float*>(smem + G.off_b[cur]);
                for (int kk = 0; kk < TK; kk += 8) {
                    uint32_t ahi[4], alo[4];
                    const float* ar = As + (16 * rg + g) * G.a_stride + kk + tq;
                    split_tf32(ar[0], ahi[0], alo[0]);
                    split_tf32(ar[8 * G.a_stride], ahi[1], alo[1]);
                    split_tf32(ar[4], ahi[2], alo[2]);
                    split_tf32(ar[8 * G.a_stride + 4], ahi[3], alo[3]);
#pragma unroll
                    for (int nb = 0; nb < kDenseMaxNB; ++nb) {
                        if (nb < G.NBW) {
                            const float* br = Bs + (kk + tq) * G.b_stride + cb0 + nb * 8 + g;
                            uint32_t bhi0, blo0, bhi1, blo1;
                            split_tf32(br[0], bhi0, blo0);
                            split_tf32(br[4 * G.b_stride], bhi1, blo1);
                            mma_tf32(part[nb], alo, bhi0, bhi1);
                            mma_tf32(part[nb], ahi, blo0, blo1);
                            mma_tf32(part[nb], ahi, bhi0, bhi1);
                        }
                    }
                }
#pragma unroll
                for (int nb = 0; nb < kDenseMaxNB; ++nb)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[nb][e] += part[nb][e];
            }
            __syncthreads();  // buffer cur may be restaged for tile t + 2
        }
        cp_async_wait<0>();
        // this pass's columns into the shared result tile
#pragma unroll
        for (int nb = 0; nb < kDenseMaxNB; ++nb) {
            if (nb < G.NBW) {
                const int col = p0 + cg * G.NBW * 8 + nb * 8 + 2 * tq;
                if (col < K) {
                    const int r = 16 * rg + g;
                    *reinterpret_cast<float2*>(Cs + r * G.cs_stride + col) = make_float2(acc[nb][0], acc[nb][1]);
                    *reinterpret_cast<float2*>(Cs + (r + 8) * G.cs_stride + col) = make_float2(acc[nb][2], acc[nb][3]);
                }
            }
        }
    }
    __syncthreads();
    dense_deliver_rows<L, VPL, BF16, HINT>(D, di, w, Cs, G.cs_stride, meta, pol);
}

// The window's rows: the tensor-core part (Cs, TM x K FP32 in shared memory) plus the rows'
// absorbed residual on the CUDA cores, then delivery (stored, or piece 0 of a split row).
// Latency first: one pass loads every row's id, residual range and split id (a thread per row,
// into `meta`); then each warp takes its rows (r = warp, warp + 4, ...) and gathers all of their
// residual nonzeros as one list, 32 entries per load and four B rows in flight, adding them into
// the rows of Cs it owns; last, the rows are delivered from Cs.
template <int L, int VPL, bool BF16, bool HINT>
__device__ void dense_deliver_rows(const ExecDesc& D, int32_t di, int32_t w, float* Cs, int cs_stride,
                                   int4* meta, const Policies& pol)
{
    const int TM = D.TM, K = D.K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool absorb = __ldg(D.dwin_absorb + di) != 0;
    const int nv = K >> 2;
    const int grp = lane / L, li = lane % L;
    // ---- row metadata: (row id, first residual nonzero, residual length, split id) ----
    for (int r = threadIdx.x; r < TM; r += kExecThreads) {
        int32_t i = __ldg(D.win_rows + (int64_t)w * TM + r);
        int32_t z0 = 0, n = 0, sp = -1;
        if (i >= D.m) {  // guard: corrupt plan
            atomicOr(D.status, kStatusInternal);
            i = -1;
        }
        if (i >= 0) sp = __ldg(D.row_split + i);
        if (i >= 0 && absorb) {
            z0 = __ldg(D.res_rowptr + i);
            const int32_t z1 = __ldg(D.res_rowptr + i + 1);
            n = z1 - z0;
            if (z0 < 0 || n < 0 || (int64_t)z0 + n > D.n_res) {  // guard: corrupt plan
                atomicOr(D.status, kStatusInternal);
                n = 0;
            }
        }
        meta[r] = make_int4(i, z0, n, sp);
    }
    __syncthreads();
    // ---- absorbed residual: this warp's rows as one list of nonzeros ----
    const int nrw = (TM - warp + kExecWarps - 1) / kExecWarps;  // rows warp, warp + 4, ... (<= 16)
    int len = 0, z0l = 0;
    if (lane < nrw) {
        const int4 mt = meta[warp + kExecWarps * lane];
        len = mt.z;
        z0l = mt.y;
    }
    int start = len;  // inclusive scan over the warp's rows
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start += y;
    }
    const int total = __shfl_sync(0xffffffffu, start, 15);
    start -= len;  // exclusive
    for (int e0 = 0; e0 < total; e0 += 32) {
        // entry e0 + lane: its row l (largest l with start_l <= e), then its column and value
        const int e = e0 + lane;
        int l = 0;
#pragma unroll
        for (int step = 8; step >= 1; step >>= 1) {
            const int s_l = __shfl_sync(0xffffffffu, start, (l + step) & 31);
            if (l + step < nrw && s_l <= e) l += step;
        }
        const int zl = __shfl_sync(0xffffffffu, z0l, l & 31);
        const int sl = __shfl_sync(0xffffffffu, start, l & 31);
        int32_t ec = -1;
        float ev = 0.f;
        if (e < total) {
            const int64_t z = (int64_t)zl + (e - sl);
            ec = __ldg(D.res_col + z);
            ev = __ldg(D.res_val + z);
            if ((unsigned)ec >= (unsigned)D.n) {  // guard: never gather outside B
                atomicOr(D.status, kStatusInternal);
                ec = -1;
            }
        }
        const int er = warp + kExecWarps * l;  // the entry's row in the window
        const int cnt = total - e0 < 32 ? total - e0 : 32;
        // the warp gathers the listed B rows, four in flight, lanes across the row
        for (int j0 = 0; j0 < cnt; j0 += 4) {
            BRaw<BF16> b[4][VPL];
            float val[4];
            int row[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u;
                const int32_t col = __shfl_sync(0xffffffffu, ec, j & 31);
                val[u] = __shfl_sync(0xffffffffu, ev, j & 31);
                row[u] = __shfl_sync(0xffffffffu, er, j & 31);
                const bool have = j < cnt && col >= 0;
                if (!have) val[u] = 0.f;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int v = li + L * q;
                    const int64_t off = (int64_t)(have ? col : 0) * D.ldb + 4 * v;
                    b[u][q] = (have && grp == 0 && v < nv)
                                  ? ld_braw<BF16, HINT>(static_cast<const unsigned char*>(D.B) + off * (BF16 ? 2 : 4), pol.last)
                                  : braw_zero<BF16>();
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j0 + u >= cnt) break;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int v = li + L * q;
                    if (grp == 0 && v < nv) {
                        float4* cp = reinterpret_cast<float4*>(Cs + row[u] * cs_stride + 4 * v);
                        *cp = f4_fma(val[u], widen(b[u][q]), *cp);
                    }
                }
            }
        }
    }
    __syncwarp();
    // ---- delivery, a warp per row ----
    for (int r = warp; r < TM; r += kExecWarps) {
        const int4 mt = meta[r];
        const int32_t i = mt.x;
        if (i < 0) continue;
        float4 acc[VPL];
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            const int v = li + L * q;
            acc[q] = (grp == 0 && v < nv) ? *reinterpret_cast<const float4*>(Cs + r * cs_stride + 4 * v)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        deliver_row<L, VPL, HINT>(D, i, 0, true, acc, lane, pol.first, mt.w);
    }
    __syncthreads();  // shared memory is reused by the next item
}

}  // namespace ns
