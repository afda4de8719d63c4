/*
 * ns_oracle.c -- FP64 CPU oracle for the hybrid SpMM C = A * B.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this file:
 * only the tests, the package's smoke() check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or table with the CUDA library; the two meet only in the seeded
 * inputs drawn by the `synth` module.
 *
 * Two things live here:
 *
 *  1. orc_spmm_rows -- the plain definition of SpMM (Section 5.1, both execution models compute
 *     the same product):  C[i,:] = sum_{p in row i} vals[p] * B[colidx[p], :], evaluated in
 *     double precision with A's FP32 values and B's values (FP32, or BF16 widened exactly)
 *     first widened to double, accumulated in ascending p.
 *
 *  2. orc_plan_build -- the CPU reference partition of A.  It takes the method's planning steps
 *     in the paper's order (Section 5.2.2 row/column extraction with the Len rule of Eq. 4-5,
 *     Section 6.1 local reordering, row windows and column compaction, the tile density rule
 *     derived from the cost model of Eq. 1-3, the residual of Section 5.2.2) with the integer
 *     readings written down in the project design notes.  The device planner must reproduce
 *     every array it emits bit for bit.  How the execute kernel then schedules that partition
 *     (residual chunks, split rows, the work-list order) is not the paper's partition and is not
 *     restated here: the tests check it by invariants and by the product.
 *
 * Everything is deliberately simple: loops, qsort, binary search.  No blocking, no fusion.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAU_INF 2147483647

/* ---------------------------------------------------------------------------------------- */
/* scalar helpers                                                                            */
/* ---------------------------------------------------------------------------------------- */

static double orc_bf16_to_double(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16; /* BF16 is the upper half of an IEEE-754 binary32 */
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Round-to-nearest-even of a binary32 to BF16 on the bit pattern: add 0x7FFF plus the
 * lowest kept bit, then truncate.  Inputs carry no NaNs. */
uint16_t orc_f32_to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void orc_f32_to_bf16_array(const float* x, int64_t count, uint16_t* out)
{
    for (int64_t i = 0; i < count; ++i) out[i] = orc_f32_to_bf16(x[i]);
}

/* ---------------------------------------------------------------------------------------- */
/* 1. the SpMM definition                                                                    */
/* ---------------------------------------------------------------------------------------- */

/* C_out[r, :] = sum over row rows[r] of A, for r in [0, nrows).  B is n x K with leading
 * dimension ldb (elements); b_bf16 selects uint16 BF16 storage.  C_out is nrows x K doubles. */
int orc_spmm_rows(int32_t m, int32_t n, int32_t K, const int32_t* rowptr, const int32_t* colidx,
                  const float* vals, const void* B, int32_t b_bf16, int64_t ldb,
                  const int32_t* rows, int64_t nrows, double* C_out)
{
    if (K < 0 || ldb < K) return 1;
    for (int64_t r = 0; r < nrows; ++r) {
        int32_t i = rows[r];
        double* c = C_out + r * (int64_t)K;
        for (int32_t k = 0; k < K; ++k) c[k] = 0.0;
        if (i < 0 || i >= m) return 1;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = colidx[p];
            if (j < 0 || j >= n) return 1;
            double a = (double)vals[p];
            if (b_bf16) {
                const uint16_t* b = (const uint16_t*)B + (int64_t)j * ldb;
                for (int32_t k = 0; k < K; ++k) c[k] += a * orc_bf16_to_double(b[k]);
            } else {
                const float* b = (const float*)B + (int64_t)j * ldb;
                for (int32_t k = 0; k < K; ++k) c[k] += a * (double)b[k];
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* 2. the reference partition                                                                */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
    int32_t TM;          /* row-window height (Section 6.1: windows match the tile's M)         */
    int32_t TK;          /* compacted columns per tile                                           */
    int32_t tau_tile;    /* tile is dense iff tile_nnz >= tau_tile (alpha * TM * TK, rounded up) */
    int32_t tau_row;     /* row goes to the residual iff Len(row) <= tau_row (Eq. 4-5)           */
    int32_t tau_col;     /* column (inside the window rows) to residual iff count <= tau_col      */
    int32_t col_order;   /* 0: count descending then column ascending; 1: column ascending       */
    int32_t reorder;     /* Section 6.1 local reordering: windows per cluster (0: off)            */
} orc_tune;

typedef struct {
    int64_t m, n, nnz, K, b_bf16, TM, TK;
    int64_t m_aic, n_win, n_dtiles, n_dwin, n_dvals, n_res;
    int32_t* aic_rows;   /* rows kept for windows, in window order                               */
    int32_t* win_rows;   /* n_win * TM rows, the last window padded with -1                      */
    int32_t* win_dptr;   /* dense tiles of window w: [win_dptr[w], win_dptr[w + 1])              */
    int32_t* dtile_cols; /* TK column ids per dense tile (-1 past the window's last column)      */
    uint32_t* dtile_bits;/* TM x TK row-major bitmap per dense tile                              */
    int32_t* dtile_voff; /* first packed value of each dense tile (padded to 8 per tile)         */
    void* dtile_vals;    /* packed values in bitmap order (FP32, or BF16 rounded to nearest even) */
    int32_t* res_rowptr; /* residual CSR over the original m rows                                */
    int32_t* res_col;
    float* res_val;
} orc_plan;

typedef struct {
    int32_t col, cnt;
} orc_ucol;

static int cmp_int32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int cmp_ucol_count_desc(const void* a, const void* b)
{
    const orc_ucol* x = (const orc_ucol*)a;
    const orc_ucol* y = (const orc_ucol*)b;
    if (x->cnt != y->cnt) return (x->cnt < y->cnt) - (x->cnt > y->cnt);
    return (x->col > y->col) - (x->col < y->col);
}

/* position of column j inside the sorted row segment colidx[b, e); -1 if absent */
static int64_t find_in_row(const int32_t* colidx, int64_t b, int64_t e, int32_t j)
{
    while (b < e) {
        int64_t mid = b + (e - b) / 2;
        if (colidx[mid] == j) return mid;
        if (colidx[mid] < j) b = mid + 1;
        else e = mid;
    }
    return -1;
}

void orc_plan_free(orc_plan* p)
{
    if (!p) return;
    free(p->aic_rows); free(p->win_rows); free(p->win_dptr);
    free(p->dtile_cols); free(p->dtile_bits); free(p->dtile_voff); free(p->dtile_vals);
    free(p->res_rowptr); free(p->res_col); free(p->res_val);
    free(p);
}

/* growable buffer helper */
static int grow(void** buf, int64_t* cap, int64_t need, size_t esize)
{
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    void* nb = realloc(*buf, (size_t)nc * esize);
    if (!nb) return 1;
    *buf = nb;
    *cap = nc;
    return 0;
}

/* Returns 0 on success, 1 on an invalid CSR or tune, 2 on allocation failure. */
int orc_plan_build(int32_t m, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                   const float* vals, int32_t K, int32_t b_bf16, const orc_tune* tu,
                   orc_plan** out)
{
    *out = NULL;
    /* ---- input checks: sorted unique in-range columns, monotone row pointers ---- */
    if (m < 0 || n < 0 || K < 1) return 1;
    if (rowptr[0] != 0) return 1;
    for (int32_t i = 0; i < m; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return 1;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            if (colidx[p] < 0 || colidx[p] >= n) return 1;
            if (p > rowptr[i] && colidx[p] <= colidx[p - 1]) return 1;
        }
    }
    const int32_t TM = tu->TM, TK = tu->TK;
    if (!(TM == 16 || TM == 32 || TM == 64) || !(TK == 16 || TK == 32)) return 1;
    if (tu->reorder < 0) return 1;
    const int64_t nnz = rowptr[m];
    const int32_t BW = TM * TK / 32; /* bitmap words per tile */

    orc_plan* P = (orc_plan*)calloc(1, sizeof(orc_plan));
    if (!P) return 2;
    P->m = m; P->n = n; P->nnz = nnz; P->K = K; P->b_bf16 = b_bf16 ? 1 : 0; P->TM = TM; P->TK = TK;

    int32_t* len = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    uint8_t* is_dense_elem = (uint8_t*)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    uint8_t* aic_col = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    if (!len || !is_dense_elem || !aic_col) { free(len); free(is_dense_elem); free(aic_col); orc_plan_free(P); return 2; }

    /* ---- Eq. 4: Len(row); Eq. 5 rule with an integer threshold: row to residual iff
     *      Len <= tau_row.  Windows (and with them the whole extraction) exist only when a
     *      tile can be dense at all, i.e. tau_tile is finite. ---- */
    for (int32_t i = 0; i < m; ++i) len[i] = rowptr[i + 1] - rowptr[i];
    const int windows_on = tu->tau_tile != ORC_TAU_INF;
    int64_t m_aic = 0;
    if (windows_on)
        for (int32_t i = 0; i < m; ++i) m_aic += len[i] > tu->tau_row;
    P->m_aic = m_aic;
    P->aic_rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m_aic > 0 ? m_aic : 1));
    {
        int64_t k = 0;
        if (windows_on)
            for (int32_t i = 0; i < m; ++i)
                if (len[i] > tu->tau_row) P->aic_rows[k++] = i;
    }

    /* ---- second extraction stage: column lengths inside the rows kept for windows ---- */
    for (int32_t j = 0; j < n; ++j) aic_col[j] = 1;
    if (windows_on && tu->tau_col > 0) {
        int32_t* colcount = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
        for (int64_t k = 0; k < m_aic; ++k) {
            int32_t i = P->aic_rows[k];
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) colcount[colidx[p]]++;
        }
        for (int32_t j = 0; j < n; ++j) aic_col[j] = colcount[j] > tu->tau_col;
        free(colcount);
    }

    /* ---- Section 6.1 local reordering: inside clusters of reorder*TM consecutive kept rows,
     *      rebuild windows greedily.  The anchor is the first unassigned row of the cluster in the
     *      current order; it takes the TM-1 unassigned rows most similar to it by Jaccard
     *      similarity of their kept-column sets (ties: earlier position), best first. ---- */
    if (windows_on && tu->reorder > 0 && m_aic > 0) {
        const int64_t CR = (int64_t)tu->reorder * TM;
        int32_t* neworder = (int32_t*)malloc(sizeof(int32_t) * (size_t)m_aic);
        int64_t* klen = (int64_t*)malloc(sizeof(int64_t) * (size_t)m_aic);
        uint8_t* used = (uint8_t*)calloc((size_t)m_aic, 1);
        for (int64_t k = 0; k < m_aic; ++k) {
            int32_t i = P->aic_rows[k];
            int64_t c = 0;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) c += aic_col[colidx[p]] ? 1 : 0;
            klen[k] = c;
        }
        for (int64_t c0 = 0; c0 < m_aic; c0 += CR) {
            const int64_t c1 = c0 + CR < m_aic ? c0 + CR : m_aic;
            int64_t out = c0;
            for (int64_t a = c0; a < c1; ++a) {
                if (used[a]) continue;
                used[a] = 1;
                neworder[out++] = P->aic_rows[a];
                const int32_t ia = P->aic_rows[a];
                for (int32_t pick = 0; pick < TM - 1; ++pick) {
                    int64_t best = -1, bn = 0, bd = 1;
                    for (int64_t b = c0; b < c1; ++b) {
                        if (used[b]) continue;
                        /* |intersection| over kept columns: merge of the two sorted rows */
                        const int32_t ib = P->aic_rows[b];
                        int64_t inter = 0;
                        int32_t p = rowptr[ia], q = rowptr[ib];
                        while (p < rowptr[ia + 1] && q < rowptr[ib + 1]) {
                            if (colidx[p] < colidx[q]) ++p;
                            else if (colidx[p] > colidx[q]) ++q;
                            else {
                                inter += aic_col[colidx[p]] ? 1 : 0;
                                ++p;
                                ++q;
                            }
                        }
                        const int64_t uni = klen[a] + klen[b] - inter;
                        const int64_t num = uni > 0 ? inter : 0, den = uni > 0 ? uni : 1;
                        if (best < 0 || num * bd > bn * den) {  /* strictly better; ties keep the earlier */
                            best = b;
                            bn = num;
                            bd = den;
                        }
                    }
                    if (best < 0) break;
                    used[best] = 1;
                    neworder[out++] = P->aic_rows[best];
                }
            }
        }
        memcpy(P->aic_rows, neworder, sizeof(int32_t) * (size_t)m_aic);
        free(neworder);
        free(klen);
        free(used);
    }

    /* ---- windows: consecutive kept rows, TM per window, the last padded with -1 ---- */
    const int64_t n_win = (m_aic + TM - 1) / TM;
    P->n_win = n_win;
    P->win_rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_win * TM > 0 ? n_win * TM : 1));
    for (int64_t s = 0; s < n_win * TM; ++s) P->win_rows[s] = s < m_aic ? P->aic_rows[s] : -1;
    P->win_dptr = (int32_t*)calloc((size_t)(n_win + 1), sizeof(int32_t));

    /* growable outputs of the window pass */
    int32_t* dcols = NULL; int64_t dcols_cap = 0;       /* n_dtiles * TK */
    uint32_t* dbits = NULL; int64_t dbits_cap = 0;      /* n_dtiles * BW */
    int32_t* dtnnz = NULL; int64_t dtnnz_cap = 0;       /* n_dtiles */
    int64_t n_dt = 0;
    int32_t* win_ntile_dense_rows = NULL; /* unused */
    (void)win_ntile_dense_rows;

    /* scratch per window */
    int32_t* wcols = NULL; int64_t wcols_cap = 0;
    orc_ucol* uc = NULL; int64_t uc_cap = 0;
    int32_t* uasc = NULL; int64_t uasc_cap = 0;     /* ascending unique columns */
    int32_t* upos = NULL; int64_t upos_cap = 0;     /* canonical position of each ascending entry */
    int32_t* tile_rank = NULL; int64_t tile_rank_cap = 0; /* dense rank of tile t or -1 */

    for (int64_t w = 0; w < n_win; ++w) {
        /* collect the window's kept columns (Section 6.1: compaction drops empty columns) */
        int64_t cnt = 0;
        for (int32_t r = 0; r < TM; ++r) {
            int32_t i = P->win_rows[w * TM + r];
            if (i < 0) continue;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                if (!aic_col[colidx[p]]) continue;
                if (grow((void**)&wcols, &wcols_cap, cnt + 1, sizeof(int32_t))) goto oom;
                wcols[cnt++] = colidx[p];
            }
        }
        qsort(wcols, (size_t)cnt, sizeof(int32_t), cmp_int32);
        int64_t U = 0;
        for (int64_t q = 0; q < cnt; ++q) {
            if (q == 0 || wcols[q] != wcols[q - 1]) {
                if (grow((void**)&uc, &uc_cap, U + 1, sizeof(orc_ucol))) goto oom;
                uc[U].col = wcols[q];
                uc[U].cnt = 1;
                ++U;
            } else {
                uc[U - 1].cnt++;
            }
        }
        if (grow((void**)&uasc, &uasc_cap, U + 1, sizeof(int32_t))) goto oom;
        if (grow((void**)&upos, &upos_cap, U + 1, sizeof(int32_t))) goto oom;
        for (int64_t q = 0; q < U; ++q) uasc[q] = uc[q].col;
        /* canonical column order inside the window */
        if (tu->col_order == 0) qsort(uc, (size_t)U, sizeof(orc_ucol), cmp_ucol_count_desc);
        for (int64_t q = 0; q < U; ++q) {
            int64_t a = find_in_row(uasc, 0, U, uc[q].col);
            upos[a] = (int32_t)q;
        }
        /* tiles of TK consecutive positions; dense iff tile_nnz >= tau_tile */
        int64_t ntile = (U + TK - 1) / TK;
        if (grow((void**)&tile_rank, &tile_rank_cap, ntile + 1, sizeof(int32_t))) goto oom;
        int64_t dt_begin = n_dt;
        for (int64_t t = 0; t < ntile; ++t) {
            int64_t tnnz = 0;
            for (int64_t q = t * TK; q < (t + 1) * TK && q < U; ++q) tnnz += uc[q].cnt;
            if (tnnz >= tu->tau_tile) {
                tile_rank[t] = (int32_t)(n_dt - dt_begin);
                if (grow((void**)&dcols, &dcols_cap, (n_dt + 1) * TK, sizeof(int32_t))) goto oom;
                if (grow((void**)&dbits, &dbits_cap, (n_dt + 1) * BW, sizeof(uint32_t))) goto oom;
                if (grow((void**)&dtnnz, &dtnnz_cap, n_dt + 1, sizeof(int32_t))) goto oom;
                for (int32_t c = 0; c < TK; ++c) {
                    int64_t q = t * TK + c;
                    dcols[n_dt * TK + c] = q < U ? uc[q].col : -1;
                }
                for (int32_t b = 0; b < BW; ++b) dbits[n_dt * BW + b] = 0;
                dtnnz[n_dt] = (int32_t)tnnz;
                ++n_dt;
            } else {
                tile_rank[t] = -1;
            }
        }
        P->win_dptr[w + 1] = (int32_t)n_dt;
        /* mark each window element that fell into a dense tile and set its bitmap bit */
        for (int32_t r = 0; r < TM; ++r) {
            int32_t i = P->win_rows[w * TM + r];
            if (i < 0) continue;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                if (!aic_col[colidx[p]]) continue;
                int64_t a = find_in_row(uasc, 0, U, colidx[p]);
                int32_t pos = upos[a];
                int32_t t = pos / TK, c = pos % TK;
                if (tile_rank[t] < 0) continue;
                int64_t d = dt_begin + tile_rank[t];
                int32_t bit = r * TK + c;
                dbits[d * BW + bit / 32] |= 1u << (bit % 32);
                is_dense_elem[p] = 1;
            }
        }
    }
    P->n_dtiles = n_dt;

    /* ---- dense tile values, packed in bitmap order, each tile padded to 8 values ---- */
    P->dtile_voff = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_dt + 1));
    P->dtile_voff[0] = 0;
    for (int64_t d = 0; d < n_dt; ++d)
        P->dtile_voff[d + 1] = P->dtile_voff[d] + ((dtnnz[d] + 7) / 8) * 8;
    P->n_dvals = P->dtile_voff[n_dt];
    P->dtile_vals = calloc((size_t)(P->n_dvals > 0 ? P->n_dvals : 1), b_bf16 ? 2 : 4);
    P->dtile_cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_dt * TK > 0 ? n_dt * TK : 1));
    P->dtile_bits = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_dt * BW > 0 ? n_dt * BW : 1));
    if (n_dt) {
        memcpy(P->dtile_cols, dcols, sizeof(int32_t) * (size_t)(n_dt * TK));
        memcpy(P->dtile_bits, dbits, sizeof(uint32_t) * (size_t)(n_dt * BW));
    }
    for (int64_t w = 0; w < n_win; ++w) {
        for (int64_t d = P->win_dptr[w]; d < P->win_dptr[w + 1]; ++d) {
            int64_t v = P->dtile_voff[d];
            for (int32_t bit = 0; bit < TM * TK; ++bit) {
                if (!((P->dtile_bits[d * BW + bit / 32] >> (bit % 32)) & 1u)) continue;
                int32_t r = bit / TK, c = bit % TK;
                int32_t i = P->win_rows[w * TM + r];
                int32_t j = P->dtile_cols[d * TK + c];
                int64_t p = find_in_row(colidx, rowptr[i], rowptr[i + 1], j);
                if (b_bf16) ((uint16_t*)P->dtile_vals)[v] = orc_f32_to_bf16(vals[p]);
                else ((float*)P->dtile_vals)[v] = vals[p];
                ++v;
            }
        }
    }

    /* ---- residual CSR: every element not in a dense tile, original rows, column order ---- */
    P->res_rowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    P->res_rowptr[0] = 0;
    for (int32_t i = 0; i < m; ++i) {
        int32_t c = 0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) c += !is_dense_elem[p];
        P->res_rowptr[i + 1] = P->res_rowptr[i] + c;
    }
    P->n_res = P->res_rowptr[m];
    P->res_col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->n_res > 0 ? P->n_res : 1));
    P->res_val = (float*)malloc(sizeof(float) * (size_t)(P->n_res > 0 ? P->n_res : 1));
    {
        int64_t z = 0;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                if (!is_dense_elem[p]) { P->res_col[z] = colidx[p]; P->res_val[z] = vals[p]; ++z; }
    }

    /* ---- windows with at least one dense tile (the matrix engine's row-window list) ---- */
    {
        int64_t n_dwin = 0;
        for (int64_t w = 0; w < n_win; ++w) n_dwin += P->win_dptr[w + 1] > P->win_dptr[w];
        P->n_dwin = n_dwin;
    }

    free(len); free(is_dense_elem); free(aic_col);
    free(dcols); free(dbits); free(dtnnz); free(wcols); free(uc); free(uasc); free(upos); free(tile_rank);
    *out = P;
    return 0;

oom:
    free(len); free(is_dense_elem); free(aic_col);
    free(dcols); free(dbits); free(dtnnz); free(wcols); free(uc); free(uasc); free(upos); free(tile_rank);
    orc_plan_free(P);
    return 2;
}

/* ---------------------------------------------------------------------------------------- */
/* accessors for the Python wrapper                                                          */
/* ---------------------------------------------------------------------------------------- */

int64_t orc_plan_scalar(const orc_plan* P, const char* name)
{
#define S(x) if (!strcmp(name, #x)) return P->x;
    S(m) S(n) S(nnz) S(K) S(b_bf16) S(TM) S(TK) S(m_aic) S(n_win) S(n_dtiles) S(n_dwin) S(n_dvals)
    S(n_res)
#undef S
    return -1;
}

/* ptr, element count and element size (bytes) of a named array; returns 1 if unknown */
int orc_plan_array(const orc_plan* P, const char* name, const void** ptr, int64_t* count,
                   int32_t* esize)
{
    const int64_t TM = P->TM, TK = P->TK, BW = TM * TK / 32;
#define A(x, cnt, es) if (!strcmp(name, #x)) { *ptr = P->x; *count = (cnt); *esize = (es); return 0; }
    A(aic_rows, P->m_aic, 4)
    A(win_rows, P->n_win * TM, 4)
    A(win_dptr, P->n_win + 1, 4)
    A(dtile_cols, P->n_dtiles * TK, 4)
    A(dtile_bits, P->n_dtiles * BW, 4)
    A(dtile_voff, P->n_dtiles + 1, 4)
    A(dtile_vals, P->n_dvals, P->b_bf16 ? 2 : 4)
    A(res_rowptr, P->m + 1, 4)
    A(res_col, P->n_res, 4)
    A(res_val, P->n_res, 4)
#undef A
    return 1;
}
