// Internal declarations of the ALS / ALS-NCG CUDA library (sm_103a).
// The public boundary is include/als.h; everything here is private.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "als.h"

#define ALS_MAX_NF 128
#define ALS_TC_LD 128          // widest n_f of the tcgen05 Gram (one 128-row MMA tile)
#define ALS_HEAVY_MIN 512      // rows at least this long get a whole CTA in the passes (default)
#define ALS_DUAL_MAX 64        // longest row of the mixed form's light-row (n_i x n_i) solve
#define ALS_DUAL_SMALL 32      // light rows at most this long take a smaller layout (more CTAs per SM)
#define ALS_TC_PF_MIN 256      // tensor-core sweep: rows at least this long prefetch their factor rows
#define ALS_TUNE_MARGIN 0.02   // the autotuner keeps a shape unless a candidate is this much faster

// Slots of the device scalar block (double S[]).
enum {
    S_C = 0,        // c0..c4 of Q(alpha), 5 slots
    S_ALPHA = 5,    // accepted step
    S_BETA = 6,     // beta-bar of Eq. (8)
    S_S = 7,        // gbar_k . g_k
    S_GG = 8,       // |g_k|^2
    S_GBG = 9,      // gbar_{k+1} . g_{k+1}
    S_GBD = 10,     // gbar_{k+1} . (g_{k+1} - g_k)
    S_F = 11,       // f(x_k) from Q(alpha)
    S_MODE = 12,    // 1: fallback step (ALS point), 0: line-search step
    S_SHRINK = 13,  // backtracking count
    S_NFALL = 14,   // total fallbacks
    S_GG0 = 15,     // |g_0|^2
    S_RED = 16,     // 5 slots: plain reduction results (loss, |g|^2, ...)
    S_COUNT = 24
};

// Post-operations run by the last block of a reduction (one thread, FP64).
enum { POST_NONE = 0, POST_LSELECT = 1, POST_BETA = 2, POST_INIT = 3 };

struct LsParams {
    double alpha0, tau, c;
    int max_shrinks;
    int mode;   // als_ls_mode
    double c2;  // More-Thuente curvature tolerance
    int beta;   // als_beta_form
};

// Per-kernel-class launch timing of a sweep (als_time_sweep): when a context
// holds a KTimer, each sweep launch records a CUDA event pair on the stream
// it is launched on.  Classes: 0 k_sweep_tc prefetching variant, 1 k_sweep_tc,
// 2 k_sweep_dual, 3 k_sweep_fma, 4 the split heavy rows (all their launches).
enum { KT_TC_PF = 0, KT_TC = 1, KT_DUAL = 2, KT_FMA = 3, KT_SPLIT = 4, KT_TC_SEG = 5, KT_NCLASS = 6 };
struct KTimer {
    static constexpr int kMax = 16;          // launches per class between two reads
    cudaEvent_t ev[KT_NCLASS][kMax][2];
    int n[KT_NCLASS];
    int depth;                               // > 0 inside the split part: its own launches
                                             // (but for KT_TC_SEG, the tensor-core segment launches)
    bool serial;                             // the split part runs on the context's stream
};
void kt_begin(struct als_ctx *c, int cls, cudaStream_t st);
void kt_end(struct als_ctx *c, int cls, cudaStream_t st);

struct DevAlloc {
    void *p;
    size_t bytes;
};

struct als_ctx {
    als_config cfg;
    int64_t n_u = 0, n_m = 0, nnz = 0;
    int nf = 0, ld = 0;
    bool f64 = true;
    int dev = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side_stream = nullptr;   // split heavy rows run here, beside the light rows
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    size_t allocated = 0;
    std::vector<DevAlloc> allocs;

    // ratings: by user (CSR) and by item (CSC); rows in degree-descending order
    int64_t *uptr = nullptr, *mptr = nullptr;
    int32_t *uidx = nullptr, *midx = nullptr;
    float *uval = nullptr, *mval = nullptr;
    int32_t *uorder = nullptr, *morder = nullptr;
    int64_t nheavy_u = 0, nheavy_m = 0;
    int64_t maxdeg_u = 0, maxdeg_m = 0;

    // iterate and NCG vectors, (n_u + n_m) x ld each, element size esz
    size_t esz = 8;
    void *X = nullptr, *Xbar = nullptr, *Gbar = nullptr, *G[2] = {nullptr, nullptr}, *P = nullptr;
    int gcur = 0;
    void *tmpvec = nullptr;          // staging for user-supplied vectors

    // deterministic reductions
    double *rowterm = nullptr;   // 5 x (n_u + n_m)
    double *partial = nullptr;   // 5 x RED_MAXB
    unsigned *ticket = nullptr;
    double *S = nullptr;         // S_COUNT scalars
    int *dflags = nullptr;       // [0] rows not SPD, [1] validation errors, [2] duplicates
    double *hS = nullptr;        // pinned host mirror of S
    int *hflags = nullptr;

    // Algorithm 2 state
    bool ncg_ready = false;
    int64_t k = 0;
    bool use_tc = false;

    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};   // kernel nodes per captured iteration

    // launch shapes (defaults, or chosen by als_autotune)
    int heavy_min = ALS_HEAVY_MIN;     // rows with >= this many ratings: a CTA each in the passes
    int grid_mult = 32;                // pass grids: at most grid_mult x sm_count CTAs
    int sweep_bin_min = 0;             // FMA sweep, n_f <= 32: rows with >= this many ratings use a CTA (0: none)
    int64_t sweep_big[2] = {0, 0};     // ... their count per side (a prefix of the degree order)
    int chol_tc = 1;
    int dual_warp = 1;                 // light rows of <= ALS_DUAL_SMALL ratings: a warp per row (1)                   // tensor-core sweep: Cholesky from TMEM, trailing updates as MMAs (1)
    int tc_chunk16 = 0;                // tensor-core sweep, rows below 256 ratings: chunks of 16 ratings (1) or 32 (0)
    int gather_tma = 0;                // tensor-core sweep: heavy rows' factor rows gathered by TMA (1)
                                       // or by cp.async (0)
    int dual_max = ALS_DUAL_MAX;       // mixed tensor-core sweep: rows of <= min(dual_max, n_f) ratings
                                       // are solved through their n_i x n_i matrix (0: none)
    int64_t sweep_dual[2] = {0, 0};    // ... their count per side (a suffix of the degree order)
    int64_t sweep_dual_small[2] = {0, 0};  // ... of which the last ones, of <= ALS_DUAL_SMALL ratings
    int64_t sweep_pf[2] = {0, 0};      // tensor-core sweep: rows of >= ALS_TC_PF_MIN ratings after the
                                       // split rows (a prefix of the rest of the degree order)
    std::vector<int32_t> h_deg[2];     // degrees in degree order (host), filled on first use
    std::vector<int64_t> h_beg[2];     // first rating of each row, in degree order (host)

    // heavy rows split into segments (a prefix of each side's degree order)
    int split_min = 16384;             // rows with >= this many ratings are split
    int seg_len = 4096;                // ratings per segment
    int64_t nsplit[2] = {0, 0};        // split rows per side
    int64_t nseg[2] = {0, 0};          // segments per side
    int32_t *seg_row[2] = {nullptr, nullptr};
    int64_t *seg_beg[2] = {nullptr, nullptr};
    int32_t *seg_len_d[2] = {nullptr, nullptr};
    int32_t *hseg_off[2] = {nullptr, nullptr};   // [nsplit + 1] first segment of each split row
    void *seg_part = nullptr;          // partials: max nseg x seg_stride (element size esz)
    int64_t seg_stride = 0;
    float *hfac = nullptr;             // mixed: factored matrices of the split rows, packed lower triangles
    int32_t *hflag = nullptr;          // mixed: split rows that take another correction

    // batched problems (n_prob > 1): block-diagonal layout, per-problem scalars
    int n_prob = 1;
    int64_t *segu = nullptr, *segm = nullptr;  // device [n_prob + 1] user / item offsets
    int32_t *rowprob = nullptr;                // device [n_u + n_m] problem of each row
    std::vector<int64_t> h_segu, h_segm;

    KTimer *kt = nullptr;                      // set only inside als_time_sweep
};

#define RED_MAXB 512

// Compensated (Kahan) accumulation s += x with the lost low part kept in c
// (the sum is s - c).  Used for the FP32 sums over a row's ratings, which run
// to tens of thousands of terms; for double it is a plain add (FP64 issue is
// scarce on this GPU and its rounding is already far below what the FP64
// form needs).
template <typename T>
__device__ __forceinline__ void kadd(T &s, T &c, T x) {
    if constexpr (sizeof(T) == 4) {
        const T y = x - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    } else {
        s += x;
    }
}

// ---------------------------------------------------------------------------
// error reporting
void als_set_error(const std::string &msg);
#define ALS_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            als_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
            return ALS_ECUDA;                                                           \
        }                                                                               \
    } while (0)

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it: contexts driven from other threads (a
// server's worker, say) may launch the same kernel with a larger size at the
// same time, and a lowered limit would fail their launch.
als_status raise_smem_limit(const void *func, size_t bytes);

// allocation through the configured hooks, counted against the HBM budget
als_status ctx_alloc(als_ctx *c, void **p, size_t bytes);
void ctx_free(als_ctx *c, void *p);

// ---------------------------------------------------------------------------
// builder (builder.cu)
als_status build_ratings(als_ctx *c, const int32_t *rows, const int64_t *rowptr,
                         const int32_t *cols, const float *vals, int on_device);

// ---------------------------------------------------------------------------
// sweep (sweep.cu): one half of Algorithm 1 over a list of rows
struct SweepArgs {
    const int64_t *ptr;     // row r's ratings: [ptr[r], ptr[r+1])
    const int32_t *idx;     // fixed-side ids
    const float *val;       // ratings
    const int32_t *order;   // rows to process, in this order (nullptr = 0..nrows-1)
    int64_t nrows;
    const void *F;          // fixed-side factors, ld-strided (T)
    int64_t nF = 0;         // rows of F (0: unknown; the TMA-fed kernel then is not used)
    const void *Xin;        // current rows (warm start; Gbar = Xin - Xout); may be null
    void *Xout;             // solved rows
    void *Gbar;             // optional Gbar rows
    int nf, ld;
    double lambda;
    int refine;
    int *notspd;
    int *timeout;           // set when a bounded device wait expired
    cudaStream_t stream = nullptr;  // launch stream (nullptr: the context's)
    int64_t nbig = 0;       // FMA sweep: the first nbig rows of `order` get a CTA each
    uint64_t wait_ns = 2000000000ull;  // limit of each bounded device wait
    int withhold = 0;       // self-test of the waits: no MMA is issued, so every wait runs out
    int64_t npf = 0;        // tensor-core sweep: the first npf rows of `order` take the prefetching kernel
    // mixed tensor-core sweep: the last ndual rows of `order` (each with at
    // most dual_nmax <= ALS_DUAL_MAX ratings) take the light-row solve
    int64_t ndual = 0;
    int dual_nmax = 0;
    int64_t ndual_small = 0;   // ... the last of which have at most ALS_DUAL_SMALL ratings
    // mixed form: the gradient rows g_i = -2 (r0 - lambda n_i x_i) of this half,
    // r0 the first FP32 residual at the current row (nullptr: not written)
    void *Gout = nullptr;
    // segment mode (split heavy rows): "row" r is segment r, a slice
    // [seg_beg[r], seg_beg[r] + seg_len[r]) of the ratings of row
    // order[seg_row[r]]; the kernel writes that slice's partial Gram matrix
    // (packed lower triangle, TRI = n_f (n_f + 1) / 2 values) and partial
    // right-hand side (FP64 form) or residual at the row's current value
    // (mixed form), n_f values, to seg_out + r * seg_stride, and solves nothing
    const int32_t *seg_row = nullptr;
    const int64_t *seg_beg = nullptr;
    const int32_t *seg_len = nullptr;
    void *seg_out = nullptr;
    int64_t seg_stride = 0;
};
als_status launch_sweep(als_ctx *c, const SweepArgs &a, bool f64, bool tc);
// heavy rows split across CTAs (sweep_split.cu): segment lists and buffers
// for the current split_min / seg_len, then the split part of a half sweep
als_status load_degrees(als_ctx *c);
als_status build_split(als_ctx *c);
// sweep_dual[] (for the current dual_max, split rows and lambda) and sweep_pf[]
void count_sweep_rows(als_ctx *c);
als_status launch_split_sweep(als_ctx *c, const SweepArgs &a, int side);

// ---------------------------------------------------------------------------
// passes (passes.cu)
struct PassArgs {
    const int64_t *ptr;
    const int32_t *idx;
    const float *val;
    const int32_t *order;
    int64_t row_begin, nrows;   // positions [row_begin, row_begin + nrows) of order
    const void *Xs;             // this side's rows (x)
    const void *Ps;             // this side's direction rows (p), may be null
    const void *Xo;             // other side's rows (x)
    const void *Po;             // other side's direction rows (p), may be null
    void *Gout;                 // gradient rows out
    const void *Gbar;           // this side's gbar rows (may be null)
    const void *Gprev;          // this side's previous gradient rows (may be null)
    int nf, ld;
    double lambda;
    double *rowterm;            // rowterm[t * stride + rowoff + row]
    int64_t stride, rowoff;
};
als_status launch_grad(als_ctx *c, const PassArgs &a, bool heavy);
// the row terms of gradient rows already in a.Gout (rows 0 .. nrows - 1)
als_status launch_grad_terms(als_ctx *c, const PassArgs &a);
als_status launch_lscoef(als_ctx *c, const PassArgs &a, bool heavy);
als_status launch_lscoef_reg(als_ctx *c, const PassArgs &a);  // rows without rating terms
als_status launch_reduce(als_ctx *c, int nterms, int64_t n, int s_off, int post,
                         const LsParams &lp);
als_status launch_update_x(als_ctx *c);   // x <- x + alpha p, or x <- xbar on fallback
als_status launch_update_p(als_ctx *c);   // p <- -gbar + beta p
als_status launch_neg_copy(als_ctx *c, void *dst, const void *src, size_t n);  // dst = -src
als_status launch_convert_in(als_ctx *c, void *dst, const void *src, int64_t rows, int src_dtype,
                             int src_ld);
als_status launch_convert_out(als_ctx *c, void *dst, const void *src, int64_t rows, int dst_dtype,
                              int dst_ld);
// batched problems: local ids + per-problem offsets -> global ids (and checks)
als_status launch_offset_ids(als_ctx *c, const int64_t *nnzoff, int n_prob, const int64_t *segu,
                             const int64_t *segm, int32_t *rows, int32_t *cols, int64_t nnz, int *flag);
als_status launch_rowprob(als_ctx *c);
als_status launch_check_requests(als_ctx *c, const int64_t *ptr, int64_t nreq, const int32_t *idx,
                                 const float *val, int64_t total, int64_t bound, int *flag);
