// C ABI (include/als.h) and the host drivers of Algorithm 1 (ALS) and
// Algorithm 2 (ALS-NCG).  The host only enqueues kernels: every arithmetic
// step runs on the device, and the scalar decisions of Algorithm 2/3
// (alpha, beta-bar, the fallback) are taken by device code, so an iteration
// needs no host round trip and can be replayed as a CUDA graph.
//
// One Algorithm 2 iteration, k -> k+1 (x, p, g_k, gbar_k, s_k = gbar_k.g_k on
// the device):
//   1. Q coefficients c0..c4 at (x_k, p_k), one by-user pass (§V-C);
//   2. Algorithm 3 on Q -> alpha_k (or the ALS-point fallback);
//   3. x_{k+1} = x_k + alpha_k p_k;
//   4. xbar = P(x_{k+1}) (U half, then M half), gbar_{k+1} = x_{k+1} - xbar;
//   5. g_{k+1} = grad f(x_{k+1}) with gbar.g and gbar.(g_{k+1} - g_k) fused;
//   6. beta-bar (Eq. 8), p_{k+1} = -gbar_{k+1} + beta-bar p_k.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.cuh"

static thread_local std::string g_err;

void als_set_error(const std::string &msg) { g_err = msg; }

extern "C" const char *als_last_error(void) { return g_err.c_str(); }

als_status raise_smem_limit(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    ALS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[{dev, func}];
    if (bytes > cur) {
        ALS_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        cur = bytes;
    }
    return ALS_OK;
}

extern "C" const char *als_version(void) { return "als-ncg-gb300 1.0 (sm_103a)"; }

als_status ctx_alloc(als_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (c->cfg.hbm_budget_bytes && c->allocated + bytes > c->cfg.hbm_budget_bytes) {
        als_set_error("allocation of " + std::to_string(bytes) + " bytes exceeds hbm_budget_bytes");
        return ALS_EBUDGET;
    }
    if (c->cfg.alloc) {
        *p = c->cfg.alloc(bytes, (void *)c->stream, c->cfg.alloc_user);
        if (!*p) {
            als_set_error("allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
            return ALS_ENOMEM;
        }
    } else {
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            als_set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return ALS_ENOMEM;
        }
    }
    c->allocs.push_back({*p, bytes});
    c->allocated += bytes;
    return ALS_OK;
}

void ctx_free(als_ctx *c, void *p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i) {
        if (c->allocs[i].p == p) {
            const size_t bytes = c->allocs[i].bytes;
            if (c->cfg.free) c->cfg.free(p, bytes, (void *)c->stream, c->cfg.alloc_user);
            else cudaFree(p);
            c->allocated -= bytes;
            c->allocs.erase(c->allocs.begin() + (long)i);
            return;
        }
    }
}

namespace {

bool valid_dtype(int d) { return d == ALS_DT_F64 || d == ALS_DT_F32; }
size_t dtype_size(int d) { return d == ALS_DT_F64 ? 8 : 4; }

LsParams ls_params(const als_ctx *c) {
    LsParams p;
    p.alpha0 = c->cfg.ls_alpha0;
    p.tau = c->cfg.ls_tau;
    p.c = c->cfg.ls_c;
    p.max_shrinks = c->cfg.ls_max_shrinks;
    p.mode = c->cfg.ls_mode;
    p.c2 = c->cfg.ls_c2;
    p.beta = c->cfg.beta_form;
    return p;
}

char *vrow(const als_ctx *c, void *v, int64_t row) { return (char *)v + (size_t)row * c->ld * c->esz; }
void *ublk(const als_ctx *c, void *v) { return v; }
void *mblk(const als_ctx *c, void *v) { return vrow(c, v, c->n_u); }

// One half of P(x): side 0 solves users from the M rows in F_M, side 1 items
// from the U rows in F_U.
als_status half_sweep(als_ctx *c, int side, const void *F, const void *Xin, void *Xout, void *Gbar,
                      void *Gout = nullptr) {
    SweepArgs a;
    a.ptr = side ? c->mptr : c->uptr;
    a.idx = side ? c->midx : c->uidx;
    a.val = side ? c->mval : c->uval;
    a.order = side ? c->morder : c->uorder;
    a.nrows = side ? c->n_m : c->n_u;
    a.F = F;
    a.nF = side ? c->n_u : c->n_m;
    a.Xin = Xin;
    a.Xout = Xout;
    a.Gbar = Gbar;
    a.Gout = Gout;
    a.nf = c->nf;
    a.ld = c->ld;
    a.lambda = c->cfg.lambda;
    a.refine = c->cfg.refine_steps;
    a.notspd = c->dflags;
    a.timeout = c->dflags + 7;
    a.nbig = c->sweep_big[side];
    a.ndual = c->sweep_dual[side];
    a.ndual_small = c->sweep_dual_small[side];
    a.npf = c->sweep_pf[side];
    a.dual_nmax = std::min(c->dual_max, c->nf);
    const int64_t H = c->nsplit[side];
    if (H == 0) return launch_sweep(c, a, c->f64, c->use_tc);
    if (c->kt && c->kt->serial) {
        // per-kernel timing: every launch on the context's stream, so that
        // each one's events time it alone
        als_status s = launch_split_sweep(c, a, side);
        if (s != ALS_OK) return s;
        a.order += H;
        a.nrows -= H;
        a.nbig = std::max<int64_t>(0, a.nbig - H);
        return launch_sweep(c, a, c->f64, c->use_tc);
    }
    // the heaviest rows, split across CTAs, on the side stream; the rest, one
    // CTA (or warp) each, beside them on the context's stream (inside a
    // captured iteration the two become parallel branches of the graph)
    ALS_CUDA_TRY(cudaEventRecord(c->ev_fork, c->stream));
    ALS_CUDA_TRY(cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    SweepArgs h = a;
    h.stream = c->side_stream;
    als_status s = launch_split_sweep(c, h, side);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaEventRecord(c->ev_join, c->side_stream));
    a.order += H;
    a.nrows -= H;
    a.nbig = std::max<int64_t>(0, a.nbig - H);
    s = launch_sweep(c, a, c->f64, c->use_tc);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    return ALS_OK;
}

// xbar = P(x) with gbar = x - xbar, or in place (x <- P(x)) when Xout == X.
// G (may be null): with the fused gradient, the users' rows of grad f(X)
// are written into G by the U half (its first residuals)
als_status sweep_into(als_ctx *c, void *X, void *Xout, void *Gbar, void *G = nullptr) {
    als_status s = half_sweep(c, 0, mblk(c, X), ublk(c, X), ublk(c, Xout), Gbar ? ublk(c, Gbar) : nullptr,
                              G ? ublk(c, G) : nullptr);
    if (s != ALS_OK) return s;
    return half_sweep(c, 1, ublk(c, Xout), mblk(c, X), mblk(c, Xout), Gbar ? mblk(c, Gbar) : nullptr);
}

// The mixed tensor-core sweep forms, for every user row, the FP32 residual
// r0 = sum_e f_e (r_e - f_e . x_i) at the current row, whose -2 (r0 -
// lambda n_i x_i) is that row of grad f(x): so P(x) can write the users'
// gradient rows and the gradient pass then forms only their FP64 terms (the
// items' rows need U of x, not the new U of the sweep's first half).  The
// FMA sweeps (FP64 form, n_f <= 32) form the right-hand side instead.
bool fused_grad(const als_ctx *c) { return c->use_tc && !c->f64; }

PassArgs pass_args(const als_ctx *c, int side) {
    PassArgs a;
    std::memset(&a, 0, sizeof a);
    a.ptr = side ? c->mptr : c->uptr;
    a.idx = side ? c->midx : c->uidx;
    a.val = side ? c->mval : c->uval;
    a.order = side ? c->morder : c->uorder;
    a.nf = c->nf;
    a.ld = c->ld;
    a.lambda = c->cfg.lambda;
    a.rowterm = c->rowterm;
    a.stride = c->n_u + c->n_m;
    a.rowoff = side ? c->n_u : 0;
    return a;
}

// gradient of Eq. (1) at X into Gout; per-row terms |g|^2, gbar.g,
// gbar.(g-gprev) and, with P (the Hestenes-Stiefel form of beta-bar),
// p.(g-gprev).  Gbar == Gout: gbar is the gradient itself (plain NCG).
// users_written: the users' gradient rows are already in Gout (the fused
// sweep), only their row terms are formed
als_status grad_into(als_ctx *c, void *X, void *Gout, void *Gbar, void *Gprev, void *P = nullptr,
                     bool users_written = false) {
    for (int side = 0; side < 2; ++side) {
        PassArgs a = pass_args(c, side);
        a.Xs = side ? mblk(c, X) : ublk(c, X);
        a.Xo = side ? ublk(c, X) : mblk(c, X);
        a.Gout = side ? mblk(c, Gout) : ublk(c, Gout);
        a.Gbar = Gbar ? (side ? mblk(c, Gbar) : ublk(c, Gbar)) : nullptr;
        a.Gprev = Gprev ? (side ? mblk(c, Gprev) : ublk(c, Gprev)) : nullptr;
        a.Ps = (P && Gprev) ? (side ? mblk(c, P) : ublk(c, P)) : nullptr;
        const int64_t n = side ? c->n_m : c->n_u;
        const int64_t nh = side ? c->nheavy_m : c->nheavy_u;
        if (side == 0 && users_written) {
            a.row_begin = 0;
            a.nrows = n;
            als_status s = launch_grad_terms(c, a);
            if (s != ALS_OK) return s;
            continue;
        }
        a.row_begin = 0;
        a.nrows = nh;
        als_status s = launch_grad(c, a, true);
        if (s != ALS_OK) return s;
        a.row_begin = nh;
        a.nrows = n - nh;
        s = launch_grad(c, a, false);
        if (s != ALS_OK) return s;
    }
    return ALS_OK;
}

// Q coefficients at (X, P) (P == nullptr: only c0 = f(X)) into rowterm
als_status lscoef_into(als_ctx *c, void *X, void *P) {
    PassArgs a = pass_args(c, 0);
    a.Xs = ublk(c, X);
    a.Xo = mblk(c, X);
    a.Ps = P ? ublk(c, P) : nullptr;
    a.Po = P ? mblk(c, P) : nullptr;
    a.row_begin = 0;
    a.nrows = c->nheavy_u;
    als_status s = launch_lscoef(c, a, true);
    if (s != ALS_OK) return s;
    a.row_begin = c->nheavy_u;
    a.nrows = c->n_u - c->nheavy_u;
    s = launch_lscoef(c, a, false);
    if (s != ALS_OK) return s;
    PassArgs b = pass_args(c, 1);
    b.Xs = mblk(c, X);
    b.Ps = P ? mblk(c, P) : nullptr;
    b.row_begin = 0;
    b.nrows = c->n_m;
    return launch_lscoef_reg(c, b);
}

als_status read_scalars(als_ctx *c) {
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hS, c->S, (size_t)c->n_prob * S_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->hflags[7]) {
        // reported once: the flag is cleared here, so that the context runs
        // again after the caller restores a checkpoint (als_set_state) or
        // sets new factors; what was computed since the expiry is not valid
        c->hflags[7] = 0;
        ALS_CUDA_TRY(cudaMemsetAsync(c->dflags + 7, 0, sizeof(int), c->stream));
        ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        als_set_error("a bounded device wait of the tensor-core sweep expired; results since the last "
                      "successful call are not valid: restore a checkpoint (als_set_state) or set new factors");
        return ALS_ETIMEOUT;
    }
    return ALS_OK;
}

bool plain_ncg(const als_ctx *c) { return c->cfg.preconditioner == ALS_PRECOND_NONE; }

// plain NCG: gbar = g (copied from the gradient just formed) and xbar = x
// (a failed line search keeps x and restarts along -g)
als_status plain_gbar(als_ctx *c, void *G) {
    const size_t bytes = (size_t)(c->n_u + c->n_m) * c->ld * c->esz;
    ALS_CUDA_TRY(cudaMemcpyAsync(c->Gbar, G, bytes, cudaMemcpyDeviceToDevice, c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->Xbar, c->X, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return ALS_OK;
}

als_status ncg_init(als_ctx *c) {
    // gbar_0 = x_0 - P(x_0), g_0 = grad f(x_0), p_0 = -gbar_0, s_0 = gbar_0 . g_0
    als_status s;
    if (plain_ncg(c)) {
        s = grad_into(c, c->X, c->G[c->gcur], c->G[c->gcur], nullptr);
        if (s != ALS_OK) return s;
        s = plain_gbar(c, c->G[c->gcur]);
    } else {
        const bool fg = fused_grad(c);
        s = sweep_into(c, c->X, c->Xbar, c->Gbar, fg ? c->G[c->gcur] : nullptr);
        if (s != ALS_OK) return s;
        s = grad_into(c, c->X, c->G[c->gcur], c->Gbar, nullptr, nullptr, fg);
    }
    if (s != ALS_OK) return s;
    s = launch_reduce(c, 3, c->n_u + c->n_m, S_RED, POST_INIT, ls_params(c));
    if (s != ALS_OK) return s;
    s = launch_neg_copy(c, c->P, c->Gbar, (size_t)(c->n_u + c->n_m) * c->ld);
    if (s != ALS_OK) return s;
    c->ncg_ready = true;
    c->k = 0;
    return ALS_OK;
}

// enqueue one Algorithm 2 iteration (graph-capturable: no host sync)
als_status ncg_iter(als_ctx *c, int gcur) {
    als_status s = lscoef_into(c, c->X, c->P);
    if (s != ALS_OK) return s;
    s = launch_reduce(c, 5, c->n_u + c->n_m, S_C, POST_LSELECT, ls_params(c));
    if (s != ALS_OK) return s;
    s = launch_update_x(c);
    if (s != ALS_OK) return s;
    const bool hs = c->cfg.beta_form == ALS_BETA_HS;
    if (plain_ncg(c)) {
        s = grad_into(c, c->X, c->G[gcur ^ 1], c->G[gcur ^ 1], c->G[gcur], hs ? c->P : nullptr);
        if (s != ALS_OK) return s;
        s = plain_gbar(c, c->G[gcur ^ 1]);
    } else {
        const bool fg = fused_grad(c);
        s = sweep_into(c, c->X, c->Xbar, c->Gbar, fg ? c->G[gcur ^ 1] : nullptr);
        if (s != ALS_OK) return s;
        s = grad_into(c, c->X, c->G[gcur ^ 1], c->Gbar, c->G[gcur], hs ? c->P : nullptr, fg);
    }
    if (s != ALS_OK) return s;
    s = launch_reduce(c, hs ? 4 : 3, c->n_u + c->n_m, S_RED, POST_BETA, ls_params(c));
    if (s != ALS_OK) return s;
    return launch_update_p(c);
}

// sum over the problems of a per-problem scalar slot (one problem: the slot)
double sum_slot(const als_ctx *c, int slot) {
    double s = 0.0;
    for (int q = 0; q < c->n_prob; ++q) s += c->hS[(size_t)q * S_COUNT + slot];
    return s;
}

// the worst problem's |g_k| / |g_0|
double worst_rel_gnorm(const als_ctx *c) {
    double w = 0.0;
    for (int q = 0; q < c->n_prob; ++q) {
        const double *S = c->hS + (size_t)q * S_COUNT;
        const double r = S[S_GG0] > 0.0 ? std::sqrt(S[S_GG] / S[S_GG0]) : 0.0;
        w = std::max(w, r);
    }
    return w;
}

void fill_info_q(const als_ctx *c, int q, als_iter_info *o) {
    const double *S = c->hS + (size_t)q * S_COUNT;
    o->k = c->k;
    o->f = S[S_F];
    o->gnorm = std::sqrt(S[S_GG]);
    o->gnorm0 = std::sqrt(S[S_GG0]);
    o->alpha = S[S_ALPHA];
    o->beta = S[S_BETA];
    for (int i = 0; i < 5; ++i) o->c[i] = S[S_C + i];
    o->shrinks = (int32_t)S[S_SHRINK];
    o->fallback = S[S_MODE] != 0.0;
    o->fallbacks = (int64_t)S[S_NFALL];
    o->notspd = c->hflags[0];
    o->kernels = 0;
}

// one record for the whole context: problem 0, or for a batch the sums of f
// and |g|^2 over the problems (alpha, beta, c: problem 0)
void fill_info(const als_ctx *c, als_iter_info *o) {
    fill_info_q(c, 0, o);
    if (c->n_prob > 1) {
        o->f = sum_slot(c, S_F);
        o->gnorm = std::sqrt(sum_slot(c, S_GG));
        o->gnorm0 = std::sqrt(sum_slot(c, S_GG0));
        o->fallbacks = (int64_t)sum_slot(c, S_NFALL);
    }
}

als_status loss_now(als_ctx *c, double *f) {
    als_status s = lscoef_into(c, c->X, nullptr);
    if (s != ALS_OK) return s;
    s = launch_reduce(c, 1, c->n_u + c->n_m, S_RED, POST_NONE, ls_params(c));
    if (s != ALS_OK) return s;
    s = read_scalars(c);
    if (s != ALS_OK) return s;
    *f = sum_slot(c, S_RED);
    return ALS_OK;
}

void destroy_graphs(als_ctx *c) {
    for (int i = 0; i < 2; ++i) {
        if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
        c->graph[i] = nullptr;
    }
}

als_status capture_graphs(als_ctx *c) {
    for (int p = 0; p < 2; ++p) {
        if (c->graph[p]) continue;
        cudaGraph_t g = nullptr;
        ALS_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        als_status s = ncg_iter(c, p);
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s != ALS_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) {
            als_set_error(std::string("graph capture: ") + cudaGetErrorString(e));
            return ALS_ECUDA;
        }
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        int64_t nk = 0;
        for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
        }
        c->graph_kernels[p] = nk;
        const cudaError_t e2 = cudaGraphInstantiate(&c->graph[p], g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            c->graph[p] = nullptr;
            als_set_error(std::string("graph instantiate: ") + cudaGetErrorString(e2));
            return ALS_ECUDA;
        }
    }
    return ALS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" void als_config_default(als_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->n_f = 10;
    cfg->lambda = 0.05;
    cfg->precision = ALS_FP64;
    cfg->ls_mode = ALS_LS_BACKTRACK;
    cfg->ls_alpha0 = 10.0;
    cfg->ls_tau = 0.9;
    cfg->ls_c = 0.5;
    cfg->ls_max_shrinks = 200;
    cfg->refine_steps = 2;
    cfg->gram_path = ALS_GRAM_AUTO;
    cfg->beta_form = ALS_BETA_PR;
    cfg->preconditioner = ALS_PRECOND_ALS;
    cfg->ls_c2 = 1e-2;
}

namespace {
// batched problems: per-problem sizes (host) for create_impl
struct BatchSpec {
    int n_prob;
    std::vector<int64_t> segu, segm, nnzoff;  // prefix sums, n_prob + 1 entries each
};
}  // namespace

static als_status create_impl(const als_config *cfg, int64_t n_u, int64_t n_m, int64_t nnz,
                              const int32_t *rows_or_null, const int64_t *rowptr_or_null, const int32_t *cols,
                              const float *vals, int on_device, void *cuda_stream, als_ctx **out,
                              const BatchSpec *bs);

extern "C" als_status als_create(const als_config *cfg, int64_t n_u, int64_t n_m, int64_t nnz,
                                 const int32_t *rows_or_null, const int64_t *rowptr_or_null,
                                 const int32_t *cols, const float *vals, int on_device, void *cuda_stream,
                                 als_ctx **out) {
    return create_impl(cfg, n_u, n_m, nnz, rows_or_null, rowptr_or_null, cols, vals, on_device, cuda_stream, out,
                       nullptr);
}

extern "C" als_status als_create_batched(const als_config *cfg, int32_t n_prob, const int64_t *n_u,
                                         const int64_t *n_m, const int64_t *nnz, const int32_t *rows,
                                         const int32_t *cols, const float *vals, int on_device, void *cuda_stream,
                                         als_ctx **out) {
    if (!out) { als_set_error("als_create_batched: out is NULL"); return ALS_EINVAL; }
    *out = nullptr;
    if (n_prob < 1 || n_prob > (1 << 20) || !n_u || !n_m || !nnz) {
        als_set_error("als_create_batched: need 1 <= n_prob <= 2^20 and per-problem size arrays");
        return ALS_EINVAL;
    }
    BatchSpec bs;
    bs.n_prob = n_prob;
    bs.segu.assign(1, 0);
    bs.segm.assign(1, 0);
    bs.nnzoff.assign(1, 0);
    for (int q = 0; q < n_prob; ++q) {
        if (n_u[q] < 1 || n_m[q] < 1 || nnz[q] < 0) {
            als_set_error("als_create_batched: every problem needs n_u, n_m >= 1 and nnz >= 0");
            return ALS_EINVAL;
        }
        bs.segu.push_back(bs.segu.back() + n_u[q]);
        bs.segm.push_back(bs.segm.back() + n_m[q]);
        bs.nnzoff.push_back(bs.nnzoff.back() + nnz[q]);
    }
    return create_impl(cfg, bs.segu.back(), bs.segm.back(), bs.nnzoff.back(), rows, nullptr, cols, vals, on_device,
                       cuda_stream, out, &bs);
}

static als_status create_impl(const als_config *cfg, int64_t n_u, int64_t n_m, int64_t nnz,
                              const int32_t *rows_or_null, const int64_t *rowptr_or_null, const int32_t *cols,
                              const float *vals, int on_device, void *cuda_stream, als_ctx **out,
                              const BatchSpec *bs) {
    if (!out) { als_set_error("als_create: out is NULL"); return ALS_EINVAL; }
    *out = nullptr;
    if (!cfg) { als_set_error("als_create: cfg is NULL"); return ALS_EINVAL; }
    if (cfg->n_f < 1 || cfg->n_f > ALS_MAX_NF) { als_set_error("als_create: n_f must be in 1..128"); return ALS_EINVAL; }
    if (!(cfg->lambda >= 0.0) || !std::isfinite(cfg->lambda)) { als_set_error("als_create: lambda must be finite and >= 0"); return ALS_EINVAL; }
    if (cfg->precision != ALS_FP64 && cfg->precision != ALS_MIXED) { als_set_error("als_create: bad precision"); return ALS_EINVAL; }
    if (cfg->ls_mode != ALS_LS_BACKTRACK && cfg->ls_mode != ALS_LS_EXACT && cfg->ls_mode != ALS_LS_MORE_THUENTE) {
        als_set_error("als_create: bad ls_mode");
        return ALS_EINVAL;
    }
    if (cfg->beta_form < ALS_BETA_PR || cfg->beta_form > ALS_BETA_PR_PLUS) { als_set_error("als_create: bad beta_form"); return ALS_EINVAL; }
    if (cfg->preconditioner != ALS_PRECOND_ALS && cfg->preconditioner != ALS_PRECOND_NONE) {
        als_set_error("als_create: bad preconditioner");
        return ALS_EINVAL;
    }
    if (cfg->ls_mode == ALS_LS_MORE_THUENTE && !(cfg->ls_c2 > cfg->ls_c && cfg->ls_c2 < 1.0 && cfg->ls_max_shrinks >= 1)) {
        als_set_error("als_create: the More-Thuente search needs 0 < ls_c < ls_c2 < 1 and ls_max_shrinks >= 1");
        return ALS_EINVAL;
    }
    if (!(cfg->ls_alpha0 > 0) || !(cfg->ls_tau > 0 && cfg->ls_tau < 1) || !(cfg->ls_c > 0 && cfg->ls_c < 1) || cfg->ls_max_shrinks < 0) {
        als_set_error("als_create: line-search parameters need alpha0 > 0, 0 < tau < 1, 0 < c < 1");
        return ALS_EINVAL;
    }
    if (cfg->refine_steps < 1 || cfg->refine_steps > 8) { als_set_error("als_create: refine_steps must be 1..8"); return ALS_EINVAL; }
    if (n_u < 1 || n_m < 1 || n_u >= (1ll << 31) || n_m >= (1ll << 31) || nnz < 0 || nnz >= (1ll << 40)) {
        als_set_error("als_create: need 1 <= n_u, n_m < 2^31 and 0 <= nnz < 2^40");
        return ALS_EINVAL;
    }
    if (nnz > 0 && (!cols || !vals || (!rows_or_null && !rowptr_or_null))) {
        als_set_error("als_create: ratings arrays are NULL");
        return ALS_EINVAL;
    }
    if (rowptr_or_null == nullptr && nnz > 0 && rows_or_null == nullptr) { als_set_error("als_create: rows is NULL"); return ALS_EINVAL; }
    if (nnz >= (1ll << 32)) { als_set_error("als_create: nnz >= 2^32 is not supported by the builder"); return ALS_ENOTSUP; }

    als_ctx *c = new als_ctx();
    c->cfg = *cfg;
    c->n_u = n_u; c->n_m = n_m; c->nnz = nnz;
    c->nf = cfg->n_f;
    c->ld = (cfg->n_f + 3) & ~3;
    c->f64 = cfg->precision == ALS_FP64;
    c->esz = c->f64 ? 8 : 4;
    auto fail = [&](als_status s) { als_destroy(c); return s; };
    if (cudaGetDevice(&c->dev) != cudaSuccess) { cudaGetLastError(); als_set_error("als_create: no CUDA device"); return fail(ALS_ECUDA); }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->dev) != cudaSuccess) { cudaGetLastError(); als_set_error("als_create: cudaGetDeviceProperties failed"); return fail(ALS_ECUDA); }
    if (!(prop.major == 10 && prop.minor == 3)) {
        char b[160];
        snprintf(b, sizeof b, "als_create: this library is built for sm_103a (GB300); device is sm_%d%d", prop.major, prop.minor);
        als_set_error(b);
        return fail(ALS_ENOTSUP);
    }
    c->sm_count = prop.multiProcessorCount;
    c->stream = (cudaStream_t)cuda_stream;
    if (!c->stream) {
        // the legacy default stream cannot be captured into a graph: own a stream
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            als_set_error("als_create: cudaStreamCreateWithFlags failed");
            return fail(ALS_ECUDA);
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        als_set_error("als_create: stream or event creation failed");
        return fail(ALS_ECUDA);
    }
    c->use_tc = !c->f64 && c->nf > 32 && cfg->gram_path != ALS_GRAM_FMA;
    if (cfg->gram_path == ALS_GRAM_TC && c->f64) { als_set_error("als_create: the tensor-core Gram needs ALS_MIXED"); return fail(ALS_EINVAL); }
    if (cfg->gram_path == ALS_GRAM_TC) c->use_tc = true;

    const int64_t nrows = n_u + n_m;
    const size_t vbytes = (size_t)nrows * c->ld * c->esz;
    als_status s;
#define ALLOC(ptr, bytes) do { void *_p = nullptr; s = ctx_alloc(c, &_p, (bytes)); if (s != ALS_OK) return fail(s); ptr = (decltype(ptr))_p; } while (0)
    ALLOC(c->uptr, (n_u + 1) * sizeof(int64_t));
    ALLOC(c->mptr, (n_m + 1) * sizeof(int64_t));
    ALLOC(c->uidx, nnz * sizeof(int32_t));
    ALLOC(c->midx, nnz * sizeof(int32_t));
    ALLOC(c->uval, nnz * sizeof(float));
    ALLOC(c->mval, nnz * sizeof(float));
    ALLOC(c->uorder, n_u * sizeof(int32_t));
    ALLOC(c->morder, n_m * sizeof(int32_t));
    ALLOC(c->X, vbytes);
    ALLOC(c->Xbar, vbytes);
    ALLOC(c->Gbar, vbytes);
    ALLOC(c->G[0], vbytes);
    ALLOC(c->G[1], vbytes);
    ALLOC(c->P, vbytes);
    ALLOC(c->tmpvec, (size_t)nrows * c->ld * 8);
    ALLOC(c->rowterm, 5 * (size_t)nrows * sizeof(double));
    ALLOC(c->partial, 5 * RED_MAXB * sizeof(double));
    ALLOC(c->ticket, 256);
    c->n_prob = bs ? bs->n_prob : 1;
    ALLOC(c->S, (size_t)c->n_prob * S_COUNT * sizeof(double));
    ALLOC(c->dflags, 16 * sizeof(int));
    if (bs) {
        ALLOC(c->segu, (bs->n_prob + 1) * sizeof(int64_t));
        ALLOC(c->segm, (bs->n_prob + 1) * sizeof(int64_t));
        ALLOC(c->rowprob, nrows * sizeof(int32_t));
        c->h_segu = bs->segu;
        c->h_segm = bs->segm;
    }
#undef ALLOC
    if (cudaMallocHost(&c->hS, (size_t)c->n_prob * S_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hflags, 16 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        als_set_error("als_create: pinned host allocation failed");
        return fail(ALS_ENOMEM);
    }
    for (void *p : {c->X, c->Xbar, c->Gbar, c->G[0], c->G[1], c->P}) {
        if (cudaMemsetAsync(p, 0, vbytes, c->stream) != cudaSuccess) { cudaGetLastError(); als_set_error("als_create: memset failed"); return fail(ALS_ECUDA); }
    }
    if (cudaMemsetAsync(c->ticket, 0, 256, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->S, 0, (size_t)c->n_prob * S_COUNT * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->dflags, 0, 16 * sizeof(int), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->rowterm, 0, 5 * (size_t)nrows * sizeof(double), c->stream) != cudaSuccess) {
        cudaGetLastError();
        als_set_error("als_create: memset failed");
        return fail(ALS_ECUDA);
    }
    if (bs) {
        // batched: per-problem local ids -> global ids of the block-diagonal problem
        int32_t *drows = nullptr, *dcols = nullptr;
        float *dvals = nullptr;
        int64_t *dnnz = nullptr;
        auto tmp = [&](void **p, size_t b) { return ctx_alloc(c, p, b); };
        if ((s = tmp((void **)&drows, std::max<int64_t>(nnz, 1) * sizeof(int32_t))) != ALS_OK) return fail(s);
        if ((s = tmp((void **)&dcols, std::max<int64_t>(nnz, 1) * sizeof(int32_t))) != ALS_OK) return fail(s);
        if ((s = tmp((void **)&dvals, std::max<int64_t>(nnz, 1) * sizeof(float))) != ALS_OK) return fail(s);
        if ((s = tmp((void **)&dnnz, (bs->n_prob + 1) * sizeof(int64_t))) != ALS_OK) return fail(s);
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        bool okc = cudaMemcpyAsync(c->segu, bs->segu.data(), (bs->n_prob + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
                   cudaMemcpyAsync(c->segm, bs->segm.data(), (bs->n_prob + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
                   cudaMemcpyAsync(dnnz, bs->nnzoff.data(), (bs->n_prob + 1) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
        if (okc && nnz > 0)
            okc = cudaMemcpyAsync(drows, rows_or_null, nnz * sizeof(int32_t), kind, c->stream) == cudaSuccess &&
                  cudaMemcpyAsync(dcols, cols, nnz * sizeof(int32_t), kind, c->stream) == cudaSuccess &&
                  cudaMemcpyAsync(dvals, vals, nnz * sizeof(float), kind, c->stream) == cudaSuccess;
        if (!okc) {
            als_set_error(std::string("als_create_batched: copy failed: ") + cudaGetErrorString(cudaGetLastError()));
            return fail(ALS_ECUDA);
        }
        if ((s = launch_offset_ids(c, dnnz, bs->n_prob, c->segu, c->segm, drows, dcols, nnz, c->dflags + 8)) != ALS_OK)
            return fail(s);
        if ((s = launch_rowprob(c)) != ALS_OK) return fail(s);
        int bad = 0;
        if (cudaMemcpyAsync(&bad, c->dflags + 8, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            als_set_error("als_create_batched: synchronisation failed");
            return fail(ALS_ECUDA);
        }
        if (bad) {
            als_set_error("als_create_batched: " + std::to_string(bad) + " ratings with a local id out of range");
            return fail(ALS_EINVAL);
        }
        s = build_ratings(c, drows, nullptr, dcols, dvals, 1);
        ctx_free(c, drows);
        ctx_free(c, dcols);
        ctx_free(c, dvals);
        ctx_free(c, dnnz);
    } else {
        s = build_ratings(c, rows_or_null, rowptr_or_null, cols, vals, on_device);
    }
    if (s != ALS_OK) return fail(s);
    s = build_split(c);  // segment lists of the heaviest rows
    if (s != ALS_OK) return fail(s);
    count_sweep_rows(c);
    if (cudaMemsetAsync(c->dflags, 0, 16 * sizeof(int), c->stream) != cudaSuccess) { cudaGetLastError(); return fail(ALS_ECUDA); }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        als_set_error(std::string("als_create: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(ALS_ECUDA);
    }
    *out = c;
    return ALS_OK;
}

extern "C" als_status als_get_ratings(als_ctx *c, int64_t *uptr, int32_t *uidx, float *uval, int64_t *mptr,
                                      int32_t *midx, float *mval, int32_t *uorder, int32_t *morder) {
    if (!c) { als_set_error("als_get_ratings: ctx is NULL"); return ALS_EINVAL; }
    const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
    if (uptr) ALS_CUDA_TRY(cudaMemcpyAsync(uptr, c->uptr, (c->n_u + 1) * sizeof(int64_t), k, c->stream));
    if (mptr) ALS_CUDA_TRY(cudaMemcpyAsync(mptr, c->mptr, (c->n_m + 1) * sizeof(int64_t), k, c->stream));
    if (c->nnz > 0) {
        if (uidx) ALS_CUDA_TRY(cudaMemcpyAsync(uidx, c->uidx, c->nnz * sizeof(int32_t), k, c->stream));
        if (uval) ALS_CUDA_TRY(cudaMemcpyAsync(uval, c->uval, c->nnz * sizeof(float), k, c->stream));
        if (midx) ALS_CUDA_TRY(cudaMemcpyAsync(midx, c->midx, c->nnz * sizeof(int32_t), k, c->stream));
        if (mval) ALS_CUDA_TRY(cudaMemcpyAsync(mval, c->mval, c->nnz * sizeof(float), k, c->stream));
    }
    if (uorder) ALS_CUDA_TRY(cudaMemcpyAsync(uorder, c->uorder, c->n_u * sizeof(int32_t), k, c->stream));
    if (morder) ALS_CUDA_TRY(cudaMemcpyAsync(morder, c->morder, c->n_m * sizeof(int32_t), k, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ALS_OK;
}

extern "C" als_status als_set_factors(als_ctx *c, const void *U, const void *M, int dtype, int on_device) {
    if (!c || !U || !M || !valid_dtype(dtype)) { als_set_error("als_set_factors: bad argument"); return ALS_EINVAL; }
    const size_t es = dtype_size(dtype);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ALS_CUDA_TRY(cudaMemcpyAsync(c->tmpvec, U, (size_t)c->n_u * c->nf * es, kind, c->stream));
    als_status s = launch_convert_in(c, c->X, c->tmpvec, c->n_u, dtype, c->nf);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaMemcpyAsync(c->tmpvec, M, (size_t)c->n_m * c->nf * es, kind, c->stream));
    s = launch_convert_in(c, mblk(c, c->X), c->tmpvec, c->n_m, dtype, c->nf);
    if (s != ALS_OK) return s;
    // new factors: an unreported expiry of a bounded wait no longer matters
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags + 7, 0, sizeof(int), c->stream));
    if (!on_device) ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->ncg_ready = false;
    c->k = 0;
    return ALS_OK;
}

extern "C" als_status als_get_factors(als_ctx *c, void *U, void *M, int dtype, int on_device) {
    if (!c || !U || !M || !valid_dtype(dtype)) { als_set_error("als_get_factors: bad argument"); return ALS_EINVAL; }
    const size_t es = dtype_size(dtype);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    als_status s = launch_convert_out(c, c->tmpvec, c->X, c->n_u, dtype, c->nf);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaMemcpyAsync(U, c->tmpvec, (size_t)c->n_u * c->nf * es, kind, c->stream));
    if (!on_device) ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    s = launch_convert_out(c, c->tmpvec, mblk(c, c->X), c->n_m, dtype, c->nf);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaMemcpyAsync(M, c->tmpvec, (size_t)c->n_m * c->nf * es, kind, c->stream));
    if (!on_device) ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ALS_OK;
}

extern "C" als_status als_get_state(als_ctx *c, void *x, void *p, void *g, void *gbar, void *xbar,
                                    double scalars[4], int dtype, int on_device) {
    if (!c || !valid_dtype(dtype)) { als_set_error("als_get_state: bad argument"); return ALS_EINVAL; }
    if (!c->ncg_ready) { als_set_error("als_get_state: ALS-NCG has not started"); return ALS_EINVAL; }
    if (c->n_prob > 1) { als_set_error("als_get_state: not supported for batched contexts"); return ALS_ENOTSUP; }
    const int64_t rows = c->n_u + c->n_m;
    const size_t bytes = (size_t)rows * c->nf * dtype_size(dtype);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    void *src[5] = {c->X, c->P, c->G[c->gcur], c->Gbar, c->Xbar};
    void *dst[5] = {x, p, g, gbar, xbar};
    for (int i = 0; i < 5; ++i) {
        if (!dst[i]) continue;
        als_status s = launch_convert_out(c, c->tmpvec, src[i], rows, dtype, c->nf);
        if (s != ALS_OK) return s;
        ALS_CUDA_TRY(cudaMemcpyAsync(dst[i], c->tmpvec, bytes, kind, c->stream));
        if (!on_device) ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    als_status s = read_scalars(c);
    if (s != ALS_OK) return s;
    if (scalars) {
        scalars[0] = c->hS[S_S];
        scalars[1] = c->hS[S_GG0];
        scalars[2] = (double)c->k;
        scalars[3] = c->hS[S_NFALL];
    }
    return ALS_OK;
}

extern "C" als_status als_set_state(als_ctx *c, const void *x, const void *p, const void *g, const void *gbar,
                                    const void *xbar, const double scalars[4], int dtype, int on_device) {
    if (!c || !x || !p || !g || !gbar || !xbar || !scalars || !valid_dtype(dtype)) {
        als_set_error("als_set_state: bad argument");
        return ALS_EINVAL;
    }
    if (c->n_prob > 1) { als_set_error("als_set_state: not supported for batched contexts"); return ALS_ENOTSUP; }
    const int64_t rows = c->n_u + c->n_m;
    const size_t bytes = (size_t)rows * c->nf * dtype_size(dtype);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const void *src[5] = {x, p, g, gbar, xbar};
    void *dst[5] = {c->X, c->P, c->G[c->gcur], c->Gbar, c->Xbar};
    for (int i = 0; i < 5; ++i) {
        ALS_CUDA_TRY(cudaMemcpyAsync(c->tmpvec, src[i], bytes, kind, c->stream));
        als_status s = launch_convert_in(c, dst[i], c->tmpvec, rows, dtype, c->nf);
        if (s != ALS_OK) return s;
        if (!on_device) ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    const double hs[4] = {scalars[0], scalars[1], scalars[3], 0.0};
    ALS_CUDA_TRY(cudaMemcpyAsync(c->S + S_S, &hs[0], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->S + S_GG0, &hs[1], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->S + S_NFALL, &hs[2], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->S + S_MODE, &hs[3], sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // a restored checkpoint replaces whatever an expired bounded wait left
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags + 7, 0, sizeof(int), c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->k = (int64_t)scalars[2];
    c->ncg_ready = true;
    return ALS_OK;
}

extern "C" als_status als_sweep(als_ctx *c, int32_t n_sweeps) {
    if (!c || n_sweeps < 0) { als_set_error("als_sweep: bad argument"); return ALS_EINVAL; }
    for (int i = 0; i < n_sweeps; ++i) {
        als_status s = sweep_into(c, c->X, c->X, nullptr);
        if (s != ALS_OK) return s;
    }
    c->ncg_ready = false;
    return ALS_OK;
}

extern "C" als_status alsncg_step(als_ctx *c, als_iter_info *out) {
    if (!c) { als_set_error("alsncg_step: ctx is NULL"); return ALS_EINVAL; }
    als_status s;
    if (!c->ncg_ready) {
        s = ncg_init(c);
        if (s != ALS_OK) return s;
    }
    s = capture_graphs(c);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaGraphLaunch(c->graph[c->gcur], c->stream));
    const int64_t nk = c->graph_kernels[c->gcur];
    c->gcur ^= 1;
    c->k += 1;
    if (out) {
        s = read_scalars(c);
        if (s != ALS_OK) return s;
        fill_info(c, out);
        out->kernels = nk;
        if (out->fallback) {
            double f;
            s = loss_now(c, &f);
            if (s != ALS_OK) return s;
            out->f = f;
        }
    }
    return ALS_OK;
}

extern "C" als_status alsncg_run(als_ctx *c, int32_t max_iter, double rel_tol, int32_t check_every,
                                 als_iter_info *last, int32_t *iters_done) {
    if (!c || max_iter < 0 || check_every < 1) { als_set_error("alsncg_run: bad argument"); return ALS_EINVAL; }
    als_status s;
    if (!c->ncg_ready) {
        s = ncg_init(c);
        if (s != ALS_OK) return s;
    }
    s = capture_graphs(c);
    if (s != ALS_OK) return s;
    int32_t done = 0;
    int64_t nk = 0;
    bool converged = false;
    while (done < max_iter && !converged) {
        ALS_CUDA_TRY(cudaGraphLaunch(c->graph[c->gcur], c->stream));
        nk += c->graph_kernels[c->gcur];
        c->gcur ^= 1;
        c->k += 1;
        ++done;
        if (done % check_every == 0 || done == max_iter) {
            s = read_scalars(c);
            if (s != ALS_OK) return s;
            converged = worst_rel_gnorm(c) <= rel_tol;
        }
    }
    if (iters_done) *iters_done = done;
    if (last) {
        s = read_scalars(c);
        if (s != ALS_OK) return s;
        fill_info(c, last);
        last->kernels = nk;
    }
    return ALS_OK;
}

extern "C" als_status als_loss(als_ctx *c, double *f) {
    if (!c || !f) { als_set_error("als_loss: bad argument"); return ALS_EINVAL; }
    return loss_now(c, f);
}

extern "C" als_status als_grad(als_ctx *c, void *g_out, int dtype, int on_device, double *gnorm) {
    if (!c || (g_out && !valid_dtype(dtype))) { als_set_error("als_grad: bad argument"); return ALS_EINVAL; }
    // G[gcur ^ 1] is free between ALS-NCG iterations (the next one overwrites it)
    void *G = c->G[c->gcur ^ 1];
    als_status s = grad_into(c, c->X, G, nullptr, nullptr);
    if (s != ALS_OK) return s;
    if (gnorm) {
        s = launch_reduce(c, 1, c->n_u + c->n_m, S_RED, POST_NONE, ls_params(c));
        if (s != ALS_OK) return s;
    }
    if (g_out) {
        const size_t es = dtype_size(dtype);
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        s = launch_convert_out(c, c->tmpvec, G, c->n_u + c->n_m, dtype, c->nf);
        if (s != ALS_OK) return s;
        ALS_CUDA_TRY(cudaMemcpyAsync(g_out, c->tmpvec, (size_t)(c->n_u + c->n_m) * c->nf * es, kind, c->stream));
    }
    if (gnorm) {
        s = read_scalars(c);
        if (s != ALS_OK) return s;
        *gnorm = std::sqrt(sum_slot(c, S_RED));
    } else if (g_out && !on_device) {
        ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return ALS_OK;
}

extern "C" als_status als_linesearch_coeffs(als_ctx *c, const void *p, int dtype, int on_device, double cf[5]) {
    if (!c || !cf || (p && !valid_dtype(dtype))) { als_set_error("als_linesearch_coeffs: bad argument"); return ALS_EINVAL; }
    void *P = c->P;
    if (p) {
        // stage the caller's direction in G[gcur^1] (unused between iterations)
        void *dst = c->G[c->gcur ^ 1];
        const size_t es = dtype_size(dtype);
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        ALS_CUDA_TRY(cudaMemcpyAsync(c->tmpvec, p, (size_t)(c->n_u + c->n_m) * c->nf * es, kind, c->stream));
        als_status s = launch_convert_in(c, dst, c->tmpvec, c->n_u + c->n_m, dtype, c->nf);
        if (s != ALS_OK) return s;
        P = dst;
    } else if (!c->ncg_ready) {
        als_set_error("als_linesearch_coeffs: no direction given and ALS-NCG has not started");
        return ALS_EINVAL;
    }
    als_status s = lscoef_into(c, c->X, P);
    if (s != ALS_OK) return s;
    s = launch_reduce(c, 5, c->n_u + c->n_m, S_RED, POST_NONE, ls_params(c));
    if (s != ALS_OK) return s;
    s = read_scalars(c);
    if (s != ALS_OK) return s;
    for (int i = 0; i < 5; ++i) cf[i] = sum_slot(c, S_RED + i);
    return ALS_OK;
}

extern "C" als_status als_foldin(als_ctx *c, int64_t n_req, const int64_t *req_ptr, const int32_t *items,
                                 const float *vals, int on_device_in, void *u_out, int dtype, int on_device_out) {
    if (!c || n_req < 0 || (n_req > 0 && (!req_ptr || !u_out)) || !valid_dtype(dtype)) {
        als_set_error("als_foldin: bad argument");
        return ALS_EINVAL;
    }
    if (n_req == 0) return ALS_OK;
    int64_t total = 0;
    const cudaMemcpyKind kin = on_device_in ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    ALS_CUDA_TRY(cudaMemcpyAsync(&total, req_ptr + n_req, sizeof(int64_t), kin, c->stream));
    int64_t first = 0;
    ALS_CUDA_TRY(cudaMemcpyAsync(&first, req_ptr, sizeof(int64_t), kin, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (first != 0 || total < 0 || (total > 0 && (!items || !vals))) {
        als_set_error("als_foldin: req_ptr[0] must be 0 and req_ptr[n_req] >= 0");
        return ALS_EINVAL;
    }
    // device copies of the requests
    int64_t *dptr = nullptr;
    int32_t *didx = nullptr;
    float *dval = nullptr;
    void *dout = nullptr;
    int32_t *dord = nullptr;
    als_status s;
    auto cleanup = [&]() {
        ctx_free(c, dptr); ctx_free(c, didx); ctx_free(c, dval); ctx_free(c, dout); ctx_free(c, dord);
    };
    if ((s = ctx_alloc(c, (void **)&dptr, (n_req + 1) * sizeof(int64_t))) != ALS_OK) { cleanup(); return s; }
    if ((s = ctx_alloc(c, (void **)&didx, std::max<int64_t>(total, 1) * sizeof(int32_t))) != ALS_OK) { cleanup(); return s; }
    if ((s = ctx_alloc(c, (void **)&dval, std::max<int64_t>(total, 1) * sizeof(float))) != ALS_OK) { cleanup(); return s; }
    if ((s = ctx_alloc(c, (void **)&dout, (size_t)n_req * c->ld * 8)) != ALS_OK) { cleanup(); return s; }
    const cudaMemcpyKind k2 = on_device_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
#define TRY(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { cleanup(); als_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); return ALS_ECUDA; } } while (0)
    TRY(cudaMemcpyAsync(dptr, req_ptr, (n_req + 1) * sizeof(int64_t), k2, c->stream));
    if (total > 0) {
        TRY(cudaMemcpyAsync(didx, items, total * sizeof(int32_t), k2, c->stream));
        TRY(cudaMemcpyAsync(dval, vals, total * sizeof(float), k2, c->stream));
    }
    // reject out-of-range item ids, non-finite values and a decreasing req_ptr
    s = launch_check_requests(c, dptr, n_req, didx, dval, total, c->n_m, c->dflags + 6);
    if (s != ALS_OK) { cleanup(); return s; }
    TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    if (c->hflags[6]) {
        cleanup();
        als_set_error("als_foldin: item id out of range, non-finite rating or decreasing req_ptr");
        return ALS_EINVAL;
    }
    // requests by descending degree (ties by position), as a sweep orders its
    // rows: the heaviest take the prefetching tensor-core kernel, the lightest
    // (mixed form, lambda > 0) the light-row solve
    std::vector<int64_t> hp(n_req + 1);
    TRY(cudaMemcpyAsync(hp.data(), dptr, (n_req + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> hord(n_req);
    for (int64_t q = 0; q < n_req; ++q) hord[q] = (int32_t)q;
    std::stable_sort(hord.begin(), hord.end(),
                     [&](int32_t x, int32_t y) { return hp[x + 1] - hp[x] > hp[y + 1] - hp[y]; });
    const int T = std::min(c->dual_max, c->nf);
    const bool dual = c->use_tc && !c->f64 && c->cfg.lambda > 0.0 && T > 0;
    int64_t npf = 0, ndual = 0, nsmall = 0;
    for (int64_t q = 0; q < n_req; ++q) {
        const int64_t d = hp[hord[q] + 1] - hp[hord[q]];
        if (d >= ALS_TC_PF_MIN) ++npf;
        if (dual && d <= T) ++ndual;
        if (dual && d <= std::min(T, ALS_DUAL_SMALL)) ++nsmall;
    }
    if ((s = ctx_alloc(c, (void **)&dord, n_req * sizeof(int32_t))) != ALS_OK) { cleanup(); return s; }
    TRY(cudaMemcpyAsync(dord, hord.data(), n_req * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    SweepArgs a;
    a.ptr = dptr;
    a.idx = didx;
    a.val = dval;
    a.order = dord;
    a.nrows = n_req;
    a.npf = npf;
    a.ndual = ndual;
    a.ndual_small = nsmall;
    a.dual_nmax = dual ? T : 0;
    a.F = mblk(c, c->X);
    a.nF = c->n_m;
    a.Xin = nullptr;
    a.Xout = dout;
    a.Gbar = nullptr;
    a.nf = c->nf;
    a.ld = c->ld;
    a.lambda = c->cfg.lambda;
    a.refine = c->cfg.refine_steps + 1;  // cold start: one more correction
    a.notspd = c->dflags + 5;
    a.timeout = c->dflags + 7;
    s = launch_sweep(c, a, c->f64, c->use_tc);
    if (s != ALS_OK) { cleanup(); return s; }
    s = launch_convert_out(c, c->tmpvec, dout, n_req, dtype, c->nf);
    if (s != ALS_OK) { cleanup(); return s; }
    const cudaMemcpyKind ko = on_device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TRY(cudaMemcpyAsync(u_out, c->tmpvec, (size_t)n_req * c->nf * dtype_size(dtype), ko, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
#undef TRY
    cleanup();
    return ALS_OK;
}

extern "C" als_status als_batch_info(als_ctx *c, int32_t n_prob, als_iter_info *out) {
    if (!c || !out || n_prob != c->n_prob) {
        als_set_error("als_batch_info: bad argument (n_prob must equal the context's problem count)");
        return ALS_EINVAL;
    }
    als_status s = read_scalars(c);
    if (s != ALS_OK) return s;
    for (int q = 0; q < n_prob; ++q) fill_info_q(c, q, out + q);
    return ALS_OK;
}

extern "C" als_status als_batch_grad_norms(als_ctx *c, int32_t n_prob, double *gnorm) {
    if (!c || !gnorm || n_prob != c->n_prob) {
        als_set_error("als_batch_grad_norms: bad argument (n_prob must equal the context's problem count)");
        return ALS_EINVAL;
    }
    // G[gcur ^ 1] is free between ALS-NCG iterations (the next one overwrites it)
    als_status s = grad_into(c, c->X, c->G[c->gcur ^ 1], nullptr, nullptr);
    if (s != ALS_OK) return s;
    s = launch_reduce(c, 1, c->n_u + c->n_m, S_RED, POST_NONE, ls_params(c));
    if (s != ALS_OK) return s;
    s = read_scalars(c);
    if (s != ALS_OK) return s;
    for (int q = 0; q < n_prob; ++q) gnorm[q] = std::sqrt(c->hS[(size_t)q * S_COUNT + S_RED]);
    return ALS_OK;
}

extern "C" als_status als_sync(als_ctx *c) {
    if (!c) { als_set_error("als_sync: ctx is NULL"); return ALS_EINVAL; }
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ALS_OK;
}

extern "C" void als_destroy(als_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    while (!c->allocs.empty()) ctx_free(c, c->allocs.back().p);
    if (c->hS) cudaFreeHost(c->hS);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

// ---------------------------------------------------------------------------
// Autotuner: launch shapes timed on this context's own data.  Only launch
// geometry changes (which kernel variant a row goes to, grid caps, the Gram
// path of the mixed form); every variant computes the same quantities, so
// the FP64 form's results change only in summation order.

namespace {

template <typename Fn>
als_status time_best_ms(als_ctx *c, int reps, Fn &&fn, double *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ALS_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaGetLastError();
        als_set_error("als_autotune: event creation failed");
        return ALS_ECUDA;
    }
    als_status s = fn();  // warm-up
    double best = 1e300;
    for (int r = 0; r < reps && s == ALS_OK; ++r) {
        cudaEventRecord(e0, c->stream);
        s = fn();
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            als_set_error("als_autotune: timed launch failed");
            s = ALS_ECUDA;
            break;
        }
        float el = 0.0f;
        cudaEventElapsedTime(&el, e0, e1);
        best = std::min(best, (double)el);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

// rows of `side` with at least t ratings (a prefix of the degree order)
int64_t rows_at_least(const als_ctx *c, int side, int64_t t) {
    const std::vector<int32_t> &d = c->h_deg[side];
    return std::partition_point(d.begin(), d.end(), [&](int32_t x) { return (int64_t)x >= t; }) - d.begin();
}

}  // namespace

namespace {

void fill_launch(const als_ctx *c, als_launch *o) {
    o->heavy_min = c->heavy_min;
    o->grid_mult = c->grid_mult;
    o->sweep_bin_min = c->sweep_bin_min;
    o->split_min = c->split_min;
    o->seg_len = c->seg_len;
    o->gram_path = c->f64 ? ALS_GRAM_FMA : (c->use_tc ? ALS_GRAM_TC : ALS_GRAM_FMA);
    o->dual_max = c->dual_max;
    o->gather_tma = c->gather_tma;
    o->tc_chunk = c->tc_chunk16 ? 16 : 32;
    o->chol_tc = c->chol_tc;
    o->dual_warp = c->dual_warp;
}

// apply launch shapes (validated by the caller); rebuilds what depends on them
als_status apply_launch(als_ctx *c, const als_launch &l) {
    als_status s = load_degrees(c);
    if (s != ALS_OK) return s;
    c->heavy_min = l.heavy_min;
    c->nheavy_u = rows_at_least(c, 0, l.heavy_min);
    c->nheavy_m = rows_at_least(c, 1, l.heavy_min);
    c->grid_mult = l.grid_mult;
    c->sweep_bin_min = l.sweep_bin_min;
    c->sweep_big[0] = l.sweep_bin_min > 0 ? rows_at_least(c, 0, l.sweep_bin_min) : 0;
    c->sweep_big[1] = l.sweep_bin_min > 0 ? rows_at_least(c, 1, l.sweep_bin_min) : 0;
    if (!c->f64) {
        c->use_tc = l.gram_path == ALS_GRAM_TC;
    }
    if (l.split_min != c->split_min || l.seg_len != c->seg_len || (c->split_min > 0 && !c->seg_part)) {
        c->split_min = l.split_min;
        c->seg_len = l.seg_len;
        if ((s = build_split(c)) != ALS_OK) return s;
    }
    c->dual_max = l.dual_max;
    c->gather_tma = l.gather_tma;
    c->tc_chunk16 = l.tc_chunk == 16;
    c->chol_tc = l.chol_tc;
    c->dual_warp = l.dual_warp;
    count_sweep_rows(c);
    destroy_graphs(c);  // the captured iterations hold the old launch shapes
    return ALS_OK;
}

bool launch_valid(const als_ctx *c, const als_launch &l) {
    if (l.heavy_min < 1 || l.grid_mult < 1 || l.grid_mult > 64 || l.sweep_bin_min < 0 || l.split_min < 0 ||
        l.seg_len < 32 || l.dual_max < 0 || l.dual_max > ALS_DUAL_MAX || l.gather_tma < 0 || l.gather_tma > 1 ||
        (l.tc_chunk != 16 && l.tc_chunk != 32) || l.chol_tc < 0 || l.chol_tc > 1 ||
        l.dual_warp < 0 || l.dual_warp > 1)
        return false;
    if (l.gram_path != ALS_GRAM_FMA && l.gram_path != ALS_GRAM_TC) return false;
    if (l.gram_path == ALS_GRAM_TC && (c->f64 || c->nf > ALS_TC_LD)) return false;
    return true;
}

}  // namespace

extern "C" als_status als_get_launch(als_ctx *c, als_launch *out) {
    if (!c || !out) { als_set_error("als_get_launch: bad argument"); return ALS_EINVAL; }
    fill_launch(c, out);
    return ALS_OK;
}

extern "C" als_status als_set_launch(als_ctx *c, const als_launch *in) {
    if (!c || !in || !launch_valid(c, *in)) {
        als_set_error("als_set_launch: bad argument (heavy_min >= 1, grid_mult 1..64, sweep_bin_min >= 0, "
                      "split_min >= 0, seg_len >= 32, gram_path FMA, or TC for the mixed form, dual_max 0..64, "
                      "gather_tma 0 or 1, tc_chunk 16 or 32, chol_tc 0 or 1, dual_warp 0 or 1)");
        return ALS_EINVAL;
    }
    return apply_launch(c, *in);
}

extern "C" als_status als_autotune(als_ctx *c, int32_t reps, als_tune_report *out) {
    if (!c || reps < 1 || reps > 100) { als_set_error("als_autotune: bad argument"); return ALS_EINVAL; }
    als_status s = load_degrees(c);
    if (s != ALS_OK) return s;
    void *scratch = c->tmpvec;  // n_u + n_m rows of ld doubles: holds any result vector
    als_tune_report rep;
    std::memset(&rep, 0, sizeof rep);
    als_launch cur;
    fill_launch(c, &cur);
    auto passes = [&]() -> als_status {
        als_status st = grad_into(c, c->X, scratch, c->Gbar, c->G[0]);
        if (st != ALS_OK) return st;
        return lscoef_into(c, c->X, c->P);
    };
    auto sweep = [&]() -> als_status { return sweep_into(c, c->X, scratch, nullptr); };
    // time `fn` with `cand` applied; keep it in `cur` when faster than `best`
    auto trial = [&](const als_launch &cand, bool pass, double &best) -> als_status {
        if (!launch_valid(c, cand)) return ALS_OK;
        als_status st = apply_launch(c, cand);
        if (st != ALS_OK) return st;
        double ms;
        st = pass ? time_best_ms(c, reps, passes, &ms) : time_best_ms(c, reps, sweep, &ms);
        if (st != ALS_OK) return st;
        ++rep.candidates;
        if (ms < best * (1.0 - ALS_TUNE_MARGIN)) {
            best = ms;
            cur = cand;
        }
        return apply_launch(c, cur);
    };

    // 1. passes: heavy-row threshold, then the grid cap
    if ((s = time_best_ms(c, reps, passes, &rep.pass_ms_default)) != ALS_OK) return s;
    double best = rep.pass_ms_default;
    for (int h : {256, 512, 1024, 2048, 4096, 8192, 1 << 30}) {
        als_launch cand = cur;
        cand.heavy_min = h;
        if ((s = trial(cand, true, best)) != ALS_OK) return s;
    }
    for (int g : {4, 8, 16, 32, 64}) {
        als_launch cand = cur;
        cand.grid_mult = g;
        if ((s = trial(cand, true, best)) != ALS_OK) return s;
    }
    rep.pass_ms_tuned = best;

    // 2. sweep: Gram path (mixed, 16 < n_f <= 64), heavy-row split, FMA degree bin
    if ((s = time_best_ms(c, reps, sweep, &rep.sweep_ms_default)) != ALS_OK) return s;
    best = rep.sweep_ms_default;
    if (!c->f64 && c->cfg.gram_path == ALS_GRAM_AUTO && c->nf > 16 && c->nf <= 64) {
        als_launch cand = cur;
        cand.gram_path = cur.gram_path == ALS_GRAM_TC ? ALS_GRAM_FMA : ALS_GRAM_TC;
        if ((s = trial(cand, false, best)) != ALS_OK) return s;
    }
    {
        // every candidate splits rows above 65536 ratings: a whole row's
        // Gram matrix accumulated in FP32 over millions of ratings is too
        // inexact for the mixed form's refinement (f 1.4e-5 off the FP64 run
        // with rows of 2.7e6 ratings); segment partials added in FP64 are not
        const int split_c[][2] = {{2048, 1024}, {2048, 2048}, {4096, 1024}, {4096, 2048}, {4096, 4096},
                                  {8192, 2048}, {8192, 4096}, {16384, 4096}, {65536, 4096}};
        for (const auto &sc : split_c) {
            als_launch cand = cur;
            cand.split_min = sc[0];
            cand.seg_len = sc[1];
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
    }
    if (!c->f64 && cur.gram_path == ALS_GRAM_TC) {
        // the heavy rows' gather: cp.async by the lanes, or TMA gather4
        for (int g : {0, 1}) {
            als_launch cand = cur;
            cand.gather_tma = g;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
        // the other rows' chunk: 16 ratings (7 CTAs per SM) or 32 (5)
        for (int kc : {16, 32}) {
            als_launch cand = cur;
            cand.tc_chunk = kc;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
        // the rows' Cholesky: CUDA cores in shared memory, or TMEM panels
        // with the trailing updates on the tensor core
        for (int ct : {0, 1}) {
            als_launch cand = cur;
            cand.chol_tc = ct;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
    }
    if (!c->f64 && cur.gram_path == ALS_GRAM_TC && c->cfg.lambda > 0.0) {
        // light-row solve through n_i x n_i matrices: the longest such row
        for (int d : {0, 16, 32, 48, 64}) {
            als_launch cand = cur;
            cand.dual_max = d;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
        // the light rows of <= 32 ratings: a CTA or a warp each
        for (int w : {0, 1}) {
            als_launch cand = cur;
            cand.dual_warp = w;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
    }
    if (c->nf <= 32 && cur.gram_path == ALS_GRAM_FMA) {
        for (int b : {0, 16384, 4096, 1024, 256}) {
            als_launch cand = cur;
            cand.sweep_bin_min = b;
            if ((s = trial(cand, false, best)) != ALS_OK) return s;
        }
    }
    rep.sweep_ms_tuned = best;
    if ((s = apply_launch(c, cur)) != ALS_OK) return s;
    rep.chosen = cur;
    if (out) *out = rep;
    return ALS_OK;
}

// ---------------------------------------------------------------------------
// Groups of contexts (problems of different n_f): every member's captured
// iteration is launched on the member's own stream, so the members' kernels
// overlap on the GPU; the host only enqueues.

extern "C" als_status als_group_run(als_ctx **ctxs, int32_t n, int32_t max_iter, double rel_tol,
                                    int32_t check_every, als_iter_info *last, int32_t *iters_done) {
    if (!ctxs || n < 1 || max_iter < 0 || check_every < 1) {
        als_set_error("als_group_run: bad argument");
        return ALS_EINVAL;
    }
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i]) { als_set_error("als_group_run: a member is NULL"); return ALS_EINVAL; }
        for (int32_t j = 0; j < i; ++j) {
            if (ctxs[j] == ctxs[i]) {
                als_set_error("als_group_run: members must be distinct contexts");
                return ALS_EINVAL;
            }
        }
    }
    als_status s;
    for (int32_t i = 0; i < n; ++i) {
        als_ctx *c = ctxs[i];
        if (!c->ncg_ready && (s = ncg_init(c)) != ALS_OK) return s;
        if ((s = capture_graphs(c)) != ALS_OK) return s;
    }
    std::vector<int64_t> nk(n, 0);
    int32_t done = 0;
    bool converged = false;
    while (done < max_iter && !converged) {
        for (int32_t i = 0; i < n; ++i) {
            als_ctx *c = ctxs[i];
            ALS_CUDA_TRY(cudaGraphLaunch(c->graph[c->gcur], c->stream));
            nk[i] += c->graph_kernels[c->gcur];
            c->gcur ^= 1;
            c->k += 1;
        }
        ++done;
        if (done % check_every == 0 || done == max_iter) {
            double worst = 0.0;
            for (int32_t i = 0; i < n; ++i) {
                if ((s = read_scalars(ctxs[i])) != ALS_OK) return s;
                worst = std::max(worst, worst_rel_gnorm(ctxs[i]));
            }
            converged = worst <= rel_tol;
        }
    }
    if (iters_done) *iters_done = done;
    if (last) {
        for (int32_t i = 0; i < n; ++i) {
            if ((s = read_scalars(ctxs[i])) != ALS_OK) return s;
            fill_info(ctxs[i], last + i);
            last[i].kernels = nk[i];
        }
    }
    return ALS_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded device waits: one half sweep of the tensor-core
// kernel in which no MMA is issued and nothing signals the mbarriers, so every
// CTA's wait runs out after limit_s; each records the expiry, frees its TMEM
// and returns.  Nothing is left in flight; the expiry stays recorded in the
// context as a real one would be.

extern "C" als_status als_selftest_wait_expiry(als_ctx *c, double limit_s, int64_t *expired) {
    if (!c || !(limit_s > 0.0) || limit_s > 10.0) {
        als_set_error("als_selftest_wait_expiry: bad argument (0 < limit_s <= 10)");
        return ALS_EINVAL;
    }
    if (!c->use_tc) {
        als_set_error("als_selftest_wait_expiry: needs the tensor-core Gram (ALS_MIXED)");
        return ALS_ENOTSUP;
    }
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags, 0, 16 * sizeof(int), c->stream));
    SweepArgs a;
    a.ptr = c->uptr;
    a.idx = c->uidx;
    a.val = c->uval;
    a.order = c->uorder;
    a.nrows = c->n_u;
    a.F = mblk(c, c->X);
    a.nF = c->n_m;
    a.Xin = ublk(c, c->X);
    a.Xout = c->tmpvec;   // scratch: the factors are not touched
    a.Gbar = nullptr;
    a.nf = c->nf;
    a.ld = c->ld;
    a.lambda = c->cfg.lambda;
    a.refine = c->cfg.refine_steps;
    a.notspd = c->dflags;
    a.timeout = c->dflags + 7;
    a.wait_ns = (uint64_t)(limit_s * 1e9);
    a.withhold = 1;
    als_status s = launch_sweep(c, a, false, true);
    if (s != ALS_OK) return s;
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int64_t n = c->hflags[7];
    // the expiry stays recorded, as after a real one inside a sweep: the next
    // call that reads the context's status reports ALS_ETIMEOUT once, and
    // als_set_state / als_set_factors clear it; the other flags are reset
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags, 0, 7 * sizeof(int), c->stream));
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags + 8, 0, 8 * sizeof(int), c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (expired) *expired = n;
    if (n == 0) {
        als_set_error("als_selftest_wait_expiry: no wait ran out");
        return ALS_OK;
    }
    als_set_error("als_selftest_wait_expiry: the bounded waits ran out as designed");
    return ALS_ETIMEOUT;
}

// ---------------------------------------------------------------------------
// Per-kernel-class timing of one sweep (events on each launch's own stream).

void kt_begin(als_ctx *c, int cls, cudaStream_t st) {
    KTimer *k = c->kt;
    if (!k || (k->depth > 0 && cls != KT_TC_SEG) || k->n[cls] >= KTimer::kMax) return;
    cudaEventRecord(k->ev[cls][k->n[cls]][0], st);
}

void kt_end(als_ctx *c, int cls, cudaStream_t st) {
    KTimer *k = c->kt;
    if (!k || (k->depth > 0 && cls != KT_TC_SEG) || k->n[cls] >= KTimer::kMax) return;
    cudaEventRecord(k->ev[cls][k->n[cls]][1], st);
    k->n[cls] += 1;
}

extern "C" als_status als_time_sweep(als_ctx *c, int32_t reps, als_sweep_timing *out) {
    if (!c || !out || reps < 1 || reps > 1000) {
        als_set_error("als_time_sweep: bad argument (1 <= reps <= 1000, out not NULL)");
        return ALS_EINVAL;
    }
    als_status s = load_degrees(c);
    if (s != ALS_OK) return s;
    std::memset(out, 0, sizeof *out);
    // rows and ratings of each class, from the degree order: split rows first,
    // then (tensor-core sweep) the prefetching rows, the other tensor-core
    // rows and the light rows; or (FMA sweep) every other row
    const bool tc = c->use_tc && !c->f64;
    for (int side = 0; side < 2; ++side) {
        const std::vector<int32_t> &d = c->h_deg[side];
        const int64_t n = (int64_t)d.size();
        const int64_t H = c->nsplit[side];
        auto add = [&](int cls, int64_t b, int64_t e) {
            b = std::max<int64_t>(0, std::min(b, n));
            e = std::max<int64_t>(b, std::min(e, n));
            out->rows[cls] += e - b;
            for (int64_t r = b; r < e; ++r) out->ratings[cls] += d[r];
        };
        add(KT_SPLIT, 0, H);
        if (tc) add(KT_TC_SEG, 0, H);
        if (tc) {
            const int64_t npf = std::min(c->sweep_pf[side], n - H);
            const int64_t nd = std::min(c->sweep_dual[side], n - H);
            add(KT_TC_PF, H, H + npf);
            add(KT_TC, H + npf, n - nd);
            add(KT_DUAL, n - nd, n);
        } else {
            add(KT_FMA, H, n);
        }
    }
    KTimer kt;
    std::memset(&kt, 0, sizeof kt);
    kt.serial = true;
    for (int a = 0; a < KT_NCLASS; ++a)
        for (int i = 0; i < KTimer::kMax; ++i)
            for (int j = 0; j < 2; ++j)
                if (cudaEventCreate(&kt.ev[a][i][j]) != cudaSuccess) {
                    als_set_error("als_time_sweep: cudaEventCreate failed");
                    kt.ev[a][i][j] = nullptr;
                }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto cleanup = [&]() {
        c->kt = nullptr;
        for (int a = 0; a < KT_NCLASS; ++a)
            for (int i = 0; i < KTimer::kMax; ++i)
                for (int j = 0; j < 2; ++j)
                    if (kt.ev[a][i][j]) cudaEventDestroy(kt.ev[a][i][j]);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    // x is not changed: xbar = P(x) and gbar = x - xbar are written, which is
    // what they already hold between ALS-NCG iterations (the kernels are
    // deterministic)
    for (int rep = 0; rep < reps; ++rep) {
        for (int a = 0; a < KT_NCLASS; ++a) kt.n[a] = 0;
        c->kt = &kt;
        cudaEventRecord(e0, c->stream);
        s = sweep_into(c, c->X, c->Xbar, c->Gbar);
        cudaEventRecord(e1, c->stream);
        c->kt = nullptr;
        if (s != ALS_OK) { cleanup(); return s; }
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cleanup();
            als_set_error(std::string("als_time_sweep: ") + cudaGetErrorString(e));
            return ALS_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        out->sweep_ms += ms / reps;
        for (int a = 0; a < KT_NCLASS; ++a) {
            out->launches[a] = kt.n[a];
            for (int i = 0; i < kt.n[a]; ++i) {
                float m = 0.f;
                cudaEventElapsedTime(&m, kt.ev[a][i][0], kt.ev[a][i][1]);
                out->ms[a] += m / reps;
            }
        }
    }
    cleanup();
    ALS_CUDA_TRY(cudaGetLastError());
    return read_scalars(c);
}
