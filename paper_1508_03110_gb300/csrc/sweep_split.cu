// Heavy rows of a half sweep split across CTAs.  A row with many ratings
// would otherwise be walked chunk after chunk by a single CTA while the rest
// of the grid idles (ML20M-shaped data: the 1,152 items with >= 4096 ratings
// hold two thirds of all ratings, the largest 33k; Zipf-1.1 data reaches
// 2e5).  Each such row's ratings are cut into segments of about seg_len:
//   1. one CTA per segment forms the segment's part of Eq. (3)/(4): its
//      partial Gram matrix sum_e f_e f_e^T and, for the FP64 form, its part
//      of the right-hand side sum_e r_e f_e, or, for the mixed form, its part
//      of the residual sum_e f_e (r_e - f_e . x_i) at the current row (the
//      same kernels as whole rows, in segment mode);
//   2. one CTA per split row adds its segments' partials in FP64 in segment
//      order (deterministic), adds lambda n_i I, factors and solves -- the
//      FP64 form exactly (the definition), the mixed form as the first
//      correction of the refinement from x_i -- and keeps the factored matrix
//      (mixed form: packed lower triangle, as the tensor-core kernel's);
//   3. mixed form only, up to refine_steps - 1 times, for the rows whose last
//      correction was not yet negligible: one CTA per segment forms its part
//      of the FP32 residual at the new row, one CTA per row adds them, solves
//      with the kept factor and applies the correction.
// Accuracy: a segment's tensor-core partial accumulates at most seg_len
// ratings in FP32 and the segments are added in FP64, so a split row's Gram
// matrix is more accurate than a whole row's: its relative error is that of
// one segment's, 2^-17 (the BF16 split) + seg_len 2^-24 (FP32 accumulation),
// plus one FP32 rounding of the sum.  The refinement's stopping rule
// (sw_correction_small) therefore takes min(n_i, seg_len) ratings for a
// split row rather than n_i, so long rows stop as soon as a row of seg_len
// ratings would.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

struct SplitArgs {
    const int32_t *order;     // the side's degree order (split rows first)
    const int64_t *ptr;       // the side's row pointers (degree of a row)
    const int32_t *hseg_off;  // [nsplit + 1]
    const int32_t *seg_row;   // segment -> split row
    const int64_t *seg_beg;
    const int32_t *seg_len;
    const int32_t *idx;       // fixed-side ids of the side's ratings
    const float *val;
    const void *part;         // partials, seg_stride elements per segment
    int64_t seg_stride;
    const void *F;            // fixed-side factors (ld-strided)
    const void *Xin;          // current rows (x_i), may be null
    void *Xout;
    void *Gbar;               // may be null
    float *hfac;              // mixed: factored matrices, n_f x (n_f + 1) per split row
    int32_t *hflag;           // mixed: rows that take another correction
    int *notspd;
    int nf, ld;
    double lambda;
    int more;                 // mixed: corrections still allowed after this one
    int seg_cap;              // the most ratings of any segment (seg_len)
    void *Gout;               // mixed: the rows' gradient -2 (r0 - lambda n x_i), or null
};

constexpr int HT = 128;  // threads per CTA

__device__ __forceinline__ void tri_index(int e, int &m, int &c) {
    m = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((m + 1) * (m + 2) / 2 <= e) ++m;
    while (m * (m + 1) / 2 > e) --m;
    c = e - m * (m + 1) / 2;
}

// step 2: sum the partials, factor, solve (one CTA per split row)
template <typename T>
__global__ void __launch_bounds__(HT) k_split_solve(SplitArgs s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nf = s.nf, ldA = nf + 1, t = threadIdx.x;
    T *A = reinterpret_cast<T *>(smem_raw);
    T *vec = A + (((size_t)nf * ldA + 3) & ~(size_t)3);
    T *u = vec, *v1 = vec + 128, *v2 = vec + 256, *colk = vec + 384, *diag = vec + 512;
    float *work = reinterpret_cast<float *>(vec + 640);  // FP32 Cholesky scratch / reduction
    const int h = blockIdx.x;
    const int64_t row = s.order[h];
    const int64_t n = s.ptr[row + 1] - s.ptr[row];
    const T lam_n = (T)(s.lambda * (double)n);
    const int tri = nf * (nf + 1) / 2;
    const int s0 = s.hseg_off[h], s1 = s.hseg_off[h + 1];
    const T *P = reinterpret_cast<const T *>(s.part);
    const T *xi = s.Xin ? reinterpret_cast<const T *>(s.Xin) + row * s.ld : nullptr;
    for (int k = t; k < nf; k += HT) u[k] = xi ? xi[k] : T(0);
    // FP64 form: square A (column Cholesky); mixed form: packed lower triangle
    for (int e = t; e < tri + nf; e += HT) {
        double acc = 0.0;
        for (int q = s0; q < s1; ++q) acc += (double)P[(int64_t)q * s.seg_stride + e];
        if (e < tri) {
            if constexpr (sizeof(T) == 8) {
                int m, c;
                tri_index(e, m, c);
                A[m * ldA + c] = (T)acc;
            } else {
                A[e] = (T)acc;
            }
        } else {
            v1[e - tri] = (T)acc;
        }
    }
    __syncthreads();
    if (t < nf) {
        A[sizeof(T) == 8 ? t * ldA + t : tri_off(t) + t] += lam_n;
        if (sizeof(T) == 4) v1[t] -= lam_n * u[t];  // mixed: residual at x_i
    }
    if (sizeof(T) == 4 && s.Gout && t < s.ld)
        reinterpret_cast<float *>(s.Gout)[row * s.ld + t] = t < nf ? -2.0f * (float)v1[t] : 0.0f;
    __syncthreads();
    bool ok;
    if constexpr (sizeof(T) == 8) {
        ok = sw_cholesky<T, HT>(A, ldA, nf, colk, diag, t);
        if (ok) sw_trisolve<T, HT>(A, ldA, nf, diag, v1, v2, u, t);
    } else {
        ok = chol_blocked128(reinterpret_cast<float *>(A), nf, reinterpret_cast<float *>(diag), work, t);
        if (ok) {
            invert_diag_blocks128(reinterpret_cast<float *>(A), nf, reinterpret_cast<float *>(diag), t);
            trisolve_inv128(reinterpret_cast<float *>(A), nf, reinterpret_cast<float *>(v1),
                            reinterpret_cast<float *>(v2), reinterpret_cast<float *>(colk), t);
            for (int k = t; k < nf; k += HT) u[k] += colk[k];
            float *hf = s.hfac + (size_t)h * tri;
            for (int e = t; e < tri; e += HT) hf[e] = A[e];
            __syncthreads();
            const bool small = sw_correction_small<float, HT>(colk, u, nf, (int)(n < s.seg_cap ? n : (int64_t)s.seg_cap), work, t);
            if (t == 0) s.hflag[h] = (s.more > 0 && !small) ? 1 : 0;
        }
    }
    if (!ok) {
        if (t == 0) {
            atomicAdd(s.notspd, 1);
            if (sizeof(T) == 4) s.hflag[h] = 0;
        }
        for (int k = t; k < nf; k += HT) u[k] = xi ? xi[k] : T(0);
    }
    __syncthreads();
    T *xo = reinterpret_cast<T *>(s.Xout) + row * s.ld;
    T *gb = s.Gbar ? reinterpret_cast<T *>(s.Gbar) + row * s.ld : nullptr;
    for (int k = t; k < s.ld; k += HT) {
        const T uk = k < nf ? u[k] : T(0);
        xo[k] = uk;
        if (gb) gb[k] = (xi ? xi[k] : T(0)) - uk;
    }
}

// step 3a: a segment's part of the FP32 residual at the row's current value
__global__ void __launch_bounds__(HT) k_split_resid(SplitArgs s) {
    __shared__ float part[4][128];
    const int r = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int h = s.seg_row[r];
    if (!s.hflag[h]) return;
    const int64_t row = s.order[h];
    const float *ur = reinterpret_cast<const float *>(s.Xout) + row * s.ld;
    const bool act = 4 * lane < s.ld;
    float uu[4], acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i) uu[i] = (4 * lane + i < s.nf) ? ur[4 * lane + i] : 0.0f;
    const int64_t b = s.seg_beg[r], e1 = b + s.seg_len[r];
    const float *F = reinterpret_cast<const float *>(s.F);
    for (int64_t e = b + warp; e < e1; e += 32) resid8(F, s.ld, s.idx + e, s.val + e, e1 - e, uu, lane, act, acc, cmp);
#pragma unroll
    for (int i = 0; i < 4; ++i) part[warp][4 * lane + i] = acc[i] - cmp[i];
    __syncthreads();
    float *po = const_cast<float *>(reinterpret_cast<const float *>(s.part)) + (int64_t)r * s.seg_stride +
                s.nf * (s.nf + 1) / 2;
    if (t < s.nf) po[t] = (part[0][t] + part[1][t]) + (part[2][t] + part[3][t]);
}

// step 3b: add the residual parts, solve with the kept factor, correct
__global__ void __launch_bounds__(HT) k_split_refine(SplitArgs s) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nf = s.nf, ldA = nf + 1, t = threadIdx.x, h = blockIdx.x;
    if (!s.hflag[h]) return;
    float *A = reinterpret_cast<float *>(smem_raw);
    float *vec = A + (((size_t)nf * ldA + 3) & ~(size_t)3);
    float *u = vec, *v1 = vec + 128, *v2 = vec + 256, *colk = vec + 384;
    float *red = vec + 640;
    const int64_t row = s.order[h];
    const int64_t n = s.ptr[row + 1] - s.ptr[row];
    const float lam_n = (float)(s.lambda * (double)n);
    const int tri = nf * (nf + 1) / 2;
    const int s0 = s.hseg_off[h], s1 = s.hseg_off[h + 1];
    const float *P = reinterpret_cast<const float *>(s.part);
    float *xo = reinterpret_cast<float *>(s.Xout) + row * s.ld;
    const int tri0 = nf * (nf + 1) / 2;
    const float *hf = s.hfac + (size_t)h * tri0;
    for (int e = t; e < tri0; e += HT) A[e] = hf[e];
    for (int k = t; k < nf; k += HT) {
        double acc = 0.0;
        for (int q = s0; q < s1; ++q) acc += (double)P[(int64_t)q * s.seg_stride + tri + k];
        u[k] = xo[k];
        v1[k] = (float)acc - lam_n * u[k];
    }
    trisolve_inv128(A, nf, v1, v2, colk, t);  // starts with a barrier
    for (int k = t; k < nf; k += HT) u[k] += colk[k];
    __syncthreads();
    const bool small = sw_correction_small<float, HT>(colk, u, nf, (int)(n < s.seg_cap ? n : (int64_t)s.seg_cap), red, t);
    if (t == 0) s.hflag[h] = (s.more > 0 && !small) ? 1 : 0;
    const float *xi = s.Xin ? reinterpret_cast<const float *>(s.Xin) + row * s.ld : nullptr;
    float *gb = s.Gbar ? reinterpret_cast<float *>(s.Gbar) + row * s.ld : nullptr;
    for (int k = t; k < nf; k += HT) {
        xo[k] = u[k];
        if (gb) gb[k] = (xi ? xi[k] : 0.0f) - u[k];
    }
}

size_t solve_smem(int nf, size_t esz) {
    const size_t a = (((size_t)nf * (nf + 1) + 3) & ~(size_t)3) * esz;
    return a + 640 * esz + (16 * 128 + 256 + 16) * sizeof(float);
}

}  // namespace

als_status load_degrees(als_ctx *c) {
    for (int side = 0; side < 2; ++side) {
        if (!c->h_deg[side].empty() || (side ? c->n_m : c->n_u) == 0) continue;
        const int64_t n = side ? c->n_m : c->n_u;
        std::vector<int64_t> ptr(n + 1);
        std::vector<int32_t> ord(n);
        ALS_CUDA_TRY(cudaMemcpyAsync(ptr.data(), side ? c->mptr : c->uptr, (n + 1) * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, c->stream));
        ALS_CUDA_TRY(cudaMemcpyAsync(ord.data(), side ? c->morder : c->uorder, n * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, c->stream));
        ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->h_deg[side].resize(n);
        c->h_beg[side].resize(n);
        for (int64_t r = 0; r < n; ++r) {
            c->h_deg[side][r] = (int32_t)(ptr[ord[r] + 1] - ptr[ord[r]]);
            c->h_beg[side][r] = ptr[ord[r]];
        }
    }
    return ALS_OK;
}

als_status build_split(als_ctx *c) {
    als_status st = load_degrees(c);
    if (st != ALS_OK) return st;
    // release the previous lists and buffers
    for (int side = 0; side < 2; ++side) {
        ctx_free(c, c->seg_row[side]);
        ctx_free(c, c->seg_beg[side]);
        ctx_free(c, c->seg_len_d[side]);
        ctx_free(c, c->hseg_off[side]);
        c->seg_row[side] = nullptr;
        c->seg_beg[side] = nullptr;
        c->seg_len_d[side] = nullptr;
        c->hseg_off[side] = nullptr;
        c->nsplit[side] = c->nseg[side] = 0;
    }
    ctx_free(c, c->seg_part);
    ctx_free(c, c->hfac);
    ctx_free(c, c->hflag);
    c->seg_part = nullptr;
    c->hfac = nullptr;
    c->hflag = nullptr;
    if (c->split_min <= 0) return ALS_OK;  // splitting off
    const int tri = c->nf * (c->nf + 1) / 2;
    c->seg_stride = ((int64_t)tri + c->nf + 3) & ~(int64_t)3;
    int64_t max_seg = 0, max_split = 0;
    for (int side = 0; side < 2; ++side) {
        const std::vector<int32_t> &d = c->h_deg[side];
        const int64_t H =
            std::partition_point(d.begin(), d.end(), [&](int32_t x) { return x >= c->split_min; }) - d.begin();
        if (H == 0) continue;
        std::vector<int32_t> srow, slen, off(H + 1, 0);
        std::vector<int64_t> sbeg;
        for (int64_t h = 0; h < H; ++h) {
            const int64_t deg = d[h];
            const int64_t ns = (deg + c->seg_len - 1) / c->seg_len;
            const int64_t len = (deg + ns - 1) / ns;  // balanced segments
            for (int64_t q = 0; q < ns; ++q) {
                const int64_t b = q * len;
                srow.push_back((int32_t)h);
                sbeg.push_back(c->h_beg[side][h] + b);
                slen.push_back((int32_t)std::min<int64_t>(len, deg - b));
            }
            off[h + 1] = (int32_t)srow.size();
        }
        const int64_t S = (int64_t)srow.size();
#define ALLOC_UP(dst, vec, type)                                                                            \
    do {                                                                                                   \
        void *p_ = nullptr;                                                                                \
        if ((st = ctx_alloc(c, &p_, (vec).size() * sizeof(type))) != ALS_OK) return st;                  \
        dst = (decltype(dst))p_;                                                                           \
        ALS_CUDA_TRY(cudaMemcpyAsync(p_, (vec).data(), (vec).size() * sizeof(type), cudaMemcpyHostToDevice, \
                                     c->stream));                                                          \
    } while (0)
        ALLOC_UP(c->seg_row[side], srow, int32_t);
        ALLOC_UP(c->seg_beg[side], sbeg, int64_t);
        ALLOC_UP(c->seg_len_d[side], slen, int32_t);
        ALLOC_UP(c->hseg_off[side], off, int32_t);
#undef ALLOC_UP
        ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
        c->nsplit[side] = H;
        c->nseg[side] = S;
        max_seg = std::max(max_seg, S);
        max_split = std::max(max_split, H);
    }
    if (max_seg == 0) return ALS_OK;
    void *p = nullptr;
    if ((st = ctx_alloc(c, &p, (size_t)max_seg * c->seg_stride * c->esz)) != ALS_OK) return st;
    c->seg_part = p;
    if (!c->f64) {
        if ((st = ctx_alloc(c, &p, (size_t)max_split * (c->nf * (c->nf + 1) / 2) * sizeof(float))) != ALS_OK)
            return st;
        c->hfac = (float *)p;
        if ((st = ctx_alloc(c, &p, (size_t)max_split * sizeof(int32_t))) != ALS_OK) return st;
        c->hflag = (int32_t *)p;
    }
    return ALS_OK;
}

// Rows of the light-row solve per side: those with at most min(dual_max, n_f)
// ratings (a suffix of the degree-descending order), never a split row; none
// in the FP64 form, past the tensor-core width, or without regularisation
// (lambda = 0 leaves A singular for n_i < n_f, which the solve through G
// would hide).  And the rows of the prefetching tensor-core kernel: those of
// at least ALS_TC_PF_MIN ratings that are not split (a prefix of the order
// once the split rows are taken off).
void count_sweep_rows(als_ctx *c) {
    for (int side = 0; side < 2; ++side) {
        const std::vector<int32_t> &d = c->h_deg[side];
        const int64_t n = (int64_t)d.size();
        const int64_t heavy =
            std::partition_point(d.begin(), d.end(), [&](int32_t x) { return x >= ALS_TC_PF_MIN; }) - d.begin();
        c->sweep_pf[side] = std::max<int64_t>(0, heavy - c->nsplit[side]);
        c->sweep_dual[side] = 0;
        c->sweep_dual_small[side] = 0;
        const int T = std::min(c->dual_max, c->nf);
        if (c->f64 || T <= 0 || !(c->cfg.lambda > 0.0) || c->nf > ALS_TC_LD || n == 0) continue;
        const int64_t first =
            std::partition_point(d.begin(), d.end(), [&](int32_t x) { return x > T; }) - d.begin();
        c->sweep_dual[side] = std::max<int64_t>(0, std::min<int64_t>(n - first, n - c->nsplit[side]));
        const int Ts = std::min(T, ALS_DUAL_SMALL);
        const int64_t first_small =
            std::partition_point(d.begin(), d.end(), [&](int32_t x) { return x > Ts; }) - d.begin();
        c->sweep_dual_small[side] = std::min<int64_t>(n - first_small, c->sweep_dual[side]);
    }
}

als_status split_sweep_launches(als_ctx *c, const SweepArgs &a, int side, cudaStream_t stream);

als_status launch_split_sweep(als_ctx *c, const SweepArgs &a, int side) {
    const int64_t H = c->nsplit[side];
    if (H == 0) return ALS_OK;
    cudaStream_t stream = a.stream ? a.stream : c->stream;
    kt_begin(c, KT_SPLIT, stream);
    if (c->kt) c->kt->depth++;
    const als_status st = split_sweep_launches(c, a, side, stream);
    if (c->kt) c->kt->depth--;
    kt_end(c, KT_SPLIT, stream);
    return st;
}

// the launches of launch_split_sweep (timed there as one class)
als_status split_sweep_launches(als_ctx *c, const SweepArgs &a, int side, cudaStream_t stream) {
    const int64_t H = c->nsplit[side], S = c->nseg[side];
    // 1. segment partials
    SweepArgs b = a;
    b.nbig = 0;
    b.ndual = 0;
    b.seg_row = c->seg_row[side];
    b.seg_beg = c->seg_beg[side];
    b.seg_len = c->seg_len_d[side];
    b.seg_out = c->seg_part;
    b.seg_stride = c->seg_stride;
    b.nrows = S;
    b.Gout = nullptr;  // a segment's residual is a partial
    als_status st = launch_sweep(c, b, c->f64, c->use_tc);
    if (st != ALS_OK) return st;
    // 2. per split row: sum, factor, solve
    SplitArgs s;
    s.order = a.order;
    s.ptr = a.ptr;
    s.hseg_off = c->hseg_off[side];
    s.seg_row = c->seg_row[side];
    s.seg_beg = c->seg_beg[side];
    s.seg_len = c->seg_len_d[side];
    s.idx = a.idx;
    s.val = a.val;
    s.part = c->seg_part;
    s.seg_stride = c->seg_stride;
    s.F = a.F;
    s.Xin = a.Xin;
    s.Xout = a.Xout;
    s.Gbar = a.Gbar;
    s.hfac = c->hfac;
    s.hflag = c->hflag;
    s.notspd = a.notspd;
    s.nf = a.nf;
    s.ld = a.ld;
    s.lambda = a.lambda;
    s.more = a.refine - 1;
    s.seg_cap = c->seg_len;
    s.Gout = a.Gout;
    const size_t smem = solve_smem(a.nf, c->esz);
    if (c->f64) {
        if (raise_smem_limit((const void *)k_split_solve<double>, smem) != ALS_OK) return ALS_ECUDA;
        k_split_solve<double><<<(unsigned)H, HT, smem, stream>>>(s);
        ALS_CUDA_TRY(cudaGetLastError());
        return ALS_OK;
    }
    if (raise_smem_limit((const void *)k_split_solve<float>, smem) != ALS_OK) return ALS_ECUDA;
    k_split_solve<float><<<(unsigned)H, HT, smem, stream>>>(s);
    ALS_CUDA_TRY(cudaGetLastError());
    // 3. further corrections of the rows that still need them
    if (raise_smem_limit((const void *)k_split_refine, smem) != ALS_OK) return ALS_ECUDA;
    for (int q = 1; q < a.refine; ++q) {
        s.more = a.refine - 1 - q;
        k_split_resid<<<(unsigned)S, HT, 0, stream>>>(s);
        k_split_refine<<<(unsigned)H, HT, smem, stream>>>(s);
        ALS_CUDA_TRY(cudaGetLastError());
    }
    return ALS_OK;
}
