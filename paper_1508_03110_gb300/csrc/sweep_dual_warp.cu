// Mixed-precision light rows of at most 32 ratings, one warp per row
// (launch shape dual_warp).  The row's system is solved as in k_sweep_dual
// (sweep_dual.cu): through G = F F^T + lambda n_i I, n_i x n_i, with the
// Woodbury identity A^{-1} v = (v - F^T G^{-1} F v) / (lambda n_i) as the
// approximate inverse of an FP32 refinement started at the current row
// (readings 15-17 of the design notes).  What differs is the mapping: a
// whole CTA per row spends most of its instructions on barriers and on
// loops a 32 x 32 matrix cannot fill, so here one warp owns a row and no
// step waits for another warp:
//   1. gather: the row's factor rows are read once (a lane per 4-wide slot,
//      eight ratings at a time), stored into the warp's shared memory, and
//      give the first FP32 residual sum_e f_e (r_e - f_e . u0);
//   2. G: the lower triangle by 2 x 2 tiles of rows, a lane per tile;
//   3. Cholesky of G with lane l holding row l in registers: column j's
//      pivot and entries reach the other lanes by shuffles (rows past n_i
//      are the identity);
//   4. each correction: w = F v (lane e: rating e), L z = w by columns
//      (shuffles), L^T x = z by rows of L from shared memory, q = F^T x (a
//      lane per slot), dx = (v - q) / (lambda n_i);
//   5. further corrections (the shared stopping rule, sw_correction_small's
//      rule over the warp) recompute the FP32 residual from the rows in
//      shared memory.
// Rows of at most 16 ratings run the 16-wide forms of steps 3-4.  Two rows
// per CTA (~16 KB of shared memory each for n_f = 100, 128 registers: 7
// CTAs per SM).  The code takes R rows per lane; two (rows of 33..64
// ratings, 255 registers, one warp per CTA at ~35 KB, 6 warps per SM) ran
// 1.6x slower on those rows than a CTA per row (k_sweep_dual), so only
// R = 1 is launched.
#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

// rows per CTA (a warp each): two for rows of at most 32 ratings, one for
// longer rows (whose factor rows take twice the shared memory)
__host__ __device__ constexpr int wd_warps(int R) { return R == 1 ? 2 : 1; }

struct WarpDualLayout {
    int S;         // row stride of the factor rows (floats), S / 4 odd
    int G;         // packed lower triangle of G, then of its factor L (float offset)
    int vec;       // u, v [2][128] (float offset)
    int per_warp;  // floats per warp
};

// R: rows per lane (up to 32 R ratings)
__host__ __device__ inline WarpDualLayout wdual_layout(int nf, int R) {
    WarpDualLayout L;
    int S = (nf + 3) & ~3;
    if (((S >> 2) & 1) == 0) S += 4;
    L.S = S;
    const int rows = 32 * R;
    L.G = rows * S;
    L.vec = L.G + ((rows * (rows + 1) / 2 + 3) & ~3);
    L.per_warp = (L.vec + 256 + 3) & ~3;
    return L;
}

__device__ __forceinline__ float dot4v(const float4 a, const float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// sum over the warp, every lane receiving it
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One row of n <= 32 R ratings by one warp: row i of G (and of its factor)
// is held by lane i % 32 in slot i / 32; NB = 16, 32 or 64 is the width of
// the unrolled factorisation and solves (rows past n: the identity).
template <int R, int NB>
__device__ __forceinline__ void dual_warp_row(const SweepArgs &a, float *Fs, float *Gs, float *us, float *vs, int S,
                                              int64_t beg, int n, float lam_n, int lane, float (&u)[4], bool &ok,
                                              float *go) {
    static_assert(NB <= 32 * R, "rows per lane");
    const int nf = a.nf, nf4 = (nf + 3) & ~3;
    const bool act = 4 * lane < nf4;
    const float *F = reinterpret_cast<const float *>(a.F);
    // ---- 1. factor rows into shared memory, the first residual ------------
    float rv[R];  // lane l, slot r: the rating of row l + 32 r
#pragma unroll
    for (int r = 0; r < R; ++r) rv[r] = 0.0f;
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    for (int e0 = 0; e0 < n; e0 += 8) {
        float f[8][4], d[8], rr[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q;
            const bool in = e < n;
            const int64_t j = in ? a.idx[beg + e] : 0;
            rr[q] = in ? a.val[beg + e] : 0.0f;
            if (in && act) ld4f(F + j * a.ld + 4 * lane, f[q]);
            else f[q][0] = f[q][1] = f[q][2] = f[q][3] = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * lane + i >= nf) f[q][i] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            d[q] = u[0] * f[q][0];
#pragma unroll
            for (int i = 1; i < 4; ++i) d[q] = fmaf(u[i], f[q][i], d[q]);
        }
        warp_allsum8(d, lane);
        float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float er = e0 + q < n ? rr[q] - d[q] : 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) cs[i] = fmaf(er, f[q][i], cs[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], cs[i]);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + q;
            if (e < n && act)
                *reinterpret_cast<float4 *>(Fs + e * S + 4 * lane) = make_float4(f[q][0], f[q][1], f[q][2], f[q][3]);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (lane + 32 * r == e) rv[r] = rr[q];
        }
    }
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = 4 * lane + i < nf ? (acc[i] - cmp[i]) - lam_n * u[i] : 0.0f;
    // the row's gradient -2 (r0 - lambda n u0)
    if (go && 4 * lane < a.ld)
        *reinterpret_cast<float4 *>(go + 4 * lane) = make_float4(-2.0f * v[0], -2.0f * v[1], -2.0f * v[2], -2.0f * v[3]);
    __syncwarp();
    // ---- 2. G = F F^T (packed lower triangle), 2 x 2 tiles of rows ---------
    {
        const int np = (n + 1) >> 1, ntile = np * (np + 1) / 2;
        for (int tt = lane; tt < ntile; tt += 32) {
            int p, q;
            lt_first(tt, p, q);  // p >= q
            const float *a0 = Fs + 2 * p * S, *a1 = a0 + S, *b0 = Fs + 2 * q * S, *b1 = b0 + S;
            float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
            for (int k = 0; k < nf4; k += 4) {
                const float4 x0 = *reinterpret_cast<const float4 *>(a0 + k);
                const float4 x1 = *reinterpret_cast<const float4 *>(a1 + k);
                const float4 y0 = *reinterpret_cast<const float4 *>(b0 + k);
                const float4 y1 = *reinterpret_cast<const float4 *>(b1 + k);
                s00 += dot4v(x0, y0);
                s01 += dot4v(x0, y1);
                s10 += dot4v(x1, y0);
                s11 += dot4v(x1, y1);
            }
            // rows at or past n (an odd n's pair) hold stale values: their
            // entries are written but never read
            Gs[tri_off(2 * p) + 2 * q] = s00;
            if (p != q) Gs[tri_off(2 * p) + 2 * q + 1] = s01;
            Gs[tri_off(2 * p + 1) + 2 * q] = s10;
            Gs[tri_off(2 * p + 1) + 2 * q + 1] = s11;
        }
    }
    __syncwarp();
    // ---- 3. Cholesky of G + lambda n I --------------------------------------
    float g[R][NB];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float x = (i == j) ? 1.0f : 0.0f;
            if (i < n && j <= i) x = Gs[tri_off(i) + j] + (j == i ? lam_n : 0.0f);
            g[r][j] = x;
        }
    }
    bool bad = false;
    float rd[R];  // 1 / L[i][i] of the lane's rows
#pragma unroll
    for (int r = 0; r < R; ++r) rd[r] = 1.0f;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const float pj = __shfl_sync(0xffffffffu, g[j >> 5][j], j & 31);
        bad |= !(pj > 0.0f);
        const float rj = rsqrtf(pj);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            if (i == j) {
                g[r][j] = pj * rj;
                rd[r] = rj;
            } else if (i > j) {
                g[r][j] *= rj;
            }
        }
#pragma unroll
        for (int k = 1; k < NB; ++k) {
            if (k <= j) continue;
            const float lk = __shfl_sync(0xffffffffu, g[k >> 5][j], k & 31);
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (lane + 32 * r >= k) g[r][k] = fmaf(-g[r][j], lk, g[r][k]);
        }
    }
    if (bad) {
        ok = false;
        if (lane == 0) atomicAdd(a.notspd, 1);
        return;
    }
    // rows of L into shared memory: the backward solve reads its columns
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j <= i && i < NB) Gs[tri_off(i) + j] = g[r][j];
    }
    __syncwarp();
    const float inv_lam_n = 1.0f / lam_n;
    float dx[4];
    // dx = A^{-1} v = (v - F^T G^{-1} F v) / (lambda n); u += dx
    auto apply_inv = [&]() {
        if (act) *reinterpret_cast<float4 *>(vs + 4 * lane) = make_float4(v[0], v[1], v[2], v[3]);
        __syncwarp();
        float b[R], z[R], x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {  // lane l, slot r: f_e . v for rating e = l + 32 r
            const int e = lane + 32 * r;
            float w0 = 0.f, w1 = 0.f;
            if (e < n) {
                const float *fe = Fs + e * S;
                int k = 0;
                for (; k + 8 <= nf4; k += 8) {
                    w0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(vs + k));
                    w1 += dot4v(*reinterpret_cast<const float4 *>(fe + k + 4),
                                *reinterpret_cast<const float4 *>(vs + k + 4));
                }
                if (k < nf4)
                    w0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(vs + k));
            }
            b[r] = w0 + w1;
            z[r] = 0.0f;
            x[r] = 0.0f;
        }
        // L z = w, column by column
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float zj = __shfl_sync(0xffffffffu, b[j >> 5] * rd[j >> 5], j & 31);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = lane + 32 * r;
                if (i > j) b[r] = fmaf(-g[r][j], zj, b[r]);
                if (i == j) z[r] = zj;
            }
        }
        // L^T x = z, row j of L from shared memory
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
            const float xj = __shfl_sync(0xffffffffu, z[j >> 5] * rd[j >> 5], j & 31);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = lane + 32 * r;
                if (i < j) z[r] = fmaf(-Gs[tri_off(j) + i], xj, z[r]);
                if (i == j) x[r] = xj;
            }
        }
        // q = F^T x, a lane per 4-wide slot
        float qv[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = 0; e < n; ++e) {
            const float xe = R == 1 ? __shfl_sync(0xffffffffu, x[0], e & 31)
                                    : __shfl_sync(0xffffffffu, e < 32 ? x[0] : x[R - 1], e & 31);
            if (act) {
                const float4 fe = *reinterpret_cast<const float4 *>(Fs + e * S + 4 * lane);
                qv[0] = fmaf(fe.x, xe, qv[0]);
                qv[1] = fmaf(fe.y, xe, qv[1]);
                qv[2] = fmaf(fe.z, xe, qv[2]);
                qv[3] = fmaf(fe.w, xe, qv[3]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            dx[i] = 4 * lane + i < nf ? (v[i] - qv[i]) * inv_lam_n : 0.0f;
            u[i] += dx[i];
        }
        __syncwarp();
    };
    apply_inv();
    for (int s = 1; s < a.refine; ++s) {
        // the stopping rule of sw_correction_small, over the warp
        float d2 = 0.f, u2 = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            d2 = fmaf(dx[i], dx[i], d2);
            u2 = fmaf(u[i], u[i], u2);
        }
        d2 = warp_sum(d2);
        u2 = warp_sum(u2);
        const float rho = 0x1p-17f + (float)n * 0x1p-24f;
        if (d2 * rho * rho <= 0x1p-42f * u2) break;
        // the FP32 residual at u: lane l forms r_e - f_e . u for its ratings
        // e = l + 32 r, then a lane per slot sums f_e (r_e - f_e . u) over the
        // ratings (compensated by 8)
        if (act) *reinterpret_cast<float4 *>(us + 4 * lane) = make_float4(u[0], u[1], u[2], u[3]);
        __syncwarp();
        float er[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = lane + 32 * r;
            float de0 = 0.f, de1 = 0.f;
            if (e < n) {
                const float *fe = Fs + e * S;
                int k = 0;
                for (; k + 8 <= nf4; k += 8) {
                    de0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(us + k));
                    de1 += dot4v(*reinterpret_cast<const float4 *>(fe + k + 4),
                                 *reinterpret_cast<const float4 *>(us + k + 4));
                }
                if (k < nf4)
                    de0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(us + k));
            }
            er[r] = e < n ? rv[r] - (de0 + de1) : 0.0f;
        }
        float ra[4] = {0.f, 0.f, 0.f, 0.f}, rc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e0 = 0; e0 < n; e0 += 8) {
            float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q;
                const float ere = R == 1 ? __shfl_sync(0xffffffffu, er[0], e & 31)
                                         : __shfl_sync(0xffffffffu, e < 32 ? er[0] : er[R - 1], e & 31);
                if (e < n && act) {
                    const float4 fe = *reinterpret_cast<const float4 *>(Fs + e * S + 4 * lane);
                    cs[0] = fmaf(ere, fe.x, cs[0]);
                    cs[1] = fmaf(ere, fe.y, cs[1]);
                    cs[2] = fmaf(ere, fe.z, cs[2]);
                    cs[3] = fmaf(ere, fe.w, cs[3]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) kadd(ra[i], rc[i], cs[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = 4 * lane + i < nf ? (ra[i] - rc[i]) - lam_n * u[i] : 0.0f;
        __syncwarp();
        apply_inv();
    }
}

template <int R>
__global__ void __launch_bounds__(32 * wd_warps(R)) k_sweep_dual_warp(SweepArgs a, int nmax) {
    extern __shared__ __align__(16) float smw[];
    const int nf = a.nf;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpDualLayout L = wdual_layout(nf, R);
    float *Fs = smw + warp * L.per_warp;
    float *Gs = Fs + L.G;
    float *us = Fs + L.vec, *vs = us + 128;
    const int64_t r = (int64_t)blockIdx.x * wd_warps(R) + warp;
    if (r >= a.nrows) return;  // a whole warp: nothing below waits for another warp
    const int64_t row = a.order ? a.order[r] : r;
    const int64_t beg = a.ptr[row];
    const int n = (int)(a.ptr[row + 1] - beg);
    const float *xi = a.Xin ? reinterpret_cast<const float *>(a.Xin) + row * a.ld : nullptr;
    float *xo = reinterpret_cast<float *>(a.Xout) + row * a.ld;
    float *gb = a.Gbar ? reinterpret_cast<float *>(a.Gbar) + row * a.ld : nullptr;
    float *go = a.Gout ? reinterpret_cast<float *>(a.Gout) + row * a.ld : nullptr;
    const float lam_n = (float)(a.lambda * (double)n);
    // rows longer than the launch's bound are not this kernel's (the host
    // never passes one): they keep their value and count as not solved
    bool ok = n > 0 && n <= nmax && lam_n > 0.0f;
    if (n > nmax && lane == 0) atomicAdd(a.notspd, 1);
    float u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
    if (ok) {
        if constexpr (R == 1) {
            if (n <= 16) dual_warp_row<1, 16>(a, Fs, Gs, us, vs, L.S, beg, n, lam_n, lane, u, ok, go);
            else dual_warp_row<1, 32>(a, Fs, Gs, us, vs, L.S, beg, n, lam_n, lane, u, ok, go);
        } else {
            dual_warp_row<2, 64>(a, Fs, Gs, us, vs, L.S, beg, n, lam_n, lane, u, ok, go);
        }
    }
    if (!ok) {
        // no ratings (lambda n_i = 0): the row's solution is 0; a
        // factorisation failure keeps the current value
#pragma unroll
        for (int i = 0; i < 4; ++i) u[i] = (n > 0 && xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
    }
    if (4 * lane < a.ld) {
        float o[4], xk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[i] = 4 * lane + i < nf ? u[i] : 0.0f;
            xk[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
        }
        *reinterpret_cast<float4 *>(xo + 4 * lane) = make_float4(o[0], o[1], o[2], o[3]);
        if (gb) *reinterpret_cast<float4 *>(gb + 4 * lane) = make_float4(xk[0] - o[0], xk[1] - o[1], xk[2] - o[2],
                                                                         xk[3] - o[3]);
        if (go && n <= 0) *reinterpret_cast<float4 *>(go + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

}  // namespace

// rows (a suffix of the degree order) of at most nmax <= ALS_DUAL_SMALL
// ratings: a warp each
als_status launch_sweep_dual_warp(als_ctx *c, const SweepArgs &a, int nmax) {
    if (a.nrows <= 0) return ALS_OK;
    if (a.nf > ALS_TC_LD || nmax < 1 || nmax > ALS_DUAL_SMALL) {
        als_set_error("sweep: the warp light-row solve supports n_f <= 128 and rows of at most 32 ratings");
        return ALS_ENOTSUP;
    }
    constexpr int R = 1;
    const int warps = wd_warps(R);
    const int64_t blocks = (a.nrows + warps - 1) / warps;
    if (blocks > (int64_t)INT32_MAX) {
        als_set_error("sweep: more rows than CTAs in one launch");
        return ALS_ENOTSUP;
    }
    const WarpDualLayout L = wdual_layout(a.nf, R);
    const size_t smem = (size_t)warps * L.per_warp * sizeof(float);
    const void *fn = (const void *)k_sweep_dual_warp<R>;
    if (raise_smem_limit(fn, smem) != ALS_OK) return ALS_ECUDA;
    ALS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    cudaStream_t st = a.stream ? a.stream : c->stream;
    kt_begin(c, KT_DUAL, st);
    k_sweep_dual_warp<R><<<(unsigned)blocks, 32 * warps, smem, st>>>(a, nmax);
    kt_end(c, KT_DUAL, st);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}
