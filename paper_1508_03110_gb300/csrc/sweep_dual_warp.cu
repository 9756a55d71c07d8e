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
//   3. Cholesky of G with lane i holding row i in registers: column j's
//      pivot and entries reach the other lanes by shuffles (rows past n_i
//      are the identity);
//   4. each correction: w = F v (lane e: rating e), L z = w by columns
//      (shuffles), L^T x = z by rows of L from shared memory, q = F^T x (a
//      lane per slot), dx = (v - q) / (lambda n_i);
//   5. further corrections (the shared stopping rule, sw_correction_small's
//      rule over the warp) recompute the FP32 residual from the rows in
//      shared memory.
// Rows of at most 16 ratings run the 16-wide forms of steps 3-4.
#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

constexpr int WD_WARPS = 2;  // rows per CTA

struct WarpDualLayout {
    int S;         // row stride of the factor rows (floats), S / 4 odd
    int G;         // [32][33] G, then its factor L (float offset)
    int vec;       // u, v [2][128] (float offset)
    int per_warp;  // floats per warp
};

__host__ __device__ inline WarpDualLayout wdual_layout(int nf) {
    WarpDualLayout L;
    int S = (nf + 3) & ~3;
    if (((S >> 2) & 1) == 0) S += 4;
    L.S = S;
    L.G = 32 * S;
    L.vec = L.G + 32 * 33;
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

template <int NB>
__device__ __forceinline__ void dual_warp_row(const SweepArgs &a, float *Fs, float *Gs, float *us, float *vs, int S,
                                              int64_t beg, int n, const float *xi, float lam_n, int lane,
                                              float (&u)[4], bool &ok) {
    const int nf = a.nf, nf4 = (nf + 3) & ~3;
    const bool act = 4 * lane < nf4;
    const float *F = reinterpret_cast<const float *>(a.F);
    // ---- 1. factor rows into shared memory, the first residual ------------
    float rv = 0.0f;  // lane e: rating e
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
            if (lane == e) rv = rr[q];
        }
    }
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = 4 * lane + i < nf ? (acc[i] - cmp[i]) - lam_n * u[i] : 0.0f;
    __syncwarp();
    // ---- 2. G = F F^T (lower triangle), 2 x 2 tiles of rows ----------------
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
            Gs[(2 * p) * 33 + 2 * q] = s00;
            Gs[(2 * p) * 33 + 2 * q + 1] = s01;
            Gs[(2 * p + 1) * 33 + 2 * q] = s10;
            Gs[(2 * p + 1) * 33 + 2 * q + 1] = s11;
        }
    }
    __syncwarp();
    // ---- 3. Cholesky of G + lambda n I, lane i = row i ------------------------
    float g[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        float x = (lane == j) ? 1.0f : 0.0f;
        if (lane < n && j <= lane) x = Gs[lane * 33 + j] + (j == lane ? lam_n : 0.0f);
        g[j] = x;
    }
    bool bad = false;
    float rd = 1.0f;  // 1 / L[lane][lane]
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const float pj = __shfl_sync(0xffffffffu, g[j], j);
        bad |= !(pj > 0.0f);
        const float rj = rsqrtf(pj);
        if (lane == j) {
            g[j] = pj * rj;
            rd = rj;
        } else if (lane > j) {
            g[j] *= rj;
        }
#pragma unroll
        for (int k = 1; k < NB; ++k) {
            if (k <= j) continue;
            const float lk = __shfl_sync(0xffffffffu, g[j], k);
            if (lane >= k) g[k] = fmaf(-g[j], lk, g[k]);
        }
    }
    if (bad) {
        ok = false;
        if (lane == 0) atomicAdd(a.notspd, 1);
        return;
    }
    // rows of L into shared memory: the backward solve reads its columns
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j <= lane && lane < NB) Gs[lane * 33 + j] = g[j];
    __syncwarp();
    const float inv_lam_n = 1.0f / lam_n;
    float dx[4];
    // dx = A^{-1} v = (v - F^T G^{-1} F v) / (lambda n); u += dx
    auto apply_inv = [&]() {
        if (act) *reinterpret_cast<float4 *>(vs + 4 * lane) = make_float4(v[0], v[1], v[2], v[3]);
        __syncwarp();
        float w0 = 0.f, w1 = 0.f;  // lane e: f_e . v
        if (lane < n) {
            const float *fe = Fs + lane * S;
            int k = 0;
            for (; k + 8 <= nf4; k += 8) {
                w0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(vs + k));
                w1 += dot4v(*reinterpret_cast<const float4 *>(fe + k + 4),
                            *reinterpret_cast<const float4 *>(vs + k + 4));
            }
            if (k < nf4)
                w0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(vs + k));
        }
        // L z = w, column by column
        float b = w0 + w1, z = 0.0f;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float zj = __shfl_sync(0xffffffffu, b * rd, j);
            if (lane > j) b = fmaf(-g[j], zj, b);
            if (lane == j) z = zj;
        }
        // L^T x = z, row j of L from shared memory
        float x = 0.0f;
#pragma unroll
        for (int j = NB - 1; j >= 0; --j) {
            const float xj = __shfl_sync(0xffffffffu, z * rd, j);
            if (lane < j) z = fmaf(-Gs[j * 33 + lane], xj, z);
            if (lane == j) x = xj;
        }
        // q = F^T x, a lane per 4-wide slot
        float qv[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = 0; e < n; ++e) {
            const float xe = __shfl_sync(0xffffffffu, x, e);
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
        // the FP32 residual at u: lane e forms r_e - f_e . u, then a lane per
        // slot sums f_e (r_e - f_e . u) over the ratings (compensated by 8)
        if (act) *reinterpret_cast<float4 *>(us + 4 * lane) = make_float4(u[0], u[1], u[2], u[3]);
        __syncwarp();
        float de0 = 0.f, de1 = 0.f;
        if (lane < n) {
            const float *fe = Fs + lane * S;
            int k = 0;
            for (; k + 8 <= nf4; k += 8) {
                de0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(us + k));
                de1 += dot4v(*reinterpret_cast<const float4 *>(fe + k + 4),
                             *reinterpret_cast<const float4 *>(us + k + 4));
            }
            if (k < nf4)
                de0 += dot4v(*reinterpret_cast<const float4 *>(fe + k), *reinterpret_cast<const float4 *>(us + k));
        }
        const float er = lane < n ? rv - (de0 + de1) : 0.0f;
        float ra[4] = {0.f, 0.f, 0.f, 0.f}, rc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e0 = 0; e0 < n; e0 += 8) {
            float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q;
                const float ere = __shfl_sync(0xffffffffu, er, e & 31);
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

__global__ void __launch_bounds__(32 * WD_WARPS) k_sweep_dual_warp(SweepArgs a) {
    extern __shared__ __align__(16) float smw[];
    const int nf = a.nf;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpDualLayout L = wdual_layout(nf);
    float *Fs = smw + warp * L.per_warp;
    float *Gs = Fs + L.G;
    float *us = Fs + L.vec, *vs = us + 128;
    const int64_t r = (int64_t)blockIdx.x * WD_WARPS + warp;
    if (r >= a.nrows) return;  // a whole warp: nothing below waits for another warp
    const int64_t row = a.order ? a.order[r] : r;
    const int64_t beg = a.ptr[row];
    const int n = (int)(a.ptr[row + 1] - beg);
    const float *xi = a.Xin ? reinterpret_cast<const float *>(a.Xin) + row * a.ld : nullptr;
    float *xo = reinterpret_cast<float *>(a.Xout) + row * a.ld;
    float *gb = a.Gbar ? reinterpret_cast<float *>(a.Gbar) + row * a.ld : nullptr;
    const float lam_n = (float)(a.lambda * (double)n);
    // rows longer than 32 ratings are not this kernel's (the host never
    // passes one): they keep their value and count as not solved
    bool ok = n > 0 && n <= 32 && lam_n > 0.0f;
    if (n > 32 && lane == 0) atomicAdd(a.notspd, 1);
    float u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
    if (ok) {
        if (n <= 16) dual_warp_row<16>(a, Fs, Gs, us, vs, L.S, beg, n, xi, lam_n, lane, u, ok);
        else dual_warp_row<32>(a, Fs, Gs, us, vs, L.S, beg, n, xi, lam_n, lane, u, ok);
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
    }
}

}  // namespace

// the suffix of the degree order with at most 32 ratings per row: a warp each
als_status launch_sweep_dual_warp(als_ctx *c, const SweepArgs &a) {
    if (a.nrows <= 0) return ALS_OK;
    if (a.nf > ALS_TC_LD) {
        als_set_error("sweep: the light-row solve supports n_f <= 128");
        return ALS_ENOTSUP;
    }
    const int64_t blocks = (a.nrows + WD_WARPS - 1) / WD_WARPS;
    if (blocks > (int64_t)INT32_MAX) {
        als_set_error("sweep: more rows than CTAs in one launch");
        return ALS_ENOTSUP;
    }
    const WarpDualLayout L = wdual_layout(a.nf);
    const size_t smem = (size_t)WD_WARPS * L.per_warp * sizeof(float);
    if (raise_smem_limit((const void *)k_sweep_dual_warp, smem) != ALS_OK) return ALS_ECUDA;
    ALS_CUDA_TRY(cudaFuncSetAttribute(k_sweep_dual_warp, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    cudaStream_t st = a.stream ? a.stream : c->stream;
    kt_begin(c, KT_DUAL, st);
    k_sweep_dual_warp<<<(unsigned)blocks, 32 * WD_WARPS, smem, st>>>(a);
    kt_end(c, KT_DUAL, st);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}
