// Mixed-precision half sweep for light rows: a row with n_i <= 64 ratings
// and n_i <= n_f is solved through the n_i x n_i matrix
//     G = F F^T + lambda n_i I        (F: the row's n_i fixed-side factor rows)
// instead of the n_f x n_f matrix A = F^T F + lambda n_i I of Eq. (4).  The
// two give the same solution of Eq. (4): by the Woodbury identity
//     A^{-1} v = (v - F^T G^{-1} F v) / (lambda n_i),
// so A^{-1} is applied with a Cholesky factorisation of G alone, n_i^3 / 3
// flops instead of n_f^3 / 3 (a user of ML20M size has a median of 42
// ratings against n_f = 100).
//
// The refinement is the tensor-core kernel's: from u0 = x_i, u <- u + A^{-1}
// res with res = sum_e f_e (r_e - f_e . u) - lambda n_i u in FP32
// (compensated), the first residual formed while the factor rows are read,
// and the same stopping rule.  Only the approximate inverse differs: G in FP32
// from the FP32 factor rows.  Its error, like that of the Cholesky factor of
// A, is of order kappa(A) times FP32 rounding.
//
// One CTA of 128 threads per row.  The row's factor rows are read from global
// memory once, into shared memory (row stride S floats, S / 4 odd, so that
// 16-byte accesses of eight consecutive rows fall in distinct bank groups);
// every later product with F, F^T and every later residual reads them there.
#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

constexpr int DU_THREADS = 128;

struct DualLayout {
    int S;        // shared-memory row stride of F (floats)
    int G;        // packed lower triangle of G (float offset)
    int vec;      // vectors (float offset)
    int total;    // floats
};

// nmax: the most ratings of any row of the launch (<= ALS_DUAL_MAX)
__host__ __device__ inline DualLayout dual_layout(int nf, int nmax) {
    DualLayout L;
    int S = (nf + 3) & ~3;
    if (((S >> 2) & 1) == 0) S += 4;
    L.S = S;
    const int rows = (nmax + 3) & ~3;
    L.G = rows * S;
    L.vec = L.G + ((nmax * (nmax + 1) / 2 + 3) & ~3);
    // u, v, dx [3][132]; w, z, zz, diag, rv [5][64]; part [4][128] aliased
    // with the Cholesky scratch (8 * 128 + 64 + 1 floats, padded)
    L.total = L.vec + 3 * 132 + 5 * 64 + 1104;
    return L;
}

// sum over k < nf4 of p[k] q[k] for 16-byte aligned p, q (shared memory)
__device__ __forceinline__ float dot_sm(const float *p, const float *q, int nf4, int k0, int kstep) {
    float s0 = 0.0f, s1 = 0.0f;
    for (int k = 4 * k0; k < nf4; k += 4 * kstep) {
        const float4 a = *reinterpret_cast<const float4 *>(p + k);
        const float4 b = *reinterpret_cast<const float4 *>(q + k);
        s0 = fmaf(a.x, b.x, s0);
        s1 = fmaf(a.y, b.y, s1);
        s0 = fmaf(a.z, b.z, s0);
        s1 = fmaf(a.w, b.w, s1);
    }
    return s0 + s1;
}

template <int MINB>
__global__ void __launch_bounds__(DU_THREADS, MINB) k_sweep_dual(SweepArgs a, int nmax) {
    extern __shared__ __align__(16) float sm[];
    const int nf = a.nf, nf4 = (nf + 3) & ~3;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const DualLayout L = dual_layout(nf, nmax);
    const int S = L.S;
    float *Fs = sm;
    float *G = sm + L.G;
    float *vec = sm + L.vec;
    float *u = vec, *v = vec + 132, *dx = vec + 264;
    float *w = vec + 396, *z = w + 64, *zz = w + 128, *diag = w + 192, *rv = w + 256;
    float *part = w + 320;   // residual partials [4][128] (residual phases)
    float *work = w + 320;   // Cholesky scratch (factorisation phase)
    const float *F = reinterpret_cast<const float *>(a.F);

    for (int64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {
        const int64_t row = a.order ? a.order[r] : r;
        const int64_t beg = a.ptr[row];
        const int n = (int)(a.ptr[row + 1] - beg);
        const float *xi = a.Xin ? reinterpret_cast<const float *>(a.Xin) + row * a.ld : nullptr;
        float *xo = reinterpret_cast<float *>(a.Xout) + row * a.ld;
        float *gb = a.Gbar ? reinterpret_cast<float *>(a.Gbar) + row * a.ld : nullptr;
        const float lam_n = (float)(a.lambda * (double)n);
        // rows longer than the launch's bound are not this kernel's (the host
        // never passes one): they keep their value and count as not solved
        bool ok = n > 0 && n <= nmax && lam_n > 0.0f;
        if (n > nmax && t == 0) atomicAdd(a.notspd, 1);
        const bool act = 4 * lane < nf4;
        float uu[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) uu[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
        for (int k = t; k < 132; k += DU_THREADS) u[k] = (xi && k < nf) ? xi[k] : 0.0f;
        if (ok) {
            // ---- 1. factor rows into shared memory (features >= n_f zeroed),
            //      with the first residual sum_e f_e (r_e - f_e . u0) ---------
            float acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
            for (int e0 = 0; e0 < n; e0 += 32) {
                int32_t cj[8];
                float cr[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = e0 + warp + 4 * q;
                    cj[q] = e < n ? a.idx[beg + e] : -1;
                    cr[q] = e < n ? a.val[beg + e] : 0.0f;
                }
                float f[8][4];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (cj[q] >= 0 && act) ld4f(F + (int64_t)cj[q] * a.ld + 4 * lane, f[q]);
                    else f[q][0] = f[q][1] = f[q][2] = f[q][3] = 0.0f;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (4 * lane + i >= nf) f[q][i] = 0.0f;
                }
                float d[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    d[q] = uu[0] * f[q][0];
#pragma unroll
                    for (int i = 1; i < 4; ++i) d[q] = fmaf(uu[i], f[q][i], d[q]);
                }
                warp_allsum8(d, lane);
                float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float er = cj[q] >= 0 ? cr[q] - d[q] : 0.0f;
#pragma unroll
                    for (int i = 0; i < 4; ++i) cs[i] = fmaf(er, f[q][i], cs[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], cs[i]);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = e0 + warp + 4 * q;
                    if (e < n) {
                        if (act)
                            *reinterpret_cast<float4 *>(Fs + e * S + 4 * lane) =
                                make_float4(f[q][0], f[q][1], f[q][2], f[q][3]);
                        if (lane == 0) rv[e] = cr[q];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) part[warp * 128 + 4 * lane + i] = acc[i] - cmp[i];
            __syncthreads();
            // v = r0 - lambda n u0 (fixed order over the warps), zero past n_f
            for (int k = t; k < nf4; k += DU_THREADS)
                v[k] = k < nf ? ((part[k] + part[128 + k]) + (part[256 + k] + part[384 + k])) - lam_n * u[k] : 0.0f;
            // the row's gradient -2 (r0 - lambda n u0) (ld = nf4 slots)
            if (a.Gout)
                for (int k = t; k < a.ld; k += DU_THREADS)
                    reinterpret_cast<float *>(a.Gout)[row * a.ld + k] = k < nf ? -2.0f * v[k] : 0.0f;
            // ---- 2. G = F F^T + lambda n I, lower triangle, 4 x 4 tiles ------
            {
                const int nt = (n + 3) >> 2;
                const int ntiles = nt * (nt + 1) / 2;
                for (int p = t; p < ntiles; p += DU_THREADS) {
                    int ti = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
                    while (ti * (ti + 1) / 2 > p) --ti;
                    while ((ti + 1) * (ti + 2) / 2 <= p) ++ti;
                    const int tj = p - ti * (ti + 1) / 2;
                    float g[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) g[i][j] = 0.0f;
                    // rows past n (tile padding) are read but never stored
                    const float *Fi = Fs + 4 * ti * S, *Fj = Fs + 4 * tj * S;
                    for (int k = 0; k < nf4; k += 4) {
                        float4 x[4], y[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            x[i] = *reinterpret_cast<const float4 *>(Fi + i * S + k);
                            y[i] = *reinterpret_cast<const float4 *>(Fj + i * S + k);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                g[i][j] = fmaf(x[i].x, y[j].x, g[i][j]);
                                g[i][j] = fmaf(x[i].y, y[j].y, g[i][j]);
                                g[i][j] = fmaf(x[i].z, y[j].z, g[i][j]);
                                g[i][j] = fmaf(x[i].w, y[j].w, g[i][j]);
                            }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int gi = 4 * ti + i, gj = 4 * tj + j;
                            if (gi < n && gj <= gi) G[tri_off(gi) + gj] = g[i][j] + (gi == gj ? lam_n : 0.0f);
                        }
                }
            }
            __syncthreads();
            // ---- 3. Cholesky of G (inverted diagonal blocks) -----------------
            ok = chol_blocked128(G, n, diag, work, t, 32 * (int)(blockIdx.x & 3));
            if (ok) invert_diag_blocks128(G, n, diag, t);
            if (!ok && t == 0) atomicAdd(a.notspd, 1);
        }
        if (ok) {
            const float inv_lam_n = 1.0f / lam_n;
            // dx = A^{-1} v = (v - F^T G^{-1} F v) / (lambda n); u += dx
            auto apply_inv = [&]() {
                __syncthreads();  // v complete
                {
                    const int e = t >> 1, h = t & 1;  // two threads per rating
                    float s = e < n ? dot_sm(Fs + e * S, v, nf4, h, 2) : 0.0f;
                    s += __shfl_xor_sync(0xffffffffu, s, 1);
                    if (e < n && h == 0) w[e] = s;
                }
                trisolve_inv128(G, n, w, zz, z, t);  // barriers on entry and exit
                for (int k = t; k < nf; k += DU_THREADS) {
                    float q0 = 0.0f, q1 = 0.0f;
                    int e = 0;
                    for (; e + 1 < n; e += 2) {
                        q0 = fmaf(Fs[e * S + k], z[e], q0);
                        q1 = fmaf(Fs[(e + 1) * S + k], z[e + 1], q1);
                    }
                    if (e < n) q0 = fmaf(Fs[e * S + k], z[e], q0);
                    dx[k] = (v[k] - (q0 + q1)) * inv_lam_n;
                    u[k] += dx[k];
                }
            };
            apply_inv();
            for (int s = 1; s < a.refine; ++s) {
                if (sw_correction_small<float, DU_THREADS>(dx, u, nf, n, part, t)) break;
                // residual at u from the factor rows in shared memory: a warp
                // takes ratings warp + 4 q, a lane a 4-wide slot of the row
                float uk[4], ak[4] = {0.f, 0.f, 0.f, 0.f}, ck[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 4; ++i) uk[i] = (4 * lane + i < nf) ? u[4 * lane + i] : 0.0f;
                for (int e0 = 0; e0 < n; e0 += 32) {
                    float f[8][4], d[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int e = e0 + warp + 4 * q;
                        if (e < n && act) ld4f(Fs + e * S + 4 * lane, f[q]);
                        else f[q][0] = f[q][1] = f[q][2] = f[q][3] = 0.0f;
                        d[q] = uk[0] * f[q][0];
#pragma unroll
                        for (int i = 1; i < 4; ++i) d[q] = fmaf(uk[i], f[q][i], d[q]);
                    }
                    warp_allsum8(d, lane);
                    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int e = e0 + warp + 4 * q;
                        const float er = e < n ? rv[e] - d[q] : 0.0f;
#pragma unroll
                        for (int i = 0; i < 4; ++i) cs[i] = fmaf(er, f[q][i], cs[i]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) kadd(ak[i], ck[i], cs[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) part[warp * 128 + 4 * lane + i] = ak[i] - ck[i];
                __syncthreads();
                for (int k = t; k < nf4; k += DU_THREADS)
                    v[k] = k < nf ? ((part[k] + part[128 + k]) + (part[256 + k] + part[384 + k])) - lam_n * u[k]
                                  : 0.0f;
                apply_inv();
            }
        } else {
            // no ratings (lambda n_i = 0): the row's solution is 0; a
            // factorisation failure keeps the current value
            for (int k = t; k < nf; k += DU_THREADS) u[k] = (n > 0 && xi) ? xi[k] : 0.0f;
        }
        __syncthreads();
        for (int k = t; k < a.ld; k += DU_THREADS) {
            const float uk = k < nf ? u[k] : 0.0f;
            const float xk = xi ? xi[k] : 0.0f;
            xo[k] = uk;
            if (gb) gb[k] = xk - uk;
            if (a.Gout && n <= 0) reinterpret_cast<float *>(a.Gout)[row * a.ld + k] = 0.0f;
        }
        __syncthreads();
    }
}

}  // namespace

als_status launch_sweep_dual_warp(als_ctx *c, const SweepArgs &a, int nmax);  // sweep_dual_warp.cu

namespace {

// nmax <= ALS_DUAL_SMALL: a layout of ~23 KB (n_f = 100) and a register
// budget of 72 per thread, so that 7 CTAs fit per SM; longer rows ~43 KB, 5
template <int MINB>
als_status launch_dual(als_ctx *c, const SweepArgs &a, int nmax) {
    const DualLayout L = dual_layout(a.nf, nmax);
    const size_t smem = (size_t)L.total * sizeof(float);
    if (raise_smem_limit((const void *)k_sweep_dual<MINB>, smem) != ALS_OK) return ALS_ECUDA;
    ALS_CUDA_TRY(cudaFuncSetAttribute(k_sweep_dual<MINB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    cudaStream_t st = a.stream ? a.stream : c->stream;
    kt_begin(c, KT_DUAL, st);
    k_sweep_dual<MINB><<<(unsigned)a.nrows, DU_THREADS, smem, st>>>(a, nmax);
    kt_end(c, KT_DUAL, st);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

}  // namespace

als_status launch_sweep_dual(als_ctx *c, const SweepArgs &a, int nmax) {
    if (a.nrows <= 0) return ALS_OK;
    if (a.nf > ALS_TC_LD || nmax < 1 || nmax > ALS_DUAL_MAX) {
        als_set_error("sweep: the light-row solve supports n_f <= 128 and rows of at most 64 ratings");
        return ALS_ENOTSUP;
    }
    if (a.nrows > (int64_t)INT32_MAX) {
        als_set_error("sweep: more rows than CTAs in one launch");
        return ALS_ENOTSUP;
    }
    if (nmax <= ALS_DUAL_SMALL) return c->dual_warp ? launch_sweep_dual_warp(c, a, nmax) : launch_dual<7>(c, a, nmax);
    // the rows (a suffix of the degree order) of at most ALS_DUAL_SMALL
    // ratings in the smaller layout, the longer ones before them
    const int64_t ns = a.order ? std::max<int64_t>(0, std::min(a.ndual_small, a.nrows)) : 0;
    if (ns < a.nrows) {
        SweepArgs l = a;
        l.nrows = a.nrows - ns;
        als_status s = launch_dual<5>(c, l, nmax);
        if (s != ALS_OK) return s;
    }
    if (ns == 0) return ALS_OK;
    SweepArgs sm = a;
    sm.order = a.order + (a.nrows - ns);
    sm.nrows = ns;
    return c->dual_warp ? launch_sweep_dual_warp(c, sm, ALS_DUAL_SMALL) : launch_dual<7>(c, sm, ALS_DUAL_SMALL);
}
