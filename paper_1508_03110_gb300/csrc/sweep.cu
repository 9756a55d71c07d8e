// One half of an ALS sweep (Algorithm 1): for every row i of one side, with
// the other side F fixed,
//     A_i = sum_{e in row i} f_e f_e^T + lambda n_i I,   v_i = sum_e r_e f_e,
//     x_i <- A_i^{-1} v_i                                   (Eq. 3 / Eq. 4)
// fused in one kernel per row group: the gathered factor rows are staged in
// shared memory, the Gram matrix is accumulated in registers, factored by a
// right-looking Cholesky in shared memory and solved by two triangular
// sweeps; nothing but the solved row (and gbar = x - xbar) reaches HBM.
//
// FP64 (parity form): the definition above, solved from scratch.
// FP32 (mixed form): the Gram matrix is the (approximate) preconditioner of an
// iterative refinement started at the current row x_i:
//     res = sum_e f_e (r_e - f_e . u) - lambda n_i u   (FP32, matrix free)
//     u  <- u + A_i^{-1} res                           (refine times)
// which converges to the same A_i^{-1} v_i; its error shrinks with the step.
// The tensor-core Gram (n_f > 64) lives in sweep_tc.cu and shares the solve
// code below.
#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

constexpr int CH = 32;  // ratings staged per chunk

template <typename T>
__host__ __device__ inline size_t group_smem_elems(int nf) {
    const int ldA = nf + 1;
    return (size_t)nf * ldA + (size_t)CH * ldA + 2 * CH + 5 * (size_t)nf;
}

// upper-triangle entry enumeration (k <= l), row-major in k
__device__ __forceinline__ void tri_first(int t, int nf, int &k, int &l) {
    k = 0;
    int rem = t;
    while (k < nf && rem >= nf - k) { rem -= nf - k; ++k; }
    l = k + rem;
}
__device__ __forceinline__ void tri_next(int step, int nf, int &k, int &l) {
    int rem = l - k + step;
    while (k < nf && rem >= nf - k) { rem -= nf - k; ++k; }
    l = k + rem;
}

template <typename T, int TPR>
__device__ __forceinline__ void stage_chunk(const SweepArgs &a, const T *F, int64_t base, int cn, T *Fc,
                                            T *rc, int ldA, int t) {
    const int nv = a.ld / 4;
    for (int q = t; q < cn * nv; q += TPR) {
        const int c = q / nv, v = q - c * nv;
        const int64_t j = a.idx[base + c];
        T x[4];
        sw_ld4(F + j * a.ld + 4 * v, x);
        T *dst = Fc + c * ldA + 4 * v;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * v + i < a.nf) dst[i] = x[i];
    }
    for (int c = t; c < cn; c += TPR) rc[c] = (T)a.val[base + c];
}

template <typename T, int TPR, int MAXE, bool WARM>
__global__ void __launch_bounds__(128) k_sweep_fma(SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nf = a.nf, ldA = nf + 1;
    const int G = blockDim.x / TPR, g = threadIdx.x / TPR, t = threadIdx.x - g * TPR;
    T *A = reinterpret_cast<T *>(smem_raw) + (size_t)g * group_smem_elems<T>(nf);
    T *Fc = A + nf * ldA;
    T *rc = Fc + CH * ldA;
    T *err = rc + CH;
    T *colk = err + CH;
    T *v1 = colk + nf;
    T *v2 = v1 + nf;
    T *u = v2 + nf;
    T *diag = u + nf;
    const T *F = reinterpret_cast<const T *>(a.F);
    const int NT = nf * (nf + 1) / 2;

    for (int64_t r = (int64_t)blockIdx.x * G + g; r < a.nrows; r += (int64_t)gridDim.x * G) {
        const bool seg = a.seg_out != nullptr;  // a slice of a split row: partials only
        const int64_t row = seg ? a.order[a.seg_row[r]] : (a.order ? a.order[r] : r);
        const int64_t beg = seg ? a.seg_beg[r] : a.ptr[row];
        const int n = seg ? a.seg_len[r] : (int)(a.ptr[row + 1] - beg);
        const T *xi = a.Xin ? reinterpret_cast<const T *>(a.Xin) + row * a.ld : nullptr;
        T *xo = reinterpret_cast<T *>(a.Xout) + row * a.ld;
        T *gb = a.Gbar ? reinterpret_cast<T *>(a.Gbar) + row * a.ld : nullptr;
        const T lam_n = (T)(a.lambda * (double)n);
        bool ok = n > 0;
        if (ok) {
            // ---- Gram matrix (upper triangle in registers) and, cold, the RHS
            T acc[MAXE];
#pragma unroll
            for (int q = 0; q < MAXE; ++q) acc[q] = T(0);
            T vacc = T(0), vcmp = T(0);
            if (WARM && seg) {  // the slice's residual is taken at the row's current value
                for (int k = t; k < nf; k += TPR) u[k] = xi ? xi[k] : T(0);
            }
            for (int c0 = 0; c0 < n; c0 += CH) {
                const int cn = min(CH, n - c0);
                sw_gsync<TPR>();
                stage_chunk<T, TPR>(a, F, beg + c0, cn, Fc, rc, ldA, t);
                sw_gsync<TPR>();
                if (WARM && seg) {
                    for (int c = t; c < cn; c += TPR) {
                        T d = T(0);
                        for (int k = 0; k < nf; ++k) d = fma(Fc[c * ldA + k], u[k], d);
                        err[c] = rc[c] - d;
                    }
                    sw_gsync<TPR>();
                    if (t < nf)
                        for (int c = 0; c < cn; ++c) kadd(vacc, vcmp, err[c] * Fc[c * ldA + t]);
                }
                int k, l;
                tri_first(t, nf, k, l);
#pragma unroll
                for (int q = 0; q < MAXE; ++q) {
                    if (t + q * TPR < NT) {
                        const T *pk = Fc + k, *pl = Fc + l;
                        T s = T(0);
                        for (int c = 0; c < cn; ++c) s = fma(pk[c * ldA], pl[c * ldA], s);
                        acc[q] += s;
                        tri_next(TPR, nf, k, l);
                    }
                }
                if (!WARM && t < nf) {
                    T s = T(0);
                    for (int c = 0; c < cn; ++c) s = fma(rc[c], Fc[c * ldA + t], s);
                    vacc += s;
                }
            }
            sw_gsync<TPR>();
            if (seg) {
                // the slice's partials: packed lower triangle (entry (l, k),
                // k <= l, at l (l + 1) / 2 + k), then its right-hand side
                // (FP64 form) or its residual at the current value (mixed)
                T *po = reinterpret_cast<T *>(a.seg_out) + r * a.seg_stride;
                int k, l;
                tri_first(t, nf, k, l);
#pragma unroll
                for (int q = 0; q < MAXE; ++q) {
                    if (t + q * TPR < NT) {
                        po[l * (l + 1) / 2 + k] = acc[q];
                        tri_next(TPR, nf, k, l);
                    }
                }
                if (t < nf) po[NT + t] = WARM ? vacc - vcmp : vacc;
                sw_gsync<TPR>();
                continue;
            }
            {
                int k, l;
                tri_first(t, nf, k, l);
#pragma unroll
                for (int q = 0; q < MAXE; ++q) {
                    if (t + q * TPR < NT) {
                        A[l * ldA + k] = acc[q] + (k == l ? lam_n : T(0));
                        tri_next(TPR, nf, k, l);
                    }
                }
            }
            if (!WARM && t < nf) v1[t] = vacc;
            sw_gsync<TPR>();
            ok = sw_cholesky<T, TPR>(A, ldA, nf, colk, diag, t);
            if (!ok && t == 0) atomicAdd(a.notspd, 1);
        }
        if (ok) {
            if (!WARM) {
                sw_trisolve<T, TPR>(A, ldA, nf, diag, v1, v2, u, t);
            } else {
                for (int k = t; k < nf; k += TPR) u[k] = xi ? xi[k] : T(0);
                for (int s = 0; s < a.refine; ++s) {
                    if (s > 0 && sw_correction_small<T, TPR>(colk, u, nf, n, err, t)) break;
                    // res = sum_e f_e (r_e - f_e . u) - lambda n u
                    T rv = T(0), rcmp = T(0);
                    for (int c0 = 0; c0 < n; c0 += CH) {
                        const int cn = min(CH, n - c0);
                        sw_gsync<TPR>();
                        stage_chunk<T, TPR>(a, F, beg + c0, cn, Fc, rc, ldA, t);
                        sw_gsync<TPR>();
                        for (int c = t; c < cn; c += TPR) {
                            T d = T(0);
                            for (int k = 0; k < nf; ++k) d = fma(Fc[c * ldA + k], u[k], d);
                            err[c] = rc[c] - d;
                        }
                        sw_gsync<TPR>();
                        if (t < nf)
                            for (int c = 0; c < cn; ++c) kadd(rv, rcmp, err[c] * Fc[c * ldA + t]);
                    }
                    sw_gsync<TPR>();
                    if (t < nf) v1[t] = (rv - rcmp) - lam_n * u[t];
                    sw_trisolve<T, TPR>(A, ldA, nf, diag, v1, v2, colk, t);
                    for (int k = t; k < nf; k += TPR) u[k] += colk[k];
                    sw_gsync<TPR>();
                }
            }
        } else {
            // empty row: held at zero; system not SPD: row left unchanged
            for (int k = t; k < nf; k += TPR) u[k] = (n > 0 && xi) ? xi[k] : T(0);
        }
        sw_gsync<TPR>();
        for (int k = t; k < a.ld; k += TPR) {
            const T uk = k < nf ? u[k] : T(0);
            const T xk = xi ? xi[k] : T(0);
            xo[k] = uk;
            if (gb) gb[k] = xk - uk;
        }
        sw_gsync<TPR>();
    }
}

template <typename T, int TPR, int MAXE, bool WARM>
als_status sweep_launch(als_ctx *c, const SweepArgs &a) {
    if (a.nrows <= 0) return ALS_OK;
    const int G = 128 / TPR;
    const size_t smem = (size_t)G * group_smem_elems<T>(a.nf) * sizeof(T);
    auto kern = k_sweep_fma<T, TPR, MAXE, WARM>;
    if (raise_smem_limit((const void *)kern, smem) != ALS_OK) return ALS_ECUDA;
    ALS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    int occ = 0;
    ALS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem));
    if (occ < 1) {
        als_set_error("sweep: the row working set does not fit in shared memory");
        return ALS_ENOTSUP;
    }
    // one row group per CTA: the hardware packs as many CTAs per SM as fit
    const int64_t want = (a.nrows + G - 1) / G;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)INT32_MAX));
    cudaStream_t st = a.stream ? a.stream : c->stream;
    kt_begin(c, KT_FMA, st);
    kern<<<grid, 128, smem, st>>>(a);
    kt_end(c, KT_FMA, st);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

}  // namespace

als_status launch_sweep_tc(als_ctx *c, const SweepArgs &a);                // sweep_tc.cu
als_status launch_sweep_dual(als_ctx *c, const SweepArgs &a, int nmax);    // sweep_dual.cu

als_status launch_sweep(als_ctx *c, const SweepArgs &a, bool f64, bool tc) {
    if (tc && !f64) {
        // the lightest rows (a suffix of the degree order) through their
        // n_i x n_i matrix, the rest on the tensor cores
        const int64_t nd = (a.order && !a.seg_out && a.dual_nmax > 0) ? std::min(a.ndual, a.nrows) : 0;
        if (nd <= 0) return launch_sweep_tc(c, a);
        SweepArgs h = a;
        h.nrows = a.nrows - nd;
        als_status s = launch_sweep_tc(c, h);
        if (s != ALS_OK) return s;
        SweepArgs l = a;
        l.order = a.order + h.nrows;
        l.nrows = nd;
        return launch_sweep_dual(c, l, a.dual_nmax);
    }
    if (a.nf <= 32) {
        // degree bin: the heaviest rows (a prefix of the degree order) get a
        // CTA each, the rest a warp each
        const int64_t nbig = a.order ? std::min<int64_t>(a.nbig, a.nrows) : 0;
        als_status s = ALS_OK;
        if (nbig > 0) {
            SweepArgs b = a;
            b.nrows = nbig;
            s = f64 ? sweep_launch<double, 128, 65, false>(c, b) : sweep_launch<float, 128, 65, true>(c, b);
            if (s != ALS_OK) return s;
        }
        SweepArgs r = a;
        r.order = a.order ? a.order + nbig : nullptr;
        r.nrows = a.nrows - nbig;
        return f64 ? sweep_launch<double, 32, 17, false>(c, r) : sweep_launch<float, 32, 17, true>(c, r);
    }
    return f64 ? sweep_launch<double, 128, 65, false>(c, a) : sweep_launch<float, 128, 65, true>(c, a);
}

