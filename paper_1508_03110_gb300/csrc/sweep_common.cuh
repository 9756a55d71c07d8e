// Per-row dense kernels shared by the sweep variants: group barrier, the
// right-looking Cholesky factorisation in shared memory (Golub & Van Loan's
// outer-product form) and the two triangular solves.  A group is TPR
// threads; TPR == 32 groups are one warp, TPR == blockDim groups the CTA.
#pragma once

#include "internal.cuh"

template <int TPR>
__device__ __forceinline__ void sw_gsync() {
    if (TPR == 32) __syncwarp();
    else __syncthreads();
}

__device__ __forceinline__ void sw_ld4(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void sw_ld4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// lower-triangle (a >= b) local enumeration of an m x m trailing block
__device__ __forceinline__ void lt_first(int t, int &a, int &b) {
    a = 0;
    int rem = t;
    while (rem >= a + 1) { rem -= a + 1; ++a; }
    b = rem;
}
__device__ __forceinline__ void lt_next(int step, int &a, int &b) {
    int rem = b + step;
    while (rem >= a + 1) { rem -= a + 1; ++a; }
    b = rem;
}

// In place: A's strict lower triangle becomes L's, diag[k] = L[k][k].
// Returns false (in every thread of the group) if a pivot is not positive.
template <typename T, int TPR>
__device__ bool sw_cholesky(T *A, int ldA, int nf, T *colk, T *diag, int t) {
    for (int k = 0; k < nf; ++k) {
        sw_gsync<TPR>();
        const T akk = A[k * ldA + k];
        if (!(akk > T(0))) {
            sw_gsync<TPR>();
            return false;
        }
        const T dk = sqrt(akk);
        for (int i = k + 1 + t; i < nf; i += TPR) {
            const T v = A[i * ldA + k] / dk;
            A[i * ldA + k] = v;
            colk[i] = v;
        }
        if (t == 0) diag[k] = dk;
        sw_gsync<TPR>();
        const int m = nf - k - 1;
        if (m > 0) {
            int aa, bb;
            lt_first(t, aa, bb);
            while (aa < m) {
                const int i = k + 1 + aa, j = k + 1 + bb;
                A[i * ldA + j] -= colk[i] * colk[j];
                lt_next(TPR, aa, bb);
            }
        }
    }
    sw_gsync<TPR>();
    return true;
}

// Solve L L^T x = b (b in `b`, consumed; z scratch; result in x).
template <typename T, int TPR>
__device__ void sw_trisolve(const T *A, int ldA, int nf, const T *diag, T *b, T *z, T *x, int t) {
    for (int k = 0; k < nf; ++k) {
        sw_gsync<TPR>();
        const T zk = b[k] / diag[k];
        for (int i = k + 1 + t; i < nf; i += TPR) b[i] -= A[i * ldA + k] * zk;
        if (t == 0) z[k] = zk;
    }
    for (int k = nf - 1; k >= 0; --k) {
        sw_gsync<TPR>();
        const T xk = z[k] / diag[k];
        for (int i = t; i < k; i += TPR) z[i] -= A[k * ldA + i] * xk;
        if (t == 0) x[k] = xk;
    }
    sw_gsync<TPR>();
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky (panels of 16 columns) for n <= 128, FP32,
// by a CTA of exactly 128 threads.  Panel: thread t holds row kb+t of the
// panel in registers, one column at a time (pivot, scale, rank-1 update of
// the panel).  Trailing update A22 -= L21 L21^T with 4x4 register blocks
// from the transposed panel PT in shared memory.
// A: lower triangle used; on return its lower triangle holds L (diagonal
// included) and diag[k] = 1 / L[k][k] (reciprocal, for the solves).  work: >= 16*128 + 256 + 2 floats, 16-byte
// aligned.  Returns false (in every thread) on a non-positive pivot.
__device__ __forceinline__ bool chol_blocked128(float *A, int ldA, int n, float *diag, float *work, int t) {
    float *PT = work;              // [16][128]
    float *lcol = work + 16 * 128; // [2][128]
    float *piv = lcol + 256;       // [2]
    for (int kb = 0; kb < n; kb += 16) {
        const int nb = min(16, n - kb), mp = n - kb;
        float row[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) row[c] = (t < mp && c < nb) ? A[(kb + t) * ldA + kb + c] : 0.0f;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            if (c < nb) {
                if (t == c) piv[c & 1] = row[c];
                __syncthreads();
                const float p = piv[c & 1];
                if (!(p > 0.0f)) return false;
                const float rd = rsqrtf(p);   // 1 / L[k][k]
                float l = 0.0f;
                if (t > c && t < mp) {
                    l = row[c] * rd;
                    row[c] = l;
                }
                if (t == c) {
                    row[c] = p * rd;
                    diag[kb + c] = rd;
                }
                lcol[(c & 1) * 128 + t] = l;
                __syncthreads();
                if (t > c && t < mp) {
#pragma unroll
                    for (int cc = c + 1; cc < 16; ++cc) row[cc] -= l * lcol[(c & 1) * 128 + cc];
                }
            }
        }
        if (t < mp) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < nb && c <= t) A[(kb + t) * ldA + kb + c] = row[c];
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) PT[c * 128 + t] = (t < mp && c < nb && t > c) ? row[c] : 0.0f;
        __syncthreads();
        const int m = mp - nb;
        if (m > 0) {
            const int mb = (m + 3) >> 2, nblk = mb * (mb + 1) / 2;
            for (int bidx = t; bidx < nblk; bidx += 128) {
                int bi = (int)((sqrtf(8.0f * (float)bidx + 1.0f) - 1.0f) * 0.5f);
                while ((bi + 1) * (bi + 2) / 2 <= bidx) ++bi;
                while (bi * (bi + 1) / 2 > bidx) --bi;
                const int bj = bidx - bi * (bi + 1) / 2;
                const int pi = nb + 4 * bi, pj = nb + 4 * bj;
                float acc[4][4];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float4 li = *reinterpret_cast<const float4 *>(PT + c * 128 + pi);
                    const float4 lj = *reinterpret_cast<const float4 *>(PT + c * 128 + pj);
                    const float a4[4] = {li.x, li.y, li.z, li.w}, b4[4] = {lj.x, lj.y, lj.z, lj.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a4[p], b4[q], acc[p][q]);
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int i = kb + pi + p;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = kb + pj + q;
                        if (i < n && j <= i) A[i * ldA + j] -= acc[p][q];
                    }
                }
            }
        }
        __syncthreads();
    }
    return true;
}

// L L^T x = b with L from chol_blocked128 (diag = reciprocals), blocks of 16: the diagonal block
// is solved by warp 0 with shuffles, the rows outside it are updated by all
// 128 threads.  b is consumed; z is scratch; x receives the solution (x may
// alias z).
__device__ __forceinline__ void trisolve_blocked128(const float *A, int ldA, int n, const float *diag, float *b,
                                                    float *z, float *x, int t) {
    const int warp = t >> 5, lane = t & 31;
    for (int kb = 0; kb < n; kb += 16) {
        const int nb = min(16, n - kb);
        __syncthreads();
        if (warp == 0) {
            float bv = lane < nb ? b[kb + lane] : 0.0f;
            for (int c = 0; c < nb; ++c) {
                const float zc = __shfl_sync(0xffffffffu, bv, c) * diag[kb + c];
                if (lane == c) z[kb + c] = zc;
                if (lane > c && lane < nb) bv -= A[(kb + lane) * ldA + kb + c] * zc;
            }
        }
        __syncthreads();
        for (int i = kb + nb + t; i < n; i += 128) {
            float s = 0.0f;
            for (int c = 0; c < nb; ++c) s = fmaf(A[i * ldA + kb + c], z[kb + c], s);
            b[i] -= s;
        }
    }
    const int last = ((n - 1) / 16) * 16;
    for (int kb = last; kb >= 0; kb -= 16) {
        const int nb = min(16, n - kb);
        __syncthreads();
        if (warp == 0) {
            float zv = lane < nb ? z[kb + lane] : 0.0f;
            for (int c = nb - 1; c >= 0; --c) {
                const float xc = __shfl_sync(0xffffffffu, zv, c) * diag[kb + c];
                if (lane == c) x[kb + c] = xc;
                if (lane < c) zv -= A[(kb + c) * ldA + kb + lane] * xc;
            }
        }
        __syncthreads();
        for (int i = t; i < kb; i += 128) {
            float s = 0.0f;
            for (int c = 0; c < nb; ++c) s = fmaf(A[(kb + c) * ldA + i], x[kb + c], s);
            z[i] -= s;
        }
    }
    __syncthreads();
}
