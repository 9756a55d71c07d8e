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

// ---------------------------------------------------------------------------
// Blocked Cholesky with inverted diagonal blocks, n <= 128, FP32, exactly 128
// threads.  Per panel of 16 columns:
//   1. warp 0 factors the 16 x 16 diagonal block warp-synchronously (lane i
//      holds row i; pivots and column entries move by shuffles), then each
//      lane j computes column j of the block's inverse, which overwrites the
//      block (lower triangle) -- the solves only need the inverse;
//   2. every row below the block: L21 row = A21 row * inv(L_kk)^T (a 16-wide
//      matvec per thread, no dependency chain), stored in A and transposed
//      into PT;
//   3. trailing update A22 -= L21 L21^T with 4 x 4 register blocks.
// Three CTA barriers per panel.  On return: off-diagonal blocks of A hold L,
// diagonal blocks hold inv(L_kk), diag[k] = 1 / L[k][k].  work: >= 16*128 + 4
// floats, 16-byte aligned.  Returns false (in every thread) on a
// non-positive pivot.
__device__ __forceinline__ bool chol_inv128(float *A, int ldA, int n, float *diag, float *work, int t) {
    float *PT = work;                                     // [16][128]
    int *flag = reinterpret_cast<int *>(work + 16 * 128);  // non-SPD flag
    const int warp = t >> 5, lane = t & 31;
    if (t == 0) *flag = 0;
    for (int kb = 0; kb < n; kb += 16) {
        const int nb = min(16, n - kb), mp = n - kb;
        __syncthreads();
        if (warp == 0) {
            float row[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) row[c] = (lane < nb && c < nb) ? A[(kb + lane) * ldA + kb + c] : 0.0f;
            bool bad = false;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                if (c < nb) {
                    const float p = __shfl_sync(0xffffffffu, row[c], c);
                    if (!(p > 0.0f)) bad = true;
                    const float rd = rsqrtf(p);
                    const float l = (lane > c) ? row[c] * rd : 0.0f;
                    if (lane > c) row[c] = l;
                    if (lane == c) {
                        row[c] = p * rd;
                        diag[kb + c] = rd;
                    }
#pragma unroll
                    for (int cc = c + 1; cc < 16; ++cc) {
                        const float lcc = __shfl_sync(0xffffffffu, l, cc);
                        if (lane >= cc) row[cc] -= l * lcc;
                    }
                }
            }
            if (bad && lane == 0) *flag = 1;
            // L_kk into shared memory, then column `lane` of its inverse
            if (lane < nb) {
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c <= lane) A[(kb + lane) * ldA + kb + c] = row[c];
            }
            __syncwarp();
            float inv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float v = 0.0f;
                if (i < nb && i >= lane) {
                    if (i == lane) {
                        v = diag[kb + i];
                    } else {
                        float s = 0.0f;
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (c >= lane && c < i) s = fmaf(A[(kb + i) * ldA + kb + c], inv[c], s);
                        v = -s * diag[kb + i];
                    }
                }
                inv[i] = v;
            }
            __syncwarp();
            if (lane < nb) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i < nb && i >= lane) A[(kb + i) * ldA + kb + lane] = inv[i];
            }
        }
        __syncthreads();
        if (*flag) return false;
        // rows below the diagonal block: L21 = A21 inv(L_kk)^T
        {
            float l[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) l[c] = 0.0f;
            if (t >= nb && t < mp) {
                float a21[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) a21[c] = (c < nb) ? A[(kb + t) * ldA + kb + c] : 0.0f;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (c < nb) {
                        float s = 0.0f;
#pragma unroll
                        for (int cc = 0; cc <= c; ++cc) s = fmaf(a21[cc], A[(kb + c) * ldA + kb + cc], s);
                        l[c] = s;
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c < nb) A[(kb + t) * ldA + kb + c] = l[c];
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) PT[c * 128 + t] = l[c];
        }
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
    }
    __syncthreads();
    return true;
}

// L L^T x = b with A from chol_inv128 (inverted diagonal blocks): per block
// a 16-wide triangular matvec with the inverse, then the update of the rows
// outside the block, by all 128 threads.  b is consumed; z scratch; x result.
__device__ __forceinline__ void trisolve_inv128(const float *A, int ldA, int n, float *b, float *z, float *x,
                                                int t) {
    for (int kb = 0; kb < n; kb += 16) {
        const int nb = min(16, n - kb);
        __syncthreads();
        if (t < nb) {
            float s = 0.0f;
            for (int c = 0; c <= t; ++c) s = fmaf(A[(kb + t) * ldA + kb + c], b[kb + c], s);
            z[kb + t] = s;
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
        if (t < nb) {
            float s = 0.0f;
            for (int c = t; c < nb; ++c) s = fmaf(A[(kb + c) * ldA + kb + t], z[kb + c], s);
            x[kb + t] = s;
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

// After chol_blocked128: replace every 16 x 16 diagonal block of L by its
// inverse (lower triangular), all blocks at once -- thread t computes column
// t % 16 of block t / 16 by forward substitution (n <= 128: 8 blocks x 16
// columns = 128 threads).  diag holds 1 / L[k][k].  Afterwards the solves of
// trisolve_inv128 apply.
__device__ __forceinline__ void invert_diag_blocks128(float *A, int ldA, int n, const float *diag, int t) {
    const int b = t >> 4, j = t & 15, kb = 16 * b;
    const int nb = kb < n ? min(16, n - kb) : 0;
    float inv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float v = 0.0f;
        if (j < nb && i < nb && i >= j) {
            if (i == j) {
                v = diag[kb + i];
            } else {
                float s = 0.0f;
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c >= j && c < i) s = fmaf(A[(kb + i) * ldA + kb + c], inv[c], s);
                v = -s * diag[kb + i];
            }
        }
        inv[i] = v;
    }
    __syncthreads();
    if (j < nb) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i < nb && i >= j) A[(kb + i) * ldA + kb + j] = inv[i];
    }
    __syncthreads();
}
