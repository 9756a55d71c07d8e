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
