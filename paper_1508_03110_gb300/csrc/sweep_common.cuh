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

__device__ __forceinline__ void ld4f(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

// d[q] <- sum of d[q] over the warp's 32 lanes, for 8 values at once: three
// halving exchanges leave each lane one value summed over 8 lanes, two more
// finish the sum over the warp, and 8 reads gather the totals (17 shuffles
// instead of 40)
__device__ __forceinline__ void warp_allsum8(float (&d)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float e4[4], e2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? d[i] : d[i + 4];
        e4[i] = (b4 ? d[i + 4] : d[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? e4[i] : e4[i + 2];
        e2[i] = (b3 ? e4[i + 2] : e4[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float e1 = (b2 ? e2[1] : e2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? e2[0] : e2[1], 4);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
    // lane l now holds the total of value 4 b4 + 2 b3 + b2
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = __shfl_sync(0xffffffffu, e1, ((q >> 2) & 1) * 16 + ((q >> 1) & 1) * 8 + (q & 1) * 4);
}

// acc += sum over q < 8 with 4 q < cnt of f_q (r_q - f_q . u), f_q the FP32
// factor row of id ix[4 q] and r_q = vx[4 q]: the warp's share of the FP32
// residual of the row's normal equations (lane = 4-wide slot of the row).
// All eight rows are requested before any is used, so one gather latency
// covers them.
__device__ __forceinline__ void resid8(const float *F, int ld, const int32_t *ix, const float *vx, int64_t cnt,
                                       const float (&uu)[4], int lane, bool act, float (&acc)[4],
                                       float (&cmp)[4]) {
    float f[8][4], d[8], r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool in = 4 * q < cnt;
        const int64_t j = in ? ix[4 * q] : 0;
        r[q] = in ? vx[4 * q] : 0.0f;
        if (in && act) ld4f(F + j * ld + 4 * lane, f[q]);
        else f[q][0] = f[q][1] = f[q][2] = f[q][3] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        d[q] = uu[0] * f[q][0];
#pragma unroll
        for (int i = 1; i < 4; ++i) d[q] = fmaf(uu[i], f[q][i], d[q]);
    }
    warp_allsum8(d, lane);
    // the 8 terms in plain FP32, then one compensated add into the running sum
    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float er = 4 * q < cnt ? r[q] - d[q] : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) cs[i] = fmaf(er, f[q][i], cs[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], cs[i]);
}

// Stopping test of the mixed form's refinement u <- u + Ahat^-1 (v - A u)
// for a row with n ratings: true when rho(n) |dx| <= 2^-21 |u|, dx the last
// correction.  A correction leaves at most rho |dx|, rho = |I - Ahat^-1 A|;
// rho(n) = 2^-17 + n 2^-24 bounds it from above -- the BF16 split's own error
// plus FP32 accumulation over n ratings (measured at ML20M size: 2e-6 for
// rows of ~150 ratings, 8e-6 at 9e3, 1.7e-4 at 3.2e4, each under the bound).
// So a row stops once what is left is below ~5e-7 of it, under the mixed
// form's FP32 storage floor; light rows rarely need a second correction.
// One group of TPR threads (a warp, or the CTA when TPR > 32); red: 2 * TPR /
// 32 elements of scratch for the CTA case.
template <typename T, int TPR>
__device__ __forceinline__ bool sw_correction_small(const T *dx, const T *u, int nf, int n, T *red, int t) {
    T d2 = T(0), u2 = T(0);
    for (int k = t; k < nf; k += TPR) {
        d2 = fma(dx[k], dx[k], d2);
        u2 = fma(u[k], u[k], u2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        u2 += __shfl_xor_sync(0xffffffffu, u2, o);
    }
    if constexpr (TPR > 32) {
        if ((t & 31) == 0) {
            red[2 * (t >> 5)] = d2;
            red[2 * (t >> 5) + 1] = u2;
        }
        __syncthreads();
        d2 = T(0);
        u2 = T(0);
#pragma unroll
        for (int w = 0; w < TPR / 32; ++w) {
            d2 += red[2 * w];
            u2 += red[2 * w + 1];
        }
        __syncthreads();
    }
    const T rho = T(0x1p-17) + T(n) * T(0x1p-24);
    return d2 * rho * rho <= T(0x1p-42) * u2;
}

// Packed lower-triangular storage of the symmetric matrices of the
// tensor-core path: entry (i, j), j <= i, at tri_off(i) + j.
__device__ __forceinline__ int tri_off(int i) { return i * (i + 1) / 2; }

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky (panels of 8 columns) for n <= 128, FP32, by
// a CTA of exactly 128 threads, two CTA barriers per panel:
//   1. one thread factors the 8 x 8 diagonal block in registers (no
//      communication inside the block) and publishes L_kk;
//   2. every thread below the block turns its row of A21 into its row of
//      L21 = A21 L_kk^-T by forward substitution against L_kk, stores it and
//      its transpose (PT);
//   3. trailing update A22 -= L21 L21^T by row strips of 16 columns: a warp
//      takes consecutive rows of one strip, so the update of A (row stride
//      ldA odd) is conflict-free and the strip's L21 columns are broadcast
//      loads (a strip's columns end at 16 ceil((n - kb - 8) / 16) + 7 <= 127).
// Measured on a GB300 (100 x 100, 4 CTAs per SM): 39.8k cycles per
// factorisation, against 58.6k for one barrier pair per column.  The thread
// that factors the diagonal blocks is spread over the SM's sub-partitions by
// the caller's `lead`.
// A: lower triangle used; on return its lower triangle holds L (diagonal
// included) and diag[k] = 1 / L[k][k].  work: >= 8*128 + 64 + 1 floats,
// 16-byte aligned.  Returns false (in every thread) on a non-positive pivot.
__device__ __forceinline__ bool chol_blocked128(float *A, int n, float *diag, float *work, int t,
                                                int lead = 0) {
    float *PT = work;              // [8][128] L21, transposed
    float *Lk = work + 8 * 128;    // [8][8] L_kk, Lk[c * 8 + r] = L[r][c]
    int *flag = reinterpret_cast<int *>(Lk + 64);
    if (t == lead) *flag = 0;
    for (int kb = 0; kb < n; kb += 8) {
        const int nb = min(8, n - kb), mp = n - kb;
        if (t == lead) {
            float d[36];  // lower triangle of the block, row-major; unit diagonal past nb
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j)
                    d[i * (i + 1) / 2 + j] = (i < nb && j < nb) ? A[tri_off(kb + i) + kb + j] : (i == j ? 1.0f : 0.0f);
            bool bad = false;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float p = d[c * (c + 1) / 2 + c];
                bad |= !(p > 0.0f);
                const float rd = rsqrtf(p);
                d[c * (c + 1) / 2 + c] = p * rd;
                if (c < nb) diag[kb + c] = rd;
#pragma unroll
                for (int i = c + 1; i < 8; ++i) d[i * (i + 1) / 2 + c] *= rd;
#pragma unroll
                for (int i = c + 1; i < 8; ++i)
#pragma unroll
                    for (int j = c + 1; j <= i; ++j)
                        d[i * (i + 1) / 2 + j] = fmaf(-d[i * (i + 1) / 2 + c], d[j * (j + 1) / 2 + c], d[i * (i + 1) / 2 + j]);
            }
            if (bad) *flag = 1;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) {
                    Lk[j * 8 + i] = d[i * (i + 1) / 2 + j];
                    if (i < nb && j < nb) A[tri_off(kb + i) + kb + j] = d[i * (i + 1) / 2 + j];
                }
        }
        __syncthreads();
        if (*flag) return false;
        float a[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = 0.0f;
        const bool own = t >= nb && t < mp;
        if (own) {
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = (c < nb) ? A[tri_off(kb + t) + kb + c] : 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                a[c] *= diag[kb + c];
#pragma unroll
                for (int cc = c + 1; cc < 8; ++cc) a[cc] = fmaf(-a[c], Lk[c * 8 + cc], a[cc]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < nb) A[tri_off(kb + t) + kb + c] = a[c];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) PT[c * 128 + t] = own ? a[c] : 0.0f;
        __syncthreads();
        const int m = mp - nb;
        if (m > 0) {
            const int G = (m + 15) >> 4;
            const int total = G * m - 8 * G * (G - 1);  // sum over g of (m - 16 g)
            for (int q = t; q < total; q += 128) {
                int g = 0, qq = q;
                while (qq >= m - 16 * g) {
                    qq -= m - 16 * g;
                    ++g;
                }
                const int i = nb + 16 * g + qq, j0 = nb + 16 * g;
                float acc[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float li = PT[c * 128 + i];
                    const float4 *lj = reinterpret_cast<const float4 *>(PT + c * 128 + j0);
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float4 w = lj[v];
                        acc[4 * v] = fmaf(li, w.x, acc[4 * v]);
                        acc[4 * v + 1] = fmaf(li, w.y, acc[4 * v + 1]);
                        acc[4 * v + 2] = fmaf(li, w.z, acc[4 * v + 2]);
                        acc[4 * v + 3] = fmaf(li, w.w, acc[4 * v + 3]);
                    }
                }
                float *ar = A + tri_off(kb + i) + kb + j0;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (j0 + k <= i) ar[k] -= acc[k];
            }
        }
        __syncthreads();
    }
    return true;
}

// L L^T x = b with A from chol_blocked128 after invert_diag_blocks128 (the
// diagonal blocks hold inv(L_kk)): per block of 16, z_blk = inv(L_kk) b_blk
// by 16 threads, then the rows outside the block are updated by all 128
// threads.  Every dot product is a fixed 16-term loop (predicated), so its
// shared-memory loads issue together.  b is consumed; z scratch; x result.
__device__ __forceinline__ void trisolve_inv128(const float *A, int n, float *b, float *z, float *x,
                                                int t) {
    for (int kb = 0; kb < n; kb += 16) {
        const int nb = min(16, n - kb);
        __syncthreads();
        if (t < nb) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                if (c <= t) s0 = fmaf(A[tri_off(kb + t) + kb + c], b[kb + c], s0);
                if (c + 1 <= t) s1 = fmaf(A[tri_off(kb + t) + kb + c + 1], b[kb + c + 1], s1);
            }
            z[kb + t] = s0 + s1;
        }
        __syncthreads();
        for (int i = kb + nb + t; i < n; i += 128) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                if (c < nb) s0 = fmaf(A[tri_off(i) + kb + c], z[kb + c], s0);
                if (c + 1 < nb) s1 = fmaf(A[tri_off(i) + kb + c + 1], z[kb + c + 1], s1);
            }
            b[i] -= s0 + s1;
        }
    }
    const int last = ((n - 1) / 16) * 16;
    for (int kb = last; kb >= 0; kb -= 16) {
        const int nb = min(16, n - kb);
        __syncthreads();
        if (t < nb) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                if (c >= t && c < nb) s0 = fmaf(A[tri_off(kb + c) + kb + t], z[kb + c], s0);
                if (c + 1 >= t && c + 1 < nb) s1 = fmaf(A[tri_off(kb + c + 1) + kb + t], z[kb + c + 1], s1);
            }
            x[kb + t] = s0 + s1;
        }
        __syncthreads();
        for (int i = t; i < kb; i += 128) {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                if (c < nb) s0 = fmaf(A[tri_off(kb + c) + i], x[kb + c], s0);
                if (c + 1 < nb) s1 = fmaf(A[tri_off(kb + c + 1) + i], x[kb + c + 1], s1);
            }
            z[i] -= s0 + s1;
        }
    }
    __syncthreads();
}

// After chol_blocked128: replace every 16 x 16 diagonal block of L by its
// inverse (lower triangular), all blocks at once -- thread t computes column
// t % 16 of block t / 16 by forward substitution (n <= 128: 8 blocks x 16
// columns = 128 threads).  diag holds 1 / L[k][k].  Afterwards the solves of
// trisolve_inv128 apply.
__device__ __forceinline__ void invert_diag_blocks128(float *A, int n, const float *diag, int t) {
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
                    if (c >= j && c < i) s = fmaf(A[tri_off(kb + i) + kb + c], inv[c], s);
                v = -s * diag[kb + i];
            }
        }
        inv[i] = v;
    }
    __syncthreads();
    if (j < nb) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i < nb && i >= j) A[tri_off(kb + i) + kb + j] = inv[i];
    }
    __syncthreads();
}
