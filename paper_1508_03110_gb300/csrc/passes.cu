// Rating passes, deterministic reductions and NCG vector kernels.
//
//  * k_grad: gradient of Eq. (1) for one side (§V-C "Gradient Evaluation"):
//      g_i = 2 lambda n_i x_i - 2 sum_{e in row i} (r_e - x_i . f_e) f_e,
//    with the fixed side f, plus per-row FP64 terms |g_i|^2,
//    gbar_i . g_i and gbar_i . (g_i - gprev_i) for Eq. (8).
//  * k_lscoef: the five coefficients of Q(alpha) = f(x + alpha p) (§V-C
//    "Line Search & Loss Function Evaluation"), one pass over the by-user
//    ratings with four dot products per rating; with p = 0 it is the loss.
//  * k_reduce: fixed-order two-level FP64 sums of the per-row terms, and the
//    scalar step that follows them (Algorithm 3 on Q, beta-bar of Eq. 8).
//  * vector kernels: x <- x + alpha p (or the ALS point on a fallback),
//    p <- -gbar + beta p, conversions.
//
// Layout: a row of n_f values is stored in ld = round_up(n_f, 4) slots (the
// padding is kept at zero).  A group of LPR lanes owns one row, each lane one
// 4-wide slot, so a rating costs one 16 B (float) / 32 B (double) load per
// lane and a log2(LPR)-step shuffle reduction for each dot product.  Rows of
// at least ALS_HEAVY_MIN ratings are processed by a whole CTA (contiguous
// segments per group, combined in a fixed order).  No floating-point atomics
// anywhere: every per-row term lands in its own slot and is summed in a fixed
// order, so results are bit-reproducible.
#include <cmath>

#include "internal.cuh"
#include "sweep_common.cuh"

namespace {

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st4<float>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

template <typename T>
__device__ __forceinline__ void zero4(T (&v)[4]) { v[0] = v[1] = v[2] = v[3] = T(0); }

template <typename T>
__device__ __forceinline__ T dot4(const T (&a)[4], const T (&b)[4]) {
    T s = a[0] * b[0];
    s = fma(a[1], b[1], s);
    s = fma(a[2], b[2], s);
    s = fma(a[3], b[3], s);
    return s;
}

template <int LPR, typename V>
__device__ __forceinline__ V gsum(V x, unsigned mask) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

template <int LPR>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if constexpr (LPR == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << LPR) - 1u) << ((lane / LPR) * LPR);
    }
}

// Totals over the group of each of N FP64 values, in every lane of the group.
// A whole warp halves the values at each of its first log2(P) exchanges (P =
// N rounded up to 4 or 8), so that each lane then carries one value summed
// over 2, 4 or 8 lanes; the remaining exchanges finish it and P reads gather
// the totals (6 or 9 additions in all instead of 5 N, on the slow FP64 pipe).
// Smaller groups add each value over their own exchanges.
template <int LPR, int N>
__device__ __forceinline__ void tsum_n(double (&t)[N], unsigned mask, int lane) {
    if constexpr (LPR == 32 && N >= 3 && N <= 8) {
        constexpr int P = N <= 4 ? 4 : 8;
        double d[P];
#pragma unroll
        for (int i = 0; i < P; ++i) d[i] = i < N ? t[i] : 0.0;
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        double e[P / 2];
#pragma unroll
        for (int i = 0; i < P / 2; ++i)
            e[i] = (b4 ? d[i + P / 2] : d[i]) + __shfl_xor_sync(mask, b4 ? d[i] : d[i + P / 2], 16);
        double f[P / 4];
#pragma unroll
        for (int i = 0; i < P / 4; ++i)
            f[i] = (b3 ? e[i + P / 4] : e[i]) + __shfl_xor_sync(mask, b3 ? e[i] : e[i + P / 4], 8);
        double v;
        if constexpr (P == 8) v = (b2 ? f[1] : f[0]) + __shfl_xor_sync(mask, b2 ? f[0] : f[1], 4);
        else v = f[0] + __shfl_xor_sync(mask, f[0], 4);
        v += __shfl_xor_sync(mask, v, 2);
        v += __shfl_xor_sync(mask, v, 1);
        // lane l now holds the total of value 4 b4 + 2 b3 + b2 (P = 8) or
        // 2 b4 + b3 (P = 4)
#pragma unroll
        for (int q = 0; q < N; ++q)
            t[q] = __shfl_sync(mask, v,
                               P == 8 ? ((q >> 2) & 1) * 16 + ((q >> 1) & 1) * 8 + (q & 1) * 4
                                      : ((q >> 1) & 1) * 16 + (q & 1) * 8);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) t[q] = gsum<LPR>(t[q], mask);
    }
}

// ---------------------------------------------------------------------------
// gradient
// ---------------------------------------------------------------------------
// the per-row FP64 terms of Eq. (8) from the row's gradient g (this lane's
// 4-wide slot): |g|^2, gbar . g, gbar . (g - gprev) and, with Ps,
// p . (g - gprev), summed over the group and written to rowterm
template <typename T, int LPR>
__device__ __forceinline__ void grad_terms(const PassArgs &a, int64_t row, int gl, int lane, unsigned mask,
                                           const T (&g)[4]) {
    const int nslot = a.ld / 4;
    const bool act = gl < nslot;
    double tg = 0, tgb = 0, tgd = 0, tpd = 0;
    if (act) {
#pragma unroll
        for (int i = 0; i < 4; ++i) tg += (double)g[i] * (double)g[i];
        if (a.Gbar) {
            // Gbar == Gout: plain NCG, gbar is this gradient
            T gb[4];
            if (a.Gbar == a.Gout) {
#pragma unroll
                for (int i = 0; i < 4; ++i) gb[i] = g[i];
            } else {
                ld4(reinterpret_cast<const T *>(a.Gbar) + row * a.ld + 4 * gl, gb);
            }
            T gp[4];
            if (a.Gprev) ld4(reinterpret_cast<const T *>(a.Gprev) + row * a.ld + 4 * gl, gp);
            else zero4(gp);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                tgb += (double)gb[i] * (double)g[i];
                tgd += (double)gb[i] * ((double)g[i] - (double)gp[i]);
            }
            if (a.Ps) {
                // p_k . (g_{k+1} - g_k): the Hestenes-Stiefel denominator
                T pk[4];
                ld4(reinterpret_cast<const T *>(a.Ps) + row * a.ld + 4 * gl, pk);
#pragma unroll
                for (int i = 0; i < 4; ++i) tpd += (double)pk[i] * ((double)g[i] - (double)gp[i]);
            }
        }
    }
    double tt[4] = {tg, tgb, tgd, tpd};
    tsum_n<LPR, 4>(tt, mask, lane);
    if (gl == 0) {
        const int64_t o = a.rowoff + row;
        a.rowterm[o] = tt[0];
        a.rowterm[a.stride + o] = tt[1];
        a.rowterm[2 * a.stride + o] = tt[2];
        if (a.Ps) a.rowterm[3 * a.stride + o] = tt[3];
    }
}

// g_i = 2 lambda n_i x_i - 2 acc, stored, then its row terms
template <typename T, int LPR>
__device__ __forceinline__ void grad_finish(const PassArgs &a, int64_t row, int64_t n, int gl, int lane,
                                            unsigned mask, const T (&x)[4], const T (&acc)[4]) {
    const T l2 = (T)(2.0 * a.lambda * (double)n);
    T g[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) g[i] = l2 * x[i] - T(2) * acc[i];
    if (gl < a.ld / 4) st4(reinterpret_cast<T *>(a.Gout) + row * a.ld + 4 * gl, g);
    grad_terms<T, LPR>(a, row, gl, lane, mask, g);
}

// the row terms of gradient rows already in Gout (the mixed tensor-core
// sweep writes a side's gradient rows while it solves them: its first
// residual is that gradient); rows 0 .. nrows - 1 of the side
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_grad_terms(PassArgs a) {
    const int lane = threadIdx.x & 31, gl = lane % LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / LPR;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR; row < a.nrows; row += ngroups) {
        T g[4];
        if (gl < a.ld / 4) ld4(reinterpret_cast<const T *>(a.Gout) + row * a.ld + 4 * gl, g);
        else zero4(g);
        grad_terms<T, LPR>(a, row, gl, lane, mask, g);
    }
}

// d[q] <- sum of d[q] over the LPR-lane group, for 4 values at once; for a
// whole warp (LPR == 32) two halving exchanges and three more leave each lane
// one total and 4 reads gather them (10 shuffles instead of 20)
template <int LPR, typename T>
__device__ __forceinline__ void gsum4(T (&d)[4], unsigned mask, int lane) {
    if constexpr (LPR == 32) {
        const bool b4 = lane & 16, b3 = lane & 8;
        T e2[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) e2[i] = (b4 ? d[i + 2] : d[i]) + __shfl_xor_sync(mask, b4 ? d[i] : d[i + 2], 16);
        T e1 = (b3 ? e2[1] : e2[0]) + __shfl_xor_sync(mask, b3 ? e2[0] : e2[1], 8);
        e1 += __shfl_xor_sync(mask, e1, 4);
        e1 += __shfl_xor_sync(mask, e1, 2);
        e1 += __shfl_xor_sync(mask, e1, 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = __shfl_sync(mask, e1, ((q >> 1) & 1) * 16 + (q & 1) * 8);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = gsum<LPR>(d[q], mask);
    }
}

// acc (compensated in FP32) += sum over the 4 ratings e .. e + 3 of
// f_e (r_e - x . f_e), f_e the gathered rows; all 4 rows are requested
// before any is used
template <typename T, int LPR>
__device__ __forceinline__ void grad4(const PassArgs &a, const T *Xo, const T (&x)[4], int64_t e, int gl, int lane,
                                      unsigned mask, bool act, T (&acc)[4], T (&cmp)[4]) {
    T f[4][4], d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t j = a.idx[e + q];
        if (act) ld4(Xo + j * a.ld + 4 * gl, f[q]);
        else zero4(f[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = dot4(x, f[q]);
    gsum4<LPR>(d, mask, lane);
    T cs[4];
    zero4(cs);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T er = (T)a.val[e + q] - d[q];
#pragma unroll
        for (int i = 0; i < 4; ++i) cs[i] = fma(er, f[q][i], cs[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], cs[i]);
}

template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_grad(PassArgs a) {
    const int lane = threadIdx.x & 31, gl = lane % LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const int nslot = a.ld / 4;
    const bool act = gl < nslot;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / LPR;
    const T *Xs = reinterpret_cast<const T *>(a.Xs);
    const T *Xo = reinterpret_cast<const T *>(a.Xo);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR; r < a.nrows; r += ngroups) {
        const int64_t row = a.order[a.row_begin + r];
        const int64_t beg = a.ptr[row], n = a.ptr[row + 1] - beg;
        T x[4], acc[4], cmp[4];
        zero4(acc);
        zero4(cmp);
        if (act) ld4(Xs + row * a.ld + 4 * gl, x); else zero4(x);
        int64_t e = 0;
        for (; e + 4 <= n; e += 4) grad4<T, LPR>(a, Xo, x, beg + e, gl, lane, mask, act, acc, cmp);
        for (; e < n; ++e) {
            const int64_t j0 = a.idx[beg + e];
            T f0[4];
            if (act) ld4(Xo + j0 * a.ld + 4 * gl, f0); else zero4(f0);
            const T d0 = gsum<LPR>(dot4(x, f0), mask);
            const T e0 = (T)a.val[beg + e] - d0;
#pragma unroll
            for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], e0 * f0[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] -= cmp[i];
        grad_finish<T, LPR>(a, row, n, gl, lane, mask, x, acc);
    }
}

// one CTA (256 threads) per heavy row; groups take contiguous segments
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_grad_heavy(PassArgs a) {
    constexpr int NG = 256 / LPR;
    __shared__ T part[NG][LPR][4];
    const int lane = threadIdx.x & 31, gl = lane % LPR, gi = threadIdx.x / LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const bool act = gl < a.ld / 4;
    const T *Xs = reinterpret_cast<const T *>(a.Xs);
    const T *Xo = reinterpret_cast<const T *>(a.Xo);
    for (int64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {
        const int64_t row = a.order[a.row_begin + r];
        const int64_t beg = a.ptr[row], n = a.ptr[row + 1] - beg;
        const int64_t seg = (n + NG - 1) / NG;
        const int64_t e0 = beg + gi * seg, e1 = min(beg + n, e0 + seg);
        T x[4], acc[4], cmp[4];
        zero4(acc);
        zero4(cmp);
        if (act) ld4(Xs + row * a.ld + 4 * gl, x); else zero4(x);
        int64_t e = e0;
        for (; e + 4 <= e1; e += 4) grad4<T, LPR>(a, Xo, x, e, gl, lane, mask, act, acc, cmp);
        for (; e < e1; ++e) {
            const int64_t j = a.idx[e];
            T f[4];
            if (act) ld4(Xo + j * a.ld + 4 * gl, f); else zero4(f);
            const T d = gsum<LPR>(dot4(x, f), mask);
            const T er = (T)a.val[e] - d;
#pragma unroll
            for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], er * f[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) part[gi][gl][i] = acc[i] - cmp[i];
        __syncthreads();
        if (gi == 0) {
            T tot[4];
            zero4(tot);
            for (int q = 0; q < NG; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) tot[i] += part[q][gl][i];
            grad_finish<T, LPR>(a, row, n, gl, lane, mask, x, tot);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// line-search coefficients (and the loss when Ps == Po == null)
// ---------------------------------------------------------------------------
// One rating's four dot products are reduced over the group; lane `owner`
// parks them (in the storage precision) and every LPR ratings the whole group
// turns its parked values into FP64 terms at once.  A warp-wide FP64
// instruction costs the FP64 pipe the same whether 1 or 32 lanes are active,
// so this keeps the FP64 instruction count at ~12 per LPR ratings.
template <typename T>
struct LsPending {
    T r, d0, d1, d2, d3;
    bool have;
};

// A lane's sums of the five rating terms of Q.  FP64 form: FP64 terms, FP64
// sums.  Mixed form, without the FP64 pipe (1/64 of the FP32 rate here):
// e0 = r - d0 and a = d1 + d2 are formed exactly as float pairs by Knuth's
// two-sum, each product as its exact leading part (x y = p + e, e = fma(x, y,
// -p)) plus the cross terms of the pairs' low parts, and the five sums are
// kept as float pairs (hi, lo) by two-sum, which carries the rounding error of
// every addition (Knuth, TAOCP vol. 2, 4.2.2; Dekker 1971).  Every term then
// matches the one formed in FP64 from the same FP32 dot products to about
// 2^-47 of itself and a lane's sum keeps FP64-like accuracy; the FP64 pipe
// adds hi and lo once per row instead of taking about 17 instructions per 32
// ratings.
template <typename T>
struct LsAcc {
    double t[5];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 5; ++q) t[q] = 0.0;
    }
    template <bool HAS_P>
    __device__ __forceinline__ void add(const LsPending<T> &p) {
        const double e0 = (double)p.r - (double)p.d0;
        if (HAS_P) {
            const double aa = (double)p.d1 + (double)p.d2, b = (double)p.d3;
            t[0] += e0 * e0;
            t[1] += -2.0 * e0 * aa;
            t[2] += aa * aa - 2.0 * e0 * b;
            t[3] += 2.0 * aa * b;
            t[4] += b * b;
        } else {
            t[0] += e0 * e0;
        }
    }
    __device__ __forceinline__ void out(double (&o)[5]) const {
#pragma unroll
        for (int q = 0; q < 5; ++q) o[q] = t[q];
    }
};

// s + e = a + b exactly (two-sum); the _rn intrinsics are never contracted
// into an FMA, which would break the exact splits
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

template <>
struct LsAcc<float> {
    float h[5], l[5];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 5; ++q) h[q] = l[q] = 0.0f;
    }
    // (h, l) += (xh + xl)(yh + yl), dropping xl yl (2^-48 of the product)
    __device__ __forceinline__ void prod(int q, float xh, float xl, float yh, float yl) {
        const float p = __fmul_rn(xh, yh), e = fmaf(xh, yh, -p);
        const float c = fmaf(xh, yl, __fmul_rn(xl, yh));
        float s, err;
        two_sum(h[q], p, s, err);
        h[q] = s;
        l[q] = __fadd_rn(l[q], __fadd_rn(err, __fadd_rn(e, c)));
    }
    template <bool HAS_P>
    __device__ __forceinline__ void add(const LsPending<float> &p) {
        float e0h, e0l;
        two_sum(p.r, -p.d0, e0h, e0l);
        prod(0, e0h, e0l, e0h, e0l);
        if (HAS_P) {
            float ah, al;
            two_sum(p.d1, p.d2, ah, al);
            const float b = p.d3;
            prod(1, -2.0f * e0h, -2.0f * e0l, ah, al);
            prod(2, ah, al, ah, al);
            prod(2, -2.0f * e0h, -2.0f * e0l, b, 0.0f);
            prod(3, 2.0f * ah, 2.0f * al, b, 0.0f);
            prod(4, b, 0.0f, b, 0.0f);
        }
    }
    __device__ __forceinline__ void out(double (&o)[5]) const {
#pragma unroll
        for (int q = 0; q < 5; ++q) o[q] = (double)h[q] + (double)l[q];
    }
};

template <typename T, bool HAS_P>
__device__ __forceinline__ void ls_flush(LsPending<T> &q, LsAcc<T> &t) {
    if (!q.have) return;
    t.template add<HAS_P>(q);
    q.have = false;
}

template <typename T, int LPR, bool HAS_P>
__device__ __forceinline__ void lscoef_rating(const T (&xu)[4], const T (&pu)[4], const T *Xo,
                                              const T *Po, int64_t j, float r, int ld, int gl,
                                              bool act, unsigned mask, int &owner, LsPending<T> &q,
                                              LsAcc<T> &t) {
    T xm[4], pm[4];
    if (act) {
        ld4(Xo + j * ld + 4 * gl, xm);
        if (HAS_P) ld4(Po + j * ld + 4 * gl, pm); else zero4(pm);
    } else {
        zero4(xm); zero4(pm);
    }
    const T d0 = gsum<LPR>(dot4(xu, xm), mask);
    T d1 = T(0), d2 = T(0), d3 = T(0);
    if (HAS_P) {
        d1 = gsum<LPR>(dot4(xu, pm), mask);
        d2 = gsum<LPR>(dot4(pu, xm), mask);
        d3 = gsum<LPR>(dot4(pu, pm), mask);
    }
    if (owner == gl) {
        q.r = (T)r; q.d0 = d0; q.d1 = d1; q.d2 = d2; q.d3 = d3;
        q.have = true;
    }
    if (++owner == LPR) {
        owner = 0;
        ls_flush<T, HAS_P>(q, t);
    }
}

// ratings [e, e1) of one row.  Mixed form with whole-warp groups: two
// ratings per step, their four rows requested together and their eight dot
// products all-reduced at once (17 shuffles instead of 40); otherwise one
// rating at a time.
template <typename T, int LPR, bool HAS_P>
__device__ __forceinline__ void lscoef_range(const PassArgs &a, const T (&xu)[4], const T (&pu)[4], const T *Xo,
                                             const T *Po, int64_t e, int64_t e1, int gl, int lane, bool act,
                                             unsigned mask, int &owner, LsPending<T> &q, LsAcc<T> &t) {
    if constexpr (sizeof(T) == 4 && LPR == 32 && HAS_P) {
        for (; e + 2 <= e1; e += 2) {
            const int64_t j0 = a.idx[e], j1 = a.idx[e + 1];
            const float r0 = a.val[e], r1 = a.val[e + 1];
            float xm0[4], pm0[4], xm1[4], pm1[4];
            if (act) {
                ld4(Xo + j0 * a.ld + 4 * gl, xm0);
                ld4(Po + j0 * a.ld + 4 * gl, pm0);
                ld4(Xo + j1 * a.ld + 4 * gl, xm1);
                ld4(Po + j1 * a.ld + 4 * gl, pm1);
            } else {
                zero4(xm0); zero4(pm0); zero4(xm1); zero4(pm1);
            }
            float d[8] = {dot4(xu, xm0), dot4(xu, pm0), dot4(pu, xm0), dot4(pu, pm0),
                          dot4(xu, xm1), dot4(xu, pm1), dot4(pu, xm1), dot4(pu, pm1)};
            warp_allsum8(d, lane);
            if (owner == gl) {
                q.r = r0; q.d0 = d[0]; q.d1 = d[1]; q.d2 = d[2]; q.d3 = d[3];
                q.have = true;
            }
            if (owner + 1 == gl) {
                q.r = r1; q.d0 = d[4]; q.d1 = d[5]; q.d2 = d[6]; q.d3 = d[7];
                q.have = true;
            }
            owner += 2;
            if (owner == LPR) {
                owner = 0;
                ls_flush<T, HAS_P>(q, t);
            }
        }
    }
    for (; e < e1; ++e)
        lscoef_rating<T, LPR, HAS_P>(xu, pu, Xo, Po, a.idx[e], a.val[e], a.ld, gl, act, mask, owner, q, t);
}

// t: this lane's shares of the five rating terms; the row's regulariser
// lambda n_i |x + alpha p|^2 adds this lane's slots of x.x, 2 x.p and p.p
// to them, and one reduction over the group gives the row's five terms
template <typename T, int LPR, bool HAS_P>
__device__ __forceinline__ void lscoef_finish(const PassArgs &a, int64_t row, int64_t n, int gl, int lane,
                                              unsigned mask, const T (&xu)[4], const T (&pu)[4],
                                              double (&t)[5]) {
    double xx = 0, xp = 0, pp = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        xx += (double)xu[i] * (double)xu[i];
        if (HAS_P) {
            xp += (double)xu[i] * (double)pu[i];
            pp += (double)pu[i] * (double)pu[i];
        }
    }
    const double ln = a.lambda * (double)n;
    t[0] += ln * xx;
    if (HAS_P) {
        t[1] += ln * 2.0 * xp;
        t[2] += ln * pp;
        tsum_n<LPR, 5>(t, mask, lane);
    } else {
        t[0] = gsum<LPR>(t[0], mask);
    }
    if (gl == 0) {
        const int64_t o = a.rowoff + row;
        const int nt = HAS_P ? 5 : 1;
        for (int q = 0; q < nt; ++q) a.rowterm[q * a.stride + o] = t[q];
    }
}

template <typename T, int LPR, bool HAS_P>
__global__ void __launch_bounds__(256) k_lscoef(PassArgs a) {
    const int lane = threadIdx.x & 31, gl = lane % LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const bool act = gl < a.ld / 4;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / LPR;
    const T *Xs = reinterpret_cast<const T *>(a.Xs), *Ps = reinterpret_cast<const T *>(a.Ps);
    const T *Xo = reinterpret_cast<const T *>(a.Xo), *Po = reinterpret_cast<const T *>(a.Po);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR; r < a.nrows; r += ngroups) {
        const int64_t row = a.order[a.row_begin + r];
        const int64_t beg = a.ptr[row], n = a.ptr[row + 1] - beg;
        T xu[4], pu[4];
        if (act) {
            ld4(Xs + row * a.ld + 4 * gl, xu);
            if (HAS_P) ld4(Ps + row * a.ld + 4 * gl, pu); else zero4(pu);
        } else {
            zero4(xu); zero4(pu);
        }
        LsAcc<T> acc;
        acc.init();
        int owner = 0;
        LsPending<T> q;
        q.have = false;
        lscoef_range<T, LPR, HAS_P>(a, xu, pu, Xo, Po, beg, beg + n, gl, lane, act, mask, owner, q, acc);
        ls_flush<T, HAS_P>(q, acc);
        double t[5];
        acc.out(t);
        lscoef_finish<T, LPR, HAS_P>(a, row, n, gl, lane, mask, xu, pu, t);
    }
}

template <typename T, int LPR, bool HAS_P>
__global__ void __launch_bounds__(256) k_lscoef_heavy(PassArgs a) {
    constexpr int NG = 256 / LPR;
    __shared__ double part[NG][5];
    const int lane = threadIdx.x & 31, gl = lane % LPR, gi = threadIdx.x / LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const bool act = gl < a.ld / 4;
    const T *Xs = reinterpret_cast<const T *>(a.Xs), *Ps = reinterpret_cast<const T *>(a.Ps);
    const T *Xo = reinterpret_cast<const T *>(a.Xo), *Po = reinterpret_cast<const T *>(a.Po);
    for (int64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {
        const int64_t row = a.order[a.row_begin + r];
        const int64_t beg = a.ptr[row], n = a.ptr[row + 1] - beg;
        const int64_t seg = (n + NG - 1) / NG;
        const int64_t e0 = beg + gi * seg, e1 = min(beg + n, e0 + seg);
        T xu[4], pu[4];
        if (act) {
            ld4(Xs + row * a.ld + 4 * gl, xu);
            if (HAS_P) ld4(Ps + row * a.ld + 4 * gl, pu); else zero4(pu);
        } else {
            zero4(xu); zero4(pu);
        }
        LsAcc<T> acc;
        acc.init();
        int owner = 0;
        LsPending<T> q;
        q.have = false;
        lscoef_range<T, LPR, HAS_P>(a, xu, pu, Xo, Po, e0, e1, gl, lane, act, mask, owner, q, acc);
        ls_flush<T, HAS_P>(q, acc);
        double t[5];
        acc.out(t);
        if constexpr (HAS_P) tsum_n<LPR, 5>(t, mask, lane);
        else t[0] = gsum<LPR>(t[0], mask);
        if (gl == 0)
            for (int q = 0; q < 5; ++q) part[gi][q] = t[q];
        __syncthreads();
        if (gi == 0) {
            // the groups' sums in group order, as lane 0's share
            double tot[5] = {0, 0, 0, 0, 0};
            if (gl == 0)
                for (int q = 0; q < NG; ++q)
                    for (int s = 0; s < 5; ++s) tot[s] += part[q][s];
            lscoef_finish<T, LPR, HAS_P>(a, row, n, gl, lane, mask, xu, pu, tot);
        }
        __syncthreads();
    }
}

// rows whose ratings are handled from the other side: only the lambda terms
template <typename T, int LPR, bool HAS_P>
__global__ void __launch_bounds__(256) k_lscoef_reg(PassArgs a) {
    const int lane = threadIdx.x & 31, gl = lane % LPR;
    const unsigned mask = group_mask<LPR>(lane);
    const bool act = gl < a.ld / 4;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / LPR;
    const T *Xs = reinterpret_cast<const T *>(a.Xs), *Ps = reinterpret_cast<const T *>(a.Ps);
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR; row < a.nrows; row += ngroups) {
        const int64_t n = a.ptr[row + 1] - a.ptr[row];
        T xu[4], pu[4];
        if (act) {
            ld4(Xs + row * a.ld + 4 * gl, xu);
            if (HAS_P) ld4(Ps + row * a.ld + 4 * gl, pu); else zero4(pu);
        } else {
            zero4(xu); zero4(pu);
        }
        double t[5] = {0, 0, 0, 0, 0};
        lscoef_finish<T, LPR, HAS_P>(a, row, n, gl, lane, mask, xu, pu, t);
        if (HAS_P && gl == 0) {
            a.rowterm[3 * a.stride + a.rowoff + row] = 0.0;
            a.rowterm[4 * a.stride + a.rowoff + row] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// fixed-order reduction + scalar post-operations
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

// Q(alpha) - Q(0), Horner form, no contraction
__device__ double q_delta(const double *c, double al) {
    double t = dadd(c[3], dmul(al, c[4]));
    t = dadd(c[2], dmul(al, t));
    t = dadd(c[1], dmul(al, t));
    return dmul(al, t);
}

// Real roots of a x^3 + b x^2 + c x + d = 0 (Cardano / trigonometric form,
// each polished by two Newton steps).  Returns the number of roots.
__device__ int cubic_roots(double a, double b, double c, double d, double *r) {
    int n = 0;
    if (fabs(a) <= 1e-300) {
        if (fabs(b) <= 1e-300) {
            if (fabs(c) > 1e-300) r[n++] = -d / c;
            return n;
        }
        const double disc = c * c - 4 * b * d;
        if (disc >= 0) {
            const double s = sqrt(disc);
            const double q = -0.5 * (c + (c >= 0 ? s : -s));
            r[n++] = q / b;
            if (q != 0) r[n++] = d / q;
        }
        return n;
    }
    const double B = b / a, C = c / a, D = d / a;
    const double p = C - B * B / 3.0, q = 2.0 * B * B * B / 27.0 - B * C / 3.0 + D;
    const double disc = 0.25 * q * q + p * p * p / 27.0;
    if (disc > 0) {
        const double s = sqrt(disc);
        r[n++] = cbrt(-0.5 * q + s) + cbrt(-0.5 * q - s) - B / 3.0;
    } else if (p == 0) {
        r[n++] = -B / 3.0;
    } else {
        const double m = 2.0 * sqrt(-p / 3.0);
        double arg = 3.0 * q / (p * m);
        arg = fmax(-1.0, fmin(1.0, arg));
        const double th = acos(arg) / 3.0;
        for (int k = 0; k < 3; ++k) r[n++] = m * cos(th - 2.0943951023931957 * k) - B / 3.0;
    }
    for (int i = 0; i < n; ++i) {
        for (int it = 0; it < 2; ++it) {
            const double x = r[i];
            const double f = ((a * x + b) * x + c) * x + d, fp = (3 * a * x + 2 * b) * x + c;
            if (fp != 0) r[i] = x - f / fp;
        }
    }
    return n;
}

// ---- More-Thuente search on Q (variant; More & Thuente 1994) -------------
// The same steps as the published algorithm: trial steps in an interval of
// uncertainty updated by the four cases of its Section 4, first on
// psi(a) = phi(a) - ftol a phi'(0), then on phi; bisection when the interval
// fails to shrink by 0.66 over two trials; extrapolation in
// [1.1, 4] x the last move before anything is bracketed.  phi = Q - c0.
// Every product and sum is rounded on its own (no contraction).
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

__device__ double q_slope(const double *c, double al) {   // Q'(alpha)
    double t = dmul(dmul(al, 4.0), c[4]);
    t = dadd(dmul(3.0, c[3]), t);
    t = dadd(dmul(2.0, c[2]), dmul(al, t));
    return dadd(c[1], dmul(al, t));
}

// minimiser of the cubic through (a, fa; slope da) and (b, fb; slope db);
// false if it has none
__device__ bool mt_cubic(double a, double fa, double da, double b, double fb, double db, double *out) {
    const double d1 = dsub(dadd(da, db), ddiv(dmul(3.0, dsub(fa, fb)), dsub(a, b)));
    const double disc = dsub(dmul(d1, d1), dmul(da, db));
    if (disc < 0.0) return false;
    const double d2 = copysign(__dsqrt_rn(disc), dsub(b, a));
    const double den = dadd(dsub(db, da), dmul(2.0, d2));
    if (den == 0.0) return false;
    *out = dsub(b, ddiv(dmul(dsub(b, a), dsub(dadd(db, d2), d1)), den));
    return true;
}

__device__ double mt_quad(double a, double fa, double da, double b, double fb) {
    const double h = dsub(b, a);
    return dadd(a, ddiv(dmul(dmul(0.5, da), dmul(h, h)), dadd(dsub(fa, fb), dmul(da, h))));
}

__device__ double mt_secant(double a, double da, double b, double db) {
    return dsub(b, ddiv(dmul(db, dsub(b, a)), dsub(db, da)));
}

struct MtEnds {
    double x, fx, dx, y, fy, dy;
};

// one trial-step choice and interval update; returns the next trial
__device__ double mt_trial(MtEnds &e, double t, double ft, double dt, bool &brackt, double lo, double hi) {
    const bool same = dmul(dt, copysign(1.0, e.dx)) > 0.0;
    double nxt, cc;
    if (ft > e.fx) {                                   // case 1
        const double q = mt_quad(e.x, e.fx, e.dx, t, ft);
        if (!mt_cubic(e.x, e.fx, e.dx, t, ft, dt, &cc)) cc = q;
        nxt = fabs(dsub(cc, e.x)) < fabs(dsub(q, e.x)) ? cc : dadd(cc, dmul(0.5, dsub(q, cc)));
        brackt = true;
    } else if (!same) {                                // case 2
        const double sc = mt_secant(e.x, e.dx, t, dt);
        if (!mt_cubic(e.x, e.fx, e.dx, t, ft, dt, &cc)) cc = sc;
        nxt = fabs(dsub(cc, t)) >= fabs(dsub(sc, t)) ? cc : sc;
        brackt = true;
    } else if (fabs(dt) < fabs(e.dx)) {                // case 3
        const bool have = mt_cubic(e.x, e.fx, e.dx, t, ft, dt, &cc);
        const bool beyond = have && dmul(dsub(cc, t), dsub(t, e.x)) > 0.0;
        if (!beyond) cc = t > e.x ? hi : lo;
        const double sc = mt_secant(e.x, e.dx, t, dt);
        if (brackt) {
            nxt = fabs(dsub(cc, t)) < fabs(dsub(sc, t)) ? cc : sc;
            const double lim = dadd(t, dmul(0.66, dsub(e.y, t)));
            nxt = t > e.x ? fmin(lim, nxt) : fmax(lim, nxt);
        } else {
            nxt = fabs(dsub(cc, t)) > fabs(dsub(sc, t)) ? cc : sc;
            nxt = fmin(hi, fmax(lo, nxt));
        }
    } else {                                           // case 4
        if (brackt) {
            if (!mt_cubic(t, ft, dt, e.y, e.fy, e.dy, &nxt)) nxt = dmul(0.5, dadd(t, e.y));
        } else {
            nxt = t > e.x ? hi : lo;
        }
    }
    if (ft > e.fx) {
        e.y = t; e.fy = ft; e.dy = dt;
    } else {
        if (!same) { e.y = e.x; e.fy = e.fx; e.dy = e.dx; }
        e.x = t; e.fx = ft; e.dx = dt;
    }
    return nxt;
}

// returns ok; *alpha the step, *dq = Q(alpha) - Q(0), *nfev the evaluations
__device__ bool more_thuente(const double *c, const LsParams &lp, double *alpha, double *dq, int *nfev) {
    const double g0 = c[1];
    const double ftol = lp.c, gtol = lp.c2, xtol = 1e-15, stpmin = 1e-15, stpmax = 1e15;
    const double gtest = dmul(ftol, g0);
    bool brackt = false, stage1 = true;
    double width = dsub(stpmax, stpmin), width_prev = dmul(2.0, width);
    MtEnds e{0.0, 0.0, g0, 0.0, 0.0, g0};
    double lo = 0.0, hi = dadd(lp.alpha0, dmul(4.0, lp.alpha0));
    double t = fmin(fmax(lp.alpha0, stpmin), stpmax);
    bool have_best = false;
    double best_t = 0.0, best_f = 0.0;
    int n = 0;
    while (n < lp.max_shrinks) {
        ++n;
        const double ft = q_delta(c, t), dt = q_slope(c, t);
        const double ftest = dmul(t, gtest);
        if (ft <= ftest && (!have_best || ft < best_f)) { have_best = true; best_t = t; best_f = ft; }
        if (stage1 && ft <= ftest && dt >= 0.0) stage1 = false;
        if (ft <= ftest && fabs(dt) <= dmul(-gtol, g0)) {
            *alpha = t; *dq = ft; *nfev = n;
            return true;
        }
        if ((brackt && (t <= lo || t >= hi)) || (brackt && dsub(hi, lo) <= dmul(xtol, hi)) ||
            (t == stpmax && ft <= ftest && dt <= gtest) || (t == stpmin && (ft > ftest || dt >= gtest)))
            break;
        double tn;
        if (stage1 && ft <= e.fx && ft > ftest) {
            // the auxiliary function psi = phi - a gtest
            MtEnds m{e.x, dsub(e.fx, dmul(e.x, gtest)), dsub(e.dx, gtest),
                     e.y, dsub(e.fy, dmul(e.y, gtest)), dsub(e.dy, gtest)};
            tn = mt_trial(m, t, dsub(ft, dmul(t, gtest)), dsub(dt, gtest), brackt, lo, hi);
            e.x = m.x; e.fx = dadd(m.fx, dmul(m.x, gtest)); e.dx = dadd(m.dx, gtest);
            e.y = m.y; e.fy = dadd(m.fy, dmul(m.y, gtest)); e.dy = dadd(m.dy, gtest);
        } else {
            tn = mt_trial(e, t, ft, dt, brackt, lo, hi);
        }
        if (brackt) {
            if (fabs(dsub(e.y, e.x)) >= dmul(0.66, width_prev)) tn = dadd(e.x, dmul(0.5, dsub(e.y, e.x)));
            width_prev = width;
            width = fabs(dsub(e.y, e.x));
            lo = fmin(e.x, e.y);
            hi = fmax(e.x, e.y);
        } else {
            lo = dadd(tn, dmul(1.1, dsub(tn, e.x)));
            hi = dadd(tn, dmul(4.0, dsub(tn, e.x)));
        }
        tn = fmin(fmax(tn, stpmin), stpmax);
        if ((brackt && (tn <= lo || tn >= hi)) || (brackt && dsub(hi, lo) <= dmul(xtol, hi))) tn = e.x;
        t = tn;
    }
    *nfev = n;
    if (have_best) {   // no strong-Wolfe step: the best step with sufficient decrease
        *alpha = best_t; *dq = best_f;
        return true;
    }
    return false;
}

__device__ void post_lselect(double *S, const LsParams lp) {
    const double *c = S + S_C;
    double alpha = 0.0, dq = 0.0;
    int ok = 0, k = 0;
    if (c[1] < 0.0) {
        if (lp.mode == ALS_LS_MORE_THUENTE) {
            ok = more_thuente(c, lp, &alpha, &dq, &k) ? 1 : 0;
        } else if (lp.mode == ALS_LS_EXACT) {
            double r[3];
            const int n = cubic_roots(4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1], r);
            double best = 0.0;
            for (int i = 0; i < n; ++i) {
                if (r[i] > 0.0) {
                    const double v = q_delta(c, r[i]);
                    if (!ok || v < best) { best = v; alpha = r[i]; ok = 1; }
                }
            }
            dq = best;
        } else {
            alpha = lp.alpha0;
            for (k = 0; k <= lp.max_shrinks; ++k) {
                dq = q_delta(c, alpha);
                const double rhs = dmul(dmul(alpha, lp.c), c[1]);
                if (dq <= rhs) { ok = 1; break; }
                alpha = dmul(alpha, lp.tau);
            }
            if (!ok) k = lp.max_shrinks;
        }
    }
    if (ok) {
        S[S_ALPHA] = alpha;
        S[S_MODE] = 0.0;
        S[S_F] = dadd(c[0], dq);
    } else {
        S[S_ALPHA] = 0.0;
        S[S_MODE] = 1.0;
        S[S_F] = __longlong_as_double(0x7ff8000000000000ll);  // unknown until evaluated
        S[S_NFALL] += 1.0;
    }
    S[S_SHRINK] = (double)k;
}

// scalar step after a reduction, on one problem's scalars (one thread)
__device__ void run_post(double *S, int s_off, int post, const LsParams &lp) {
    if (post == POST_LSELECT) {
        post_lselect(S, lp);
    } else if (post == POST_BETA) {
        const double gg = S[s_off], gbg = S[s_off + 1], gbd = S[s_off + 2];
        const double sk = S[S_S];
        double beta = 0.0;
        if (S[S_MODE] == 0.0) {   // after a fallback the direction restarts
            if (lp.beta == ALS_BETA_FR) {
                beta = sk != 0.0 ? gbg / sk : 0.0;
            } else if (lp.beta == ALS_BETA_HS) {
                const double pd = S[s_off + 3];
                beta = pd != 0.0 ? gbd / pd : 0.0;
            } else {
                beta = sk != 0.0 ? gbd / sk : 0.0;
                if (lp.beta == ALS_BETA_PR_PLUS) beta = fmax(0.0, beta);
            }
        }
        S[S_BETA] = beta;
        S[S_S] = gbg;
        S[S_GG] = gg;
    } else if (post == POST_INIT) {
        S[S_GG] = S[s_off];
        S[S_GG0] = S[s_off];
        S[S_S] = S[s_off + 1];
        S[S_MODE] = 0.0;
        S[S_BETA] = 0.0;
        S[S_NFALL] = 0.0;
        S[S_ALPHA] = 0.0;
        S[S_SHRINK] = 0.0;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const double *__restrict__ rowterm, int64_t n,
                                                        int nterms, double *__restrict__ partial,
                                                        unsigned *__restrict__ ticket, double *__restrict__ S,
                                                        int s_off, int post, LsParams lp) {
    __shared__ double red[RED_THREADS];
    __shared__ bool last;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int t = 0; t < nterms; ++t) {
        double s = 0.0;
        for (int64_t i = b0 + threadIdx.x; i < b1; i += RED_THREADS) s += rowterm[t * n + i];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[t * RED_MAXB + blockIdx.x] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(ticket, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int t = 0; t < nterms; ++t) {
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += RED_THREADS) s += partial[t * RED_MAXB + i];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) S[s_off + t] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *ticket = 0u;
        run_post(S, s_off, post, lp);
    }
}

// Batched problems: block q reduces problem q's user rows [segu[q], segu[q+1])
// and item rows [n_u + segm[q], n_u + segm[q+1]) in a fixed order, then runs
// the post-operation on problem q's scalars S + q * S_COUNT.
__global__ void __launch_bounds__(RED_THREADS) k_reduce_seg(const double *__restrict__ rowterm, int64_t n, int nterms,
                                                            const int64_t *__restrict__ segu,
                                                            const int64_t *__restrict__ segm, int64_t n_u,
                                                            double *__restrict__ S, int s_off, int post, LsParams lp) {
    __shared__ double red[RED_THREADS];
    const int q = blockIdx.x;
    double *Sq = S + (size_t)q * S_COUNT;
    const int64_t u0 = segu[q], u1 = segu[q + 1], m0 = n_u + segm[q], m1 = n_u + segm[q + 1];
    for (int t = 0; t < nterms; ++t) {
        double s = 0.0;
        for (int64_t i = u0 + threadIdx.x; i < u1; i += RED_THREADS) s += rowterm[t * n + i];
        for (int64_t i = m0 + threadIdx.x; i < m1; i += RED_THREADS) s += rowterm[t * n + i];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) Sq[s_off + t] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) run_post(Sq, s_off, post, lp);
}

// ---------------------------------------------------------------------------
// vectors
// ---------------------------------------------------------------------------
// rowprob == nullptr: one problem; otherwise the scalars of row i / ld's problem
template <typename T>
__global__ void k_update_x(T *__restrict__ X, const T *__restrict__ Xbar, const T *__restrict__ P,
                           const double *__restrict__ S, const int32_t *__restrict__ rowprob, int ld, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *Sq = rowprob ? S + (size_t)rowprob[i / ld] * S_COUNT : S;
        const bool fallback = Sq[S_MODE] != 0.0;
        const T al = (T)Sq[S_ALPHA];
        X[i] = fallback ? Xbar[i] : fma(al, P[i], X[i]);
    }
}

template <typename T>
__global__ void k_update_p(T *__restrict__ P, const T *__restrict__ Gbar, const double *__restrict__ S,
                           const int32_t *__restrict__ rowprob, int ld, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *Sq = rowprob ? S + (size_t)rowprob[i / ld] * S_COUNT : S;
        const T be = (T)Sq[S_BETA];
        P[i] = fma(be, P[i], -Gbar[i]);
    }
}

template <typename T>
__global__ void k_neg(T *__restrict__ d, const T *__restrict__ s, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = -s[i];
}

// user layout (dtype S_, row stride nf) -> internal (T, row stride ld, zero pad)
template <typename TS, typename TD>
__global__ void k_convert(TD *__restrict__ dst, const TS *__restrict__ src, int64_t rows, int nf,
                          int src_ld, int dst_ld) {
    const int64_t n = rows * dst_ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / dst_ld;
        const int k = (int)(i - r * dst_ld);
        if (k < nf) dst[i] = (TD)src[r * src_ld + k];
        else if (k < dst_ld) dst[i] = TD(0);
    }
}

inline unsigned grid_for(als_ctx *c, int64_t n, int threads) {
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)c->sm_count * c->grid_mult;
    return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

template <int LPR>
struct Lpr {};

inline int lpr_for(int ld) {
    const int slots = ld / 4;
    if (slots <= 4) return 4;
    if (slots <= 8) return 8;
    if (slots <= 16) return 16;
    return 32;
}

template <typename T, int LPR>
als_status grad_launch(als_ctx *c, const PassArgs &a, bool heavy) {
    if (a.nrows <= 0) return ALS_OK;
    if (heavy) {
        const unsigned g = (unsigned)std::min<int64_t>(a.nrows, 65535);
        k_grad_heavy<T, LPR><<<g, 256, 0, c->stream>>>(a);
    } else {
        const int64_t groups_per_block = 256 / LPR;
        const int64_t want = (a.nrows + groups_per_block - 1) / groups_per_block;
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->sm_count * c->grid_mult));
        k_grad<T, LPR><<<g, 256, 0, c->stream>>>(a);
    }
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

template <typename T, int LPR, bool HAS_P>
als_status lscoef_launch(als_ctx *c, const PassArgs &a, int kind) {  // 0 rows, 1 heavy, 2 reg
    if (a.nrows <= 0) return ALS_OK;
    if (kind == 1) {
        const unsigned g = (unsigned)std::min<int64_t>(a.nrows, 65535);
        k_lscoef_heavy<T, LPR, HAS_P><<<g, 256, 0, c->stream>>>(a);
    } else {
        const int64_t groups_per_block = 256 / LPR;
        const int64_t want = (a.nrows + groups_per_block - 1) / groups_per_block;
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->sm_count * c->grid_mult));
        if (kind == 0) k_lscoef<T, LPR, HAS_P><<<g, 256, 0, c->stream>>>(a);
        else k_lscoef_reg<T, LPR, HAS_P><<<g, 256, 0, c->stream>>>(a);
    }
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

template <typename T>
als_status grad_dispatch(als_ctx *c, const PassArgs &a, bool heavy) {
    switch (lpr_for(a.ld)) {
        case 4: return grad_launch<T, 4>(c, a, heavy);
        case 8: return grad_launch<T, 8>(c, a, heavy);
        case 16: return grad_launch<T, 16>(c, a, heavy);
        default: return grad_launch<T, 32>(c, a, heavy);
    }
}

template <typename T, int LPR>
als_status grad_terms_launch(als_ctx *c, const PassArgs &a) {
    if (a.nrows <= 0) return ALS_OK;
    const int64_t groups_per_block = 256 / LPR;
    const int64_t want = (a.nrows + groups_per_block - 1) / groups_per_block;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->sm_count * c->grid_mult));
    k_grad_terms<T, LPR><<<g, 256, 0, c->stream>>>(a);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

template <typename T>
als_status grad_terms_dispatch(als_ctx *c, const PassArgs &a) {
    switch (lpr_for(a.ld)) {
        case 4: return grad_terms_launch<T, 4>(c, a);
        case 8: return grad_terms_launch<T, 8>(c, a);
        case 16: return grad_terms_launch<T, 16>(c, a);
        default: return grad_terms_launch<T, 32>(c, a);
    }
}

template <typename T, bool HAS_P>
als_status lscoef_dispatch(als_ctx *c, const PassArgs &a, int kind) {
    switch (lpr_for(a.ld)) {
        case 4: return lscoef_launch<T, 4, HAS_P>(c, a, kind);
        case 8: return lscoef_launch<T, 8, HAS_P>(c, a, kind);
        case 16: return lscoef_launch<T, 16, HAS_P>(c, a, kind);
        default: return lscoef_launch<T, 32, HAS_P>(c, a, kind);
    }
}

}  // namespace

als_status launch_grad(als_ctx *c, const PassArgs &a, bool heavy) {
    return c->f64 ? grad_dispatch<double>(c, a, heavy) : grad_dispatch<float>(c, a, heavy);
}

als_status launch_grad_terms(als_ctx *c, const PassArgs &a) {
    return c->f64 ? grad_terms_dispatch<double>(c, a) : grad_terms_dispatch<float>(c, a);
}

als_status launch_lscoef(als_ctx *c, const PassArgs &a, bool heavy) {
    const int kind = heavy ? 1 : 0;
    if (a.Ps) return c->f64 ? lscoef_dispatch<double, true>(c, a, kind) : lscoef_dispatch<float, true>(c, a, kind);
    return c->f64 ? lscoef_dispatch<double, false>(c, a, kind) : lscoef_dispatch<float, false>(c, a, kind);
}

als_status launch_lscoef_reg(als_ctx *c, const PassArgs &a) {
    if (a.Ps) return c->f64 ? lscoef_dispatch<double, true>(c, a, 2) : lscoef_dispatch<float, true>(c, a, 2);
    return c->f64 ? lscoef_dispatch<double, false>(c, a, 2) : lscoef_dispatch<float, false>(c, a, 2);
}

als_status launch_reduce(als_ctx *c, int nterms, int64_t n, int s_off, int post, const LsParams &lp) {
    if (c->n_prob > 1) {
        k_reduce_seg<<<(unsigned)c->n_prob, RED_THREADS, 0, c->stream>>>(c->rowterm, n, nterms, c->segu, c->segm,
                                                                         c->n_u, c->S, s_off, post, lp);
        ALS_CUDA_TRY(cudaGetLastError());
        return ALS_OK;
    }
    const int64_t want = (n + 8191) / 8192;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, RED_MAXB));
    k_reduce<<<g, RED_THREADS, 0, c->stream>>>(c->rowterm, n, nterms, c->partial, c->ticket, c->S, s_off,
                                               post, lp);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_update_x(als_ctx *c) {
    const int64_t n = (c->n_u + c->n_m) * c->ld;
    const unsigned g = grid_for(c, n, 256);
    if (c->f64) k_update_x<double><<<g, 256, 0, c->stream>>>((double *)c->X, (const double *)c->Xbar, (const double *)c->P, c->S, c->rowprob, c->ld, n);
    else k_update_x<float><<<g, 256, 0, c->stream>>>((float *)c->X, (const float *)c->Xbar, (const float *)c->P, c->S, c->rowprob, c->ld, n);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_update_p(als_ctx *c) {
    const int64_t n = (c->n_u + c->n_m) * c->ld;
    const unsigned g = grid_for(c, n, 256);
    if (c->f64) k_update_p<double><<<g, 256, 0, c->stream>>>((double *)c->P, (const double *)c->Gbar, c->S, c->rowprob, c->ld, n);
    else k_update_p<float><<<g, 256, 0, c->stream>>>((float *)c->P, (const float *)c->Gbar, c->S, c->rowprob, c->ld, n);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_neg_copy(als_ctx *c, void *dst, const void *src, size_t n) {
    const unsigned g = grid_for(c, (int64_t)n, 256);
    if (c->f64) k_neg<double><<<g, 256, 0, c->stream>>>((double *)dst, (const double *)src, (int64_t)n);
    else k_neg<float><<<g, 256, 0, c->stream>>>((float *)dst, (const float *)src, (int64_t)n);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_convert_in(als_ctx *c, void *dst, const void *src, int64_t rows, int src_dtype, int src_ld) {
    if (rows <= 0) return ALS_OK;
    const unsigned g = grid_for(c, rows * c->ld, 256);
    if (c->f64) {
        if (src_dtype == ALS_DT_F64) k_convert<double, double><<<g, 256, 0, c->stream>>>((double *)dst, (const double *)src, rows, c->nf, src_ld, c->ld);
        else k_convert<float, double><<<g, 256, 0, c->stream>>>((double *)dst, (const float *)src, rows, c->nf, src_ld, c->ld);
    } else {
        if (src_dtype == ALS_DT_F64) k_convert<double, float><<<g, 256, 0, c->stream>>>((float *)dst, (const double *)src, rows, c->nf, src_ld, c->ld);
        else k_convert<float, float><<<g, 256, 0, c->stream>>>((float *)dst, (const float *)src, rows, c->nf, src_ld, c->ld);
    }
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_convert_out(als_ctx *c, void *dst, const void *src, int64_t rows, int dst_dtype, int dst_ld) {
    if (rows <= 0) return ALS_OK;
    const unsigned g = grid_for(c, rows * dst_ld, 256);
    if (c->f64) {
        if (dst_dtype == ALS_DT_F64) k_convert<double, double><<<g, 256, 0, c->stream>>>((double *)dst, (const double *)src, rows, c->nf, c->ld, dst_ld);
        else k_convert<double, float><<<g, 256, 0, c->stream>>>((float *)dst, (const double *)src, rows, c->nf, c->ld, dst_ld);
    } else {
        if (dst_dtype == ALS_DT_F64) k_convert<float, double><<<g, 256, 0, c->stream>>>((double *)dst, (const float *)src, rows, c->nf, c->ld, dst_ld);
        else k_convert<float, float><<<g, 256, 0, c->stream>>>((float *)dst, (const float *)src, rows, c->nf, c->ld, dst_ld);
    }
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

namespace {
__global__ void k_check_requests(const int64_t *__restrict__ ptr, int64_t nreq, const int32_t *__restrict__ idx,
                                 const float *__restrict__ val, int64_t total, int64_t bound, int *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride)
        if (idx[e] < 0 || idx[e] >= bound || !isfinite(val[e])) atomicAdd(flag, 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nreq; q += stride)
        if (ptr[q + 1] < ptr[q] || ptr[q + 1] > total) atomicAdd(flag, 1);
}
}  // namespace

als_status launch_check_requests(als_ctx *c, const int64_t *ptr, int64_t nreq, const int32_t *idx, const float *val,
                                 int64_t total, int64_t bound, int *flag) {
    ALS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    const unsigned g = grid_for(c, std::max(total, nreq), 256);
    k_check_requests<<<g, 256, 0, c->stream>>>(ptr, nreq, idx, val, total, bound, flag);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

// ---------------------------------------------------------------------------
// batched problems: global ids and the row -> problem map
// ---------------------------------------------------------------------------
namespace {
__global__ void k_offset_ids(const int64_t *__restrict__ nnzoff, int n_prob, const int64_t *__restrict__ segu,
                             const int64_t *__restrict__ segm, int32_t *__restrict__ rows, int32_t *__restrict__ cols,
                             int64_t nnz, int *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        int lo = 0, hi = n_prob;  // last q with nnzoff[q] <= e
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (nnzoff[mid] <= e) lo = mid; else hi = mid;
        }
        const int64_t nu = segu[lo + 1] - segu[lo], nm = segm[lo + 1] - segm[lo];
        const int32_t r = rows[e], c = cols[e];
        if (r < 0 || r >= nu || c < 0 || c >= nm) {
            atomicAdd(flag, 1);
            rows[e] = -1;
            cols[e] = -1;
        } else {
            rows[e] = (int32_t)(r + segu[lo]);
            cols[e] = (int32_t)(c + segm[lo]);
        }
    }
}

__global__ void k_rowprob(const int64_t *__restrict__ segu, const int64_t *__restrict__ segm, int n_prob, int64_t n_u,
                          int64_t n, int32_t *__restrict__ rowprob) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t *seg = i < n_u ? segu : segm;
        const int64_t v = i < n_u ? i : i - n_u;
        int lo = 0, hi = n_prob;  // last q with seg[q] <= v
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg[mid] <= v) lo = mid; else hi = mid;
        }
        rowprob[i] = lo;
    }
}
}  // namespace

als_status launch_offset_ids(als_ctx *c, const int64_t *nnzoff, int n_prob, const int64_t *segu, const int64_t *segm,
                             int32_t *rows, int32_t *cols, int64_t nnz, int *flag) {
    if (nnz <= 0) return ALS_OK;
    k_offset_ids<<<grid_for(c, nnz, 256), 256, 0, c->stream>>>(nnzoff, n_prob, segu, segm, rows, cols, nnz, flag);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status launch_rowprob(als_ctx *c) {
    const int64_t n = c->n_u + c->n_m;
    k_rowprob<<<grid_for(c, n, 256), 256, 0, c->stream>>>(c->segu, c->segm, c->n_prob, c->n_u, n, c->rowprob);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}
