// Mixed-precision half sweep with the Gram matrices on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// For each row i (one CTA of 4 warps per row, 4 CTAs per SM), with the fixed
// side F kept in a BF16 shadow of 128 columns:
//   1. gather: each factor row is held as two BF16 rows, hi = bf16(f) and
//      lo2 = bf16(2 (f - hi)); the rows of the row's ratings, 32 per chunk,
//      are copied with cp.async into two 128-byte-swizzled, MN-major shared
//      tiles H and L (rating k of the chunk is K index k, the factor index is
//      the M/N index);
//   2. Gram: one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//      M = 128, N = round_up(n_f, 16), K = 16 per instruction): D += H H^T
//      and D += H L^T, so D = sum_e hi_e (hi_e + 2 lo_e)^T accumulates in
//      TMEM; its symmetric part is sum_e (hi hi^T + hi lo^T + lo hi^T), the
//      Gram matrix with ~2^-17 relative error (the lo lo^T term is dropped).
//      Chunks are double buffered; tcgen05.commit on an mbarrier releases a
//      stage;
//   3. tcgen05.ld moves D into FP32 shared memory (row m of D is TMEM lane
//      m), A = (D + D^T)/2 + lambda n_i I;
//   4. blocked Cholesky of A (inverted diagonal blocks) and the refinement of
//      the ALS solve from the current row u0 = x_i: res = sum_e f_e (r_e -
//      f_e . u) - lambda n_i u in FP32 from the FP32 factors, u <- u +
//      A^{-1} res.  The first residual (at u0) is gathered inside the Gram
//      loop, while the chunk's copies and MMAs are in flight.
// Every mbarrier wait is bounded (%globaltimer): on expiry the CTA records a
// timeout, waits for its copies, frees its TMEM and returns.
#include "internal.cuh"
#include "sweep_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_THREADS = 128;
constexpr int KCH = 32;                          // ratings per chunk
constexpr int TILE_BYTES = KCH * ALS_TC_LD * 2;  // 8 KB: one BF16 tile (H or L)
constexpr int STAGE_BYTES = 2 * TILE_BYTES;      // H and L
constexpr int NSTAGE = 2;
constexpr uint32_t LBO = 1024;  // byte distance between the two 64-wide MN atoms
constexpr uint32_t SBO = 2048;  // byte distance between groups of 8 K rows
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int TMEM_COLS = 128;

struct TcLayout {
    int ring, meta, A, vec, mbar, holder, total;
};

__host__ __device__ inline TcLayout tc_layout(int nf) {
    TcLayout L;
    L.ring = 0;
    L.A = 0;  // the FP32 matrix reuses the gather ring once the MMAs are done
    L.meta = NSTAGE * STAGE_BYTES;  // per stage: the chunk's ids, then its ratings
    int big = L.meta + NSTAGE * KCH * 8;
    const int a_bytes = nf * (nf + 1) * 4;
    if (a_bytes > big) big = a_bytes;
    big = (big + 15) & ~15;
    L.vec = big;  // colk, v1, v2, u, diag [5][128]; then part[4][128] / Cholesky work (aliased)
    L.mbar = L.vec + (5 * 128 + 16 * 128 + 256 + 16) * 4;
    L.holder = L.mbar + 16;
    L.total = L.holder + 16;
    return L;
}

__global__ void __launch_bounds__(TC_THREADS, 4) k_sweep_tc(SweepArgs a, int ntc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char *base = smem_raw + pad;
    const uint32_t sbase = raw + pad;
    const int nf = a.nf, ldA = nf + 1;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const TcLayout L = tc_layout(nf);
    float *A = reinterpret_cast<float *>(base + L.A);
    float *vec = reinterpret_cast<float *>(base + L.vec);
    float *colk = vec, *v1 = vec + 128, *v2 = vec + 256, *u = vec + 384, *diag = vec + 512;
    float *part = vec + 640;   // residual partials (residual phase)
    float *work = vec + 640;   // Cholesky panel scratch (factorisation phase)
    int32_t *meta_i = reinterpret_cast<int32_t *>(base + L.meta);          // [NSTAGE][KCH]
    float *meta_v = reinterpret_cast<float *>(base + L.meta + NSTAGE * KCH * 4);
    const uint32_t mbar[2] = {sbase + L.mbar, sbase + L.mbar + 8};
    uint32_t *holder = reinterpret_cast<uint32_t *>(base + L.holder);

    if (t == 0) {
        mbar_init(mbar[0], 1);
        mbar_init(mbar[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(sbase + L.holder, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    const uint32_t idesc = idesc_bf16_f32_mn((uint32_t)ntc);
    const float *F = reinterpret_cast<const float *>(a.F);
    const __nv_bfloat16 *Fb = a.Fbf;
    uint32_t phase[2] = {0u, 0u};
    bool bail = false;

    for (int64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {
        const bool seg = a.seg_out != nullptr;  // a slice of a split row: partials only
        const int64_t row = seg ? a.order[a.seg_row[r]] : (a.order ? a.order[r] : r);
        const int64_t beg = seg ? a.seg_beg[r] : a.ptr[row];
        const int n = seg ? a.seg_len[r] : (int)(a.ptr[row + 1] - beg);
        const float *xi = a.Xin ? reinterpret_cast<const float *>(a.Xin) + row * a.ld : nullptr;
        float *xo = reinterpret_cast<float *>(a.Xout) + row * a.ld;
        float *gb = a.Gbar ? reinterpret_cast<float *>(a.Gbar) + row * a.ld : nullptr;
        const float lam_n = (float)(a.lambda * (double)n);
        bool ok = n > 0;
        // current row u0 = x_i (fold-in: 0), one 4-wide slot per lane
        const bool act = 4 * lane < a.ld;
        float uu[4], acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) uu[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
        for (int k = t; k < nf; k += TC_THREADS) u[k] = xi ? xi[k] : 0.0f;
        if (ok) {
            // ---- 1-2. gather + tensor-core Gram, with the first FP32 residual
            //      r0 = sum_e f_e (r_e - f_e . u0) of the chunk's ratings computed
            //      while the chunk's copies and MMAs are in flight -------------
            const int nch = (n + KCH - 1) / KCH;
            int pend[2] = {0, 0};
            // ids and ratings of the next chunk to gather: thread t copies
            // ratings k0 + 8 j (j < 4) of a chunk, k0 = (t / 16) % 8
            const int k0 = (t >> 4) & 7;
            int32_t pj[4];
            float pv[4];
            auto prefetch = [&](int ch) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t e = beg + (int64_t)ch * KCH + k0 + 8 * j;
                    const bool in = ch < nch && e < beg + n;
                    pj[j] = in ? a.idx[e] : -1;
                    pv[j] = in ? a.val[e] : 0.0f;
                }
            };
            auto gather = [&](int st) {
                const uint32_t stage = sbase + L.ring + st * STAGE_BYTES;
#pragma unroll
                for (int i = 0; i < (2 * KCH * 16) / TC_THREADS; ++i) {
                    const int p = t + TC_THREADS * i;
                    const int part_ = p >> 9, k = (p >> 4) & (KCH - 1), q = p & 15;
                    const uint32_t dst = stage + part_ * TILE_BYTES + (k >> 3) * SBO + (q >> 3) * LBO + (k & 7) * 128 +
                                         ((uint32_t)((q & 7) ^ (k & 7)) << 4);
                    const int32_t j = pj[i & 3];
                    if (j >= 0) cp_async16(dst, Fb + (int64_t)j * (2 * ALS_TC_LD) + part_ * ALS_TC_LD + q * 8);
                    else cp_async16_zero(dst, Fb);
                }
                cp_async_commit();
                if ((t & 15) == 0) {  // the chunk's ids and ratings for its residual
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        meta_i[st * KCH + k0 + 8 * j] = pj[j];
                        meta_v[st * KCH + k0 + 8 * j] = pv[j];
                    }
                }
            };
            prefetch(0);
            gather(0);
            prefetch(1);
            __syncthreads();  // chunk 0's ids and ratings visible to every warp
            for (int ch = 0; ch < nch; ++ch) {
                const int st = ch & 1;
                if (ch + 1 < nch) {
                    const int sn = st ^ 1;
                    if (pend[sn]) {  // the MMAs of chunk ch-1 still read stage sn
                        const bool w = mbar_wait_bounded(mbar[sn], phase[sn], WAIT_NS);
                        if (__syncthreads_or(!w)) { bail = true; break; }
                        phase[sn] ^= 1u;
                        pend[sn] = 0;
                    }
                    gather(sn);
                    prefetch(ch + 2);
                }
                {
                    const int cnt = (n - ch * KCH < KCH) ? n - ch * KCH : KCH;
                    resid8(F, a.ld, meta_i + st * KCH + warp, meta_v + st * KCH + warp, cnt - warp, uu, lane, act,
                           acc, cmp);
                }
                if (ch + 1 < nch) cp_async_wait<1>();
                else cp_async_wait<0>();
                fence_proxy_async_smem();
                __syncthreads();
                if (t == 0) {
                    tc_fence_after();
                    const uint32_t stage = sbase + L.ring + st * STAGE_BYTES;
#pragma unroll
                    for (int s = 0; s < KCH / 16; ++s) {
                        const uint64_t dh = smem_desc_sw128(stage + (uint32_t)s * 2u * SBO, LBO, SBO);
                        const uint64_t dl = smem_desc_sw128(stage + TILE_BYTES + (uint32_t)s * 2u * SBO, LBO, SBO);
                        tc_mma_bf16(tmem, dh, dh, idesc, (ch > 0 || s > 0) ? 1u : 0u);
                        tc_mma_bf16(tmem, dh, dl, idesc, 1u);
                    }
                    tc_commit(mbar[st]);
                }
                pend[st] = 1;
            }
            if (bail) break;
            for (int s = 0; s < 2; ++s) {
                if (pend[s]) {
                    const bool w = mbar_wait_bounded(mbar[s], phase[s], WAIT_NS);
                    if (__syncthreads_or(!w)) { bail = true; break; }
                    phase[s] ^= 1u;
                    pend[s] = 0;
                }
            }
            if (bail) break;
#pragma unroll
            for (int i = 0; i < 4; ++i) part[warp * 128 + 4 * lane + i] = acc[i] - cmp[i];
            tc_fence_after();
            // ---- 3. TMEM -> FP32 A (row m of D is TMEM lane m) -----------------
            {
                const int m = 32 * warp + lane;
                for (int c0 = 0; c0 < ntc; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
                    if (m < nf) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int col = c0 + i;
                            if (col < nf) A[m * ldA + col] = v[i];
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            if (seg) {
                // the slice's partials: packed lower triangle of the symmetric
                // part of D (row m at m (m + 1) / 2), then its residual at u0
                float *po = reinterpret_cast<float *>(a.seg_out) + r * a.seg_stride;
                const int tri = nf * (nf + 1) / 2;
                for (int e = t; e < tri; e += TC_THREADS) {
                    int m = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                    while ((m + 1) * (m + 2) / 2 <= e) ++m;
                    while (m * (m + 1) / 2 > e) --m;
                    const int cc = e - m * (m + 1) / 2;
                    po[e] = 0.5f * (A[m * ldA + cc] + A[cc * ldA + m]);
                }
                if (t < nf) po[tri + t] = (part[t] + part[128 + t]) + (part[256 + t] + part[384 + t]);
                __syncthreads();
                continue;
            }
            // symmetric part of D, lower triangle, plus lambda n I; the first
            // residual v1 = r0 - lambda n u0 (fixed order over the warps)
            if (t < nf) {
                for (int c = 0; c < t; ++c) A[t * ldA + c] = 0.5f * (A[t * ldA + c] + A[c * ldA + t]);
                A[t * ldA + t] += lam_n;
                v1[t] = ((part[t] + part[128 + t]) + (part[256 + t] + part[384 + t])) - lam_n * u[t];
            }
            __syncthreads();
            // ---- 4. Cholesky (inverted diagonal blocks), refinement ------------
            ok = chol_blocked128(A, ldA, nf, diag, work, t);
            if (ok) invert_diag_blocks128(A, ldA, nf, diag, t);
            if (!ok && t == 0) atomicAdd(a.notspd, 1);
        }
        if (ok) {
            trisolve_inv128(A, ldA, nf, v1, v2, colk, t);
            for (int k = t; k < nf; k += TC_THREADS) u[k] += colk[k];
            for (int s = 1; s < a.refine; ++s) {
                if (sw_correction_small<float, TC_THREADS>(colk, u, nf, n, part, t)) break;
                float uk[4], ak[4] = {0.f, 0.f, 0.f, 0.f}, ck[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 4; ++i) uk[i] = (4 * lane + i < nf) ? u[4 * lane + i] : 0.0f;
                for (int64_t e = beg + warp; e < beg + n; e += 32)
                    resid8(F, a.ld, a.idx + e, a.val + e, beg + n - e, uk, lane, act, ak, ck);
#pragma unroll
                for (int i = 0; i < 4; ++i) part[warp * 128 + 4 * lane + i] = ak[i] - ck[i];
                __syncthreads();
                if (t < nf) v1[t] = ((part[t] + part[128 + t]) + (part[256 + t] + part[384 + t])) - lam_n * u[t];
                trisolve_inv128(A, ldA, nf, v1, v2, colk, t);
                for (int k = t; k < nf; k += TC_THREADS) u[k] += colk[k];
            }
        } else {
            for (int k = t; k < nf; k += TC_THREADS) u[k] = (n > 0 && xi) ? xi[k] : 0.0f;
        }
        __syncthreads();
        for (int k = t; k < a.ld; k += TC_THREADS) {
            const float uk = k < nf ? u[k] : 0.0f;
            const float xk = xi ? xi[k] : 0.0f;
            xo[k] = uk;
            if (gb) gb[k] = xk - uk;
        }
        __syncthreads();
    }
    // ---- teardown: no copies in flight, TMEM returned -------------------------
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
    if (bail && t == 0) atomicAdd(a.timeout, 1);
}

}  // namespace

als_status launch_sweep_tc(als_ctx *c, const SweepArgs &a) {
    if (a.nrows <= 0) return ALS_OK;
    if (a.nf > ALS_TC_LD) {
        als_set_error("sweep: the tensor-core Gram supports n_f <= 128");
        return ALS_ENOTSUP;
    }
    const int ntc = (a.nf + 15) / 16 * 16;
    const TcLayout L = tc_layout(a.nf);
    // 46..56 KB of shared memory per CTA keeps exactly 4 CTAs (4 x 128 TMEM
    // columns = the SM's 512) resident per SM, so tcgen05.alloc never waits.
    size_t smem = (size_t)L.total + 1024;
    if (smem < 46 * 1024) smem = 46 * 1024;
    if (raise_smem_limit((const void *)k_sweep_tc, smem) != ALS_OK) return ALS_ECUDA;
    // the whole L1/shared array as shared memory, so that 4 CTAs fit per SM
    ALS_CUDA_TRY(cudaFuncSetAttribute(k_sweep_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    // One CTA per row (rows in degree-descending order): the hardware keeps as
    // many CTAs resident per SM as shared memory allows (at most 4 here), and
    // each one holds its TMEM columns only for the row it solves.
    const int64_t grid = std::min<int64_t>(a.nrows, (int64_t)INT32_MAX);
    k_sweep_tc<<<(unsigned)grid, TC_THREADS, smem, a.stream ? a.stream : c->stream>>>(a, ntc);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}
