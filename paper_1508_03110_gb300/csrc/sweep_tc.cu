// Mixed-precision half sweep with the Gram matrices on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// For each row i (one CTA of 4 warps per row, 5 CTAs per SM), with the fixed
// side F (FP32 factor rows):
//   1. gather: the row's ratings are taken 32 per chunk, a warp 8 of them;
//      each rating's factor row f is read once, into registers, and split
//      into hi = bf16(f) and lo = bf16(f - hi), stored into two
//      128-byte-swizzled, MN-major shared tiles H and L (rating k of the chunk
//      is K index k, the factor index is the M/N index); the same FP32 values
//      give the chunk's part of the first residual sum_e f_e (r_e - f_e . u0)
//      at the current row u0 = x_i;
//   2. Gram: one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//      M = 128, N = round_up(n_f, 16), K = 16 per instruction): D += H H^T,
//      D += H L^T and D += L H^T, so D = sum_e (hi hi^T + hi lo^T + lo hi^T)
//      accumulates in TMEM: the Gram matrix with ~2^-17 relative error (the
//      lo lo^T term is dropped), symmetric by construction.  Two stages:
//      while the MMAs of one chunk run, the next chunk's rows are read and
//      split; tcgen05.commit on an mbarrier releases a stage;
//   3. tcgen05.ld moves D's lower triangle into packed FP32 shared memory
//      (row m of D is TMEM lane m), A = D + lambda n_i I; the CTA then frees
//      its TMEM columns, which it holds only from the Gram to this read-out;
//   4. blocked Cholesky of A (inverted diagonal blocks) and the refinement of
//      the ALS solve from u0: u <- u + A^{-1} res, res = sum_e f_e (r_e -
//      f_e . u) - lambda n_i u in FP32 from the FP32 factors (the first
//      residual comes from step 1).
// With the launch shape chol_tc, steps 3-4 factor A in place in TMEM instead
// (chol_tmem: panels of 16 columns, trailing updates as tcgen05 MMAs), and the
// CTA holds its TMEM columns until the factorisation ends.
// With a.Gout the kernel also writes the row's gradient of Eq. (1) at the
// current factors, -2 v1 with v1 = r0 - lambda n_i x_i the first residual:
// the gradient pass then only forms the rows' FP64 terms.
// Every mbarrier wait is bounded (%globaltimer): on expiry the CTA gives each
// stage whose MMAs may still be in flight one more bounded wait, records a
// timeout, frees its TMEM and returns.  The rows of such a launch are not
// valid; the host reports the expiry once.
//
// Heavy rows (and split-row segments) take the prefetching variant (PF): the
// next chunk's factor rows are copied into a staging tile with cp.async
// while the current chunk is split, stored and multiplied, so the gather's L2
// latency is paid once per row rather than once per chunk.  The staging tile
// costs 12.8 KB of shared memory (n_f = 100), i.e. 4 CTAs per SM instead of 5.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "sweep_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_THREADS = 128;
// ratings per chunk: 32 for the heavy rows' variants, 16 for the rest (a
// smaller ring, so that more CTAs fit per SM); a tile (H or L) is KC x 128
// BF16 values, a stage H and L
__host__ __device__ constexpr int tile_bytes(int kc) { return kc * ALS_TC_LD * 2; }
__host__ __device__ constexpr int stage_bytes(int kc) { return 2 * tile_bytes(kc); }
constexpr int NSTAGE = 2;
constexpr uint32_t LBO = 1024;  // byte distance between the two 64-wide MN atoms
constexpr uint32_t SBO = 2048;  // byte distance between groups of 8 K rows
constexpr int TMEM_COLS = 128;
// the Cholesky's trailing-update operands: 128 rows x 16 BF16 K values,
// K-major without swizzle (core matrices of 8 rows x 16 bytes: the two K
// halves 128 bytes apart, groups of 8 rows 256 bytes apart)
constexpr int CH_TILE = 128 * 16 * 2;
constexpr uint32_t CH_LBO = 128;
constexpr uint32_t CH_SBO = 256;

// Variants of the gather (template PFM): 0 each lane loads its factor rows
// from global memory; 1 (prefetching) the next chunk's rows are copied into a
// staging tile with cp.async by the lanes that will read them; 2 (TMA) the
// rows of the chunk after next are gathered into one of two staging tiles by
// tile::gather4 TMA copies, issued by 8 lanes of warp 0, four rows each, and
// counted on the stage's mbarrier.
constexpr int NSTG = 1;   // TMA staging tiles (gathers run NSTG chunks ahead)

// bytes between two groups of four gathered rows in a TMA staging tile
// (each group's destination must be 128-byte aligned)
__host__ __device__ inline int tma_group_bytes(int ld) { return (4 * ld * 4 + 127) & ~127; }

struct TcLayout {
    int ring, A, ops, vec, mbar, holder, stg, total;
};

// mode 1: a staging tile of kc factor rows of ld floats; mode 2: NSTG TMA
// staging tiles of kc / 4 row groups; chol_tc: room for the TMEM
// factorisation's operand tiles after A
__host__ __device__ inline TcLayout tc_layout(int nf, int ld, int mode, int kc, int chol_tc) {
    TcLayout L;
    L.ring = 0;
    L.A = 0;  // the FP32 matrix reuses the gather ring once the MMAs are done
    int big = NSTAGE * stage_bytes(kc);
    const int a_bytes = nf * (nf + 1) / 2 * 4;  // packed lower triangle
    // then the Cholesky's operand tiles (BF16 hi and lo, 128 rows x 16 K)
    L.ops = (a_bytes + 127) & ~127;
    const int a_end = chol_tc ? L.ops + 2 * CH_TILE : a_bytes;
    if (a_end > big) big = a_end;
    big = (big + 15) & ~15;
    L.vec = big;  // colk, v1, v2, u, diag [5][128]; then part[4][128] / Cholesky work (aliased)
    L.mbar = L.vec + (5 * 128 + 1104) * 4;   // [0..1] MMA stages, [2..3] TMA staging tiles
    L.holder = L.mbar + 32;
    L.stg = L.holder + 16;
    if (mode == 2) L.stg = (L.stg + 127) & ~127;
    L.total = L.stg + (mode == 1 ? kc * ld * 4 : mode == 2 ? NSTG * (kc / 4) * tma_group_bytes(ld) : 0);
    return L;
}

// d[q] <- sum of d[q] over the warp for Q = 8 (warp_allsum8) or Q = 4 values:
// two halving exchanges leave each lane one value summed over 4 lanes, three
// more finish it over the warp, and 4 reads gather the totals
template <int Q>
__device__ __forceinline__ void warp_allsum_q(float (&d)[Q], int lane) {
    if constexpr (Q == 8) {
        warp_allsum8(d, lane);
    } else {
        static_assert(Q == 4, "chunks of 16 or 32 ratings");
        const bool b4 = lane & 16, b3 = lane & 8;
        float e2[2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
            e2[i] = (b4 ? d[i + 2] : d[i]) + __shfl_xor_sync(0xffffffffu, b4 ? d[i] : d[i + 2], 16);
        float e1 = (b3 ? e2[1] : e2[0]) + __shfl_xor_sync(0xffffffffu, b3 ? e2[0] : e2[1], 8);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 4);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = __shfl_sync(0xffffffffu, e1, ((q >> 1) & 1) * 16 + (q & 1) * 8);
    }
}

// Cholesky factorisation of A = D + lambda n I with the Gram matrix D in TMEM
// (row m in lane m, entry j in column j), right-looking by panels of 16
// columns; the trailing updates run on the tensor core:
//   1. every thread loads its row's 16 entries of the panel (tcgen05.ld) and
//      adds lambda n on the diagonal;
//   2. the warp holding the panel's 16 diagonal rows factors the 16 x 16
//      diagonal block in registers, one row per lane, exchanging the columns
//      of L by shuffles, and publishes L_kk: into packed A, transposed into
//      l11t, and 1 / L[k][k] into diag;
//   3. every row below the block forms its row of L21 = A21 L_kk^-T by
//      forward substitution, stores it into packed A and, split into BF16
//      hi + lo, into a K-major operand tile (zero rows elsewhere);
//   4. one thread issues D[:, c0 + 16 :] -= L21 L21^T as tcgen05.mma with A
//      negated, hi hi^T + hi lo^T + lo hi^T (lo lo^T dropped, as in the
//      Gram), committed to an mbarrier that the next panel waits on.
// So the O(n_f^3) part of the factorisation is three MMAs per panel, and
// no FP32 trailing update is left on the CUDA cores.  On return A's lower
// triangle holds L and diag[k] = 1 / L[k][k] (as chol_blocked128 leaves
// them); false (in every thread) on a non-positive pivot; bail set when a
// bounded wait ran out (the last panel's MMAs may still be in flight: the
// caller waits once more before freeing TMEM).  l11t: 257 floats of scratch.
__device__ __forceinline__ bool chol_tmem(uint32_t tmem, int nf, int ntc, float lam_n, float *A, float *diag, float *l11t,
                          uint32_t ops, uint32_t mbar, uint32_t &phase, uint64_t wait_ns, bool withhold, int t,
                          bool &bail) {
    const int warp = t >> 5, lane = t & 31;
    int *flag = reinterpret_cast<int *>(l11t + 256);
    const uint32_t rowoff = (uint32_t)(t >> 3) * CH_SBO + (uint32_t)(t & 7) * 16;
    for (int c0 = 0; c0 < nf; c0 += 16) {
        if (c0 > 0) {  // the previous panel's update has reached TMEM
            const bool w = mbar_wait_bounded(mbar, phase, wait_ns);
            if (__syncthreads_or(!w)) {
                bail = true;
                return false;
            }
            phase ^= 1u;
        }
        tc_fence_after();
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        const int li = t - c0;
        // rows and columns past n_f: the identity in the diagonal block, zero
        // elsewhere
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (t >= nf) v[j] = (li == j) ? 1.0f : 0.0f;
            else if (c0 + j >= nf) v[j] = 0.0f;
            else if (li == j) v[j] += lam_n;
        }
        if (warp == (c0 >> 5)) {
            const int base = c0 & 31;
            const bool inb = li >= 0 && li < 16;
            bool bad = false;
            float rdo = 1.0f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float pj = __shfl_sync(0xffffffffu, v[j], base + j);
                bad |= !(pj > 0.0f);
                const float rj = rsqrtf(pj);
                if (inb && li == j) {
                    v[j] = pj * rj;
                    rdo = rj;
                } else if (inb && li > j) {
                    v[j] *= rj;
                }
#pragma unroll
                for (int k = 1; k < 16; ++k) {
                    if (k <= j) continue;
                    const float lk = __shfl_sync(0xffffffffu, v[j], base + k);
                    if (inb && li >= k) v[k] = fmaf(-v[j], lk, v[k]);
                }
            }
            if (inb) {
                diag[t] = rdo;
                if (t < nf) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j <= li) A[tri_off(t) + c0 + j] = v[j];
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) l11t[j * 16 + li] = (j <= li) ? v[j] : 0.0f;
            }
            if (lane == base) *flag = bad ? 1 : 0;
        }
        __syncthreads();
        if (*flag) return false;
        // rows below the block: L21 = A21 L_kk^-T, column by column
        const bool below = li >= 16 && t < nf;
        float a[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            a[c] = below ? v[c] * diag[c0 + c] : 0.0f;
            const float4 *col = reinterpret_cast<const float4 *>(l11t + c * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (4 * q + 3 <= c) continue;
                const float4 w = col[q];
                if (4 * q > c) v[4 * q] = fmaf(-a[c], w.x, v[4 * q]);
                if (4 * q + 1 > c) v[4 * q + 1] = fmaf(-a[c], w.y, v[4 * q + 1]);
                if (4 * q + 2 > c) v[4 * q + 2] = fmaf(-a[c], w.z, v[4 * q + 2]);
                v[4 * q + 3] = fmaf(-a[c], w.w, v[4 * q + 3]);
            }
        }
        if (below) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c0 + c < nf) A[tri_off(t) + c0 + c] = a[c];
        }
        uint32_t hw[8], lw[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(a[2 * i], a[2 * i + 1]);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(a[2 * i] - hf.x, a[2 * i + 1] - hf.y);
            hw[i] = *reinterpret_cast<const uint32_t *>(&h);
            lw[i] = *reinterpret_cast<const uint32_t *>(&l);
        }
        st_shared_v4(ops + rowoff, hw[0], hw[1], hw[2], hw[3]);
        st_shared_v4(ops + rowoff + CH_LBO, hw[4], hw[5], hw[6], hw[7]);
        st_shared_v4(ops + CH_TILE + rowoff, lw[0], lw[1], lw[2], lw[3]);
        st_shared_v4(ops + CH_TILE + rowoff + CH_LBO, lw[4], lw[5], lw[6], lw[7]);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        const int ncol = ntc - c0 - 16;  // trailing columns (a multiple of 16)
        if (ncol > 0 && t == 0 && !withhold) {
            tc_fence_after();
            const uint32_t id = idesc_bf16_f32_k_nega((uint32_t)ncol);
            const uint32_t boff = (uint32_t)((c0 + 16) >> 3) * CH_SBO;
            const uint64_t ah = smem_desc_noswz(ops, CH_LBO, CH_SBO);
            const uint64_t al = smem_desc_noswz(ops + CH_TILE, CH_LBO, CH_SBO);
            const uint64_t bh = smem_desc_noswz(ops + boff, CH_LBO, CH_SBO);
            const uint64_t bl = smem_desc_noswz(ops + CH_TILE + boff, CH_LBO, CH_SBO);
            const uint32_t dcol = tmem + (uint32_t)(c0 + 16);
            tc_mma_bf16(dcol, ah, bh, id, 1u);
            tc_mma_bf16(dcol, ah, bl, id, 1u);
            tc_mma_bf16(dcol, al, bh, id, 1u);
            tc_commit(mbar);
        }
    }
    return true;
}

// resident CTAs per SM the register budget is set for
__host__ __device__ constexpr int tc_min_blocks(int pfm, int kc) {
    return pfm == 2 ? (NSTG == 1 ? 4 : 3) : (pfm == 1 ? 4 : (kc == 16 ? 7 : 5));
}

// CT: the factorisation in TMEM (launch shape chol_tc); a template parameter
// so that each kernel carries only the code of its own factorisation
template <int PFM, int KC, int CT>
__global__ void __launch_bounds__(TC_THREADS, tc_min_blocks(PFM, KC))
    k_sweep_tc(SweepArgs a, int ntc, const __grid_constant__ CUtensorMap tmap) {
    constexpr bool PF = PFM == 1;
    constexpr bool TM = PFM == 2;
    constexpr int KCH = KC;
    constexpr int Q = KC / 4;                 // ratings of a chunk per warp
    constexpr int TILE_BYTES = tile_bytes(KC);
    constexpr int STAGE_BYTES = stage_bytes(KC);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char *base = smem_raw + pad;
    const uint32_t sbase = raw + pad;
    const int nf = a.nf;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const TcLayout L = tc_layout(nf, a.ld, PFM, KC, CT);
    float *A = reinterpret_cast<float *>(base + L.A);
    const float *stg = reinterpret_cast<const float *>(base + L.stg);
    float *vec = reinterpret_cast<float *>(base + L.vec);
    float *colk = vec, *v1 = vec + 128, *v2 = vec + 256, *u = vec + 384, *diag = vec + 512;
    float *part = vec + 640;   // residual partials (residual phase)
    float *work = vec + 640;   // Cholesky panel scratch (factorisation phase)
    const uint32_t mbar[2] = {sbase + L.mbar, sbase + L.mbar + 8};
    const uint32_t sbar[2] = {sbase + L.mbar + 16, sbase + L.mbar + 24};   // TMA staging tiles (NSTG used)
    uint32_t *holder = reinterpret_cast<uint32_t *>(base + L.holder);
    const int gsf = tma_group_bytes(a.ld) / 4;           // floats between row groups (TMA tiles)
    const int stgf = (KCH / 4) * gsf;                    // floats per TMA staging tile

    if (t == 0) {
        mbar_init(mbar[0], 1);
        mbar_init(mbar[1], 1);
        if constexpr (TM) {
            mbar_init(sbar[0], 1);
            if (NSTG > 1) mbar_init(sbar[1], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t tmem = 0;
    bool held = false;  // TMEM columns are held only from a row's Gram to its read-out
    const uint32_t idesc = idesc_bf16_f32_mn((uint32_t)ntc);
    const float *F = reinterpret_cast<const float *>(a.F);
    uint32_t phase[2] = {0u, 0u};
    uint32_t sphase = 0u;   // TMA staging tiles: parity of the next completion (bit s: tile s)
    uint32_t spend = 0u;    // ... and whether a gather into it is in flight (bit s)
    bool bail = false;

    for (int64_t r = blockIdx.x; r < a.nrows; r += gridDim.x) {  // one row per CTA (grid = rows)
        const bool seg = a.seg_out != nullptr;  // a slice of a split row: partials only
        const int64_t row = seg ? a.order[a.seg_row[r]] : (a.order ? a.order[r] : r);
        const int64_t beg = seg ? a.seg_beg[r] : a.ptr[row];
        const int n = seg ? a.seg_len[r] : (int)(a.ptr[row + 1] - beg);
        const float *xi = a.Xin ? reinterpret_cast<const float *>(a.Xin) + row * a.ld : nullptr;
        float *xo = reinterpret_cast<float *>(a.Xout) + row * a.ld;
        float *gb = a.Gbar ? reinterpret_cast<float *>(a.Gbar) + row * a.ld : nullptr;
        // the row's gradient g_i = 2 lambda n_i x_i - 2 r0 = -2 v1, v1 the first
        // residual below (whole rows only: a segment's is a partial)
        float *go = (a.Gout && !seg) ? reinterpret_cast<float *>(a.Gout) + row * a.ld : nullptr;
        const float lam_n = (float)(a.lambda * (double)n);
        bool ok = n > 0;
        // current row u0 = x_i (fold-in: 0), one 4-wide slot per lane
        const bool act = 4 * lane < a.ld;
        float uu[4], acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) uu[i] = (xi && 4 * lane + i < nf) ? xi[4 * lane + i] : 0.0f;
        for (int k = t; k < nf; k += TC_THREADS) u[k] = xi ? xi[k] : 0.0f;
        if (ok) {
            // TMEM for this row's accumulator (5 CTAs share an SM's 512 columns:
            // if none are free the allocation waits for a CTA that is past its
            // read-out, which every CTA reaches after bounded waits)
            if (warp == 0) tmem_alloc(sbase + L.holder, TMEM_COLS);
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            tmem = *holder;
            held = true;
            // ---- 1-2. gather + tensor-core Gram, with the first FP32 residual
            //      r0 = sum_e f_e (r_e - f_e . u0) of the chunk's ratings computed
            //      while the chunk's copies and MMAs are in flight -------------
            const int nch = (n + KCH - 1) / KCH;
            int pend[2] = {0, 0};
            // ids and ratings of this warp's ratings k = warp + 4 q (q < Q) of
            // the next chunk, fetched one chunk ahead (PF: two ahead, the next
            // chunk's rows being copied already)
            int32_t nj[Q], nnj[Q];
            float nr[Q], nnr[Q];
            auto fetch = [&](int ch, int32_t (&oj)[Q], float (&orr)[Q]) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int64_t e = beg + (int64_t)ch * KCH + warp + 4 * q;
                    const bool in = ch < nch && e < beg + n;
                    // TMA: the rows arrive by id in the staging tile; only
                    // whether the rating exists matters here
                    oj[q] = in ? (TM ? 0 : a.idx[e]) : -1;
                    orr[q] = in ? a.val[e] : 0.0f;
                }
            };
            // TMA: gather chunk ch's factor rows into staging tile sg (warp 0:
            // lane g < 8 copies rows 4 g .. 4 g + 3; past the row's end, row 0
            // stands in, in bounds and unused)
            // the ids of the four rows lane g < 8 of warp 0 gathers for chunk ch
            auto tma_ids = [&](int ch, int32_t (&y)[4]) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t e = beg + (int64_t)ch * KCH + 4 * lane + i;
                    y[i] = (warp == 0 && lane < KCH / 4 && ch < nch && e < beg + n) ? a.idx[e] : 0;
                }
            };
            int32_t ty[4];   // TMA: ids of the next chunk to gather, loaded a chunk early
            auto tma_chunk = [&](int ch, int sg, const int32_t (&y)[4]) {
                if (warp == 0) {
                    const uint32_t bar = sg ? sbar[1] : sbar[0];
                    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(KCH * a.ld * 4));
                    __syncwarp();
                    if (lane < KCH / 4) {
                        fence_proxy_async_smem();
                        tma_gather4(sbase + (uint32_t)L.stg + (uint32_t)((sg * stgf + lane * gsf) * 4), &tmap, 0,
                                    y[0], y[1], y[2], y[3], bar);
                    }
                }
                spend |= 1u << sg;
            };
            // PF: copy the factor rows of ids jj into the staging tile (row k =
            // warp + 4 q, this lane's 16 bytes: the lane later reads only those)
            auto stage_rows = [&](const int32_t (&jj)[Q]) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    if (jj[q] >= 0 && act)
                        cp_async16(sbase + (uint32_t)L.stg + (uint32_t)(((warp + 4 * q) * a.ld + 4 * lane) * 4),
                                   F + (int64_t)jj[q] * a.ld + 4 * lane);
                cp_async_commit();
            };
            fetch(0, nj, nr);
            if constexpr (PF) {
                stage_rows(nj);
                fetch(1, nnj, nnr);
            }
            if constexpr (TM) {
                for (int c0 = 0; c0 < NSTG && c0 < nch; ++c0) {
                    tma_ids(c0, ty);
                    tma_chunk(c0, c0, ty);
                }
            }
            for (int ch = 0; ch < nch; ++ch) {
                const int st = ch & 1;
                bool swait = true;   // TMA: this chunk's rows arrived in time
                const int sg = ch % NSTG;   // TMA: this chunk's staging tile
                if constexpr (TM) tma_ids(ch + NSTG, ty);   // in flight while this chunk is split
                // the MMAs of chunk ch-2 read stage st: each thread waits for
                // them before it writes its part of the stage (no CTA barrier
                // here; a wait that ran out is noticed at the chunk's barrier
                // and its thread writes nothing)
                bool sok = true;
                if (pend[st]) {
                    sok = mbar_wait_bounded(mbar[st], phase[st], a.wait_ns);
                    if (sok) {
                        phase[st] ^= 1u;
                        pend[st] = 0;
                    }
                }
                int32_t cj[Q];
                float cr[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    cj[q] = nj[q];
                    cr[q] = nr[q];
                }
                if constexpr (PF) {
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        nj[q] = nnj[q];
                        nr[q] = nnr[q];
                    }
                    fetch(ch + 2, nnj, nnr);
                } else {
                    fetch(ch + 1, nj, nr);
                }
                // each factor row is read once, in FP32: it feeds the residual
                // at u0 and, split into BF16 hi + lo, the operand tiles of stage st
                {
                    float f[Q][4];
                    if constexpr (PF) cp_async_wait_all();  // this lane's copies of chunk ch
                    if constexpr (TM) {
                        swait = mbar_wait_bounded(sg ? sbar[1] : sbar[0], (sphase >> sg) & 1u, a.wait_ns);
                        sphase ^= 1u << sg;
                        spend &= ~(1u << sg);
                    }
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        if (cj[q] >= 0 && act) {
                            const int k = warp + 4 * q;
                            if constexpr (PF) ld4f(stg + k * a.ld + 4 * lane, f[q]);
                            else if constexpr (TM) ld4f(stg + sg * stgf + (k >> 2) * gsf + (k & 3) * a.ld + 4 * lane, f[q]);
                            else ld4f(F + (int64_t)cj[q] * a.ld + 4 * lane, f[q]);
                        } else {
                            f[q][0] = f[q][1] = f[q][2] = f[q][3] = 0.0f;
                        }
                    }
                    float d[Q];
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        d[q] = uu[0] * f[q][0];
#pragma unroll
                        for (int i = 1; i < 4; ++i) d[q] = fmaf(uu[i], f[q][i], d[q]);
                    }
                    // PF: the staged rows are in registers now (the dot products
                    // used them all): the next chunk's copies may overwrite them
                    if constexpr (PF)
                        if (ch + 1 < nch) stage_rows(nj);
                    warp_allsum_q(d, lane);
                    {
                        // the chunk's Q terms in plain FP32, then one compensated
                        // add into the row's running sum
                        float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                        for (int q = 0; q < Q; ++q) {
                            const float er = cj[q] >= 0 ? cr[q] - d[q] : 0.0f;
#pragma unroll
                            for (int i = 0; i < 4; ++i) cs[i] = fmaf(er, f[q][i], cs[i]);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) kadd(acc[i], cmp[i], cs[i]);
                    }
                    if (act && sok) {
                        const uint32_t stage = sbase + L.ring + st * STAGE_BYTES;
#pragma unroll
                        for (int q = 0; q < Q; ++q) {
                            const int k = warp + 4 * q;   // K index (rating within the chunk)
                            const int qq = lane >> 1;     // 16-byte column chunk: factors 8 qq .. 8 qq + 7
                            const uint32_t off = (uint32_t)(k >> 3) * SBO + (uint32_t)(qq >> 3) * LBO +
                                                 (uint32_t)(k & 7) * 128 + ((uint32_t)((qq & 7) ^ (k & 7)) << 4) +
                                                 (uint32_t)(lane & 1) * 8;
                            uint32_t hw[2], lw[2];
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const __nv_bfloat162 h = __floats2bfloat162_rn(f[q][2 * i], f[q][2 * i + 1]);
                                const float2 hf = __bfloat1622float2(h);
                                const __nv_bfloat162 l =
                                    __floats2bfloat162_rn(f[q][2 * i] - hf.x, f[q][2 * i + 1] - hf.y);
                                hw[i] = *reinterpret_cast<const uint32_t *>(&h);
                                lw[i] = *reinterpret_cast<const uint32_t *>(&l);
                            }
                            st_shared_v2(stage + off, hw[0], hw[1]);
                            st_shared_v2(stage + TILE_BYTES + off, lw[0], lw[1]);
                        }
                    }
                }
                fence_proxy_async_smem();
                // every thread has read staging tile st and written stage st;
                // a wait that ran out is noticed by all
                if (__syncthreads_or(!swait || !sok)) { bail = true; break; }
                if (t == 0 && !a.withhold) {
                    tc_fence_after();
                    const uint32_t stage = sbase + L.ring + st * STAGE_BYTES;
#pragma unroll
                    for (int s = 0; s < KCH / 16; ++s) {
                        const uint64_t dh = smem_desc_sw128(stage + (uint32_t)s * 2u * SBO, LBO, SBO);
                        const uint64_t dl = smem_desc_sw128(stage + TILE_BYTES + (uint32_t)s * 2u * SBO, LBO, SBO);
                        tc_mma_bf16(tmem, dh, dh, idesc, (ch > 0 || s > 0) ? 1u : 0u);
                        tc_mma_bf16(tmem, dh, dl, idesc, 1u);
                        tc_mma_bf16(tmem, dl, dh, idesc, 1u);
                    }
                    tc_commit(mbar[st]);
                }
                pend[st] = 1;
                // staging tile sg is free (every thread read it before the
                // barrier): the rows of chunk ch + NSTG go there
                if constexpr (TM)
                    if (ch + NSTG < nch) tma_chunk(ch + NSTG, sg, ty);
            }
            if constexpr (PF) cp_async_wait_all();  // nothing in flight past the gather
            if (!bail) {
                for (int s = 0; s < 2; ++s) {
                    if (pend[s]) {
                        const bool w = mbar_wait_bounded(mbar[s], phase[s], a.wait_ns);
                        if (__syncthreads_or(!w)) { bail = true; break; }
                        phase[s] ^= 1u;
                        pend[s] = 0;
                    }
                }
            }
            if (bail) {
                // a wait ran out: the MMAs of a stage may still be reading this
                // CTA's shared tiles and writing its TMEM, so every stage still
                // pending gets one more bounded wait before the teardown frees
                // the columns (the self-test issued none: nothing to wait for)
                if (t == 0 && !a.withhold)
                    for (int s = 0; s < 2; ++s)
                        if (pend[s]) (void)mbar_wait_bounded(mbar[s], phase[s], a.wait_ns);
                // TMA gathers still in flight write this CTA's staging tiles
                if (t == 0)
                    for (int s = 0; s < NSTG; ++s)
                        if ((spend >> s) & 1u) (void)mbar_wait_bounded(sbar[s], (sphase >> s) & 1u, a.wait_ns);
                __syncthreads();
                break;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) part[warp * 128 + 4 * lane + i] = acc[i] - cmp[i];
            tc_fence_after();
            // TMEM -> FP32 A, D's lower triangle packed (row m of D is TMEM
            // lane m), then TMEM is returned
            auto read_out = [&]() {
                const int m = 32 * warp + lane;
                for (int c0 = 0; c0 < ntc; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
                    if (m < nf) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int col = c0 + i;
                            if (col <= m) A[tri_off(m) + col] = v[i];
                        }
                    }
                }
                tc_fence_before();
                __syncthreads();
                if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);  // read out: another CTA may take it
                held = false;
            };
            if (seg) {
                // ---- 3. a slice of a split row: its Gram partial, packed as A
                //      is, then its residual at u0 --------------------------------
                read_out();
                float *po = reinterpret_cast<float *>(a.seg_out) + r * a.seg_stride;
                const int tri = nf * (nf + 1) / 2;
                for (int e = t; e < tri; e += TC_THREADS) po[e] = A[e];
                if (t < nf) po[tri + t] = (part[t] + part[128 + t]) + (part[256 + t] + part[384 + t]);
                __syncthreads();
                continue;
            }
            if constexpr (CT) {
                // the first residual v1 = r0 - lambda n u0 (fixed order over
                // the warps)
                __syncthreads();
                if (t < nf) v1[t] = ((part[t] + part[128 + t]) + (part[256 + t] + part[384 + t])) - lam_n * u[t];
                if (go && t < a.ld) go[t] = t < nf ? -2.0f * v1[t] : 0.0f;
                // ---- 3-4. Cholesky of A = D + lambda n I from TMEM, trailing
                //      updates on the tensor core --------------------------------
                ok = chol_tmem(tmem, nf, ntc, lam_n, A, diag, work + 512, sbase + (uint32_t)L.ops, mbar[0],
                               phase[0], a.wait_ns, a.withhold, t, bail);
                if (bail) {
                    // the last panel's MMAs may still write this CTA's TMEM
                    if (t == 0 && !a.withhold) (void)mbar_wait_bounded(mbar[0], phase[0], a.wait_ns);
                    __syncthreads();
                    break;
                }
                tc_fence_before();
                __syncthreads();
                if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);  // factored: another CTA may take it
                held = false;
            } else {
                // ---- 3. TMEM -> FP32 A; A = D + lambda n I, the first residual
                //      v1 = r0 - lambda n u0 (fixed order over the warps) --------
                read_out();
                if (t < nf) {
                    A[tri_off(t) + t] += lam_n;
                    v1[t] = ((part[t] + part[128 + t]) + (part[256 + t] + part[384 + t])) - lam_n * u[t];
                }
                if (go && t < a.ld) go[t] = t < nf ? -2.0f * v1[t] : 0.0f;
                __syncthreads();
                // ---- 4. blocked Cholesky of A in shared memory ---------------
                ok = chol_blocked128(A, nf, diag, work, t, 32 * (int)(blockIdx.x & 3));
            }
            if (ok) invert_diag_blocks128(A, nf, diag, t);
            if (!ok && t == 0) atomicAdd(a.notspd, 1);
        }
        if (ok) {
            trisolve_inv128(A, nf, v1, v2, colk, t);
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
                trisolve_inv128(A, nf, v1, v2, colk, t);
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
            if (go && n <= 0) go[k] = 0.0f;  // no ratings: the gradient row is 0
        }
        __syncthreads();
    }
    // ---- teardown: TMEM returned ----------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (held && warp == 0) tmem_dealloc(tmem, TMEM_COLS);
    if (bail && t == 0) atomicAdd(a.timeout, 1);
}

// tensor map of the fixed side F for the TMA gathers: nF rows of ld FP32
// values, one row per box (tile::gather4 takes four of them)
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

als_status fixed_side_map(const SweepArgs &a, CUtensorMap *m) {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    });
    if (!g_encode) {
        als_set_error("sweep: cuTensorMapEncodeTiled is not available");
        return ALS_ENOTSUP;
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)a.ld, (cuuint64_t)a.nF};
    const cuuint64_t gstride[1] = {(cuuint64_t)a.ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)a.ld, 1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(a.F), gdim, gstride, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        als_set_error("sweep: cuTensorMapEncodeTiled failed for the fixed side");
        return ALS_ECUDA;
    }
    return ALS_OK;
}

template <int PFM, int KC, int CT>
als_status launch_tc_ct(als_ctx *c, const SweepArgs &a, int ntc) {
    if (a.nrows <= 0) return ALS_OK;
    const TcLayout L = tc_layout(a.nf, a.ld, PFM, KC, CT);
    // ~40 KB of shared memory per CTA (n_f = 100): 5 CTAs per SM; cp.async
    // prefetching ~54 KB: 4; TMA-fed ~67 KB: 3
    size_t smem = (size_t)L.total + 1024;
    if (raise_smem_limit((const void *)k_sweep_tc<PFM, KC, CT>, smem) != ALS_OK) return ALS_ECUDA;
    // the whole L1/shared array as shared memory, so that 5-7 CTAs fit per SM
    ALS_CUDA_TRY(cudaFuncSetAttribute(k_sweep_tc<PFM, KC, CT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    if (PFM == 2) {
        als_status s = fixed_side_map(a, &tm);
        if (s != ALS_OK) return s;
    }
    // One CTA per row (rows in degree-descending order): the hardware keeps as
    // many CTAs resident per SM as shared memory and registers allow, and
    // each holds its 128 TMEM columns only from its Gram to the read-out.
    // Exactly one row per CTA: a CTA allocates TMEM once (the allocation
    // relinquishes the CTA's permit to allocate again).
    if (a.nrows > (int64_t)INT32_MAX) {
        als_set_error("sweep: more rows than CTAs in one launch");
        return ALS_ENOTSUP;
    }
    cudaStream_t st = a.stream ? a.stream : c->stream;
    const int cls = a.seg_out ? KT_TC_SEG : (PFM ? KT_TC_PF : KT_TC);
    kt_begin(c, cls, st);
    k_sweep_tc<PFM, KC, CT><<<(unsigned)a.nrows, TC_THREADS, smem, st>>>(a, ntc, tm);
    kt_end(c, cls, st);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

// segments factor nothing: always the kernel without the TMEM factorisation
template <int PFM, int KC>
als_status launch_tc(als_ctx *c, const SweepArgs &a, int ntc) {
    return (c->chol_tc && !a.seg_out) ? launch_tc_ct<PFM, KC, 1>(c, a, ntc) : launch_tc_ct<PFM, KC, 0>(c, a, ntc);
}

}  // namespace

als_status launch_sweep_tc(als_ctx *c, const SweepArgs &a) {
    if (a.nrows <= 0) return ALS_OK;
    if (a.nf > ALS_TC_LD) {
        als_set_error("sweep: the tensor-core Gram supports n_f <= 128");
        return ALS_ENOTSUP;
    }
    const int ntc = (a.nf + 15) / 16 * 16;
    // split-row segments are long: all prefetching; otherwise the first npf
    // rows of the order (the heaviest), then the rest
    // the heavy rows' gather: TMA-fed when the context asks for it and the
    // fixed side's extent is known, else cp.async
    const bool tma = c->gather_tma && a.nF > 0;
    if (a.seg_out) return tma ? launch_tc<2, 32>(c, a, ntc) : launch_tc<1, 32>(c, a, ntc);
    const int64_t npf = a.order ? std::max<int64_t>(0, std::min(a.npf, a.nrows)) : 0;
    if (npf > 0) {
        SweepArgs h = a;
        h.nrows = npf;
        als_status s = tma ? launch_tc<2, 32>(c, h, ntc) : launch_tc<1, 32>(c, h, ntc);
        if (s != ALS_OK) return s;
    }
    SweepArgs l = a;
    l.order = a.order ? a.order + npf : nullptr;
    l.nrows = a.nrows - npf;
    // the other rows: 32-rating chunks (5 CTAs per SM), or 16 (a 16 KB ring,
    // 7 CTAs per SM: measured 5% slower at ML20M size, kept as a launch shape)
    return c->tc_chunk16 ? launch_tc<0, 16>(c, l, ntc) : launch_tc<0, 32>(c, l, ntc);
}
