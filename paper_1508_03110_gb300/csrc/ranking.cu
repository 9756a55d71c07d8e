// Ranking accuracy of the top-t recommendations (§IV, the modified
// Kendall-tau metric of the serial experiments).
//
// For user i the predicted ratings of all items are the scores s_j = u_i . m_j
// (one row of U^T M); a ranking lists the items by descending score, ties by
// ascending item id (a strict total order, "j precedes l").
//   * als_rank_topt: the first t items of each user's ranking (the reference
//     ranking p1 is taken from a converged solution).
//   * als_rank_accuracy: for each user, the swaps s_i that move the reference
//     top-t items a_0 .. a_{t-1} one after the other to the front of the
//     current ranking p2; the k-th move costs the number of items still ahead
//     of a_k that are not among a_0 .. a_{k-1}:
//       s_i = sum_k [ pos2(a_k) - #{l < k : pos2(a_l) < pos2(a_k)} ],
//     pos2(a) = #{j : j precedes a in p2}; q_i = 1 - s_i / s_max with
//     s_max = t (2 n_m - t - 1) / 2, and the mean of q_i over the users.
//
// Both kernels are tiles of the dense product U^T M: a CTA of 256 threads
// owns 32 users (their factor rows in shared memory) and walks all items in
// tiles of 128 (their rows staged in shared memory, padded to a bank-conflict
// free stride); each thread forms 4 x 4 scores in registers with FMAs in the
// factor order, so a score is the same number in every kernel that forms it.
//   * counting: the reference items' own scores, sorted once per user, are
//     the bin edges; each tile score finds its bin by binary search and adds
//     one to a shared histogram, whose prefix sums are the positions pos2;
//   * selection: the tile's scores go to shared memory and each warp merges
//     its users' candidates into their running top-t lists (only candidates
//     that beat the list's last entry are inserted).
// Integer counts only: the results are exact for the scores as formed, and
// bit-reproducible.
#include <cfloat>

#include "internal.cuh"

namespace {

constexpr int RK_USERS = 32;
constexpr int RK_ITEMS = 128;
constexpr int RK_THREADS = 256;
constexpr int RK_TMAX = 64;

template <typename T>
struct RankArgs {
    const T *U;          // n_u rows of ld
    const T *M;          // n_m rows of ld
    int64_t n_u, n_m;
    int nf, ld, t;
    const int32_t *top_ref;  // counting: n_u x t reference item ids
    int32_t *top_out;        // selection: n_u x t item ids
    double *q_out;           // counting: q_i per user
};

// (score, id) precedence of the rankings: higher score first, then lower id
template <typename T>
__device__ __forceinline__ bool precedes(T sa, int32_t ia, T sb, int32_t ib) {
    return sa > sb || (sa == sb && ia < ib);
}

template <typename T>
struct RankSmem {
    int ldm, nfp;
    size_t u, m, extra, total;
};

template <typename T>
__host__ __device__ inline RankSmem<T> rank_smem(int nf, int t, bool select) {
    RankSmem<T> L;
    L.nfp = nf;
    L.ldm = nf + 1;
    L.u = 0;
    L.m = L.u + (size_t)RK_USERS * nf * sizeof(T);
    L.m = (L.m + 15) & ~(size_t)15;
    L.extra = L.m + (size_t)RK_ITEMS * L.ldm * sizeof(T);
    L.extra = (L.extra + 15) & ~(size_t)15;
    if (select)  // tile scores + the users' lists (score, id)
        L.total = L.extra + (size_t)RK_USERS * RK_ITEMS * sizeof(T) + (size_t)RK_USERS * t * (sizeof(T) + 4);
    else         // sorted edges (score, id, k), histograms
        L.total = L.extra + (size_t)RK_USERS * t * (sizeof(T) + 8) + (size_t)RK_USERS * (t + 1) * 4;
    return L;
}

// stage the users' rows (zero past n_u) and the scores of one tile of items
template <typename T>
__device__ __forceinline__ void load_users(const RankArgs<T> &a, T *sU, int64_t u0) {
    for (int e = threadIdx.x; e < RK_USERS * a.nf; e += RK_THREADS) {
        const int r = e / a.nf, k = e - r * a.nf;
        const int64_t u = u0 + r;
        sU[r * a.nf + k] = u < a.n_u ? a.U[u * a.ld + k] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void load_items(const RankArgs<T> &a, T *sM, int ldm, int64_t j0) {
    for (int e = threadIdx.x; e < RK_ITEMS * a.nf; e += RK_THREADS) {
        const int r = e / a.nf, k = e - r * a.nf;
        const int64_t j = j0 + r;
        sM[r * ldm + k] = j < a.n_m ? a.M[j * a.ld + k] : T(0);
    }
}

// scores of users ty + 8 b (b < 4) and items tx + 32 c (c < 4) of the tile
template <typename T>
__device__ __forceinline__ void tile_scores(const T *sU, const T *sM, int nf, int ldm, int tx, int ty,
                                            T (&s)[4][4]) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) s[b][c] = T(0);
    for (int k = 0; k < nf; ++k) {
        T uv[4], mv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) uv[b] = sU[(ty + 8 * b) * nf + k];
#pragma unroll
        for (int c = 0; c < 4; ++c) mv[c] = sM[(tx + 32 * c) * ldm + k];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) s[b][c] = fma(uv[b], mv[c], s[b][c]);
    }
}

// one score the same way (factor order, FMA from zero)
template <typename T>
__device__ __forceinline__ T one_score(const T *u, const T *m, int nf) {
    T s = T(0);
    for (int k = 0; k < nf; ++k) s = fma(u[k], m[k], s);
    return s;
}

template <typename T>
__global__ void __launch_bounds__(RK_THREADS) k_rank_count(RankArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RankSmem<T> L = rank_smem<T>(a.nf, a.t, false);
    T *sU = reinterpret_cast<T *>(smem + L.u);
    T *sM = reinterpret_cast<T *>(smem + L.m);
    T *eS = reinterpret_cast<T *>(smem + L.extra);                      // [32][t] edge scores
    int32_t *eI = reinterpret_cast<int32_t *>(eS + RK_USERS * a.t);     // [32][t] edge ids
    int32_t *eK = eI + RK_USERS * a.t;                                  // [32][t] reference index k
    int32_t *hist = eK + RK_USERS * a.t;                                // [32][t + 1]
    const int t = a.t, tx = threadIdx.x & 31, ty = threadIdx.x >> 5, warp = ty, lane = tx;
    const int64_t u0 = (int64_t)blockIdx.x * RK_USERS;
    load_users(a, sU, u0);
    for (int e = threadIdx.x; e < RK_USERS * (t + 1); e += RK_THREADS) hist[e] = 0;
    __syncthreads();
    // edges: each reference item's own score, sorted by precedence (a warp per
    // user: lane k holds entries k and k + 32; its rank is the number of
    // entries that precede it)
    for (int r = warp; r < RK_USERS; r += RK_THREADS / 32) {
        const int64_t u = u0 + r;
        T sc[2];
        int32_t id[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            sc[h] = T(0);
            id[h] = -1;
            if (u < a.n_u && k < t) {
                id[h] = a.top_ref[u * t + k];
                sc[h] = one_score(sU + r * a.nf, a.M + (int64_t)id[h] * a.ld, a.nf);
            }
        }
        int rank[2] = {0, 0};
        for (int l = 0; l < t; ++l) {
            const T ls = __shfl_sync(0xffffffffu, sc[l >> 5], l & 31);
            const int32_t li = __shfl_sync(0xffffffffu, id[l >> 5], l & 31);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < t && precedes(ls, li, sc[h], id[h])) ++rank[h];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k < t) {
                eS[r * t + rank[h]] = sc[h];
                eI[r * t + rank[h]] = id[h];
                eK[r * t + rank[h]] = k;
            }
        }
    }
    __syncthreads();
    for (int64_t j0 = 0; j0 < a.n_m; j0 += RK_ITEMS) {
        load_items(a, sM, L.ldm, j0);
        __syncthreads();
        T s[4][4];
        tile_scores(sU, sM, a.nf, L.ldm, tx, ty, s);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = ty + 8 * b;
            const T *es = eS + r * t;
            const int32_t *ei = eI + r * t;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int32_t j = (int32_t)(j0 + tx + 32 * c);
                if (j >= a.n_m) continue;
                // m* = entries that precede (s, j); an item that is itself an
                // edge precedes only the edges after it
                int lo = 0, hi = t;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (precedes(es[mid], ei[mid], s[b][c], j)) lo = mid + 1;
                    else hi = mid;
                }
                const int bin = lo + ((lo < t && es[lo] == s[b][c] && ei[lo] == j) ? 1 : 0);
                atomicAdd(&hist[r * (t + 1) + bin], 1);
            }
        }
        __syncthreads();
    }
    // pos2 of edge m = items that precede it = sum of bins 0..m; then the
    // swaps in the reference order (a warp per user)
    for (int r = warp; r < RK_USERS; r += RK_THREADS / 32) {
        const int64_t u = u0 + r;
        if (u >= a.n_u) continue;
        int pos[2] = {0, 0}, ref[2] = {-1, -1};
        int run = 0;
        for (int m = 0; m < t; ++m) {
            run += hist[r * (t + 1) + m];
            if (m == lane) { pos[0] = run; ref[0] = eK[r * t + m]; }
            if (m == lane + 32) { pos[1] = run; ref[1] = eK[r * t + m]; }
        }
        long long sw = 0;
        for (int l = 0; l < t; ++l) {
            const int lp = __shfl_sync(0xffffffffu, pos[l >> 5], l & 31);
            const int lk = __shfl_sync(0xffffffffu, ref[l >> 5], l & 31);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (lane + 32 * h >= t) continue;
                if (l == lane + 32 * h) sw += pos[h];                // pos2(a_k)
                else if (lk < ref[h] && lp < pos[h]) sw -= 1;        // a_l, l < k, ahead of a_k
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, o);
        if (lane == 0) {
            const double smax = 0.5 * (double)t * (2.0 * (double)a.n_m - (double)t - 1.0);
            a.q_out[u] = smax > 0.0 ? 1.0 - (double)sw / smax : 1.0;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RK_THREADS) k_rank_topt(RankArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RankSmem<T> L = rank_smem<T>(a.nf, a.t, true);
    T *sU = reinterpret_cast<T *>(smem + L.u);
    T *sM = reinterpret_cast<T *>(smem + L.m);
    T *sS = reinterpret_cast<T *>(smem + L.extra);                      // [32][128] tile scores
    T *lS = sS + RK_USERS * RK_ITEMS;                                   // [32][t] list scores
    int32_t *lI = reinterpret_cast<int32_t *>(lS + RK_USERS * a.t);    // [32][t] list ids
    const int t = a.t, tx = threadIdx.x & 31, ty = threadIdx.x >> 5, warp = ty, lane = tx;
    const int64_t u0 = (int64_t)blockIdx.x * RK_USERS;
    load_users(a, sU, u0);
    for (int e = threadIdx.x; e < RK_USERS * t; e += RK_THREADS) {
        lS[e] = -(T)INFINITY;
        lI[e] = INT32_MAX;   // every real (score, id) precedes this sentinel
    }
    __syncthreads();
    for (int64_t j0 = 0; j0 < a.n_m; j0 += RK_ITEMS) {
        load_items(a, sM, L.ldm, j0);
        __syncthreads();
        T s[4][4];
        tile_scores(sU, sM, a.nf, L.ldm, tx, ty, s);
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) sS[(ty + 8 * b) * RK_ITEMS + tx + 32 * c] = s[b][c];
        __syncthreads();
        // merge: warp w owns users w, w + 8, w + 16, w + 24
        for (int r = warp; r < RK_USERS; r += RK_THREADS / 32) {
            T *ls = lS + r * t;
            int32_t *li = lI + r * t;
            for (int c = 0; c < RK_ITEMS / 32; ++c) {
                const int32_t j = (int32_t)(j0 + lane + 32 * c);
                const T sc = sS[r * RK_ITEMS + lane + 32 * c];
                bool want = j < a.n_m && precedes(sc, j, ls[t - 1], li[t - 1]);
                unsigned ball = __ballot_sync(0xffffffffu, want);
                while (ball) {
                    const int src = __ffs(ball) - 1;
                    ball &= ball - 1;
                    const T cs = __shfl_sync(0xffffffffu, sc, src);
                    const int32_t cj = __shfl_sync(0xffffffffu, j, src);
                    // still beats the last entry? (earlier inserts moved it)
                    if (!precedes(cs, cj, ls[t - 1], li[t - 1])) continue;
                    // position = entries that precede the candidate
                    int p = 0;
                    T oS[2];
                    int32_t oI[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = lane + 32 * h;
                        oS[h] = m < t ? ls[m] : T(0);
                        oI[h] = m < t ? li[m] : 0;
                        p += __popc(__ballot_sync(0xffffffffu, m < t && precedes(oS[h], oI[h], cs, cj)));
                    }
                    __syncwarp();
                    // shift entries p .. t-2 down by one (all read above), then
                    // place the candidate
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = lane + 32 * h;
                        if (m < t - 1 && m >= p) {
                            ls[m + 1] = oS[h];
                            li[m + 1] = oI[h];
                        }
                    }
                    __syncwarp();
                    if (lane == 0) {
                        ls[p] = cs;
                        li[p] = cj;
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < RK_USERS * t; e += RK_THREADS) {
        const int r = e / t;
        const int64_t u = u0 + r;
        if (u < a.n_u) a.top_out[u * t + (e - r * t)] = lI[e];
    }
}

// reference lists: every id an item, no id twice in a user's list
__global__ void k_check_topt(const int32_t *__restrict__ top, int64_t n_u, int64_t n_m, int t, int *flag) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_u; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *l = top + u * t;
        bool bad = false;
        for (int k = 0; k < t && !bad; ++k) {
            if (l[k] < 0 || l[k] >= n_m) bad = true;
            for (int q = 0; q < k && !bad; ++q)
                if (l[q] == l[k]) bad = true;
        }
        if (bad) atomicAdd(flag, 1);
    }
}

als_status launch_check_topt(als_ctx *c, const int32_t *top, int t, int *flag) {
    ALS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((c->n_u + 255) / 256, 4096));
    k_check_topt<<<grid, 256, 0, c->stream>>>(top, c->n_u, c->n_m, t, flag);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

template <typename T>
als_status launch_rank(als_ctx *c, bool select, int t, const int32_t *top_ref, int32_t *top_out, double *q_out) {
    RankArgs<T> a;
    a.U = reinterpret_cast<const T *>(c->X);
    a.M = reinterpret_cast<const T *>(c->X) + (size_t)c->n_u * c->ld;
    a.n_u = c->n_u;
    a.n_m = c->n_m;
    a.nf = c->nf;
    a.ld = c->ld;
    a.t = t;
    a.top_ref = top_ref;
    a.top_out = top_out;
    a.q_out = q_out;
    const RankSmem<T> L = rank_smem<T>(c->nf, t, select);
    const void *fn = select ? (const void *)k_rank_topt<T> : (const void *)k_rank_count<T>;
    if (raise_smem_limit(fn, L.total) != ALS_OK) return ALS_ECUDA;
    const unsigned grid = (unsigned)((c->n_u + RK_USERS - 1) / RK_USERS);
    if (select) k_rank_topt<T><<<grid, RK_THREADS, L.total, c->stream>>>(a);
    else k_rank_count<T><<<grid, RK_THREADS, L.total, c->stream>>>(a);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

als_status rank_checks(als_ctx *c, int32_t t, const char *who) {
    if (!c) { als_set_error(std::string(who) + ": ctx is NULL"); return ALS_EINVAL; }
    if (c->n_prob > 1) { als_set_error(std::string(who) + ": not supported for batched contexts"); return ALS_ENOTSUP; }
    if (t < 1 || t > RK_TMAX || t > c->n_m) {
        als_set_error(std::string(who) + ": need 1 <= t <= min(64, n_m)");
        return ALS_EINVAL;
    }
    if (c->n_u > (int64_t)INT32_MAX * RK_USERS) { als_set_error(std::string(who) + ": too many users"); return ALS_ENOTSUP; }
    return ALS_OK;
}

}  // namespace

extern "C" als_status als_rank_topt(als_ctx *c, int32_t t, int32_t *top, int on_device) {
    als_status s = rank_checks(c, t, "als_rank_topt");
    if (s != ALS_OK) return s;
    if (!top) { als_set_error("als_rank_topt: top is NULL"); return ALS_EINVAL; }
    int32_t *dtop = top;
    const size_t bytes = (size_t)c->n_u * t * sizeof(int32_t);
    if (!on_device && (s = ctx_alloc(c, (void **)&dtop, bytes)) != ALS_OK) return s;
    s = c->f64 ? launch_rank<double>(c, true, t, nullptr, dtop, nullptr)
               : launch_rank<float>(c, true, t, nullptr, dtop, nullptr);
    if (s == ALS_OK && !on_device) {
        const cudaError_t e1 = cudaMemcpyAsync(top, dtop, bytes, cudaMemcpyDeviceToHost, c->stream);
        const cudaError_t e2 = cudaStreamSynchronize(c->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            als_set_error(std::string("als_rank_topt: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            s = ALS_ECUDA;
        }
    }
    if (!on_device) ctx_free(c, dtop);
    return s;
}

extern "C" als_status als_rank_accuracy(als_ctx *c, int32_t t, const int32_t *top_ref, int on_device,
                                        double *q_mean, double *q_user) {
    als_status s = rank_checks(c, t, "als_rank_accuracy");
    if (s != ALS_OK) return s;
    if (!top_ref || !q_mean) { als_set_error("als_rank_accuracy: top_ref or q_mean is NULL"); return ALS_EINVAL; }
    const size_t bytes = (size_t)c->n_u * t * sizeof(int32_t);
    int32_t *dref = const_cast<int32_t *>(top_ref);
    if (!on_device) {
        if ((s = ctx_alloc(c, (void **)&dref, bytes)) != ALS_OK) return s;
        if (cudaMemcpyAsync(dref, top_ref, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            ctx_free(c, dref);
            als_set_error("als_rank_accuracy: copy of top_ref failed");
            return ALS_ECUDA;
        }
    }
    // reference ids must be items, distinct within a user's list
    s = launch_check_topt(c, dref, t, c->dflags + 9);
    if (s == ALS_OK) {
        int bad = 0;
        if (cudaMemcpyAsync(&bad, c->dflags + 9, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            s = ALS_ECUDA;
            als_set_error("als_rank_accuracy: validation failed");
        } else if (bad) {
            s = ALS_EINVAL;
            als_set_error("als_rank_accuracy: top_ref holds an item id out of range or a repeated id");
        }
    }
    // q_i per user in the first row-term slots, then the fixed-order mean
    if (s == ALS_OK)
        s = c->f64 ? launch_rank<double>(c, false, t, dref, nullptr, c->rowterm)
                   : launch_rank<float>(c, false, t, dref, nullptr, c->rowterm);
    if (s == ALS_OK && q_user &&
        cudaMemcpyAsync(q_user, c->rowterm, (size_t)c->n_u * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess) {
        s = ALS_ECUDA;
        als_set_error("als_rank_accuracy: copy of q failed");
    }
    if (s == ALS_OK) s = launch_reduce(c, 1, c->n_u, S_RED, POST_NONE, LsParams{});
    if (s == ALS_OK) {
        double sum = 0.0;
        if (cudaMemcpyAsync(&sum, c->S + S_RED, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            s = ALS_ECUDA;
            als_set_error("als_rank_accuracy: read-back failed");
        } else {
            *q_mean = sum / (double)c->n_u;
        }
    }
    if (!on_device) ctx_free(c, dref);
    return s;
}
