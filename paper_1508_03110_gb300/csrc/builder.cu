// Ratings builder (§V-B: R is stored twice, by user and by item, in
// compressed row blocks).  On one GPU the two copies are a by-user CSR and a
// by-item CSC in HBM, built on the device from COO/CSR input:
//   1. validate ids and values;
//   2. stable LSD radix sort of (user, item) keys -> CSR order (items of each
//      user ascending), duplicate check, user degrees n_ui, row pointers;
//   3. stable radix sort of the CSR sequence by item -> CSC order (users of
//      each item ascending), item degrees n_mj, column pointers;
//   4. rows of each side ordered by descending degree (stable), which the
//      sweep and the passes use to balance heavy rows.
// The sort is an 8-bit-digit LSD radix sort: per-tile digit histograms,
// one exclusive scan, and a stable scatter that ranks equal digits with warp
// match masks.  Integer atomics only; the result is deterministic.
#include <algorithm>
#include <cstdio>

#include "internal.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                          int32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t e = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                             int shift, const int64_t *__restrict__ off, int64_t nblocks) {
    __shared__ int32_t wcnt[RS_THREADS / 32][256];
    __shared__ int32_t woff[RS_THREADS / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][threadIdx.x] = 0;
    const int64_t tile_off = off[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    int32_t running = 0;  // items of digit threadIdx.x in earlier rounds of this tile
    __shared__ int64_t sbase[256];
    sbase[threadIdx.x] = tile_off;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t e = base + (int64_t)r * RS_THREADS + threadIdx.x;
        const bool valid = e < n;
        uint64_t key = valid ? kin[e] : 0;
        uint32_t val = valid ? vin[e] : 0;
        const unsigned d = valid ? (unsigned)((key >> shift) & 0xFF) : 0x100u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int32_t s = running;
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                woff[w][threadIdx.x] = s;
                s += wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = 0;
            }
            running = s;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = sbase[d] + woff[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// Exclusive scan helpers (int32 counts -> int64 prefix), three phases.
__global__ void k_scan_tile_sums(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t red[SCAN_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (e < n) s += in[e];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = SCAN_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// single block, in place exclusive scan of int64 values; total -> *total
__global__ void k_scan_single(int64_t *__restrict__ a, int64_t n, int64_t *__restrict__ total) {
    __shared__ int64_t buf[SCAN_THREADS];
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_THREADS) {
        const int64_t e = base + threadIdx.x;
        const int64_t v = e < n ? a[e] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int w = 1; w < SCAN_THREADS; w <<= 1) {
            const int64_t t = threadIdx.x >= w ? buf[threadIdx.x - w] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (e < n) a[e] = carry + buf[threadIdx.x] - v;
        const int64_t blk = buf[SCAN_THREADS - 1];
        __syncthreads();
        carry += blk;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const int32_t *__restrict__ in, int64_t n, const int64_t *__restrict__ sums,
                             int64_t *__restrict__ out) {
    __shared__ int64_t buf[SCAN_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t loc[SCAN_ITEMS];
    int64_t s = 0;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + i;
        loc[i] = s;
        s += e < n ? in[e] : 0;
    }
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int w = 1; w < SCAN_THREADS; w <<= 1) {
        const int64_t t = threadIdx.x >= w ? buf[threadIdx.x - w] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    const int64_t pre = sums[blockIdx.x] + buf[threadIdx.x] - s;
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        const int64_t e = base + i;
        if (e < n) out[e] = pre + loc[i];
    }
}

__global__ void k_expand_rows(const int64_t *__restrict__ rowptr, int64_t n_rows, int64_t nnz,
                              int32_t *__restrict__ rows) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int64_t lo = 0, hi = n_rows;  // last r with rowptr[r] <= e
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (rowptr[mid] <= e) lo = mid; else hi = mid;
    }
    rows[e] = (int32_t)lo;
}

__global__ void k_make_keys(const int32_t *__restrict__ rows, const int32_t *__restrict__ cols,
                            const float *__restrict__ vals, int64_t nnz, int64_t n_u, int64_t n_m,
                            int cbits, uint64_t *__restrict__ keys, uint32_t *__restrict__ pay,
                            int *__restrict__ flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int32_t r = rows[e], c = cols[e];
    const float v = vals[e];
    if (r < 0 || r >= n_u || c < 0 || c >= n_m || !isfinite(v)) {
        atomicAdd(&flags[1], 1);
        keys[e] = 0;
    } else {
        keys[e] = ((uint64_t)r << cbits) | (uint64_t)c;
    }
    pay[e] = __float_as_uint(v);
}

__global__ void k_csr_fill(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ pay,
                           int64_t nnz, int cbits, int32_t *__restrict__ uidx, float *__restrict__ uval,
                           int32_t *__restrict__ ucnt, uint64_t *__restrict__ ckeys,
                           uint32_t *__restrict__ cpay, int *__restrict__ flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const uint64_t k = keys[e];
    const uint64_t cmask = (cbits >= 64) ? ~0ull : ((1ull << cbits) - 1);
    const int32_t col = (int32_t)(k & cmask), row = (int32_t)(k >> cbits);
    if (e > 0 && keys[e - 1] == k) atomicAdd(&flags[2], 1);
    uidx[e] = col;
    uval[e] = __uint_as_float(pay[e]);
    atomicAdd(&ucnt[row], 1);
    ckeys[e] = (uint64_t)col;
    cpay[e] = (uint32_t)e;
}

__global__ void k_csc_fill(const uint64_t *__restrict__ skeys, const uint32_t *__restrict__ cpos,
                           const float *__restrict__ uval, int64_t nnz, int cbits,
                           int32_t *__restrict__ midx, float *__restrict__ mval,
                           int32_t *__restrict__ mcnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const uint32_t src = cpos[e];
    const uint64_t k = skeys[src];
    const uint64_t cmask = (1ull << cbits) - 1;
    midx[e] = (int32_t)(k >> cbits);
    mval[e] = uval[src];
    atomicAdd(&mcnt[(int32_t)(k & cmask)], 1);
}

__global__ void k_degree_keys(const int64_t *__restrict__ ptr, int64_t n, int64_t maxdeg,
                              uint64_t *__restrict__ keys, uint32_t *__restrict__ pay,
                              int *__restrict__ nheavy) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t d = ptr[r + 1] - ptr[r];
    keys[r] = (uint64_t)(maxdeg - d);
    pay[r] = (uint32_t)r;
    if (d >= ALS_HEAVY_MIN) atomicAdd(nheavy, 1);
}

__global__ void k_max_degree(const int64_t *__restrict__ ptr, int64_t n, unsigned long long *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    atomicMax(out, (unsigned long long)(ptr[r + 1] - ptr[r]));
}

__global__ void k_copy_u32_to_i32(const uint32_t *__restrict__ a, int64_t n, int32_t *__restrict__ b) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) b[r] = (int32_t)a[r];
}

int bits_for(int64_t n) {  // bits needed to represent values 0..n-1
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < n) ++b;
    return b;
}

inline unsigned grid1d(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct Scratch {
    als_ctx *c;
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) ctx_free(c, p);
    }
    template <typename T>
    als_status get(T **p, size_t count) {
        void *q = nullptr;
        als_status s = ctx_alloc(c, &q, std::max<size_t>(count, 1) * sizeof(T));
        if (s != ALS_OK) return s;
        ptrs.push_back(q);
        *p = (T *)q;
        return ALS_OK;
    }
};

// exclusive scan of counts[n] into out[n+1] (out[n] = total)
als_status scan_counts(als_ctx *c, Scratch &sc, const int32_t *counts, int64_t n, int64_t *out) {
    const int64_t nb = std::max<int64_t>(1, (n + SCAN_TILE - 1) / SCAN_TILE);
    int64_t *sums = nullptr;
    als_status s = sc.get(&sums, (size_t)nb);
    if (s != ALS_OK) return s;
    if (n > 0) k_scan_tile_sums<<<(unsigned)nb, SCAN_THREADS, 0, c->stream>>>(counts, n, sums);
    else ALS_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(int64_t), c->stream));
    k_scan_single<<<1, SCAN_THREADS, 0, c->stream>>>(sums, nb, out + n);
    if (n > 0) k_scan_apply<<<(unsigned)nb, SCAN_THREADS, 0, c->stream>>>(counts, n, sums, out);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}

// stable LSD radix sort over bits [0, nbits); result ends in (*k0, *v0)
als_status radix_sort(als_ctx *c, Scratch &sc, uint64_t **k0, uint32_t **v0, uint64_t *k1,
                      uint32_t *v1, int64_t n, int nbits) {
    if (n <= 1 || nbits <= 0) return ALS_OK;
    const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    int32_t *hist = nullptr;
    int64_t *off = nullptr;
    als_status s = sc.get(&hist, (size_t)(256 * nb));
    if (s != ALS_OK) return s;
    s = sc.get(&off, (size_t)(256 * nb + 1));
    if (s != ALS_OK) return s;
    uint64_t *ka = *k0, *kb = k1;
    uint32_t *va = *v0, *vb = v1;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, c->stream>>>(ka, n, shift, hist, nb);
        s = scan_counts(c, sc, hist, 256 * nb, off);
        if (s != ALS_OK) return s;
        k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, c->stream>>>(ka, va, kb, vb, n, shift, off, nb);
        ALS_CUDA_TRY(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *k0 = ka;
    *v0 = va;
    return ALS_OK;
}

}  // namespace

als_status build_ratings(als_ctx *c, const int32_t *rows_in, const int64_t *rowptr_in,
                         const int32_t *cols_in, const float *vals_in, int on_device) {
    const int64_t nnz = c->nnz, n_u = c->n_u, n_m = c->n_m;
    Scratch sc{c, {}};
    als_status s;
    int32_t *rows = nullptr, *cols = nullptr;
    float *vals = nullptr;
    s = sc.get(&rows, (size_t)nnz); if (s) return s;
    s = sc.get(&cols, (size_t)nnz); if (s) return s;
    s = sc.get(&vals, (size_t)nnz); if (s) return s;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nnz > 0) {
        ALS_CUDA_TRY(cudaMemcpyAsync(cols, cols_in, nnz * sizeof(int32_t), kind, c->stream));
        ALS_CUDA_TRY(cudaMemcpyAsync(vals, vals_in, nnz * sizeof(float), kind, c->stream));
    }
    if (rowptr_in) {
        int64_t *rp = nullptr;
        s = sc.get(&rp, (size_t)(n_u + 1)); if (s) return s;
        ALS_CUDA_TRY(cudaMemcpyAsync(rp, rowptr_in, (n_u + 1) * sizeof(int64_t), kind, c->stream));
        // the CSR must be well formed: rowptr[0] = 0, non-decreasing, rowptr[n_u] = nnz
        int64_t h0 = 0, hn = 0;
        ALS_CUDA_TRY(cudaMemcpyAsync(&h0, rp, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        ALS_CUDA_TRY(cudaMemcpyAsync(&hn, rp + n_u, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (h0 != 0 || hn != nnz) {
            als_set_error("als_create: rowptr[0] must be 0 and rowptr[n_u] must equal nnz");
            return ALS_EINVAL;
        }
        if (nnz > 0) k_expand_rows<<<grid1d(nnz, 256), 256, 0, c->stream>>>(rp, n_u, nnz, rows);
    } else if (nnz > 0) {
        ALS_CUDA_TRY(cudaMemcpyAsync(rows, rows_in, nnz * sizeof(int32_t), kind, c->stream));
    }
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags, 0, 8 * sizeof(int), c->stream));

    const int cbits = std::max(1, bits_for(n_m)), rbits = std::max(1, bits_for(n_u));
    uint64_t *ka = nullptr, *kb = nullptr;
    uint32_t *va = nullptr, *vb = nullptr;
    s = sc.get(&ka, (size_t)nnz); if (s) return s;
    s = sc.get(&kb, (size_t)nnz); if (s) return s;
    s = sc.get(&va, (size_t)nnz); if (s) return s;
    s = sc.get(&vb, (size_t)nnz); if (s) return s;
    if (nnz > 0)
        k_make_keys<<<grid1d(nnz, 256), 256, 0, c->stream>>>(rows, cols, vals, nnz, n_u, n_m, cbits,
                                                             ka, va, c->dflags);
    ALS_CUDA_TRY(cudaGetLastError());
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->hflags[1]) {
        char buf[160];
        snprintf(buf, sizeof buf, "als_create: %d ratings with an id out of range or a non-finite value",
                 c->hflags[1]);
        als_set_error(buf);
        return ALS_EINVAL;
    }
    // by-user order
    s = radix_sort(c, sc, &ka, &va, kb, vb, nnz, rbits + cbits); if (s) return s;
    int32_t *ucnt = nullptr, *mcnt = nullptr;
    s = sc.get(&ucnt, (size_t)n_u); if (s) return s;
    s = sc.get(&mcnt, (size_t)n_m); if (s) return s;
    ALS_CUDA_TRY(cudaMemsetAsync(ucnt, 0, n_u * sizeof(int32_t), c->stream));
    ALS_CUDA_TRY(cudaMemsetAsync(mcnt, 0, n_m * sizeof(int32_t), c->stream));
    uint64_t *ck = nullptr, *ck2 = nullptr;
    uint32_t *cp = nullptr, *cp2 = nullptr;
    s = sc.get(&ck, (size_t)nnz); if (s) return s;
    s = sc.get(&ck2, (size_t)nnz); if (s) return s;
    s = sc.get(&cp, (size_t)nnz); if (s) return s;
    s = sc.get(&cp2, (size_t)nnz); if (s) return s;
    if (nnz > 0)
        k_csr_fill<<<grid1d(nnz, 256), 256, 0, c->stream>>>(ka, va, nnz, cbits, c->uidx, c->uval, ucnt,
                                                            ck, cp, c->dflags);
    s = scan_counts(c, sc, ucnt, n_u, c->uptr); if (s) return s;
    // by-item order: stable sort of the CSR sequence by item id
    s = radix_sort(c, sc, &ck, &cp, ck2, cp2, nnz, cbits); if (s) return s;
    if (nnz > 0)
        k_csc_fill<<<grid1d(nnz, 256), 256, 0, c->stream>>>(ka, cp, c->uval, nnz, cbits, c->midx,
                                                            c->mval, mcnt);
    s = scan_counts(c, sc, mcnt, n_m, c->mptr); if (s) return s;
    ALS_CUDA_TRY(cudaGetLastError());

    // degree orders
    unsigned long long *dmax = nullptr;
    s = sc.get(&dmax, 2); if (s) return s;
    ALS_CUDA_TRY(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), c->stream));
    if (n_u > 0) k_max_degree<<<grid1d(n_u, 256), 256, 0, c->stream>>>(c->uptr, n_u, dmax);
    if (n_m > 0) k_max_degree<<<grid1d(n_m, 256), 256, 0, c->stream>>>(c->mptr, n_m, dmax + 1);
    unsigned long long hmax[2] = {0, 0};
    ALS_CUDA_TRY(cudaMemcpyAsync(hmax, dmax, sizeof hmax, cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->hflags[2]) {
        char buf[128];
        snprintf(buf, sizeof buf, "als_create: %d duplicate (user, item) ratings", c->hflags[2]);
        als_set_error(buf);
        return ALS_EINVAL;
    }
    c->maxdeg_u = (int64_t)hmax[0];
    c->maxdeg_m = (int64_t)hmax[1];
    ALS_CUDA_TRY(cudaMemsetAsync(c->dflags + 3, 0, 2 * sizeof(int), c->stream));
    for (int side = 0; side < 2; ++side) {
        const int64_t n = side ? n_m : n_u;
        const int64_t *ptr = side ? c->mptr : c->uptr;
        const int64_t maxdeg = side ? c->maxdeg_m : c->maxdeg_u;
        int32_t *order = side ? c->morder : c->uorder;
        if (n == 0) continue;
        uint64_t *k0 = nullptr, *k1 = nullptr;
        uint32_t *p0 = nullptr, *p1 = nullptr;
        s = sc.get(&k0, (size_t)n); if (s) return s;
        s = sc.get(&k1, (size_t)n); if (s) return s;
        s = sc.get(&p0, (size_t)n); if (s) return s;
        s = sc.get(&p1, (size_t)n); if (s) return s;
        k_degree_keys<<<grid1d(n, 256), 256, 0, c->stream>>>(ptr, n, maxdeg, k0, p0, c->dflags + 3 + side);
        s = radix_sort(c, sc, &k0, &p0, k1, p1, n, std::max(1, bits_for(maxdeg + 1)));
        if (s) return s;
        k_copy_u32_to_i32<<<grid1d(n, 256), 256, 0, c->stream>>>(p0, n, order);
        ALS_CUDA_TRY(cudaGetLastError());
    }
    ALS_CUDA_TRY(cudaMemcpyAsync(c->hflags, c->dflags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ALS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->nheavy_u = c->hflags[3];
    c->nheavy_m = c->hflags[4];
    return ALS_OK;
}
