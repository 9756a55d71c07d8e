// Allocation-free variant of the line-search-coefficient pass.
//
// als_linesearch_coeffs() needs a context, and building a context allocates
// device memory for the ratings, the vectors and the reduction scratch.  Some
// callers cannot allocate at the point where they need the coefficients:
// code that runs while a CUDA stream is being captured into a graph (where
// cudaMalloc is not allowed), code inside a framework that owns every byte of
// device memory through its own pool, or a latency-critical serving loop that
// must never enter the allocator.  For them this file offers one entry point
// that takes every input and output from the caller and keeps its only
// scratch -- the per-row FP64 terms and the block partials of the fixed-order
// reduction -- in a file-scope device array of fixed size.
//
// That array is part of the library image: every GPU that loads the library
// holds it (about 10 MB) until the process exits.  All calls share it, so two
// calls that overlap on the GPU (different streams, no ordering) race on it;
// calls on one stream, or otherwise ordered, are safe.
#include <mutex>

#include "internal.cuh"

#define ALS_STATIC_MAX_ROWS (1 << 18)   // n_u + n_m limit of the static entry point
#define ALS_STATIC_MAXB 256             // reduction blocks

namespace {

struct StaticScratch {
    double rowterm[5 * (size_t)ALS_STATIC_MAX_ROWS];
    double partial[5 * ALS_STATIC_MAXB];
    unsigned ticket;
};

static __device__ __align__(256) StaticScratch g_scratch;

struct StaticArgs {
    int64_t n_u, n_m;
    int nf, ld;
    double lambda;
    const int64_t *uptr;
    const int32_t *uidx;
    const float *uval;
    const int64_t *mptr;
    const void *x, *p;
    StaticScratch *scratch;   // device address of g_scratch
    double *c_out;
};

template <typename T>
__device__ __forceinline__ void sld4(const T *q, T (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = q[i];
}

template <int LPR, typename V>
__device__ __forceinline__ V ssum(V x, unsigned mask) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

// One group of LPR lanes per row: user rows (< n_u) get the rating terms of
// Q(alpha) plus their lambda terms, item rows only their lambda terms; the
// five per-row FP64 terms go to scratch->rowterm.
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_lscoef_static(StaticArgs a) {
    const int lane = threadIdx.x & 31, gl = lane % LPR;
    const unsigned mask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << ((lane / LPR) * LPR));
    const bool act = gl < a.ld / 4;
    const int64_t nrows = a.n_u + a.n_m;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / LPR;
    const T *X = reinterpret_cast<const T *>(a.x), *P = reinterpret_cast<const T *>(a.p);
    const T *XM = X + a.n_u * a.ld, *PM = P + a.n_u * a.ld;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR; row < nrows; row += ngroups) {
        T xr[4] = {0, 0, 0, 0}, pr[4] = {0, 0, 0, 0};
        if (act) {
            sld4(X + row * a.ld + 4 * gl, xr);
            sld4(P + row * a.ld + 4 * gl, pr);
        }
        double t[5] = {0, 0, 0, 0, 0};
        int64_t n;
        if (row < a.n_u) {
            const int64_t beg = a.uptr[row];
            n = a.uptr[row + 1] - beg;
            int owner = 0;
            for (int64_t e = beg; e < beg + n; ++e) {
                const int64_t j = a.uidx[e];
                T xm[4] = {0, 0, 0, 0}, pm[4] = {0, 0, 0, 0};
                if (act) {
                    sld4(XM + j * a.ld + 4 * gl, xm);
                    sld4(PM + j * a.ld + 4 * gl, pm);
                }
                T d[4] = {0, 0, 0, 0};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    d[0] += xr[i] * xm[i];
                    d[1] += xr[i] * pm[i];
                    d[2] += pr[i] * xm[i];
                    d[3] += pr[i] * pm[i];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] = ssum<LPR>(d[q], mask);
                if (owner == gl) {
                    const double e0 = (double)a.uval[e] - (double)d[0];
                    const double aa = (double)d[1] + (double)d[2], b = (double)d[3];
                    t[0] += e0 * e0;
                    t[1] += -2.0 * e0 * aa;
                    t[2] += aa * aa - 2.0 * e0 * b;
                    t[3] += 2.0 * aa * b;
                    t[4] += b * b;
                }
                owner = owner + 1 == LPR ? 0 : owner + 1;
            }
        } else {
            n = a.mptr[row - a.n_u + 1] - a.mptr[row - a.n_u];
        }
        double xx = 0, xp = 0, pp = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xx += (double)xr[i] * (double)xr[i];
            xp += (double)xr[i] * (double)pr[i];
            pp += (double)pr[i] * (double)pr[i];
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) t[q] = ssum<LPR>(t[q], mask);
        xx = ssum<LPR>(xx, mask);
        xp = ssum<LPR>(xp, mask);
        pp = ssum<LPR>(pp, mask);
        const double ln = a.lambda * (double)n;
        t[0] += ln * xx;
        t[1] += ln * 2.0 * xp;
        t[2] += ln * pp;
        if (gl == 0)
            for (int q = 0; q < 5; ++q) a.scratch->rowterm[q * nrows + row] = t[q];
    }
}

// fixed-order two-level sum of the five per-row terms into c_out[0..4]
__global__ void __launch_bounds__(256) k_reduce_static(StaticArgs a) {
    __shared__ double red[256];
    __shared__ bool last;
    StaticScratch *s = a.scratch;
    const int64_t n = a.n_u + a.n_m;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int t = 0; t < 5; ++t) {
        double v = 0.0;
        for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) v += s->rowterm[t * n + i];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) s->partial[t * ALS_STATIC_MAXB + blockIdx.x] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&s->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int t = 0; t < 5; ++t) {
        double v = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) v += s->partial[t * ALS_STATIC_MAXB + i];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.c_out[t] = red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) s->ticket = 0u;
}

// device address of g_scratch, looked up once per device and CUDA context
// (host code must not pass the symbol itself: on the host it is only a
// stand-in).  The context handle is recorded beside the address: after
// cudaDeviceReset the device's primary context is a new one, the module is
// loaded again, and the array may sit elsewhere, so a changed handle means
// the lookup is done again.
constexpr int kMaxDevices = 64;
typedef int (*CtxGetCurrentFn)(void **);
std::mutex g_mu;
StaticScratch *g_addr[kMaxDevices] = {};
void *g_ctx[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_get_tried = false;

als_status scratch_for_device(StaticScratch **out, int *sms) {
    int dev = 0;
    ALS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        als_set_error("als_linesearch_coeffs_static: device index out of range");
        return ALS_ENOTSUP;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ctx_get_tried) {
        g_ctx_get_tried = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
        cudaGetLastError();
    }
    void *ctx = nullptr;
    if (g_ctx_get && g_ctx_get(&ctx) != 0) ctx = nullptr;
    if (!g_addr[dev] || ctx != g_ctx[dev]) {
        void *p = nullptr;
        ALS_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
        int n = 0;
        ALS_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        // the lookup made the device's primary context current if it was not
        if (g_ctx_get && g_ctx_get(&ctx) != 0) ctx = nullptr;
        g_addr[dev] = reinterpret_cast<StaticScratch *>(p);
        g_ctx[dev] = ctx;
        g_sms[dev] = n;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return ALS_OK;
}

template <typename T>
void launch_static(const StaticArgs &a, unsigned grid, cudaStream_t st) {
    const int slots = a.ld / 4;
    if (slots <= 4) k_lscoef_static<T, 4><<<grid, 256, 0, st>>>(a);
    else if (slots <= 8) k_lscoef_static<T, 8><<<grid, 256, 0, st>>>(a);
    else if (slots <= 16) k_lscoef_static<T, 16><<<grid, 256, 0, st>>>(a);
    else k_lscoef_static<T, 32><<<grid, 256, 0, st>>>(a);
}

}  // namespace

extern "C" als_status als_linesearch_coeffs_static(int64_t n_u, int64_t n_m, int32_t n_f, int32_t ld,
                                                   double lambda, const int64_t *uptr, const int32_t *uidx,
                                                   const float *uval, const int64_t *mptr, const void *x,
                                                   const void *p, int dtype, double *c_out, void *stream) {
    if (n_u < 1 || n_m < 1 || n_f < 1 || n_f > ALS_MAX_NF || ld < n_f || ld % 4 != 0 || ld > ALS_MAX_NF ||
        !uptr || !uidx || !uval || !mptr || !x || !p || !c_out ||
        (dtype != ALS_DT_F64 && dtype != ALS_DT_F32) || !(lambda >= 0.0)) {
        als_set_error("als_linesearch_coeffs_static: bad argument (need 1 <= n_f <= ld <= 128, ld % 4 == 0, "
                      "device pointers, dtype F64 or F32, lambda >= 0)");
        return ALS_EINVAL;
    }
    if (n_u + n_m > ALS_STATIC_MAX_ROWS) {
        als_set_error("als_linesearch_coeffs_static: n_u + n_m = " + std::to_string(n_u + n_m) +
                      " exceeds the static scratch limit of " + std::to_string(ALS_STATIC_MAX_ROWS) +
                      " rows; use als_linesearch_coeffs with a context instead");
        return ALS_EINVAL;
    }
    StaticScratch *scr = nullptr;
    int sms = 0;
    als_status s = scratch_for_device(&scr, &sms);
    if (s != ALS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    StaticArgs a;
    a.n_u = n_u; a.n_m = n_m; a.nf = n_f; a.ld = ld; a.lambda = lambda;
    a.uptr = uptr; a.uidx = uidx; a.uval = uval; a.mptr = mptr;
    a.x = x; a.p = p; a.scratch = scr; a.c_out = c_out;
    // the ticket must start at zero (a previous call's kernel resets it, but a
    // call that failed between the two launches would not have)
    ALS_CUDA_TRY(cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned), st));
    const int64_t rows = n_u + n_m;
    const int slots = ld / 4;
    const int lpr = slots <= 4 ? 4 : slots <= 8 ? 8 : slots <= 16 ? 16 : 32;
    const int64_t want = (rows + 256 / lpr - 1) / (256 / lpr);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    if (dtype == ALS_DT_F64) launch_static<double>(a, grid, st);
    else launch_static<float>(a, grid, st);
    ALS_CUDA_TRY(cudaGetLastError());
    const unsigned rgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 8191) / 8192, ALS_STATIC_MAXB));
    k_reduce_static<<<rgrid, 256, 0, st>>>(a);
    ALS_CUDA_TRY(cudaGetLastError());
    return ALS_OK;
}
