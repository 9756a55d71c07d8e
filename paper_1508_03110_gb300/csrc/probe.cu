// Measured ALU peaks of this device (the paper has no counterpart: these are
// the denominators of the FP32 / FP64 roofline fractions of the sweep's
// Cholesky, solves and residuals, which run on the plain FMA pipes).
//
// Every thread runs eight independent FMA chains, so the pipes see no
// dependency stalls; the grid fills every SM with 2048 resident threads.
// The kernel is timed with CUDA events on its own stream, after a warm-up
// launch, best of three.  flops = threads x iterations x 8 chains x 2.
#include "internal.cuh"

namespace {

__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T b, T c, int iters, int write) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (write && s == (T)12345.678) g_probe_sink = (double)s;  // keeps the chains live
}

template <typename T>
als_status time_fma(cudaStream_t st, int sms, int iters, double *tflops) {
    const unsigned grid = (unsigned)sms * 8u;  // 8 x 256 = 2048 threads per SM
    cudaEvent_t e0, e1;
    ALS_CUDA_TRY(cudaEventCreate(&e0));
    ALS_CUDA_TRY(cudaEventCreate(&e1));
    k_fma_peak<T><<<grid, 256, 0, st>>>((T)0.999, (T)1e-4, iters, 1);
    double best = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        k_fma_peak<T><<<grid, 256, 0, st>>>((T)0.999, (T)1e-4, iters, 1);
        cudaEventRecord(e1, st);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            als_set_error(std::string("als_probe_alu_peaks: ") + cudaGetErrorString(e));
            return ALS_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = (double)grid * 256.0 * iters * 16.0 * 8.0 * 2.0;
        best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ALS_CUDA_TRY(cudaGetLastError());
    *tflops = best;
    return ALS_OK;
}

}  // namespace

extern "C" als_status als_probe_alu_peaks(double *fp32_tflops, double *fp64_tflops) {
    if (!fp32_tflops && !fp64_tflops) {
        als_set_error("als_probe_alu_peaks: both outputs are NULL");
        return ALS_EINVAL;
    }
    int dev = 0, sms = 0;
    ALS_CUDA_TRY(cudaGetDevice(&dev));
    ALS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st;
    ALS_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    als_status s = ALS_OK;
    // about 20 ms per launch at the nominal rates (80 FP32, 1.25 FP64 TFLOP/s)
    if (fp32_tflops) s = time_fma<float>(st, sms, 10000, fp32_tflops);
    if (s == ALS_OK && fp64_tflops) s = time_fma<double>(st, sms, 200, fp64_tflops);
    cudaStreamDestroy(st);
    return s;
}
