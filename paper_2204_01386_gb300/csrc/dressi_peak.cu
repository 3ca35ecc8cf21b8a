// dressi_peak.cu -- microbenchmarks of the two units the per-tile kernels lean on, run on
// the caller's device: FP32 FMA throughput and red.global.add.v4.f32 throughput.  They give
// the measured denominators of the roofline fractions (no counterpart in the paper).
#include <algorithm>

#include "dressi_core.cuh"
#include "dressi_launch.h"

namespace dressi {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;          // independent FMA chains per thread
constexpr int PK_FMA_ITERS = 65536;  // chain steps per launch (~4 ms at the nominal rate)
constexpr int PK_RED_PER_THREAD = 1024; // reductions per thread per launch (~5 GB of payload)
constexpr int PK_RED_SCATTERED = 256;   // the same, scattered (one sector per lane)

// PK_CHAINS independent chains a <- a b + c per thread; the sums are written so that
// nothing is dead code.  FLOP per launch = threads * PK_FMA_ITERS * PK_CHAINS * 2.
__global__ void __launch_bounds__(PK_THREADS) k_peak_fma(float *out, float b, float c, int iters)
{
    float a[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) a[j] = (float)threadIdx.x * 1e-3f + (float)j;
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) a[j] = __fmaf_rn(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += a[j];
    out[blockIdx.x * (size_t)PK_THREADS + threadIdx.x] = s;
}

// every lane adds a float4 into its own 16 bytes, the launch's threads stepping through the
// buffer: with SCATTER false consecutive lanes are adjacent (one warp instruction covers 512
// contiguous bytes), with SCATTER true every lane's float4 lies in a 32-byte sector of its
// own, 4 KiB away from its neighbour lane's (one sector per lane, as the gradient scatters
// of the adjoint mostly are)
template <bool SCATTER>
__global__ void __launch_bounds__(PK_THREADS) k_peak_red(float4 *buf, long long n4, int reps)
{
    const long long nthreads = (long long)gridDim.x * PK_THREADS;
    long long i = blockIdx.x * (long long)PK_THREADS + threadIdx.x;
    const float4 v = make_float4(1.f, 2.f, 3.f, 0.f);
#pragma unroll 4
    for (int r = 0; r < reps; ++r) {
        // scattered: lane l of warp w at float4 (w * 32 + l) * 256 + r, wrapped into the buffer
        const long long a = SCATTER ? ((i * 256 + r) % n4) : (i % n4);
        atomicAdd(buf + a, v);
        i += nthreads;
    }
}

}  // namespace dressi

using namespace dressi;

extern "C" int dressi_measure_peak(int32_t which, void *dev_buf, size_t bytes, double *result, void *stream)
{
    if (which < 0 || which > 2 || !dev_buf || !result || bytes < ((size_t)64 << 20) ||
        (reinterpret_cast<uintptr_t>(dev_buf) & 15) != 0)
        return DRESSI_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DRESSI_ERR_LAUNCH;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return DRESSI_ERR_LAUNCH;
    }
    // a full SM of threads (2,048) on every SM
    const int blocks = sms * (2048 / PK_THREADS);
    const long long threads = (long long)blocks * PK_THREADS;
    const long long n4 = (long long)(bytes / 16);
    if (which == 0 && (size_t)threads * sizeof(float) > bytes) return DRESSI_ERR_ARG;
    float best = 3.0e38f;
    int rc = DRESSI_OK;
    for (int rep = 0; rep < 6; ++rep) {   // the first launch warms up; the best of the rest counts
        cudaEventRecord(e0, s);
        if (which == 0) k_peak_fma<<<blocks, PK_THREADS, 0, s>>>(static_cast<float *>(dev_buf), 0.999f, 1e-3f, PK_FMA_ITERS);
        else if (which == 1) k_peak_red<false><<<blocks, PK_THREADS, 0, s>>>(static_cast<float4 *>(dev_buf), n4, PK_RED_PER_THREAD);
        else k_peak_red<true><<<blocks, PK_THREADS, 0, s>>>(static_cast<float4 *>(dev_buf), n4, PK_RED_SCATTERED);
        count_launch(1);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = DRESSI_ERR_LAUNCH; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) rc = DRESSI_ERR_LAUNCH;
    if (rc != DRESSI_OK) return rc;
    const double sec = (double)best * 1e-3;
    if (which == 0) *result = (double)threads * PK_FMA_ITERS * PK_CHAINS * 2.0 / sec / 1e12;   // TFLOP/s
    else if (which == 1) *result = (double)threads * PK_RED_PER_THREAD * 16.0 / sec / 1e9;    // GB/s
    else *result = (double)threads * PK_RED_SCATTERED * 32.0 / sec / 1e9;                     // GB/s of sectors
    return DRESSI_OK;
}
