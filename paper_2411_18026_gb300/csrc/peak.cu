// Measured arithmetic peaks of the current GPU: the roofline denominators of
// the FP64 steps (kernel evaluation, CPQR, merges, top LU) and of the FP32
// sweep and forward operator.  A register-resident loop of independent fused
// multiply-adds, enough warps per SM to hide the pipe latency, timed with CUDA
// events: the rate a kernel of this kind can reach at the clock the GPU runs.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "fds.h"

namespace {

constexpr int CHAINS = 8;    // independent accumulators per thread
constexpr int UNROLL = 16;   // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, T b, T c, int iters) {
    T a[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int j = 0; j < CHAINS; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += a[j];
    if (s == (T)-1.25e-30) out[0] = s;   // never true for these inputs; keeps the chains live
}

template <typename T>
int measure(double *tflops) {
    int dev = 0, sms = 0;
    FDS_CUDA_TRY(cudaGetDevice(&dev));
    FDS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T *out = nullptr;
    FDS_CUDA_TRY(cudaMalloc((void **)&out, sizeof(T)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    auto run = [&](int iters, float *ms) -> int {
        cudaEventRecord(e0, 0);
        fds_count_launch(), k_fma_peak<T><<<blocks, threads>>>(out, (T)0.999999, (T)1e-6, iters);
        cudaEventRecord(e1, 0);
        FDS_CUDA_TRY(cudaGetLastError());
        FDS_CUDA_TRY(cudaEventSynchronize(e1));
        cudaEventElapsedTime(ms, e0, e1);
        return FDS_OK;
    };
    // calibrate to ~60 ms per launch, then best of three
    float ms = 0;
    int iters = 64, rc = run(iters, &ms);
    if (rc == FDS_OK) rc = run(iters, &ms);
    if (rc == FDS_OK) {
        iters = (int)std::min(4.0e6, std::max(64.0, iters * 60.0 / std::max(ms, 1e-3f)));
        double best = 0;
        for (int r = 0; r < 3 && rc == FDS_OK; ++r) {
            rc = run(iters, &ms);
            const double fl = 2.0 * CHAINS * UNROLL * (double)iters * blocks * threads;
            best = std::max(best, fl / (ms * 1e-3) / 1e12);
        }
        *tflops = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int fds_alu_peak(int32_t kind, double *tflops) {
    if (!tflops || (kind != 0 && kind != 1)) return FDS_ERR_ARG;
    *tflops = 0;
    return kind == 0 ? measure<double>(tflops) : measure<float>(tflops);
}
