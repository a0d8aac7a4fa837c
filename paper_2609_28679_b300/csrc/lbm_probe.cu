// Device throughput probe: the float64 fused multiply-add rate of this GPU,
// the arithmetic bound of the float64 forms of the step (their population
// traffic alone would allow several times their measured rate).
#include <cuda_runtime.h>

#include <string>

#include "lbm.h"

void lbm_set_global_error(const std::string& msg);  // lbm_abi.cu

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;     // independent dependency chains per thread
constexpr int kProbeIters = 4096;   // fused multiply-adds per chain

// Eight independent chains a <- a b + c per thread: no memory traffic, no
// dependency stall once a scheduler holds a few warps.  The result is stored
// only if it is a sentinel value, so the arithmetic cannot be dropped.
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(double b, double c, double* sink)
{
    double a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
#pragma unroll 4
    for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int lbm_fp64_peak(double* tflops, double* ms, void* stream)
{
    if (!tflops) {
        lbm_set_global_error("lbm_fp64_peak: tflops is NULL");
        return LBM_E_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kProbeThreads, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = 4 * nsm * (per_sm > 0 ? per_sm : 1);  // four full waves
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<grid, kProbeThreads, 0, st>>>(0.999999, 1e-9, nullptr);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        lbm_set_global_error(std::string("lbm_fp64_peak: ") + cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    const double flops = 2.0 * kProbeChains * kProbeIters * (double)kProbeThreads * grid;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return LBM_OK;
}
