// Measured FMA issue rate of the GPU's non-tensor pipes (FP32 or FP64), the
// ceiling of the stencil kernels: every thread runs eight independent
// multiply-add chains in registers, no memory traffic.  A multiply-add counts
// as two flops.  The paper has no counterpart; it is a measurement helper.
#include <cuda_runtime.h>

#include "internal.h"
#include "ofmlmc.h"

using ofm::fail;

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_chains(int iters, T seed, T* out) {
    T a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = seed + (T)(threadIdx.x + k);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], m, c);
    }
    T s = (T)0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == (T)-1) out[blockIdx.x] = s;   // never taken; keeps the chains live
}

template <typename T>
int probe(int iters, double* tflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_probe_fma_tflops: no device");
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_probe_fma_tflops: event creation failed");
    for (int w = 0; w < 3; ++w) fma_chains<T><<<blocks, PROBE_THREADS, 0, st>>>(iters, (T)1, (T*)nullptr);
    const int reps = 10;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) fma_chains<T><<<blocks, PROBE_THREADS, 0, st>>>(iters, (T)1, (T*)nullptr);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(OFM_ECUDA, "ofm_probe_fma_tflops: %s", cudaGetErrorString(err));
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * PROBE_THREADS * blocks * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return OFM_OK;
}

}  // namespace

extern "C" int ofm_probe_fma_tflops(int precision, double* tflops, void* stream) {
    ofm::clear_error();
    if (!tflops || (precision != OFM_FP32 && precision != OFM_FP64))
        return fail(OFM_EINVAL, "ofm_probe_fma_tflops: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    return precision == OFM_FP32 ? probe<float>(1 << 15, tflops, st) : probe<double>(1 << 10, tflops, st);
}
