// FMA-throughput probe (libhh_peaks.so): measures the FP32 and FP64 FMA
// peaks of the device that the roofline fractions of the force kernels are
// reported against.  Not part of the force path.
//
// Each thread runs kChains independent FMA chains for `iters` iterations;
// the grid is a multiple of the SM count.  FLOPs = 2 per FMA.

#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_fma_chain(T *out, int iters, T a, T b)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) acc[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) acc[c] = acc[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += acc[c];
    if (s == T(-1.2345)) out[blockIdx.x] = s;  // keeps the chains live
}

template <typename T>
int run(int device, int iters, double *tflops)
{
    if (cudaSetDevice(device) != cudaSuccess) return -3;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return -3;
    const int blocks = p.multiProcessorCount * 8, threads = 256;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-7);
    k_fma_chain<T><<<blocks, threads>>>(out, iters / 10, a, b);  // warm-up
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, threads>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return -3;
    const double flops = 2.0 * kChains * double(iters) * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}

}  // namespace

extern "C" int hh_fma_peak(int device, int fp64, int iters, double *tflops)
{
    if (!tflops || iters < 10) return -1;
    return fp64 ? run<double>(device, iters, tflops) : run<float>(device, iters, tflops);
}
