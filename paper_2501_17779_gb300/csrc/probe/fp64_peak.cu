// fp64_peak.cu -- measures this GPU's FP64 FMA throughput, the denominator of
// the roofline the FP64 kernels are reported against.  Built as its own small
// library (libfapeak.so); it is not part of the alignment ABI.
//
// Every thread runs 8 independent chains of dependent DFMAs; 16 CTAs of 256
// threads per SM keep every SM partition's FP64 pipe busy.
#include <cuda_runtime.h>

namespace {
__global__ void dfma_loop(double* out, int iters, double b, double c)
{
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-9 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.678) out[0] = s;  // keeps the loop alive; never true
}
}  // namespace

// Returns the best of `reps` timed launches in TFLOP/s (FMA = 2 flops), or a
// negative value on a CUDA error.  Runs on the current device and stream 0.
extern "C" double fa_probe_fp64_fma_tflops(int reps)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    double* d = nullptr;
    if (cudaMalloc(&d, 64) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 16, threads = 256, iters = 2048;
    dfma_loop<<<blocks, threads>>>(d, 64, 1.0000001, 1e-9);
    double best = 0;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        dfma_loop<<<blocks, threads>>>(d, iters, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { best = -1; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * 8 * iters * (double)blocks * threads;
        const double tf = fl / (ms * 1e-3) / 1e12;
        if (tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return best;
}
