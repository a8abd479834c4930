// FP64 DFMA throughput probe: independent chains, all SMs busy.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/bench_fp64_peak bench_fp64_peak.cu && /tmp/bench_fp64_peak
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k_dfma(double *out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
int main() {
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int threads = 256;
    for (int per_sm : {4, 8}) {
        const int blocks = sms * per_sm;
        double *out = nullptr;
        cudaMalloc(&out, sizeof(double) * blocks * threads);
        const int iters = 1 << 14;
        k_dfma<<<blocks, threads>>>(out, 16, 0.999999, 1e-7);
        cudaDeviceSynchronize();
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0); cudaEventCreate(&e1);
        cudaEventRecord(e0);
        k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0; cudaEventElapsedTime(&ms, e0, e1);
        const double fmas = (double)blocks * threads * iters * 8;
        const double rate = fmas / (ms * 1e-3);
        printf("blocks/SM %d: %.3f ms, %.1f G DFMA/s = %.3f TFLOP/s, %.3f DFMA lane-ops/clk/SM at max clock %d MHz\n",
               per_sm, ms, rate / 1e9, 2 * rate / 1e12, rate / (sms * (clk * 1e3)), clk / 1000);
        cudaFree(out);
    }
    printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
