// FP64 throughput vs active lanes; rcp.approx.f64 and cvt rates
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/bench_fp64_issue bench_fp64_issue.cu && /tmp/bench_fp64_issue
#include <cstdio>
#include <cuda_runtime.h>
constexpr int ITERS = 2048;
__global__ void k_dfma(double *out, int active, double a, double b) {
    double x[8];
    for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
    if ((threadIdx.x & 31) < active) {
        for (int it = 0; it < ITERS; ++it) {
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
        }
    }
    double s = 0; for (int q = 0; q < 8; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_rcp(double *out, int active) {
    double x[8];
    for (int q = 0; q < 8; ++q) x[q] = 1.5 + threadIdx.x * 1e-3 + q;
    if ((threadIdx.x & 31) < active) {
        for (int it = 0; it < ITERS; ++it) {
#pragma unroll
            for (int q = 0; q < 8; ++q) { double r; asm volatile("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x[q])); x[q] = r; }
        }
    }
    double s = 0; for (int q = 0; q < 8; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_cvt(double *out, int active) {
    double x[8];
    for (int q = 0; q < 8; ++q) x[q] = 1.5 + threadIdx.x * 1e-3 + q;
    if ((threadIdx.x & 31) < active) {
        for (int it = 0; it < ITERS; ++it) {
#pragma unroll
            for (int q = 0; q < 8; ++q) { float f; asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(x[q])); asm volatile("cvt.f64.f32 %0, %1;" : "=d"(x[q]) : "f"(f)); }
        }
    }
    double s = 0; for (int q = 0; q < 8; ++q) s += x[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
    int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int blocks = sms * 8, threads = 256;
    double *out; cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    const double warps = (double)blocks * threads / 32;
    for (int pass = 0; pass < 2; ++pass) {
        for (int act : {32, 16, 8, 4, 1}) {
            float ms;
            cudaEventRecord(e0); k_dfma<<<blocks, threads>>>(out, act, 0.999, 1e-3); cudaEventRecord(e1);
            cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
            double wi = warps * ITERS * 8;   // warp instructions
            printf("DFMA active=%2d: %.3f ms  warp-instr/clk/SM %.4f  lane-ops/clk/SM %.3f (at %d MHz)\n", act, ms,
                   wi / (ms * 1e-3 * clk * 1e3) / sms, wi * act / (ms * 1e-3 * clk * 1e3) / sms, clk / 1000);
            cudaEventRecord(e0); k_rcp<<<blocks, threads>>>(out, act); cudaEventRecord(e1);
            cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
            printf("RCP64 active=%2d: %.3f ms  warp-instr/clk/SM %.4f\n", act, ms, wi / (ms * 1e-3 * clk * 1e3) / sms);
            cudaEventRecord(e0); k_cvt<<<blocks, threads>>>(out, act); cudaEventRecord(e1);
            cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
            printf("CVT f64->f32->f64 pair active=%2d: %.3f ms  pairs warp-instr/clk/SM %.4f\n", act, ms, wi / (ms * 1e-3 * clk * 1e3) / sms);
        }
    }
    printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
