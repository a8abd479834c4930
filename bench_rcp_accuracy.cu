// relative error of rcp.approx.ftz.f64 and of one / two Newton steps, vs 1/x
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/bench_rcp_accuracy bench_rcp_accuracy.cu && /tmp/bench_rcp_accuracy
#include <cstdio>
#include <cmath>
#include <cuda_runtime.h>
__global__ void k_acc(unsigned long long seed, int n, double lo_exp, double hi_exp, double *worst) {
    // worst[0..2]: max rel err raw, 1 step, 2 steps; per-block atomics avoided: one thread per slot
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    unsigned long long s = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(t + 1);
    s ^= s >> 31; s *= 0xBF58476D1CE4E5B9ull; s ^= s >> 27; s *= 0x94D049BB133111EBull; s ^= s >> 31;
    const double u = (double)(s >> 11) * 0x1p-53;
    const double x = exp2(lo_exp + (hi_exp - lo_exp) * u) * ((s & 1) ? -1.0 : 1.0);
    double r; asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double q = 1.0 / x;
    double e = fma(-x, r, 1.0);
    const double r1 = fma(r, e, r);
    e = fma(-x, r1, 1.0);
    const double r2 = fma(r1, e, r1);
    worst[3 * t + 0] = fabs(r - q) / fabs(q);
    worst[3 * t + 1] = fabs(r1 - q) / fabs(q);
    worst[3 * t + 2] = fabs(r2 - q) / fabs(q);
}
int main() {
    const int n = 1 << 22;
    double *w; cudaMalloc(&w, (size_t)3 * n * sizeof(double));
    double *h = new double[(size_t)3 * n];
    double ranges[3][2] = {{0, 1}, {-60, 60}, {-1000, 1000}};
    for (auto &rg : ranges) {
        k_acc<<<n / 256, 256>>>(12345, n, rg[0], rg[1], w);
        cudaMemcpy(h, w, (size_t)3 * n * sizeof(double), cudaMemcpyDeviceToHost);
        double m[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) for (int k = 0; k < 3; ++k) m[k] = fmax(m[k], h[3 * i + k]);
        printf("x in 2^[%g,%g): max rel err raw %.3e (2^%.2f), 1 Newton %.3e (2^%.2f), 2 Newton %.3e (2^%.2f)\n",
               rg[0], rg[1], m[0], log2(m[0]), m[1], log2(m[1]), m[2], log2(m[2]));
    }
    printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
