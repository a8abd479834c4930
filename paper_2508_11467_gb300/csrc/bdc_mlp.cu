// Training kernels of the root-start MLP (network and features in
// bdc_mlp.cuh).  The network is fitted on (features, r) pairs harvested from
// FP64 divide-and-conquer runs, r = y - y_q the gap between the logit of the
// converged root's position and its analytic estimate, with the Huber loss
//   loss = mean over samples of h(g - r),  h(u) = u^2/2 for |u| <= delta,
//   delta (|u| - delta/2) beyond  (delta <= 0: plain least squares),
// which keeps the rare roots that sit within an ulp of a pole (|r| up to 40)
// from dominating the fit.
//
//   k_mlp_init      feature means / inverse deviations (FP64 sums), Glorot
//                   uniform hidden weights from a counter-based generator,
//                   zero biases and a zero output layer (the untrained
//                   network leaves the analytic estimate unchanged).
//   k_mlp_grad      forward and backward over blocks of 64 samples held in
//                   shared memory; each CTA accumulates its gradient in
//                   registers and writes one partial row.
//   k_mlp_reduce    sums the partial rows in a fixed order (the gradient is
//                   deterministic for a given sample order).
//   k_mlp_adam      one Adam update (the normalisation entries stay).
//   k_mlp_predict   one thread per sample through the same inference code
//                   the root solver uses.
#include "bdc_internal.cuh"
#include "bdc_mlp.cuh"

namespace bdc {

namespace {

constexpr int kMB = 64;                 // samples per block
constexpr int kGT = 256;                // threads of the gradient kernel
constexpr int kPad = 65;                // row stride of the 64 x 64 activations
constexpr int kPAl = (kMlpParams + 3) & ~3;
constexpr int kGradSmemFloats = kPAl + 2 * kMlpH * kMlpH + kMB * kMlpIn + 4 * kMB * kPad + kMB;
// the float4 reads of W2 and its transpose need 16-byte aligned rows
static_assert(kPAl % 4 == 0 && kMlpH % 4 == 0, "shared-memory copies of W2 must stay 16-byte aligned");

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// ---------------------------------------------------------------- init
__global__ void __launch_bounds__(1024) k_mlp_init(float *__restrict__ P, const float *__restrict__ feat,
                                                   int count, unsigned long long seed) {
    __shared__ double red[32][2 * kMlpIn];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    double s1[kMlpIn], s2[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) s1[k] = s2[k] = 0.0;
    for (int i = t; i < count; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            const double v = feat[(size_t)i * kMlpIn + k];
            s1[k] += v;
            s2[k] = fma(v, v, s2[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) { s1[k] = warp_sum(s1[k]); s2[k] = warp_sum(s2[k]); }
    if (lane == 0) {
        for (int k = 0; k < kMlpIn; ++k) { red[w][k] = s1[k]; red[w][kMlpIn + k] = s2[k]; }
    }
    __syncthreads();
    if (t < kMlpIn) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[q][t]; b += red[q][kMlpIn + t]; }
        const double cnt = count > 0 ? (double)count : 1.0;
        const double mean = a / cnt;
        const double var = fmax(b / cnt - mean * mean, 0.0);
        P[kOffMean + t] = (float)mean;
        P[kOffIstd + t] = (float)(1.0 / fmax(sqrt(var), 1e-3));
    }
    if (t == 0) P[kOffB3] = 0.f;
    // Glorot-uniform hidden weights, zero biases and output layer
    for (int p = kOffW1 + t; p < kOffB3; p += blockDim.x) {
        float lim = 0.f;
        if (p < kOffB1) lim = sqrtf(6.f / (kMlpIn + kMlpH));
        else if (p >= kOffW2 && p < kOffB2) lim = sqrtf(6.f / (kMlpH + kMlpH));
        const unsigned long long r = mix64(seed * 0x100000001B3ull + (unsigned long long)p);
        const float u = (float)((double)(r >> 11) * 0x1.0p-53) * 2.f - 1.f;
        P[p] = lim * u;
    }
}

// ---------------------------------------------------------------- gradient
__global__ void __launch_bounds__(kGT) k_mlp_grad(const float *__restrict__ Pg, const float *__restrict__ feat,
                                                  const float *__restrict__ targ, int count, float huber,
                                                  float *__restrict__ part) {
    extern __shared__ __align__(16) float smf[];
    float *P = smf;                                  // parameters
    float *W2t = P + kPAl;                           // W2 transposed: W2t[k*64 + j] = W2[j][k]
    float *W2s = W2t + kMlpH * kMlpH;                // W2 row-major, 16-byte aligned rows
    float *X = W2s + kMlpH * kMlpH;                  // normalised inputs [64][kMlpIn]
    float *H1 = X + kMB * kMlpIn;                    // [64][kPad]
    float *H2 = H1 + kMB * kPad;
    float *D2 = H2 + kMB * kPad;                     // dL/dZ2
    float *D1 = D2 + kMB * kPad;                     // dL/dZ1
    float *dy = D1 + kMB * kPad;                     // dL/dy [64]
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;

    for (int p = t; p < kMlpParams; p += kGT) P[p] = Pg[p];
    for (int p = t; p < kMlpH * kMlpH; p += kGT) {
        const int j = p >> 6, k = p & 63;
        const float w = Pg[kOffW2 + p];
        W2t[k * kMlpH + j] = w;
        W2s[p] = w;
    }
    __syncthreads();

    const float inv_count = 1.f / (float)count;
    const int jg = t >> 2, kq = t & 3;               // gradient ownership
    float gW2[16], gW1[3], gv = 0.f, lsum = 0.f;   // gW1[c]: input kq + 4c (< kMlpIn)
#pragma unroll
    for (int c = 0; c < 16; ++c) gW2[c] = 0.f;
    gW1[0] = gW1[1] = gW1[2] = 0.f;
    const int sb = (t >> 4) * 4, cb = (t & 15) * 4;  // 4 x 4 output tile of the 64 x 64 products
    const int nblk = (count + kMB - 1) / kMB;

    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int base = blk * kMB;
        // inputs
        for (int q = t; q < kMB * kMlpIn; q += kGT) {
            const int s = q / kMlpIn, k = q - s * kMlpIn;
            const float v = (base + s < count) ? feat[(size_t)(base + s) * kMlpIn + k] : 0.f;
            X[q] = (v - P[kOffMean + k]) * P[kOffIstd + k];
        }
        __syncthreads();
        // layer 1
        {
            const int s = t >> 2;
#pragma unroll 4
            for (int q = 0; q < 16; ++q) {
                const int j = kq + 4 * q;
                float a = P[kOffB1 + j];
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) a = fmaf(P[kOffW1 + j * kMlpIn + k], X[s * kMlpIn + k], a);
                H1[s * kPad + j] = tanhf(a);
            }
        }
        __syncthreads();
        // layer 2: H2 = tanh(H1 W2^T + b2)
        {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = P[kOffB2 + cb + b];
#pragma unroll 4
            for (int k = 0; k < kMlpH; ++k) {
                const float4 wv = *reinterpret_cast<const float4 *>(W2t + k * kMlpH + cb);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float h = H1[(sb + a) * kPad + k];
                    acc[a][0] = fmaf(h, wv.x, acc[a][0]);
                    acc[a][1] = fmaf(h, wv.y, acc[a][1]);
                    acc[a][2] = fmaf(h, wv.z, acc[a][2]);
                    acc[a][3] = fmaf(h, wv.w, acc[a][3]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) H2[(sb + a) * kPad + cb + b] = tanhf(acc[a][b]);
        }
        __syncthreads();
        // output and dL/dy (warp w: samples 8w .. 8w+7)
        for (int q = 0; q < 8; ++q) {
            const int s = w * 8 + q;
            float o = H2[s * kPad + lane] * P[kOffW3 + lane] + H2[s * kPad + lane + 32] * P[kOffW3 + lane + 32];
            for (int sh = 16; sh > 0; sh >>= 1) o += __shfl_xor_sync(0xffffffffu, o, sh);
            if (lane == 0) {
                float g = 0.f;
                if (base + s < count) {
                    const float r = o + P[kOffB3] - targ[base + s];
                    if (huber > 0.f && fabsf(r) > huber) {
                        lsum += huber * (fabsf(r) - 0.5f * huber);
                        g = copysignf(huber, r) * inv_count;
                    } else {
                        lsum = fmaf(0.5f * r, r, lsum);
                        g = r * inv_count;
                    }
                }
                dy[s] = g;
            }
        }
        __syncthreads();
        // dZ2 = dy W3 (1 - H2^2)
        for (int q = t; q < kMB * kMlpH; q += kGT) {
            const int s = q >> 6, j = q & 63;
            const float h = H2[s * kPad + j];
            D2[s * kPad + j] = dy[s] * P[kOffW3 + j] * (1.f - h * h);
        }
        __syncthreads();
        // dZ1 = (dZ2 W2) (1 - H1^2)
        {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
            for (int j = 0; j < kMlpH; ++j) {
                const float4 wv = *reinterpret_cast<const float4 *>(W2s + j * kMlpH + cb);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float g = D2[(sb + a) * kPad + j];
                    acc[a][0] = fmaf(g, wv.x, acc[a][0]);
                    acc[a][1] = fmaf(g, wv.y, acc[a][1]);
                    acc[a][2] = fmaf(g, wv.z, acc[a][2]);
                    acc[a][3] = fmaf(g, wv.w, acc[a][3]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float h = H1[(sb + a) * kPad + cb + b];
                    D1[(sb + a) * kPad + cb + b] = acc[a][b] * (1.f - h * h);
                }
        }
        __syncthreads();
        // parameter gradients of this block
        for (int s = 0; s < kMB; ++s) {
            const float g2 = D2[s * kPad + jg], g1 = D1[s * kPad + jg];
#pragma unroll
            for (int c = 0; c < 16; ++c) gW2[c] = fmaf(g2, H1[s * kPad + kq * 16 + c], gW2[c]);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (kq + 4 * c < kMlpIn) gW1[c] = fmaf(g1, X[s * kMlpIn + kq + 4 * c], gW1[c]);
            if (kq == 0) gv += g2;                                  // b2[jg]
            else if (kq == 1) gv += g1;                             // b1[jg]
            else if (kq == 2) gv = fmaf(dy[s], H2[s * kPad + jg], gv);   // W3[jg]
            else if (jg == 0) gv += dy[s];                          // b3
        }
        __syncthreads();
    }
    float *out = part + (size_t)blockIdx.x * (kMlpParams + 1);
#pragma unroll
    for (int c = 0; c < 16; ++c) out[kOffW2 + jg * kMlpH + kq * 16 + c] = gW2[c];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (kq + 4 * c < kMlpIn) out[kOffW1 + jg * kMlpIn + kq + 4 * c] = gW1[c];
    if (kq == 0) out[kOffB2 + jg] = gv;
    else if (kq == 1) out[kOffB1 + jg] = gv;
    else if (kq == 2) out[kOffW3 + jg] = gv;
    else if (jg == 0) out[kOffB3] = gv;
    if (t < kOffW1) out[t] = 0.f;
    // loss: warp lane 0 values
    __shared__ float lred[kGT / 32];
    if (lane == 0) lred[w] = lsum;
    __syncthreads();
    if (t == 0) {
        float l = 0.f;
        for (int q = 0; q < kGT / 32; ++q) l += lred[q];
        out[kMlpParams] = l;
    }
}

__global__ void k_mlp_reduce(const float *__restrict__ part, int G, float *__restrict__ grad,
                             float *__restrict__ loss, int count) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    float a = 0.f;
    for (int g = 0; g < G; ++g) a += part[(size_t)g * (kMlpParams + 1) + p];
    if (p < kMlpParams) grad[p] = a;
    else if (loss) *loss = a / (float)count;
}

__global__ void k_mlp_zero(float *__restrict__ grad, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMlpParams) grad[p] = 0.f;
    if (p == 0 && loss) *loss = 0.f;
}

// ---------------------------------------------------------------- Adam
__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    const int p = kOffW1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMlpParams) return;
    const float gi = g[p];
    const float mi = b1 * m[p] + (1.f - b1) * gi;
    const float vi = b2 * v[p] + (1.f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    P[p] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// ---------------------------------------------------------------- inference
__global__ void __launch_bounds__(128) k_mlp_predict(const float *__restrict__ P, const float *__restrict__ feat,
                                                     int count, float *__restrict__ out) {
    __shared__ float Ps[kMlpParams];
    for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) Ps[p] = P[p];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float f[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) f[k] = feat[(size_t)i * kMlpIn + k];
    out[i] = mlp_predict_thread(Ps, f);
}

int grad_ctas(int count) {
    const int nblk = (count + kMB - 1) / kMB;
    return nblk < 152 ? (nblk > 0 ? nblk : 1) : 152;    // one CTA per SM (122 KB shared memory)
}

}  // namespace

size_t mlp_grad_workspace(int count) {
    return sizeof(float) * (size_t)grad_ctas(count) * (kMlpParams + 1);
}

cudaError_t launch_mlp_init(float *P, const float *feat, int count, unsigned long long seed,
                            cudaStream_t st) {
    k_mlp_init<<<1, 1024, 0, st>>>(P, feat, count, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float *P, const float *feat, const float *targ, int count, float huber,
                            float *grad, float *loss, float *work, cudaStream_t st) {
    if (count <= 0) {
        k_mlp_zero<<<(kMlpParams + 255) / 256, 256, 0, st>>>(grad, loss);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(float) * (size_t)kGradSmemFloats;
    cudaError_t ea = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
    const int G = grad_ctas(count);
    k_mlp_grad<<<G, kGT, smem, st>>>(P, feat, targ, count, huber, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_reduce<<<(kMlpParams + 1 + 255) / 256, 256, 0, st>>>(work, G, grad, loss, count);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *P, const float *grad, float *m, float *v, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st) {
    const float c1 = 1.f / (1.f - powf(b1, (float)step));
    const float c2 = 1.f / (1.f - powf(b2, (float)step));
    const int n = kMlpParams - kOffW1;
    k_mlp_adam<<<(n + 255) / 256, 256, 0, st>>>(P, grad, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_predict(const float *P, const float *feat, int count, float *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_mlp_predict<<<(unsigned)(((long long)count + 127) / 128), 128, 0, st>>>(P, feat, count, out);
    return cudaGetLastError();
}

int mlp_param_count() { return kMlpParams; }
int mlp_feature_count() { return kMlpIn; }

}  // namespace bdc
