// Start points for the secular roots (Eq. M-svd-val): an analytic local
// estimate, the features of the small correcting MLP, its parameter layout
// and warp-level inference.  Shared by the root solver and the training
// kernels.
//
// Root i (0 <= i < N-1) lies in (d_i, d_{i+1}).  With D2 = d_{i+1}^2 - d_i^2
// its position is t = (w^2 - d_i^2) / D2 in (0, 1), held as the logit
// y = ln(t / (1 - t)).
//
// Analytic estimate y_q.  In t the secular function is
//   f = c(t) - a / t + b / (1 - t),  a = z_i^2 / D2,  b = z_{i+1}^2 / D2,
// with c(t) = 1 + (the sum over every other pole).  Freezing c at the
// interval midpoint m = (d_i + d_{i+1}) / 2 leaves a quadratic,
//   c t^2 - (c + a + b) t + a = 0,
// whose root in (0, 1) and its complement s = 1 - t are taken in
// cancellation-free form (both discriminants equal (c -+ a +- b)^2 + 4ab):
//   t = 2a / (p + sqrt(p^2 - 4ca))  or, for p < 0, (p - sqrt(..)) / (2c),
//   s = 2b / (q + sqrt(q^2 + 4cb))  or, for q < 0, (q - sqrt(..)) / (-2c),
//   p = c + a + b,  q = a + b - c,  y_q = ln t - ln s.
// c is estimated in O(1) per root: the kNear poles on each side exactly,
// every farther pole on a side through the first two moments of its z^2
// weights in d^2 (sum z^2 / (d^2 - m^2) ~ M / (mu - m^2) * (1 + var /
// (mu - m^2)^2), M = sum z^2, mu and var the z^2-weighted mean and variance
// of d^2), from prefix / suffix sums formed once per merge.
//
// MLP correction.  yhat = y_q + g(f), g an 11 -> 64 -> 64 -> 1 tanh network
// in FP32 on the features (each clamped to [-40, 40]):
//   f0 = ln a          f1 = ln b          f2 = ln(rho / D2), rho = sum z^2
//   f3 = ln(gap_{i-1} / gap_i)  (0 at i = 0)       gap_k = d_{k+1} - d_k
//   f4 = ln(gap_{i+1} / gap_i)  (0 at i = N-2)
//   f5 = ln(z_{i-1}^2 / D2)     (-40 at i = 0)
//   f6 = ln(z_{i+2}^2 / D2)     (-40 at i = N-2)
//   f7 = asinh(near-pole part of c - 1)   f8 = asinh(far-pole part)
//   f9 = y_q           f10 = d_i / d_{i+1}
// The last root (no right pole) always uses the plain start.
//
// Parameter vector (FP32, kMlpParams entries):
//   [0, 11) feature means, [11, 22) inverse standard deviations,
//   W1 64 x 11 (row j = hidden unit j), b1[64], W2 64 x 64, b2[64], W3[64], b3.
#pragma once
#include <cuda_runtime.h>

namespace bdc {

constexpr int kMlpIn = 11, kMlpH = 64, kMlpNear = 8;
constexpr int kOffMean = 0, kOffIstd = kMlpIn, kOffW1 = 2 * kMlpIn, kOffB1 = kOffW1 + kMlpH * kMlpIn,
              kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH, kOffW3 = kOffB2 + kMlpH,
              kOffB3 = kOffW3 + kMlpH, kMlpParams = kOffB3 + 1;

// z^2-weighted moments of the far poles on one side: sum z^2, sum z^2 d^2,
// sum z^2 d^4
struct FarSums {
    double m0, m1, m2;
};

__device__ __forceinline__ float clamp40(double v) { return (float)fmin(40.0, fmax(-40.0, v)); }

// second-moment estimate of sum over a far side of z^2 / (d^2 - m2)
__device__ __forceinline__ double far_part(const FarSums &s, double m2) {
    if (!(s.m0 > 0.0)) return 0.0;
    const double mu = s.m1 / s.m0;
    const double var = fmax(s.m2 / s.m0 - mu * mu, 0.0);
    const double den = mu - m2;
    if (!(fabs(den) > 0.0)) return 0.0;
    const double r = s.m0 / den * (1.0 + var / (den * den));
    return isfinite(r) ? r : 0.0;
}

// Features of root i (i < N - 1) of the sorted problem (d, z) and the
// analytic estimate y_q (FP64, unclamped); rho = sum z^2, L / R the far sums
// of poles j <= i - kNear - 1 and j >= i + kNear + 2.  One thread's work
// (FP64 is scarce: spread roots over threads, not one root over a warp).
__device__ __forceinline__ double mlp_features(const double *__restrict__ d, const double *__restrict__ z, int N,
                                               int i, double rho, const FarSums &L, const FarSums &R,
                                               float (&f)[kMlpIn]) {
    const double dl = d[i], du = d[i + 1];
    const double gap = du - dl, D2 = gap * (du + dl);
    const double m = 0.5 * (dl + du);
    const double a = z[i] * z[i] / D2, b = z[i + 1] * z[i + 1] / D2;
    double bn = 0.0;
    const int jlo = i - kMlpNear > 0 ? i - kMlpNear : 0;
    const int jhi = i + 1 + kMlpNear < N - 1 ? i + 1 + kMlpNear : N - 1;
    for (int j = jlo; j <= jhi; ++j) {
        if (j == i || j == i + 1) continue;
        const double dj = d[j];
        bn += z[j] * z[j] / ((dj - m) * (dj + m));
    }
    const double bf = far_part(L, m * m) + far_part(R, m * m);
    const double c = 1.0 + bn + bf;
    const double p = c + a + b, q = a + b - c;
    const double rp = sqrt(fmax(p * p - 4.0 * c * a, 0.0)), rq = sqrt(fmax(q * q + 4.0 * c * b, 0.0));
    const double t = (p >= 0.0) ? 2.0 * a / (p + rp) : (p - rp) / (2.0 * c);
    const double s = (q >= 0.0) ? 2.0 * b / (q + rq) : (q - rq) / (-2.0 * c);
    double yq = log(t) - log(s);
    if (!isfinite(yq)) yq = (yq > 0.0) ? 700.0 : -700.0;    // t or s underflowed
    yq = fmin(700.0, fmax(-700.0, yq));
    f[0] = clamp40(log(a));
    f[1] = clamp40(log(b));
    f[2] = clamp40(log(rho / D2));
    f[3] = (i >= 1) ? clamp40(log((dl - d[i - 1]) / gap)) : 0.f;
    f[4] = (i + 2 < N) ? clamp40(log((d[i + 2] - du) / gap)) : 0.f;
    f[5] = (i >= 1) ? clamp40(log(z[i - 1] * z[i - 1] / D2)) : -40.f;
    f[6] = (i + 2 < N) ? clamp40(log(z[i + 2] * z[i + 2] / D2)) : -40.f;
    f[7] = clamp40(asinh(bn));
    f[8] = clamp40(asinh(bf));
    f[9] = clamp40(yq);
    f[10] = (float)(dl / du);
    return yq;
}

// network output g(f) for one root, computed by one thread; P may sit in
// shared memory (all threads of a warp read the same weight: broadcast)
__device__ __forceinline__ float mlp_predict_thread(const float *__restrict__ P, const float (&f)[kMlpIn]) {
    float xn[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) xn[k] = (f[k] - P[kOffMean + k]) * P[kOffIstd + k];
    float h1[kMlpH];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float a = P[kOffB1 + j];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) a = fmaf(P[kOffW1 + j * kMlpIn + k], xn[k], a);
        h1[j] = tanhf(a);
    }
    float o = P[kOffB3];
#pragma unroll 2
    for (int j = 0; j < kMlpH; ++j) {
        float a = P[kOffB2 + j];
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) a = fmaf(P[kOffW2 + j * kMlpH + k], h1[k], a);
        o = fmaf(P[kOffW3 + j], tanhf(a), o);
    }
    return o;
}

}  // namespace bdc
