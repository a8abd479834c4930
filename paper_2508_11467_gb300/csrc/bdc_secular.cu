// Merge step of Algorithm 2, part (b) (lasd3 without the products):
//
// k_secular  one lane group per root of the secular equation (Eq. M-svd-val)
//            f(w) = 1 + sum_j z_j^2 / (d_j^2 - w^2), root i in (d_i, d_{i+1}).
//            The unknown is held relative to the nearer pole d_o as
//            x = w^2 - d_o^2 (then tau = w - d_o), so d_j^2 - w^2 is formed as
//            (d_j - d_o)(d_j + d_o) - x without cancellation.  Each step fits
//            the two nearest poles with a rational model matching f and f'
//            (a "middle way" step in the sense of R.-C. Li), solved for the
//            new iterate itself, safeguarded by a bracket; the last root
//            lumps the other poles at d_{N-2} and keeps its own exact.  An
//            FP32 pre-iteration starts the FP64 one.  The group's lanes (4
//            to 32, about 16 poles each) split the pole sums and reduce
//            with shuffles.
//            Stopping rule: |f| <= 16 eps (1 + sum |terms|), or a step below
//            4 eps |x|.  Optionally the start comes from a small MLP
//            (bdc_mlp.cuh) instead of the interval midpoint; the stopping
//            rule is the same, so the MLP only changes the iteration count.
// k_lowner   one lane group per i: |z~_i| of Eq. (bdc-zi) as a product over
//            k of (w_k^2 - d_i^2) / (d_{k'}^2 - d_i^2) (every factor lies in
//            (0, 1] by interlacing), lane partial products, then a shuffle
//            product reduction; sign from z_i.
// k_vectors_warp  one lane group per column i: v_i, u_i of Eq. (M-svd-vec),
//            normalised, written in the K order of the merge product.
//
// All arithmetic is in real_t: FP64, or FP32 in the FP32 build.  The root
// starts (k_root_start, bdc_mlp.cuh) and the standalone step kernels are
// FP64 only.
#include "bdc_internal.cuh"
#ifndef BDC_FP32
#include "bdc_mlp.cuh"
#endif

namespace BDC_NS {

namespace {

// A root (or Loewner product) is served by a group of G lanes (G = 4, 8,
// 16 or 32, aligned within the warp): the per-pole work is split over the
// group and the scalar steps of the iteration are shared by G lanes, not
// 32.  Group reductions shuffle within the group's own lanes.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    return ((1u << (G & 31)) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
    const unsigned m = group_mask<G>();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}
template <int G, typename T>
__device__ __forceinline__ T group_prod(T v) {
    const unsigned m = group_mask<G>();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v *= __shfl_xor_sync(m, v, o);
    return v;
}
// lanes per group for a merge with N survivors: about 16 poles per lane
// (at most 16 below G = 32: the vector kernel caches 16 entries per lane)
__host__ __device__ __forceinline__ int group_size(int N) {
    return N <= 64 ? 4 : N <= 128 ? 8 : N <= 256 ? 16 : 32;
}
static_assert(64 <= 4 * 16 && 128 <= 8 * 16 && 256 <= 16 * 16, "group_size must keep N <= 16 G below G = 32");
// Warps per node of the lane-group kernels for merges of order <= mmax: a
// warp serves 32 / G roots (columns), and G = group_size(N) <= group_size(mmax)
// for the device-side survivor count N <= mmax, so ceil(mmax / (32 / G(mmax)))
// warps cover every root of every node; launching mmax warps per node left
// most warps of the small merges with nothing to do.
__host__ __device__ __forceinline__ int group_warps(int mmax) {
    const int per = 32 / group_size(mmax);
    return (mmax + per - 1) / per;
}

// Lanes per root of the secular solve: about kSecPoles poles per lane.  An
// FP64 instruction costs its warp the same issue slot whatever the number of
// active lanes, so the scalar steps of an iteration (model, bracket, stopping
// test) cost a warp instruction per group of 32 / G roots: fewer lanes per
// root share them among more roots, at the price of a longer pole loop.
constexpr int kSecPoles = 16;
__host__ __device__ __forceinline__ int secular_group_size(int N) {
    return N <= 4 * kSecPoles ? 4 : N <= 8 * kSecPoles ? 8 : N <= 16 * kSecPoles ? 16 : 32;
}
// warps per node: ceil(N G(N) / 32) grows with N, so mmax bounds it
__host__ __device__ __forceinline__ int secular_group_warps(int mmax) {
    return (int)(((long long)mmax * secular_group_size(mmax) + 31) / 32);
}

// Warps per CTA of the lane-group kernels (k_secular, k_lowner,
// k_vectors_warp, k_rows_update).  Their grids hold the warps of every node's
// roots in node order, and deflation leaves only the first warps of a node
// with work, so small CTAs spread the working warps over more SMs and
// sub-partitions (each sub-partition issues one FP64 warp instruction per
// ~64 cycles).
constexpr int kLgWarps = 2;
constexpr int kLgThreads = 32 * kLgWarps;

struct Sums {
    real_t psi, dpsi, phi, dphi;
};

// Per-lane cache of the shifted poles lam_j = (d_j - d_o)(d_j + d_o) of a
// root's current origin o, in shared memory (column stride 32, up to
// kLamCache terms per lane): every pole sum at a new x of the same origin
// then forms d_j^2 - w^2 = lam_j - x with one subtraction instead of three
// FP64 operations.  (One more rounding than the fused form: lam_j - x
// cancels only for j = o, where lam_o = 0 exactly, or for a farther pole
// than the other interval pole, which the nearer-pole origin rules out.)
constexpr int kLamCache = 16;
struct LamCache {
    real_t *p;   // this lane's column (nullptr: no cache)
    int o;       // origin of the cached entries (-1: none)
};

// pole sums at x = w^2 - d_o^2; left group j <= k (psi), right j > k (phi).
// Interior roots split at k = i (psi < 0 < phi); the last root at k = N-2,
// so that phi is its origin pole's term alone.
template <int G>
__device__ __forceinline__ Sums pole_sums(const real_t *__restrict__ d, const real_t *__restrict__ z,
                                          int N, int k, int o, real_t dor, real_t x, int lane, LamCache &lc) {
    Sums s{R(0.0), R(0.0), R(0.0), R(0.0)};
    const bool use = lc.p != nullptr && lc.o == o, fill = lc.p != nullptr && !use;
    int t = 0;                                   // this lane's term number (its cache slot)
    auto shifted = [&](int j) -> real_t {
        if (use && t < kLamCache) return lc.p[32 * t];
        const real_t dj = d[j];
        const real_t lam = (dj - dor) * (dj + dor);
        if (fill && t < kLamCache) lc.p[32 * t] = lam;
        return lam;
    };
    if constexpr (G < 32) {
        // several roots per warp split their poles at different k: one loop
        // over all poles (the same trip count for every group of the warp)
        for (int j = lane; j < N; j += G, ++t) {
            const real_t zj = z[j];
            const real_t tq = quot(zj, shifted(j) - x);
            if (j <= k) {
                s.psi = fma(zj, tq, s.psi);
                s.dpsi = fma(tq, tq, s.dpsi);
            } else {
                s.phi = fma(zj, tq, s.phi);
                s.dphi = fma(tq, tq, s.dphi);
            }
        }
    } else {
        for (int j = lane; j <= k; j += G, ++t) {
            const real_t zj = z[j];
            const real_t tq = quot(zj, shifted(j) - x);
            s.psi = fma(zj, tq, s.psi);
            s.dpsi = fma(tq, tq, s.dpsi);
        }
        for (int j = k + 1 + lane; j < N; j += G, ++t) {
            const real_t zj = z[j];
            const real_t tq = quot(zj, shifted(j) - x);
            s.phi = fma(zj, tq, s.phi);
            s.dphi = fma(tq, tq, s.dphi);
        }
    }
    if (fill) lc.o = o;
    s.psi = group_sum<G>(s.psi);
    s.dpsi = group_sum<G>(s.dpsi);
    s.phi = group_sum<G>(s.phi);
    s.dphi = group_sum<G>(s.dphi);
    return s;
}

struct RootState {
    int o;                       // origin pole index
    real_t dor;                  // d_o
    real_t lo, hi;               // bracket for x = w^2 - d_o^2
    real_t lamL, lamR;           // the two interval poles relative to d_o^2
    real_t x;
    real_t dl, du;               // the interval poles d_i, d_{i+1}
    Sums s;
    LamCache lc;
};

// Next iterate from the rational model of f (Eq. M-svd-val) at x: psi's poles
// lumped into one at lamL and phi's into one at lamR, each matching value
// and slope at x, plus a constant C.  The model's quadratic is solved for
// the new iterate y itself, measured from the origin pole (one of lamL,
// lamR is 0, so the constant coefficient has a single term), rather than
// for a step from x: x + step would cancel for a root within eps |x| of
// its pole and leave only bisection to reach it.  An interior root takes
// the model root between lamL and lamR (the quadratic's smaller one); the
// last root (psi: every pole but the origin, lumped at lamL = d_{N-2}^2 -
// d_{N-1}^2; phi: the origin term alone, exact) the one right of 0.
// Returns NaN when the model has no such root.
// the model step's quotients: FP32 (the pre-iterations) as written, FP64 by
// the reciprocal-estimate quotient (within about an ulp; the iteration
// corrects its own rounding, the stopping rule is on f)
__device__ __forceinline__ float mdiv(float a, float b) { return a / b; }
#ifndef BDC_FP32
__device__ __forceinline__ double mdiv(double a, double b) { return quot(a, b); }
#endif

template <typename T>
__device__ __forceinline__ T model_next(T f, T dpsi, T dphi, T x, T lamL, T lamR, bool last) {
    const T DL = lamL - x, DR = lamR - x;
    const T sL = DL * DL * dpsi, sR = DR * DR * dphi;
    const T C = f - DL * dpsi - DR * dphi;
    const T a = C * (lamL + lamR) + sL + sR;
    const T b = sL * lamR + sR * lamL;
    if (!last) {
        if (C == T(0)) return mdiv(b, a);
        const T disc = sqrt(fabs(a * a - T(4) * b * C));
        return (a > T(0)) ? mdiv(T(2) * b, a + disc) : mdiv(a - disc, T(2) * C);
    }
    if (!(C > T(0))) return T(NAN);
    const T disc = sqrt(fabs(a * a - T(4) * b * C));
    return (a >= T(0)) ? mdiv(a + disc, T(2) * C) : mdiv(T(2) * b, a - disc);
}

// Safeguarded rational iteration from r.x; returns the iterations used or
// -1 when max_iter did not suffice.  All lanes return the same result.
template <int G>
__device__ __forceinline__ int root_iterate(const real_t *__restrict__ d, const real_t *__restrict__ z, int N, int i, bool last,
                            int max_iter, RootState &r) {
    const int lane = threadIdx.x & (G - 1);
    const int k = last ? i - 1 : i;
    int it = 0;
    for (;;) {
        const real_t f = R(1.0) + r.s.psi + r.s.phi;
        const real_t scale = R(1.0) + fabs(r.s.psi) + fabs(r.s.phi);
        if (fabs(f) <= R(16.0) * kEps * scale) break;
        if (f > R(0.0)) r.hi = r.x; else r.lo = r.x;
        if (it >= max_iter) return -1;
        real_t xn = model_next<real_t>(f, r.s.dpsi, r.s.dphi, r.x, r.lamL, r.lamR, last);
        if (!(xn > r.lo && xn < r.hi)) xn = R(0.5) * (r.lo + r.hi);
        const real_t step = xn - r.x;
        r.x = xn;
        ++it;
        if (!last) {
            // keep the origin at the nearer pole: an iterate past the interval
            // midpoint is re-expressed from the other pole (x and D2 are
            // within a factor 2, so x -+ D2 is exact); from the midpoint start
            // the bracket never crosses, from a predicted start it may
            const real_t D2 = r.lamR - r.lamL;
            if (r.o == i && r.x > R(0.5) * D2) {
                r.o = i + 1; r.dor = r.du; r.x -= D2; r.lo -= D2; r.hi -= D2; r.lamL = -D2; r.lamR = R(0.0);
            } else if (r.o == i + 1 && r.x < -R(0.5) * D2) {
                r.o = i; r.dor = r.dl; r.x += D2; r.lo += D2; r.hi += D2; r.lamL = R(0.0); r.lamR = D2;
            }
        }
        r.s = pole_sums<G>(d, z, N, k, r.o, r.dor, r.x, lane, r.lc);
        if (fabs(step) <= R(4.0) * kEps * fabs(r.x)) break;
    }
    return it;
}

// FP32 pre-iteration of root i from r.x: the same rational model and
// bracket as root_iterate, on FP32 copies of d and z, with the shifted
// differences of the two poles the model lumps at (j = k and k + 1: lamL
// and lamR) taken exactly from r.  FP32 runs on GB300 at ~80x the FP64
// rate, so this is nearly free; it stops at a relative step of 2^-17 (or
// after 16 steps, or where an FP32 sum overflows) and the FP64 iteration
// then finishes from there.  Other poles within ~2^-23 relative of the
// origin are only approximate in FP32: that costs FP64 steps, never
// accuracy.  Updates r.x (r.lo, r.hi untouched); all lanes agree.
template <int G>
__device__ __forceinline__ void fp32_phase(const float *__restrict__ d32, const float *__restrict__ z32, int N,
                                           int i, bool last, RootState &r) {
    const int lane = threadIdx.x & (G - 1);
    const int k = last ? i - 1 : i;
    const float lamL = (float)r.lamL, lamR = (float)r.lamR;
    const float dor = d32[r.o];
    float x = (float)r.x, lo = (float)r.lo, hi = (float)r.hi;
    for (int it = 0; it < 16; ++it) {
        float psi = 0.f, dpsi = 0.f, phi = 0.f, dphi = 0.f;
        for (int j = lane; j < N; j += G) {
            const float dj = d32[j], zj = z32[j];
            const float c = (j == k) ? lamL : (j == k + 1) ? lamR : (dj - dor) * (dj + dor);
            const float t = __fdividef(zj, c - x);   // approximate: this phase only starts the FP64 one
            if (j <= k) { psi = fmaf(zj, t, psi); dpsi = fmaf(t, t, dpsi); }
            else { phi = fmaf(zj, t, phi); dphi = fmaf(t, t, dphi); }
        }
        psi = group_sum<G>(psi); dpsi = group_sum<G>(dpsi); phi = group_sum<G>(phi); dphi = group_sum<G>(dphi);
        const float f = 1.f + psi + phi;
        if (!(fabsf(f) + dpsi + dphi < INFINITY)) break;   // no usable FP32 information at x
        if (f > 0.f) hi = x; else lo = x;
        float xn = model_next<float>(f, dpsi, dphi, x, lamL, lamR, last);
        if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
        const float step = xn - x;
        x = xn;
        if (fabsf(step) <= 0x1p-17f * fabsf(x)) break;
    }
    const real_t xd = (real_t)x;
    if (xd > r.lo && xd < r.hi) r.x = xd;
}

// Solve root i of (d, z) (N entries, d[0] = 0 < d[1] < ...).  Returns the
// number of iterations used, or -1 if not converged.  All lanes return the
// same result.  vstart (NaN = none) is a predicted start (start_fraction of
// a predicted logit, see bdc_mlp.cuh); with it the solver starts there
// instead of evaluating the interval midpoint.  d32, z32 (nullptr = none):
// FP32 copies for fp32_phase, which then also replaces the FP64 midpoint
// evaluation that picks the origin.  A start that may sit on the farther
// half is polished from the nearer pole at the end.
template <int G>
__device__ __forceinline__ int solve_root(const real_t *__restrict__ d, const real_t *__restrict__ z, int N, int i,
                          int max_iter, real_t zz, int &org_out, real_t &tau_out, real_t &x_out, real_t vstart,
                          const float *__restrict__ d32 = nullptr, const float *__restrict__ z32 = nullptr,
                          real_t *lam_cache = nullptr) {
    const int lane = threadIdx.x & (G - 1);
    if (N == 1) {
        org_out = 0;
        tau_out = fabs(z[0]);
        x_out = tau_out * tau_out;
        return 0;
    }
    const bool last = (i == N - 1);
    const real_t dl = d[i];
    const real_t du = last ? sqrt(dl * dl + zz) : d[i + 1];
    const real_t h = R(0.5) * (du - dl);
    const bool pre32 = d32 != nullptr;
    const bool use_mlp = !last && ((vstart == vstart) || pre32);
    RootState r;
    r.dl = dl;
    r.du = du;
    r.lc = LamCache{lam_cache, -1};
    if (pre32 && !last && !(vstart == vstart)) {
        // FP32 sign at the interval midpoint picks the origin (a wrong pick
        // near the midpoint is repaired by the origin switch)
        const float xm = (float)(h * (R(2.0) * dl + h)), D2f = (float)((du - dl) * (du + dl));
        const float di = (float)dl;
        float s = 0.f;
        for (int j = lane; j < N; j += G) {
            const float dj = d32[j], zj = z32[j];
            const float c = (j == i) ? 0.f : (j == i + 1) ? D2f : (dj - di) * (dj + di);
            s = fmaf(zj, __fdividef(zj, c - xm), s);
        }
        s = group_sum<G>(s);
        vstart = (1.f + s >= 0.f) ? R(0.25) : R(-0.25);     // the midpoint seen from the chosen pole
    }
    if (use_mlp) {
        const real_t D2 = (du - dl) * (du + dl);
        if (vstart > R(0.0)) {
            r.o = i; r.dor = dl; r.lo = R(0.0); r.hi = D2; r.lamL = R(0.0); r.lamR = D2; r.x = vstart * D2;
        } else {
            r.o = i + 1; r.dor = du; r.lo = -D2; r.hi = R(0.0); r.lamL = -D2; r.lamR = R(0.0); r.x = vstart * D2;
        }
        if (!(r.x > r.lo && r.x < r.hi)) r.x = R(0.5) * (r.lo + r.hi);
        if (pre32) fp32_phase<G>(d32, z32, N, i, false, r);
        r.s = pole_sums<G>(d, z, N, i, r.o, r.dor, r.x, lane, r.lc);
    } else if (!last) {
        // sign of f at the interval midpoint picks the nearer pole as origin
        const real_t xmid = h * (R(2.0) * dl + h);
        r.s = pole_sums<G>(d, z, N, i, i, dl, xmid, lane, r.lc);
        const real_t fmid = R(1.0) + r.s.psi + r.s.phi;
        if (fmid >= R(0.0)) {
            r.o = i; r.dor = dl; r.lo = R(0.0); r.hi = xmid;
            r.lamL = R(0.0); r.lamR = (du - dl) * (du + dl);
            r.x = xmid;
        } else {
            r.o = i + 1; r.dor = du; r.lo = -h * (R(2.0) * du - h); r.hi = R(0.0);
            r.lamL = -(du - dl) * (du + dl); r.lamR = R(0.0);
            r.x = r.lo;                    // the same point, measured from d_{i+1}
        }
    } else {
        // last root, w in (d_{N-1}, sqrt(d_{N-1}^2 + |z|^2)): origin d_{N-1};
        // the other poles lumped at d_{N-2}^2 - d_{N-1}^2
        const real_t dp = d[i - 1];
        r.o = i; r.dor = dl; r.lo = R(0.0); r.hi = zz;
        r.lamL = -(dl - dp) * (dl + dp); r.lamR = R(0.0);
        r.x = R(0.5) * zz;
        if (pre32) fp32_phase<G>(d32, z32, N, i, true, r);
        r.s = pole_sums<G>(d, z, N, i - 1, r.o, r.dor, r.x, lane, r.lc);
    }
    int it = root_iterate<G>(d, z, N, i, last, max_iter, r);
    if (use_mlp && it >= 0) {
        // the origin must be the nearer pole (no cancellation in d_j - w)
        const real_t D2 = (du - dl) * (du + dl);
        bool sw = false;
        if (r.o == i && r.x > R(0.5) * D2) {
            r.o = i + 1; r.dor = du; r.x -= D2; r.lo = -D2; r.hi = R(0.0); r.lamL = -D2; r.lamR = R(0.0); sw = true;
        } else if (r.o == i + 1 && r.x < -R(0.5) * D2) {
            r.o = i; r.dor = dl; r.x += D2; r.lo = R(0.0); r.hi = D2; r.lamL = R(0.0); r.lamR = D2; sw = true;
        }
        if (sw) {
            if (!(r.x > r.lo && r.x < r.hi)) r.x = R(0.5) * (r.lo + r.hi);
            r.s = pole_sums<G>(d, z, N, i, r.o, r.dor, r.x, lane, r.lc);
            const int it2 = root_iterate<G>(d, z, N, i, last, max_iter, r);
            it = (it2 < 0) ? -1 : it + 1 + it2;
        }
    }
    org_out = r.o;
    x_out = r.x;
    // tau = w - d_o from x = (w - d_o)(w + d_o)
    tau_out = r.x / (r.dor + sqrt(r.dor * r.dor + r.x));
    return it;
}

#ifndef BDC_FP32   // root starts: FP64 only
// far-pole moment sums of root i from the merge's prefix (poles j <= i-9)
// and suffix (poles j >= i+10) sums
__device__ __forceinline__ void far_from_scans(const double *__restrict__ pz, long long stride, int N, int i,
                                               FarSums &L, FarSums &R) {
    const int jl = i - kMlpNear - 1, jr = i + kMlpNear + 2;
    L = (jl >= 0) ? FarSums{pz[jl], pz[stride + jl], pz[2 * stride + jl]} : FarSums{0.0, 0.0, 0.0};
    R = (jr <= N - 1) ? FarSums{pz[3 * stride + jr], pz[4 * stride + jr], pz[5 * stride + jr]}
                      : FarSums{0.0, 0.0, 0.0};
}

// the same sums formed directly by one warp (standalone entry points)
__device__ __forceinline__ void far_direct(const double *__restrict__ d, const double *__restrict__ z, int N,
                                           int i, int lane, FarSums &L, FarSums &R) {
    double l0 = 0.0, l1 = 0.0, l2 = 0.0, r0 = 0.0, r1 = 0.0, r2 = 0.0;
    for (int j = lane; j < N; j += 32) {
        const double z2 = z[j] * z[j], d2 = d[j] * d[j];
        if (j <= i - kMlpNear - 1) { l0 += z2; l1 += z2 * d2; l2 += z2 * d2 * d2; }
        if (j >= i + kMlpNear + 2) { r0 += z2; r1 += z2 * d2; r2 += z2 * d2 * d2; }
    }
    L = FarSums{warp_sum(l0), warp_sum(l1), warp_sum(l2)};
    R = FarSums{warp_sum(r0), warp_sum(r1), warp_sum(r2)};
}

// natural log of a positive FP64 value to FP32 accuracy without a call:
// exponent from the bits, FP32 log of the mantissa in [1, 2)
__device__ __forceinline__ double log_approx(double v) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0 || ex == 0x7ff) return (v > 0.0 && ex == 0x7ff) ? 1e300 : -1e300;   // 0, subnormal, inf
    const double mant = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
    return (double)(ex - 1023) * 0.6931471805599453 + (double)__logf((float)mant);
}

// logit of the converged root's position, from x relative to its origin
__device__ __forceinline__ double root_logit(int o, int i, double x, double D2) {
    return (o == i) ? log_approx(x) - log_approx(D2 - x) : log_approx(D2 + x) - log_approx(-x);
}

// start fraction of a predicted logit y: +t for t = sigmoid(y) <= 1/2
// (origin d_i, x = t D2), -(1 - t) otherwise (origin d_{i+1}, x = -(1-t) D2)
// The logit is limited to +-36 (t >= 2e-16): a start closer to a pole than
// that gains nothing and can leave the root finder crawling back.
__device__ __forceinline__ double start_fraction(double y) {
    const double ey = exp(-fmin(fabs(y), 36.0));
    const double small = ey / (1.0 + ey);
    return (y <= 0.0) ? small : -small;
}

// The analytic start alone (no network, no harvest), in FP32 on the FP32
// copies of the survivors: the same estimate as y_q in mlp_features (near
// poles exact, far poles by their moments, the quadratic in cancellation-free
// form), returned as the start fraction without forming the logit:
// sigmoid(ln(t / s)) = t / (t + s).  The FP32 root pre-iteration that follows
// works at the same precision; a start that is not finite means "no start".
__device__ __forceinline__ double start_analytic32(const float *__restrict__ d, const float *__restrict__ z,
                                                   int N, int i, const FarSums &L, const FarSums &Rs) {
    const float dl = d[i], du = d[i + 1];
    const float gap = du - dl, D2 = gap * (du + dl);
    const float m = 0.5f * (dl + du), m2 = m * m;
    const float a = z[i] * z[i] / D2, b = z[i + 1] * z[i + 1] / D2;
    float bn = 0.f;
    const int jlo = i - kMlpNear > 0 ? i - kMlpNear : 0;
    const int jhi = i + 1 + kMlpNear < N - 1 ? i + 1 + kMlpNear : N - 1;
    for (int j = jlo; j <= jhi; ++j) {
        if (j == i || j == i + 1) continue;
        const float dj = d[j];
        bn += z[j] * z[j] / ((dj - m) * (dj + m));
    }
    auto far32 = [&](const FarSums &s) {
        const float m0 = (float)s.m0;
        if (!(m0 > 0.f)) return 0.f;
        const float mu = (float)s.m1 / m0;
        const float var = fmaxf((float)s.m2 / m0 - mu * mu, 0.f);
        const float den = mu - m2;
        if (!(fabsf(den) > 0.f)) return 0.f;
        const float r = m0 / den * (1.f + var / (den * den));
        return isfinite(r) ? r : 0.f;
    };
    const float c = 1.f + bn + far32(L) + far32(Rs);
    const float p = c + a + b, q = a + b - c;
    const float rp = sqrtf(fmaxf(p * p - 4.f * c * a, 0.f)), rq = sqrtf(fmaxf(q * q + 4.f * c * b, 0.f));
    const float t = (p >= 0.f) ? 2.f * a / (p + rp) : (p - rp) / (2.f * c);
    const float sc = (q >= 0.f) ? 2.f * b / (q + rq) : (q - rq) / (-2.f * c);
    const float tot = t + sc;
    if (!(t > 0.f && sc > 0.f && isfinite(tot))) return __longlong_as_double(0x7ff8000000000000ll);
    constexpr float kMin = 2.3195228e-16f;           // sigmoid(-36): the logit is limited to +-36
    return (t <= sc) ? (double)fmaxf(t / tot, kMin) : -(double)fmaxf(sc / tot, kMin);
}

// Start of every root but each merge's last: one thread per root computes
// the features and the analytic estimate y_q, and with an MLP the corrected
// start y_q + g (weights staged in shared memory).  Writes ystart (and,
// when harvesting, the features and y_q for k_secular to append).  The
// analytic start alone takes start_analytic32.
__global__ void __launch_bounds__(128) k_root_start(const NodeDesc *__restrict__ nodes,
                                                    const MatDesc *__restrict__ mats,
                                                    const NodeState *__restrict__ state, int mmax, int nnodes,
                                                    int seed_mode, const float *__restrict__ mlp) {
    extern __shared__ float Ps[];
    const bool use_net = (seed_mode == BDC_SEED_MLP);
    if (use_net) {
        for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) Ps[p] = mlp[p];
        __syncthreads();
    }
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int node = (int)(idx / mmax), i = (int)(idx % mmax);
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const int N = state[nd.id].N;
    if (i >= N - 1) return;
    const MatDesc &md = mats[nd.mat];
    const double *d = md.dM + nd.r0, *z = md.zM + nd.r0;
    FarSums L, R;
    far_from_scans(md.pz + nd.r0, md.n, N, i, L, R);
    if (seed_mode == BDC_SEED_ANALYTIC && md.feat == nullptr) {
        md.ystart[nd.r0 + i] = start_analytic32(md.d32 + nd.r0, md.z32 + nd.r0, N, i, L, R);
        return;
    }
    float f[kMlpIn];
    const double yq = mlp_features(d, z, N, i, state[nd.id].rho, L, R, f);
    double ys = yq;
    if (use_net) ys += (double)mlp_predict_thread(Ps, f);
    md.ystart[nd.r0 + i] = start_fraction(ys);
    if (md.feat != nullptr) {
        md.yq[nd.r0 + i] = yq;
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) md.fs[(size_t)(nd.r0 + i) * kMlpIn + k] = f[k];
    }
}
#endif  // BDC_FP32

// root i of one merge by a group of G lanes
template <int G>
__device__ __forceinline__ void secular_group(const NodeDesc &nd, const MatDesc &md, NodeState *__restrict__ state,
                                              int N, real_t zz, int i, int max_iter, int seed_mode,
                                              int fp32_start, real_t *lam_cache) {
    const real_t *d = md.dM + nd.r0, *z = md.zM + nd.r0;
    real_t vstart = R(NAN);                                    // NaN: plain start
    if (seed_mode != BDC_SEED_PLAIN && i < N - 1) vstart = md.ystart[nd.r0 + i];
    int o;
    real_t tau, x;
    const int it = solve_root<G>(d, z, N, i, max_iter, zz, o, tau, x, vstart,
                                 fp32_start ? md.d32 + nd.r0 : nullptr, fp32_start ? md.z32 + nd.r0 : nullptr,
                                 lam_cache);
    if ((threadIdx.x & (G - 1)) == 0) {
        md.org[nd.r0 + i] = o;
        md.tau[nd.r0 + i] = tau;
        md.omega[nd.r0 + i] = d[o] + tau;
        if (it < 0) atomicAdd(md.info, 1);
        atomicAdd(&state[nd.id].iters, (unsigned long long)(it < 0 ? max_iter : it));
#ifndef BDC_FP32
        if (md.feat != nullptr && i < N - 1 && it >= 0) {
            // harvest (features, y - y_q): the network learns the correction
            const double D2 = (d[i + 1] - d[i]) * (d[i + 1] + d[i]);
            const int slot = atomicAdd(md.hcount, 1);
            if (slot < md.hcap) {
                const float *fr = md.fs + (size_t)(nd.r0 + i) * kMlpIn;
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) md.feat[(size_t)slot * kMlpIn + k] = fr[k];
                md.targ[slot] = clamp40(root_logit(o, i, x, D2) - md.yq[nd.r0 + i]);
            }
        }
#endif
    }
}

// Warp w of a node (secular_group_warps(mmax) per node) serves roots w * (32 / G) + (lane / G),
// G = secular_group_size(N) from the node's survivor count, known only here.
__global__ void __launch_bounds__(kLgThreads, 16 / kLgWarps) k_secular(const NodeDesc *__restrict__ nodes,
                                                 const MatDesc *__restrict__ mats,
                                                 NodeState *__restrict__ state, int wpn,
                                                 int max_iter, int nnodes, int seed_mode, int fp32_start) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / wpn, w = warp % wpn;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    const int N = ns.N, G = secular_group_size(N), per = 32 / G;
    const int i = w * per + lane / G;
    if (i >= N) return;                              // whole groups leave together
    const MatDesc &md = mats[nd.mat];
    const real_t zz = ns.rho;                        // sum z^2 (computed by the merge prep)
    __shared__ real_t s_lam[kLgWarps][kLamCache * 32];   // shifted poles of each lane's root (pole_sums)
    real_t *lc = &s_lam[threadIdx.x >> 5][lane];
    switch (G) {
    case 4: secular_group<4>(nd, md, state, N, zz, i, max_iter, seed_mode, fp32_start, lc); break;
    case 8: secular_group<8>(nd, md, state, N, zz, i, max_iter, seed_mode, fp32_start, lc); break;
    case 16: secular_group<16>(nd, md, state, N, zz, i, max_iter, seed_mode, fp32_start, lc); break;
    default: secular_group<32>(nd, md, state, N, zz, i, max_iter, seed_mode, fp32_start, lc); break;
    }
}

#ifndef BDC_FP32   // standalone step kernels: FP64 only
__device__ __forceinline__ double warp_sumsq(const double *__restrict__ z, int N, int lane) {
    double zz = 0.0;
    for (int j = lane; j < N; j += 32) zz = fma(z[j], z[j], zz);
    return warp_sum(zz);
}

__global__ void __launch_bounds__(256, 2) k_secular_single(int N, const double *d, const double *z, int *org,
                                                        double *tau, double *omega, int max_iter,
                                                        int *info, int seed_mode, const float *__restrict__ mlp,
                                                        int *iters) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= N) return;
    const bool need_rho = (i == N - 1) || seed_mode != BDC_SEED_PLAIN;
    const double zz = need_rho ? warp_sumsq(z, N, lane) : 0.0;
    double ystart = __longlong_as_double(0x7ff8000000000000ll);
    if (seed_mode != BDC_SEED_PLAIN && i < N - 1) {
        float f[kMlpIn];
        FarSums L, R;
        far_direct(d, z, N, i, lane, L, R);
        const double yq = mlp_features(d, z, N, i, zz, L, R, f);
        ystart = start_fraction((seed_mode == BDC_SEED_MLP) ? yq + (double)mlp_predict_thread(mlp, f) : yq);
    }
    int o;
    double t, x;
    const int it = solve_root<32>(d, z, N, i, max_iter, zz, o, t, x, ystart);
    if (lane == 0) {
        org[i] = o;
        tau[i] = t;
        omega[i] = d[o] + t;
        if (iters) iters[i] = it;
        if (it < 0) atomicAdd(info, 1);
    }
}

// features and analytic estimates of roots 0..N-2 of one secular problem
__global__ void __launch_bounds__(256) k_mlp_features_single(int N, const double *d, const double *z,
                                                             float *feat, double *yq_out) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= N - 1) return;
    const double zz = warp_sumsq(z, N, lane);
    FarSums L, R;
    far_direct(d, z, N, i, lane, L, R);
    float f[kMlpIn];
    const double yq = mlp_features(d, z, N, i, zz, L, R, f);
    if (lane < kMlpIn) {
        float v = f[0];
#pragma unroll
        for (int k = 1; k < kMlpIn; ++k) if (lane == k) v = f[k];
        feat[(size_t)i * kMlpIn + lane] = v;
    }
    if (lane == 0 && yq_out) yq_out[i] = yq;
}

#endif  // BDC_FP32

// |z~_i|^2 of Eq. (bdc-zi), 0-based: (w_{N-1}^2 - d_i^2) *
//   prod_{k<i} (w_k^2 - d_i^2)/(d_k^2 - d_i^2) * prod_{i<=k<N-1} (w_k^2 - d_i^2)/(d_{k+1}^2 - d_i^2)
// by a group of G lanes.  FP64: numerators and denominators are multiplied
// separately and divided once per 8 factors (by the reciprocal-estimate
// quotient `quot`: four FP64 operations where a division costs about nine on
// GB300), sooner when either product falls below
// 2^-300; every factor of the product lies in (0, 1] by interlacing.
template <int G>
__device__ __forceinline__ real_t lowner_one(const real_t *__restrict__ d, const real_t *__restrict__ z,
                                             const int *__restrict__ org, const real_t *__restrict__ tau,
                                             const real_t *__restrict__ omega, int N, int i, int lane) {
    const real_t di = d[i];
    real_t prod = R(1.0);
#ifdef BDC_FP32
    for (int k = lane; k < N - 1; k += G) {
        const int ok = org[k];
        const real_t wmd = (d[ok] - di) + tau[k];        // w_k - d_i
        const real_t wpd = d[ok] + tau[k] + di;          // w_k + d_i
        const int kk = (k < i) ? k : k + 1;
        const real_t den = (d[kk] - di) * (d[kk] + di);
        prod *= (wmd * wpd) / den;
    }
#else
    double num = 1.0, den = 1.0;
    int cnt = 0;
    constexpr long long kLow = (long long)(1023 - 300) << 52;   // bits of 2^-300
    for (int k = lane; k < N - 1; k += G) {
        const int ok = org[k];
        const double wmd = (d[ok] - di) + tau[k];        // w_k - d_i
        const double wpd = (omega ? omega[k] : d[ok] + tau[k]) + di;   // w_k + d_i
        const int kk = (k < i) ? k : k + 1;
        num *= wmd * wpd;
        den *= (d[kk] - di) * (d[kk] + di);
        if (++cnt == 8 || (__double_as_longlong(num) & 0x7fffffffffffffffll) < kLow ||
            (__double_as_longlong(den) & 0x7fffffffffffffffll) < kLow) {
            prod *= quot(num, den);
            num = den = 1.0;
            cnt = 0;
        }
    }
    if (cnt) prod *= quot(num, den);
#endif
    prod = group_prod<G>(prod);
    const int oN = org[N - 1];
    const real_t last = ((d[oN] - di) + tau[N - 1]) * (d[oN] + tau[N - 1] + di);
    const real_t zt = sqrt(fabs(last * prod));
    return (z[i] < R(0.0)) ? -zt : zt;
}

__global__ void __launch_bounds__(kLgThreads) k_lowner(const NodeDesc *__restrict__ nodes,
                                                const MatDesc *__restrict__ mats,
                                                const NodeState *__restrict__ state, int wpn, int nnodes) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / wpn, w = warp % wpn;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    const int N = ns.N, G = group_size(N), per = 32 / G;
    const int i = w * per + lane / G;
    if (i >= N) return;                              // whole groups leave together
    const MatDesc &md = mats[nd.mat];
    const int r0 = nd.r0, gl = lane & (G - 1);
    const real_t *d = md.dM + r0, *z = md.zM + r0, *tau = md.tau + r0;
    const int *org = md.org + r0;
    real_t zt;
    switch (G) {
    case 4: zt = lowner_one<4>(d, z, org, tau, md.omega + r0, N, i, gl); break;
    case 8: zt = lowner_one<8>(d, z, org, tau, md.omega + r0, N, i, gl); break;
    case 16: zt = lowner_one<16>(d, z, org, tau, md.omega + r0, N, i, gl); break;
    default: zt = lowner_one<32>(d, z, org, tau, md.omega + r0, N, i, gl); break;
    }
    if (gl == 0) md.zt[r0 + i] = zt;
}

#ifndef BDC_FP32
__global__ void __launch_bounds__(256) k_lowner_single(int N, const double *d, const double *z,
                                                       const int *org, const double *tau, double *zt) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= N) return;
    const double v = lowner_one<32>(d, z, org, tau, nullptr, N, i, lane);
    if (lane == 0) zt[i] = v;
}
#endif

#ifndef BDC_FP32   // the single-problem vector kernel: FP64 only
__device__ __forceinline__ real_t block_sum256(real_t v, real_t *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    real_t r = R(0.0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    __syncthreads();
    return r;
}

// column i of U_M and V_M, rows in K order (invK: K position -> M index, -1 =
// zero row; nullptr = identity), one CTA (standalone step entry point)
__device__ void vectors_one(const real_t *__restrict__ d, const real_t *__restrict__ zt, int N, int i,
                            int o, real_t tau, const int *__restrict__ invK, int Ktot,
                            real_t *__restrict__ UMcol, real_t *__restrict__ VMcol, real_t *sh) {
    const real_t dor = d[o];
    const real_t wsum = dor + tau;   // w_i: d_j + w_i formed once per entry (a sum of positives)
    real_t sv = R(0.0), su = R(0.0);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const real_t dj = d[j];
        const real_t v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
        const real_t u = (j == 0) ? -R(1.0) : dj * v;
        sv = fma(v, v, sv);
        su = fma(u, u, su);
    }
    sv = block_sum256(sv, sh);
    su = block_sum256(su, sh);
    const real_t iv = R(1.0) / sqrt(sv), iu = R(1.0) / sqrt(su);
    for (int p = threadIdx.x; p < Ktot; p += blockDim.x) {
        const int j = invK ? invK[p] : p;
        real_t uo = R(0.0), vo = R(0.0);
        if (j >= 0) {
            const real_t dj = d[j];
            const real_t v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
            vo = v * iv;
            uo = ((j == 0) ? -R(1.0) : dj * v) * iu;
        }
        UMcol[p] = uo;
        VMcol[p] = vo;
    }
}

#endif  // BDC_FP32

// The same with a lane group per column (G = 4 to 32 lanes, about 16 rows
// each), for heights whose merges have N <= 1024 survivors: each lane keeps
// its entries v_j (j = lane, lane + G, ...) in registers between the norm and
// the write, so every entry costs one division; rows are written at their K
// positions (kposM), the padding rows [n1, P1) of the K order as zeros.
template <int G, int T>
__device__ __forceinline__ void vectors_group(const real_t *__restrict__ d, const real_t *__restrict__ zt,
                                              const int *__restrict__ kpos, int N, int n1, int P1, real_t dor,
                                              real_t tau, real_t *__restrict__ UMcol, real_t *__restrict__ VMcol,
                                              int gl, bool wu) {
    const real_t wsum = dor + tau;   // w_i: d_j + w_i formed once per entry (a sum of positives)
    real_t vr[T];
    real_t sv = R(0.0), su = R(0.0);
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int j = gl + t * G;
        real_t v = R(0.0);
        if (j < N) {
            const real_t dj = d[j];
            v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
            const real_t u = (j == 0) ? -R(1.0) : dj * v;
            sv = fma(v, v, sv);
            su = fma(u, u, su);
        }
        vr[t] = v;
    }
    sv = group_sum<G>(sv);
    su = group_sum<G>(su);
    const real_t iv = R(1.0) / sqrt(sv), iu = R(1.0) / sqrt(su);
    for (int p = n1 + gl; p < P1; p += G) {
        if (wu) UMcol[p] = R(0.0);
        VMcol[p] = R(0.0);
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int j = gl + t * G;
        if (j < N) {
            const int kp = kpos[j];
            VMcol[kp] = vr[t] * iv;
            if (wu) UMcol[kp] = ((j == 0) ? -R(1.0) : d[j] * vr[t]) * iu;
        }
    }
}

// the same for N > 32 * 32 survivors (a warp per column, entries recomputed
// for the write instead of cached)
__device__ __forceinline__ void vectors_warp_long(const real_t *__restrict__ d, const real_t *__restrict__ zt,
                                                  const int *__restrict__ kpos, int N, int n1, int P1, real_t dor,
                                                  real_t tau, real_t *__restrict__ UMcol,
                                                  real_t *__restrict__ VMcol, int lane, bool wu) {
    const real_t wsum = dor + tau;   // w_i: d_j + w_i formed once per entry (a sum of positives)
    real_t sv = R(0.0), su = R(0.0);
    for (int j = lane; j < N; j += 32) {
        const real_t dj = d[j];
        const real_t v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
        const real_t u = (j == 0) ? -R(1.0) : dj * v;
        sv = fma(v, v, sv);
        su = fma(u, u, su);
    }
    sv = warp_sum(sv);
    su = warp_sum(su);
    const real_t iv = R(1.0) / sqrt(sv), iu = R(1.0) / sqrt(su);
    for (int p = n1 + lane; p < P1; p += 32) {
        if (wu) UMcol[p] = R(0.0);
        VMcol[p] = R(0.0);
    }
    for (int j = lane; j < N; j += 32) {
        const real_t dj = d[j];
        const real_t v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
        const int kp = kpos[j];
        VMcol[kp] = v * iv;
        if (wu) UMcol[kp] = ((j == 0) ? -R(1.0) : dj * v) * iu;
    }
}

__global__ void __launch_bounds__(kLgThreads) k_vectors_warp(const NodeDesc *__restrict__ nodes,
                                                      const MatDesc *__restrict__ mats,
                                                      const NodeState *__restrict__ state, int wpn,
                                                      int nnodes) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / wpn, w = warp % wpn;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    const int N = ns.N, G = group_size(N), per = 32 / G;
    const int i = w * per + lane / G;
    if (i >= N) return;                              // whole groups leave together
    const MatDesc &md = mats[nd.mat];
    const int r0 = nd.r0, Ktot = ns.Ktot, gl = lane & (G - 1);
    const long long wb = (long long)r0 * md.wstride;
    const real_t *d = md.dM + r0, *zt = md.zt + r0;
    const int *kpos = md.kposM + r0;
    const real_t dor = d[md.org[r0 + i]], tau = md.tau[r0 + i];
    real_t *UMcol = md.UM + wb + (size_t)i * Ktot, *VMcol = md.VM + wb + (size_t)i * Ktot;
    // the register cache holds 16 entries per lane below G = 32 (group_size
    // keeps N <= 16 G there)
    const bool wu = md.want_u != 0;
    switch (G) {
    case 4: vectors_group<4, 16>(d, zt, kpos, N, ns.n1, ns.P1, dor, tau, UMcol, VMcol, gl, wu); break;
    case 8: vectors_group<8, 16>(d, zt, kpos, N, ns.n1, ns.P1, dor, tau, UMcol, VMcol, gl, wu); break;
    case 16: vectors_group<16, 16>(d, zt, kpos, N, ns.n1, ns.P1, dor, tau, UMcol, VMcol, gl, wu); break;
    default:
        if (N <= 32 * 32) vectors_group<32, 32>(d, zt, kpos, N, ns.n1, ns.P1, dor, tau, UMcol, VMcol, gl, wu);
        else vectors_warp_long(d, zt, kpos, N, ns.n1, ns.P1, dor, tau, UMcol, VMcol, gl, wu);
        break;
    }
}

// values only: the node's first and last rows of V for the survivors, row
// times the normalised v_i of Eq. (M-svd-vec) computed on the fly (a lane
// group per root; no U_M / V_M is stored)
template <int G>
__device__ __forceinline__ void rows_group(const real_t *__restrict__ d, const real_t *__restrict__ zt,
                                           const int *__restrict__ kpos, const real_t *__restrict__ FK,
                                           const real_t *__restrict__ LK, int N, real_t dor, real_t tau,
                                           real_t *vf, real_t *vl, int gl) {
    const real_t wsum = dor + tau;   // w_i: d_j + w_i formed once per entry (a sum of positives)
    real_t sv = R(0), sf = R(0), sl = R(0);
    for (int j = gl; j < N; j += G) {
        const real_t dj = d[j];
        const real_t v = quot(zt[j], ((dj - dor) - tau) * (dj + wsum));
        const int kp = kpos[j];
        sv = fma(v, v, sv);
        sf = fma(FK[kp], v, sf);
        sl = fma(LK[kp], v, sl);
    }
    sv = group_sum<G>(sv);
    sf = group_sum<G>(sf);
    sl = group_sum<G>(sl);
    if (gl == 0) {
        const real_t iv = R(1) / sqrt(sv);
        *vf = sf * iv;
        *vl = sl * iv;
    }
}

__global__ void __launch_bounds__(kLgThreads) k_rows_update(const NodeDesc *__restrict__ nodes,
                                                     const MatDesc *__restrict__ mats,
                                                     const NodeState *__restrict__ state, int wpn, int nnodes) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / wpn, w = warp % wpn;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    const int N = ns.N, G = group_size(N), per = 32 / G;
    const int i = w * per + lane / G;
    if (i >= N) return;                              // whole groups leave together
    const MatDesc &md = mats[nd.mat];
    const int r0 = nd.r0, gl = lane & (G - 1);
    const real_t *d = md.dM + r0, *zt = md.zt + r0;
    const int *kpos = md.kposM + r0;
    const real_t *FK = md.FK + nd.kbase, *LK = md.LK + nd.kbase;
    const real_t dor = d[md.org[r0 + i]], tau = md.tau[r0 + i];
    real_t *vf = md.vf[nd.buf] + r0 + i, *vl = md.vl[nd.buf] + r0 + i;
    switch (G) {
    case 4: rows_group<4>(d, zt, kpos, FK, LK, N, dor, tau, vf, vl, gl); break;
    case 8: rows_group<8>(d, zt, kpos, FK, LK, N, dor, tau, vf, vl, gl); break;
    case 16: rows_group<16>(d, zt, kpos, FK, LK, N, dor, tau, vf, vl, gl); break;
    default: rows_group<32>(d, zt, kpos, FK, LK, N, dor, tau, vf, vl, gl); break;
    }
}

#ifndef BDC_FP32
__global__ void __launch_bounds__(256) k_mvectors_single(int N, const double *d, const double *zt,
                                                         const int *org, const double *tau, double *UM,
                                                         int ldum, double *VM, int ldvm) {
    __shared__ double sh[8];
    const int i = blockIdx.x;
    vectors_one(d, zt, N, i, org[i], tau[i], nullptr, N, UM + (size_t)i * ldum, VM + (size_t)i * ldvm, sh);
}
#endif

}  // namespace

cudaError_t launch_secular(const NodeDesc *nodes, int nnodes, const MatDesc *mats, NodeState *state,
                           int mmax, int max_iter, int seed_mode, const float *mlp, int harvest, int fp32_start,
                           cudaStream_t st) {
#ifdef BDC_FP32
    fp32_start = 0;   // already single precision
#endif
    if (nnodes <= 0) return cudaSuccess;
    const long long roots = (long long)nnodes * mmax;
    const long long gwarps = (long long)nnodes * group_warps(mmax);
    cudaError_t e = cudaSuccess;
    {
    StageScope sc(st, BDC_STAGE_SECULAR, (seed_mode != BDC_SEED_PLAIN || harvest) ? 2 : 1, 0.0);
#ifdef BDC_FP32
    if (seed_mode != BDC_SEED_PLAIN || harvest) return cudaErrorInvalidValue;   // starts: FP64 only
    (void)mlp;
#else
    if (seed_mode != BDC_SEED_PLAIN || harvest) {
        const size_t smem = (seed_mode == BDC_SEED_MLP) ? sizeof(float) * kMlpParams : 0;
        if (smem > 48 * 1024) return cudaErrorInvalidValue;
        k_root_start<<<(unsigned)((roots + 127) / 128), 128, smem, st>>>(nodes, mats, state, mmax, nnodes,
                                                                          seed_mode, mlp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
#endif
    const long long swarps = (long long)nnodes * secular_group_warps(mmax);
    k_secular<<<(unsigned)((swarps + kLgWarps - 1) / kLgWarps), kLgThreads, 0, st>>>(
        nodes, mats, state, secular_group_warps(mmax), max_iter, nnodes, seed_mode, fp32_start);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    }
    StageScope sc(st, BDC_STAGE_LOWNER, 1, 0.0);
    k_lowner<<<(unsigned)((gwarps + kLgWarps - 1) / kLgWarps), kLgThreads, 0, st>>>(nodes, mats, state,
                                                                                   group_warps(mmax), nnodes);
    return cudaGetLastError();
}

cudaError_t launch_vectors(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                           int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    const long long warps = (long long)nnodes * group_warps(mmax);
    k_vectors_warp<<<(unsigned)((warps + kLgWarps - 1) / kLgWarps), kLgThreads, 0, st>>>(nodes, mats, state,
                                                                                        group_warps(mmax), nnodes);
    return cudaGetLastError();
}

cudaError_t launch_rows_update(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                               int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    const long long warps = (long long)nnodes * group_warps(mmax);
    k_rows_update<<<(unsigned)((warps + kLgWarps - 1) / kLgWarps), kLgThreads, 0, st>>>(nodes, mats, state,
                                                                                       group_warps(mmax), nnodes);
    return cudaGetLastError();
}

#ifndef BDC_FP32   // standalone step entry points: FP64 only
cudaError_t launch_secular_single(int N, const double *d, const double *z, int *org, double *tau,
                                  double *omega, int max_iter, int *info, int seed_mode, const float *mlp,
                                  int *iters, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_secular_single<<<(N + 7) / 8, 256, 0, st>>>(N, d, z, org, tau, omega, max_iter, info, seed_mode, mlp,
                                                   iters);
    return cudaGetLastError();
}

cudaError_t launch_mlp_features_single(int N, const double *d, const double *z, float *feat, double *yq,
                                       cudaStream_t st) {
    if (N <= 1) return cudaSuccess;
    k_mlp_features_single<<<(N - 1 + 7) / 8, 256, 0, st>>>(N, d, z, feat, yq);
    return cudaGetLastError();
}

cudaError_t launch_lowner_single(int N, const double *d, const double *z, const int *org,
                                 const double *tau, double *zt, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_lowner_single<<<(N + 7) / 8, 256, 0, st>>>(N, d, z, org, tau, zt);
    return cudaGetLastError();
}

cudaError_t launch_mvectors_single(int N, const double *d, const double *zt, const int *org,
                                   const double *tau, double *UM, int ldum, double *VM, int ldvm,
                                   cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_mvectors_single<<<N, 256, 0, st>>>(N, d, zt, org, tau, UM, ldum, VM, ldvm);
    return cudaGetLastError();
}
#endif  // BDC_FP32

}  // namespace BDC_NS
