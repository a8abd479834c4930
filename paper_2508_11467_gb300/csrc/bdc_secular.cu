// Merge step of Algorithm 2, part (b) (lasd3 without the products):
//
// k_secular  one warp per root of the secular equation (Eq. M-svd-val)
//            f(w) = 1 + sum_j z_j^2 / (d_j^2 - w^2), root i in (d_i, d_{i+1}).
//            The unknown is held relative to the nearer pole d_o as
//            x = w^2 - d_o^2 (then tau = w - d_o), so d_j^2 - w^2 is formed as
//            (d_j - d_o)(d_j + d_o) - x without cancellation.  Each step fits
//            the two nearest poles with a rational model matching f and f'
//            (a "middle way" step in the sense of R.-C. Li), safeguarded by a
//            bracket; lanes split the pole sums and reduce with shuffles.
//            Stopping rule: |f| <= 16 eps (1 + sum |terms|), or a step below
//            4 eps |x|.
// k_lowner   one warp per i: |z~_i| of Eq. (bdc-zi) as a product over k of
//            (w_k^2 - d_i^2) / (d_{k'}^2 - d_i^2) (every factor lies in (0, 1]
//            by interlacing), lane partial products, then a shuffle product
//            reduction; sign from z_i.
// k_vectors  one CTA per column i: v_i, u_i of Eq. (M-svd-vec), normalised,
//            written in the K order of the merge product (coalesced down the
//            column).
//
// All arithmetic is FP64.
#include "bdc_internal.cuh"

namespace bdc {

namespace {

struct Sums {
    double psi, dpsi, phi, dphi;
};

// pole sums at x = w^2 - d_o^2; left group j <= i (psi < 0), right j > i
__device__ __forceinline__ Sums pole_sums(const double *__restrict__ d, const double *__restrict__ z,
                                          int N, int i, double dor, double x, int lane) {
    Sums s{0.0, 0.0, 0.0, 0.0};
    for (int j = lane; j <= i; j += 32) {
        const double dj = d[j], zj = z[j];
        const double del = (dj - dor) * (dj + dor) - x;
        const double t = zj / del;
        s.psi = fma(zj, t, s.psi);
        s.dpsi = fma(t, t, s.dpsi);
    }
    for (int j = i + 1 + lane; j < N; j += 32) {
        const double dj = d[j], zj = z[j];
        const double del = (dj - dor) * (dj + dor) - x;
        const double t = zj / del;
        s.phi = fma(zj, t, s.phi);
        s.dphi = fma(t, t, s.dphi);
    }
    s.psi = warp_sum(s.psi);
    s.dpsi = warp_sum(s.dpsi);
    s.phi = warp_sum(s.phi);
    s.dphi = warp_sum(s.dphi);
    return s;
}

// Solve root i of (d, z) (N entries, d[0] = 0 < d[1] < ...).  Returns the
// number of iterations used, or -1 if not converged.  All lanes return the
// same result.  x0 (optional, NaN = none) is a proposed start w^2 - d_o^2
// relative to the origin chosen here.
__device__ int solve_root(const double *__restrict__ d, const double *__restrict__ z, int N, int i,
                          int max_iter, double zz, int &org_out, double &tau_out, double start_frac) {
    const int lane = threadIdx.x & 31;
    if (N == 1) {
        org_out = 0;
        tau_out = fabs(z[0]);
        return 0;
    }
    const bool last = (i == N - 1);
    const double dl = d[i];
    const double du = last ? sqrt(dl * dl + zz) : d[i + 1];
    const double h = 0.5 * (du - dl);
    int o;
    double dor, lo, hi, lamL, lamR, x;
    Sums s;
    if (!last) {
        // sign of f at the interval midpoint picks the nearer pole as origin
        const double xmid = h * (2.0 * dl + h);
        s = pole_sums(d, z, N, i, dl, xmid, lane);
        const double fmid = 1.0 + s.psi + s.phi;
        if (fmid >= 0.0) {
            o = i; dor = dl; lo = 0.0; hi = xmid;
            lamL = 0.0; lamR = (du - dl) * (du + dl);
            x = xmid;
        } else {
            o = i + 1; dor = du; lo = -h * (2.0 * du - h); hi = 0.0;
            lamL = -(du - dl) * (du + dl); lamR = 0.0;
            x = lo;                        // the same point, measured from d_{i+1}
        }
    } else {
        o = i; dor = dl; lo = 0.0; hi = zz;
        lamL = 0.0; lamR = 0.0;
        x = 0.5 * zz;
        s = pole_sums(d, z, N, i, dor, x, lane);
    }
    if (!(start_frac != start_frac)) {     // proposed start inside the bracket
        const double xs = lo + start_frac * (hi - lo);
        if (xs > lo && xs < hi) {
            x = xs;
            s = pole_sums(d, z, N, i, dor, x, lane);
        }
    }
    int it = 0;
    for (;;) {
        const double f = 1.0 + s.psi + s.phi;
        const double scale = 1.0 + s.phi - s.psi;
        if (fabs(f) <= 16.0 * kEps * scale) break;
        if (f > 0.0) hi = x; else lo = x;
        if (it >= max_iter) { it = -1; break; }
        // rational model through the two nearest poles (value and slope)
        const double DL = lamL - x;
        double eta;
        bool ok = true;
        if (!last) {
            const double DR = lamR - x;
            const double sL = DL * DL * s.dpsi, sR = DR * DR * s.dphi;
            const double C = f - DL * s.dpsi - DR * s.dphi;
            const double a = C * (DL + DR) + sL + sR;
            const double b = C * DL * DR + sL * DR + sR * DL;
            if (C == 0.0) {
                eta = b / a;
            } else {
                const double disc = sqrt(fabs(a * a - 4.0 * b * C));
                eta = (a > 0.0) ? (2.0 * b / (a + disc)) : ((a - disc) / (2.0 * C));
            }
        } else {
            const double sL = DL * DL * s.dpsi;
            const double C = f - DL * s.dpsi;
            if (C > 0.0) eta = DL + sL / C; else { eta = 0.0; ok = false; }
        }
        double xn = x + eta;
        if (!ok || !(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double step = xn - x;
        x = xn;
        ++it;
        s = pole_sums(d, z, N, i, dor, x, lane);
        if (fabs(step) <= 4.0 * kEps * fabs(x)) break;
    }
    org_out = o;
    // tau = w - d_o from x = (w - d_o)(w + d_o)
    tau_out = x / (dor + sqrt(dor * dor + x));
    return it;
}

__global__ void __launch_bounds__(256) k_secular(const NodeDesc *__restrict__ nodes,
                                                 const MatDesc *__restrict__ mats,
                                                 NodeState *__restrict__ state, int mmax,
                                                 int max_iter, int nnodes) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / mmax, i = warp % mmax;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    if (i >= ns.N) return;
    const MatDesc md = mats[nd.mat];
    const double *d = md.dM + nd.r0, *z = md.zM + nd.r0;
    const int N = ns.N;
    double zz = 0.0;
    if (i == N - 1) {
        for (int j = lane; j < N; j += 32) zz = fma(z[j], z[j], zz);
        zz = warp_sum(zz);
    }
    int o;
    double tau;
    const int it = solve_root(d, z, N, i, max_iter, zz, o, tau, __longlong_as_double(0x7ff8000000000000ll));
    if (lane == 0) {
        md.org[nd.r0 + i] = o;
        md.tau[nd.r0 + i] = tau;
        md.omega[nd.r0 + i] = d[o] + tau;
        if (it < 0) atomicAdd(md.info, 1);
        atomicAdd(&state[nd.id].iters, (unsigned long long)(it < 0 ? max_iter : it));
    }
}

__global__ void __launch_bounds__(256) k_secular_single(int N, const double *d, const double *z, int *org,
                                                        double *tau, double *omega, int max_iter,
                                                        int *info) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= N) return;
    double zz = 0.0;
    if (i == N - 1) {
        for (int j = lane; j < N; j += 32) zz = fma(z[j], z[j], zz);
        zz = warp_sum(zz);
    }
    int o;
    double t;
    const int it = solve_root(d, z, N, i, max_iter, zz, o, t, __longlong_as_double(0x7ff8000000000000ll));
    if (lane == 0) {
        org[i] = o;
        tau[i] = t;
        omega[i] = d[o] + t;
        if (it < 0) atomicAdd(info, 1);
    }
}

// |z~_i|^2 of Eq. (bdc-zi), 0-based: (w_{N-1}^2 - d_i^2) *
//   prod_{k<i} (w_k^2 - d_i^2)/(d_k^2 - d_i^2) * prod_{i<=k<N-1} (w_k^2 - d_i^2)/(d_{k+1}^2 - d_i^2)
__device__ __forceinline__ double lowner_one(const double *__restrict__ d, const double *__restrict__ z,
                                             const int *__restrict__ org, const double *__restrict__ tau,
                                             int N, int i, int lane) {
    const double di = d[i];
    double prod = 1.0;
    for (int k = lane; k < N - 1; k += 32) {
        const int ok = org[k];
        const double wmd = (d[ok] - di) + tau[k];        // w_k - d_i
        const double wpd = d[ok] + tau[k] + di;          // w_k + d_i
        const int kk = (k < i) ? k : k + 1;
        const double den = (d[kk] - di) * (d[kk] + di);
        prod *= (wmd * wpd) / den;
    }
    for (int o = 16; o > 0; o >>= 1) prod *= __shfl_down_sync(0xffffffffu, prod, o);
    prod = __shfl_sync(0xffffffffu, prod, 0);
    const int oN = org[N - 1];
    const double last = ((d[oN] - di) + tau[N - 1]) * (d[oN] + tau[N - 1] + di);
    const double zt = sqrt(fabs(last * prod));
    return (z[i] < 0.0) ? -zt : zt;
}

__global__ void __launch_bounds__(256) k_lowner(const NodeDesc *__restrict__ nodes,
                                                const MatDesc *__restrict__ mats,
                                                const NodeState *__restrict__ state, int mmax, int nnodes) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int node = warp / mmax, i = warp % mmax;
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    if (i >= ns.N) return;
    const MatDesc md = mats[nd.mat];
    const int r0 = nd.r0;
    const double zt = lowner_one(md.dM + r0, md.zM + r0, md.org + r0, md.tau + r0, ns.N, i, lane);
    if (lane == 0) md.zt[r0 + i] = zt;
}

__global__ void __launch_bounds__(256) k_lowner_single(int N, const double *d, const double *z,
                                                       const int *org, const double *tau, double *zt) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= N) return;
    const double v = lowner_one(d, z, org, tau, N, i, lane);
    if (lane == 0) zt[i] = v;
}

__device__ __forceinline__ double block_sum256(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    __syncthreads();
    return r;
}

// column i of U_M and V_M, rows in K order (invK: K position -> M index, -1 = zero row)
__device__ void vectors_one(const double *__restrict__ d, const double *__restrict__ zt, int N, int i,
                            int o, double tau, const int *__restrict__ invK, int Ktot,
                            double *__restrict__ UMcol, double *__restrict__ VMcol, double *sh) {
    const double dor = d[o];
    double sv = 0.0, su = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double dj = d[j];
        const double v = zt[j] / (((dj - dor) - tau) * (dj + dor + tau));
        const double u = (j == 0) ? -1.0 : dj * v;
        sv = fma(v, v, sv);
        su = fma(u, u, su);
    }
    sv = block_sum256(sv, sh);
    su = block_sum256(su, sh);
    const double iv = 1.0 / sqrt(sv), iu = 1.0 / sqrt(su);
    for (int p = threadIdx.x; p < Ktot; p += blockDim.x) {
        const int j = invK ? invK[p] : p;
        double uo = 0.0, vo = 0.0;
        if (j >= 0) {
            const double dj = d[j];
            const double v = zt[j] / (((dj - dor) - tau) * (dj + dor + tau));
            vo = v * iv;
            uo = ((j == 0) ? -1.0 : dj * v) * iu;
        }
        UMcol[p] = uo;
        VMcol[p] = vo;
    }
}

__global__ void __launch_bounds__(256) k_vectors(const NodeDesc *__restrict__ nodes,
                                                 const MatDesc *__restrict__ mats,
                                                 const NodeState *__restrict__ state, int mmax) {
    __shared__ double sh[8];
    const int node = blockIdx.x / mmax, i = blockIdx.x % mmax;
    const NodeDesc nd = nodes[node];
    const NodeState ns = state[nd.id];
    if (i >= ns.N) return;
    const MatDesc md = mats[nd.mat];
    const int r0 = nd.r0;
    const long long wb = (long long)r0 * md.wstride;
    vectors_one(md.dM + r0, md.zt + r0, ns.N, i, md.org[r0 + i], md.tau[r0 + i], md.invK + nd.kbase,
                ns.Ktot, md.UM + wb + (size_t)i * ns.Ktot, md.VM + wb + (size_t)i * ns.Ktot, sh);
}

__global__ void __launch_bounds__(256) k_mvectors_single(int N, const double *d, const double *zt,
                                                         const int *org, const double *tau, double *UM,
                                                         int ldum, double *VM, int ldvm) {
    __shared__ double sh[8];
    const int i = blockIdx.x;
    vectors_one(d, zt, N, i, org[i], tau[i], nullptr, N, UM + (size_t)i * ldum, VM + (size_t)i * ldvm, sh);
}

}  // namespace

cudaError_t launch_secular(const NodeDesc *nodes, int nnodes, const MatDesc *mats, NodeState *state,
                           int mmax, int max_iter, int seed_mode, const float *mlp, cudaStream_t st) {
    (void)seed_mode; (void)mlp;
    if (nnodes <= 0) return cudaSuccess;
    const long long warps = (long long)nnodes * mmax;
    k_secular<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(nodes, mats, state, mmax, max_iter, nnodes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lowner<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(nodes, mats, state, mmax, nnodes);
    return cudaGetLastError();
}

cudaError_t launch_vectors(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                           int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    k_vectors<<<(unsigned)nnodes * mmax, 256, 0, st>>>(nodes, mats, state, mmax);
    return cudaGetLastError();
}

cudaError_t launch_secular_single(int N, const double *d, const double *z, int *org, double *tau,
                                  double *omega, int max_iter, int *info, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_secular_single<<<(N + 7) / 8, 256, 0, st>>>(N, d, z, org, tau, omega, max_iter, info);
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

}  // namespace bdc
