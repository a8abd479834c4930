// Checked mode (bdc_opts.checked = 1): the invariants of every merge of
// Algorithm 2 verified on the device between the stages, a violation
// recorded in the matrix's status word as BDC_ERR_CHECK (the first error of
// a matrix is kept; nothing traps).
//
// k_check_prep   after the deflation (Sec. 4.2.1): 1 <= N <= m, the type
//                counts add up to N - 1 with the K order [n1 | pad to 8 |
//                d_0 | n2 | n3] of the merge products, the survivors' d
//                strictly ascending from d_0 = 0 (Eq. M-condition leaves
//                distinct values), z finite and non-zero, the K positions a
//                permutation (invK o kposM = identity), and (with vectors)
//                every slot of the node's column maps inside [0, n).
// k_check_roots  after the secular solve and z~ (Eqs. M-svd-val, bdc-zi):
//                root i has its origin at d_i or d_{i+1} (the last root at
//                d_{N-1}), its offset tau on the interval's side of that
//                origin and shorter than the interval, and z~_i finite.
// k_check_final  after the final sort: S finite, non-negative, descending.
#include "bdc_internal.cuh"

namespace BDC_NS {

namespace {

__device__ __forceinline__ bool finite(real_t x) { return abits(x) < abits(R(INFINITY)); }

__device__ __forceinline__ void flag(const MatDesc &md, bool bad) {
    if (bad) set_error(md.info, BDC_ERR_CHECK);
}

__global__ void __launch_bounds__(256) k_check_prep(const NodeDesc *__restrict__ nodes,
                                                    const MatDesc *__restrict__ mats,
                                                    const NodeState *__restrict__ state) {
    const NodeDesc nd = nodes[blockIdx.x];
    const MatDesc &md = mats[nd.mat];
    const NodeState ns = state[nd.id];
    const int m = nd.m, r0 = nd.r0, t = threadIdx.x;
    const int N = ns.N;
    const bool counts = N >= 1 && N <= m && ns.n1 >= 0 && ns.n2 >= 0 && ns.n3 >= 0 &&
                        ns.n1 + ns.n2 + ns.n3 == N - 1 && ns.P1 == ((ns.n1 + 7) & ~7) &&
                        ns.Ktot == ns.P1 + 1 + ns.n2 + ns.n3 && ns.Ktot <= m + 8;
    if (t == 0) flag(md, !counts);
    if (!counts) return;                     // the loops below index with these counts
    const real_t *dM = md.dM + r0, *zM = md.zM + r0;
    const int *kpos = md.kposM + r0, *invK = md.invK + nd.kbase;
    bool bad = false;
    for (int i = t; i < N; i += blockDim.x) {
        const real_t di = dM[i], zi = zM[i];
        bad |= !finite(di) || !finite(zi) || zi == R(0);
        bad |= (i == 0) ? (di != R(0)) : !(di > dM[i - 1]);
        const int kp = kpos[i];
        bad |= kp < 0 || kp >= ns.Ktot;
        if (kp >= 0 && kp < ns.Ktot) bad |= invK[kp] != i;
    }
    for (int kp = ns.n1 + t; kp < ns.P1; kp += blockDim.x) bad |= invK[kp] != -1;
    if (!md.vals) {
        const int *nus = md.us[nd.buf] + r0, *nvs = md.vs[nd.buf] + r0;
        for (int c = t; c < m; c += blockDim.x) bad |= nus[c] < 0 || nus[c] >= md.n || nvs[c] < 0 || nvs[c] >= md.n;
    }
    flag(md, bad);
}

// one thread per root (node = blockIdx.y)
__global__ void __launch_bounds__(256) k_check_roots(const NodeDesc *__restrict__ nodes,
                                                     const MatDesc *__restrict__ mats,
                                                     const NodeState *__restrict__ state) {
    const NodeDesc nd = nodes[blockIdx.y];
    const MatDesc &md = mats[nd.mat];
    const int N = state[nd.id].N;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || N < 1 || N > nd.m) return;
    const int r0 = nd.r0;
    const real_t *dM = md.dM + r0;
    const int o = md.org[r0 + i];
    const real_t tau = md.tau[r0 + i], zt = md.zt[r0 + i];
    bool bad = !finite(tau) || !finite(zt);
    if (i == N - 1) {
        bad |= o != i || !(tau > R(0));
    } else if (o == i) {
        bad |= !(tau > R(0)) || !(tau < dM[i + 1] - dM[i]);
    } else if (o == i + 1) {
        bad |= !(tau < R(0)) || !(-tau < dM[i + 1] - dM[i]);
    } else {
        bad = true;
    }
    flag(md, bad);
}

__global__ void __launch_bounds__(256) k_check_final(const MatDesc *__restrict__ mats) {
    const MatDesc &md = mats[blockIdx.x];
    bool bad = false;
    for (int c = threadIdx.x; c < md.n; c += blockDim.x) {
        const real_t s = md.So[c];
        bad |= !finite(s) || s < R(0) || (c + 1 < md.n && !(s >= md.So[c + 1]));
    }
    flag(md, bad);
}

// test hook (BDC_TEST_CORRUPT_ROOT): moves root 0 of the first node of a
// height to the wrong side of its origin, a value-only change that the root
// check must report (no index is derived from it)
__global__ void k_corrupt_root(const NodeDesc *__restrict__ nodes, const MatDesc *__restrict__ mats) {
    const NodeDesc nd = nodes[0];
    const MatDesc &md = mats[nd.mat];
    md.tau[nd.r0] = -md.tau[nd.r0];
}

}  // namespace

cudaError_t launch_check_prep(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                              cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    k_check_prep<<<nnodes, 256, 0, st>>>(nodes, mats, state);
    return cudaGetLastError();
}

cudaError_t launch_check_roots(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                               int mmax, bool corrupt, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    if (corrupt) {
        k_corrupt_root<<<1, 1, 0, st>>>(nodes, mats);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int n0 = 0; n0 < nnodes; n0 += 65535) {
        const int nn = nnodes - n0 < 65535 ? nnodes - n0 : 65535;
        k_check_roots<<<dim3((unsigned)((mmax + 255) / 256), (unsigned)nn), 256, 0, st>>>(nodes + n0, mats, state);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_check_final(const MatDesc *mats, int nmat, cudaStream_t st) {
    if (nmat <= 0) return cudaSuccess;
    k_check_final<<<nmat, 256, 0, st>>>(mats);
    return cudaGetLastError();
}

}  // namespace BDC_NS
