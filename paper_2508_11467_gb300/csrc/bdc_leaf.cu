// Leaf SVDs of Algorithm 2, step (1): "solve subproblems by QR iteration".
//
// One warp per leaf, the whole leaf in shared memory.  A leaf is the
// m x (m+sqre) upper bidiagonal of rows r0..r0+m-1 (Sec. 4.2.1: every left
// child is (k-1) x k, a right child inherits its parent's shape).  For
// sqre = 1 the extra column is first rotated away by right rotations
// (bottom to top), which leaves the right null vector in the last column of
// V.  The square part is then diagonalised by Golub-Kahan implicit-shift QR
// sweeps (Wilkinson shift, zero-diagonal chases).  Lane 0 computes each
// sweep's rotation sequence (the sweep is sequential), then all lanes apply
// it to their rows of U and V (one row per lane, rows stride 32).  Output:
// singular values sorted ascending into D, the node's U and V blocks, and
// the identity order in Q.
#include "bdc_internal.cuh"

namespace BDC_NS {

namespace {

enum { ACT_DONE = 0, ACT_SWEEP = 1, ACT_CHASE_ROW = 2, ACT_CHASE_COL = 3, ACT_NOOP = 4 };

struct LeafCtl {
    int act, lo, hi, k, cnt, info;
};

// columns a, b of an SMEM column-major matrix, rows handled by this lane
__device__ __forceinline__ void rot_rows(real_t *X, int ld, int rows, int lane, int a, int b,
                                         real_t c, real_t s) {
    for (int r = lane; r < rows; r += 32) {
        real_t u = X[a * ld + r], v = X[b * ld + r];
        X[a * ld + r] = c * u + s * v;
        X[b * ld + r] = -s * u + c * v;
    }
}

__global__ void __launch_bounds__(32) k_leaf(const NodeDesc *__restrict__ leaves,
                                             const MatDesc *__restrict__ mats, int L,
                                             int max_sweeps) {
    extern __shared__ real_t sm[];
    const int lane = threadIdx.x;
    const NodeDesc nd = leaves[blockIdx.x];
    const MatDesc md = mats[nd.mat];
    const int m = nd.m, sq = nd.sqre, mc = m + sq;
    // singular values only: U is not accumulated and V keeps just its first
    // and last rows (2 x mc, rows 0 and mc-1 of the leaf's V)
    const bool vals = md.vals != 0;
    const int ldu = L, ldv = vals ? 2 : L + 1, vrows = vals ? 2 : mc;
    real_t *Us = sm;
    real_t *Vs = Us + (size_t)L * L;
    real_t *dd = Vs + (size_t)(L + 1) * (L + 1);
    real_t *ee = dd + (L + 1);
    real_t *c1 = ee + (L + 1);
    real_t *s1 = c1 + (L + 1);
    real_t *c2 = s1 + (L + 1);
    real_t *s2 = c2 + (L + 1);
    int *perm = (int *)(s2 + (L + 1));
    volatile LeafCtl *ctl = (volatile LeafCtl *)(perm + L + 2);

    if (!vals)
        for (int j = 0; j < m; ++j)
            for (int r = lane; r < m; r += 32) Us[j * ldu + r] = (r == j) ? R(1) : R(0);
    for (int j = 0; j < mc; ++j)
        for (int r = lane; r < vrows; r += 32) {
            const int row = (vals && r == 1) ? mc - 1 : r;
            Vs[j * ldv + r] = (row == j) ? R(1) : R(0);
        }
    for (int i = lane; i < m; i += 32) dd[i] = md.dsc[nd.r0 + i];
    for (int i = lane; i < m - 1 + sq; i += 32) ee[i] = md.esc[nd.r0 + i];
    if (lane == 0) { ctl->info = 0; ctl->hi = m - 1; }
    __syncwarp();

    // ---- rectangular leaf: rotate the extra column (index m) away
    if (sq) {
        if (lane == 0) {
            real_t x = ee[m - 1];
            for (int j = m - 1; j >= 0; --j) {
                real_t c, s, r;
                make_rot(dd[j], x, c, s, r);
                dd[j] = r;
                c1[j] = c; s1[j] = s;
                if (j > 0) { x = -s * ee[j - 1]; ee[j - 1] = c * ee[j - 1]; }
            }
            ee[m - 1] = R(0);
        }
        __syncwarp();
        for (int j = m - 1; j >= 0; --j) rot_rows(Vs, ldv, vrows, lane, j, m, c1[j], s1[j]);
        __syncwarp();
    }

    // leaf-local norm for the zero-diagonal threshold
    real_t bn = R(0);
    for (int i = lane; i < m; i += 32) bn = fmax(bn, fabs(dd[i]));
    for (int i = lane; i < m - 1; i += 32) bn = fmax(bn, fabs(ee[i]));
    bn = warp_max(bn);
    const real_t dtiny = kEps * bn;

    long long budget = (long long)max_sweeps * (m > 0 ? m : 1);
    for (;;) {
        if (lane == 0) {
            int act = ACT_NOOP;
            int hi = ctl->hi;
            if (hi <= 0) {
                act = ACT_DONE;
            } else if (fabs(ee[hi - 1]) <= kEps * (fabs(dd[hi - 1]) + fabs(dd[hi])) ||
                       fabs(ee[hi - 1]) <= dtiny * kEps) {
                ee[hi - 1] = R(0);
                ctl->hi = hi - 1;
                act = ACT_NOOP;
            } else {
                int lo = hi - 1;
                while (lo > 0 && fabs(ee[lo - 1]) > kEps * (fabs(dd[lo - 1]) + fabs(dd[lo])) &&
                       fabs(ee[lo - 1]) > dtiny * kEps)
                    --lo;
                if (lo > 0) ee[lo - 1] = R(0);
                int kz = -1;
                for (int k = lo; k <= hi; ++k)
                    if (fabs(dd[k]) <= dtiny) { kz = k; break; }
                if (kz >= 0) {
                    dd[kz] = R(0);
                    if (kz < hi) {            // clear row kz with rows kz+1..hi
                        real_t x = ee[kz];
                        ee[kz] = R(0);
                        int cnt = 0;
                        for (int j = kz + 1; j <= hi && x != R(0); ++j) {
                            real_t c, s, r;
                            make_rot(dd[j], x, c, s, r);
                            dd[j] = r;
                            if (j < hi) { x = -s * ee[j]; ee[j] = c * ee[j]; }
                            c2[j] = c; s2[j] = s;
                            cnt = j - kz;
                        }
                        act = ACT_CHASE_ROW; ctl->k = kz; ctl->cnt = cnt;
                    } else {                  // clear column hi with columns hi-1..lo
                        real_t x = ee[hi - 1];
                        ee[hi - 1] = R(0);
                        int jend = hi;
                        for (int j = hi - 1; j >= lo && x != R(0); --j) {
                            real_t c, s, r;
                            make_rot(dd[j], x, c, s, r);
                            dd[j] = r;
                            if (j > lo) { x = -s * ee[j - 1]; ee[j - 1] = c * ee[j - 1]; }
                            c1[j] = c; s1[j] = s;
                            jend = j;
                        }
                        act = ACT_CHASE_COL; ctl->k = jend;
                    }
                    ctl->lo = lo;
                } else if (budget-- <= 0) {
                    int cnt = 0;
                    for (int i = 0; i < hi; ++i) cnt += (ee[i] != R(0));
                    ctl->info = cnt > 0 ? cnt : 1;
                    act = ACT_DONE;
                } else {
                    // Golub-Kahan sweep on [lo, hi] with a Wilkinson shift
                    real_t dm = dd[hi - 1], dn = dd[hi], em = ee[hi - 1];
                    real_t el = (hi - 1 > lo) ? ee[hi - 2] : R(0);
                    real_t t11 = dm * dm + el * el, t22 = dn * dn + em * em, t12 = dm * em;
                    real_t delta = R(0.5) * (t11 - t22);
                    real_t sg = (delta >= R(0)) ? R(1) : R(-1);
                    real_t den = delta + sg * hypot(delta, t12);
                    real_t mu = (den != R(0)) ? t22 - t12 * t12 / den : t22;
                    real_t y = dd[lo] * dd[lo] - mu;
                    real_t z = dd[lo] * ee[lo];
                    for (int k = lo; k < hi; ++k) {
                        real_t c, s, r;
                        make_rot(y, z, c, s, r);
                        if (k > lo) ee[k - 1] = r;
                        real_t dk = dd[k], ek = ee[k], dk1 = dd[k + 1];
                        dd[k] = c * dk + s * ek;
                        ee[k] = -s * dk + c * ek;
                        real_t bulge = s * dk1;
                        dd[k + 1] = c * dk1;
                        c1[k] = c; s1[k] = s;
                        make_rot(dd[k], bulge, c, s, r);
                        dd[k] = r;
                        ek = ee[k]; dk1 = dd[k + 1];
                        ee[k] = c * ek + s * dk1;
                        dd[k + 1] = -s * ek + c * dk1;
                        if (k < hi - 1) {
                            real_t ek1 = ee[k + 1];
                            z = s * ek1;
                            ee[k + 1] = c * ek1;
                            y = ee[k];
                        }
                        c2[k] = c; s2[k] = s;
                    }
                    act = ACT_SWEEP;
                    ctl->lo = lo;
                }
            }
            ctl->act = act;
        }
        __syncwarp();
        const int act = ctl->act;
        if (act == ACT_DONE) break;
        if (act == ACT_SWEEP) {
            const int lo = ctl->lo, hi = ctl->hi;
            for (int k = lo; k < hi; ++k) rot_rows(Vs, ldv, vrows, lane, k, k + 1, c1[k], s1[k]);
            if (!vals)
                for (int k = lo; k < hi; ++k) rot_rows(Us, ldu, m, lane, k, k + 1, c2[k], s2[k]);
        } else if (act == ACT_CHASE_ROW) {
            const int kz = ctl->k, cnt = ctl->cnt;
            if (!vals)
                for (int j = kz + 1; j <= kz + cnt; ++j) rot_rows(Us, ldu, m, lane, j, kz, c2[j], s2[j]);
        } else if (act == ACT_CHASE_COL) {
            const int hi = ctl->hi, jend = ctl->k;
            for (int j = hi - 1; j >= jend; --j) rot_rows(Vs, ldv, vrows, lane, j, hi, c1[j], s1[j]);
        }
        __syncwarp();
    }

    // non-negative values: flip the matching right vector
    for (int j = 0; j < m; ++j) {
        if (dd[j] < R(0)) {
            for (int r = lane; r < vrows; r += 32) Vs[j * ldv + r] = -Vs[j * ldv + r];
        }
    }
    __syncwarp();
    for (int j = lane; j < m; j += 32) dd[j] = fabs(dd[j]);
    __syncwarp();
    // ascending order (ties by index)
    for (int j = lane; j < m; j += 32) {
        real_t v = dd[j];
        int rank = 0;
        for (int i = 0; i < m; ++i) {
            real_t w = dd[i];
            rank += (w < v) || (w == v && i < j);
        }
        perm[rank] = j;
    }
    __syncwarp();
    const long long ld = md.n;
    const int r0 = nd.r0;
    if (vals) {
        real_t *VF = md.vf[nd.buf], *VL = md.vl[nd.buf];
        for (int p = lane; p < m; p += 32) {
            VF[r0 + p] = Vs[perm[p] * ldv + 0];
            VL[r0 + p] = Vs[perm[p] * ldv + 1];
        }
        if (sq && lane == 0) {
            VF[r0 + m] = Vs[m * ldv + 0];
            VL[r0 + m] = Vs[m * ldv + 1];
        }
    } else {
        // node column p in slot r0 + p (rows r0..r0+m-1 of U, r0..r0+mc-1 of V)
        real_t *Uo = md.U, *Vo = md.V;
        for (int p = 0; p < m; ++p) {
            const int j = perm[p];
            for (int r = lane; r < m; r += 32) Uo[(size_t)(r0 + p) * ld + r0 + r] = Us[j * ldu + r];
            for (int r = lane; r < mc; r += 32) Vo[(size_t)(r0 + p) * ld + r0 + r] = Vs[j * ldv + r];
        }
        if (sq)
            for (int r = lane; r < mc; r += 32) Vo[(size_t)(r0 + m) * ld + r0 + r] = Vs[m * ldv + r];
        for (int p = lane; p < mc; p += 32) {
            if (p < m) {
                md.us[nd.buf][r0 + p] = r0 + p;
                md.ulo[r0 + p] = r0;
                md.uhi[r0 + p] = r0 + m;
            }
            md.vs[nd.buf][r0 + p] = r0 + p;
            md.vlo[r0 + p] = r0;
            md.vhi[r0 + p] = r0 + mc;
        }
    }
    for (int p = lane; p < m; p += 32) {
        md.D[r0 + p] = dd[perm[p]];
        md.Q[r0 + p] = p;
    }
    if (lane == 0 && ctl->info != 0) atomicAdd(md.info, ctl->info);
}

}  // namespace

cudaError_t launch_leaves(const NodeDesc *leaves, int nleaves, const MatDesc *mats, int leafmax,
                          int max_sweeps, cudaStream_t st) {
    if (nleaves <= 0) return cudaSuccess;
    const int L = leafmax;
    size_t smem = sizeof(real_t) * ((size_t)L * L + (size_t)(L + 1) * (L + 1) + 6 * (size_t)(L + 1)) +
                  sizeof(int) * (L + 2) + sizeof(LeafCtl) + 16;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_leaf<<<nleaves, 32, smem, st>>>(leaves, mats, L, max_sweeps);
    return cudaGetLastError();
}

}  // namespace BDC_NS
