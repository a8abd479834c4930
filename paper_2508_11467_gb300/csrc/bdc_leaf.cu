// Leaf SVDs of Algorithm 2, step (1): "solve subproblems by QR iteration".
//
// A leaf is the m x (m+sqre) upper bidiagonal of rows r0..r0+m-1 (Sec. 4.2.1:
// every left child is (k-1) x k, a right child inherits its parent's shape).
// For sqre = 1 the extra column is first rotated away by right rotations
// (bottom to top), which leaves the right null vector in the last column of
// V.  The square part is then diagonalised by Golub-Kahan implicit-shift QR
// sweeps (Wilkinson shift, zero-diagonal chases).  Output: singular values
// sorted ascending into D, the node's columns of U and V in slots r0 + p, and
// the identity order in Q.
//
// The rotations of a sweep form one sequential chain, and GB300's FP64 pipe
// charges an instruction the same whether 1 or 32 lanes issue it, so the
// chain is not run by one lane of a warp while 31 wait.  Two kernels:
//   k_leaf_rotations  the QR iteration on d and e alone, one leaf per lane
//                     (ceil(leaves / (4 SMs)) leaves per warp),
//                     writing every action and its rotations to a per-leaf
//                     log;
//   k_leaf_vectors    one warp per leaf: replays the log on U and V (each lane
//                     carries one row of U or V through a whole action),
//                     then fixes signs, sorts and writes the node.
// A leaf whose log would outgrow its fixed capacity is marked, and
// k_leaf_vectors runs the QR iteration for it itself (lane 0 forms each
// action's rotations, all lanes apply them).  Singular values only: the
// first kernel applies the V rotations to the two tracked rows of V itself
// and writes the leaf's outputs; the second kernel is not launched.
#include <cstdlib>

#include "bdc_internal.cuh"

namespace BDC_NS {

namespace {

enum { ACT_DONE = 0, ACT_SWEEP = 1, ACT_CHASE_ROW = 2, ACT_CHASE_COL = 3, ACT_NOOP = 4, ACT_SQRE = 5 };

// Rotation log of one leaf (leaf_log_bytes apart):
//   real_t cs[cs_cap(L)]   the actions' rotations, in order:
//     ACT_SQRE            (c, s) for j = m-1 .. 0: V columns (j, m)
//     ACT_SWEEP lo hi     (c1, s1, c2, s2) for k = lo .. hi-1: V columns
//                         (k, k+1) by (c1, s1), U columns (k, k+1) by (c2, s2)
//     ACT_CHASE_ROW kz n  (c, s) for j = kz+1 .. kz+n: U columns (j, kz)
//     ACT_CHASE_COL je hi (c, s) for j = hi-1 down to je: V columns (j, hi)
//   int hdr[hdr_cap(L)]    hdr[0] = number of actions, or -1 when the log
//                          overflowed; hdr[1 + a] = act | p1 << 8 | p2 << 16
// A rotation of columns (a, b) by (c, s): X_a <- c X_a + s X_b,
// X_b <- -s X_a + c X_b.
__host__ __device__ __forceinline__ int cs_cap(int L) { return 8 * L * L + 64; }
__host__ __device__ __forceinline__ int hdr_cap(int L) { return 6 * L + 32; }
__host__ __device__ __forceinline__ size_t cs_bytes(int L) {
    return ((sizeof(real_t) * (size_t)cs_cap(L)) + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t log_stride(int L) {
    return cs_bytes(L) + ((sizeof(int) * (size_t)hdr_cap(L) + 15) & ~(size_t)15);
}

// plane rotation for the leaf iteration (same convention as make_rot).  FP64:
// with both magnitudes inside [2^-500, 2^500) (exponents compared as
// integers) r^2 = f^2 + g^2 cannot overflow or underflow, and one reciprocal
// square root gives c, s and r (r = r^2 / r), in place of hypot and two
// divisions; other inputs take make_rot.
__device__ __forceinline__ void leaf_rot(real_t f, real_t g, real_t &c, real_t &s, real_t &r) {
#ifdef BDC_FP32
    make_rot(f, g, c, s, r);
#else
    const long long fb = __double_as_longlong(f), gb = __double_as_longlong(g);
    if ((gb << 1) == 0) { c = 1.0; s = 0.0; r = f; return; }
    if ((fb << 1) == 0) { c = 0.0; s = 1.0; r = g; return; }
    const int ef = (int)((fb >> 52) & 0x7ff), eg = (int)((gb >> 52) & 0x7ff);
    const int em = ef > eg ? ef : eg;
    if (em >= 1023 - 500 && em < 1023 + 500) {
        const double t = fma(g, g, f * f);
        const double y = rsqrt(t);
        c = f * y; s = g * y; r = t * y;
        return;
    }
    make_rot(f, g, c, s, r);
#endif
}

#ifdef BDC_FP32
constexpr int kMant = 23, kEpsExp = 23;   // kEps = 2^-23
#else
constexpr int kMant = 52, kEpsExp = 52;   // kEps = 2^-52
#endif

// The leaf's negligibility test |e| <= kEps (|d1| + |d2|) or |e| <= tabs,
// decided on the bit patterns where that is exact (|e| > 2^(1-kEpsExp)
// max|d| is never negligible, |e| <= 2^-kEpsExp max|d| always is) and in
// floating point only in the factor-2 band between (same results as the
// floating-point test alone).
__device__ __forceinline__ bool negligible(real_t e, real_t d1, real_t d2, rbits_t tabs) {
    const rbits_t be = abits(e);
    if (be <= tabs) return true;
    const rbits_t b1 = abits(d1), b2 = abits(d2), bm = b1 > b2 ? b1 : b2;
    if (bm >= ((rbits_t)(kEpsExp + 1) << kMant)) {
        if (be > bm - ((rbits_t)(kEpsExp - 1) << kMant)) return false;
        if (be <= bm - ((rbits_t)kEpsExp << kMant)) return true;
    }
    return fabs(e) <= kEps * (fabs(d1) + fabs(d2));
}

// ---------------------------------------------------------------- kernel 1
// one leaf per lane; the leaf's d, e (and, for singular values only, its two
// rows of V) live in shared memory with a stride of 32 (lane-interleaved)
struct LaneVec {
    real_t *p;
    __device__ __forceinline__ real_t &operator[](int i) const { return p[i * 32]; }
};

__global__ void __launch_bounds__(32) k_leaf_rotations(const NodeDesc *__restrict__ leaves,
                                                       const MatDesc *__restrict__ mats, int nleaves, int L,
                                                       int per_warp, int max_sweeps, int ccap,
                                                       char *__restrict__ log, NodeState *__restrict__ state) {
    extern __shared__ real_t sm[];
    const int lane = threadIdx.x;
    const int li = blockIdx.x * per_warp + lane;
    if (lane >= per_warp || li >= nleaves) return;
    const NodeDesc nd = leaves[li];
    const MatDesc &md = mats[nd.mat];
    const int m = nd.m, sq = nd.sqre, mc = m + sq, r0 = nd.r0;
    const bool vals = md.vals != 0;
    const LaneVec dd{sm + lane}, ee{sm + 32 * (L + 1) + lane};
    const LaneVec vf{sm + 64 * (L + 1) + lane}, vl{sm + 96 * (L + 1) + lane};
    real_t *cs = nullptr;
    int *hdr = nullptr;
    if (!vals) {
        char *lg = log + (size_t)li * log_stride(L);
        cs = (real_t *)lg;
        hdr = (int *)(lg + cs_bytes(L));
    }
    const int hcap = hdr_cap(L);
    int na = 0, nc = 0;
    bool ovf = false;
    // room for one more action with `need` log entries (always true for values only)
    auto room = [&](int need) {
        if (vals) return true;
        if (na + 2 > hcap || nc + need > ccap) ovf = true;
        return !ovf;
    };
    auto put = [&](real_t c, real_t s) { if (!vals) { cs[nc] = c; cs[nc + 1] = s; } nc += 2; };
    auto act = [&](int a, int p1, int p2) { if (!vals) hdr[1 + na] = a | (p1 << 8) | (p2 << 16); ++na; };
    // values only: V columns (a, b) on the two tracked rows
    auto vrot = [&](int a, int b, real_t c, real_t s) {
        real_t u = vf[a], v = vf[b];
        vf[a] = c * u + s * v;
        vf[b] = -s * u + c * v;
        u = vl[a]; v = vl[b];
        vl[a] = c * u + s * v;
        vl[b] = -s * u + c * v;
    };

    for (int i = 0; i < m; ++i) dd[i] = md.dsc[r0 + i];
    for (int i = 0; i < m - 1 + sq; ++i) ee[i] = md.esc[r0 + i];
    if (vals)
        for (int j = 0; j < mc; ++j) { vf[j] = (j == 0) ? R(1) : R(0); vl[j] = (j == mc - 1) ? R(1) : R(0); }

    // ---- rectangular leaf: rotate the extra column (index m) away
    if (sq && room(2 * m)) {
        real_t x = ee[m - 1];
        for (int j = m - 1; j >= 0; --j) {
            real_t c, s, r;
            leaf_rot(dd[j], x, c, s, r);
            dd[j] = r;
            if (j > 0) { x = -s * ee[j - 1]; ee[j - 1] = c * ee[j - 1]; }
            put(c, s);
            if (vals) vrot(j, m, c, s);
        }
        ee[m - 1] = R(0);
        act(ACT_SQRE, m, 0);
    }

    // leaf-local norm for the zero-diagonal threshold (max of the bit patterns)
    rbits_t bb = 0;
    for (int i = 0; i < m; ++i) { const rbits_t b = abits(dd[i]); bb = b > bb ? b : bb; }
    for (int i = 0; i < m - 1; ++i) { const rbits_t b = abits(ee[i]); bb = b > bb ? b : bb; }
#ifdef BDC_FP32
    const real_t dtiny = kEps * __int_as_float(bb);
#else
    const real_t dtiny = kEps * __longlong_as_double(bb);
#endif
    const rbits_t tiny_b = abits(dtiny), tabs = abits(dtiny * kEps);

    long long budget = (long long)max_sweeps * (m > 0 ? m : 1);
    int info = 0, hi = m - 1;
    // One action per pass, the bottom deflations of a pass included, so that
    // the lanes of a warp (different leaves) start their sweeps together
    while (!ovf) {
        while (hi > 0 && negligible(ee[hi - 1], dd[hi - 1], dd[hi], tabs)) {
            ee[hi - 1] = R(0);
            --hi;
        }
        if (hi <= 0) break;
        int lo = hi - 1;
        while (lo > 0 && !negligible(ee[lo - 1], dd[lo - 1], dd[lo], tabs)) --lo;
        if (lo > 0) ee[lo - 1] = R(0);
        int kz = -1;
        for (int k = lo; k <= hi; ++k)
            if (abits(dd[k]) <= tiny_b) { kz = k; break; }
        if (kz < 0 && budget-- <= 0) {
            int cnt = 0;
            for (int i = 0; i < hi; ++i) cnt += (ee[i] != R(0));
            info = cnt > 0 ? cnt : 1;
            break;
        }
        if (!room(kz >= 0 ? 2 * (hi - lo + 1) : 4 * (hi - lo))) break;
        if (kz >= 0) {
            dd[kz] = R(0);
            if (kz < hi) {            // clear row kz with rows kz+1..hi (U rotations)
                real_t x = ee[kz];
                ee[kz] = R(0);
                int cnt = 0;
                for (int j = kz + 1; j <= hi && x != R(0); ++j) {
                    real_t c, s, r;
                    leaf_rot(dd[j], x, c, s, r);
                    dd[j] = r;
                    if (j < hi) { x = -s * ee[j]; ee[j] = c * ee[j]; }
                    put(c, s);
                    cnt = j - kz;
                }
                act(ACT_CHASE_ROW, kz, cnt);
            } else {                  // clear column hi with columns hi-1..lo (V rotations)
                real_t x = ee[hi - 1];
                ee[hi - 1] = R(0);
                int jend = hi;
                for (int j = hi - 1; j >= lo && x != R(0); --j) {
                    real_t c, s, r;
                    leaf_rot(dd[j], x, c, s, r);
                    dd[j] = r;
                    if (j > lo) { x = -s * ee[j - 1]; ee[j - 1] = c * ee[j - 1]; }
                    put(c, s);
                    if (vals) vrot(j, hi, c, s);
                    jend = j;
                }
                act(ACT_CHASE_COL, jend, hi);
            }
            continue;
        }
        // Golub-Kahan sweep on [lo, hi] with a Wilkinson shift
        const real_t dm = dd[hi - 1], dn = dd[hi], em = ee[hi - 1];
        const real_t el = (hi - 1 > lo) ? ee[hi - 2] : R(0);
        const real_t t11 = dm * dm + el * el, t22 = dn * dn + em * em, t12 = dm * em;
        const real_t delta = R(0.5) * (t11 - t22);
        const real_t sg = (delta >= R(0)) ? R(1) : R(-1);
        const real_t den = delta + sg * hypot(delta, t12);
        const real_t mu = (den != R(0)) ? t22 - t12 * t12 / den : t22;
        // the chain runs in registers: dk, ek are d_k, e_k as updated by the
        // previous step, dk1, ek1 the untouched d_{k+1}, e_{k+1}, loaded one
        // step ahead; every store is final (e_{k-1} takes the next step's r)
        real_t dk = dd[lo], ek = ee[lo];
        real_t dk1 = dd[lo + 1], ek1 = (lo + 1 < hi) ? ee[lo + 1] : R(0);
        real_t y = dk * dk - mu;
        real_t z = dk * ek;
        for (int k = lo; k < hi; ++k) {
            const real_t dk2 = (k + 2 <= hi) ? dd[k + 2] : R(0);
            const real_t ek2 = (k + 2 < hi) ? ee[k + 2] : R(0);
            real_t c, s, r;
            leaf_rot(y, z, c, s, r);
            if (k > lo) ee[k - 1] = r;
            const real_t dka = c * dk + s * ek;
            const real_t eka = -s * dk + c * ek;
            const real_t bulge = s * dk1;
            const real_t dk1a = c * dk1;
            put(c, s);
            if (vals) vrot(k, k + 1, c, s);
            leaf_rot(dka, bulge, c, s, r);
            dd[k] = r;
            const real_t ekb = c * eka + s * dk1a;      // e_k after this step (y of the next)
            const real_t dk1b = -s * eka + c * dk1a;    // d_{k+1} after this step
            if (k < hi - 1) {
                z = s * ek1;
                ek = c * ek1;
                y = ekb;
            } else {
                ee[k] = ekb;
                dd[k + 1] = dk1b;
            }
            dk = dk1b;
            dk1 = dk2;
            ek1 = ek2;
            if (!vals) { cs[nc] = c; cs[nc + 1] = s; }
            nc += 2;
        }
        act(ACT_SWEEP, lo, hi);
    }

    // rotations formed (the stage profiler's FP64 operation count); leaves
    // have no other use for their node state
    state[nd.id].iters = (unsigned long long)(nc / 2);
    if (!vals) {
        if (ovf) { hdr[0] = -1; return; }       // k_leaf_vectors iterates this leaf itself
        for (int i = 0; i < m; ++i) md.D[r0 + i] = dd[i];   // signed; sorted by k_leaf_vectors
        hdr[0] = na;
        if (info) atomicAdd(md.info, info);
        return;
    }
    // values only: non-negative values (flip the matching column of V), ascending order
    for (int j = 0; j < m; ++j)
        if (dd[j] < R(0)) { dd[j] = -dd[j]; vf[j] = -vf[j]; vl[j] = -vl[j]; }
    real_t *VF = md.vf[nd.buf], *VL = md.vl[nd.buf];
    for (int j = 0; j < m; ++j) {
        const real_t v = dd[j];
        int rank = 0;
        for (int i = 0; i < m; ++i) {
            const real_t w = dd[i];
            rank += (w < v) || (w == v && i < j);
        }
        md.D[r0 + rank] = v;
        VF[r0 + rank] = vf[j];
        VL[r0 + rank] = vl[j];
        md.Q[r0 + j] = j;
    }
    if (sq) { VF[r0 + m] = vf[m]; VL[r0 + m] = vl[m]; }
    if (info) atomicAdd(md.info, info);
}

// ---------------------------------------------------------------- kernel 2
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

// The QR iteration of a leaf whose log overflowed: lane 0 forms each action's
// rotations (the same steps as k_leaf_rotations), all lanes apply them.
__device__ void leaf_iterate(real_t *Us, real_t *Vs, real_t *dd, real_t *ee, real_t *c1, real_t *s1, real_t *c2,
                             real_t *s2, volatile LeafCtl *ctl, int m, int sq, int L, int max_sweeps, int lane) {
    const int ldu = L, ldv = L + 1, mc = m + sq;
    if (sq) {
        if (lane == 0) {
            real_t x = ee[m - 1];
            for (int j = m - 1; j >= 0; --j) {
                real_t c, s, r;
                leaf_rot(dd[j], x, c, s, r);
                dd[j] = r;
                c1[j] = c; s1[j] = s;
                if (j > 0) { x = -s * ee[j - 1]; ee[j - 1] = c * ee[j - 1]; }
            }
            ee[m - 1] = R(0);
        }
        __syncwarp();
        for (int j = m - 1; j >= 0; --j) rot_rows(Vs, ldv, mc, lane, j, m, c1[j], s1[j]);
        __syncwarp();
    }
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
                    if (kz < hi) {
                        real_t x = ee[kz];
                        ee[kz] = R(0);
                        int cnt = 0;
                        for (int j = kz + 1; j <= hi && x != R(0); ++j) {
                            real_t c, s, r;
                            leaf_rot(dd[j], x, c, s, r);
                            dd[j] = r;
                            if (j < hi) { x = -s * ee[j]; ee[j] = c * ee[j]; }
                            c2[j] = c; s2[j] = s;
                            cnt = j - kz;
                        }
                        act = ACT_CHASE_ROW; ctl->k = kz; ctl->cnt = cnt;
                    } else {
                        real_t x = ee[hi - 1];
                        ee[hi - 1] = R(0);
                        int jend = hi;
                        for (int j = hi - 1; j >= lo && x != R(0); --j) {
                            real_t c, s, r;
                            leaf_rot(dd[j], x, c, s, r);
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
                        leaf_rot(y, z, c, s, r);
                        if (k > lo) ee[k - 1] = r;
                        real_t dk = dd[k], ek = ee[k], dk1 = dd[k + 1];
                        dd[k] = c * dk + s * ek;
                        ee[k] = -s * dk + c * ek;
                        real_t bulge = s * dk1;
                        dd[k + 1] = c * dk1;
                        c1[k] = c; s1[k] = s;
                        leaf_rot(dd[k], bulge, c, s, r);
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
            for (int k = lo; k < hi; ++k) rot_rows(Vs, ldv, mc, lane, k, k + 1, c1[k], s1[k]);
            for (int k = lo; k < hi; ++k) rot_rows(Us, ldu, m, lane, k, k + 1, c2[k], s2[k]);
        } else if (act == ACT_CHASE_ROW) {
            const int kz = ctl->k, cnt = ctl->cnt;
            for (int j = kz + 1; j <= kz + cnt; ++j) rot_rows(Us, ldu, m, lane, j, kz, c2[j], s2[j]);
        } else if (act == ACT_CHASE_COL) {
            const int hi = ctl->hi, jend = ctl->k;
            for (int j = hi - 1; j >= jend; --j) rot_rows(Vs, ldv, mc, lane, j, hi, c1[j], s1[j]);
        }
        __syncwarp();
    }
}

// One chain of rotations on one row x (stride ld) of U or V: columns
// (first + i*step, pivot) for i = 0..n-1 with (c, s) = st[2 i], st[2 i + 1]
// (stride w between pairs); the pivot column's entry is carried in a register.
__device__ __forceinline__ void chain_pivot(real_t *x, int ld, int first, int step, int n, int pivot,
                                            const real_t *st, int w) {
    real_t carry = x[pivot * ld];
    for (int i = 0; i < n; ++i) {
        const int j = first + i * step;
        const real_t c = st[w * i], s = st[w * i + 1];
        const real_t a = x[j * ld];
        x[j * ld] = c * a + s * carry;
        carry = -s * a + c * carry;
    }
    x[pivot * ld] = carry;
}

__global__ void __launch_bounds__(32) k_leaf_vectors(const NodeDesc *__restrict__ leaves,
                                                     const MatDesc *__restrict__ mats, int L, int max_sweeps,
                                                     const char *__restrict__ log) {
    extern __shared__ real_t sm[];
    const int lane = threadIdx.x;
    const NodeDesc nd = leaves[blockIdx.x];
    const MatDesc &md = mats[nd.mat];
    const int m = nd.m, sq = nd.sqre, mc = m + sq;
    const int ldu = L, ldv = L + 1;
    real_t *Us = sm;
    real_t *Vs = Us + (size_t)L * L;
    real_t *dd = Vs + (size_t)(L + 1) * (L + 1);
    real_t *ee = dd + (L + 1);
    real_t *st = ee + (L + 1);               // 4 (L + 1): staged rotations / c1 s1 c2 s2
    int *perm = (int *)(st + 4 * (L + 1));
    volatile LeafCtl *ctl = (volatile LeafCtl *)(perm + L + 2);
    const char *lg = log + (size_t)blockIdx.x * log_stride(L);
    const real_t *cs = (const real_t *)lg;
    const int *hdr = (const int *)(lg + cs_bytes(L));
    const int na = hdr[0];
    const int r0 = nd.r0;

    for (int j = 0; j < m; ++j)
        for (int r = lane; r < m; r += 32) Us[j * ldu + r] = (r == j) ? R(1) : R(0);
    for (int j = 0; j < mc; ++j)
        for (int r = lane; r < mc; r += 32) Vs[j * ldv + r] = (r == j) ? R(1) : R(0);

    if (na >= 0) {
        for (int i = lane; i < m; i += 32) dd[i] = md.D[r0 + i];
        int pos = 0;
        for (int a = 0; a < na; ++a) {
            const int code = hdr[1 + a];
            const int act = code & 255, p1 = (code >> 8) & 255, p2 = code >> 16;
            const int w = (act == ACT_SWEEP) ? 4 : 2;
            const int cnt = (act == ACT_SQRE) ? p1 : (act == ACT_SWEEP) ? p2 - p1
                          : (act == ACT_CHASE_ROW) ? p2 : p2 - p1;
            __syncwarp();
            for (int i = lane; i < w * cnt; i += 32) st[i] = cs[pos + i];
            __syncwarp();
            pos += w * cnt;
            if (act == ACT_SWEEP) {
                // V rows then U rows, one row per task; (k, k+1) for k = p1 .. p2-1
                for (int t = lane; t < mc + m; t += 32) {
                    const bool isv = t < mc;
                    real_t *x = isv ? Vs + t : Us + (t - mc);
                    const int ld = isv ? ldv : ldu;
                    const real_t *cp = st + (isv ? 0 : 2);
                    real_t carry = x[p1 * ld];
                    for (int k = p1; k < p2; ++k) {
                        const real_t c = cp[4 * (k - p1)], s = cp[4 * (k - p1) + 1];
                        const real_t b = x[(k + 1) * ld];
                        x[k * ld] = c * carry + s * b;
                        carry = -s * carry + c * b;
                    }
                    x[p2 * ld] = carry;
                }
            } else if (act == ACT_SQRE) {
                for (int t = lane; t < mc; t += 32) chain_pivot(Vs + t, ldv, m - 1, -1, m, m, st, 2);
            } else if (act == ACT_CHASE_ROW) {
                for (int t = lane; t < m; t += 32) chain_pivot(Us + t, ldu, p1 + 1, 1, p2, p1, st, 2);
            } else {   // ACT_CHASE_COL
                for (int t = lane; t < mc; t += 32) chain_pivot(Vs + t, ldv, p2 - 1, -1, p2 - p1, p2, st, 2);
            }
        }
        __syncwarp();
    } else {
        for (int i = lane; i < m; i += 32) dd[i] = md.dsc[r0 + i];
        for (int i = lane; i < m - 1 + sq; i += 32) ee[i] = md.esc[r0 + i];
        if (lane == 0) { ctl->info = 0; ctl->hi = m - 1; }
        __syncwarp();
        leaf_iterate(Us, Vs, dd, ee, st, st + (L + 1), st + 2 * (L + 1), st + 3 * (L + 1), ctl, m, sq, L,
                     max_sweeps, lane);
    }

    // non-negative values: flip the matching right vector
    for (int j = 0; j < m; ++j) {
        if (dd[j] < R(0)) {
            for (int r = lane; r < mc; r += 32) Vs[j * ldv + r] = -Vs[j * ldv + r];
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
    // node column p in slot r0 + p (rows r0..r0+m-1 of U, r0..r0+mc-1 of V)
    const long long ld = md.n;
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
    __syncwarp();
    for (int p = lane; p < m; p += 32) {
        md.D[r0 + p] = dd[perm[p]];
        md.Q[r0 + p] = p;
    }
    if (na < 0 && lane == 0 && ctl->info != 0) atomicAdd(md.info, ctl->info);
}

int leaf_sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

}  // namespace

size_t leaf_log_bytes(int leafmax) { return log_stride(leafmax < 1 ? 1 : leafmax); }

cudaError_t launch_leaves(const NodeDesc *leaves, int nleaves, const MatDesc *mats, int leafmax,
                          int max_sweeps, int vals, void *log, NodeState *state, cudaStream_t st) {
    if (nleaves <= 0) return cudaSuccess;
    const int L = leafmax;
    // up to four warps per SM, one per sub-partition: the chain of one leaf
    // is bound by the issue rate of its sub-partition's FP64 unit, so the
    // leaves are spread over as many sub-partitions as possible before they
    // share a warp
    const int target = 4 * leaf_sm_count();
    // log capacity: cs_cap(L) entries; the environment variable
    // BDC_LEAF_LOG_ENTRIES can lower it (tests use it to send leaves through
    // the fallback iteration of k_leaf_vectors)
    int ccap = cs_cap(L);
    if (const char *env = std::getenv("BDC_LEAF_LOG_ENTRIES")) {
        const int v = std::atoi(env);
        if (v >= 0 && v < ccap) ccap = v;
    }
    int per_warp = (nleaves + target - 1) / target;
    per_warp = per_warp < 1 ? 1 : per_warp > 32 ? 32 : per_warp;
    const size_t smem1 = sizeof(real_t) * 32 * (size_t)(L + 1) * (vals ? 4 : 2);
    if (smem1 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf_rotations, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem1);
        if (e != cudaSuccess) return e;
    }
    k_leaf_rotations<<<(nleaves + per_warp - 1) / per_warp, 32, smem1, st>>>(leaves, mats, nleaves, L, per_warp,
                                                                             max_sweeps, ccap, (char *)log, state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || vals) return e;
    const size_t smem2 = sizeof(real_t) * ((size_t)L * L + (size_t)(L + 1) * (L + 1) + 6 * (size_t)(L + 1)) +
                         sizeof(int) * (L + 2) + sizeof(LeafCtl) + 16;
    if (smem2 > 48 * 1024) {
        e = cudaFuncSetAttribute(k_leaf_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
    }
    k_leaf_vectors<<<nleaves, 32, smem2, st>>>(leaves, mats, L, max_sweeps, (const char *)log);
    return cudaGetLastError();
}

}  // namespace BDC_NS
