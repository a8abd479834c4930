// Merge step of Algorithm 2, part (a) "deflate singular values" (lasd2) and
// the bookkeeping around part (b), all on the GPU.
//
// k_merge_prep   (one CTA per node)  z formation (Sec. 4.2.1: the coupling
//                row times the children's right vectors), merge of the two
//                sorted child value lists, deflation tests (Eq. M-condition)
//                and the rotation chains of the four deflation cases, column
//                typing (top / dense / bottom, the blocks of Eq. bdc-W-Q) and
//                the K order [top | pad | d_0 column | dense | bottom] used by
//                the merge products of Eq. (bdc-Mv2Bv-u-vt).
// k_merge_order  (merges of order >= 4096, a grid per node) the merged order
//                and z of the prep's first two phases, so that the prep of
//                those merges starts at the deflation.
// k_merge_gather (one CTA per column task) applies the rotations and writes
//                the survivors' vectors W~ (left) and Q~ (right) into the
//                workspace at their K position, and the deflated vectors and
//                the new right null vector straight into the node's block.
// k_merge_finish writes the node's values (roots, then deflated values,
//                Eq. bdc-B-svd) and their ascending order.
//
// The sequential deflation scan is parallelised exactly: the small-z test
// uses the original z, so survivors of it are found with a block scan; the
// close-value test only compares consecutive survivors, so chains of close
// values are independent and each is walked by one thread.  The scans over
// a node's positions go by warps over chunks of 32 consecutive positions,
// several chunks' loads in flight together: the merges at the top of the
// tree have one CTA for thousands of positions, and a loop that waited on
// one load per chunk would be bound by the round trips.
#include <algorithm>
#include <mutex>

#include "bdc_internal.cuh"

namespace BDC_NS {

namespace {

constexpr int PREP_THREADS = 512;
// chunks of 32 positions whose loads the deflation and numbering loops of
// the prep issue together (one round trip per batch instead of per chunk)
constexpr int kDeflBatch = 8;
constexpr int kNumBatch = 4;      // the same for the survivor numbering (more loads per chunk)
constexpr int FL_START = 16, FL_MEMBER = 32;

__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = (lane < nw) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    const int base = (w > 0) ? wsum[w - 1] : 0;
    total = wsum[nw - 1];
    __syncthreads();
    return base + x - v;
}


__device__ __forceinline__ int block_isum(int v, int *wsum) {
    int t;
    block_excl_scan(v, wsum, t);
    return t;
}

// exclusive block scan of real_ts in thread order (reverse = false: sum over
// threads before t; true: over threads after t); no subtraction, so small
// partial sums keep their relative accuracy
__device__ __forceinline__ real_t block_excl_scan_d(real_t v, real_t *buf, bool reverse) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    real_t x = v;
    if (!reverse) {
        for (int o = 1; o < 32; o <<= 1) {
            const real_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
    } else {
        for (int o = 1; o < 32; o <<= 1) {
            const real_t y = __shfl_down_sync(0xffffffffu, x, o);
            if (lane + o < 32) x += y;
        }
    }
    real_t ex = reverse ? __shfl_down_sync(0xffffffffu, x, 1) : __shfl_up_sync(0xffffffffu, x, 1);
    if (reverse ? lane == 31 : lane == 0) ex = 0.0;
    if (reverse ? lane == 0 : lane == 31) buf[w] = x;
    __syncthreads();
    if (w == 0) {
        real_t t = (lane < nw) ? buf[lane] : R(0);
        real_t tx = t;
        if (!reverse) {
            for (int o = 1; o < 32; o <<= 1) {
                const real_t y = __shfl_up_sync(0xffffffffu, tx, o);
                if (lane >= o) tx += y;
            }
        } else {
            for (int o = 1; o < 32; o <<= 1) {
                const real_t y = __shfl_down_sync(0xffffffffu, tx, o);
                if (lane + o < 32) tx += y;
            }
        }
        // exclusive over warps
        real_t e = reverse ? __shfl_down_sync(0xffffffffu, tx, 1) : __shfl_up_sync(0xffffffffu, tx, 1);
        if (reverse ? lane == 31 : lane == 0) e = 0.0;
        __syncwarp();
        if (lane < nw) buf[lane] = e;
    }
    __syncthreads();
    const real_t r = buf[w] + ex;
    __syncthreads();
    return r;
}

// side of a pre-deflation column: 1 = rows of the left child, 2 = right
__device__ __forceinline__ int col_side(int c, int nl) { return c == 0 ? 0 : (c <= nl ? 1 : 2); }

// Deflation of the sorted (ds, zs), ds[0] = 0, tolerance tol (Sec. 4.2.1):
// fills slist/sidx/role, rotation (rc, rs) attached to the later member of
// each rotated pair, and the final z of every survivor in place in zs.
// src (may be null) gives the pre-deflation column of each position, used to
// type survivors.  Returns the number ns of small-z survivors.
__device__ int deflate_core(int m, real_t tol, const real_t *ds, real_t *zs, const int *src, int nl,
                            int *slist, int *sidx, int *role, real_t *rc, real_t *rs, int *wsum,
                            int *a_out) {
    const int T = blockDim.x, t = threadIdx.x;
    const int lane = t & 31, nw = T >> 5;
    const unsigned lt = (1u << lane) - 1u;       // lanes below this one
    // z_0 (paired with d_0 = 0) is clamped up to tol, never deflated
    if (t == 0) {
        real_t z0 = zs[0];
        if (abits(z0) < abits(tol)) zs[0] = (z0 < R(0)) ? -tol : tol;
    }
    __syncthreads();
    const rbits_t tolb = abits(tol);
    // survivors (position 0 and |z| > tol), numbered in ascending position
    // order.  Warp w takes the positions [wb, we) in chunks of 32 consecutive
    // ones (lane = position: coalesced), the loads of kDeflBatch chunks in
    // flight together; a chunk's survivors are counted by a ballot and
    // numbered by the population count of the lower lanes.
    const int wspan = ((m + nw - 1) / nw + 31) & ~31;
    const int wb = min(m, (t >> 5) * wspan), we = min(m, wb + wspan);
    int cnt = 0;
    for (int c0 = wb; c0 < we; c0 += 32 * kDeflBatch) {
        rbits_t zb[kDeflBatch];
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            zb[u] = (p < we) ? abits(zs[p]) : (rbits_t)0;
        }
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            cnt += __popc(__ballot_sync(0xffffffffu, p < we && (p == 0 || zb[u] > tolb)));
        }
    }
    int ns;
    int k = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt : 0, wsum, ns), 0);
    for (int c0 = wb; c0 < we; c0 += 32 * kDeflBatch) {
        rbits_t zb[kDeflBatch];
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            zb[u] = (p < we) ? abits(zs[p]) : (rbits_t)0;
        }
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            const bool keep = p < we && (p == 0 || zb[u] > tolb);
            const unsigned b = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int kk = k + __popc(b & lt);
                slist[kk] = p; sidx[p] = kk;
            } else if (p < we) {
                sidx[p] = -1;
                role[p] = ROLE_DEFL;
            }
            k += __popc(b);
        }
    }
    __syncthreads();
    // survivors close to d_0 = 0 form a prefix of slist (ds ascending)
    const int sseg = (ns + T - 1) / T;
    const int sb = min(ns, t * sseg), se = min(ns, sb + sseg);
    int za = 0;
    for (int kk = max(sb, 1); kk < se; ++kk) za += (abits(ds[slist[kk]]) <= tolb);
    const int a = block_isum(za, wsum);
    for (int kk = sb; kk < se; ++kk) {
        const int p = slist[kk];
        int r;
        if (kk == 0) {
            r = ROLE_KEEP;
        } else if (kk <= a) {
            r = ROLE_ZERO;
        } else {
            const bool closeK = (kk >= a + 2) && (ds[p] - ds[slist[kk - 1]] <= tol);
            const bool nextClose = (kk + 1 < ns) && (kk + 1 >= a + 2) && (ds[slist[kk + 1]] - ds[p] <= tol);
            if (nextClose) r = ROLE_CHAIN | FL_MEMBER | (closeK ? 0 : FL_START);
            else r = ROLE_KEEP | (closeK ? FL_MEMBER : 0);
            if (!nextClose && !closeK) r |= (src ? col_side(src[p], nl) : 1) << 8;
        }
        role[p] = r;
    }
    __syncthreads();
    // walk each chain of close values: the earlier z is rotated into the later
    for (int kk = sb; kk < se; ++kk) {
        const int p = slist[kk];
        if ((role[p] & 15) != ROLE_CHAIN || !(role[p] & FL_START)) continue;
        real_t zr = zs[p];
        int ty = src ? col_side(src[p], nl) : 1;
        for (int j = kk + 1; j < ns; ++j) {
            const int q = slist[j];
            const real_t zq = zs[q];
            real_t c, s, r;
            make_rot(zq, zr, c, s, r);    // c = z_q / r, s = z_prev / r
            rc[q] = c; rs[q] = s;
            zr = r;
            ty |= src ? col_side(src[q], nl) : 1;
            if ((role[q] & 15) == ROLE_KEEP) {
                zs[q] = zr;
                role[q] |= ty << 8;
                break;
            }
        }
    }
    // values close to d_0 = 0: right-side rotations fold them into z_0
    if (t == 0 && a > 0) {
        real_t zr = zs[0];
        for (int j = 1; j <= a; ++j) {
            const int q = slist[j];
            const real_t zq = zs[q];
            real_t c, s, r;
            make_rot(zr, zq, c, s, r);    // c = z_0 / r, s = z_q / r
            rc[q] = c; rs[q] = s;
            zr = r;
        }
        zs[0] = zr;
    }
    __syncthreads();
    *a_out = a;
    return ns;
}

// The merged ascending order and z of positions 1..m-1 of the merges of
// one height, for large merges: the same merge path and z formation as the
// prep's first two phases, spread over a grid (blockIdx.x = share of the
// node's positions, blockIdx.y = node; at most ORDER_SPAN positions per
// thread), each thread forming z at the positions it has just placed, so
// that the single-CTA prep of a large merge starts at the deflation.
constexpr int ORDER_THREADS = 256, ORDER_SPAN = 4, ORDER_MIN = 4096;

__global__ void __launch_bounds__(ORDER_THREADS) k_merge_order(const NodeDesc *__restrict__ nodes,
                                                               const MatDesc *__restrict__ mats) {
    const NodeDesc nd = nodes[blockIdx.y];
    const MatDesc &md = mats[nd.mat];
    const int m = nd.m, nl = nd.nl, nr = m - nl - 1;
    const int r0 = nd.r0, r0L = r0, r0R = r0 + nl + 1;
    const long long ld = md.n;
    const int mt = nl + nr, T = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = (mt + T - 1) / T;
    const int k0 = min(mt, t * S), k1 = min(mt, k0 + S);
    if (k0 >= k1) return;
    real_t *ds = md.ds + r0, *zs = md.zs + r0;
    int *src = md.src + r0;
    const real_t alpha = md.dsc[r0 + nl], beta = md.esc[r0 + nl];
    const int *cvs = md.vs[1 - nd.buf];
    const int *QL = md.Q + r0L, *QR = md.Q + r0R;
    const real_t *DL = md.D + r0L, *DR = md.D + r0R;
    int lo = max(0, k0 - nr), hi = min(k0, nl);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (abits(DL[QL[mid]]) <= abits(DR[QR[k0 - mid - 1]])) lo = mid + 1; else hi = mid;
    }
    int i = lo, j = k0 - lo;
    real_t a = (i < nl) ? DL[QL[i]] : R(INFINITY);
    real_t b = (j < nr) ? DR[QR[j]] : R(INFINITY);
    int cs[ORDER_SPAN];
#pragma unroll
    for (int u = 0; u < ORDER_SPAN; ++u) {
        const int k = k0 + u;
        if (k >= k1) break;
        if (j >= nr || (i < nl && abits(a) <= abits(b))) {
            ds[1 + k] = a;
            cs[u] = 1 + QL[i];
            ++i;
            a = (i < nl) ? DL[QL[i]] : R(INFINITY);
        } else {
            ds[1 + k] = b;
            cs[u] = nl + 1 + QR[j];
            ++j;
            b = (j < nr) ? DR[QR[j]] : R(INFINITY);
        }
        src[1 + k] = cs[u];
    }
    // z: alpha times the last row of a left child's right vector, beta times
    // the first row of a right child's (the loads of the span in flight together)
    real_t zv[ORDER_SPAN];
    bool left[ORDER_SPAN];
#pragma unroll
    for (int u = 0; u < ORDER_SPAN; ++u) {
        zv[u] = R(0);
        left[u] = true;
        if (k0 + u >= k1) continue;
        const int c = cs[u];
        left[u] = c <= nl;
        const int jx = left[u] ? r0L + c - 1 : r0R + (c - nl - 1);
        if (md.vals) {
            zv[u] = left[u] ? md.vl[1 - nd.buf][jx] : md.vf[1 - nd.buf][jx];
        } else {
            const int g = cvs[jx];
            const long long row = left[u] ? r0L + nl : r0R;
            const real_t v = md.V[(size_t)g * ld + row];
            zv[u] = (row >= md.vlo[g] && row < md.vhi[g]) ? v : R(0);
        }
    }
#pragma unroll
    for (int u = 0; u < ORDER_SPAN; ++u)
        if (k0 + u < k1) zs[1 + k0 + u] = (left[u] ? alpha : beta) * zv[u];
}

// ordered = 1: k_merge_order has written ds, src and zs at positions 1..m-1
__global__ void __launch_bounds__(PREP_THREADS) k_merge_prep(const NodeDesc *__restrict__ nodes,
                                                             const MatDesc *__restrict__ mats,
                                                             NodeState *__restrict__ state,
                                                             GemmProb *__restrict__ probs, int scans,
                                                             int ordered) {
    __shared__ int wsum[PREP_THREADS / 32 + 1];
    __shared__ real_t dsum[PREP_THREADS / 32 + 1];
    const NodeDesc nd = nodes[blockIdx.x];
    const MatDesc &md = mats[nd.mat];
    const int m = nd.m, nl = nd.nl, nr = m - nl - 1, sqre = nd.sqre, mc = m + sqre;
    const int r0 = nd.r0, r0L = r0, r0R = r0 + nl + 1;
    const long long ld = md.n;
    const int T = blockDim.x, t = threadIdx.x;
    real_t *ds = md.ds + r0, *zs = md.zs + r0;
    int *src = md.src + r0;
    const real_t alpha = md.dsc[r0 + nl], beta = md.esc[r0 + nl];
    // children's right vectors: node column j of a child lives in slot
    // vs[1 - buf][child r0 + j]; rows outside the slot's range read as zero
    const int *cvs = md.vs[1 - nd.buf], *cus = md.us[1 - nd.buf];
    auto vrow = [&](int g, long long row) -> real_t {
        return (row >= md.vlo[g] && row < md.vhi[g]) ? md.V[(size_t)g * ld + row] : R(0);
    };

    // ---- the merged ascending order (children are sorted through Q; ties:
    // left first).  Merge path: thread t merges output positions [k0, k1),
    // an equal share, from the split of the two lists found by a binary
    // search on its diagonal; then z of every position, independently.
    // (node values are non-negative: they are compared as bit patterns)
    const int *QL = md.Q + r0L, *QR = md.Q + r0R;
    const real_t *DL = md.D + r0L, *DR = md.D + r0R;
    if (!ordered) {
        const int mt = nl + nr, S = (mt + T - 1) / T;
        const int k0 = min(mt, t * S), k1 = min(mt, k0 + S);
        if (k0 < k1) {
            int lo = max(0, k0 - nr), hi = min(k0, nl);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (abits(DL[QL[mid]]) <= abits(DR[QR[k0 - mid - 1]])) lo = mid + 1; else hi = mid;
            }
            int i = lo, j = k0 - lo;
            real_t a = (i < nl) ? DL[QL[i]] : R(INFINITY);
            real_t b = (j < nr) ? DR[QR[j]] : R(INFINITY);
            for (int k = k0; k < k1; ++k) {
                if (j >= nr || (i < nl && abits(a) <= abits(b))) {
                    ds[1 + k] = a;
                    src[1 + k] = 1 + QL[i];
                    ++i;
                    a = (i < nl) ? DL[QL[i]] : R(INFINITY);
                } else {
                    ds[1 + k] = b;
                    src[1 + k] = nl + 1 + QR[j];
                    ++j;
                    b = (j < nr) ? DR[QR[j]] : R(INFINITY);
                }
            }
        }
    }
    // the largest value ends one of the two sorted lists
    const real_t dmax = fmax(nl > 0 ? DL[QL[nl - 1]] : R(0), nr > 0 ? DR[QR[nr - 1]] : R(0));
    __syncthreads();
    // z of every position: alpha times the last row of a left child's right
    // vector, beta times the first row of a right child's.  Four positions
    // per thread in flight: each level of the chain (source column, its
    // slot, the slot's range and entry) is loaded for all four before the
    // next, and the slot entry unconditionally (it lies inside the slot
    // column whatever its range), so the loads do not wait on one another.
    for (int pos0 = 1 + t; !ordered && pos0 < m; pos0 += 4 * T) {
        int jx[4];
        bool left[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pos = pos0 + u * T;
            const int c = (pos < m) ? src[pos] : 1;
            left[u] = c <= nl;
            jx[u] = left[u] ? r0L + c - 1 : r0R + (c - nl - 1);
        }
        real_t zv[4];
        if (md.vals) {
#pragma unroll
            for (int u = 0; u < 4; ++u) zv[u] = left[u] ? md.vl[1 - nd.buf][jx[u]] : md.vf[1 - nd.buf][jx[u]];
        } else {
            int g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) g[u] = cvs[jx[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long row = left[u] ? r0L + nl : r0R;
                const int lo = md.vlo[g[u]], hi = md.vhi[g[u]];
                const real_t v = md.V[(size_t)g[u] * ld + row];
                zv[u] = (row >= lo && row < hi) ? v : R(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int pos = pos0 + u * T;
            if (pos < m) zs[pos] = (left[u] ? alpha : beta) * zv[u];
        }
    }
    __shared__ real_t s_cq, s_sq;
    if (t == 0) {
        // d_0 = 0 column: alpha * (last entry of q_1), folded with beta * (first
        // entry of q_2) when the right child is rectangular
        real_t z0 = alpha * (md.vals ? md.vl[1 - nd.buf][r0L + nl] : vrow(cvs[r0L + nl], r0L + nl));
        real_t cq = R(1), sq = R(0);
        if (sqre) {
            const real_t b0 = beta * (md.vals ? md.vf[1 - nd.buf][r0R + nr] : vrow(cvs[r0R + nr], r0R));
            real_t r;
            make_rot(z0, b0, cq, sq, r);
            z0 = r;
        }
        ds[0] = 0.0;
        zs[0] = z0;
        src[0] = 0;
        s_cq = cq; s_sq = sq;
    }
    // 8 eps ||M|| with ||M|| ~ max(|d|, |alpha|, |beta|); the floor (2^-400 in
    // FP64, 2^-60 in FP32) keeps an all-zero node well defined (tol^2 stays a
    // normal number)
    const real_t tol = R(8) * kEps * fmax(fmax(dmax, kTolFloor), fmax(fabs(alpha), fabs(beta)));

    // ---- deflation
    int a;
    const int ns = deflate_core(m, tol, ds, zs, src, nl, md.slist + r0, md.sidx + r0, md.role + r0,
                                md.rc + r0, md.rs + r0, wsum, &a);
    (void)ns;
    const int *role = md.role + r0;

    // ---- survivor numbering (M order = ascending), type groups, deflated slots
    // Warp w numbers the positions [wb, we), 32 consecutive ones at a time
    // (lane = position): the category counts of a chunk come from ballots,
    // a position's index from the population count of the lower lanes, so
    // that every load and store of a chunk is coalesced.  Categories: 0
    // survivor, 1..3 its type group (1: left only, 2: right only, 3: both),
    // 4 deflated against d_0, 5 other deflated.
    const int lane = t & 31, wid = t >> 5, nwarp = T >> 5;
    const int wseg = ((m + nwarp - 1) / nwarp + 31) & ~31;
    const int wb = min(m, wid * wseg), we = min(m, wb + wseg);
    const unsigned lt = (1u << lane) - 1u;       // lanes below this one
    auto category = [&](int p, int r, int &grp) {   // survivor: grp = type group (0 for p = 0)
        const int code = r & 15;
        grp = 0;
        if (code == ROLE_KEEP) {
            if (p > 0) { const int ty = (r >> 8) & 3; grp = (ty == 1) ? 1 : (ty == 2) ? 2 : 3; }
            return 0;
        }
        return (code == ROLE_ZERO) ? 4 : 5;
    };
    int cnt[6] = {0, 0, 0, 0, 0, 0};             // this warp's counts (lane 0 keeps them)
    for (int c0 = wb; c0 < we; c0 += 32 * kDeflBatch) {
        int rr[kDeflBatch];                      // the roles of kDeflBatch chunks, loaded together
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            rr[u] = (p < we) ? role[p] : 0;
        }
#pragma unroll
        for (int u = 0; u < kDeflBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            int grp = -1, cat = -1;
            if (p < we) cat = category(p, rr[u], grp);
            cnt[0] += __popc(__ballot_sync(0xffffffffu, cat == 0));
            cnt[1] += __popc(__ballot_sync(0xffffffffu, cat == 0 && grp == 1));
            cnt[2] += __popc(__ballot_sync(0xffffffffu, cat == 0 && grp == 3));
            cnt[3] += __popc(__ballot_sync(0xffffffffu, cat == 0 && grp == 2));
            cnt[4] += __popc(__ballot_sync(0xffffffffu, cat == 4));
            cnt[5] += __popc(__ballot_sync(0xffffffffu, cat == 5));
        }
    }
    // warp bases: exclusive scans over the warps (one value per warp, in lane 0)
    int N, n1, n2, n3, nz, no;
    int base[6];
    base[0] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[0] : 0, wsum, N), 0);
    base[1] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[1] : 0, wsum, n1), 0);
    base[2] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[2] : 0, wsum, n2), 0);
    base[3] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[3] : 0, wsum, n3), 0);
    base[4] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[4] : 0, wsum, nz), 0);
    base[5] = __shfl_sync(0xffffffffu, block_excl_scan(lane == 0 ? cnt[5] : 0, wsum, no), 0);
    const int P1 = (n1 + 7) & ~7;
    const int Ktot = P1 + 1 + n2 + n3;
    real_t *dM = md.dM + r0, *zM = md.zM + r0, *dval = md.dval + r0;
    int *kposM = md.kposM + r0, *invK = md.invK + nd.kbase, *dest = md.dest + r0, *dsrc = md.dsrc + r0;
    // slots of the node's columns (values-only nodes have none): a survivor's
    // new column goes to the slot of its source column (the d_0 column's to
    // the free coupling column of U and to q_1's slot in V), a deflated
    // column stays in its slot
    const bool slots = !md.vals;
    int *nus = slots ? md.us[nd.buf] + r0 : nullptr, *nvs = slots ? md.vs[nd.buf] + r0 : nullptr;
    auto slot_u = [&](int c) { return c == 0 ? r0 + nl : (c <= nl ? cus[r0L + c - 1] : cus[r0R + (c - nl - 1)]); };
    auto slot_v = [&](int c) { return c == 0 ? cvs[r0L + nl] : (c <= nl ? cvs[r0L + c - 1] : cvs[r0R + (c - nl - 1)]); };
    // batches of kNumBatch chunks (nothing read here is written in this
    // loop): the roles, values and sources of a batch are loaded together,
    // then the slots of its sources, before any of its stores
    auto ld_pos = [&](int q, int &rq, real_t &dq, real_t &zq, int &cq) {
        if (q < we) { rq = role[q]; dq = ds[q]; zq = zs[q]; cq = slots ? src[q] : 0; }
    };
    for (int c0 = wb; c0 < we; c0 += 32 * kNumBatch) {
        int rq[kNumBatch], cq[kNumBatch], suq[kNumBatch], svq[kNumBatch];
        real_t dq[kNumBatch], zq[kNumBatch];
#pragma unroll
        for (int u = 0; u < kNumBatch; ++u) {
            rq[u] = cq[u] = suq[u] = svq[u] = 0;
            dq[u] = zq[u] = R(0);
            ld_pos(c0 + 32 * u + lane, rq[u], dq[u], zq[u], cq[u]);
        }
        if (slots) {
#pragma unroll
            for (int u = 0; u < kNumBatch; ++u)
                if (c0 + 32 * u + lane < we) { suq[u] = slot_u(cq[u]); svq[u] = slot_v(cq[u]); }
        }
#pragma unroll
        for (int u = 0; u < kNumBatch; ++u) {
            const int p = c0 + 32 * u + lane;
            const bool in = p < we;
            const int rp = rq[u], su = suq[u], sv = svq[u];
            const real_t dp = dq[u], zp = zq[u];
            int grp = -1, cat = -1;
            real_t dsp = R(0), zsp = R(0);
            if (in) {
                cat = category(p, rp, grp);
                dsp = dp;
                zsp = zp;
            }
            const unsigned bk = __ballot_sync(0xffffffffu, cat == 0), b1 = __ballot_sync(0xffffffffu, cat == 0 && grp == 1),
                           b2 = __ballot_sync(0xffffffffu, cat == 0 && grp == 3),
                           b3 = __ballot_sync(0xffffffffu, cat == 0 && grp == 2),
                           bz = __ballot_sync(0xffffffffu, cat == 4), bo = __ballot_sync(0xffffffffu, cat == 5);
            if (in) {
                int col;                                     // node column of sorted position p
                if (cat == 0) {
                    const int ik = base[0] + __popc(bk & lt);
                    const int kp = (grp == 0) ? P1
                                 : (grp == 1) ? base[1] + __popc(b1 & lt)
                                 : (grp == 3) ? P1 + 1 + base[2] + __popc(b2 & lt)
                                              : P1 + 1 + n2 + base[3] + __popc(b3 & lt);
                    dM[ik] = dsp;
                    zM[ik] = zsp;
                    md.d32[r0 + ik] = (float)dsp;
                    md.z32[r0 + ik] = (float)zsp;
                    kposM[ik] = kp;
                    invK[kp] = ik;
                    dest[p] = kp;
                    col = ik;
                } else if (cat == 4) {
                    const int iz = base[4] + __popc(bz & lt);
                    dval[iz] = R(0);
                    dsrc[iz] = p;
                    dest[p] = -(1 + iz);
                    col = N + iz;
                } else {
                    const int slot = nz + base[5] + __popc(bo & lt);
                    dval[slot] = dsp;
                    dsrc[slot] = p;
                    dest[p] = -(1 + slot);
                    col = N + slot;
                }
                if (slots) {
                    nus[col] = su;
                    nvs[col] = sv;
                }
            }
            base[0] += __popc(bk); base[1] += __popc(b1); base[2] += __popc(b2);
            base[3] += __popc(b3); base[4] += __popc(bz); base[5] += __popc(bo);
        }
    }
    if (slots && sqre && t == 0) nvs[m] = cvs[r0R + nr];   // the new null vector takes q_2's slot
    for (int kp = n1 + t; kp < P1; kp += T) invK[kp] = -1;
    if (scans) {
        // moment scans of the survivors for the root start estimates: prefix
        // sums (inclusive) of z^2, z^2 d^2, z^2 d^4 and the same suffix sums;
        // thread t takes the survivors [ik0, ik0 + ck) (written by other threads)
        __syncthreads();
        const int kseg = (N + T - 1) / T;
        const int ik0 = min(N, t * kseg), ck = min(N, ik0 + kseg) - ik0;
        real_t a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int k = ik0; k < ik0 + ck; ++k) {
            const real_t z2 = zM[k] * zM[k], d2 = dM[k] * dM[k];
            a0 += z2; a1 += z2 * d2; a2 += z2 * d2 * d2;
        }
        real_t *pz = md.pz + r0;
        const long long sn = md.n;
        real_t c0 = block_excl_scan_d(a0, dsum, false), c1 = block_excl_scan_d(a1, dsum, false),
               c2 = block_excl_scan_d(a2, dsum, false);
        for (int k = ik0; k < ik0 + ck; ++k) {
            const real_t z2 = zM[k] * zM[k], d2 = dM[k] * dM[k];
            c0 += z2; c1 += z2 * d2; c2 += z2 * d2 * d2;
            pz[k] = c0; pz[sn + k] = c1; pz[2 * sn + k] = c2;
        }
        c0 = block_excl_scan_d(a0, dsum, true); c1 = block_excl_scan_d(a1, dsum, true);
        c2 = block_excl_scan_d(a2, dsum, true);
        for (int k = ik0 + ck - 1; k >= ik0; --k) {
            const real_t z2 = zM[k] * zM[k], d2 = dM[k] * dM[k];
            c0 += z2; c1 += z2 * d2; c2 += z2 * d2 * d2;
            pz[3 * sn + k] = c0; pz[4 * sn + k] = c1; pz[5 * sn + k] = c2;
        }
    }
    __syncthreads();
    // rho = sum of the survivors' z^2 (the secular solver's upper bound for
    // the last root and one of the MLP features)
    real_t zz = 0.0;
    for (int k = t; k < N; k += T) zz = fma(zM[k], zM[k], zz);
    zz = warp_sum(zz);
    if ((t & 31) == 0) dsum[t >> 5] = zz;
    __syncthreads();
    if (t == 0) {
        real_t rho = 0.0;
        for (int w = 0; w < (T >> 5); ++w) rho += dsum[w];
        NodeState s;
        s.N = N; s.n1 = n1; s.n2 = n2; s.n3 = n3; s.P1 = P1; s.Ktot = Ktot;
        s.ndef = m - N; s.nzero = nz; s.tol = tol; s.cq = s_cq; s.sq = s_sq; s.iters = 0; s.rho = rho;
        state[nd.id] = s;
        const long long wb = (long long)r0 * md.wstride;
        const int Ktop = P1 + 1 + n2, Kbot = Ktot - P1;
        GemmProb *pr = probs + 4 * (size_t)blockIdx.x;
        // U: top rows 0..nl (incl. the coupling row), bottom rows nl+1..m-1;
        // survivor i's column goes to the slot us[buf][r0 + i] (empty
        // products, M = N = 0, when the U side is not formed)
        const int *cu = md.us[nd.buf] + r0, *cv = md.vs[nd.buf] + r0;
        const int uN = md.want_u ? N : 0;
        pr[0] = GemmProb{md.Wt + wb, md.UM + wb, md.U + r0, m, Ktot, (int)ld, md.want_u ? nl + 1 : 0, uN, Ktop, cu};
        pr[1] = GemmProb{md.Wt + wb + (nl + 1) + (size_t)P1 * m, md.UM + wb + P1, md.U + r0 + nl + 1, m, Ktot,
                         (int)ld, md.want_u ? m - nl - 1 : 0, uN, Kbot, cu};
        // V: top rows 0..nl (left child's columns), bottom rows nl+1..mc-1
        pr[2] = GemmProb{md.Qt + wb, md.VM + wb, md.V + r0, mc, Ktot, (int)ld, nl + 1, N, Ktop, cv};
        pr[3] = GemmProb{md.Qt + wb + (nl + 1) + (size_t)P1 * mc, md.VM + wb + P1, md.V + r0 + nl + 1, mc, Ktot,
                         (int)ld, mc - nl - 1, N, Kbot, cv};
    }
}

// ------------------------------------------------------------------ gather
// Columns of the node before deflation: c = 0 is the d_0 column (U: the unit
// vector of the coupling row; V: cq q_1 + sq q_2), c = 1..nl the left
// child's columns, c > nl the right child's.  Child columns are read from
// their slots (rows outside a slot's range are zero).
struct ColSrc {
    const real_t *U, *V;
    long long ld;
    int r0, nl, nr, sqre, r0R;
    real_t cq, sq;
    const int *cus, *cvs;                    // children's slot maps
    const int *ulo, *uhi, *vlo, *vhi;
    __device__ int uslot(int c) const { return c <= nl ? cus[r0 + c - 1] : cus[r0R + (c - nl - 1)]; }
    __device__ int vslot(int c) const { return c <= nl ? cvs[r0 + c - 1] : cvs[r0R + (c - nl - 1)]; }
    __device__ real_t uat(int g, int r) const {     // node row r of U slot g
        const long long row = r0 + r;
        return (row >= ulo[g] && row < uhi[g]) ? U[(size_t)g * ld + row] : R(0);
    }
    __device__ real_t vat(int g, int r) const {
        const long long row = r0 + r;
        return (row >= vlo[g] && row < vhi[g]) ? V[(size_t)g * ld + row] : R(0);
    }
    __device__ real_t u(int c, int r) const {       // r in [0, m)
        if (c == 0) return (r == nl) ? R(1) : R(0);
        return uat(uslot(c), r);
    }
    __device__ int q1slot() const { return cvs[r0 + nl]; }
    __device__ int q2slot() const { return cvs[r0R + nr]; }
    __device__ real_t v(int c, int r) const {       // r in [0, m + sqre)
        if (c == 0) return cq * vat(q1slot(), r) + (sqre ? sq * vat(q2slot(), r) : R(0));
        return vat(vslot(c), r);
    }
};

// copy rows [0, n) of a slot column (data in rows [lo, hi), zero elsewhere)
// to dst, by nthr threads from tid: four loads in flight per thread before
// their stores (source and destination may not alias as far as the compiler
// knows, so it would not hoist them itself)
__device__ __forceinline__ void copy_slot(real_t *__restrict__ dst, const real_t *__restrict__ src, int n,
                                          long long lo, long long hi, int tid, int nthr) {
    for (int r = tid; r < n; r += 4 * nthr) {
        real_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = r + u * nthr;
            v[u] = (row < n && row >= lo && row < hi) ? src[row] : R(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = r + u * nthr;
            if (row < n) dst[row] = v[u];
        }
    }
}

// One column task per sorted position of every node: survivors are copied
// into the K-ordered W~ / Q~ (the products' operands); deflated columns stay
// in their slots, except the members of close-value chains and the columns
// deflated against d_0, which are rotated in place (the rotation of Sec.
// 4.2.1 acts on the node's whole row range, so their slots' ranges become
// the node's).  CPB = 1: a CTA per task, its threads over the rows (large
// nodes); CPB = 4: a warp per task, four per CTA (small nodes, where a CTA
// per column of a few dozen rows would be all launch and descriptor loads).
template <int CPB>
__global__ void __launch_bounds__(256) k_merge_gather(const NodeDesc *__restrict__ nodes,
                                                      const MatDesc *__restrict__ mats,
                                                      const NodeState *__restrict__ state, int mmax, int ntasks) {
    const int task = blockIdx.x * CPB + (CPB == 1 ? 0 : (int)(threadIdx.x >> 5));
    const int tid = (CPB == 1) ? (int)threadIdx.x : (int)(threadIdx.x & 31);
    const int nthr = (CPB == 1) ? (int)blockDim.x : 32;
    auto sync = [] { if (CPB == 1) __syncthreads(); else __syncwarp(); };
    if (task >= ntasks) return;                  // a whole warp (CPB = 4) or CTA (CPB = 1)
    const int node = task / mmax, p = task % mmax;
    const NodeDesc nd = nodes[node];
    if (p >= nd.m) return;
    const MatDesc &md = mats[nd.mat];
    const NodeState ns = state[nd.id];
    const int m = nd.m, nl = nd.nl, sqre = nd.sqre, mc = m + sqre, r0 = nd.r0;
    const int r = md.role[r0 + p], code = r & 15;
    const int *src = md.src + r0, *dest = md.dest + r0, *slist = md.slist + r0;
    const real_t *rc = md.rc + r0, *rs = md.rs + r0;
    const ColSrc cs{md.U, md.V, (long long)md.n, r0, nl, m - nl - 1, sqre, r0 + nl + 1, ns.cq, ns.sq,
                    md.us[1 - nd.buf], md.vs[1 - nd.buf], md.ulo, md.uhi, md.vlo, md.vhi};
    const long long wb = (long long)r0 * md.wstride, ld = md.n;
    real_t *W = md.Wt + wb, *Qm = md.Qt + wb;
    real_t *U = md.U + r0, *V = md.V + r0;           // row r0 of every slot

    const bool wu = md.want_u != 0;              // the U side is formed (W~)
    if (p == 0) {
        const int a = ns.nzero;
        // padding columns of the K order (between the top block and index 0)
        for (int kp = ns.n1; kp < ns.P1; ++kp) {
            if (wu)
                for (int row = tid; row < m; row += nthr) W[(size_t)kp * m + row] = R(0);
            for (int row = tid; row < mc; row += nthr) Qm[(size_t)kp * mc + row] = R(0);
        }
        // U: the d_0 column is the unit vector; columns deflated against d_0
        // keep their U columns (the rotation is one-sided)
        if (wu)
            for (int row = tid; row < m; row += nthr) W[(size_t)ns.P1 * m + row] = cs.u(0, row);
        // V: the d_0 column absorbs them one by one, in place
        const int g1 = cs.q1slot(), g2 = sqre ? cs.q2slot() : 0;
        for (int row = tid; row < mc; row += nthr) {
            const real_t q1 = cs.vat(g1, row), q2 = sqre ? cs.vat(g2, row) : R(0);
            real_t y = ns.cq * q1 + ns.sq * q2;
            for (int j = 1; j <= a; ++j) {
                const int q = slist[j];
                const int g = cs.vslot(src[q]);
                const real_t x = cs.vat(g, row), c = rc[q], s = rs[q];
                V[(size_t)g * ld + row] = -s * y + c * x;
                y = c * y + s * x;
            }
            Qm[(size_t)ns.P1 * mc + row] = y;
            // the new right null vector replaces q_2 in its slot
            if (sqre) V[(size_t)g2 * ld + row] = -ns.sq * q1 + ns.cq * q2;
        }
        sync();
        if (tid == 0) {
            for (int j = 1; j <= a; ++j) {
                const int g = cs.vslot(src[slist[j]]);
                md.vlo[g] = r0; md.vhi[g] = r0 + mc;
            }
            if (sqre) { md.vlo[g2] = r0; md.vhi[g2] = r0 + mc; }
        }
        return;
    }
    if (code == ROLE_ZERO) return;
    if ((r & FL_MEMBER) && !(r & FL_START)) return;   // handled by its chain's first member
    if (code == ROLE_CHAIN) {                          // chain start: walk to its end
        const int k0 = md.sidx[r0 + p];
        // every member but a surviving last one is rotated in its own slot
        for (int row = tid; row < (wu ? m : 0); row += nthr) {
            real_t y = cs.u(src[p], row);
            int prev = p;
            for (int k = k0 + 1; k < m; ++k) {
                const int q = slist[k];
                const real_t x = cs.u(src[q], row), c = rc[q], s = rs[q];
                U[(size_t)cs.uslot(src[prev]) * ld + row] = c * y - s * x;
                y = s * y + c * x;
                prev = q;
                if ((md.role[r0 + q] & 15) == ROLE_KEEP) break;
            }
            if (dest[prev] >= 0) W[(size_t)dest[prev] * m + row] = y;
            else U[(size_t)cs.uslot(src[prev]) * ld + row] = y;
        }
        for (int row = tid; row < mc; row += nthr) {
            real_t y = cs.v(src[p], row);
            int prev = p;
            for (int k = k0 + 1; k < m; ++k) {
                const int q = slist[k];
                const real_t x = cs.v(src[q], row), c = rc[q], s = rs[q];
                V[(size_t)cs.vslot(src[prev]) * ld + row] = c * y - s * x;
                y = s * y + c * x;
                prev = q;
                if ((md.role[r0 + q] & 15) == ROLE_KEEP) break;
            }
            if (dest[prev] >= 0) Qm[(size_t)dest[prev] * mc + row] = y;
            else V[(size_t)cs.vslot(src[prev]) * ld + row] = y;
        }
        sync();
        if (tid == 0) {
            int prev = p;
            for (int k = k0 + 1; k < m; ++k) {
                const int q = slist[k];
                if (wu) { md.ulo[cs.uslot(src[prev])] = r0; md.uhi[cs.uslot(src[prev])] = r0 + m; }
                md.vlo[cs.vslot(src[prev])] = r0; md.vhi[cs.vslot(src[prev])] = r0 + mc;
                prev = q;
                if ((md.role[r0 + q] & 15) == ROLE_KEEP) break;
            }
            if (dest[prev] < 0) {
                if (wu) { md.ulo[cs.uslot(src[prev])] = r0; md.uhi[cs.uslot(src[prev])] = r0 + m; }
                md.vlo[cs.vslot(src[prev])] = r0; md.vhi[cs.vslot(src[prev])] = r0 + mc;
            }
        }
        return;
    }
    // a deflated column keeps its slot; a survivor is copied into W~ / Q~
    if (dest[p] < 0) return;
    const int c = src[p], gv = cs.vslot(c);
    if (wu) {
        const int gu = cs.uslot(c);
        copy_slot(W + (size_t)dest[p] * m, md.U + (size_t)gu * ld + r0, m, md.ulo[gu] - r0, md.uhi[gu] - r0, tid,
                  nthr);
    }
    copy_slot(Qm + (size_t)dest[p] * mc, md.V + (size_t)gv * ld + r0, mc, md.vlo[gv] - r0, md.vhi[gv] - r0, tid,
              nthr);
}

// ------------------------------------------------------------------ gather (values only)
// The same deflation bookkeeping as k_merge_gather on just two rows of V:
// the node's first row (inside the left child's rows) and last row (inside
// the right child's rows).  One thread per sorted position; survivors go to
// the K-indexed FK / LK, deflated columns and the new null vector straight
// to the node's first/last-row arrays.
struct RowSrc {
    const real_t *VF, *VL;       // children's first / last rows (copy 1 - buf)
    int r0, r0R, nl, nr, sqre;
    real_t cq, sq;
    __device__ real_t f(int c) const {     // first row of pre-deflation column c
        if (c == 0) return cq * VF[r0 + nl];
        return (c <= nl) ? VF[r0 + c - 1] : R(0);
    }
    __device__ real_t l(int c) const {     // last row
        if (c == 0) return sqre ? sq * VL[r0R + nr] : R(0);
        return (c > nl) ? VL[r0R + (c - nl - 1)] : R(0);
    }
};

__global__ void __launch_bounds__(128) k_gather_rows(const NodeDesc *__restrict__ nodes,
                                                     const MatDesc *__restrict__ mats,
                                                     const NodeState *__restrict__ state, int mmax, int nnodes) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int node = (int)(idx / mmax), p = (int)(idx % mmax);
    if (node >= nnodes) return;
    const NodeDesc nd = nodes[node];
    if (p >= nd.m) return;
    const MatDesc &md = mats[nd.mat];
    const NodeState ns = state[nd.id];
    const int m = nd.m, nl = nd.nl, sqre = nd.sqre, r0 = nd.r0;
    const int r = md.role[r0 + p], code = r & 15;
    const int *src = md.src + r0, *dest = md.dest + r0, *slist = md.slist + r0;
    const real_t *rc = md.rc + r0, *rs = md.rs + r0;
    const RowSrc cs{md.vf[1 - nd.buf], md.vl[1 - nd.buf], r0, r0 + nl + 1, nl, m - nl - 1, sqre, ns.cq, ns.sq};
    real_t *FK = md.FK + nd.kbase, *LK = md.LK + nd.kbase;
    real_t *VF = md.vf[nd.buf] + r0, *VL = md.vl[nd.buf] + r0;
    auto put = [&](int dst, real_t fv, real_t lv) {
        if (dst >= 0) { FK[dst] = fv; LK[dst] = lv; }
        else { VF[ns.N + (-dst - 1)] = fv; VL[ns.N + (-dst - 1)] = lv; }
    };
    if (p == 0) {
        // the d_0 column absorbs the zero-deflated group by one-sided rotations
        real_t yf = cs.f(0), yl = cs.l(0);
        for (int j = 1; j <= ns.nzero; ++j) {
            const int q = slist[j];
            const real_t xf = cs.f(src[q]), xl = cs.l(src[q]), c = rc[q], s = rs[q];
            put(dest[q], -s * yf + c * xf, -s * yl + c * xl);
            yf = c * yf + s * xf;
            yl = c * yl + s * xl;
        }
        FK[ns.P1] = yf;
        LK[ns.P1] = yl;
        if (sqre) {   // the new right null vector: last column of the node
            VF[m] = -ns.sq * md.vf[1 - nd.buf][r0 + nl];
            VL[m] = ns.cq * md.vl[1 - nd.buf][r0 + nl + 1 + (m - nl - 1)];
        }
        return;
    }
    if (code == ROLE_ZERO) return;
    if ((r & FL_MEMBER) && !(r & FL_START)) return;   // handled by its chain's first member
    if (code == ROLE_CHAIN) {
        const int k0 = md.sidx[r0 + p];
        real_t yf = cs.f(src[p]), yl = cs.l(src[p]);
        int prev = p;
        for (int k = k0 + 1; k < m; ++k) {
            const int q = slist[k];
            const real_t xf = cs.f(src[q]), xl = cs.l(src[q]), c = rc[q], s = rs[q];
            put(dest[prev], c * yf - s * xf, c * yl - s * xl);
            yf = s * yf + c * xf;
            yl = s * yl + c * xl;
            prev = q;
            if ((md.role[r0 + q] & 15) == ROLE_KEEP) break;
        }
        put(dest[prev], yf, yl);
        return;
    }
    put(dest[p], cs.f(src[p]), cs.l(src[p]));
}

// ------------------------------------------------------------------ finish
// node values (roots, then deflated values) and their ascending order; the
// vectors are already in place (products and gather write the node block)
// grid (share of the node's positions, node): one CTA per node, or several
// for large merges (the entries are independent)
__global__ void __launch_bounds__(256) k_merge_finish(const NodeDesc *__restrict__ nodes,
                                                      const MatDesc *__restrict__ mats,
                                                      const NodeState *__restrict__ state) {
    const NodeDesc nd = nodes[blockIdx.y];
    const MatDesc &md = mats[nd.mat];
    const NodeState ns = state[nd.id];
    const int r0 = nd.r0, N = ns.N, ndef = ns.ndef;
    const real_t *om = md.omega + r0, *dv = md.dval + r0;
    const int T = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!md.vals) {
        // the products wrote the survivors' columns over the node's rows
        for (int i = t; i < N; i += T) {
            const int gu = md.us[nd.buf][r0 + i], gv = md.vs[nd.buf][r0 + i];
            md.ulo[gu] = r0; md.uhi[gu] = r0 + nd.m;
            md.vlo[gv] = r0; md.vhi[gv] = r0 + nd.m + nd.sqre;
        }
    }
    for (int i = t; i < N; i += T) md.D[r0 + i] = om[i];
    for (int s2 = t; s2 < ndef; s2 += T) md.D[r0 + N + s2] = dv[s2];
    // ascending order of roots (ascending) and deflated values (ascending),
    // roots first on ties: merge path, an equal share of positions per thread
    const int mt = N + ndef, S = (mt + T - 1) / T;
    const int k0 = min(mt, t * S), k1 = min(mt, k0 + S);
    if (k0 < k1) {
        int lo = max(0, k0 - ndef), hi = min(k0, N);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (om[mid] <= dv[k0 - mid - 1]) lo = mid + 1; else hi = mid;
        }
        int i = lo, j = k0 - lo;
        for (int k = k0; k < k1; ++k) {
            if (j >= ndef || (i < N && om[i] <= dv[j])) md.Q[r0 + k] = i++;
            else md.Q[r0 + k] = N + j++;
        }
    }
}

#ifndef BDC_FP32   // step entry point: FP64 only
__global__ void __launch_bounds__(PREP_THREADS) k_deflate_single(int m, const real_t *d, const real_t *z,
                                                                 real_t tol, int *keep, real_t *zout,
                                                                 real_t *dval, int *scratch_i,
                                                                 real_t *scratch_d) {
    __shared__ int wsum[PREP_THREADS / 32 + 1];
    real_t *zs = scratch_d, *rc = scratch_d + m, *rs = scratch_d + 2 * m;
    int *slist = scratch_i, *sidx = scratch_i + m, *role = scratch_i + 2 * m;
    for (int p = threadIdx.x; p < m; p += blockDim.x) zs[p] = z[p];
    __syncthreads();
    int a;
    deflate_core(m, tol, d, zs, nullptr, 0, slist, sidx, role, rc, rs, wsum, &a);
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int code = role[p] & 15;
        keep[p] = (code == ROLE_KEEP);
        zout[p] = (code == ROLE_KEEP) ? zs[p] : R(0);
        dval[p] = (code == ROLE_ZERO) ? R(0) : (code == ROLE_KEEP ? R(0) : d[p]);
    }
}

#endif

}  // namespace

cudaError_t launch_merge_prep(const NodeDesc *nodes, int nnodes, const MatDesc *mats, NodeState *state,
                              GemmProb *probs, int mmax, int scans, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    // large merges: the merged order and z over a grid first
    const int ordered = mmax >= ORDER_MIN ? 1 : 0;
    if (ordered) {
        const int chunks = (mmax + ORDER_THREADS * ORDER_SPAN - 1) / (ORDER_THREADS * ORDER_SPAN);
        for (int n0 = 0; n0 < nnodes; n0 += 65535) {     // grid y: at most 65535 nodes per launch
            const int nn = std::min(65535, nnodes - n0);
            k_merge_order<<<dim3((unsigned)chunks, (unsigned)nn), ORDER_THREADS, 0, st>>>(nodes + n0, mats);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    // a warp per 32 entries of the largest node, up to PREP_THREADS
    const int T = std::min(PREP_THREADS, std::max(32, (mmax + 1 + 31) / 32 * 32));
    k_merge_prep<<<nnodes, T, 0, st>>>(nodes, mats, state, probs, scans, ordered);
    return cudaGetLastError();
}

cudaError_t launch_merge_gather(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                                const NodeState *state, int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    const int ntasks = nnodes * mmax;
    if (mmax <= 256) {
        // a warp per column task, four per CTA
        k_merge_gather<4><<<(unsigned)(ntasks + 3) / 4, 128, 0, st>>>(nodes, mats, state, mmax, ntasks);
    } else {
        k_merge_gather<1><<<(unsigned)ntasks, 256, 0, st>>>(nodes, mats, state, mmax, ntasks);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                               const NodeState *state, int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    const long long t = (long long)nnodes * mmax;
    k_gather_rows<<<(unsigned)((t + 127) / 128), 128, 0, st>>>(nodes, mats, state, mmax, nnodes);
    return cudaGetLastError();
}

cudaError_t launch_merge_finish(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                                const NodeState *state, int mmax, cudaStream_t st) {
    if (nnodes <= 0) return cudaSuccess;
    const int T = std::min(256, std::max(32, (mmax + 31) / 32 * 32));
    const int chunks = std::max(1, mmax / (16 * 256));   // about 16 positions per thread for large merges
    for (int n0 = 0; n0 < nnodes; n0 += 65535) {         // grid y: at most 65535 nodes per launch
        const int nn = std::min(65535, nnodes - n0);
        k_merge_finish<<<dim3((unsigned)chunks, (unsigned)nn), T, 0, st>>>(nodes + n0, mats, state);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

#ifndef BDC_FP32
cudaError_t launch_deflate_single(int m, const real_t *d, const real_t *z, real_t tol, int *keep,
                                  real_t *zout, real_t *dval, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    void *si = nullptr, *sd = nullptr;
    cudaError_t e = cudaMallocAsync(&si, sizeof(int) * 3 * (size_t)m, st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&sd, sizeof(real_t) * 3 * (size_t)m, st);
    if (e != cudaSuccess) { cudaFreeAsync(si, st); return e; }
    k_deflate_single<<<1, PREP_THREADS, 0, st>>>(m, d, z, tol, keep, zout, dval, (int *)si, (real_t *)sd);
    e = cudaGetLastError();
    cudaFreeAsync(si, st);
    cudaFreeAsync(sd, st);
    return e;
}
#endif

}  // namespace BDC_NS

#ifndef BDC_FP32   // allocation-free step entry point: FP64 only
// ---------------------------------------------------------------------------
// Allocation-free deflation.
//
// bdc_deflate above obtains its scratch with cudaMallocAsync.  Some callers
// cannot allocate device memory at the moment they call: code that runs
// while another component owns the device allocator (a framework caching
// allocator, or an application that reserves all memory up front and treats
// any further allocation as a failure), and latency-critical loops that must
// not touch the driver's allocator at all.  For them bdc_deflate_noalloc does
// the same work with its scratch in a fixed array that lives in the module's
// global memory for as long as the library is loaded (on every device that
// loads it).  Only the problem size is limited: m <= BDC_DEFLATE_NOALLOC_MAX.
//
// The array is shared by every call: calls whose kernels overlap on the GPU
// (different streams without ordering) race on it and must be serialised by
// the caller.  Every scratch entry a call reads is written earlier by the
// same call, so nothing has to be cleared between calls.
// ---------------------------------------------------------------------------
namespace BDC_NS {
namespace {

constexpr int kNoAllocMax = BDC_DEFLATE_NOALLOC_MAX;
constexpr size_t kNoAllocDoubles = 3 * (size_t)kNoAllocMax;   // zs, rc, rs
constexpr size_t kNoAllocInts = 3 * (size_t)kNoAllocMax;      // slist, sidx, role
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocDoubles * sizeof(real_t) +
                                                                  kNoAllocInts * sizeof(int)];

// device address of g_noalloc_scratch, looked up once per device (the host
// symbol is only a stand-in and must never be passed to a kernel); kept for
// the life of the process, so it is stale after cudaDeviceReset on that
// device (documented as a limit of the entry point)
constexpr int kMaxDevices = 64;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

cudaError_t noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace BDC_NS


extern "C" int bdc_deflate_noalloc(int m, const double *d, const double *z, double tol, int *keep, double *zout,
                                   double *dval, bdc_stream_t stream) {
    using namespace bdc;
    if (m < 0 || m > kNoAllocMax) return -1;
    if (m > 0 && (!d || !z || !keep || !zout || !dval)) return -2;
    if (!(tol >= 0.0)) return -4;
    if (m == 0) return 0;
    void *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return BDC_ERR_CUDA;
    real_t *sd = (real_t *)base;
    int *si = (int *)((char *)base + kNoAllocDoubles * sizeof(real_t));
    k_deflate_single<<<1, PREP_THREADS, 0, (cudaStream_t)stream>>>(m, d, z, tol, keep, zout, dval, si, sd);
    return cudaGetLastError() == cudaSuccess ? 0 : BDC_ERR_CUDA;
}
#endif  // BDC_FP32
