// Internal data layout and helpers of the GB300 bidiagonal divide-and-conquer.
//
// Layout in HBM (one "matrix" = one bidiagonal problem of order n):
//   U, V      n x n column-major (ld = n), one copy each.  A node of the split
//             tree covers rows r0..r0+m-1 (Sec. 4.2.1: B_1 is (k-1) x k, the
//             coupling row k, B_2 below).  Its columns are not stored in a
//             block of their own: node column c lives in the slot (global
//             column index) us[b][r0 + c] of U and vs[b][r0 + c] of V, b =
//             depth % 2 (the maps are double-buffered: a node writes its map
//             while its children's maps are read).  A slot holds data only
//             in rows [lo, hi) of the node that last wrote it (ulo/uhi,
//             vlo/vhi); every reader treats the other rows as zero.  A column
//             that a merge deflates keeps its slot untouched; survivors are
//             gathered into W~/Q~ and the merge products write the new
//             columns back into the survivors' slots, so deflated columns are
//             never copied.
//   D, Q      n entries: D[r0+j] = value of node column j, Q[r0+p] = local
//             column of the p-th smallest value (node-local ascending order).
//   merge scratch (indexed from r0 or from the node's kbase) and four big
//   per-level matrices W~, Q~ (gathered/rotated vectors) and U_M, V_M (the
//   vectors of M~), node block at r0 * wstride, wstride = n + 16.
//
// The data path is compiled twice from the same sources: in FP64 (namespace
// bdc, real_t = double) and, with -DBDC_FP32, in FP32 (namespace bdc32,
// real_t = float) for the single-precision batched entry points.  Literal
// constants in arithmetic on real_t are written R(...) so that the FP32
// build does no FP64 arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bdc.h"

// a captured plan (bdc_plan_create / bdc_plan_create_f32): its CUDA graph
// and the pinned host blocks the graph's descriptor copies read from
struct bdc_plan_s {
    std::vector<void *> pinned;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int batch = 0;
};

#ifdef BDC_FP32
#define BDC_NS bdc32
#else
#define BDC_NS bdc
#endif
#define R(x) (static_cast<real_t>(x))

namespace BDC_NS {

#ifdef BDC_FP32
typedef float real_t;
constexpr real_t kEps = 1.1920928955078125e-7f;  // 2^-23
constexpr real_t kTolFloor = 0x1p-60f;           // keeps tol^2 a normal number
#else
typedef double real_t;
constexpr real_t kEps = 2.220446049250313e-16;   // 2^-52
constexpr real_t kTolFloor = 0x1p-400;
#endif

struct MatDesc {
    int n;
    int ldu, ldvt;           // user output leading dimensions
    long long wstride;       // n + 16
    const real_t *d_in, *e_in;
    real_t *Uo, *So, *VTo;   // user outputs
    real_t *dsc, *esc;       // scaled copies (esc[n-1] = 0)
    real_t *scale;           // [1] scale factor applied to d, e
    real_t *U, *V;           // column slots (n x n each, ld = n)
    int *us[2], *vs[2];      // node column -> slot, copy = tree depth % 2 (n + 1 each)
    int *ulo, *uhi, *vlo, *vhi;   // per slot: rows holding data [lo, hi) (n + 1 each)
    real_t *D;               // node values
    int *Q;                  // node-local ascending order
    // merge scratch, per node from r0 (size n) unless noted
    real_t *ds, *zs;         // sorted d, z
    int *src;                // sorted position -> encoded source column
    real_t *rc, *rs;         // rotation linking a sorted position to its chain predecessor
    int *role;               // sorted position -> role (see bdc_merge.cu)
    real_t *dM, *zM, *zt, *tau, *omega;   // survivors in M order
    int *org, *kposM;        // root origin, K position of each survivor
    int *invK;               // from kbase: K position -> M index (-1 = padding)
    real_t *dval;            // deflated values, output order
    int *dsrc;               // deflated output slot -> sorted position
    int *dest;               // sorted position -> K position (>= 0) or -(1 + deflated slot)
    int *slist;              // survivors of the small-z test, sorted positions (from r0)
    int *sidx;               // sorted position -> index in slist (-1 = small z)
    real_t *Wt, *Qt, *UM, *VM;   // big per-level matrices (node base r0 * wstride)
    int *info;               // [1] status: >0 non-convergence count, <0 error code
    real_t *pz;              // per-merge z^2 moment scans [6][n]: prefix sums of z^2, z^2 d^2,
                             // z^2 d^4 (rows 0-2), suffix sums (rows 3-5); root start features
    real_t *ystart;          // per-root start fractions (seeded starts), indexed r0 + i
    real_t *yq;              // per-root analytic estimates (harvest)
    float *fs;               // per-root features [n][kMlpIn] (harvest)
    float *d32, *z32;        // FP32 copies of the survivors' d, z (M order, from r0)
    float *feat;             // optional MLP harvest: features [hcap][kMlpIn] (nullptr = off)
    float *targ;             // harvest targets [hcap]
    int *hcount;             // harvest counter (device)
    int hcap;                // harvest capacity
    // singular values only: no U, V panels; each node keeps the first and
    // last rows of its V (the rows z is formed from), copy = depth % 2
    int vals;                // 1 = singular values only
    int want_u;              // 0: no U side (right vectors only; every merge skips W~, U_M, the
                             // U products and the U output)
    int rev;                 // 1: the solve runs on J B^T J (d, e read reversed) and its right
                             // vectors are written, rows reversed, as U (left vectors only)
    real_t *vf[2], *vl[2];   // [n + 1], node column c at r0 + c
    real_t *FK, *LK;         // K-indexed (from kbase): first/last-row entries of the survivors' columns
};

struct NodeDesc {
    int mat;     // index into the MatDesc array
    int id;      // global node id (NodeState index)
    int r0;      // first row of the node block
    int m;       // rows
    int sqre;    // 1 if the node has m+1 columns
    int nl;      // rows of the left child (coupling row = r0 + nl)
    int kbase;   // base of K-indexed scratch (invK)
    int pad;     // largest order among the nodes of this node's height
    int buf;     // U/V copy this node writes (its depth % 2); children are in 1 - buf
    int pad2;
};

struct NodeState {
    int N;       // surviving (non-deflated) entries, including index 0
    int n1, n2, n3;   // survivors of type top-only / dense / bottom-only
    int P1;      // n1 rounded up to a multiple of 8 (K position of index 0)
    int Ktot;    // P1 + 1 + n2 + n3
    int ndef;    // m - N
    int nzero;   // deflated by rotation against d_0 = 0
    real_t tol;
    real_t cq, sq;   // rotation folding the two null-vector components (sqre)
    unsigned long long iters;   // secular iterations summed over the node's roots
    real_t rho;                 // sum of z^2 over the survivors (after deflation)
};

// one product C = A * B (column-major, real_t), used by the merge GEMMs;
// with cmap, column j of the result is stored at C + cmap[j] * ldc
// Phases of a split-BF16 product launch: MIXED_A uploads the product table
// and slices the A operands (they need only the gathered W~ / Q~ blocks, so
// this can run while the roots are found); MIXED_B slices the B operands
// (U_M, V_M) and runs the tensor-core products.  MIXED_A precedes MIXED_B
// in stream order.
enum { MIXED_A = 1, MIXED_B = 2, MIXED_ALL = 3 };

struct GemmProb {
    const real_t *A; const real_t *B; real_t *C;
    int lda, ldb, ldc;
    int M, N, K;
    const int *cmap;
};

__host__ __device__ __forceinline__ size_t gemm_col(const GemmProb &p, int j) {
    return (size_t)(p.cmap ? p.cmap[j] : j) * (size_t)p.ldc;
}

// role codes for sorted positions (merge)
enum : int {
    ROLE_NONE = 0,
    ROLE_KEEP = 1,        // survivor
    ROLE_DEFL = 2,        // deflated by small z
    ROLE_CHAIN = 3,       // deflated member of a close-value chain (not last)
    ROLE_ZERO = 4         // deflated by rotation against d_0 = 0
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ real_t warp_max(real_t v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_isum(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// |x| as an ordered integer: for non-negative values the bit patterns sort
// like the values, so magnitude comparisons need no floating-point
// instruction (GB300's FP64 unit takes 64 cycles per warp instruction)
#ifdef BDC_FP32
typedef int rbits_t;
__device__ __forceinline__ rbits_t abits(real_t x) { return __float_as_int(x) & 0x7fffffff; }
#else
typedef long long rbits_t;
__device__ __forceinline__ rbits_t abits(real_t x) { return __double_as_longlong(x) & 0x7fffffffffffffffll; }
#endif

// z / x for the pole sums and vector entries.  FP64: GB300 issues an FP64
// division as about eight FP64-pipe operations, while the hardware
// reciprocal estimate (PTX rcp.approx.ftz.f64, relative error below 2^-19.9
// measured over 2^-1000..2^1000) issues at about eight times the FMA rate.
// The estimate r = (1 + d)/x is corrected to third order with the geometric
// series 1/x = r / (1 - e) = r (1 + e + e^2 + ...), e = 1 - x r = -d:
// r (1 + e + e^2) = (1 + d^3)/x, |d^3| < 2^-59; then the product with z.
// Three FMAs and a product, within about an ulp of z / x.  Outside
// 2^-1000 <= |x| <= 2^1000 the plain quotient.
__device__ __forceinline__ real_t quot(real_t z, real_t x) {
#ifdef BDC_FP32
    return z / x;
#else
    const long long xb = __double_as_longlong(x) & 0x7fffffffffffffffll;
    if (xb < (23ll << 52) || xb > (2023ll << 52)) return z / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    r = fma(r, fma(e, e, e), r);
    return z * r;
#endif
}

// plane rotation with c f + s g = r, -s f + c g = 0.  When both |f| and |g|
// lie below kRotSmall (f and g may be subnormal: a quotient of two
// subnormals carries only their few significant bits, and c^2 + s^2 would
// miss 1 by far more than an ulp), c and s are formed from copies scaled up
// by the power of two kRotUp (exact) and r is scaled back.
#ifdef BDC_FP32
constexpr float kRotSmall = 0x1p-63f, kRotUp = 0x1p64f, kRotDown = 0x1p-64f;
#else
constexpr double kRotSmall = 0x1p-511, kRotUp = 0x1p600, kRotDown = 0x1p-600;
#endif
__device__ __forceinline__ void make_rot(real_t f, real_t g, real_t &c, real_t &s, real_t &r) {
    if (g == R(0)) { c = R(1); s = R(0); r = f; return; }
    if (f == R(0)) { c = R(0); s = R(1); r = g; return; }
    if (fabs(f) < kRotSmall && fabs(g) < kRotSmall) {
        const real_t fs = f * kRotUp, gs = g * kRotUp;
        const real_t h = hypot(fs, gs);
        c = fs / h; s = gs / h; r = h * kRotDown;
        return;
    }
    const real_t h = hypot(f, g);
    c = f / h; s = g / h; r = h;
}

__device__ __forceinline__ void set_error(int *info, int code) {
    atomicCAS(info, 0, code);
}

// ------------------------------------------------------ host-side launchers
// (each returns cudaGetLastError() of its launches)
cudaError_t launch_scale(const MatDesc *mats, int nmat, int nmax, cudaStream_t st);
// leaves: `log` = leaf_log_bytes(leafmax) per leaf (unused, may be null, when vals)
size_t leaf_log_bytes(int leafmax);
cudaError_t launch_leaves(const NodeDesc *leaves, int nleaves, const MatDesc *mats, int leafmax,
                          int max_sweeps, int vals, void *log, NodeState *state, cudaStream_t st);
cudaError_t launch_merge_prep(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                              NodeState *state, GemmProb *probs, int mmax, int scans, cudaStream_t st);
cudaError_t launch_merge_gather(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                                const NodeState *state, int mmax, cudaStream_t st);
cudaError_t launch_secular(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                           NodeState *state, int mmax, int max_iter, int seed_mode,
                           const float *mlp, int harvest, int fp32_start, cudaStream_t st);
cudaError_t launch_vectors(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                           const NodeState *state, int mmax, cudaStream_t st);
cudaError_t launch_gemm64(const GemmProb *probs, int nprobs, int mmax_rows, int nmax_cols,
                          cudaStream_t st);
// singular values only (first and last rows of V instead of the panels)
cudaError_t launch_gather_rows(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                               const NodeState *state, int mmax, cudaStream_t st);
cudaError_t launch_rows_update(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                               const NodeState *state, int mmax, cudaStream_t st);
cudaError_t launch_merge_finish(const NodeDesc *nodes, int nnodes, const MatDesc *mats,
                                const NodeState *state, int mmax, cudaStream_t st);
cudaError_t launch_final(const MatDesc *mats, int nmat, int nmax, cudaStream_t st);

// checked mode (bdc_check.cu): invariants after the deflation, after the
// secular solve (corrupt: the BDC_TEST_CORRUPT_ROOT test hook) and at the end
cudaError_t launch_check_prep(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                              cudaStream_t st);
cudaError_t launch_check_roots(const NodeDesc *nodes, int nnodes, const MatDesc *mats, const NodeState *state,
                               int mmax, bool corrupt, cudaStream_t st);
cudaError_t launch_check_final(const MatDesc *mats, int nmat, cudaStream_t st);

// standalone step kernels (step entry points)
cudaError_t launch_secular_single(int N, const double *d, const double *z, int *org, double *tau,
                                  double *omega, int max_iter, int *info, int seed_mode, const float *mlp,
                                  int *iters, cudaStream_t st);
// pinned host memory owned by the plan being captured, or by the graph of a
// caller's stream capture (nullptr when no capture is active on this thread;
// callers then use their own buffers)
void *plan_pinned_alloc(size_t bytes);

// Stage profiling (bdc_profile_begin / bdc_profile_end): while profiling is
// on, a StageScope records a CUDA event pair around the launches made in its
// lifetime and books them to stage kind `stage` (BDC_STAGE_*) with the
// given launch count and algorithmic work; a no-op otherwise.
struct StageScope {
    cudaStream_t st;
    int stage;
    long long launches;
    double work;
    cudaEvent_t a = nullptr, b = nullptr;
    StageScope(cudaStream_t s, int k, long long l, double w);
    ~StageScope();
};

// Test hooks of the bounded device waits (read from the environment at each
// launch; both off by default): BDC_TEST_WAIT_NS sets the wait limit of the
// tensor-core product kernels in nanoseconds (default 2 s), and
// BDC_TEST_STALL=1 makes CTA 0 of each product launch skip the load of its
// first stage, so the barrier of that stage is never signalled and the wait
// on it must give up, set the error word and unwind.
unsigned long long test_wait_ns();
int test_stall();
// BDC_TEST_CORRUPT_ROOT=1 (checked mode only): root 0 of the top merge is
// moved to the wrong side of its origin, which the root check must report
bool test_corrupt_root();

// MLP training (bdc_mlp.cu)
size_t mlp_grad_workspace(int count);
cudaError_t launch_mlp_init(float *P, const float *feat, int count, unsigned long long seed,
                            cudaStream_t st);
cudaError_t launch_mlp_grad(const float *P, const float *feat, const float *targ, int count, float huber,
                            float *grad, float *loss, float *work, cudaStream_t st);
cudaError_t launch_mlp_adam(float *P, const float *grad, float *m, float *v, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st);
cudaError_t launch_mlp_predict(const float *P, const float *feat, int count, float *out, cudaStream_t st);
int mlp_param_count();
int mlp_feature_count();
cudaError_t launch_mlp_features_single(int N, const double *d, const double *z, float *feat, double *yq,
                                       cudaStream_t st);
cudaError_t launch_lowner_single(int N, const double *d, const double *z, const int *org,
                                 const double *tau, double *zt, cudaStream_t st);
cudaError_t launch_mvectors_single(int N, const double *d, const double *zt, const int *org,
                                   const double *tau, double *UM, int ldum, double *VM, int ldvm,
                                   cudaStream_t st);
cudaError_t launch_deflate_single(int m, const double *d, const double *z, double tol, int *keep,
                                  double *zout, double *dval, cudaStream_t st);

}  // namespace BDC_NS
