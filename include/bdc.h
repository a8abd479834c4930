/*
 * bdc.h -- C ABI of the GB300 (sm_103a) bidiagonal divide-and-conquer SVD.
 *
 * Problem (Sec. 4.2.1, first display): for the n x n upper bidiagonal B with
 * diagonal d[0..n-1] and superdiagonal e[0..n-2] compute B = U S V^T with
 * S = diag(s_0 >= s_1 >= ... >= s_{n-1} >= 0) (the ordering of Sec. 1).
 * The method is Algorithm 2: recursive splitting (Sec. 4.2.1), leaf SVDs by
 * QR iteration, bottom-up merges made of deflation (Eq. M-condition and the
 * four N = 3 cases) and the secular solve / vector update (Eqs. M-svd-val,
 * bdc-zi, M-svd-vec, bdc-Mv2Bv-u-vt), then a final sort.  Every step runs on
 * the GPU; the host only plans launches.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major doubles.  U is n x n with leading dimension
 *     ldu >= max(1, n): column i is the left singular vector of s_i.  VT is
 *     n x n with leading dimension ldvt >= max(1, n): row i is the right
 *     singular vector of s_i.
 *   - Unless stated otherwise every pointer is a DEVICE pointer owned by the
 *     caller; inputs are read only.  The library keeps no pointer to caller
 *     data after a call returns; between calls it keeps only caches (launch
 *     descriptors, pinned staging blocks, a second stream per host thread).
 *   - Return codes: 0 success; -i when argument i (1-based) is illegal;
 *     +k (k > 0) when k leaf QR iterations or secular roots failed to
 *     converge (results are then not reliable); BDC_ERR_CUDA for a CUDA
 *     launch / allocation failure; BDC_ERR_TIMEOUT when a bounded device
 *     wait gave up; BDC_ERR_NONFINITE when d or e holds NaN or Inf (a code
 *     of its own, negative, so that it cannot be read as a count of
 *     non-converged problems); BDC_ERR_CHECK when checked mode found a
 *     violated invariant.
 *   - Streams: all work is ordered on `stream` (0 = legacy default); the
 *     solves with vectors also run part of each merge on a per-thread second
 *     stream forked from and joined back to `stream` by events (see
 *     bdc_svd_ex).
 */
#ifndef BDC_H
#define BDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *bdc_stream_t; /* same object as cudaStream_t */

#define BDC_ERR_CUDA      (-1000)
#define BDC_ERR_TIMEOUT   (-1001)
#define BDC_ERR_NONFINITE (-1002)
#define BDC_ERR_INTERNAL  (-1003)
#define BDC_ERR_CHECK     (-1004)

/* Precision of the merge products W~ U_M and Q~ V_M (Eq. bdc-Mv2Bv-u-vt).
 *   BDC_FP64          FP64 products.
 *   BDC_MIXED_BF16X3  FP64 operands split into two BF16 pieces, the three
 *                     leading products hi*hi + hi*lo + lo*hi on tcgen05
 *                     tensor cores with FP32 accumulation (about 1e-6
 *                     relative: reported, not accurate to FP64).
 *   BDC_MIXED_EXACT   error-free slicing: each operand row/column is scaled
 *                     by a power of two and cut into `slices` BF16 integer
 *                     slices; slice products are accumulated exactly (FP32
 *                     in TMEM over short K chunks, then 64-bit integers) so
 *                     the result matches FP64 to ~2^-(8*slices-1) relative.
 * Deflation, secular roots, z-tilde and vector formation are always FP64. */
typedef enum { BDC_FP64 = 0, BDC_MIXED_BF16X3 = 1, BDC_MIXED_EXACT = 2 } bdc_precision;

/* Starting point of each secular root (Eq. M-svd-val):
 *   BDC_SEED_PLAIN     interval-midpoint start;
 *   BDC_SEED_MLP       analytic estimate corrected by the small MLP in `mlp`
 *                      (FP32 weights, layout of bdc_mlp_param_count);
 *   BDC_SEED_ANALYTIC  the analytic estimate alone (no network).
 * The FP64 root finder always finishes every root to the same stopping
 * rule, so the start changes the iteration count, not the accuracy. */
typedef enum { BDC_SEED_PLAIN = 0, BDC_SEED_MLP = 1, BDC_SEED_ANALYTIC = 2 } bdc_seed;

typedef struct {
    int prec;          /* bdc_precision                                   */
    int seed;          /* bdc_seed                                        */
    int leaf;          /* leaf size L (4..64; 0 = default 8)              */
    int max_iter;      /* secular / QR iteration cap (0 = default 64)     */
    int slices;        /* BDC_MIXED_EXACT slice count 4..7 (0 = automatic: 7)    */
    int checked;       /* 1: checked mode: after every merge's deflation
                          and secular solve and after the final sort, device
                          kernels verify the invariants of the solve (counts
                          and K order of the survivors, strictly ascending
                          survivor values from d_0 = 0, non-zero z, the K
                          positions a permutation, slots inside [0, n),
                          each root on its interval's side of its origin,
                          finite z~, S finite, non-negative, descending) and
                          a violation sets the status to BDC_ERR_CHECK
                          instead of trapping (0 = off)                   */
    const float *mlp;  /* device pointer to MLP weights when seed = MLP    */
    int mixed_min;     /* split-BF16 products only for merges of order >= mixed_min,
                          FP64 products below (0 = automatic: 128)           */
    int fp32_start;    /* 1: each secular root first iterates in FP32 (the
                          pole sums on FP32 copies of d and z, the two
                          interval poles exact), then finishes in FP64 to the
                          same stopping rule (bdc_opts_default: 1)        */
    int vectors;       /* bdc_vectors: which singular vectors bdc_svd_ex
                          forms (0 = both)                                */
} bdc_opts;

/* Singular vectors formed by bdc_svd_ex (Sec. 4.2 with vectors for one
 * side only, the "next" partial-vector variants of the solve):
 *   BDC_VEC_BOTH  U and V^T;
 *   BDC_VEC_V     V^T only: the merges skip the U side (its gathers, vector
 *                 columns, products and output); U may be NULL and ldu is
 *                 not checked;
 *   BDC_VEC_U     U only: solved as BDC_VEC_V on J B^T J (J the reversal,
 *                 an upper bidiagonal with diagonal d reversed and
 *                 superdiagonal e reversed, whose right singular vectors are
 *                 J U), the final kernel writing them back in row-reversed
 *                 order; VT may be NULL and ldvt is not checked.
 * The singular values are those of B in every mode. */
typedef enum { BDC_VEC_BOTH = 0, BDC_VEC_V = 1, BDC_VEC_U = 2 } bdc_vectors;

/* Fill *o with the defaults (FP64, plain seed, leaf 8, automatic slices). */
void bdc_opts_default(bdc_opts *o);

/* SVD of the n x n upper bidiagonal (d, e), FP64 defaults, synchronous:
 * returns after the result and the status are known.  Allocates its
 * workspace with cudaMallocAsync on `stream` and frees it before returning.
 * n = 0 is a no-op; n = 1 gives s = |d0|, U = sign(d0), VT = 1.
 * d[n], e[n-1] (e may be NULL when n <= 1), U, S[n], VT: device pointers. */
int bdc_svd(int n, const double *d, const double *e, double *U, double *S, double *VT,
            int ldu, int ldvt, bdc_stream_t stream);

/* Singular values only (the paper's Sec. 4.2 solve without vectors): the
 * same tree, deflation and secular roots, but each node keeps only the first
 * and last rows of its right vectors (the rows the parent's z is formed
 * from, Sec. 4.2.1) instead of the U, V panels: no vector formation, no
 * merge products, O(n) memory.  S[n] descending (device).  The _ex form
 * takes a caller workspace (bdc_svd_values_workspace bytes) and a device
 * status word, like bdc_svd_ex; o->prec is ignored (no products), o->seed
 * and o->mlp select the root starts as in bdc_svd_ex.  bdc_svd_values uses
 * the defaults and is synchronous. */
size_t bdc_svd_values_workspace(int n, const bdc_opts *o);
int bdc_svd_values_ex(int n, const double *d, const double *e, double *S, const bdc_opts *o, void *work,
                      size_t lwork, int *d_info, bdc_stream_t stream);
int bdc_svd_values(int n, const double *d, const double *e, double *S, bdc_stream_t stream);

/* Workspace bytes needed by bdc_svd_ex for order n and options o. */
size_t bdc_svd_workspace(int n, const bdc_opts *o);

/* Asynchronous form: the caller passes `work` (device, lwork bytes,
 * 256-byte aligned, at least bdc_svd_workspace(n, o)) and `d_info` (device
 * int): the status code above is written to *d_info on the stream, so the
 * whole call can be captured in a CUDA graph.  The host return value only
 * reports argument errors and launch failures.
 * Streams: the solves with vectors (this call, bdc_svd, the batched forms
 * and plans) run part of each merge (the gather, the A-operand slicing, the
 * node finish) on a second stream that the library keeps per host thread
 * and device; it forks from `stream` by an event and joins back by an event
 * before the merge's products, so all of the call's work is ordered before
 * later work on `stream`, and a capture of the call records both streams
 * into the caller's graph.  Its handles live as long as the thread, like
 * the library's other caches (not valid after cudaDeviceReset). */
int bdc_svd_ex(int n, const double *d, const double *e, double *U, double *S, double *VT,
               int ldu, int ldvt, const bdc_opts *o, void *work, size_t lwork,
               int *d_info, bdc_stream_t stream);

/* Batched SVD of `batch` independent bidiagonals of uneven sizes h_n[b]
 * (HOST array, each 1..2048).  d[b], e[b], U[b], S[b], VT[b] are device
 * pointers held in HOST arrays; h_ldu/h_ldvt are host arrays.  All
 * matrices advance level by level in the same launches (one launch per
 * stage per level for the whole batch).  Status per matrix in d_info[batch]
 * (device).  Workspace from bdc_svd_batched_workspace. */
size_t bdc_svd_batched_workspace(int batch, const int *h_n, const bdc_opts *o);
int bdc_svd_batched(int batch, const int *h_n, const double *const *d, const double *const *e,
                    double *const *U, double *const *S, double *const *VT, const int *h_ldu,
                    const int *h_ldvt, const bdc_opts *o, void *work, size_t lwork,
                    int *d_info, bdc_stream_t stream);

/* ---------------- plans: a fixed batch as one CUDA graph -----------------
 * bdc_plan_create records the whole launch sequence of bdc_svd_batched for
 * fixed sizes, pointers and options into a CUDA graph (nothing runs at
 * creation); bdc_plan_launch replays it on `stream` with one graph launch:
 * every stage of every level of every matrix, no host work per call.
 * Arguments as for bdc_svd_batched (batch >= 1; a single matrix is a batch
 * of one); `work`, the matrices and d_info must stay valid while the plan
 * is used, and launches of one plan must not overlap on the GPU (they share
 * the workspace).  The descriptors are copied from host memory that the
 * plan owns, so the plan is independent of later calls.  Returns 0 or a
 * negative argument code / BDC_ERR_CUDA; *plan is NULL on failure. */
typedef struct bdc_plan_s *bdc_plan;
int bdc_plan_create(bdc_plan *plan, int batch, const int *h_n, const double *const *d, const double *const *e,
                    double *const *U, double *const *S, double *const *VT, const int *h_ldu, const int *h_ldvt,
                    const bdc_opts *o, void *work, size_t lwork, int *d_info);
int bdc_plan_launch(bdc_plan plan, bdc_stream_t stream);
void bdc_plan_destroy(bdc_plan plan);

/* ---------------- single precision (batches) ----------------------------
 * The same batched solve with FP32 data and FP32 arithmetic in every step
 * (leaves, deflation with tol = 8 eps_32 ||M||, secular roots, z~, vectors,
 * and the merge products on CUDA cores).  Arguments as for
 * bdc_svd_batched / bdc_plan_create with float data pointers; options must
 * keep prec = 0 and seed = BDC_SEED_PLAIN (the split-BF16 products and the
 * root starts are FP64-path features).  Plans from bdc_plan_create_f32 are
 * launched and destroyed with bdc_plan_launch / bdc_plan_destroy.
 * Accuracy: relative singular-value error, residual and orthogonality
 * about n * eps_32. */
size_t bdc_svd_batched_workspace_f32(int batch, const int *h_n, const bdc_opts *o);
int bdc_svd_batched_f32(int batch, const int *h_n, const float *const *d, const float *const *e, float *const *U,
                        float *const *S, float *const *VT, const int *h_ldu, const int *h_ldvt, const bdc_opts *o,
                        void *work, size_t lwork, int *d_info, bdc_stream_t stream);
int bdc_plan_create_f32(bdc_plan *plan, int batch, const int *h_n, const float *const *d, const float *const *e,
                        float *const *U, float *const *S, float *const *VT, const int *h_ldu, const int *h_ldvt,
                        const bdc_opts *o, void *work, size_t lwork, int *d_info);
/* bdc_autotune for the FP32 path (leaf size only). */
int bdc_autotune_f32(int batch, const int *h_n, bdc_opts *o, int reps, double *ms, bdc_stream_t stream);

/* Autotuner for batches: times candidate plans on synthetic bidiagonals of
 * the given orders (d, e ~ U(0.5, 1.5), counter-based generator) and writes
 * the fastest leaf size into o->leaf, and for split-BF16 products the
 * fastest o->mixed_min (the merge order from which products use them).
 * Other fields of *o are kept.  `reps` timed graph launches per candidate
 * (0 = 3).  Allocates and frees its own device memory on `stream` and
 * synchronises it.  Results are cached per (order histogram in powers of
 * two, precision, start rule): a repeated call returns the cached choice
 * without timing.  *ms (may be NULL) gets the best time per batch. */
int bdc_autotune(int batch, const int *h_n, bdc_opts *o, int reps, double *ms, bdc_stream_t stream);

/* ---------------- step entry points (one merge stage each) ----------------
 * They run a single stage of Sec. 4.2.1 on one problem so that each kernel
 * can be checked against the oracle element by element.  d is sorted
 * ascending with d[0] = 0 and distinct entries; z has no zero entry (the
 * state after deflation, Eq. M-condition). */

/* Roots of the secular equation f(w) = 1 + sum_j z_j^2 / (d_j^2 - w^2)
 * (Eq. M-svd-val), one warp per root.  Root i is returned as
 * omega[i] = d[org[i]] + tau[i], org[i] in {i, i+1} the nearer pole.
 * Status (non-converged count) is written to *d_info. */
int bdc_secular_solve(int N, const double *d, const double *z, int *org, double *tau,
                      double *omega, int max_iter, int *d_info, bdc_stream_t stream);

/* z-tilde of Eq. (bdc-zi) from the roots (org, tau); sign taken from z. */
int bdc_lowner_z(int N, const double *d, const double *z, const int *org, const double *tau,
                 double *zt, bdc_stream_t stream);

/* Normalised singular vectors of M~ (Eq. M-svd-vec): column i of UM (N x N,
 * ld ldum) is u_i and of VM (ld ldvm) is v_i. */
int bdc_m_vectors(int N, const double *d, const double *zt, const int *org, const double *tau,
                  double *UM, int ldum, double *VM, int ldvm, bdc_stream_t stream);

/* Deflation of Sec. 4.2.1 on sorted (d, z) with tolerance tol.  Outputs
 * (device): keep[m] (1 = survivor, 0 = deflated), zout[m] (z after the
 * rotations; 0 for deflated entries), dval[m] (value of a deflated entry,
 * unspecified for survivors). */
int bdc_deflate(int m, const double *d, const double *z, double tol, int *keep, double *zout,
                double *dval, bdc_stream_t stream);

/* Allocation-free form of bdc_deflate, for callers that must not allocate
 * device memory during the call (the device allocator is owned by another
 * component, or all memory is reserved up front).  The paper has no
 * counterpart of this entry point.  Same arguments and outputs as
 * bdc_deflate; the scratch is a fixed array in the library's device memory
 * (about 2.4 MB, held on every device that loads the library until exit),
 * so m is limited to BDC_DEFLATE_NOALLOC_MAX: a larger (or negative) m
 * returns -1 before any work is queued.  No cudaMalloc / cudaFree or other
 * allocating call is made.  The first call on a device looks the array's
 * device address up (cudaGetSymbolAddress) with that device current; make
 * that first call before capturing a stream.  The address is kept for the
 * life of the process: after cudaDeviceReset on a device (a new context and
 * a new copy of the array) this entry point must not be called again on that
 * device in the same process.  All calls share the array, so calls that can
 * run at the same time on the GPU race and must be ordered by the caller. */
#define BDC_DEFLATE_NOALLOC_MAX 65536
int bdc_deflate_noalloc(int m, const double *d, const double *z, double tol, int *keep, double *zout,
                        double *dval, bdc_stream_t stream);

/* Merge product C = A * B (M x N, inner K), column-major, with the chosen
 * precision (bdc_precision): FP64, or the split BF16 tcgen05 products.  A,
 * B, C device; `work` device scratch of bdc_gemm_workspace bytes. */
size_t bdc_gemm_workspace(int M, int N, int K, int prec, int slices);
int bdc_gemm(int M, int N, int K, const double *A, int lda, const double *B, int ldb, double *C,
             int ldc, int prec, int slices, void *work, size_t lwork, bdc_stream_t stream);

/* ---------------- MLP seeding of the secular roots ----------------------
 * The paper solves every root of the secular equation (Eq. M-svd-val) from
 * a fixed start; it has no learned component.  These entry points add one.
 * Root i (0 <= i < N-1) lies in (d_i, d_{i+1}); with D2 = d_{i+1}^2 - d_i^2
 * its position t = (w_i^2 - d_i^2) / D2 is held as the logit y =
 * ln(t / (1 - t)).  The start is yhat = y_q + g(f):
 *   y_q  an analytic estimate: the two interval poles exactly, the rest of
 *        the secular function frozen at the interval midpoint (the 8
 *        nearest other poles on each side summed exactly, the farther ones
 *        through the first two moments of their z^2 weights in d^2), which
 *        leaves a quadratic in t;
 *   g    a 2 x 64 tanh MLP (FP32) trained on the gap y - y_q of roots that
 *        FP64 runs produced.
 * The solver starts at yhat instead of the interval midpoint (one pole-sum
 * evaluation fewer, and a closer start), and polishes from the nearer pole
 * if yhat lands on the wrong half.  The last root always starts plainly.
 *
 * Features (FP32, each clamped to [-40, 40]), a = z_i^2/D2, b =
 * z_{i+1}^2/D2, gap_k = d_{k+1} - d_k, rho = sum z^2:
 *   f0 = ln a   f1 = ln b   f2 = ln(rho/D2)
 *   f3 = ln(gap_{i-1}/gap_i) (0 at i = 0)   f4 = ln(gap_{i+1}/gap_i) (0 at i = N-2)
 *   f5 = ln(z_{i-1}^2/D2) (-40 at i = 0)    f6 = ln(z_{i+2}^2/D2) (-40 at i = N-2)
 *   f7 = asinh(near-pole sum)   f8 = asinh(far-pole estimate)   f9 = y_q
 *   f10 = d_i/d_{i+1}
 * Parameters (FP32, bdc_mlp_param_count entries): [0,11) feature means,
 * [11,22) inverse standard deviations, W1 (64 x 11, row per hidden unit),
 * b1[64], W2 (64 x 64), b2[64], W3[64], b3;
 * g = W3.tanh(W2 tanh(W1 xn + b1) + b2) + b3, xn = (f - mean) * istd.
 * All pointers below are device pointers; calls are asynchronous on
 * `stream`; non-zero returns: negative = argument error, BDC_ERR_CUDA. */
/* Number of FP32 parameters (5015). */
int bdc_mlp_param_count(void);
/* Number of input features per root (11). */
int bdc_mlp_feature_count(void);

/* Features of roots 0..N-2 of one sorted secular problem (d[0] = 0 <
 * d[1] < ... , z non-zero) into feat[(N-1) x 11], row-major, and the
 * analytic estimates y_q into yq[N-1] (yq may be NULL). */
int bdc_mlp_features(int N, const double *d, const double *z, float *feat, double *yq, bdc_stream_t stream);

/* bdc_secular_solve with a start rule `seed` (bdc_seed; `mlp` is needed
 * for BDC_SEED_MLP only) and the iterations each root used in iters[N]
 * (NULL = not wanted; -1 = did not converge). */
int bdc_secular_solve_ex(int N, const double *d, const double *z, int seed, const float *mlp, int *org,
                         double *tau, double *omega, int *iters, int max_iter, int *d_info, bdc_stream_t stream);

/* bdc_svd_ex that also appends, for every secular root the merges solve
 * (except each merge's last root), its features to feat[cap x 11] and its
 * training target r = y - y_q (clamped to [-40, 40]) to targ[cap].
 * *d_count (device) is the running number of samples: the caller zeroes it
 * once, later calls append; slots at or past `cap` are counted but not
 * written.  The sample order is not deterministic (roots append in
 * completion order). */
int bdc_svd_harvest(int n, const double *d, const double *e, double *U, double *S, double *VT, int ldu, int ldvt,
                    const bdc_opts *o, void *work, size_t lwork, int *d_info, float *feat, float *targ, int cap,
                    int *d_count, bdc_stream_t stream);

/* Initialise params from `count` harvested feature rows: feature means and
 * inverse standard deviations (floor 1e-3 on the deviation), Glorot-uniform
 * hidden weights from a counter-based generator keyed by `seed`, zero
 * biases and a zero output layer (g = 0: the start is y_q until trained).
 * `targ` is not read and may be NULL. */
int bdc_mlp_init(float *params, const float *feat, const float *targ, int count, unsigned long long seed,
                 bdc_stream_t stream);

/* Gradient of loss = mean over samples of h(g - r), h the Huber function
 * with threshold `huber` (h(u) = u^2/2 for |u| <= huber, huber (|u| -
 * huber/2) beyond; huber <= 0: u^2/2 everywhere), with respect to params
 * into grad[param_count] (the normalisation entries are 0: not trained);
 * *loss (may be NULL) gets the loss.  `work` is device scratch of
 * bdc_mlp_grad_workspace(count) bytes.  For a given sample order the
 * result is deterministic. */
size_t bdc_mlp_grad_workspace(int count);
int bdc_mlp_grad(const float *params, const float *feat, const float *targ, int count, float huber, float *grad,
                 float *loss, void *work, size_t lwork, bdc_stream_t stream);

/* One Adam step (step >= 1 is the bias-correction count) on the trained
 * entries (from index 22) of params; m and v (param_count entries, zeroed
 * before step 1) are the moment estimates. */
int bdc_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, float beta1,
                 float beta2, float eps, bdc_stream_t stream);

/* g for `count` feature rows into out[count], with the same inference code
 * the root solver runs. */
int bdc_mlp_predict(const float *params, const float *feat, int count, float *out, bdc_stream_t stream);

/* Fit params (device, bdc_mlp_param_count floats) to `count` harvested
 * pairs: bdc_mlp_init(seed), then `steps` full-batch Adam steps (beta1 0.9,
 * beta2 0.999, eps 1e-8) on the Huber loss of bdc_mlp_grad, the learning
 * rate decaying linearly from lr (step 1) to lr / 10 (the last step).
 * losses (device, `steps` floats, may be NULL) gets the loss before each
 * step.  Allocates its scratch with cudaMallocAsync on `stream`;
 * asynchronous.  Returns -1 (params), -2 (count <= 0 or feat, targ NULL),
 * -5 (steps < 0), -6 (lr <= 0), -7 (huber NaN) or BDC_ERR_CUDA. */
int bdc_mlp_fit(float *params, const float *feat, const float *targ, int count, int steps, float lr, float huber,
                unsigned long long seed, float *losses, bdc_stream_t stream);

/* Harvest and training in one call (the learned start of the secular roots
 * is trained on roots that FP64 solves of this library produce):
 *   1. two n x n bidiagonals are generated on the device from a
 *      counter-based generator keyed by t->seed: uniform d, e ~ U(0.5, 1.5)
 *      and graded d_k = 10^(-8k/n) U(0.5, 1.5), e_k = d_k / 2;
 *   2. both are solved with FP64 products and plain starts (the other
 *      fields of *o, e.g. leaf and max_iter, apply; o may be NULL) while
 *      every merge root but each merge's last is harvested (bdc_svd_harvest,
 *      at most 2^21 samples);
 *   3. bdc_mlp_fit(t->steps, t->lr, t->huber, t->seed) on the samples.
 * params: device output (bdc_mlp_param_count floats); losses: device,
 * t->steps floats, may be NULL; *samples (host, may be NULL): samples
 * harvested; out_path (may be NULL): the parameters are also written there
 * as raw little-endian FP32.  t may be NULL (all defaults).  Synchronous:
 * allocates and frees its buffers (about 16 n^2 + 100 MB bytes plus the
 * workspace of one solve) on `stream` and returns when training is done.
 * Returns 0; -1 (options), -2 (training options), -3 (params NULL), -6
 * (out_path not writable); a positive count when a harvest solve did not
 * converge; BDC_ERR_INTERNAL when nothing was harvested; BDC_ERR_CUDA. */
typedef struct {
    int n;                   /* order of the harvest bidiagonals, 16..65536 (0 = 8192) */
    int steps;               /* Adam steps (0 = 1500) */
    float lr;                /* initial learning rate (0 = 3e-3) */
    float huber;             /* Huber threshold (0 = 0.25; < 0: squared loss) */
    unsigned long long seed; /* generator and initialisation seed */
} bdc_mlp_train_opts;
int bdc_mlp_train(const bdc_opts *o, const bdc_mlp_train_opts *t, float *params, float *losses, int *samples,
                  const char *out_path, bdc_stream_t stream);

/* ---------------- dense front and back end (Sec. 4.1, 4.3) ---------------
 * All matrices column-major FP64 device arrays owned by the caller; every
 * call is asynchronous on `stream` unless stated; workspaces are device
 * memory of the size the matching *_workspace function returns (any
 * alignment).  Reflectors use LAPACK's sign convention and storage: a
 * reflector I - tau y y^T maps x to beta e_1 with beta = -sign(x_1) ||x||,
 * y_1 = 1 implicit.  Panels are b = 32 columns (rows) wide.  The panel
 * kernels are cooperative launches whose grid barriers wait at most 2 s; a
 * wait that gives up makes the call report BDC_ERR_TIMEOUT in *d_info.
 * Returns: 0, -i for an illegal argument i, BDC_ERR_CUDA. */

/* Bidiagonalization A = Q1 B P1^T (Sec. 4.1, Algorithm 1), m >= n: per
 * panel the b column and row reflectors (H_i, G_i, Eq. gebrd-house) with the
 * vectors y_i, x_i of Eqs. (bidiag-y-k3, bidiag-x-k3), then the merged
 * rank-(2b) update A -= P Q^T of Eq. (bidiag-A-trail3) as one FP64
 * tensor-core product.  On exit d[n] / e[n-1] hold B's diagonal and
 * superdiagonal, A holds y_i below the diagonal of column i and u_i right of
 * the superdiagonal of row i (u_i[i+1] = 1 implicit), tauq[n], taup[n] the
 * scalars (taup[n-1] = 0).  *d_info (device): 0 or BDC_ERR_TIMEOUT. */
size_t bdc_gebrd_workspace(int m, int n);
int bdc_gebrd(int m, int n, double *A, int lda, double *d, double *e, double *tauq, double *taup, void *work,
              size_t lwork, int *d_info, bdc_stream_t stream);

/* Back-transformation with the reflectors of bdc_gebrd (Sec. 4.3, ormqr /
 * ormlq): vect = 0: C (m x cdim, ldc >= m) := Q1 C; vect = 1: C (cdim x n,
 * ldc >= cdim) := C P1^T.  Each block of b reflectors is applied in the
 * modified compact-WY form: T^{-1} = Y^T Y with diagonal 1/tau (Eqs. inv_t,
 * larft_update), Z = Y^T C, a triangular solve with T^{-1}, C -= Y W. */
size_t bdc_ormbr_workspace(int m, int n, int cdim);
int bdc_ormbr(int vect, int m, int n, const double *A, int lda, const double *tau, double *C, int ldc, int cdim,
              void *work, size_t lwork, bdc_stream_t stream);

/* QR factorization A = Q R (Sec. 4.3, geqrf): per panel a cooperative
 * column-reflector kernel, then the trailing columns updated by the panel's
 * block reflector in modified compact WY.  R in the upper triangle of A,
 * reflectors below, tau[min(m, n)]. */
size_t bdc_geqrf_workspace(int m, int n);
int bdc_geqrf(int m, int n, double *A, int lda, double *tau, void *work, size_t lwork, int *d_info,
              bdc_stream_t stream);

/* The first n columns of Q = H_1 ... H_n (Eq. orgqr-q) in place of the
 * reflectors bdc_geqrf left in A (m >= n); workspace of bdc_geqrf_workspace. */
int bdc_orgqr(int m, int n, double *A, int lda, const double *tau, void *work, size_t lwork, bdc_stream_t stream);

/* Dense SVD A = U diag(S) V^T, m >= n (Sec. 4): for m >= 1.6 n first A = Q R
 * (bdc_geqrf, bdc_orgqr) and the SVD of R with U = Q U_R; then bdc_gebrd,
 * the bidiagonal SVD bdc_svd_ex with options o (precision of the merge
 * products, root starts; o->vectors must be BDC_VEC_BOTH), and the
 * back-transformations U = Q1 U2, V^T = V2^T P1^T (bdc_ormbr).  A (m x n,
 * lda) is overwritten; S[n] descending; U m x n (ldu >= m); VT n x n (ldvt
 * >= n).  *d_info (device): the status of bdc_svd_ex, or BDC_ERR_TIMEOUT. */
size_t bdc_gesvd_workspace(int m, int n, const bdc_opts *o);
int bdc_gesvd(int m, int n, double *A, int lda, double *S, double *U, int ldu, double *VT, int ldvt,
              const bdc_opts *o, void *work, size_t lwork, int *d_info, bdc_stream_t stream);

/* ---------------- stage profiling (CUDA events, host side) ---------------
 * bdc_profile_begin(1) makes every later call record a CUDA event pair
 * around each stage's launches on the call's stream; bdc_profile_end() waits
 * for them and returns, per stage kind k (BDC_STAGE_*), the summed device
 * milliseconds in ms[k], the launch count in launches[k] and the summed
 * algorithmic work in work[k]:
 *   BDC_STAGE_GEMM     tensor flops 2 M N K of every merge product at its
 *                      deflated size, times the slice pairs of the split
 *                      BF16 paths (the products the tensor cores execute);
 *   every other stage  the bytes it must move through HBM (reads + writes)
 *                      at the deflated sizes: scale 32 n; leaf the leaves'
 *                      U, V blocks; prep 80 m per merge; gather the N
 *                      survivor columns of W~, Q~ written in full and their
 *                      child-block rows read (12 N (m + m + sqre)); secular
 *                      and Loewner 0 (d, z stay in cache); vectors 16 N Ktot
 *                      (U_M, V_M written); slice (8 + 2 S)(M K + K N) per
 *                      split product; finish 24 m; final 16 n^2 (U, V^T
 *                      written).
 * BDC_STAGE_SLICE and BDC_STAGE_LOWNER are split out of BDC_STAGE_GEMM and
 * BDC_STAGE_SECULAR (operand slicing of the split-BF16 products; the z~
 * products of Eq. bdc-zi).  Arrays have BDC_NSTAGES entries (any may be
 * NULL).  Not thread safe; not for graph capture. */
enum { BDC_STAGE_SCALE = 0, BDC_STAGE_LEAF, BDC_STAGE_PREP, BDC_STAGE_GATHER, BDC_STAGE_SECULAR,
       BDC_STAGE_VECTORS, BDC_STAGE_GEMM, BDC_STAGE_FINISH, BDC_STAGE_FINAL, BDC_STAGE_SLICE, BDC_STAGE_LOWNER,
       BDC_NSTAGES };
int bdc_profile_begin(int on);
int bdc_profile_end(double *ms, long long *launches, double *work);
/* After bdc_profile_end: secular roots solved and root-finder iterations
 * spent (summed over the recorded calls), *roots and *iters (host). */
int bdc_profile_secular(long long *roots, long long *iters);
/* After bdc_profile_end: FP64 operations (lane operations, an FMA counted
 * once) per stage kind, fp64[BDC_NSTAGES] (host), from the recorded calls'
 * deflated sizes, root-finder iterations and leaf rotation counts:
 *   secular  9 per pole term, N terms per pole-sum evaluation, 1 + iters
 *            evaluations per root (the FP32 pre-iterations not counted);
 *   Loewner  10 per factor, N - 1 factors per z~ entry;
 *   vectors  15 per entry of U_M, V_M (one quotient and the norms);
 *   leaf     17 per logged rotation (forming and applying it to d, e) and
 *            6 per rotation per row of U or V it is replayed on. */
int bdc_profile_fp64(double *fp64);
/* After bdc_profile_end: per merge height k < levels (0 = the merges right
 * above the leaves) of stage kind `stage`, the summed milliseconds ms[k]
 * and work[k]: FP64 operations for the secular, Loewner and vector stages,
 * executed tensor flops for the products (either array may be NULL). */
int bdc_profile_levels(int stage, int levels, double *ms, double *work);

/* Text of the last CUDA error the library saw on this thread ("" if none);
 * reading it clears it. */
const char *bdc_last_error_string(void);

/* Human-readable text for a status code (static string). */
const char *bdc_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* BDC_H */
