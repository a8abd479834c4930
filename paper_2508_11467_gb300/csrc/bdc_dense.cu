// Dense front and back end of the SVD (FP64), all on the GPU:
//
//   Sec. 4.1, Algorithm 1  bidiagonalization A = Q1 B P1^T (m >= n) by blocks
//             of b columns and rows: one cooperative panel kernel (k_labrd)
//             forms the b column reflectors H_i, row reflectors G_i and the
//             vectors y_i, x_i of Eqs. (bidiag-y-k3) and (bidiag-x-k3), the
//             corrections of the not yet updated trailing matrix merged into
//             one pair of matrices P = [V X], Q = [Y U]; the trailing matrix
//             then takes the merged rank-(2b) update A -= P Q^T of Eq.
//             (bidiag-A-trail3) as ONE product.
//   Sec. 4.3  QR of a tall-and-skinny A (cooperative panel k_geqr2 plus a
//             block-reflector update of the trailing columns), the explicit Q
//             (Eq. orgqr-q), and the back-transformations U = Q1 U2 and
//             V^T = V2^T P1^T.  Every block reflector I - Y T Y^T is applied
//             in the modified compact-WY form of Eqs. (inv_t, larft_update):
//             T^{-1} = Y^T Y (one product) with the diagonal 1 / tau, then
//             Z = Y^T C (product), W = T Z by a triangular solve with T^{-1},
//             C -= Y W (product): products and a small triangular solve only.
//
// The products are FP64 on the tensor cores (mma.sync.m8n8k4.f64, k_dgemm):
// C = alpha op(A) op(B) + beta C with either operand transposed.  The panel
// kernels run as cooperative launches (all CTAs resident) and separate their
// phases with a grid barrier whose wait is bounded (2 s of %globaltimer): a
// barrier that gives up sets an error word, every CTA leaves at its next
// barrier, and the entry point reports BDC_ERR_TIMEOUT.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "bdc_internal.cuh"

namespace bdc {

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ GEMM
struct DGemm {
    const double *A, *B;
    double *C;
    int lda, ldb, ldc, M, N, K;
    int ta, tb;            // op(A) = A^T, op(B) = B^T
    double alpha, beta;    // beta = 0: C is not read
    int kchunk;            // split K: CTA row blockIdx.y multiplies K range [y kchunk, (y+1) kchunk)
    double *part;          // split K: partial products part[y][M x N] (then alpha, beta unused)
};

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// 64 x 64 CTA tile, four warps of 32 x 32 (4 x 4 fragments 8 x 8), K step 16,
// operands staged k-major in padded shared tiles, next step prefetched
constexpr int DBM = 64, DBN = 64, DBK = 16, DSA = DBM + 8, DSB = DBK + 4;
__global__ void __launch_bounds__(128) k_dgemm(DGemm g) {
    __shared__ double As[DBK * DSA];   // As[k][m]
    __shared__ double Bs[DBN * DSB];   // Bs[n][k]
    const int tilesN = (g.N + DBN - 1) / DBN;
    const int m0 = (blockIdx.x / tilesN) * DBM, n0 = (blockIdx.x % tilesN) * DBN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gr = lane >> 2, tg = lane & 3;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    constexpr int L = DBM * DBK / 128;   // 8 elements per thread per operand
    double ra[L], rb[L];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < L; ++r) {
            const int idx = tid + r * 128;
            int am, ak;
            if (!g.ta) { am = idx % DBM; ak = idx / DBM; } else { ak = idx % DBK; am = idx / DBK; }
            const int gm = m0 + am, gk = k0 + ak;
            ra[r] = (gm < g.M && gk < g.K) ? (g.ta ? g.A[(size_t)gm * g.lda + gk] : g.A[(size_t)gk * g.lda + gm])
                                           : 0.0;
            int bk, bn;
            if (!g.tb) { bk = idx % DBK; bn = idx / DBK; } else { bn = idx % DBN; bk = idx / DBN; }
            const int gn = n0 + bn, gk2 = k0 + bk;
            rb[r] = (gn < g.N && gk2 < g.K) ? (g.tb ? g.B[(size_t)gk2 * g.ldb + gn] : g.B[(size_t)gn * g.ldb + gk2])
                                            : 0.0;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int r = 0; r < L; ++r) {
            const int idx = tid + r * 128;
            int am, ak, bk, bn;
            if (!g.ta) { am = idx % DBM; ak = idx / DBM; } else { ak = idx % DBK; am = idx / DBK; }
            if (!g.tb) { bk = idx % DBK; bn = idx / DBK; } else { bn = idx % DBN; bk = idx / DBN; }
            As[ak * DSA + am] = ra[r];
            Bs[bn * DSB + bk] = rb[r];
        }
    };
    // K range of this CTA (all of K unless split)
    const int kb = g.part ? (int)blockIdx.y * g.kchunk : 0;
    const int ke = g.part ? min(g.K, kb + g.kchunk) : g.K;
    // operand loads are bounded by the K range end
    const int Kfull = g.K;
    g.K = ke;
    load(kb);
    for (int k0 = kb; k0 < ke; k0 += DBK) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + DBK < ke) load(k0 + DBK);
#pragma unroll
        for (int kk = 0; kk < DBK; kk += 4) {
            if (k0 + kk >= ke) break;
            double af[4], bf[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) af[i] = As[(kk + tg) * DSA + wm + i * 8 + gr];
#pragma unroll
            for (int j = 0; j < 4; ++j) bf[j] = Bs[(wn + j * 8 + gr) * DSB + kk + tg];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (m0 + wm + i * 8 < g.M && n0 + wn + j * 8 < g.N) dmma(acc[i][j], af[i], bf[j]);
        }
    }
    (void)Kfull;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + wm + i * 8 + gr;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gn = n0 + wn + j * 8 + 2 * tg + h;
                if (gn >= g.N) continue;
                if (g.part) {
                    g.part[((size_t)blockIdx.y * g.N + gn) * g.M + gm] = acc[i][j][h];
                    continue;
                }
                double *c = g.C + (size_t)gn * g.ldc + gm;
                const double v = g.alpha * acc[i][j][h];
                *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
            }
        }
    }
}

// C = beta C + alpha sum_y part[y] (the split-K partial products, summed in
// a fixed order)
__global__ void k_dgemm_reduce(const double *__restrict__ part, int splits, int M, int N, double alpha, double beta,
                               double *C, int ldc) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)M * N) return;
    const int n = (int)(k / M), m = (int)(k % M);
    double s = 0.0;
    for (int y = 0; y < splits; ++y) s += part[(size_t)y * M * N + k];
    double *c = C + (size_t)n * ldc + m;
    *c = (beta == 0.0) ? alpha * s : fma(beta, *c, alpha * s);
}

// scratch for split-K partial products (set per call sequence by the driver)
thread_local double *g_split_buf = nullptr;
thread_local size_t g_split_cap = 0;   // doubles

int sm_count_dense() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

// C = alpha op(A) op(B) + beta C.  Products with few output tiles and a long
// K (the Y^T C and C Y of the block reflectors: 32 x n outputs, K = the
// panel's rows) split K over several CTAs into partial products, summed in a
// fixed order by k_dgemm_reduce, so that the whole GPU works on them
cudaError_t dgemm(int ta, int tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                  int ldb, double beta, double *C, int ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const long long tiles = (long long)((M + DBM - 1) / DBM) * ((N + DBN - 1) / DBN);
    if (tiles > 0x7fffffffll) return cudaErrorInvalidValue;
    DGemm g{A, B, C, lda, ldb, ldc, M, N, std::max(K, 0), ta, tb, alpha, beta, 0, nullptr};
    int splits = 1;
    const int sms = sm_count_dense();
    if (K >= 128 && tiles < 2 * sms && g_split_buf) {
        splits = (int)std::min<long long>((2 * sms + tiles - 1) / tiles, K / 64);
        splits = std::min(splits, 64);
        while (splits > 1 && (size_t)splits * M * N > g_split_cap) --splits;
    }
    if (splits > 1) {
        g.kchunk = ((K + splits - 1) / splits + DBK - 1) / DBK * DBK;
        splits = (K + g.kchunk - 1) / g.kchunk;
        g.part = g_split_buf;
        k_dgemm<<<dim3((unsigned)tiles, (unsigned)splits), 128, 0, st>>>(g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const long long cnt = (long long)M * N;
        k_dgemm_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(g_split_buf, splits, M, N, alpha, beta, C, ldc);
        return cudaGetLastError();
    }
    k_dgemm<<<(unsigned)tiles, 128, 0, st>>>(g);
    return cudaGetLastError();
}

// ------------------------------------------------------------ grid barrier
struct GridBar {
    unsigned count, gen;
    int err;
    int pad;
};
constexpr unsigned long long kBarNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// all CTAs of a cooperative launch; false (and the error word set) when the
// wait gave up or another CTA gave up before
__device__ bool grid_sync(GridBar *gb) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile GridBar *v = gb;
        int ok = v->err == 0;
        if (ok) {
            const unsigned g0 = v->gen;
            __threadfence();
            const unsigned arrived = atomicAdd(&gb->count, 1u);
            if (arrived == gridDim.x - 1) {
                gb->count = 0;
                __threadfence();
                atomicAdd(&gb->gen, 1u);
            } else {
                const unsigned long long t0 = gtime();
                while (v->gen == g0) {
                    if (v->err) { ok = 0; break; }
                    if (gtime() - t0 > kBarNs) {
                        atomicExch(&gb->err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// block sum of a double over blockDim.x threads (result in every thread)
__device__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;
}

// sum over the grid's CTAs of part[k * stride] (k < count), by the whole
// block: strided loads, four in flight per thread, then a block reduction
__device__ double grid_partials(const double *part, int count, int stride, double *sh) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const int T = blockDim.x;
    int k = threadIdx.x;
    for (; k + 3 * T < count; k += 4 * T) {
        s0 += part[(size_t)k * stride];
        s1 += part[(size_t)(k + T) * stride];
        s2 += part[(size_t)(k + 2 * T) * stride];
        s3 += part[(size_t)(k + 3 * T) * stride];
    }
    for (; k < count; k += T) s0 += part[(size_t)k * stride];
    return block_sum((s0 + s1) + (s2 + s3), sh);
}

// dot product of x[r] y[r] over r = r0 + lane, r0 + lane + 32, ... < r1 by
// sum over j < cnt of a[j sa] b[j sb] + c[j sa] d[j sb] (the panel's
// earlier columns, cnt < b): two independent FMA chains and the loads of
// eight j in flight, instead of one dependent chain waiting on each j's loads
__device__ __forceinline__ double dot2(const double *__restrict__ a, const double *__restrict__ b,
                                       const double *__restrict__ c, const double *__restrict__ d, long long sa,
                                       long long sb, int cnt) {
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
#pragma unroll 4
    for (; j + 1 < cnt; j += 2) {
        s0 = fma(a[j * sa], b[j * sb], s0);
        s1 = fma(a[(j + 1) * sa], b[(j + 1) * sb], s1);
        s0 = fma(c[j * sa], d[j * sb], s0);
        s1 = fma(c[(j + 1) * sa], d[(j + 1) * sb], s1);
    }
    if (j < cnt) {
        s0 = fma(a[j * sa], b[j * sb], s0);
        s0 = fma(c[j * sa], d[j * sb], s0);
    }
    return s0 + s1;
}

// one warp (result in every lane): four independent accumulators so that
// four pairs of loads are in flight per lane
__device__ __forceinline__ double warp_dot(const double *__restrict__ x, const double *__restrict__ y, int r0,
                                           int r1) {
    const int lane = threadIdx.x & 31;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int r = r0 + lane;
    for (; r + 96 < r1; r += 128) {
        s0 = fma(x[r], y[r], s0);
        s1 = fma(x[r + 32], y[r + 32], s1);
        s2 = fma(x[r + 64], y[r + 64], s2);
        s3 = fma(x[r + 96], y[r + 96], s3);
    }
    for (; r < r1; r += 32) s0 = fma(x[r], y[r], s0);
    double s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Householder reflector from alpha and ||x_2..||^2 = sig2 (LAPACK's sign
// convention, Sec. 4.1's first display): beta = -sign(alpha) ||x||, tau =
// (beta - alpha) / beta, the vector's tail scaled by 1 / (alpha - beta);
// sig2 = 0 gives tau = 0 (H = I).  Returns the tail scale.
__device__ __forceinline__ double reflector(double alpha, double sig2, double &tau, double &beta) {
    if (sig2 == 0.0) {
        tau = 0.0;
        beta = alpha;
        return 0.0;
    }
    const double nrm = sqrt(fma(alpha, alpha, sig2));
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    return 1.0 / (alpha - beta);
}

// -------------------------------------------------------- gebrd panel
// Panel of Algorithm 1 (labrd) on the local m x n trailing matrix A (ld lda):
// nb column and row reflectors.  Workspace (all column-major):
//   PW  m x 2b: [V | X], QW  n x 2b: [Y | U] (explicit, zero outside their
//   supports), yraw[n], tv[4b] (the small products of Eqs. bidiag-y-k3 /
//   x-k3), xpart[chunks][m] (column-chunk partial sums of A u), part[grid][2]
//   (partial sums of squares).
struct LabrdArgs {
    double *A;
    int lda, m, n, nb, b;
    double *d, *e, *tauq, *taup;   // offset to the panel's first index
    double *PW, *QW, *yraw, *tv, *xpart, *part;
    int chunks, chunkw;            // column chunks of the row-wise product A u
    GridBar *bar;
};

__global__ void __launch_bounds__(256) k_labrd(LabrdArgs a) {
    __shared__ double sh[32];
    const int T = blockDim.x, G = gridDim.x;
    const int gtid = blockIdx.x * T + threadIdx.x, gthreads = G * T;
    const int lane = threadIdx.x & 31;
    const int gwarp = gtid >> 5, gwarps = gthreads >> 5;
    const int m = a.m, n = a.n, b = a.b;
    double *A = a.A;
    const long long lda = a.lda;
    double *V = a.PW, *X = a.PW + (size_t)b * m, *Y = a.QW, *U = a.QW + (size_t)b * n;
    double *t1 = a.tv, *t2 = a.tv + b, *t3 = a.tv + 2 * b, *t4 = a.tv + 3 * b;

    // zero the workspace matrices (supports are filled step by step)
    for (size_t k = gtid; k < (size_t)2 * b * m; k += gthreads) a.PW[k] = 0.0;
    for (size_t k = gtid; k < (size_t)2 * b * n; k += gthreads) a.QW[k] = 0.0;
    if (!grid_sync(a.bar)) return;

    for (int i = 0; i < a.nb; ++i) {
        // (a) column i of the panel, rows i..m-1: A - V Y^T - X U^T (Eq. bidiag-y-k2 form)
        double ss = 0.0;
        for (int r = i + gtid; r < m; r += gthreads) {
            double v = A[(size_t)i * lda + r];
            v -= dot2(V + r, Y + i, X + r, U + i, m, n, i);
            A[(size_t)i * lda + r] = v;
            if (r > i) ss = fma(v, v, ss);
        }
        ss = block_sum(ss, sh);
        if (threadIdx.x == 0) a.part[2 * blockIdx.x] = ss;
        if (!grid_sync(a.bar)) return;
        // (b) the column reflector H_i (every CTA forms the same scalars)
        double sig2 = grid_partials(a.part, G, 2, sh);
        const double alpha = A[(size_t)i * lda + i];
        double tau, beta;
        const double sc = reflector(alpha, sig2, tau, beta);
        for (int r = i + 1 + gtid; r < m; r += gthreads) {
            const double v = A[(size_t)i * lda + r] * sc;
            A[(size_t)i * lda + r] = v;
            V[(size_t)i * m + r] = v;
        }
        if (gtid == 0) {
            V[(size_t)i * m + i] = 1.0;
            a.d[i] = beta;
            a.tauq[i] = tau;
        }
        if (!grid_sync(a.bar)) return;
        if (gtid == 0) A[(size_t)i * lda + i] = beta;   // v_i[i] = 1 is implicit from here on
        // (c) yraw = A^T v over the trailing columns, t1 = V^T v, t2 = X^T v
        // (Eq. bidiag-y-k3); one warp per dot product, rows i..m-1
        const int ncol = n - i - 1;
        for (int w = gwarp; w < ncol + 2 * i; w += gwarps) {
            const double *col;
            if (w < ncol) col = A + (size_t)(i + 1 + w) * lda;
            else if (w < ncol + i) col = V + (size_t)(w - ncol) * m;
            else col = X + (size_t)(w - ncol - i) * m;
            const double s = warp_dot(col, V + (size_t)i * m, i, m);
            if (lane == 0) {
                if (w < ncol) a.yraw[i + 1 + w] = s;
                else if (w < ncol + i) t1[w - ncol] = s;
                else t2[w - ncol - i] = s;
            }
        }
        if (!grid_sync(a.bar)) return;
        if (ncol == 0) continue;   // the last column of the matrix: no row reflector
        // (d) y_i = tau (yraw - Y t1 - U t2), then row i, columns i+1..n-1:
        // A - V Y^T - X U^T with the new v_i, y_i (Eq. bidiag-x-k3 form)
        ss = 0.0;
        for (int c = i + 1 + gtid; c < n; c += gthreads) {
            double y = a.yraw[c];
            y -= dot2(Y + c, t1, U + c, t2, n, 1, i);
            y *= tau;
            Y[(size_t)i * n + c] = y;
            double v = A[(size_t)c * lda + i] - y;   // V[i][i] = 1
            v -= dot2(Y + c, V + i, U + c, X + i, n, m, i);
            A[(size_t)c * lda + i] = v;
            if (c > i + 1) ss = fma(v, v, ss);
        }
        ss = block_sum(ss, sh);
        if (threadIdx.x == 0) a.part[2 * blockIdx.x + 1] = ss;
        if (!grid_sync(a.bar)) return;
        // (e) the row reflector G_i
        sig2 = grid_partials(a.part + 1, G, 2, sh);
        const double alr = A[(size_t)(i + 1) * lda + i];
        double pi, betr;
        const double scr = reflector(alr, sig2, pi, betr);
        for (int c = i + 2 + gtid; c < n; c += gthreads) {
            const double u = A[(size_t)c * lda + i] * scr;
            A[(size_t)c * lda + i] = u;
            U[(size_t)i * n + c] = u;
        }
        if (gtid == 0) {
            U[(size_t)i * n + i + 1] = 1.0;
            a.e[i] = betr;
            a.taup[i] = pi;
        }
        if (!grid_sync(a.bar)) return;
        if (gtid == 0) A[(size_t)(i + 1) * lda + i] = betr;
        // (f) xpart = A u by column chunks (rows i+1..m-1), t3 = Y^T u, t4 = U^T u
        const int rows = m - i - 1;
        const long long items = (long long)a.chunks * rows;
        for (long long t = gtid; t < items; t += gthreads) {
            const int ch = (int)(t / rows), r = i + 1 + (int)(t % rows);
            const int c0 = i + 1 + ch * a.chunkw, c1 = min(n, c0 + a.chunkw);
            const double *ui = U + (size_t)i * n;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int c = c0;
            for (; c + 3 < c1; c += 4) {
                s0 = fma(A[(size_t)c * lda + r], ui[c], s0);
                s1 = fma(A[(size_t)(c + 1) * lda + r], ui[c + 1], s1);
                s2 = fma(A[(size_t)(c + 2) * lda + r], ui[c + 2], s2);
                s3 = fma(A[(size_t)(c + 3) * lda + r], ui[c + 3], s3);
            }
            for (; c < c1; ++c) s0 = fma(A[(size_t)c * lda + r], ui[c], s0);
            a.xpart[(size_t)ch * m + r] = (s0 + s1) + (s2 + s3);
        }
        for (int w = gwarp; w < 2 * i + 1; w += gwarps) {
            const double *col = (w <= i) ? Y + (size_t)w * n : U + (size_t)(w - i - 1) * n;
            const double s = warp_dot(col, U + (size_t)i * n, i + 1, n);
            if (lane == 0) {
                if (w <= i) t3[w] = s;
                else t4[w - i - 1] = s;
            }
        }
        if (!grid_sync(a.bar)) return;
        // (g) x_i = pi (A u - V t3 - X t4), rows i+1..m-1
        for (int r = i + 1 + gtid; r < m; r += gthreads) {
            double x = 0.0;
            for (int ch = 0; ch < a.chunks; ++ch) x += a.xpart[(size_t)ch * m + r];
            x -= dot2(V + r, t3, X + r, t4, m, 1, i) + V[(size_t)i * m + r] * t3[i];
            X[(size_t)i * m + r] = pi * x;
        }
        if (!grid_sync(a.bar)) return;
    }
}

// ---------------------------------------------------------- QR panel
// geqr2 on the local m x nb panel A (Sec. 4.3, step 1): column reflectors
// with the panel's later columns updated after each one.  part[grid][b]:
// partial products v^T A[:, c] per CTA.
struct Geqr2Args {
    double *A;
    int lda, m, nb, b;
    double *tau;
    double *part;
    GridBar *bar;
};

__global__ void __launch_bounds__(256) k_geqr2(Geqr2Args a) {
    __shared__ double sh[32];
    __shared__ double sw[64];
    const int T = blockDim.x, G = gridDim.x;
    const int gtid = blockIdx.x * T + threadIdx.x, gthreads = G * T;
    const int m = a.m, nb = a.nb, b = a.b;
    double *A = a.A;
    const long long lda = a.lda;
    for (int i = 0; i < nb; ++i) {
        double ss = 0.0;
        for (int r = i + 1 + gtid; r < m; r += gthreads) ss = fma(A[(size_t)i * lda + r], A[(size_t)i * lda + r], ss);
        ss = block_sum(ss, sh);
        if (threadIdx.x == 0) a.part[(size_t)blockIdx.x * (b + 1) + b] = ss;
        if (!grid_sync(a.bar)) return;
        double sig2 = grid_partials(a.part + b, G, b + 1, sh);
        const double alpha = A[(size_t)i * lda + i];
        double tau, beta;
        const double sc = reflector(alpha, sig2, tau, beta);
        // w_c = v^T A[i:, c] for every later panel column at once, from the
        // column before scaling (v_r = sc A[r, i] for r > i, v_i = 1; the
        // scaled v is written in the update phase, after the barrier, so no
        // CTA reads a row another one is scaling): each warp sums its rows for
        // column c = i + 1 + lane (lanes over columns, the warp's rows in
        // turn), then the warps' sums are added in shared memory in a fixed
        // order
        {
            __shared__ double wsum[8][33];
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
            const int c = i + 1 + lane;
            double acc = 0.0;
            if (c < nb) {
                for (int r = i + 1 + blockIdx.x * nwarp + wid; r < m; r += G * nwarp)
                    acc = fma(A[(size_t)i * lda + r], A[(size_t)c * lda + r], acc);
                acc *= sc;
                if (gtid < 32) acc += A[(size_t)c * lda + i];           // v_i = 1 at row i (one warp of CTA 0)
            }
            if (wid < 8) wsum[wid][lane] = acc;
            __syncthreads();
            if (threadIdx.x < 32) {
                double t = 0.0;
                for (int q = 0; q < nwarp && q < 8; ++q) t += wsum[q][threadIdx.x];
                if (i + 1 + (int)threadIdx.x < nb) a.part[(size_t)blockIdx.x * (b + 1) + i + 1 + threadIdx.x] = t;
            }
        }
        if (gtid == 0) a.tau[i] = tau;
        if (!grid_sync(a.bar)) return;
        // A[i:, c] -= tau v w_c, w_c summed over the CTAs: thread t takes
        // column offset t % 32 and every eighth CTA from t / 32
        {
            __shared__ double red[8][33];
            const int co = threadIdx.x & 31, kk = threadIdx.x >> 5, c = i + 1 + co;
            double w = 0.0;
            if (c < nb && kk < 8)
                for (int k = kk; k < G; k += 8) w += a.part[(size_t)k * (b + 1) + c];
            if (kk < 8) red[kk][co] = w;
            __syncthreads();
            if (threadIdx.x < 32) {
                double t = 0.0;
                for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
                sw[threadIdx.x] = tau * t;
            }
            __syncthreads();
        }
        for (int r = i + gtid; r < m; r += gthreads) {
            double v = 1.0;
            if (r > i) {
                v = A[(size_t)i * lda + r] * sc;        // the reflector's entry, stored scaled
                A[(size_t)i * lda + r] = v;
            }
            for (int c = i + 1; c < nb; ++c) A[(size_t)c * lda + r] -= v * sw[c - i - 1];
        }
        if (gtid == 0) A[(size_t)i * lda + i] = beta;
        if (!grid_sync(a.bar)) return;
    }
}

// ------------------------------------------------ block reflector helpers
// Y (rows x nb, ld rows) from the stored reflectors: column j is zero above
// row j + off, 1 at row j + off, then the stored entries src[j * ldsrc + r]
// (column reflectors: off = 0, src = A's panel; row reflectors: the entries
// of row j of A's panel, read with ldsrc = 1 and stride lda, off = 0 on the
// shifted rows).
__global__ void k_form_y(double *Y, int rows, int nb, const double *src, long long sr, long long sc) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)rows * nb) return;
    const int j = (int)(k / rows), r = (int)(k % rows);
    Y[k] = (r < j) ? 0.0 : (r == j) ? 1.0 : src[(size_t)j * sc + (size_t)r * sr];
}

// T^{-1} = Y^T Y with the diagonal 1 / tau (Eqs. inv_t, larft_update; only the
// upper triangle is read): the product is done by k_dgemm, this fixes the
// diagonal; a zero tau (H = I) is marked by a zero diagonal entry
__global__ void k_tinv_diag(double *Ti, int nb, const double *tau) {
    const int j = threadIdx.x;
    if (j < nb) Ti[(size_t)j * nb + j] = (tau[j] != 0.0) ? 1.0 / tau[j] : 0.0;
}

// Triangular solve with T^{-1} (nb x nb, upper, in Ti) on many right-hand
// sides: mode 0: W = T Z  (T^{-1} W = Z, column vectors of Z, nb x ncol, ld ldz)
//        mode 1: W = T^T Z (T^{-T} W = Z)
//        mode 2: W = Z T   (W T^{-1} = Z, row vectors of Z, nrow x nb, ld ldz)
//        mode 3: W = Z T^T (W T^{-T} = Z)
// in place; a zero diagonal entry (tau = 0) makes that component of W zero.
__global__ void __launch_bounds__(128) k_tsolve(const double *__restrict__ Ti, int nb, double *Z, int ldz,
                                                int count, int mode) {
    extern __shared__ double st[];   // T^{-1}, nb x nb
    for (int k = threadIdx.x; k < nb * nb; k += blockDim.x) st[k] = Ti[k];
    __syncthreads();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= count) return;
    // element p of this right-hand side
    const bool colwise = mode < 2;
    auto at = [&](int p) -> double & { return colwise ? Z[(size_t)v * ldz + p] : Z[(size_t)p * ldz + v]; };
    auto tij = [&](int i, int j) { return st[(size_t)j * nb + i]; };   // T^{-1}(i, j), i <= j
    const bool upper_solve = (mode == 0) || (mode == 3);   // T^{-1} W = Z or W T^{-T} = Z: back substitution
    if (upper_solve) {
        for (int p = nb - 1; p >= 0; --p) {
            const double dp = tij(p, p);
            if (dp == 0.0) { at(p) = 0.0; continue; }
            double s = at(p);
            for (int q = p + 1; q < nb; ++q) s -= tij(p, q) * at(q);
            at(p) = s / dp;
        }
    } else {
        for (int p = 0; p < nb; ++p) {
            const double dp = tij(p, p);
            if (dp == 0.0) { at(p) = 0.0; continue; }
            double s = at(p);
            for (int q = 0; q < p; ++q) s -= tij(q, p) * at(q);
            at(p) = s / dp;
        }
    }
}

// C (rows x cols, ldc) := H C or H^T C (left) or C H or C H^T (right), H =
// I - Y T Y^T = H_1 ... H_nb for the explicit Y (left: rows x nb; right:
// cols x nb), modified compact WY: T^{-1} = Y^T Y (diag 1/tau), Z = Y^T C
// (or C Y), W = T Z / T^T Z (or Z T / Z T^T) by the triangular solve, C -= Y W
// (or W Y^T).  Scratch: Ti (nb x nb), Z (nb x cols or rows x nb).
cudaError_t apply_block(int left, int trans, int rows, int cols, const double *Y, int nb, const double *tau,
                        double *C, int ldc, double *Ti, double *Z, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || nb <= 0) return cudaSuccess;
    const int ry = left ? rows : cols;   // rows of Y
    cudaError_t e = dgemm(1, 0, nb, nb, ry, 1.0, Y, ry, Y, ry, 0.0, Ti, nb, st);
    if (e != cudaSuccess) return e;
    k_tinv_diag<<<1, ((nb + 31) / 32) * 32, 0, st>>>(Ti, nb, tau);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = sizeof(double) * nb * nb;
    if (smem > 48 * 1024) {   // T^{-1} above the static limit: opt in to more dynamic shared memory
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [] {
            attr = cudaFuncSetAttribute(k_tsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        if (attr != cudaSuccess) return attr;
        if (smem > 200 * 1024) return cudaErrorInvalidValue;
    }
    if (left) {
        if ((e = dgemm(1, 0, nb, cols, rows, 1.0, Y, rows, C, ldc, 0.0, Z, nb, st)) != cudaSuccess) return e;
        k_tsolve<<<(cols + 127) / 128, 128, smem, st>>>(Ti, nb, Z, nb, cols, trans ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return dgemm(0, 0, rows, cols, nb, -1.0, Y, rows, Z, nb, 1.0, C, ldc, st);
    }
    if ((e = dgemm(0, 0, rows, nb, cols, 1.0, C, ldc, Y, cols, 0.0, Z, rows, st)) != cudaSuccess) return e;
    k_tsolve<<<(rows + 127) / 128, 128, smem, st>>>(Ti, nb, Z, rows, rows, trans ? 3 : 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return dgemm(0, 1, rows, cols, nb, -1.0, Z, rows, Y, cols, 1.0, C, ldc, st);
}

__global__ void k_fill(double *X, long long rows, long long cols, long long ld, double diag_val) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows * cols) return;
    const long long c = k / rows, r = k % rows;
    X[c * ld + r] = (r == c) ? diag_val : 0.0;
}

__global__ void k_copy_upper(const double *A, long long lda, double *R, long long ldr, int n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)n * n) return;
    const int c = (int)(k / n), r = (int)(k % n);
    R[(size_t)c * ldr + r] = (r <= c) ? A[(size_t)c * lda + r] : 0.0;
}

__global__ void k_zero_rows(double *X, long long ld, int r0, int r1, int cols) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = r1 - r0;
    if (rows <= 0 || k >= (long long)rows * cols) return;
    const int c = (int)(k / rows), r = r0 + (int)(k % rows);
    X[(size_t)c * ld + r] = 0.0;
}

__global__ void k_read_err(const GridBar *bar, int *info) {
    if (bar->err) *info = BDC_ERR_TIMEOUT;
}

int coop_blocks(const void *fn, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    per = std::min(per, 2);
    return std::max(1, sms * std::max(per, 1));
}

// workspace layout of the dense routines (bytes from an aligned base)
struct DenseWs {
    size_t bar, PW, QW, yraw, tv, xpart, part, Y, Ti, Z, split, split_doubles, total;
};
constexpr int kChunkW = 128;   // columns per partial sum of A u

DenseWs dense_ws(int m, int n, int b, int zcols) {
    DenseWs w{};
    size_t o = 0;
    const int chunks = (n + kChunkW - 1) / kChunkW;
    const int grid = 4 * 256;   // upper bound of the cooperative grid (partial arrays)
    w.bar = o; o += 256;
    w.PW = o; o += al256(sizeof(double) * 2 * (size_t)b * m);
    w.QW = o; o += al256(sizeof(double) * 2 * (size_t)b * n);
    w.yraw = o; o += al256(sizeof(double) * (size_t)n);
    w.tv = o; o += al256(sizeof(double) * 4 * (size_t)b);
    w.xpart = o; o += al256(sizeof(double) * (size_t)chunks * m);
    w.part = o; o += al256(sizeof(double) * (size_t)grid * (b + 1));
    w.Y = o; o += al256(sizeof(double) * (size_t)std::max(m, n) * b);
    w.Ti = o; o += al256(sizeof(double) * (size_t)b * b);
    w.Z = o; o += al256(sizeof(double) * (size_t)b * std::max(std::max(m, n), zcols));
    w.split_doubles = (size_t)16 * b * std::max(std::max(m, n), zcols);
    w.split = o; o += al256(sizeof(double) * w.split_doubles);
    w.total = o + 256;
    return w;
}

// the split-K scratch of the calling thread's dense routine
struct SplitScope {
    SplitScope(char *ws, const DenseWs &w) {
        g_split_buf = (double *)(ws + w.split);
        g_split_cap = w.split_doubles;
    }
    ~SplitScope() {
        g_split_buf = nullptr;
        g_split_cap = 0;
    }
};

cudaError_t launch_coop(const void *fn, int grid, void *args, cudaStream_t st) {
    void *params[] = {args};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), params, 0, st);
}

}  // namespace

// ---------------------------------------------------------------- drivers
// Bidiagonalization, Algorithm 1 (m >= n): per panel of b, k_labrd, then the
// merged rank-(2b) update of the trailing matrix (one product).
constexpr long long kLabrdWork = 8192;   // trailing-matrix entries per CTA of the panel kernel

cudaError_t dense_gebrd(int m, int n, double *A, int lda, double *d, double *e, double *tauq, double *taup, int b,
                        char *ws, cudaStream_t st) {
    const DenseWs w = dense_ws(m, n, b, n);
    SplitScope split_scope(ws, w);
    GridBar *bar = (GridBar *)(ws + w.bar);
    cudaError_t err = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);   // count, gen (not the error word)
    if (err != cudaSuccess) return err;
    // CTAs per panel by the work of its steps (the products with the
    // trailing matrix, ~ml nl FMAs): a small trailing matrix cannot use the
    // whole GPU, and every barrier costs more with more CTAs
    const int gmax = std::min(coop_blocks((const void *)k_labrd, 256, 0), 4 * 256);
    for (int i0 = 0; i0 < n; i0 += b) {
        const int nb = std::min(b, n - i0), ml = m - i0, nl = n - i0;
        const int grid = (int)std::max<long long>(8, std::min<long long>(gmax, (long long)ml * nl / kLabrdWork));
        LabrdArgs a{A + i0 + (size_t)i0 * lda, lda, ml, nl, nb, b,
                    d + i0, e + i0, tauq + i0, taup + i0,
                    (double *)(ws + w.PW), (double *)(ws + w.QW), (double *)(ws + w.yraw), (double *)(ws + w.tv),
                    (double *)(ws + w.xpart), (double *)(ws + w.part), (nl + kChunkW - 1) / kChunkW, kChunkW, bar};
        if ((err = launch_coop((const void *)k_labrd, grid, &a, st)) != cudaSuccess) return err;
        if (nb < nl) {
            // the merged rank-(2b) update A[nb:, nb:] -= P Q^T (Eq. bidiag-A-trail3):
            // P = [V X] (ml x 2b) and Q = [Y U] (nl x 2b) are contiguous column
            // blocks, zero in the columns a short last panel does not use, so
            // the whole update is ONE product with K = 2b
            const double *P = (const double *)(ws + w.PW), *Q = (const double *)(ws + w.QW);
            if ((err = dgemm(0, 1, ml - nb, nl - nb, 2 * b, -1.0, P + nb, ml, Q + nb, nl, 1.0,
                             A + i0 + nb + (size_t)(i0 + nb) * lda, lda, st)) != cudaSuccess)
                return err;
        }
    }
    return cudaSuccess;
}

// QR (Sec. 4.3): per panel, k_geqr2 and the update of the trailing columns by
// H^T = I - Y T^T Y^T in modified compact WY
cudaError_t dense_geqrf(int m, int n, double *A, int lda, double *tau, int b, char *ws, cudaStream_t st) {
    if (b < 1 || b > 32) return cudaErrorInvalidValue;   // k_geqr2: a lane per later panel column
    const DenseWs w = dense_ws(m, n, b, n);
    SplitScope split_scope(ws, w);
    GridBar *bar = (GridBar *)(ws + w.bar);
    cudaError_t err = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);   // count, gen (not the error word)
    if (err != cudaSuccess) return err;
    // enough CTAs for ~4 panel rows per thread: the per-column reductions over
    // the CTAs' partial sums grow with the grid
    const int grid = std::max(1, std::min(coop_blocks((const void *)k_geqr2, 256, 0), (m + 1023) / 1024));
    double *Y = (double *)(ws + w.Y), *Ti = (double *)(ws + w.Ti), *Z = (double *)(ws + w.Z);
    const int kmax = std::min(m, n);
    for (int i0 = 0; i0 < kmax; i0 += b) {
        const int nb = std::min(b, kmax - i0), ml = m - i0;
        Geqr2Args a{A + i0 + (size_t)i0 * lda, lda, ml, nb, b, tau + i0, (double *)(ws + w.part), bar};
        if ((err = launch_coop((const void *)k_geqr2, grid, &a, st)) != cudaSuccess) return err;
        if (i0 + nb < n) {
            const long long cnt = (long long)ml * nb;
            k_form_y<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Y, ml, nb, A + i0 + (size_t)i0 * lda, 1, lda);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            if ((err = apply_block(1, 1, ml, n - i0 - nb, Y, nb, tau + i0, A + i0 + (size_t)(i0 + nb) * lda, lda, Ti,
                                   Z, st)) != cudaSuccess)
                return err;
        }
    }
    return cudaSuccess;
}

// the first n columns of Q = H_1 ... H_k in place of A (Eq. orgqr-q): the
// panels from the last to the first, each panel's reflectors copied to Y
// before its columns are reset to the identity's
cudaError_t dense_orgqr(int m, int n, int k, double *A, int lda, const double *tau, int b, char *ws, cudaStream_t st) {
    const DenseWs w = dense_ws(m, n, b, n);
    SplitScope split_scope(ws, w);
    double *Y = (double *)(ws + w.Y), *Ti = (double *)(ws + w.Ti), *Z = (double *)(ws + w.Z);
    cudaError_t err = cudaSuccess;
    // columns k..n-1 start as identity columns
    if (k < n) {
        const long long cnt = (long long)m * (n - k);
        k_fill<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(A + (size_t)k * lda, m, n - k, lda, 0.0);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const long long c2 = (long long)(m - k) * (n - k);
        k_fill<<<(unsigned)((c2 + 255) / 256), 256, 0, st>>>(A + k + (size_t)k * lda, m - k, n - k, lda, 1.0);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    const int last = ((k - 1) / b) * b;
    for (int i0 = last; i0 >= 0; i0 -= b) {
        const int nb = std::min(b, k - i0), ml = m - i0;
        const long long cnt = (long long)ml * nb;
        k_form_y<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Y, ml, nb, A + i0 + (size_t)i0 * lda, 1, lda);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        // the panel's columns become identity columns (rows i0.., zero above)
        const long long c2 = (long long)m * nb;
        k_fill<<<(unsigned)((c2 + 255) / 256), 256, 0, st>>>(A + (size_t)i0 * lda, m, nb, lda, 0.0);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        k_fill<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(A + i0 + (size_t)i0 * lda, ml, nb, lda, 1.0);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = apply_block(1, 0, ml, n - i0, Y, nb, tau + i0, A + i0 + (size_t)i0 * lda, lda, Ti, Z, st)) !=
            cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

// back-transformation (Sec. 4.3): vect 0: C (m x cols) := Q1 C with the
// column reflectors of gebrd (A m x n, tauq); vect 1: C (rows x n) := C P1^T
// with the row reflectors (taup).  Panels from the last to the first.
cudaError_t dense_ormbr(int vect, int m, int n, const double *A, int lda, const double *tau, double *C, int ldc,
                        int cdim, int b, char *ws, cudaStream_t st) {
    const DenseWs w = dense_ws(m, n, b, std::max(cdim, n));
    SplitScope split_scope(ws, w);
    double *Y = (double *)(ws + w.Y), *Ti = (double *)(ws + w.Ti), *Z = (double *)(ws + w.Z);
    cudaError_t err = cudaSuccess;
    if (vect == 0) {
        const int last = ((n - 1) / b) * b;
        for (int i0 = last; i0 >= 0; i0 -= b) {
            const int nb = std::min(b, n - i0), ml = m - i0;
            const long long cnt = (long long)ml * nb;
            k_form_y<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Y, ml, nb, A + i0 + (size_t)i0 * lda, 1, lda);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            if ((err = apply_block(1, 0, ml, cdim, Y, nb, tau + i0, C + i0, ldc, Ti, Z, st)) != cudaSuccess)
                return err;
        }
        return cudaSuccess;
    }
    if (n < 2) return cudaSuccess;
    const int nr = n - 1;   // row reflectors G_0 .. G_{n-2}, acting on columns 1..n-1
    const int last = ((nr - 1) / b) * b;
    for (int i0 = last; i0 >= 0; i0 -= b) {
        const int nb = std::min(b, nr - i0), ny = n - 1 - i0;
        const long long cnt = (long long)ny * nb;
        // Y[r][j] = u_{i0+j} at column i0 + 1 + r: row i0 + j of A from column i0 + 1
        k_form_y<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(Y, ny, nb, A + i0 + (size_t)(i0 + 1) * lda, lda, 1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = apply_block(0, 1, cdim, ny, Y, nb, tau + i0, C + (size_t)(i0 + 1) * ldc, ldc, Ti, Z, st)) !=
            cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

size_t dense_ws_bytes(int m, int n, int b) { return dense_ws(m, n, b, std::max(m, n)).total; }
cudaError_t dense_clear_err(char *ws, cudaStream_t st) {
    return cudaMemsetAsync(ws + dense_ws(1, 1, 1, 1).bar, 0, sizeof(GridBar), st);
}
cudaError_t dense_read_err(char *ws, int *info, cudaStream_t st) {
    k_read_err<<<1, 1, 0, st>>>((const GridBar *)(ws + dense_ws(1, 1, 1, 1).bar), info);
    return cudaGetLastError();
}
cudaError_t dense_copy_upper(const double *A, int lda, double *R, int ldr, int n, cudaStream_t st) {
    const long long cnt = (long long)n * n;
    k_copy_upper<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(A, lda, R, ldr, n);
    return cudaGetLastError();
}
cudaError_t dense_zero_rows(double *X, int ld, int r0, int r1, int cols, cudaStream_t st) {
    const long long cnt = (long long)(r1 - r0) * cols;
    if (cnt <= 0) return cudaSuccess;
    k_zero_rows<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(X, ld, r0, r1, cols);
    return cudaGetLastError();
}
cudaError_t dense_dgemm(int ta, int tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                        int ldb, double beta, double *C, int ldc, cudaStream_t st) {
    return dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
}


}  // namespace bdc

// ------------------------------------------------------------- C ABI
using namespace bdc;

namespace {

constexpr int kDenseBlock = 32;   // b: columns / rows per panel (reflectors per block)
// reflectors per block when they are applied (back-transformation, explicit
// Q): wider blocks pass over C fewer times (Z = Y^T C and C -= Y W with
// K = kApplyBlock); T^{-1} (kApplyBlock^2 doubles) stays in shared memory
constexpr int kApplyBlock = 64;
constexpr int kWsBlock = kApplyBlock > kDenseBlock ? kApplyBlock : kDenseBlock;   // workspace sizing
constexpr double kQrRatio = 1.6;  // m >= 1.6 n: QR first (Sec. 4.3)

char *align_ws(void *work) { return (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255); }

int note_cuda(cudaError_t e) { return e == cudaSuccess ? 0 : BDC_ERR_CUDA; }

struct GesvdWs {
    size_t dense, vecs, R, UR, bdc, total;
};
GesvdWs gesvd_layout(int m, int n, const bdc_opts *o) {
    GesvdWs w{};
    size_t off = 0;
    w.dense = off; off += al256(dense_ws_bytes(m, n, kWsBlock));
    w.vecs = off; off += al256(sizeof(double) * 4 * (size_t)n + 64);
    const bool qr = m >= kQrRatio * n;
    w.R = off; off += qr ? al256(sizeof(double) * (size_t)n * n) : 0;
    w.UR = off; off += qr ? al256(sizeof(double) * (size_t)n * n) : 0;
    w.bdc = off; off += al256(bdc_svd_workspace(n, o));
    w.total = off + 512;
    return w;
}

}  // namespace

extern "C" {

size_t bdc_gebrd_workspace(int m, int n) {
    if (m < n || n < 0) return 0;
    return dense_ws_bytes(m, n, kWsBlock) + 512;
}

int bdc_gebrd(int m, int n, double *A, int lda, double *d, double *e, double *tauq, double *taup, void *work,
              size_t lwork, int *d_info, bdc_stream_t stream) {
    if (n < 0) return -2;
    if (m < n) return -1;
    if (n > 0 && !A) return -3;
    if (lda < std::max(1, m)) return -4;
    if (n > 0 && (!d || !tauq || !taup || (n > 1 && !e))) return -5;
    if (!d_info) return -12;
    cudaStream_t st = (cudaStream_t)stream;
    if (int r = note_cuda(cudaMemsetAsync(d_info, 0, sizeof(int), st))) return r;
    if (n == 0) return 0;
    if (!work) return -10;
    if (lwork < bdc_gebrd_workspace(m, n)) return -11;
    char *ws = align_ws(work);
    if (int r = note_cuda(dense_clear_err(ws, st))) return r;
    if (int r = note_cuda(cudaMemsetAsync(taup, 0, sizeof(double) * n, st))) return r;
    if (int r = note_cuda(dense_gebrd(m, n, A, lda, d, e, tauq, taup, kDenseBlock, ws, st))) return r;
    return note_cuda(dense_read_err(ws, d_info, st));
}

int bdc_ormbr(int vect, int m, int n, const double *A, int lda, const double *tau, double *C, int ldc, int cdim,
              void *work, size_t lwork, bdc_stream_t stream) {
    if (vect < 0 || vect > 1) return -1;
    if (m < n || n < 0) return -2;
    if (n > 0 && !A) return -4;
    if (lda < std::max(1, m)) return -5;
    if (n > 0 && !tau) return -6;
    if (cdim < 0) return -9;
    if (cdim > 0 && n > 0 && !C) return -7;
    if (ldc < std::max(1, vect == 0 ? m : cdim)) return -8;
    if (n == 0 || cdim == 0) return 0;
    if (!work) return -10;
    const size_t need = dense_ws_bytes(std::max(m, cdim), std::max(n, cdim), kWsBlock) + 512;
    if (lwork < need) return -11;
    return note_cuda(dense_ormbr(vect, m, n, A, lda, tau, C, ldc, cdim, kApplyBlock, align_ws(work),
                                 (cudaStream_t)stream));
}

size_t bdc_ormbr_workspace(int m, int n, int cdim) {
    if (m < n || n < 0 || cdim < 0) return 0;
    return dense_ws_bytes(std::max(m, cdim), std::max(n, cdim), kWsBlock) + 512;
}

size_t bdc_geqrf_workspace(int m, int n) {
    if (m < 0 || n < 0) return 0;
    return dense_ws_bytes(std::max(m, 1), std::max(n, 1), kWsBlock) + 512;
}

int bdc_geqrf(int m, int n, double *A, int lda, double *tau, void *work, size_t lwork, int *d_info,
              bdc_stream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m > 0 && n > 0 && !A) return -3;
    if (lda < std::max(1, m)) return -4;
    if (std::min(m, n) > 0 && !tau) return -5;
    if (!d_info) return -9;
    cudaStream_t st = (cudaStream_t)stream;
    if (int r = note_cuda(cudaMemsetAsync(d_info, 0, sizeof(int), st))) return r;
    if (std::min(m, n) == 0) return 0;
    if (!work) return -6;
    if (lwork < bdc_geqrf_workspace(m, n)) return -7;
    char *ws = align_ws(work);
    if (int r = note_cuda(dense_clear_err(ws, st))) return r;
    if (int r = note_cuda(dense_geqrf(m, n, A, lda, tau, kDenseBlock, ws, st))) return r;
    return note_cuda(dense_read_err(ws, d_info, st));
}

int bdc_orgqr(int m, int n, double *A, int lda, const double *tau, void *work, size_t lwork, bdc_stream_t stream) {
    if (m < 0) return -1;
    if (n < 0 || n > m) return -2;
    if (n > 0 && !A) return -3;
    if (lda < std::max(1, m)) return -4;
    if (n > 0 && !tau) return -5;
    if (n == 0) return 0;
    if (!work) return -6;
    if (lwork < bdc_geqrf_workspace(m, n)) return -7;
    return note_cuda(dense_orgqr(m, n, n, A, lda, tau, kApplyBlock, align_ws(work), (cudaStream_t)stream));
}

size_t bdc_gesvd_workspace(int m, int n, const bdc_opts *o) {
    if (m < n || n < 0) return 0;
    return gesvd_layout(m, std::max(n, 1), o).total;
}

int bdc_gesvd(int m, int n, double *A, int lda, double *S, double *U, int ldu, double *VT, int ldvt,
              const bdc_opts *o, void *work, size_t lwork, int *d_info, bdc_stream_t stream) {
    if (n < 0) return -2;
    if (m < n) return -1;
    if (n > 0 && !A) return -3;
    if (lda < std::max(1, m)) return -4;
    if (n > 0 && (!S || !U || !VT)) return -5;
    if (ldu < std::max(1, m)) return -7;
    if (ldvt < std::max(1, n)) return -9;
    if (!d_info) return -13;
    cudaStream_t st = (cudaStream_t)stream;
    if (int r = note_cuda(cudaMemsetAsync(d_info, 0, sizeof(int), st))) return r;
    if (n == 0) return 0;
    if (o && o->vectors != BDC_VEC_BOTH) return -10;
    if (!work) return -11;
    const GesvdWs L = gesvd_layout(m, n, o);
    if (lwork < L.total) return -12;
    char *ws = align_ws(work);
    char *dws = ws + L.dense;
    double *d = (double *)(ws + L.vecs), *e = d + n, *tq = e + n, *tp = tq + n;
    const int b = kDenseBlock;
    if (int r = note_cuda(dense_clear_err(dws, st))) return r;
    if (int r = note_cuda(cudaMemsetAsync(tp, 0, sizeof(double) * n, st))) return r;
    const size_t lwb = bdc_svd_workspace(n, o);
    int rc = 0;
    if (m >= kQrRatio * n) {
        // tall and skinny: A = Q R, the SVD of R, U = Q U_R (Sec. 4.3)
        double *R = (double *)(ws + L.R), *UR = (double *)(ws + L.UR);
        if ((rc = note_cuda(dense_geqrf(m, n, A, lda, tq, b, dws, st)))) return rc;
        if ((rc = note_cuda(dense_copy_upper(A, lda, R, n, n, st)))) return rc;
        if ((rc = note_cuda(dense_orgqr(m, n, n, A, lda, tq, kApplyBlock, dws, st)))) return rc;
        if ((rc = note_cuda(cudaMemsetAsync(tq, 0, sizeof(double) * n, st)))) return rc;
        if ((rc = note_cuda(dense_gebrd(n, n, R, n, d, e, tq, tp, b, dws, st)))) return rc;
        if ((rc = bdc_svd_ex(n, d, e, UR, S, VT, n, ldvt, o, ws + L.bdc, lwb, d_info, stream))) return rc;
        if ((rc = note_cuda(dense_ormbr(0, n, n, R, n, tq, UR, n, n, kApplyBlock, dws, st)))) return rc;
        if ((rc = note_cuda(dense_ormbr(1, n, n, R, n, tp, VT, ldvt, n, kApplyBlock, dws, st)))) return rc;
        if ((rc = note_cuda(dense_dgemm(0, 0, m, n, n, 1.0, A, lda, UR, n, 0.0, U, ldu, st)))) return rc;
    } else {
        if ((rc = note_cuda(dense_gebrd(m, n, A, lda, d, e, tq, tp, b, dws, st)))) return rc;
        if ((rc = bdc_svd_ex(n, d, e, U, S, VT, ldu, ldvt, o, ws + L.bdc, lwb, d_info, stream))) return rc;
        if ((rc = note_cuda(dense_zero_rows(U, ldu, n, m, n, st)))) return rc;
        if ((rc = note_cuda(dense_ormbr(0, m, n, A, lda, tq, U, ldu, n, kApplyBlock, dws, st)))) return rc;
        if ((rc = note_cuda(dense_ormbr(1, m, n, A, lda, tp, VT, ldvt, n, kApplyBlock, dws, st)))) return rc;
    }
    return note_cuda(dense_read_err(dws, d_info, st));
}

}  // extern "C"
