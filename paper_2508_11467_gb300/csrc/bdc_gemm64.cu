// Merge products of Eq. (bdc-Mv2Bv-u-vt) in the working precision: C = A * B,
// all column-major, a batch of independent problems per launch (four per
// merge node: the top and bottom blocks of W~ U_M and Q~ V_M).
//
// FP32 build: CUDA-core FP32 FMA, CTA tile 64 x 64, K step 16, 256 threads
// of 4 x 4 outputs, operands staged k-major in padded shared tiles (float4
// reads), the next K step prefetched into registers.
//
// FP64 build: tensor-core FP64 (DMMA, mma.sync.m8n8k4.f64).  CTA tile 64 x 64
// (32 x 32, 32 x 64 or 64 x 32 for small problems), K step 16, warps of
// 32 x 32 (4 x 4 fragments of 8 x 8).  Shared tiles are padded
// so that the fragment loads of a warp hit every bank exactly twice (the
// minimum for 32 doubles).  The next K step is prefetched into registers while
// the current one is multiplied.  Problems whose actual size (known only on
// the device after deflation) is smaller than the launch grid exit early.
#include "bdc_internal.cuh"

namespace BDC_NS {

namespace {

#ifdef BDC_FP32
constexpr int BM = 64, BN = 64, BK = 16, SP = 68;   // SP: padded row stride of both tiles (floats)

__global__ void __launch_bounds__(256) k_gemm32(const GemmProb *__restrict__ probs, int tilesN) {
    __shared__ __align__(16) float As[BK * SP];    // As[k][m]
    __shared__ __align__(16) float Bs[BK * SP];    // Bs[k][n]
    const GemmProb pr = probs[blockIdx.y];
    const int m0 = (blockIdx.x / tilesN) * BM, n0 = (blockIdx.x % tilesN) * BN;
    if (m0 >= pr.M || n0 >= pr.N) return;
    const int tid = threadIdx.x;
    const int tm = (tid >> 4) * 4, tn = (tid & 15) * 4;
    const float *__restrict__ A = pr.A;
    const float *__restrict__ B = pr.B;
    const int M = pr.M, N = pr.N, K = pr.K, lda = pr.lda, ldb = pr.ldb;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + r * 256;       // 0..1023
            const int am = idx & 63, ak = idx >> 6;
            const int gm = m0 + am, gk = k0 + ak;
            ra[r] = (gm < M && gk < K) ? A[(size_t)gk * lda + gm] : 0.f;
            const int bk = idx & 15, bn = idx >> 4;
            const int gn = n0 + bn, gk2 = k0 + bk;
            rb[r] = (gn < N && gk2 < K) ? B[(size_t)gn * ldb + gk2] : 0.f;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + r * 256;
            As[(idx >> 6) * SP + (idx & 63)] = ra[r];
            Bs[(idx & 15) * SP + (idx >> 4)] = rb[r];
        }
    };
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(As + kk * SP + tm);
            const float4 b = *reinterpret_cast<const float4 *>(Bs + kk * SP + tn);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
    }
    float *__restrict__ C = pr.C;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tn + j;
        if (gn >= N) continue;
        float *__restrict__ Cc = C + gemm_col(pr, gn);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gm = m0 + tm + i;
            if (gm < M) Cc[gm] = acc[i][j];
        }
    }
}
#else
constexpr int BK = 16;

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// CTA tile (32 WM) x (32 WN): WM x WN warps of 32 x 32 each, registers
// capped so that twelve warps fit an SM (three 2 x 2 CTAs; measured: two
// CTAs of 206 registers 29.7 ms of FP64 products at n = 16384, three 29.0,
// four with spills 29.2); the small
// tiles serve merges whose blocks are a few dozen rows (a 64 x 64 tile
// there multiplies mostly zeros at GB300's modest FP64 tensor rate)
template <int WM, int WN>
__global__ void __launch_bounds__(32 * WM * WN, 3 * 4 / (WM * WN)) k_gemm64(const GemmProb *__restrict__ probs, int tilesN) {
    constexpr int BM = 32 * WM, BN = 32 * WN, T = 32 * WM * WN;
    constexpr int SA = BM + 8;   // As[k][m] row stride (doubles)
    constexpr int SB = BK + 4;   // Bs[n][k] row stride
    constexpr int LA = BM * BK / T, LB = BN * BK / T;   // elements per thread
    __shared__ double As[BK * SA];
    __shared__ double Bs[BN * SB];
    const GemmProb pr = probs[blockIdx.y];
    const int m0 = (blockIdx.x / tilesN) * BM, n0 = (blockIdx.x % tilesN) * BN;
    if (m0 >= pr.M || n0 >= pr.N) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp / WN) * 32, wn = (warp % WN) * 32;
    const int g = lane >> 2, tg = lane & 3;
    const double *__restrict__ A = pr.A;
    const double *__restrict__ B = pr.B;
    const int M = pr.M, N = pr.N, K = pr.K, lda = pr.lda, ldb = pr.ldb;

    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    // global -> register staging: A tile (BM m x BK k), B tile (BK k x BN n)
    double ra[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int idx = tid + r * T;
            const int am = idx % BM, ak = idx / BM;
            const int gm = m0 + am, gk = k0 + ak;
            ra[r] = (gm < M && gk < K) ? A[(size_t)gk * lda + gm] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int idx = tid + r * T;
            const int bk = idx % BK, bn = idx / BK;
            const int gn = n0 + bn, gk = k0 + bk;
            rb[r] = (gn < N && gk < K) ? B[(size_t)gn * ldb + gk] : 0.0;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int idx = tid + r * T;
            As[(idx / BM) * SA + (idx % BM)] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int idx = tid + r * T;
            Bs[(idx / BK) * SB + (idx % BK)] = rb[r];
        }
    };
    load(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        store();
        __syncthreads();
        if (k0 + BK < K) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            if (k0 + kk >= K) break;               // zero padding of the last K block
            double af[4], bf[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) af[i] = As[(kk + tg) * SA + wm + i * 8 + g];
#pragma unroll
            for (int j = 0; j < 4; ++j) bf[j] = Bs[(wn + j * 8 + g) * SB + kk + tg];
            // 8 x 8 fragments wholly outside M x N are skipped (warp-uniform):
            // a merge of order 16 has blocks of about 8 x 16 in a 32 x 32 tile
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (m0 + wm + i * 8 < M && n0 + wn + j * 8 < N) dmma(acc[i][j], af[i], bf[j]);
        }
    }
    // fragment (g, 2 tg + {0,1}) of each 8 x 8 tile
    double *__restrict__ C = pr.C;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + wm + i * 8 + g;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + wn + j * 8 + 2 * tg;
            if (gn < N) C[gemm_col(pr, gn) + gm] = acc[i][j][0];
            if (gn + 1 < N) C[gemm_col(pr, gn + 1) + gm] = acc[i][j][1];
        }
    }
}

// Small blocks (merges whose blocks are at most 64 x 64): one warp per 32 x
// 32 output tile, four independent tiles (of any problems) per CTA.  The
// fragments are loaded straight from global memory (L1/L2), one K step of 4
// ahead of the MMAs, so a tile costs its loads' latency once instead of a
// shared-memory round trip per K block, and the warp's register budget
// (<= 128) keeps four CTAs of four warps per SM in flight.  Fragments wholly
// outside the block are neither loaded nor multiplied (warp-uniform).
constexpr int SW_WARPS = 4;
constexpr int kSmallRows = 64, kSmallCols = 64;   // largest blocks served by k_gemm64_warp

__global__ void __launch_bounds__(32 * SW_WARPS, 4) k_gemm64_warp(const GemmProb *__restrict__ probs, int nprobs,
                                                                   int tilesM, int tilesN) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * SW_WARPS + (threadIdx.x >> 5);
    const int tiles = tilesM * tilesN;
    const long long p = gw / tiles;
    if (p >= nprobs) return;
    const GemmProb pr = probs[p];
    const int t = (int)(gw % tiles);
    const int m0 = (t / tilesN) * 32, n0 = (t % tilesN) * 32;
    const int M = pr.M, N = pr.N, K = pr.K, lda = pr.lda, ldb = pr.ldb;
    if (m0 >= M || n0 >= N) return;
    const int fi = min(4, (M - m0 + 7) >> 3), fj = min(4, (N - n0 + 7) >> 3);   // live fragment rows / columns
    const int g = lane >> 2, tg = lane & 3;
    const double *__restrict__ A = pr.A;
    const double *__restrict__ B = pr.B;
    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
    // fragments of K step k: A (row m0 + 8 i + g, column k + tg), B (row k + tg, column n0 + 8 j + g)
    auto ldf = [&](int k, double (&af)[4], double (&bf)[4]) {
        const int kk = k + tg;
        const bool kok = kk < K;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = m0 + 8 * i + g;
            af[i] = (i < fi && kok && row < M) ? A[(size_t)kk * lda + row] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + 8 * j + g;
            bf[j] = (j < fj && kok && col < N) ? B[(size_t)col * ldb + kk] : 0.0;
        }
    };
    auto mul = [&](const double (&af)[4], const double (&bf)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i < fi && j < fj) dmma(acc[i][j], af[i], bf[j]);
    };
    double a0[4], b0[4], a1[4], b1[4];
    ldf(0, a0, b0);
    for (int k = 0; k < K; k += 8) {
        if (k + 4 < K) ldf(k + 4, a1, b1);
        mul(a0, b0);
        if (k + 4 >= K) break;
        if (k + 8 < K) ldf(k + 8, a0, b0);
        mul(a1, b1);
    }
    // fragment (g, 2 tg + {0,1}) of each 8 x 8 tile; output columns through the column map
    double *__restrict__ C = pr.C;
    size_t col0[4], col1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gn = n0 + 8 * j + 2 * tg;
        col0[j] = (j < fj && gn < N) ? gemm_col(pr, gn) : 0;
        col1[j] = (j < fj && gn + 1 < N) ? gemm_col(pr, gn + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + 8 * i + g;
        if (i >= fi || gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + 8 * j + 2 * tg;
            if (j >= fj) continue;
            if (gn < N) C[col0[j] + gm] = acc[i][j][0];
            if (gn + 1 < N) C[col1[j] + gm] = acc[i][j][1];
        }
    }
}

#endif  // BDC_FP32

}  // namespace

cudaError_t launch_gemm64(const GemmProb *probs, int nprobs, int mmax_rows, int nmax_cols, cudaStream_t st) {
    if (nprobs <= 0 || mmax_rows <= 0 || nmax_cols <= 0) return cudaSuccess;
#ifdef BDC_FP32
    const int bm = BM, bn = BN;
#else
    if (mmax_rows <= kSmallRows && nmax_cols <= kSmallCols) {
        const int tm = (mmax_rows + 31) / 32, tn = (nmax_cols + 31) / 32;
        const long long warps = (long long)nprobs * tm * tn;
        k_gemm64_warp<<<(unsigned)((warps + SW_WARPS - 1) / SW_WARPS), 32 * SW_WARPS, 0, st>>>(probs, nprobs, tm, tn);
        return cudaGetLastError();
    }
    // 32-row / 32-column tiles when the problems are that small
    const int wm = mmax_rows <= 32 ? 1 : 2, wn = nmax_cols <= 32 ? 1 : 2;
    const int bm = 32 * wm, bn = 32 * wn;
#endif
    const int tilesN = (nmax_cols + bn - 1) / bn, tilesM = (mmax_rows + bm - 1) / bm;
    for (int p0 = 0; p0 < nprobs; p0 += 65535) {
        const int np = (nprobs - p0 < 65535) ? nprobs - p0 : 65535;
        dim3 grid((unsigned)tilesN * tilesM, np);
#ifdef BDC_FP32
        k_gemm32<<<grid, 256, 0, st>>>(probs + p0, tilesN);
#else
        if (wm == 1 && wn == 1) k_gemm64<1, 1><<<grid, 32, 0, st>>>(probs + p0, tilesN);
        else if (wm == 1) k_gemm64<1, 2><<<grid, 64, 0, st>>>(probs + p0, tilesN);
        else if (wn == 1) k_gemm64<2, 1><<<grid, 64, 0, st>>>(probs + p0, tilesN);
        else k_gemm64<2, 2><<<grid, 128, 0, st>>>(probs + p0, tilesN);
#endif
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace BDC_NS
