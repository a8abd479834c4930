// Mixed-precision merge products of Eq. (bdc-Mv2Bv-u-vt) on tcgen05 tensor
// cores (sm_103a): C = A B with FP64 A (M x K), B (K x N), C, column-major.
//
// BDC_MIXED_EXACT (error-free slicing, after Ozaki, Ogita, Oishi and Rump):
//   every row r of A is scaled by 2^-E_r (|A_rk| 2^-E_r <= 1/2) and written as
//   S balanced base-256 digits n_1..n_S (|n_s| <= 128, value sum n_s 2^-8s),
//   every column c of B likewise with 2^-F_c.  Slice s is stored in BF16 as
//   n_s 2^-8(s-1) (exact: 8 significant bits).  The products of slice pairs
//   (i, j) with i + j <= S + 1 (1-based) are summed on the tensor cores in
//   FP32.  The tensor core truncates when it aligns the addends of an
//   accumulation, so an FP32 accumulator is only trusted where every partial
//   sum is an integer multiple of its group's unit 2^-8g below 2^22 (then
//   nothing is cut): groups g = i + j - 2 <= 4 accumulate in such short K
//   chunks and are drained into integer registers; the groups g >= 5 (weight
//   <= 2^-40 of the result) are restarted every 32 of K and summed in FP32
//   registers.  Relative error about 2^-(8S-2) of |A_r| |B_c| (S = 6:
//   ~1.4e-14); see MODE_E / MODE_L below.
// BDC_MIXED_BF16X3: A = hi + lo, B = hi + lo elementwise in BF16 and
//   hi*hi + hi*lo + lo*hi accumulated in FP32 (~1e-5 relative; reported).
//
// Data path per product (several products per launch):
//   k_slice_a : 32 rows per CTA, two passes over K through shared memory
//               (row maxima, then integer digit extraction), row-major
//               K-contiguous BF16 slices [slice][row][Kld] + exponents E.
//   k_slice_b : 8 or 32 lanes per column (B is K-contiguous), same digits + F.
//   k_mma     : persistent, one CTA per SM over the list of non-empty
//               128 x 128 tiles; K staged 32 at a time by TMA (3-D box
//               32 x 128 x slices, 64-byte swizzle) into a ring of 2-4 stages
//               (the exact-group kernel loads slices 1..4 only); warp 0
//               issues TMA, warp 1 allocates TMEM (512 columns) and one lane
//               issues tcgen05.mma kind::f16 (BF16 x BF16 -> FP32), warps
//               2-17 (4 per TMEM lane quarter, 32 columns each) drain and
//               store.  Ring stages and accumulator chunks are
//               counted across tiles, so loads and MMAs of the next tile
//               overlap the current tile's conversion and stores.  Every
//               mbarrier wait is bounded (2 s of %globaltimer); a timeout
//               sets an error word and unwinds.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "bdc_internal.cuh"

namespace bdc {

struct MixProb {
    int a_row0;   // first row of the product in the A slice array
    int b_col0;   // first column in the B slice array
    int tile0;    // first tile of the product in the launch grid
    int tilesN;   // tiles along N (for the host-known bound Nmax)
    int Mmax, Nmax;
    int pad0, pad1;
};

namespace {

constexpr int TM = 128, TK = 32, TN_MAX = 128;
constexpr int TNX = 128;   // tile width along N of the MMA kernels
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr int CPT = TN_MAX * 4 / EPI_WARPS;      // accumulator columns per epilogue thread (32)
constexpr unsigned long long kDrainNs = 2000000000ull;   // bounded drains of in-flight work: 2 s

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; returns false (and flags err) after wait_ns nanoseconds
// (2 s unless the BDC_TEST_WAIT_NS hook shortens it)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, volatile int *abort_flag,
                                          unsigned long long wait_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > wait_ns) {
            atomicCAS(err, 0, 1);
            *abort_flag = 1;
            return false;
        }
    }
}
// bounded wait that ignores the abort flag: a role that stopped early still
// lets its own asynchronous copies / MMAs land before the CTA exits (always
// the full 2 s: the test hook never shortens it)
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > kDrainNs) return;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand in shared memory, 64-byte swizzle: rows of 64 B, 8-row
// groups 512 B apart (SBO), start address advanced by 32 B per K step of 16.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
           (4ull << 61);
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ double pow2(int e) {   // 2^e for -1022 <= e <= 1023
    return __longlong_as_double((long long)(e + 1023) << 52);
}
__device__ __forceinline__ double ldexp_safe(double x, int e) {
    if (e > 1000) return x * pow2(1000) * pow2(e - 1000);
    if (e < -1000) return x * pow2(-1000) * pow2(e + 1000);
    return x * pow2(e);
}

// v 2^e rounded to nearest (ties to even) as an FP64 value, built with
// integer operations only (GB300's FP64 pipe is 1.6 op/clk/SM, the integer
// pipes are far wider); falls back to FP64 arithmetic when the result
// leaves the normal range
__device__ __forceinline__ double i64_ldexp(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    const unsigned long long m = a << lz;            // leading one at bit 63
    unsigned long long mant = m >> 11;               // 53 bits with the leading one
    const unsigned long long rest = m & 0x7FFull;
    if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) mant += 1ull;
    int ex = 63 - lz + e;                            // unbiased exponent of the result
    if (mant >> 53) { mant >>= 1; ex += 1; }         // rounding carried into bit 53
    if (ex < -1022 || ex > 1023) return ldexp_safe((double)v, e);
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) |
                                            (mant & 0x000FFFFFFFFFFFFFull)));
}

// x 2^e exactly for an FP32 value x (integer operations; FP64 fallback
// outside the normal range and for subnormal x)
__device__ __forceinline__ double f32_ldexp(float x, int e) {
    const unsigned int b = __float_as_uint(x);
    const int ef = (int)((b >> 23) & 0xFF);
    if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
    const int ex = ef - 127 + e;
    if (ef == 0 || ef == 0xFF || ex < -1022 || ex > 1023) return ldexp_safe((double)x, e);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// --------------------------------------------------------------- slicing
// exponent E with 2^E >= 2 max|x| > 2^(E-1)  (0 for an all-zero set)
__device__ __forceinline__ int scale_exp(unsigned long long maxbits) {
    if (maxbits == 0) return 0;
    const int ef = (int)(maxbits >> 52);
    if (ef == 0) return -1022 + 2;               // subnormal maximum
    return ef - 1023 + 2;
}

// balanced base-256 digits of round(x 2^(8S - E)): slices n_1..n_S, |n_s| <= 128
template <int S>
__device__ __forceinline__ void digits(double x, int E, int (&n)[S]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7FF);
    long long X = 0;
    if (ef != 0) {
        const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
        const int shift = ef - 1075 - E + 8 * S;   // X = mant * 2^shift
        if (shift >= 0) X = mant << shift;
        else if (shift > -63) X = (mant + (1ll << (-shift - 1))) >> (-shift);
        if (b >> 63) X = -X;
    }
    // balanced base-256 digits from the bytes of X (two's complement), least
    // significant first, on 32-bit words: a byte of 128 or more becomes
    // byte - 256 and carries one into the next
    const unsigned lo = (unsigned)X, hi = (unsigned)((unsigned long long)X >> 32);
    int c = 0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const unsigned w = (k < 4) ? lo : hi;
        const int t = (int)((w >> (8 * (k & 3))) & 255u) + c;
        c = (t + 128) >> 8;
        n[S - 1 - k] = t - (c << 8);
    }
    // what is left above the S digits joins the top one (only when |x| 2^-E = 1/2)
    const int rem = (8 * S >= 32) ? ((int)hi >> (8 * S >= 32 ? 8 * S - 32 : 0)) : (int)(X >> (8 * S < 64 ? 8 * S : 0));
    n[0] += (rem + c) << 8;
}

// n 2^-8s (s = 0-based slice, |n| <= 256) in BF16 without conversion
// instructions: n becomes an FP32 value exactly by the 1.5 2^23 offset trick
// (one FP32 add), scales by 2^-8s (one multiply), and having at most 8
// significant bits its BF16 pattern is the top half of the FP32 pattern
__device__ __forceinline__ __nv_bfloat16 slice_bf16(int n, int s) {
    const float f = (__int_as_float(0x4B400000 + n) - 12582912.0f) * __uint_as_float((uint32_t)(127 - 8 * s) << 23);
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// A operand: 32 rows per CTA (256 threads), A column-major; grid (row blocks
// of the largest product, products from p0), blocks past their product's
// rows exit
template <int S, bool EXACT>
__global__ void __launch_bounds__(256) k_slice_a(const GemmProb *__restrict__ probs, const MixProb *__restrict__ mix,
                                                int p0, __nv_bfloat16 *__restrict__ As, int *__restrict__ Ea,
                                                int rowsA, int Kld) {
    __shared__ unsigned long long smax[8][33];
    __shared__ __nv_bfloat16 tile[S][32][72];
    const int p = p0 + blockIdx.y;
    const GemmProb pr = probs[p];
    const MixProb mx = mix[p];
    const int r0 = blockIdx.x * 32;
    if (r0 >= mx.Mmax || pr.M <= 0 || pr.N <= 0) return;   // empty products have no tiles to feed
    const int tr = threadIdx.x & 31, tc = threadIdx.x >> 5;   // row within block, column lane
    const int row = r0 + tr;
    const bool rowok = row < pr.M;
    const int K = pr.K;
    int E = 0;
    if (EXACT) {
        unsigned long long mx2 = 0;
        if (rowok)
            #pragma unroll 4
            for (int k = tc; k < K; k += 8) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(pr.A[(size_t)k * pr.lda + row]) &
                                             0x7FFFFFFFFFFFFFFFull;
                mx2 = b > mx2 ? b : mx2;
            }
        smax[tc][tr] = mx2;
        __syncthreads();
        unsigned long long m = 0;
        for (int q = 0; q < 8; ++q) m = smax[q][tr] > m ? smax[q][tr] : m;
        E = scale_exp(m);
        if (tc == 0 && row < mx.Mmax) Ea[mx.a_row0 + row] = rowok ? E : 0;
    }
    // second pass: digits, staged through shared memory so rows are written
    // K-contiguous; only up to the last 32-wide stage the MMA reads
    const int Kend = min(Kld, (K + TK - 1) / TK * TK);
    for (int k0 = 0; k0 < Kend; k0 += 64) {
        for (int kk = tc; kk < 64; kk += 8) {
            const int k = k0 + kk;
            const double x = (rowok && k < K) ? pr.A[(size_t)k * pr.lda + row] : 0.0;
            if (EXACT) {
                int n[S];
                digits<S>(x, E, n);
#pragma unroll
                for (int s = 0; s < S; ++s) tile[s][tr][kk] = slice_bf16(n[s], s);
            } else {
                const float xf = (float)x;
                const __nv_bfloat16 h = __float2bfloat16_rn(xf);
                tile[0][tr][kk] = h;
                tile[1][tr][kk] = __float2bfloat16_rn(xf - __bfloat162float(h));
            }
        }
        __syncthreads();
        // 32 rows x 64 columns x S slices out, 8 columns (16 B) per thread-store
        for (int idx = threadIdx.x; idx < S * 32 * 8; idx += 256) {
            const int s = idx / 256, rem = idx % 256, rr = rem >> 3, seg = rem & 7;
            const int grow = r0 + rr;
            if (grow < mx.Mmax && k0 + seg * 8 < Kend) {
                const uint4 v = *reinterpret_cast<const uint4 *>(&tile[s][rr][seg * 8]);
                *reinterpret_cast<uint4 *>(As + ((size_t)s * rowsA + mx.a_row0 + grow) * Kld + k0 + seg * 8) = v;
            }
        }
        __syncthreads();
    }
}

constexpr int kSliceRegs = 16;   // entries per lane held in registers by the one-pass B slicing

// B operand: LANES lanes per column (column-major B is K-contiguous),
// 32 / LANES columns per warp; grid (columns of the host bound of the
// largest product / (256 / LANES), products from p0).  K is a merge's
// survivor count: eight lanes per column for the small merges (a few
// dozen K, where a whole warp per column would mostly wait on its loads),
// a warp per column for the large ones.  Only the columns the MMA tiles
// read are written: those below N, and zeros up to N rounded up to the
// tile width; lanes past them exit (N, the survivor count, is known only on
// the device and is often far below the host bound).  Columns of up to
// LANES kSliceRegs entries are read once into registers; longer ones in two
// passes (maximum, then digits).
template <int S, bool EXACT, int LANES>
__global__ void __launch_bounds__(256) k_slice_b(const GemmProb *__restrict__ probs, const MixProb *__restrict__ mix,
                                                int p0, __nv_bfloat16 *__restrict__ Bs, int *__restrict__ Fb, int colsB,
                                                int Kld) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) / LANES, l = threadIdx.x & (LANES - 1);
    const unsigned gmask = (LANES == 32) ? 0xffffffffu : ((1u << (LANES & 31)) - 1) << (threadIdx.x & (32 - LANES));
    const int p = p0 + blockIdx.y;
    const GemmProb pr = probs[p];
    const MixProb mx = mix[p];
    // whole lane groups leave together; empty products have no tiles to feed
    if (c >= mx.Nmax || c >= (pr.N + TNX - 1) / TNX * TNX || pr.M <= 0) return;
    const bool colok = c < pr.N;
    const int K = pr.K;
    const double *col = pr.B + (size_t)c * pr.ldb;
    __nv_bfloat16 *dst = Bs + (size_t)(mx.b_col0 + c) * Kld;
    if (K <= LANES * kSliceRegs) {
        // one pass: the column's entries held in registers (every load issued
        // before the maximum is needed); K <= LANES kSliceRegs covers Kend
        double xv[kSliceRegs];
        unsigned long long m = 0;
#pragma unroll
        for (int q = 0; q < kSliceRegs; ++q) {
            const int k = l + q * LANES;
            xv[q] = (colok && k < K) ? col[k] : 0.0;
            const unsigned long long b = (unsigned long long)__double_as_longlong(xv[q]) & 0x7FFFFFFFFFFFFFFFull;
            m = b > m ? b : m;
        }
        int F = 0;
        if (EXACT) {
            for (int o = LANES / 2; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(gmask, m, o);
                m = y > m ? y : m;
            }
            F = scale_exp(m);
            if (l == 0) Fb[mx.b_col0 + c] = colok ? F : 0;
        }
        const int Kend = min(Kld, (K + TK - 1) / TK * TK);
#pragma unroll
        for (int q = 0; q < kSliceRegs; ++q) {
            const int k = l + q * LANES;
            if (k >= Kend) break;
            if (EXACT) {
                int n[S];
                digits<S>(xv[q], F, n);
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2) dst[(size_t)s2 * colsB * Kld + k] = slice_bf16(n[s2], s2);
            } else {
                const float xf = (float)xv[q];
                const __nv_bfloat16 h = __float2bfloat16_rn(xf);
                dst[k] = h;
                dst[(size_t)colsB * Kld + k] = __float2bfloat16_rn(xf - __bfloat162float(h));
            }
        }
        return;
    }
    int F = 0;
    if (EXACT) {
        unsigned long long m = 0;
        if (colok)
            #pragma unroll 4
            for (int k = l; k < K; k += LANES) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(col[k]) & 0x7FFFFFFFFFFFFFFFull;
                m = b > m ? b : m;
            }
        for (int o = LANES / 2; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(gmask, m, o);
            m = y > m ? y : m;
        }
        F = scale_exp(m);
        if (l == 0) Fb[mx.b_col0 + c] = colok ? F : 0;
    }
    const int Kend = min(Kld, (K + TK - 1) / TK * TK);
    #pragma unroll 4
    for (int k = l; k < Kend; k += LANES) {
        const double x = (colok && k < K) ? col[k] : 0.0;
        if (EXACT) {
            int n[S];
            digits<S>(x, F, n);
#pragma unroll
            for (int s = 0; s < S; ++s) dst[(size_t)s * colsB * Kld + k] = slice_bf16(n[s], s);
        } else {
            const float xf = (float)x;
            const __nv_bfloat16 h = __float2bfloat16_rn(xf);
            dst[k] = h;
            dst[(size_t)colsB * Kld + k] = __float2bfloat16_rn(xf - __bfloat162float(h));
        }
    }
}

// ------------------------------------------------------------- MMA kernels
// Three kernel modes share the TMA producer, the 128 x 128 tile and four
// 128-column TMEM accumulators at columns 0, 128, 256, 384:
//   MODE_E   exact groups g = 0..3 (10 slice pairs), K chunks of 64 split in
//            two staggered sets, set A = {g0, g3} over stages {0,1},{2,3},...
//            and set B = {g1, g2} over {0},{1,2},{3,4},...; each set drains
//            into the 64-bit integers L (unit 2^-24) while the other set's
//            MMAs run.  Writes C = 2^(E+F-40) L.
//   MODE_L   the remaining groups g >= 4: group 4 in its own accumulator,
//            exact per 32-wide stage (|I_4| <= 5 * 2^14 * 32 < 2^22), the rest
//            (weight <= 2^-40) in a second one, both restarted every stage and
//            summed over the stages in FP32 registers (round to nearest); two
//            accumulator buffers alternate per stage.  Adds 2^(E+F-16) SL to C.
//   MODE_X3  BF16x3: (hi, lo) pairs (0,0), (0,1), (1,0) in one accumulator
//            over the whole K.  Writes C.
enum { MODE_E = 0, MODE_L = 1, MODE_X3 = 2 };

// Slices loaded per stage (MODE_E multiplies slices 1..4 only), bytes per
// stage, and ring depth: as many stages as fit in ~200 KB of shared memory,
// 2 to 4 (a deeper ring hides more TMA latency; the operand traffic per
// MMA is what bounds these small-K products)
template <int S, int MODE>
__host__ __device__ constexpr int stage_slices() { return (MODE == MODE_E && S > 4) ? 4 : S; }
template <int S, int MODE>
__host__ __device__ constexpr int stage_bytes() { return 2 * stage_slices<S, MODE>() * TM * TK * 2; }
template <int S, int MODE>
__host__ __device__ constexpr int stage_count() {
    return (200 * 1024) / stage_bytes<S, MODE>() < 2 ? 2
           : (200 * 1024) / stage_bytes<S, MODE>() > 4 ? 4
                                                         : (200 * 1024) / stage_bytes<S, MODE>();
}

template <int S, int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_mma(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB,
                                                     const GemmProb *__restrict__ probs,
                                                     const MixProb *__restrict__ mix, int nprobs,
                                                     const int *__restrict__ Ea, const int *__restrict__ Fb,
                                                     int *__restrict__ err, const int2 *__restrict__ tiles,
                                                     const int *__restrict__ ntiles, unsigned long long wait_ns,
                                                     int stall) {
    constexpr int TILE = TM * TK * 2;                 // one 128 x 32 BF16 slice tile (A or B)
    constexpr int SL = stage_slices<S, MODE>();       // slices per operand in a stage
    constexpr int STAGE_BYTES = stage_bytes<S, MODE>();
    constexpr int NSTAGE = stage_count<S, MODE>();
    // kind::f16 instruction descriptor: D = F32, A = B = BF16, K-major,
    // N/8 in bits 17-22, M/16 in bits 24-28
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TNX >> 3) << 17) |
                               ((uint32_t)(TM >> 4) << 24);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + NSTAGE * STAGE_BYTES);
    uint64_t *empty = full + NSTAGE;
    uint64_t *accfull = empty + NSTAGE;      // [2]: set A / set B (MODE_E) or buffer 0 / 1 (MODE_L)
    uint64_t *accempty = accfull + 2;        // [2]
    uint32_t *tmem_slot = (uint32_t *)(accempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    (void)nprobs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent: the CTA walks the device-built list of non-empty tiles
    // (sizes after deflation), so no CTA is launched for an empty tile.  The
    // barriers live for the whole kernel and every role walks the same tiles
    // with running stage / chunk counters (phases continue across tiles):
    // the producer loads the next tile and the MMAs start on it while the
    // epilogue still converts and stores the current one.
    const int count = *ntiles;
    if ((int)blockIdx.x >= count) return;
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int i = 0; i < NSTAGE; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&accfull[i], 1); mbar_init(&accempty[i], 32 * EPI_WARPS); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int G = 0;                                  // stages loaded so far (all tiles)
            bool ok = true;
            // the next tile's coordinates are loaded while this one streams
            int2 tcn = tiles[blockIdx.x];
            MixProb mxn = mix[tcn.x];
            int Kn = probs[tcn.x].K;
            for (int ti = blockIdx.x; ti < count && ok; ti += gridDim.x) {
                const int2 tc = tcn;
                const MixProb mx = mxn;
                const int m0 = (tc.y >> 16) * TM, n0 = (tc.y & 0xffff) * TNX;
                const int nk = (Kn + TK - 1) / TK;
                if (ti + (int)gridDim.x < count) {
                    tcn = tiles[ti + gridDim.x];
                    mxn = mix[tcn.x];
                    Kn = probs[tcn.x].K;
                }
                for (int s = 0; s < nk; ++s, ++G) {
                    const int buf = G % NSTAGE;
                    if (G >= NSTAGE && !mbar_wait(&empty[buf], ((G / NSTAGE) - 1) & 1, err, abort_flag, wait_ns)) {
                        ok = false;
                        break;
                    }
                    // test hook (BDC_TEST_STALL): CTA 0 never loads its first stage,
                    // so the MMA issuer's wait on that stage's barrier must give up
                    if (stall && blockIdx.x == 0 && G == 0) continue;
                    mbar_expect_tx(&full[buf], STAGE_BYTES);
                    const uint32_t dstA = smem_u32(smem + buf * STAGE_BYTES);
                    tma_load_3d(dstA, &tmA, s * TK, mx.a_row0 + m0, 0, &full[buf]);
                    tma_load_3d(dstA + SL * TILE, &tmB, s * TK, mx.b_col0 + n0, 0, &full[buf]);
                }
            }
            // copies still in flight (after an abort) land before the CTA exits
            // (a stage skipped by the test hook has none)
            for (int g = (G > NSTAGE ? G - NSTAGE : 0); g < G; ++g)
                if (!(stall && blockIdx.x == 0 && g == 0)) mbar_drain(&full[g % NSTAGE], (g / NSTAGE) & 1);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (one lane)
        if (lane == 0) {
            // descriptor of the ring's first tile; a slice tile's descriptor adds
            // its byte offset / 16 to the 14-bit address field (shared memory
            // addresses stay below 256 KB, so the field never carries), and the
            // K step of 16 (32 B) adds 2
            const uint64_t d0 = sdesc(smem_u32(smem));
            int G = 0;                                  // stages consumed so far (all tiles)
            int nA = 0, nB = 0;                         // accumulator chunks committed: set A / set B
                                                        // (MODE_E), tiles (MODE_X3)
            bool ok = true;
            // a fresh chunk of an accumulator set waits until the epilogue has
            // drained the set's previous chunk
            auto wait_drained = [&](int set, int done) {
                if (done > 0 && !mbar_wait(&accempty[set], (done - 1) & 1, err, abort_flag, wait_ns)) ok = false;
                fence_after();
            };
            int Kn = probs[tiles[blockIdx.x].x].K;     // the next tile's K, loaded ahead
            for (int ti = blockIdx.x; ti < count && ok; ti += gridDim.x) {
                const int nk = (Kn + TK - 1) / TK;
                if (ti + (int)gridDim.x < count) Kn = probs[tiles[ti + gridDim.x].x].K;
                for (int s = 0; s < nk && ok; ++s, ++G) {
                    const int buf = G % NSTAGE;
                    if (!mbar_wait(&full[buf], (G / NSTAGE) & 1, err, abort_flag, wait_ns)) { ok = false; break; }
                    fence_after();
                    // operand "addresses" below are (buffer, tile index, K step) handles
                    auto mma = [&](uint32_t col, int ia, int ib, int kk, uint32_t acc) {
                        const uint64_t a = d0 + (uint64_t)((buf * STAGE_BYTES + ia * TILE) >> 4) + 2 * kk;
                        const uint64_t b = d0 + (uint64_t)((buf * STAGE_BYTES + (SL + ib) * TILE) >> 4) + 2 * kk;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                            "p;\n}\n" ::"r"(tmem + col),
                            "l"(a), "l"(b), "r"(idesc), "r"(acc)
                            : "memory");
                    };
                    if constexpr (MODE == MODE_X3) {
                        if (s == 0) wait_drained(0, nA);
                        if (!ok) break;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            mma(0, 0, 0, kk, (s == 0 && kk == 0) ? 0u : 1u);
                            mma(0, 0, 1, kk, 1u);
                            mma(0, 1, 0, kk, 1u);
                        }
                        umma_commit(&empty[buf]);
                        if (s == nk - 1) { umma_commit(&accfull[0]); ++nA; }
                    } else if constexpr (MODE == MODE_L) {
                        const int b = G & 1;                   // accumulator buffer of this stage
                        if (G >= 2) {
                            if (!mbar_wait(&accempty[b], ((G >> 1) - 1) & 1, err, abort_flag, wait_ns)) { ok = false; break; }
                            fence_after();
                        }
                        const uint32_t c4 = 256 * b, cl = 256 * b + 128;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                            for (int i = 0; i <= 4; ++i)
                                if (i < S && 4 - i < S)
                                    mma(c4, i, 4 - i, kk, (kk == 0 && i == 0) ? 0u : 1u);
                            bool first = true;
#pragma unroll
                            for (int g = 5; g <= S - 1; ++g)
#pragma unroll
                                for (int i = 0; i <= g; ++i) {
                                    const int j = g - i;
                                    if (i >= S || j >= S) continue;
                                    mma(cl, i, j, kk, (kk == 0 && first) ? 0u : 1u);
                                    first = false;
                                }
                        }
                        umma_commit(&empty[buf]);
                        umma_commit(&accfull[b]);
                    } else {
                        // MODE_E: set A = {g0 @0, g3 @384}, set B = {g1 @128, g2 @256}
                        auto issueA = [&](bool fresh) {
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                mma(0, 0, 0, kk, (fresh && kk == 0) ? 0u : 1u);
#pragma unroll
                                for (int i = 0; i <= 3; ++i) mma(384, i, 3 - i, kk, (fresh && kk == 0 && i == 0) ? 0u : 1u);
                            }
                        };
                        auto issueB = [&](bool fresh) {
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                                for (int i = 0; i <= 1; ++i) mma(128, i, 1 - i, kk, (fresh && kk == 0 && i == 0) ? 0u : 1u);
#pragma unroll
                                for (int i = 0; i <= 2; ++i) mma(256, i, 2 - i, kk, (fresh && kk == 0 && i == 0) ? 0u : 1u);
                            }
                        };
                        bool issued = false;
                        if ((s & 1) == 0) {
                            if (s == 0) wait_drained(1, nB);   // set B starts a chunk at a tile's first stage
                            if (ok) { issueB(s == 0); issued = true; }   // and continues at the other even stages
                            if (ok) wait_drained(0, nA);       // set A starts a chunk
                            if (ok) issueA(true);
                        } else {
                            issueA(false);
                            issued = true;
                            wait_drained(1, nB);
                            if (ok) issueB(true);
                        }
                        if (!ok) {
                            // stopped part-way: the MMAs already issued still report to the
                            // stage barrier, which the drain below waits for
                            if (issued) { umma_commit(&empty[buf]); ++G; }
                            break;
                        }
                        umma_commit(&empty[buf]);
                        if (((s & 1) == 0) || s == nk - 1) { umma_commit(&accfull[1]); ++nB; }   // set B chunk ends
                        if (((s & 1) == 1) || s == nk - 1) { umma_commit(&accfull[0]); ++nA; }   // set A chunk ends
                    }
                }
            }
            // every MMA issued has completed (its stage's commit arrived) before
            // the CTA frees TMEM and exits
            for (int g = (G > NSTAGE ? G - NSTAGE : 0); g < G; ++g) mbar_drain(&empty[g % NSTAGE], (g / NSTAGE) & 1);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        const int q = warp & 3;                    // TMEM lane quarter this warp may access
        const int part = (warp - 2) >> 2;          // column part (CPT columns)
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + CPT * part;
        bool ok = true;
        int cA = 0, cB = 0;                        // drains done: set A / set B (MODE_E), tiles (MODE_X3)
        int GL = 0;                                // stages drained (MODE_L)
        for (int ti = blockIdx.x; ti < count && ok; ti += gridDim.x) {
            const int2 tc = tiles[ti];
            const GemmProb pr = probs[tc.x];
            const MixProb mx = mix[tc.x];
            const int m0 = (tc.y >> 16) * TM, n0 = (tc.y & 0xffff) * TNX;
            const int nk = (pr.K + TK - 1) / TK;
            const int row = m0 + 32 * q + lane;
            const int c0 = n0 + CPT * part;
            const bool rowok = row < pr.M;
            const long long ldc = pr.ldc;
            // this warp's CPT columns: their exponents F and output columns
            // (slots), coalesced loads, handed to the final loop by shuffles
            // instead of one dependent global load per column
            int fbl[CPT / 32], cml[CPT / 32];
            auto column_tables = [&]() {
#pragma unroll
                for (int h2 = 0; h2 < CPT / 32; ++h2) {
                    const int col = c0 + 32 * h2 + lane;
                    const bool cok = col < pr.N;
                    fbl[h2] = (cok && MODE != MODE_X3) ? Fb[mx.b_col0 + col] : 0;
                    cml[h2] = cok ? (pr.cmap ? pr.cmap[col] : col) : 0;
                }
            };
            if constexpr (MODE == MODE_E) {
                // unsigned: the magic offsets wrap modulo 2^64 and cancel exactly at the end
                unsigned long long L[CPT];
#pragma unroll
                for (int i = 0; i < CPT; ++i) L[i] = 0;
                int tA = 0, tB = 0;                    // this tile's drains
                for (int s = 0; s < nk && ok; ++s) {
                    if (((s & 1) == 0) || s == nk - 1) {                // set B: g1, g2
                        if (!mbar_wait(&accfull[1], cB & 1, err, abort_flag, wait_ns)) { ok = false; break; }
                        fence_after();
#pragma unroll
                        for (int cb = 0; cb < CPT / 8; ++cb) {
                            float v1[8], v2[8];
                            tmem_ld8(tl + 128 + 8 * cb, v1);
                            tmem_ld8(tl + 256 + 8 * cb, v2);
                            tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                // raw magic bits b = I + 0x4B400000; the offsets are removed once at the end
                                const unsigned b1 = __float_as_uint(fmaf(v1[i], 256.0f, 12582912.0f));
                                const unsigned b2 = __float_as_uint(fmaf(v2[i], 65536.0f, 12582912.0f));
                                L[8 * cb + i] += ((unsigned long long)b1 << 16) + ((unsigned long long)b2 << 8);
                            }
                        }
                        fence_before();
                        mbar_arrive(&accempty[1]);
                        ++cB; ++tB;
                    }
                    if (((s & 1) == 1) || s == nk - 1) {                // set A: g0, g3
                        if (!mbar_wait(&accfull[0], cA & 1, err, abort_flag, wait_ns)) { ok = false; break; }
                        fence_after();
#pragma unroll
                        for (int cb = 0; cb < CPT / 8; ++cb) {
                            float v0[8], v3[8];
                            tmem_ld8(tl + 8 * cb, v0);
                            tmem_ld8(tl + 384 + 8 * cb, v3);
                            tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const unsigned b0 = __float_as_uint(fmaf(v0[i], 1.0f, 12582912.0f));
                                const unsigned b3 = __float_as_uint(fmaf(v3[i], 16777216.0f, 12582912.0f));
                                L[8 * cb + i] += ((unsigned long long)b0 << 24) + (unsigned long long)b3;
                            }
                        }
                        fence_before();
                        mbar_arrive(&accempty[0]);
                        ++cA; ++tA;
                    }
                }
                ok = __all_sync(0xffffffffu, ok);          // the shuffles below need the whole warp
                if (ok) {
                    // remove the magic offsets: every set-A drain added M (2^24 + 1),
                    // every set-B drain M (2^16 + 2^8), M = 0x4B400000
                    const unsigned long long M = 0x4B400000ull;
                    const unsigned long long corr = (unsigned long long)tA * M * ((1ull << 24) + 1) +
                                                    (unsigned long long)tB * M * ((1ull << 16) + (1ull << 8));
                    const int Er = rowok ? Ea[mx.a_row0 + row] : 0;
                    column_tables();
#pragma unroll
                    for (int cb = 0; cb < CPT / 8; ++cb) {
                        int F[8], cj[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = 8 * cb + i;
                            F[i] = __shfl_sync(0xffffffffu, fbl[k >> 5], k & 31);
                            cj[i] = __shfl_sync(0xffffffffu, cml[k >> 5], k & 31);
                        }
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = 8 * cb + i;
                            if (rowok && c0 + k < pr.N)
                                pr.C[cj[i] * ldc + row] = i64_ldexp((long long)(L[k] - corr), Er + F[i] - 40);
                        }
                    }
                }
            } else if constexpr (MODE == MODE_L) {
                // group 4 is exact per stage (and weighs <= 2^-32), groups >= 5 weigh
                // <= 2^-40: both are summed over the stages in FP32 registers
                float SL[CPT];
#pragma unroll
                for (int i = 0; i < CPT; ++i) SL[i] = 0.f;
                // the final read-modify-write of C waits on its loads while the
                // next tile's stages wait on this warp: pull this warp's 32 rows of
                // its CPT columns into L2 now (lane = column, 256 B each), while
                // the stages below accumulate
                const int Er = rowok ? Ea[mx.a_row0 + row] : 0;
                column_tables();
                {
                    const int rw0 = m0 + 32 * q;
#pragma unroll
                    for (int h2 = 0; h2 < CPT / 32; ++h2) {
                        const int col = c0 + 32 * h2 + lane;
                        if (col < pr.N && rw0 < pr.M) {
                            const double *pc = pr.C + (long long)cml[h2] * ldc + rw0;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pc));
                            if (rw0 + 16 < pr.M) asm volatile("prefetch.global.L2 [%0];" ::"l"(pc + 16));
                        }
                    }
                }
                for (int s = 0; s < nk; ++s, ++GL) {
                    const int b = GL & 1;
                    if (!mbar_wait(&accfull[b], (GL >> 1) & 1, err, abort_flag, wait_ns)) { ok = false; break; }
                    fence_after();
#pragma unroll
                    for (int cb = 0; cb < CPT / 8; ++cb) {
                        float v4[8], vl[8];
                        tmem_ld8(tl + 256 * b + 8 * cb, v4);
                        if (S > 5) tmem_ld8(tl + 256 * b + 128 + 8 * cb, vl);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            SL[8 * cb + i] += v4[i];
                            if (S > 5) SL[8 * cb + i] += vl[i];
                        }
                    }
                    fence_before();
                    mbar_arrive(&accempty[b]);
                }
                ok = __all_sync(0xffffffffu, ok);          // the shuffles below need the whole warp
                if (ok) {
                    // C += 2^(E+F-16) SL, 8 columns at a time: their loads of C are
                    // issued together
#pragma unroll
                    for (int cb = 0; cb < CPT / 8; ++cb) {
                        int F[8];
                        long long off[8];
                        double cv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = 8 * cb + i;
                            F[i] = __shfl_sync(0xffffffffu, fbl[k >> 5], k & 31);
                            off[i] = __shfl_sync(0xffffffffu, cml[k >> 5], k & 31) * ldc;
                            cv[i] = (rowok && c0 + k < pr.N) ? pr.C[off[i] + row] : 0.0;
                        }
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = 8 * cb + i;
                            if (rowok && c0 + k < pr.N) pr.C[off[i] + row] = cv[i] + f32_ldexp(SL[k], Er + F[i] - 16);
                        }
                    }
                }
            } else {
                if (!mbar_wait(&accfull[0], cA & 1, err, abort_flag, wait_ns)) ok = false;
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }   // the shuffles need the whole warp
                fence_after();
                column_tables();
#pragma unroll
                for (int cb = 0; cb < CPT / 16; ++cb) {
                    float v[16];
                    tmem_ld16(tl + 16 * cb, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int k = 16 * cb + i;
                        const long long off = __shfl_sync(0xffffffffu, cml[k >> 5], k & 31) * ldc;
                        if (rowok && c0 + k < pr.N) pr.C[off + row] = f32_ldexp(v[i], 0);
                    }
                }
                fence_before();
                mbar_arrive(&accempty[0]);
                ++cA;
            }
        }
        (void)cB;
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// list of the non-empty 128 x 128 tiles of every product (one CTA per
// product, sizes as deflated on the device); bands of 8 row blocks walk the
// column blocks together so that neighbouring tiles share operands in L2
__global__ void k_tile_list(const GemmProb *__restrict__ probs, const MixProb *__restrict__ mix,
                            int2 *__restrict__ tiles, int *__restrict__ ntiles) {
    const int p = blockIdx.x;
    const GemmProb pr = probs[p];
    const MixProb mx = mix[p];
    const int M = min(pr.M, mx.Mmax), N = min(pr.N, mx.Nmax);
    if (M <= 0 || N <= 0 || pr.K <= 0) return;
    const int tilesM = (M + TM - 1) / TM, tilesN = (N + TNX - 1) / TNX;
    const int cnt = tilesM * tilesN;
    __shared__ int base;
    if (threadIdx.x == 0) base = atomicAdd(ntiles, cnt);
    __syncthreads();
    constexpr int G = 8;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int band = t / (G * tilesN), in_band = t % (G * tilesN);
        const int bm0 = band * G, bsz = min(G, tilesM - bm0);
        const int mb = bm0 + in_band % bsz, nb = in_band / bsz;
        tiles[base + t] = make_int2(p, (mb << 16) | nb);
    }
}

// ------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 3-D map over [slice][row][Kld] BF16 (S slices) with a 32 x box_rows x
// box_slices box (slices 0 .. box_slices-1) and 64 B swizzle
bool make_map(CUtensorMap *m, void *base, int rows, int Kld, int S, int box_slices, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kld, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)Kld * 2, (cuuint64_t)rows * Kld * 2};
    cuuint32_t box[3] = {TK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t offA, offB, offE, offF, offErr, offMix, offTiles, total;
};

// tiles: capacity of the non-empty tile list (the no-deflation bound)
Layout layout(long long rowsA, long long colsB, int Kld, int S, int nprobs, long long tiles) {
    Layout L{};
    size_t o = 0;
    L.offA = o; o += align256((size_t)S * rowsA * Kld * 2);
    L.offB = o; o += align256((size_t)S * colsB * Kld * 2);
    L.offE = o; o += align256(sizeof(int) * (size_t)rowsA);
    L.offF = o; o += align256(sizeof(int) * (size_t)colsB);
    L.offErr = o; o += 256;                       // error word, tile count at +16
    L.offMix = o; o += align256(sizeof(MixProb) * (size_t)nprobs);
    L.offTiles = o; o += align256(sizeof(int2) * (size_t)tiles);
    L.total = o;
    return L;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

template <int S, bool EXACT>
cudaError_t run_mixed(const GemmProb *probs, int nprobs, const std::vector<MixProb> &hm, int rowsA, int colsB,
                      int Kld, char *scratch, const Layout &L, int *err, int phase, cudaStream_t st) {
    __nv_bfloat16 *As = (__nv_bfloat16 *)(scratch + L.offA);
    __nv_bfloat16 *Bs = (__nv_bfloat16 *)(scratch + L.offB);
    int *E = (int *)(scratch + L.offE), *F = (int *)(scratch + L.offF);
    MixProb *dmix = (MixProb *)(scratch + L.offMix);
    // largest row and column counts of one product (the slicing grids)
    int mrows = 1, ncols = 1, tiles = 0;
    for (int p = 0; p < nprobs; ++p) {
        mrows = std::max(mrows, hm[p].Mmax);
        ncols = std::max(ncols, hm[p].Nmax);
        tiles = hm[p].tile0 + ((hm[p].Mmax + TM - 1) / TM) * hm[p].tilesN;
    }
    if (hm.size() && hm[0].tilesN != (hm[0].Nmax + TNX - 1) / TNX) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (phase & MIXED_A) {   // the product table, then the A slices (W~ / Q~ blocks only)
        // small tables through pinned host memory: the capturing plan's own
        // blocks, else a shared ring (copies stay valid until the ring wraps)
        static std::mutex mu;
        static char *ring = nullptr;
        static size_t ring_off = 0;
        constexpr size_t kRing = 64ull << 20;
        const size_t need = sizeof(MixProb) * nprobs + 256;
        if (need > kRing) return cudaErrorInvalidValue;
        char *h = (char *)plan_pinned_alloc(need);
        if (!h) {
            std::lock_guard<std::mutex> lk(mu);
            if (!ring && cudaMallocHost((void **)&ring, kRing) != cudaSuccess) return cudaErrorMemoryAllocation;
            if (ring_off + need > kRing) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                cudaStreamIsCapturing(st, &cs);
                if (cs == cudaStreamCaptureStatusNone) cudaDeviceSynchronize();
                ring_off = 0;
            }
            h = ring + ring_off;
            ring_off += (need + 255) & ~(size_t)255;
        }
        char *hp = h;
        std::memcpy(hp, hm.data(), sizeof(MixProb) * nprobs);
        e = cudaMemcpyAsync(dmix, hp, sizeof(MixProb) * nprobs, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;

        {   // A operand slicing
            StageScope slice_scope(st, BDC_STAGE_SLICE, 1, 0.0);
            for (int p0 = 0; p0 < nprobs; p0 += 65535) {
                const int np = std::min(nprobs - p0, 65535);
                k_slice_a<S, EXACT><<<dim3((mrows + 31) / 32, np), 256, 0, st>>>(probs, dmix, p0, As, E, rowsA, Kld);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
    }
    if (!(phase & MIXED_B)) return cudaSuccess;

    int *ntiles = (int *)(scratch + L.offErr);
    int2 *tlist = (int2 *)(scratch + L.offTiles);
    if ((e = cudaMemsetAsync(ntiles, 0, sizeof(int), st)) != cudaSuccess) return e;   // tile count

    {   // B operand slicing
        StageScope slice_scope(st, BDC_STAGE_SLICE, 1, 0.0);
        for (int p0 = 0; p0 < nprobs; p0 += 65535) {
            const int np = std::min(nprobs - p0, 65535);
            if (ncols <= 128)
                k_slice_b<S, EXACT, 8><<<dim3((ncols + 31) / 32, np), 256, 0, st>>>(probs, dmix, p0, Bs, F, colsB, Kld);
            else
                k_slice_b<S, EXACT, 32><<<dim3((ncols + 7) / 8, np), 256, 0, st>>>(probs, dmix, p0, Bs, F, colsB, Kld);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }

    // tensor maps: boxes of all S slices, and (exact mode) of the first
    // stage_slices<S, MODE_E> slices for the exact-group kernel
    constexpr int SE = stage_slices<S, MODE_E>();
    CUtensorMap ma, mb, mae, mbe;
    if (!make_map(&ma, As, rowsA, Kld, S, S, TM) || !make_map(&mb, Bs, colsB, Kld, S, S, TNX))
        return cudaErrorInvalidValue;
    if (EXACT && (!make_map(&mae, As, rowsA, Kld, S, SE, TM) || !make_map(&mbe, Bs, colsB, Kld, S, SE, TNX)))
        return cudaErrorInvalidValue;
    auto smem_of = [](int stage, int count) { return (size_t)stage * count + 1024 + 256; };
    const size_t smemE = smem_of(stage_bytes<S, MODE_E>(), stage_count<S, MODE_E>());
    const size_t smemL = smem_of(stage_bytes<S, MODE_L>(), stage_count<S, MODE_L>());
    const size_t smemX = smem_of(stage_bytes<S, MODE_X3>(), stage_count<S, MODE_X3>());
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        if constexpr (EXACT) {
            attr_err = cudaFuncSetAttribute(k_mma<S, MODE_E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemE);
            if (attr_err == cudaSuccess)
                attr_err =
                    cudaFuncSetAttribute(k_mma<S, MODE_L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemL);
        } else {
            attr_err = cudaFuncSetAttribute(k_mma<S, MODE_X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemX);
        }
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (tiles <= 0) return cudaSuccess;
    StageScope mma_scope(st, BDC_STAGE_GEMM, (EXACT && S > 4) ? 3 : 2, 0.0);
    const unsigned long long wait_ns = test_wait_ns();
    const int stall = test_stall();
    k_tile_list<<<nprobs, 128, 0, st>>>(probs, dmix, tlist, ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int grid = tiles < sm_count() ? tiles : sm_count();   // persistent: one CTA per SM
    if constexpr (EXACT) {
        k_mma<S, MODE_E><<<grid, THREADS, smemE, st>>>(mae, mbe, probs, dmix, nprobs, E, F, err, tlist, ntiles,
                                                       wait_ns, stall);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if constexpr (S > 4)
            k_mma<S, MODE_L><<<grid, THREADS, smemL, st>>>(ma, mb, probs, dmix, nprobs, E, F, err, tlist, ntiles,
                                                           wait_ns, 0);
    } else {
        k_mma<S, MODE_X3><<<grid, THREADS, smemX, st>>>(ma, mb, probs, dmix, nprobs, E, F, err, tlist, ntiles,
                                                        wait_ns, stall);
    }
    return cudaGetLastError();
}

}  // namespace

// tiles: the largest sum over one launch's products of ceil(Mmax/128) ceil(Nmax/128)
size_t gemm_mixed_scratch(long long rows_total, long long cols_total, int kmax, int prec, int slices,
                          long long tiles) {
    const int S = (prec == BDC_MIXED_BF16X3) ? 2 : slices;
    const int Kld = (kmax + TK - 1) / TK * TK;
    const int nprobs = 1 << 16;
    return layout(rows_total + TM, cols_total + TN_MAX, Kld, S, nprobs, tiles).total + 1024;
}

// probs: device problem table (M, N, K known on the device); hm: host layout
cudaError_t launch_gemm_mixed_tab(const GemmProb *probs, int nprobs, const std::vector<MixProb> &hm, int rowsA,
                                  int colsB, int kmax, int prec, int slices, void *scratch, size_t scratch_bytes,
                                  int *err, int phase, cudaStream_t st) {
    if (nprobs <= 0) return cudaSuccess;
    const int S = (prec == BDC_MIXED_BF16X3) ? 2 : slices;
    const int Kld = (kmax + TK - 1) / TK * TK;
    long long tiles = 0;
    for (const MixProb &m : hm) tiles += (long long)((m.Mmax + TM - 1) / TM) * m.tilesN;
    const Layout L = layout(rowsA + TM, colsB + TN_MAX, Kld, S, nprobs, tiles);
    if (L.total > scratch_bytes) return cudaErrorInvalidValue;
    char *sc = (char *)scratch;
    const int ra = rowsA + TM, cbn = colsB + TN_MAX;
    if (prec == BDC_MIXED_BF16X3) return run_mixed<2, false>(probs, nprobs, hm, ra, cbn, Kld, sc, L, err, phase, st);
    switch (S) {
        case 4: return run_mixed<4, true>(probs, nprobs, hm, ra, cbn, Kld, sc, L, err, phase, st);
        case 5: return run_mixed<5, true>(probs, nprobs, hm, ra, cbn, Kld, sc, L, err, phase, st);
        case 6: return run_mixed<6, true>(probs, nprobs, hm, ra, cbn, Kld, sc, L, err, phase, st);
        case 7: return run_mixed<7, true>(probs, nprobs, hm, ra, cbn, Kld, sc, L, err, phase, st);
        default: return cudaErrorInvalidValue;
    }
}

// simple layout: products packed one after another (rows by M bound, columns by N bound)
cudaError_t launch_gemm_mixed(const GemmProb *probs, int nprobs, const int *Mmax, const int *Nmax, int kmax, int prec,
                              int slices, void *scratch, size_t scratch_bytes, int *err, int phase, cudaStream_t st) {
    std::vector<MixProb> hm(nprobs);
    int rows = 0, cols = 0, tiles = 0;
    const int tn = TNX;
    for (int p = 0; p < nprobs; ++p) {
        MixProb m{};
        m.a_row0 = rows; m.b_col0 = cols; m.tile0 = tiles;
        m.Mmax = Mmax[p]; m.Nmax = Nmax[p];
        m.tilesN = (m.Nmax + tn - 1) / tn;
        tiles += ((m.Mmax + TM - 1) / TM) * m.tilesN;
        rows += m.Mmax; cols += m.Nmax;
        hm[p] = m;
    }
    return launch_gemm_mixed_tab(probs, nprobs, hm, rows, cols, kmax, prec, slices, scratch, scratch_bytes, err, phase,
                                 st);
}


}  // namespace bdc
