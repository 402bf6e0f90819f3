// FP64 operator applications C <- A [B1; B2] (Sec. 2.1, Eq. 1) on the
// fifth-generation tensor cores by exact splitting (FR_FP64S).
//
// GB300's FP64 pipe issues about two FMAs per clock per SM, so a dense
// FP64 operator product is bound by that pipe (two FLOP per loaded value
// per operator row).  Here the product is formed from integer digits on the
// BF16 tensor cores instead, exactly, and rounded once to FP64:
//   * every operator row i (host, x64_pack) and state column n (a pre-pass,
//     k_colexp) gets the largest biased exponent E of its values, so that
//     |x| < 2^(E - 1022); each value becomes the integer
//     X = round(x 2^(56 - (E - 1022))), |X| < 2^56, written as eight signed
//     base-128 digits, X = sum_p d_p 128^(7 - p), d_0 in [-128, 128] and
//     d_1..d_7 in [-64, 63] (all exact in bf16);
//   * sum_k Xa Xb = sum_L S_L 128^(14 - L) with the level sums
//     S_L = sum_{p + q = L} sum_k a_q b_p.  A digit product is below 2^14
//     (2^13 and 2^12 away from the leading digits), so |S_L| < 2^24 for
//     K <= 409: the FP32 accumulation of the tensor cores is exact.  The
//     levels 0..7 are kept (36 digit pairs per 16-wide K step); the dropped
//     ones are below 2^-52 of the column-times-row scale;
//   * the epilogue converts the eight level sums to integers and combines
//     them into W = sum_L S_L 128^(7 - L) (two 64-bit halves; W / 2^11
//     formed exactly), which frees the accumulators for the next tile's
//     MMAs; then it rounds W once to the FP64 value W 2^(Ei + En - 2096 +
//     11) and applies the mode's FP64 epilogue (the same arithmetic as the
//     FMA kernel, fr_gemm_body.cuh).
// The error of a result is that of rounding the operands to 56 bits below
// their row and column maxima, about 2^-56 K max|A_i.| max|B_.n|, below
// the FP64 FMA chain's own rounding.
//
// The MMA's roles match the split-BF16 kernel (fr_gemm_tc.cu): the state
// tile is the A operand (M = 128 state columns = TMEM lanes), the operator
// the B operand (N = the row block's rows padded to 16, at most 64), one
// accumulator per level at TMEM columns L Nmma (8 x 64 = all 512 columns;
// two accumulator sets when Nmma <= 32).
//
// Shared memory, per ring slot (one 16-wide K stage):
//   staging  the stage's FP64 state rows, a 16 x 128 box (one 2-D
//            tensor-map TMA load; rows past B1 or B2 zero-filled);
//   digits   eight bf16 tiles (128 x 16, K-major core matrices, LBO 128 B,
//            SBO 256 B), written by the two converter warps of the slot;
//   slab     the operator's eight digit slabs of the stage (Nmma x 16
//            each), one bulk copy from the packed image.
// Warp roles (16 warps): 0-5 converters (warps 2s, 2s + 1 own slot s, one
// half of the tile's columns each), 6-13 epilogue (TMEM lane quarter =
// warp % 4, the two warps of a quarter take alternate 8-row groups or
// points), 14 TMEM allocation and the single MMA-issuing thread, 15 the
// producer (one thread).  Every wait is bounded (fr_async.cuh): on expiry
// the CTA records an error code, all roles leave their loops, the producer
// and the MMA thread wait for what they issued, and TMEM is freed.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fr_async.cuh"
#include "fr_kernels.h"

namespace fr {
namespace {

// 16 warps, four per SM sub-partition, whose register file (16K) then holds
// 128 registers per thread
constexpr int kMaxSlots = 3;
constexpr int kConvWarps = 2 * kMaxSlots, kEpiWarps = 8;
constexpr int kMmaWarp = kConvWarps + kEpiWarps, kProdWarp = kMmaWarp + 1;
constexpr int kThreads = (kProdWarp + 1) * 32;
static_assert(kThreads == 512, "four warps per sub-partition");
constexpr uint32_t kStagingBytes = kStageK * kTileN * 8;  // 16 KB of FP64
constexpr uint32_t kDigitTile = kTileN * kStageK * 2;     // 4 KB: 128 x 16 bf16
constexpr int kSmemLimit = 232448;
constexpr int kColsTmem = 512;
// X + kOff: the digits d_1..d_7 shifted to [0, 127]
constexpr long long kOff =
    64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) + (1ll << 7) + 1ll);
static_assert(kOff < (1ll << 49), "offset below the leading digit");

struct Bars {
    uint64_t loaded[kMaxSlots];     // the stage's box and operator slab landed (tx)
    uint64_t converted[kMaxSlots];  // both converter warps of the slot wrote its digits
    uint64_t freed[kMaxSlots];      // the MMAs reading the slot completed
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, Bars *bars, int *err, int code) {
    return mbar_wait_abort(b, parity, &bars->abort, err, code);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start, leading-dimension byte offset (K
// direction), stride byte offset (8-row groups), descriptor version 1, no
// swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, float &v) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    v = __uint_as_float(r);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// X = round(x 2^(56 - (E - 1022))) (half away from zero) for |x| < 2^(E - 1022)
__device__ __forceinline__ long long fixed56(double x, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int be = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (be) m |= 1ull << 52;
    else be = 1;
    // X = round(8 m / 2^sh), sh = E - be >= 0 (E bounds the column): 8 m <
    // 2^56, so a shift of 63 already gives 0 (with its rounding half)
    const int sh = E - be < 63 ? E - be : 63;
    const unsigned long long X = ((m << 3) + ((1ull << sh) >> 1)) >> sh;
    return (b >> 63) ? -(long long)X : (long long)X;
}

// bf16 bits of the small integer u - off (u < 2^23): 2^23 + u as a float
// minus 2^23 + off is exact, and so is its bf16 (at most 8 significant bits)
__device__ __forceinline__ uint32_t digit_bits(uint32_t u, float off) {
    return __float_as_uint(__int_as_float(0x4B000000 | (int)u) - off);
}

// the eight digits of X as bf16 bits (top halves of f[p])
__device__ __forceinline__ void digits8(long long X, uint32_t (&f)[kX64Digits]) {
    const long long Y = X + kOff;
    f[0] = digit_bits((uint32_t)((int)(Y >> 49) + 128), 8388736.0f);  // 2^23 + 128
#pragma unroll
    for (int p = 1; p < kX64Digits; ++p) f[p] = digit_bits((uint32_t)(Y >> (7 * (7 - p))) & 127u, 8388672.0f);
}

// w 2^e2 rounded to the nearest FP64 value (ties to even): the conversion
// instruction rounds w, the power of two goes into the exponent field;
// results outside the normal range take the library path
__device__ __forceinline__ double ldexp_i64(long long w, int e2) {
    const double d = __ll2double_rn(w);
    const long long bits = __double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7FF) + e2;
    if (w == 0) return 0.0;
    if (ex < 1 || ex > 2046) return ldexp(d, e2);
    return __longlong_as_double(bits + ((long long)e2 << 52));
}

// the integer value of a level sum s (exact, |s| < 2^24): below 2^22 in
// magnitude, 1.5 2^23 + s is exact in [2^23, 2^24) and its low mantissa
// bits are s + 2^22; wider levels take the conversion instruction
__device__ __forceinline__ long long level_int(float s, bool wide) {
    if (wide) return (long long)__float2int_rz(s);
    return (long long)(__float_as_int(__fadd_rn(s, 12582912.0f)) - 0x4B400000);
}

// W' = floor(W / 2^11), W = sum_L s[L] 128^(7 - L) < 2^74 (two exact 64-bit
// halves, zh 2^28 + zl); s[L] are exact integers below 2^24 in magnitude
// (bit L of wide: level L may reach 2^22)
__device__ __forceinline__ long long level_sum(const float (&s)[kX64Digits], uint32_t wide) {
    const long long zh = level_int(s[0], wide & 1u) * (1ll << 21) + level_int(s[1], wide & 2u) * (1ll << 14) +
                         level_int(s[2], wide & 4u) * (1ll << 7) + level_int(s[3], wide & 8u);
    const long long zl = level_int(s[4], wide & 16u) * (1ll << 21) + level_int(s[5], wide & 32u) * (1ll << 14) +
                         level_int(s[6], wide & 64u) * (1ll << 7) + level_int(s[7], wide & 128u);
    return zh * (1ll << 17) + (zl >> 11);
}

// the product W' 2^(Ea + Eb - 2096) (= sum_L S_L 128^(7 - L) 2^(Ea + Eb -
// 2156 + 49)) as FP64: NaN for a non-finite column, 0 for a zero row or
// column
__device__ __forceinline__ double finish(long long w, int Ea, int Eb) {
    if (Eb == 2047) return __longlong_as_double(0x7FF8000000000000ll);
    if (Ea == 0 || Eb == 0) return 0.0;
    return ldexp_i64(w, Ea + Eb - 2096);
}

// The divergence epilogues (the arithmetic of gemm_block in fr_gemm_body.cuh,
// FP64 storage) of rows j0 .. j0 + nr - 1 of column n: every load of the
// group first (the rows' elements are this thread's alone), then the
// arithmetic and stores
__device__ __forceinline__ void epi_div8(const GemmArgsT<double> &g, int mode, int j0, int nr, int64_t n, int64_t e,
                                         const double (&v)[8]) {
    const double ur = mode == GEMM_DIV_RK ? g.uref[n / g.np] : 0.0;
#pragma unroll
    for (int h = 0; h < 8; h += 4) {  // four rows at a time (registers)
        double ij[4], rf[4], u[4], ua[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (h + i >= nr) break;
            const int64_t idx = (int64_t)(j0 + h + i) * g.ldc + n;
            ij[i] = __ldg(g.invJ + (int64_t)(j0 + h + i) * g.np + e);
            rf[i] = g.rfs ? __ldg(g.rfs + idx) : 0.0;
            if (mode == GEMM_DIV_RK) {
                u[i] = g.rk_last ? 0.0 : g.U[idx];
                ua[i] = (g.rk_last || !g.rk_first) ? g.Uacc[idx] : 0.0;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (h + i >= nr) break;
            const int64_t idx = (int64_t)(j0 + h + i) * g.ldc + n;
            const double rt = -ij[i] * v[h + i];
            if (mode == GEMM_DIV) {
                g.C[idx] = g.rfs ? rt + rf[i] : rt;
                continue;
            }
            double rv = rt;
            if (g.rfs) rv = __dadd_rn(rv, rf[i]);
            if (g.rk_last) {
                const double un = ua[i] + g.c_acc * rv;
                g.U[idx] = un;
                g.Us[idx] = un - ur;
            } else {
                g.Uacc[idx] = (g.rk_first ? u[i] : ua[i]) + g.c_acc * rv;
                g.Us[idx] = (u[i] - ur) + g.c_stage * rv;
            }
        }
    }
}

struct Cursor {
    int q = 0, ks = 0, rb = 0;
    uint32_t par = 0;
    int64_t tile = 0, n0 = 0, n1 = 0;
    __device__ void set(const TileMap &m, int nrb) {
        rb = (int)(tile % nrb);
        m.cols(tile / nrb, n0, n1);
    }
    __device__ void start(const TileMap &m, int nrb) {
        tile = blockIdx.x;
        set(m, nrb);
    }
    __device__ void next(const TileMap &m, int nrb, int nks, int nslot) {
        if (++q == nslot) {
            q = 0;
            par ^= 1u;
        }
        if (++ks == nks) {
            ks = 0;
            tile += gridDim.x;
            set(m, nrb);
        }
    }
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_x64(const GemmArgsT<double> g, const TileMap tm, const __grid_constant__ CUtensorMap tmB1,
               const __grid_constant__ CUtensorMap tmB2, const X64Operator op, const int *__restrict__ E, int nslot,
               int *err, int no_producer) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int Nmma = op.Nmma;
    const uint32_t slab_bytes = (uint32_t)kX64Digits * (uint32_t)Nmma * 32u;
    const uint32_t slot_bytes = kStagingBytes + kX64Digits * kDigitTile + slab_bytes;
    Bars *bars = reinterpret_cast<Bars *>(smem + (size_t)nslot * slot_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrb = op.nrb;
    const int64_t ntiles = tm.ept * tm.nvb * nrb;
    const int nks = op.Kpad / kStageK, n1st = op.K1pad / kStageK;
    const int64_t nmine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = nmine * nks;
    const uint32_t acc_stride = (uint32_t)kX64Digits * (uint32_t)Nmma;
    const int nbuf = 2u * acc_stride <= (uint32_t)kColsTmem ? 2 : 1;

    if (threadIdx.x == 0) {
        for (int q = 0; q < nslot; ++q) {
            mbar_init(&bars->loaded[q], 1);
            mbar_init(&bars->converted[q], 64);  // the slot's two converter warps
            mbar_init(&bars->freed[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], kEpiWarps * 32);
        }
        mbar_init(&bars->done, 1);
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_base)),
                     "r"(kColsTmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;

    if (warp < kConvWarps) {
        // ---- converters: warps 2s and 2s + 1 own slot s (columns 0..63 and
        // 64..127 of the tile); lane l converts columns l and l + 32 of its
        // half, each K half (8 values) into one 16-byte row of every digit tile
        const int myslot = warp >> 1, half = warp & 1;
        Cursor cu;
        cu.start(tm, nrb);
        for (int64_t idx = 0; idx < total; ++idx, cu.next(tm, nrb, nks, nslot)) {
            if (cu.q != myslot) continue;
            const int q = cu.q;
            // the columns' exponents (written by the pre-pass) before the wait
            int Ec[2];
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2) {
                const int64_t n = cu.n0 + 64 * half + 32 * c2 + lane;
                Ec[c2] = n < g.N ? __ldg(E + n) : 0;
            }
            if (!mbar_wait(&bars->loaded[q], cu.par, bars, err, 1)) break;
            uint8_t *slot = smem + (size_t)q * slot_bytes;
            const double *f = reinterpret_cast<const double *>(slot);
            uint8_t *dig = slot + kStagingBytes;
#pragma unroll 1
            for (int c2 = 0; c2 < 2; ++c2) {
                const int col = 64 * half + 32 * c2 + lane;
                int Eb = c2 ? Ec[1] : Ec[0];
                const bool live = Eb > 0 && Eb < 2047;
                if (!live) Eb = 1078;  // digits of zeros below
                const uint32_t rowoff = (uint32_t)(col >> 3) * 256u + (uint32_t)(col & 7) * 16u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t w[kX64Digits][4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        uint32_t fa[kX64Digits], fb[kX64Digits];
                        const double xa = live ? f[(8 * h + i) * kTileN + col] : 0.0;
                        const double xb = live ? f[(8 * h + i + 1) * kTileN + col] : 0.0;
                        digits8(fixed56(xa, Eb), fa);
                        digits8(fixed56(xb, Eb), fb);
#pragma unroll
                        for (int p = 0; p < kX64Digits; ++p) w[p][i >> 1] = __byte_perm(fa[p], fb[p], 0x7632);
                    }
#pragma unroll
                    for (int p = 0; p < kX64Digits; ++p)
                        *reinterpret_cast<uint4 *>(dig + (uint32_t)p * kDigitTile + rowoff + (uint32_t)h * 128u) =
                            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
                }
            }
            fence_async_smem();
            mbar_arrive(&bars->converted[q]);
        }
    } else if (warp < kConvWarps + kEpiWarps) {
        // ---- epilogue: lane quarter qq = warp % 4 holds tile rows (state
        // columns) 32 qq .. 32 qq + 31; the quarter's two warps take
        // alternate 8-row groups (points, GEMM_GRAD) of the row block.  Two
        // phases: the level sums of every row the thread owns become 64-bit
        // integers W' (registers), which releases the accumulators to the
        // next tile's MMAs; then the FP64 conversion and the mode's epilogue
        const int qq = warp & 3, part = (warp - kConvWarps) >> 2;
        const int row = qq * 32 + lane;
        int b = 0;
        uint32_t ph = 0;
        constexpr int kGroups = kX64MaxRows / 16;      // 8-row groups per warp
        constexpr int kPoints = (kX64MaxRows / 3 + 1) / 2;  // points per warp
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_full[b], ph, bars, err, 2)) break;
            tc_fence_after();
            const int rb = (int)(tile % nrb);
            int64_t n0, n1;
            tm.cols(tile / nrb, n0, n1);
            const int64_t n = n0 + row;
            const bool ok = n < n1;
            const int64_t e = n % g.np;
            const int Eb = ok ? __ldg(E + n) : 0;
            const int r0 = rb * op.rows;
            const int nrows = (g.M - r0) < op.rows ? g.M - r0 : op.rows;
            const uint32_t taddr = tmem + ((uint32_t)(qq * 32) << 16) + (uint32_t)b * acc_stride;
            if (MODE == GEMM_GRAD) {
                long long w[kPoints][3];
#pragma unroll
                for (int pi = 0; pi < kPoints; ++pi) {
                    const int pt = part + 2 * pi;
                    if (3 * pt >= nrows) break;
                    float sv[3][kX64Digits];
#pragma unroll
                    for (int L = 0; L < kX64Digits; ++L)
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            tmem_ld1(taddr + (uint32_t)L * (uint32_t)Nmma + (uint32_t)(3 * pt + d), sv[d][L]);
                    tmem_ld_wait();
#pragma unroll
                    for (int d = 0; d < 3; ++d) w[pi][d] = level_sum(sv[d], op.wide);
                }
                tc_fence_before();
                mbar_arrive(&bars->acc_empty[b]);
#pragma unroll
                for (int pi = 0; pi < kPoints; ++pi) {
                    const int pt = part + 2 * pi;
                    if (3 * pt >= nrows || !ok) break;
                    const int j = (r0 + 3 * pt) / 3;
                    const double *S = g.S + (int64_t)j * 9 * g.np + e;
                    double Sv[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) Sv[k] = __ldg(S + (int64_t)k * g.np);
                    const double ij = __ldg(g.invJ + (int64_t)j * g.np + e);
                    double gv[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) gv[d] = finish(w[pi][d], __ldg(op.rexp + 3 * j + d), Eb);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        g.C[(int64_t)(3 * j + m) * g.ldc + n] =
                            ij * (Sv[0 * 3 + m] * gv[0] + Sv[1 * 3 + m] * gv[1] + Sv[2 * 3 + m] * gv[2]);
                }
            } else {
                long long w[kGroups][8];
#pragma unroll
                for (int gi = 0; gi < kGroups; ++gi) {
                    const int g8 = part + 2 * gi;
                    if (8 * g8 >= nrows) break;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {  // four rows at a time (registers)
                        float sv[kX64Digits][4];
#pragma unroll
                        for (int L = 0; L < kX64Digits; ++L)
                            tmem_ld4(taddr + (uint32_t)L * (uint32_t)Nmma + (uint32_t)(8 * g8 + 4 * hh), sv[L]);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float sl[kX64Digits];
#pragma unroll
                            for (int L = 0; L < kX64Digits; ++L) sl[L] = sv[L][i];
                            w[gi][4 * hh + i] = level_sum(sl, op.wide);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&bars->acc_empty[b]);
                const double add = (MODE == GEMM_STORE && g.add_ref && ok) ? g.uref[n / g.np] : 0.0;
#pragma unroll
                for (int gi = 0; gi < kGroups; ++gi) {
                    const int g8 = part + 2 * gi;
                    if (8 * g8 >= nrows || !ok) break;
                    const int nr = nrows - 8 * g8 < 8 ? nrows - 8 * g8 : 8;
                    double v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        v[i] = i < nr ? finish(w[gi][i], __ldg(op.rexp + r0 + 8 * g8 + i), Eb) : 0.0;
                    if (MODE == GEMM_STORE) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (i < nr) g.C[(int64_t)(r0 + 8 * g8 + i) * g.ldc + n] = v[i] + add;
                    } else {
                        epi_div8(g, MODE, r0 + 8 * g8, nr, n, e, v);
                    }
                }
            }
            if (++b == nbuf) {
                b = 0;
                ph ^= 1u;
            }
        }
    } else if (warp == kProdWarp && lane == 0 && !no_producer) {
        // ---- producer: per stage the 16 x 128 FP64 box of the state (B1
        // rows 16 ks.. while ks < K1pad / 16, else B2 rows) and the
        // operator's digit slabs of the tile's row block
        Cursor cu;
        cu.start(tm, nrb);
        uint32_t issued = 0u, last_par = 0u;
        for (int64_t idx = 0; idx < total; ++idx, cu.next(tm, nrb, nks, nslot)) {
            const int q = cu.q;
            if (!mbar_wait(&bars->freed[q], cu.par ^ 1u, bars, err, 7)) break;
            issued |= 1u << q;
            last_par = (last_par & ~(1u << q)) | (cu.par << q);
            uint8_t *slot = smem + (size_t)q * slot_bytes;
            mbar_expect_tx(&bars->loaded[q], kStagingBytes + slab_bytes);
            const int ks = cu.ks;
            const CUtensorMap *tmap = ks < n1st ? &tmB1 : &tmB2;
            const int y = ks < n1st ? ks * kStageK : ks * kStageK - op.K1pad;
            tma_load_2d(slot, tmap, (int)cu.n0, y, &bars->loaded[q]);
            bulk_load(slot + kStagingBytes + kX64Digits * kDigitTile,
                      op.img + ((size_t)cu.rb * nks + ks) * slab_bytes, slab_bytes, &bars->loaded[q]);
        }
        if (*(volatile int *)&bars->abort)
            for (int q = 0; q < nslot; ++q)
                if ((issued >> q) & 1u) mbar_drain(&bars->loaded[q], (last_par >> q) & 1u, err, 9);
    } else if (warp == kMmaWarp && lane == 0) {
        // ---- the MMA issue loop: per stage the 36 digit pairs (p, q),
        // p + q <= 7, into the accumulator of level p + q
        // D F32 (bit 4); A and B BF16 (1 at bits 7 and 10, kind::f16);
        // K-major; N >> 3 at bit 17, M >> 4 at bit 24
        const uint32_t idesc =
            (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Nmma >> 3) << 17) | ((uint32_t)(kTileN >> 4) << 24);
        bool live = true;
        int q = 0;
        uint32_t qpar = 0;
        int b = 0;
        uint32_t aph = 0;
        for (int64_t tile = blockIdx.x; live && tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_empty[b], aph ^ 1u, bars, err, 4)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)b * acc_stride;
            for (int ks = 0; ks < nks; ++ks) {
                if (!mbar_wait(&bars->converted[q], qpar, bars, err, 5)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sl = smem_u32(smem + (size_t)q * slot_bytes);
                const uint32_t dig = sl + kStagingBytes, slab = dig + kX64Digits * kDigitTile;
#pragma unroll
                for (int p = 0; p < kX64Digits; ++p) {
                    const uint64_t ad = sdesc(dig + (uint32_t)p * kDigitTile, 128, 256);
#pragma unroll
                    for (int qd = 0; qd < kX64Digits - p; ++qd) {
                        const uint64_t bd = sdesc(slab + (uint32_t)qd * (uint32_t)Nmma * 32u, 128, 256);
                        mma_bf16(d + (uint32_t)(p + qd) * (uint32_t)Nmma, ad, bd, idesc, (ks | p) != 0);
                    }
                }
                mma_commit(&bars->freed[q]);
                if (++q == nslot) {
                    q = 0;
                    qpar ^= 1u;
                }
            }
            if (!live) break;
            mma_commit(&bars->acc_full[b]);
            if (++b == nbuf) {
                b = 0;
                aph ^= 1u;
            }
        }
        // every MMA issued above has completed once this arrives
        mma_commit(&bars->done);
        mbar_drain(&bars->done, 0, err, 6);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kColsTmem) : "memory");
}

// the pre-pass: one thread per column
__global__ void k_colexp(const double *__restrict__ B1, int64_t ldb1, int K1, const double *__restrict__ B2,
                         int64_t ldb2, int K2, int64_t N, int *__restrict__ E) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int e = 0;
    for (int k = 0; k < K1 + K2; ++k) {
        const double x = k < K1 ? __ldg(B1 + (int64_t)k * ldb1 + n) : __ldg(B2 + (int64_t)(k - K1) * ldb2 + n);
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        int be = (int)((b >> 52) & 0x7FF);
        if (!be && (b << 1)) be = 1;  // subnormal
        e = be > e ? be : e;
    }
    E[n] = e;
}

uint32_t slot_bytes_of(const X64Operator &op) {
    return kStagingBytes + kX64Digits * kDigitTile + (uint32_t)kX64Digits * (uint32_t)op.Nmma * 32u;
}
int slots_of(const X64Operator &op) {
    const int64_t n = (kSmemLimit - (int64_t)sizeof(Bars) - 1024) / slot_bytes_of(op);
    return n > kMaxSlots ? kMaxSlots : (int)n;
}

template <int MODE>
cudaError_t launch_mode(const GemmArgsT<double> &g, const TileMap &tm, const X64Operator &op, const int *E, int *err,
                        int grid, cudaStream_t s, int no_producer) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_x64<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    CUtensorMap m1, m2;
    cudaError_t e = encode_rows(&m1, g.B1, g.N, g.K1, g.ldb1);
    if (e == cudaSuccess) e = g.K2 > 0 ? encode_rows(&m2, g.B2, g.N, g.K2, g.ldb2) : encode_rows(&m2, g.B1, g.N, g.K1, g.ldb1);
    if (e != cudaSuccess) return e;
    const int nslot = slots_of(op);
    k_gemm_x64<MODE><<<grid, kThreads, x64_smem_bytes(op), s>>>(g, tm, m1, m2, op, E, nslot, err, no_producer);
    return cudaGetLastError();
}

}  // namespace

size_t x64_smem_bytes(const X64Operator &op) {
    const int n = slots_of(op);
    if (n < 2) return 0;
    return (size_t)n * slot_bytes_of(op) + sizeof(Bars);
}

cudaError_t launch_colexp(const double *B1, int64_t ldb1, int K1, const double *B2, int64_t ldb2, int K2, int64_t N,
                          int *E, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_colexp<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(B1, ldb1, K1, B2, ldb2, K2, N, E);
    return cudaGetLastError();
}

cudaError_t launch_gemm_x64(const GemmArgsT<double> &g, const X64Operator &op, const int *E, int *err,
                            cudaStream_t s, int no_producer) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (!op.img || !op.rexp || g.M != op.M || g.K1 != op.K1 || g.K2 != op.K2 || op.K1 + op.K2 > kX64MaxK ||
        op.Nmma > kX64MaxRows || op.Nmma % 16 || op.rows > op.Nmma || op.rows * op.nrb < op.M ||
        x64_smem_bytes(op) == 0)
        return cudaErrorInvalidValue;
    if (g.mode == GEMM_GRAD && op.rows % 3) return cudaErrorInvalidValue;
    if ((g.mode == GEMM_DIV || g.mode == GEMM_DIV_RK) && (g.geo_elem || g.Us0)) return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases and row strides, even column offsets
    if (((uintptr_t)g.B1 | (uintptr_t)(g.K2 > 0 ? g.B2 : g.B1)) % 16 || (g.ldb1 * 8) % 16 ||
        (g.K2 > 0 && (g.ldb2 * 8) % 16) || g.np % 2 || g.np <= 0 || g.N % g.np)
        return cudaErrorInvalidValue;
    static int nsm = 0;  // one device type per process
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    TileMap tm;
    tm.np = g.np;
    tm.nvb = (int)(g.N / g.np);
    tm.ept = (g.np + kTileN - 1) / kTileN;
    const int64_t ntiles = tm.ept * tm.nvb * op.nrb;
    const int grid = (int)(ntiles < nsm ? ntiles : nsm);
    switch (g.mode) {
        case GEMM_STORE:
            return launch_mode<GEMM_STORE>(g, tm, op, E, err, grid, s, no_producer);
        case GEMM_GRAD:
            return launch_mode<GEMM_GRAD>(g, tm, op, E, err, grid, s, no_producer);
        case GEMM_DIV:
            return launch_mode<GEMM_DIV>(g, tm, op, E, err, grid, s, no_producer);
        case GEMM_DIV_RK:
            return launch_mode<GEMM_DIV_RK>(g, tm, op, E, err, grid, s, no_producer);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fr
