// Operator applications C <- A [B1; B2] (Sec. 2.1, Eq. 1) in FP32 on the
// FP32 pipe, the FR_FP32 mode's operator kernel.
//
// The chunk-staged kernel (fr_gemm.cu) gives each thread one state column
// and RC operator rows: every FMA then needs its own operator value from
// shared memory, and the column of B is re-read once per row chunk.  Here
// one CTA takes a tile of 128 state columns through all operator rows (up
// to 240 per pass):
//   * a producer thread streams the tile's K rows in stages of 16 (one 2-D
//     tensor-map box of 16 x 128 floats, rows past B1 or B2 zero-filled by
//     the TMA unit) together with the operator's slab for that stage
//     ([16][MP] floats, a plain bulk copy) into a ring of shared-memory
//     slots, each slot guarded by an mbarrier (loaded) and released by the
//     15 compute warps (freed);
//   * compute warp w owns the 4-row blocks b = w, w + 15, w + 30, w + 45 of
//     the pass, and lane l the 4 columns 4l .. 4l + 3 of the tile: per
//     column k of a stage one 16-byte load of B (the lane's 4 columns), one
//     broadcast 16-byte load of A (the block's 4 rows) and 16 FMAs into
//     registers (8 paired FP32 FMA instructions, each lane of a pair an
//     ordinary round-to-nearest FMA).  A block whose 4 rows are all zero in column k skips it
//     (the stage's 16-bit mask per block, precomputed): the FMA chain of
//     each output is the same as the chunk-staged kernel's, k in increasing
//     order, less terms whose operator entry is zero;
//   * after the last stage of a (tile, pass) the warps store their rows
//     (16-byte stores, 512 contiguous bytes per row and warp) while the
//     producer already loads the next unit's stages.
// Every wait is bounded (fr_async.cuh); on expiry the CTA records an error
// code, all roles leave their loops, and the producer waits for its own
// copies in flight before the CTA exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fr_async.cuh"
#include "fr_kernels.h"

namespace fr {
namespace {

// 15 compute warps and the producer: 4 warps per SM sub-partition, whose
// register file (16K) then holds 128 registers per thread
constexpr int kWarps = 15;                  // compute warps
constexpr int kBlocksPerWarp = 4;           // 4-row blocks per warp and pass
constexpr int kThreads = (kWarps + 1) * 32;  // + the producer warp
static_assert(kWarps * kBlocksPerWarp * 4 == kF32RowsPerPass, "rows per pass");
constexpr int kBoxBytes = kStageK * kTileN * 4;
constexpr int kMaxSlots = 12;
constexpr int kSmemLimit = 232448;

struct Bars {
    uint64_t loaded[kMaxSlots];  // the stage's box and slab landed (tx)
    uint64_t freed[kMaxSlots];   // every compute warp is done with the slot
    int abort;
};

// (d0, d1) = (a b0 + d0, a b1 + d1): two independent round-to-nearest FMAs
// in one paired FP32 instruction (each result equals fmaf's)
__device__ __forceinline__ void fma2(float &d0, float &d1, float a, float b0, float b1) {
    asm("{\n\t.reg .b64 d, x, y;\n\tmov.b64 d, {%0, %1};\n\tmov.b64 x, {%2, %2};\n\tmov.b64 y, {%3, %4};\n\t"
        "fma.rn.f32x2 d, x, y, d;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a), "f"(b0), "f"(b1));
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_f32(const GemmArgsT<float> g, const TileMap tm, const __grid_constant__ CUtensorMap tmB1,
               const __grid_constant__ CUtensorMap tmB2, const F32Operator op, int nslot, int *err,
               int no_producer) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t slab_bytes = (uint32_t)op.MP * kStageK * 4u;
    const uint32_t slot_bytes = (uint32_t)kBoxBytes + slab_bytes;
    Bars *bars = reinterpret_cast<Bars *>(smem + (size_t)nslot * slot_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nst = op.Kpad / kStageK, n1st = op.K1pad / kStageK;
    // the operator's block masks and row map, copied once into shared
    // memory (read at every stage and tile)
    const int nmask = op.npass * nst * (op.MP / 4), nrow = op.npass * op.MP;
    int *s_row = reinterpret_cast<int *>(bars + 1);
    uint16_t *s_mask = reinterpret_cast<uint16_t *>(s_row + nrow);
    for (int i = threadIdx.x; i < nrow; i += kThreads) s_row[i] = op.rowmap[i];
    for (int i = threadIdx.x; i < nmask; i += kThreads) s_mask[i] = op.mask[i];
    const int64_t ntiles = tm.ept * tm.nvb;
    const int64_t nunits = ntiles * op.npass;  // (tile, pass), pass fastest
    const int64_t nmine = nunits > blockIdx.x ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = nmine * nst;

    if (threadIdx.x == 0) {
        for (int q = 0; q < nslot; ++q) {
            mbar_init(&bars->loaded[q], 1);
            mbar_init(&bars->freed[q], kWarps);
        }
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    __syncthreads();

    if (warp == kWarps) {
        // ---- producer: one box and one slab per stage into its slot
        if (lane == 0 && !no_producer) {
            uint32_t issued = 0u, last_par = 0u;
            int q = 0, ks = 0;
            uint32_t par = 0;
            int64_t unit = blockIdx.x;
            for (int64_t idx = 0; idx < total; ++idx) {
                if (!mbar_wait_abort(&bars->freed[q], par ^ 1u, &bars->abort, err, 7)) break;
                issued |= 1u << q;
                last_par = (last_par & ~(1u << q)) | (par << q);
                const int64_t tile = unit / op.npass;
                const int pass = (int)(unit - tile * op.npass);
                int64_t n0, n1;
                tm.cols(tile, n0, n1);
                uint8_t *slot = smem + (size_t)q * slot_bytes;
                mbar_expect_tx(&bars->loaded[q], (uint32_t)kBoxBytes + slab_bytes);
                if (ks < n1st) tma_load_2d(slot, &tmB1, (int)n0, ks * kStageK, &bars->loaded[q]);
                else tma_load_2d(slot, &tmB2, (int)n0, ks * kStageK - op.K1pad, &bars->loaded[q]);
                bulk_load(slot + kBoxBytes, op.img + ((size_t)pass * nst + ks) * op.MP * kStageK, slab_bytes,
                          &bars->loaded[q]);
                if (++q == nslot) {
                    q = 0;
                    par ^= 1u;
                }
                if (++ks == nst) {
                    ks = 0;
                    unit += gridDim.x;
                }
            }
            // after an abort: the copies issued must land before the shared
            // memory is released (a completed phase returns at once)
            if (*(volatile int *)&bars->abort)
                for (int qq = 0; qq < nslot; ++qq)
                    if ((issued >> qq) & 1u) mbar_drain(&bars->loaded[qq], (last_par >> qq) & 1u, err, 9);
        }
    } else {
        // ---- compute warps: warp w takes the 4-row blocks w + 15 bi, lane
        // l the tile's columns 4l .. 4l + 3
        const int nblk = op.MP / 4;
        float acc[kBlocksPerWarp][4][4];
        int q = 0;
        uint32_t par = 0;
        bool live = true;
        for (int64_t unit = blockIdx.x; live && unit < nunits; unit += gridDim.x) {
            const int64_t tile = unit / op.npass;
            const int pass = (int)(unit - tile * op.npass);
#pragma unroll
            for (int bi = 0; bi < kBlocksPerWarp; ++bi)
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[bi][r][c] = 0.f;
            for (int ks = 0; ks < nst; ++ks) {
                if (!mbar_wait_abort(&bars->loaded[q], par, &bars->abort, err, 1)) {
                    live = false;
                    break;
                }
                const uint8_t *slot = smem + (size_t)q * slot_bytes;
                const float *slab = reinterpret_cast<const float *>(slot + kBoxBytes);
                const uint16_t *mk = s_mask + ((size_t)pass * nst + ks) * nblk;
#pragma unroll
                for (int bi = 0; bi < kBlocksPerWarp; ++bi) {
                    const int blk = warp + kWarps * bi;
                    uint32_t m = blk < nblk ? (uint32_t)mk[blk] : 0u;
                    auto ldb = [&](int k) {
                        return *reinterpret_cast<const float4 *>(slot + k * (kTileN * 4) + lane * 16);
                    };
                    auto lda = [&](int k) { return *reinterpret_cast<const float4 *>(slab + k * op.MP + blk * 4); };
                    auto fma16 = [&](const float4 a, const float4 b) {
                        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            fma2(acc[bi][r][0], acc[bi][r][1], av[r], b.x, b.y);
                            fma2(acc[bi][r][2], acc[bi][r][3], av[r], b.z, b.w);
                        }
                    };
                    if (m == 0xFFFFu) {
                        // a dense block: the 16 columns without the bit walk
#pragma unroll
                        for (int k = 0; k < kStageK; ++k) fma16(lda(k), ldb(k));
                    } else if (m) {
                        // the listed columns in increasing order, each one's
                        // loads issued before the previous one's FMAs
                        int k = __ffs(m) - 1;
                        m &= m - 1u;
                        float4 a = lda(k), b = ldb(k);
                        while (m) {
                            k = __ffs(m) - 1;
                            m &= m - 1u;
                            const float4 a2 = lda(k), b2 = ldb(k);
                            fma16(a, b);
                            a = a2;
                            b = b2;
                        }
                        fma16(a, b);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars->freed[q]);
                if (++q == nslot) {
                    q = 0;
                    par ^= 1u;
                }
            }
            if (!live) break;
            // epilogue: the warp's rows of this pass, 4 columns per lane
            int64_t n0, n1;
            tm.cols(tile, n0, n1);
            if (4 * lane < n1 - n0) {
                const float add = g.add_ref ? (float)g.uref[n0 / g.np] : 0.f;
#pragma unroll
                for (int bi = 0; bi < kBlocksPerWarp; ++bi) {
                    const int blk = warp + kWarps * bi;
                    if (blk >= nblk) continue;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int row = s_row[pass * op.MP + blk * 4 + r];
                        if (row < 0) continue;
                        *reinterpret_cast<float4 *>(g.C + (int64_t)row * g.ldc + n0 + 4 * lane) =
                            make_float4(acc[bi][r][0] + add, acc[bi][r][1] + add, acc[bi][r][2] + add,
                                        acc[bi][r][3] + add);
                    }
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace

// the slot ring, the barriers, the row map and the block masks
size_t f32_smem_bytes(const F32Operator &op, int &nslot) {
    const size_t slot = (size_t)kBoxBytes + (size_t)op.MP * kStageK * 4;
    const size_t meta = (size_t)op.npass * op.MP * sizeof(int) +
                        (size_t)op.npass * (op.Kpad / kStageK) * (op.MP / 4) * sizeof(uint16_t);
    int64_t n = ((int64_t)kSmemLimit - (int64_t)sizeof(Bars) - (int64_t)meta - 1024) / (int64_t)slot;
    if (n > kMaxSlots) n = kMaxSlots;
    nslot = n < 0 ? 0 : (int)n;
    return (size_t)nslot * slot + sizeof(Bars) + meta;
}

void f32_pack(const double *A, int M, int K1, int K2, const std::vector<int> &perm, std::vector<float> &img,
              std::vector<uint16_t> &mask, std::vector<int> &rowmap, F32Operator &op) {
    const int K = K1 + K2;
    op.M = M;
    op.K1pad = (K1 + kStageK - 1) / kStageK * kStageK;
    op.Kpad = op.K1pad + (K2 + kStageK - 1) / kStageK * kStageK;
    op.npass = (M + kF32RowsPerPass - 1) / kF32RowsPerPass;
    const int rows1 = M < kF32RowsPerPass ? M : kF32RowsPerPass;
    op.MP = (rows1 + 3) / 4 * 4;
    const int nst = op.Kpad / kStageK, nblk = op.MP / 4;
    img.assign((size_t)op.npass * nst * kStageK * op.MP, 0.f);
    mask.assign((size_t)op.npass * nst * nblk, 0);
    rowmap.assign((size_t)op.npass * op.MP, -1);
    for (int p = 0; p < op.npass; ++p)
        for (int i = 0; i < op.MP; ++i) {
            const int gi = p * kF32RowsPerPass + i;
            if (i >= kF32RowsPerPass || gi >= M) continue;
            const int row = perm.empty() ? gi : perm[gi];
            rowmap[(size_t)p * op.MP + i] = row;
            for (int kc = 0; kc < op.Kpad; ++kc) {
                // image column kc: B1 rows in [0, K1pad), B2 rows after
                const int col = kc < op.K1pad ? (kc < K1 ? kc : -1) : (kc - op.K1pad < K2 ? K1 + kc - op.K1pad : -1);
                if (col < 0) continue;
                const float a = (float)A[(size_t)row * K + col];
                if (a == 0.f) continue;
                const int s = kc / kStageK, k = kc % kStageK;
                img[(((size_t)p * nst + s) * kStageK + k) * op.MP + i] = a;
                mask[((size_t)p * nst + s) * nblk + i / 4] |= (uint16_t)(1u << k);
            }
        }
}

cudaError_t launch_gemm_f32(const GemmArgsT<float> &g, const F32Operator &op, int *err, cudaStream_t s,
                            int no_producer) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.mode != GEMM_STORE || g.M != op.M || op.MP % 4 || op.MP > kF32RowsPerPass ||
        op.MP / 4 > kWarps * kBlocksPerWarp || op.Kpad % kStageK || op.K1pad % kStageK ||
        g.K1 > op.K1pad || g.K2 > op.Kpad - op.K1pad || !op.img || !op.mask || !op.rowmap)
        return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases and row strides; 16-byte output stores
    if (((uintptr_t)g.B1 | (uintptr_t)(g.K2 > 0 ? g.B2 : g.B1) | (uintptr_t)g.C | (uintptr_t)op.img) % 16 ||
        (g.ldb1 * 4) % 16 || (g.K2 > 0 && (g.ldb2 * 4) % 16) || g.ldc % 4 || g.np % 4)
        return cudaErrorInvalidValue;
    if (g.np <= 0 || g.N % g.np) return cudaErrorInvalidValue;
    int nslot = 0;
    const size_t smem = f32_smem_bytes(op, nslot);
    if (nslot < 2) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if (e != cudaSuccess) return e;
        configured = true;
    }
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
    const int64_t nunits = tm.ept * tm.nvb * op.npass;
    const int grid = (int)(nunits < nsm ? nunits : nsm);
    CUtensorMap m1, m2;
    cudaError_t e = encode_rows(&m1, g.B1, g.N, g.K1, g.ldb1);
    if (e == cudaSuccess)
        e = g.K2 > 0 ? encode_rows(&m2, g.B2, g.N, g.K2, g.ldb2) : encode_rows(&m2, g.B1, g.N, g.K1, g.ldb1);
    if (e != cudaSuccess) return e;
    k_gemm_f32<<<grid, kThreads, smem, s>>>(g, tm, m1, m2, op, nslot, err, no_producer);
    return cudaGetLastError();
}

}  // namespace fr
