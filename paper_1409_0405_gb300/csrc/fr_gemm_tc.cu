// Operator applications C <- A [B1; B2] (Sec. 2.1, Eq. 1) on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory),
// in split BF16 ("BF16x3") with FP32 accumulation: every FP32 value x is
// carried as hi = bf16(x) and lo = bf16(x - hi), and
//     A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the dropped A_lo B_lo term is 2^-16 of a product).
//
// The roles of the two operands are swapped against the row-major statement
// so that one accumulator lane is one state column: the MMA computes
// D[n][j] = sum_k B^T[n][k] A^T[k][j] with M = 128 state columns per tile
// (TMEM lanes), N = the operator's rows padded to 16 (TMEM columns), K the
// operator's columns.  The epilogue thread of lane n then holds every
// operator row of its column and writes C[j][n] coalesced across the warp:
// a plain store (the interpolation, and the reference gradient and raw
// divergence of an RK step, which streaming kernels finish per point) or
// the divergence of a plain RHS, -(1/J) (A B) (+ rfs).
//
// Shared memory, no swizzle, K-major core matrices (8 rows x 16 bytes):
//   operator image  [hi | lo], per 16-wide K step: Nmma/8 row groups x
//                   2 K halves x 128 B  (LBO = 128 B, SBO = 256 B); loaded
//                   once per CTA by a bulk copy (TMA engine) and kept;
//   slot ring       D slots of 8 KB, one per stage of 16 K values.  A slot
//                   first receives the stage's FP32 state rows (a 16 x 128
//                   box, one 2-D tensor-map TMA load issued by the producer:
//                   the TMA engine writes shared memory directly, so the
//                   loads in flight are bounded by the ring, not by the L1
//                   left over beside the shared memory; rows past the end
//                   of B1 or B2 are filled with zeros by the TMA unit);
//                   one converter warp reads the whole stage into registers
//                   and overwrites the slot with its bf16 hi and lo core
//                   matrices [hi | lo] (4 KB each, LBO/SBO as above), which
//                   the MMA reads; its commit frees the slot for the next
//                   load.  Converter warp w owns the slots q with q % 8 ==
//                   w, so up to eight slots are converted at once.
// Warp roles (22 warps): 0-7 converters, 8-19 epilogue (TMEM lane quarter =
// warp % 4; the three warps of a quarter take every third 24-row group), 20
// TMEM allocation, operator load and the single MMA-issuing thread, 21 the
// producer of the state loads (one thread).  Hand-offs use mbarriers; the MMA side
// signals with tcgen05.commit.  Every wait is bounded: on expiry the CTA
// records an error code, all roles leave their loops, and TMEM is freed
// after the last commit has landed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fr_async.cuh"
#include "fr_kernels.h"

namespace fr {
static int tc_sub(const TcOperator &op);  // stages per slot (below)

namespace {

constexpr int kStageBytes = 8192;  // 128 x 16 x 4 B (FP32), later 128 x 16 x (hi + lo) x 2 B
constexpr int kConvWarps = 8, kEpiWarps = 12;  // epilogue: three warps per TMEM lane quarter
constexpr int kMmaWarp = kConvWarps + kEpiWarps, kProdWarp = kMmaWarp + 1;
constexpr int kThreads = (kConvWarps + kEpiWarps + 2) * 32;

constexpr int kMaxSlots = 12;

struct Bars {
    uint64_t op_full;
    uint64_t done;
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t loaded[kMaxSlots];     // producer's copies of a slot landed (tx)
    uint64_t converted[kMaxSlots];  // the slot's converter warp wrote its bf16 (tf32) tiles
    uint64_t freed[kMaxSlots];      // the MMAs reading the slot completed
    uint32_t tmem_base;
    int abort;
};

// the bounded waits of fr_async.cuh with this CTA's abort flag
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

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

// FP32 -> TF32 (10 stored mantissa bits), round half away from zero; the
// low 13 bits cleared (what the tensor core reads of a 32-bit operand)
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
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
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Epilogue of rows [c0, c0 + 24) of state column n (element e), the
// accumulators in v.  Two epilogues: the plain store (every operator of an
// RK step: the gradient and divergence products are finished by streaming
// kernels, see the callers) and the divergence of a plain RHS evaluation,
// -(1/J) v (+ rfs), whose loads of a sub-group are issued before its
// stores so that one thread keeps several in flight.
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

template <int MODE>
__device__ __forceinline__ void epi_group(const GemmArgsT<float> &g, int c0, int64_t n, int64_t e, const float *v) {
    if (MODE == GEMM_BIAS_ACT) {
        if (g.cl_add) {
            // the closure's output layer: the RHS correction in the FR layout
#pragma unroll
            for (int t = 0; t < 24; ++t) {
                const int j = c0 + t;
                if (j < g.M) {
                    const int var = j / g.cl_nu, pt = j - var * g.cl_nu;
                    const int64_t o = ((int64_t)pt * 5 + var) * g.np + n;
                    double a = g.rfs ? g.rfs[o] : 0.0;
                    if (n < g.cl_ne) a += g.cl_scale[var] * (double)(v[t] + __ldg(g.bias + j));
                    g.cl_add[o] = a;
                }
            }
            return;
        }
        // a network layer: Z = A B + bias (kept for the backward pass), gelu
#pragma unroll
        for (int t = 0; t < 24; ++t) {
            const int j = c0 + t;
            if (j < g.M) {
                const float z = v[t] + __ldg(g.bias + j);
                if (g.Z) g.Z[(int64_t)j * g.ldc + n] = z;
                g.C[(int64_t)j * g.ldc + n] = g.act ? gelu_f(z) : z;
            }
        }
    } else if (MODE == GEMM_ACT_BACK) {
        // a layer's backward data gradient: (W^T dZ) * gelu'(Z)
#pragma unroll
        for (int t = 0; t < 24; ++t) {
            const int j = c0 + t;
            if (j < g.M) {
                const int64_t o = (int64_t)j * g.ldc + n;
                g.C[o] = v[t] * gelu_df(__ldg(g.Zin + o));
            }
        }
    } else if (MODE == GEMM_STORE) {
        const float add = g.add_ref ? (float)g.uref[n / g.np] : 0.f;
#pragma unroll
        for (int t = 0; t < 24; ++t)
            if (c0 + t < g.M) g.C[(int64_t)(c0 + t) * g.ldc + n] = v[t] + add;
    } else {
        constexpr int RG = 8;
#pragma unroll
        for (int r0 = 0; r0 < 24; r0 += RG) {
            float ij[RG];
            double rf[RG];
#pragma unroll
            for (int i = 0; i < RG; ++i) {
                const int j = c0 + r0 + i;
                if (j < g.M) {
                    ij[i] = __ldg(g.invJ + (g.geo_elem ? 0 : (int64_t)j * g.np) + e);
                    rf[i] = g.rfs ? __ldg(g.rfs + (int64_t)j * g.ldc + n) : 0.0;
                }
            }
#pragma unroll
            for (int i = 0; i < RG; ++i) {
                const int j = c0 + r0 + i;
                if (j < g.M) {
                    const float rt = -ij[i] * v[r0 + i];
                    g.C[(int64_t)j * g.ldc + n] = g.rfs ? (float)((double)rt + rf[i]) : rt;
                }
            }
        }
    }
}

// The converter's in-place order: the column group (c = 0..3, columns
// l + 32 c of the 128) whose output overwrites FP32 input row k of a stage.
// bf16: group c writes hi at bytes [1024 c, 1024 c + 1024) = rows 2c, 2c+1
// and lo at 4096 + that = rows 8 + 2c, 9 + 2c; tf32: hi at [2048 c, 2048 c +
// 2048) = rows 4c .. 4c + 3 (lo lands past the FP32 rows).
template <bool TF>
__host__ __device__ constexpr int conv_kill(int k) {
    return TF ? k / 4 : (k < 8 ? k / 2 : (k - 8) / 2);
}


// TF = false: split BF16, the operator image resident in shared memory,
// slot = 8 KB (FP32 box, then bf16 hi | lo).  TF = true: split TF32 (4-byte
// halves, MMA K step 8), slot = 16 KB (FP32 box, then tf32 hi | lo) plus
// the stage's operator slab (Nmma x 16 x (hi, lo) x 4 B), streamed with the
// state because the largest split-TF32 operators do not fit beside a ring.
template <int MODE, bool TF>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const GemmArgsT<float> g, const TileMap tm, const __grid_constant__ CUtensorMap tmB1,
              const __grid_constant__ CUtensorMap tmB2, const uint8_t *__restrict__ opimg, int Nmma, int K1pad,
              int Kpad, int nslot, uint32_t tmem_cols, int *err, int no_producer, int terms, int sub) {
    extern __shared__ __align__(1024) uint8_t smem[];
    // terms (split BF16): 3 = state and operator split (hi and lo images);
    // 2 = state split, operator hi only; 1 = both rounded to bf16, hi only
    const uint32_t op_half = TF ? 0u : (uint32_t)Nmma * (uint32_t)Kpad * 2u;  // resident image: bytes of hi (lo)
    const uint32_t op_bytes = terms == 3 ? 2u * op_half : op_half;
    const uint32_t state_bytes = TF ? 16384u : (uint32_t)kStageBytes;
    const uint32_t slab_bytes = TF ? (uint32_t)Nmma * 128u : 0u;
    // a slot holds `sub` consecutive stages (one mbarrier round trip each way
    // per slot, not per stage)
    const uint32_t sub_bytes = state_bytes + slab_bytes;
    const uint32_t slot_bytes = (uint32_t)sub * sub_bytes;
    uint8_t *slots = smem + op_bytes;
    Bars *bars = reinterpret_cast<Bars *>(slots + (size_t)nslot * slot_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = tm.ept * tm.nvb;
    const int nkst = Kpad / kStageK;
    const int nss = (nkst + sub - 1) / sub;  // slots per tile

    if (threadIdx.x == 0) {
        mbar_init(&bars->op_full, 1);
        mbar_init(&bars->done, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], kEpiWarps * 32);
        }
        for (int q = 0; q < nslot; ++q) {
            mbar_init(&bars->loaded[q], 1);
            mbar_init(&bars->converted[q], 32);  // the converting warp
            mbar_init(&bars->freed[q], 1);
        }
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    const uint32_t acc_stride = tmem_cols / 2;

    // slot fills this CTA runs (tiles blockIdx.x, + gridDim.x, ...; nss
    // each), walked with incremental counters: the slot and its phase
    // parity, the fill within the tile (stages sub ks .. sub ks + sub - 1),
    // the tile's columns
    const int64_t nmine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = nmine * nss;
    struct Cursor {
        int q = 0, ks = 0;
        uint32_t par = 0;
        int64_t tile, n0 = 0, n1 = 0;
        __device__ void start(const TileMap &m) {
            tile = blockIdx.x;
            m.cols(tile, n0, n1);
        }
        __device__ void next(const TileMap &m, int nkst, int nslot) {
            if (++q == nslot) {
                q = 0;
                par ^= 1u;
            }
            if (++ks == nkst) {
                ks = 0;
                tile += gridDim.x;
                m.cols(tile, n0, n1);
            }
        }
    };

    if (warp < kConvWarps) {
        // ---- converters: warp w converts, on its own, every stage that
        // lands in a slot q with q % 8 == w, so that up to eight slots are
        // converted at once.  A warp passes through every phase of its
        // slots in order, which the phase-parity waits require (a waiter
        // must not skip a phase of the barrier it waits on).  Lane l converts
        // columns l + 32 c (c = 0..3).  The output overwrites the FP32 rows
        // in place: the hi (bf16: and lo) core matrices of column group c
        // cover the input rows kill(k) == c, so before group c is written
        // every column group still reads those rows into registers (and
        // group c its remaining rows); the warp is the slot's only reader
        // and writer, and __syncwarp orders each read phase before the
        // writes that follow it.  At most 32 values per lane are live.
        Cursor cu;
        cu.start(tm);
        for (int64_t idx = 0; idx < total; ++idx, cu.next(tm, nss, nslot)) {
            if (cu.q % kConvWarps != warp) continue;
            const int q = cu.q;
            if (!mbar_wait(&bars->loaded[q], cu.par, bars, err, 1)) break;
            const int64_t ncol = cu.n1 - cu.n0;
            for (int u = 0; u < sub && cu.ks * sub + u < nkst; ++u) {
            uint8_t *slot = slots + (size_t)q * slot_bytes + (size_t)u * sub_bytes;
            const float *f = reinterpret_cast<const float *>(slot);
            float x[4][kStageK];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int c2 = c; c2 < 4; ++c2) {
                    const bool ok = lane + 32 * c2 < ncol;
#pragma unroll
                    for (int k = 0; k < kStageK; ++k)
                        if (conv_kill<TF>(k) == c || (c2 == c && conv_kill<TF>(k) > c))
                            x[c2][k] = ok ? f[k * kTileN + lane + 32 * c2] : 0.f;
                }
                __syncwarp();
                const uint32_t rg = (uint32_t)(4 * c + (lane >> 3)), rr = (uint32_t)(lane & 7);
                if constexpr (TF) {
                    // tf32 core matrices: 8 rows x 4 values; row group rg,
                    // K core matrix kc (0..3) at rg * 512 + kc * 128
#pragma unroll
                    for (int kc = 0; kc < 4; ++kc) {
                        float hv[4], lv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            hv[i] = tf32_round(x[c][4 * kc + i]);
                            lv[i] = tf32_round(x[c][4 * kc + i] - hv[i]);
                        }
                        const uint32_t off = rg * 512u + (uint32_t)kc * 128u + rr * 16u;
                        *reinterpret_cast<float4 *>(slot + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<float4 *>(slot + 8192 + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                    }
                } else {
                    // bf16 core matrices: row group rg, K half h at rg * 256 + h * 128
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float a0 = x[c][8 * h + 2 * i], a1 = x[c][8 * h + 2 * i + 1];
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(a0), h1 = __float2bfloat16_rn(a1);
                            hw[i] = pack2(h0, h1);
                            lw[i] = pack2(__float2bfloat16_rn(a0 - __bfloat162float(h0)),
                                          __float2bfloat16_rn(a1 - __bfloat162float(h1)));
                        }
                        const uint32_t off = rg * 256u + (uint32_t)h * 128u + rr * 16u;
                        *reinterpret_cast<uint4 *>(slot + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if (terms > 1)
                            *reinterpret_cast<uint4 *>(slot + 4096 + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
            }
            }
            fence_async_smem();
            mbar_arrive(&bars->converted[q]);
        }
    } else if (warp < kConvWarps + kEpiWarps) {
        // ---- epilogue: lane quarter q = warp % 4 holds tile rows 32q..32q+31
        const int q = warp & 3, part = (warp - kConvWarps) >> 2;
        constexpr int kParts = kEpiWarps / 4;
        const int row = q * 32 + lane;
        int b = 0;
        uint32_t ph = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_full[b], ph, bars, err, 2)) break;
            tc_fence_after();
            int64_t n0, n1;
            tm.cols(tile, n0, n1);
            const int64_t n = n0 + row;
            const bool ok = n < n1;
            const int64_t e = n % g.np;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * acc_stride;
            for (int c0 = 24 * part; c0 < g.M; c0 += 24 * kParts) {
                float v[24];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    if (c0 + cc * 8 < g.M) tmem_ld8(taddr + (uint32_t)(c0 + cc * 8), v + cc * 8);
                tmem_ld_wait();
                if (ok) epi_group<MODE>(g, c0, n, e, v);
            }
            tc_fence_before();
            mbar_arrive(&bars->acc_empty[b]);
            if (++b == 2) {
                b = 0;
                ph ^= 1u;
            }
        }
    } else if (warp == kProdWarp && lane == 0 && !no_producer) {
        // ---- producer: one 2-D TMA box (16 K rows x 128 columns) per stage
        // into its part of the slot; stage ks reads B1 rows 16 ks.. (ks <
        // K1pad / 16) or B2 rows 16 ks - K1pad..
        const int n1st = K1pad / kStageK;
        Cursor cu;
        cu.start(tm);
        // slots with a copy issued, and the phase parity of each slot's last one
        uint32_t issued = 0u, last_par = 0u;
        for (int64_t idx = 0; idx < total; ++idx, cu.next(tm, nss, nslot)) {
            const int q = cu.q;
            if (!mbar_wait(&bars->freed[q], cu.par ^ 1u, bars, err, 7)) break;
            issued |= 1u << q;
            last_par = (last_par & ~(1u << q)) | (cu.par << q);
            const int64_t n0 = cu.n0;
            const int nv = nkst - cu.ks * sub < sub ? nkst - cu.ks * sub : sub;  // stages in this fill
            mbar_expect_tx(&bars->loaded[q], (uint32_t)nv * ((uint32_t)kStageBytes + slab_bytes));
            for (int u = 0; u < nv; ++u) {
                const int ks = cu.ks * sub + u;
                const CUtensorMap *tmap = ks < n1st ? &tmB1 : &tmB2;
                const int y = ks < n1st ? ks * kStageK : ks * kStageK - K1pad;
                uint8_t *slot = slots + (size_t)q * slot_bytes + (size_t)u * sub_bytes;
                tma_load_2d(slot, tmap, (int)n0, y, &bars->loaded[q]);
                // split TF32: the stage's operator slab (stage-major image)
                if constexpr (TF) bulk_load(slot + state_bytes, opimg + (size_t)ks * slab_bytes, slab_bytes, &bars->loaded[q]);
            }
        }
        // after an abort the consumers may have left before this thread's
        // last copies landed: wait for each slot's last issued phase (a
        // completed phase returns at once)
        if (*(volatile int *)&bars->abort)
            for (int q = 0; q < nslot; ++q)
                if ((issued >> q) & 1u) mbar_drain(&bars->loaded[q], (last_par >> q) & 1u, err, 9);
    } else if (warp == kMmaWarp && lane == 0) {
        // ---- operator load, then the MMA issue loop
        const uint32_t op_s = smem_u32(smem);
        bool live = true;
        if constexpr (!TF) {
            mbar_expect_tx(&bars->op_full, op_bytes);
            for (uint32_t off = 0; off < op_bytes; off += 32768u) {
                const uint32_t sz = op_bytes - off < 32768u ? op_bytes - off : 32768u;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        op_s + off),
                    "l"(opimg + off), "r"(sz), "r"(smem_u32(&bars->op_full))
                    : "memory");
            }
            live = mbar_wait(&bars->op_full, 0, bars, err, 3);
            // the image copies must land before the shared memory is released
            if (!live) mbar_drain(&bars->op_full, 0, err, 10);
        }
        // D F32 (bit 4); A and B BF16 (1 at bits 7, 10, kind::f16) or TF32
        // (2, kind::tf32); K-major; N >> 3 at bit 17, M >> 4 at bit 24
        const uint32_t fmt = TF ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(Nmma >> 3) << 17) |
                               ((uint32_t)(kTileN >> 4) << 24);
        const uint32_t st_s = smem_u32(slots);
        int q = 0;
        uint32_t qpar = 0;
        int b = 0;
        uint32_t aph = 0;
        for (int64_t tile = blockIdx.x; live && tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_empty[b], aph ^ 1u, bars, err, 4)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)b * acc_stride;
            for (int ss = 0; ss < nss; ++ss) {
                if (!mbar_wait(&bars->converted[q], qpar, bars, err, 5)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                for (int u = 0; u < sub && ss * sub + u < nkst; ++u) {
                    const int ks = ss * sub + u;
                    const uint32_t sl = st_s + (uint32_t)q * slot_bytes + (uint32_t)u * sub_bytes;
                    if constexpr (TF) {
                        // two K steps of 8; core matrices 128 B apart along K,
                        // row groups 512 B apart; the slab's lo half after its hi
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t a_hi = sl + (uint32_t)kk * 256u, a_lo = a_hi + 8192u;
                            const uint32_t b_hi = sl + state_bytes + (uint32_t)kk * 256u;
                            const uint32_t b_lo = b_hi + (uint32_t)Nmma * 64u;
                            const uint64_t ah = sdesc(a_hi, 128, 512), al = sdesc(a_lo, 128, 512);
                            const uint64_t bh = sdesc(b_hi, 128, 512), bl = sdesc(b_lo, 128, 512);
                            mma_tf32(d, ah, bh, idesc, (ks | kk) != 0);
                            mma_tf32(d, ah, bl, idesc, 1);
                            mma_tf32(d, al, bh, idesc, 1);
                        }
                    } else {
                        const uint32_t a_hi = sl, a_lo = sl + 4096u;
                        const uint32_t b_hi = op_s + (uint32_t)ks * (uint32_t)Nmma * 32u;
                        const uint32_t b_lo = b_hi + op_half;
                        const uint64_t ah = sdesc(a_hi, 128, 256), al = sdesc(a_lo, 128, 256);
                        const uint64_t bh = sdesc(b_hi, 128, 256), bl = sdesc(b_lo, 128, 256);
                        mma_bf16(d, ah, bh, idesc, ks != 0);
                        if (terms == 3) mma_bf16(d, ah, bl, idesc, 1);
                        if (terms >= 2) mma_bf16(d, al, bh, idesc, 1);
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
            if (++b == 2) {
                b = 0;
                aph ^= 1u;
            }
        }
        // every MMA issued above has completed once this arrives (waited for
        // even after an abort: the MMAs read shared memory and write TMEM)
        mma_commit(&bars->done);
        mbar_drain(&bars->done, 0, err, 6);
    }
    // every asynchronous operation of this CTA has completed here: the
    // producer and the MMA thread drained what they issued
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

template <int MODE, bool TF>
cudaError_t launch_mode(const GemmArgsT<float> &g, const TileMap &tm, const TcOperator &op, int *err, int grid,
                        cudaStream_t s, int no_producer) {
    const int nslot = tc_stages(op);
    const size_t smem = tc_smem_bytes(op);
    // the attribute is raised once per instantiation to the largest size
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<MODE, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
        if (e != cudaSuccess) return e;
        configured = 232448;
    }
    uint32_t cols = 32;
    while (cols < 2u * (uint32_t)op.Nmma) cols <<= 1;
    CUtensorMap m1, m2;
    cudaError_t e = encode_rows(&m1, g.B1, g.N, g.K1, g.ldb1);
    if (e == cudaSuccess) e = g.K2 > 0 ? encode_rows(&m2, g.B2, g.N, g.K2, g.ldb2) : encode_rows(&m2, g.B1, g.N, g.K1, g.ldb1);
    if (e != cudaSuccess) return e;
    // network layers: the forward rounds its state to bf16 (one product), the
    // backward data gradient keeps the state's lo half (two products)
    const int terms = !op.hi_only ? 3 : (MODE == GEMM_ACT_BACK ? 2 : 1);
    k_gemm_tc<MODE, TF><<<grid, kThreads, smem, s>>>(g, tm, m1, m2, op.img, op.Nmma, op.K1pad, op.Kpad, nslot, cols,
                                                    err, no_producer, terms, tc_sub(op));
    return cudaGetLastError();
}

}  // namespace

// shared memory: the resident operator image (split BF16) and the slot
// ring (2..12 slots of one or two stages; a split-TF32 stage is 16 KB of
// state plus the operator slab)
static int64_t tc_image_bytes(const TcOperator &op) {
    return op.tf32 ? 0 : (op.hi_only ? 2 : 4) * (int64_t)op.Nmma * op.Kpad;
}
static int64_t tc_stage_bytes(const TcOperator &op) {
    return op.tf32 ? 16384 + 128 * (int64_t)op.Nmma : (int64_t)kStageBytes;
}
static int64_t tc_free(const TcOperator &op) {
    return 232448 - tc_image_bytes(op) - (int64_t)sizeof(Bars) - 1024;
}
// stages per slot: two (half the hand-offs per stage) while that leaves a
// ring of at least four slots, else one
static int tc_sub(const TcOperator &op) { return tc_free(op) / (2 * tc_stage_bytes(op)) >= 4 ? 2 : 1; }
static int64_t tc_slot_bytes(const TcOperator &op) { return tc_sub(op) * tc_stage_bytes(op); }

int tc_stages(const TcOperator &op) {
    const int64_t n = tc_free(op) / tc_slot_bytes(op);
    return n < 0 ? 0 : (n > kMaxSlots ? kMaxSlots : (int)n);
}

size_t tc_smem_bytes(const TcOperator &op) {
    const size_t used = (size_t)tc_image_bytes(op) + (size_t)tc_stages(op) * tc_slot_bytes(op) + sizeof(Bars);
    // at least 116 KB, so that no two CTAs (and their tensor memory) share an SM
    return used < 118784 ? 118784 : used;
}

namespace {
// one image element per thread: operator row i < M and column k < K (the
// operator is W, or W^T when trans: then W has K rows and M columns), in
// the K-major core-matrix layout of tc_pack (hi only)
__global__ void k_pack_hi(const float *__restrict__ W, int M, int K, int ldw, int trans, int Nmma, int Kpad,
                          __nv_bfloat16 *__restrict__ img) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Nmma * Kpad) return;
    const int i = (int)(idx / Kpad), k = (int)(idx % Kpad);
    float a = 0.f;
    if (i < M && k < K) a = trans ? W[(int64_t)k * ldw + i] : W[(int64_t)i * ldw + k];
    const int ks = k / 16, kk = k % 16;
    const int64_t off = (int64_t)ks * Nmma * 16 + ((i / 8) * 2 + kk / 8) * 64 + (i % 8) * 8 + kk % 8;
    img[off] = __float2bfloat16_rn(a);
}
}  // namespace

size_t tc_hi_image_bytes(int M, int K) { return (size_t)((M + 15) / 16 * 16) * ((K + 15) / 16 * 16) * 2; }

cudaError_t tc_pack_hi(const float *W, int rows, int cols, int ldw, int trans, uint8_t *img, TcOperator &op,
                       cudaStream_t s) {
    // the operator's shape: W's (rows x cols), or (cols x rows) for W^T
    op.img = img;
    op.M = trans ? cols : rows;
    op.K = trans ? rows : cols;
    op.Nmma = (op.M + 15) / 16 * 16;
    op.Kpad = op.K1pad = (op.K + 15) / 16 * 16;
    op.tf32 = 0;
    op.hi_only = 1;
    if (rows <= 0 || cols <= 0 || op.Nmma > 256 || ((uintptr_t)img % 16)) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)op.Nmma * op.Kpad;
    k_pack_hi<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, op.M, op.K, ldw, trans, op.Nmma, op.Kpad,
                                                         reinterpret_cast<__nv_bfloat16 *>(img));
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const GemmArgsT<float> &g, const TcOperator &op, int *err, cudaStream_t s,
                           int no_producer) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.M > op.Nmma || op.Nmma > 256 || op.Nmma % 16 || op.Kpad % kStageK || op.K1pad % kStageK ||
        g.K1 > op.K1pad || g.K2 > op.Kpad - op.K1pad || tc_stages(op) < 2)
        return cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases, row strides and column offsets
    if (((uintptr_t)g.B1 | (uintptr_t)(g.K2 > 0 ? g.B2 : g.B1)) % 16 || (g.ldb1 * 4) % 16 ||
        (g.K2 > 0 && (g.ldb2 * 4) % 16) || g.np % 4)
        return cudaErrorInvalidValue;
    static int nsm = 0;  // one device type per process
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    if (g.np <= 0 || g.N % g.np) return cudaErrorInvalidValue;
    TileMap tm;
    tm.np = g.np;
    tm.nvb = (int)(g.N / g.np);
    tm.ept = (g.np + kTileN - 1) / kTileN;
    const int64_t ntiles = tm.ept * tm.nvb;
    const int grid = (int)(ntiles < nsm ? ntiles : nsm);
#define FR_TC_MODES(TF)                                                \
    switch (g.mode) {                                                  \
        case GEMM_STORE:                                               \
            return launch_mode<GEMM_STORE, TF>(g, tm, op, err, grid, s, no_producer);   \
        case GEMM_DIV:                                                 \
            return launch_mode<GEMM_DIV, TF>(g, tm, op, err, grid, s, no_producer);     \
    }
    if (op.tf32) {
        FR_TC_MODES(true)
    } else {
        if (g.mode == GEMM_BIAS_ACT) return launch_mode<GEMM_BIAS_ACT, false>(g, tm, op, err, grid, s, no_producer);
        if (g.mode == GEMM_ACT_BACK) return launch_mode<GEMM_ACT_BACK, false>(g, tm, op, err, grid, s, no_producer);
        FR_TC_MODES(false)
    }
#undef FR_TC_MODES
    return cudaErrorInvalidValue;
}

}  // namespace fr
