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
// operator row of its column and writes C[j][n] coalesced across the warp,
// applying the same fused epilogues as the FP64/FP32 kernels (gradient
// transform, -1/J, RK update).
//
// Shared memory, no swizzle, K-major core matrices (8 rows x 16 bytes):
//   operator image  [hi | lo], per 16-wide K step: Nmma/8 row groups x
//                   2 K halves x 128 B  (LBO = 128 B, SBO = 256 B); loaded
//                   once per CTA by a bulk copy (TMA engine) and kept;
//   state stages    ring of nst stages of 32 K-values: [hi k0..15 | hi
//                   k16..31 | lo k0..15 | lo k16..31], each 128 rows x 16 K
//                   (4 KB, same LBO/SBO), written by the converter warps
//                   from coalesced FP32 loads of B.
// Warp roles (13 warps): 0-7 converters, 8-11 epilogue (TMEM lane quarter =
// warp % 4), 12 TMEM allocation, operator load and the single MMA-issuing
// thread.  Hand-offs use mbarriers; the MMA side signals with
// tcgen05.commit.  Every wait is bounded: on expiry the CTA records an error
// code, all roles leave their loops, and TMEM is freed after the last
// commit has landed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fr_kernels.h"

namespace fr {
namespace {

constexpr int kTileN = 128;         // state columns per tile (MMA M)
constexpr int kStageK = 32;         // K values per stage (two MMA K steps)
constexpr int kStageBytes = 16384;  // 128 x 32 x (hi + lo) x 2 B
constexpr int kConvWarps = 8, kEpiWarps = 4;
constexpr int kThreads = (kConvWarps + kEpiWarps + 1) * 32;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct Bars {
    uint64_t op_full;
    uint64_t done;
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t full[8];
    uint64_t empty[8];
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete.  Returns false
// (and raises the CTA's abort flag and the error code) on expiry or when
// another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, Bars *bars, int *err, int code) {
    const uint32_t a = smem_u32(b);
    const long long t0 = clock64();
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 31) == 31) {
            if (*(volatile int *)&bars->abort) return false;
            if (clock64() - t0 > kWaitCycles) {
                *(volatile int *)&bars->abort = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// epilogue of one operator row j of state column n (see gemm_block in
// fr_gemm.cu for the FP32/FP64 form of the same arithmetic)
template <int MODE>
__device__ __forceinline__ void epi_row(const GemmArgsT<float> &g, int j, int64_t n, float acc) {
    const int64_t idx = (int64_t)j * g.ldc + n;
    if (MODE == GEMM_STORE) {
        g.C[idx] = acc + (g.add_ref ? (float)g.uref[n / g.np] : 0.f);
    } else {
        const int64_t e = n % g.np;
        const float rt = -g.invJ[(int64_t)j * g.np + e] * acc;
        if (MODE == GEMM_DIV) {
            g.C[idx] = g.rfs ? (float)((double)rt + g.rfs[idx]) : rt;
        } else {
            const double ur = g.uref[n / g.np];
            const double rv = (double)rt + (g.rfs ? g.rfs[idx] : 0.0);
            const double u = g.U[idx];
            if (g.rk_last) {
                const double un = g.Uacc[idx] + g.c_acc * rv;
                g.U[idx] = un;
                g.Us[idx] = (float)(un - ur);
            } else {
                g.Uacc[idx] = (g.rk_first ? u : g.Uacc[idx]) + g.c_acc * rv;
                g.Us[idx] = (float)((u - ur) + g.c_stage * rv);
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const GemmArgsT<float> g, const uint8_t *__restrict__ opimg, int Nmma, int Kpad, int nst,
              uint32_t tmem_cols, int *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const uint32_t op_half = (uint32_t)Nmma * (uint32_t)Kpad * 2u;  // bytes of hi (or lo)
    const uint32_t op_bytes = 2u * op_half;
    uint8_t *stages = smem + op_bytes;
    Bars *bars = reinterpret_cast<Bars *>(stages + (size_t)nst * kStageBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (g.N + kTileN - 1) / kTileN;
    const int nkst = Kpad / kStageK;
    const int K = g.K1 + g.K2;

    if (threadIdx.x == 0) {
        mbar_init(&bars->op_full, 1);
        mbar_init(&bars->done, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], kEpiWarps * 32);
        }
        for (int s = 0; s < nst; ++s) {
            mbar_init(&bars->full[s], kConvWarps * 32);
            mbar_init(&bars->empty[s], 1);
        }
        bars->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == kConvWarps + kEpiWarps) {
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

    if (warp < kConvWarps) {
        // ---- converters: thread (r, h) fills row r, K half h of each stage
        const int r = threadIdx.x & (kTileN - 1), h = threadIdx.x >> 7;
        int s = 0;
        uint32_t ph = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int64_t n = tile * kTileN + r;
            const bool col_ok = n < g.N;
            for (int ks = 0; ks < nkst; ++ks) {
                float v[16];
                const int k0 = ks * kStageK + h * 16;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = k0 + i;
                    float x = 0.f;
                    if (col_ok && k < K) x = k < g.K1 ? g.B1[(int64_t)k * g.ldb1 + n] : g.B2[(int64_t)(k - g.K1) * g.ldb2 + n];
                    v[i] = x;
                }
                if (!mbar_wait(&bars->empty[s], ph ^ 1u, bars, err, 1)) goto conv_done;
                {
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]), h1 = __float2bfloat16_rn(v[2 * i + 1]);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
                        hw[i] = pack2(h0, h1);
                        lw[i] = pack2(l0, l1);
                    }
                    uint8_t *st = stages + (size_t)s * kStageBytes;
                    // K step h of this stage; row r: core matrix (r/8, half), row r%8
                    const uint32_t off = (uint32_t)h * 4096u + (uint32_t)(r >> 3) * 256u + (uint32_t)(r & 7) * 16u;
                    *reinterpret_cast<uint4 *>(st + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(st + off + 128) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                    *reinterpret_cast<uint4 *>(st + 8192 + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    *reinterpret_cast<uint4 *>(st + 8192 + off + 128) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
                }
                fence_async_smem();
                mbar_arrive(&bars->full[s]);
                if (++s == nst) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    conv_done:;
    } else if (warp < kConvWarps + kEpiWarps) {
        // ---- epilogue: lane quarter q = warp % 4 holds tile rows 32q..32q+31
        const int q = warp & 3;
        const int row = q * 32 + lane;
        int b = 0;
        uint32_t ph = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_full[b], ph, bars, err, 2)) break;
            tc_fence_after();
            const int64_t n = tile * kTileN + row;
            const bool ok = n < g.N;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * acc_stride;
            for (int c0 = 0; c0 < g.M; c0 += 24) {
                float v[24];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    if (c0 + cc * 8 < g.M) tmem_ld8(taddr + (uint32_t)(c0 + cc * 8), v + cc * 8);
                tmem_ld_wait();
                if (!ok) continue;
                if (MODE == GEMM_GRAD) {
                    const int64_t e = n % g.np;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int j = c0 / 3 + t;
                        if (3 * j >= g.M) break;
                        const float *S = g.S + (int64_t)j * 9 * g.np + e;
                        const float ij = g.invJ[(int64_t)j * g.np + e];
                        const float g0 = v[3 * t], g1 = v[3 * t + 1], g2 = v[3 * t + 2];
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const float s0 = S[(0 * 3 + m) * g.np], s1 = S[(1 * 3 + m) * g.np],
                                        s2 = S[(2 * 3 + m) * g.np];
                            g.C[(int64_t)(3 * j + m) * g.ldc + n] = ij * (s0 * g0 + s1 * g1 + s2 * g2);
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 24; ++t)
                        if (c0 + t < g.M) epi_row<MODE>(g, c0 + t, n, v[t]);
                }
            }
            tc_fence_before();
            mbar_arrive(&bars->acc_empty[b]);
            if (++b == 2) {
                b = 0;
                ph ^= 1u;
            }
        }
    } else if (lane == 0) {
        // ---- operator load, then the MMA issue loop
        const uint32_t op_s = smem_u32(smem);
        mbar_expect_tx(&bars->op_full, op_bytes);
        for (uint32_t off = 0; off < op_bytes; off += 32768u) {
            const uint32_t sz = op_bytes - off < 32768u ? op_bytes - off : 32768u;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    op_s + off),
                "l"(opimg + off), "r"(sz), "r"(smem_u32(&bars->op_full))
                : "memory");
        }
        bool live = mbar_wait(&bars->op_full, 0, bars, err, 3);
        // kind::f16: D F32 (bit 4), A and B BF16 (bits 7, 10), K-major,
        // N >> 3 at bit 17, M >> 4 at bit 24
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Nmma >> 3) << 17) |
                               ((uint32_t)(kTileN >> 4) << 24);
        const uint32_t st_s = smem_u32(stages);
        int s = 0, b = 0;
        uint32_t ph = 0, aph = 0;
        for (int64_t tile = blockIdx.x; live && tile < ntiles; tile += gridDim.x) {
            if (!mbar_wait(&bars->acc_empty[b], aph ^ 1u, bars, err, 4)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)b * acc_stride;
            for (int ks = 0; ks < nkst; ++ks) {
                if (!mbar_wait(&bars->full[s], ph, bars, err, 5)) {
                    live = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint32_t kstep = (uint32_t)(ks * 2 + kk);
                    const uint32_t a_hi = st_s + (uint32_t)s * kStageBytes + (uint32_t)kk * 4096u;
                    const uint32_t a_lo = a_hi + 8192u;
                    const uint32_t b_hi = op_s + kstep * (uint32_t)Nmma * 32u;
                    const uint32_t b_lo = b_hi + op_half;
                    const uint64_t ah = sdesc(a_hi, 128, 256), al = sdesc(a_lo, 128, 256);
                    const uint64_t bh = sdesc(b_hi, 128, 256), bl = sdesc(b_lo, 128, 256);
                    mma_bf16(d, ah, bh, idesc, (ks | kk) != 0);
                    mma_bf16(d, ah, bl, idesc, 1);
                    mma_bf16(d, al, bh, idesc, 1);
                }
                mma_commit(&bars->empty[s]);
                if (++s == nst) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!live) break;
            mma_commit(&bars->acc_full[b]);
            if (++b == 2) {
                b = 0;
                aph ^= 1u;
            }
        }
        // every MMA issued above has completed once this arrives
        mma_commit(&bars->done);
        mbar_wait(&bars->done, 0, bars, err, 6);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kConvWarps + kEpiWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

template <int MODE>
cudaError_t launch_mode(const GemmArgsT<float> &g, const TcOperator &op, int *err, int grid, cudaStream_t s) {
    const int nst = tc_stages(op);
    const size_t smem = tc_smem_bytes(op);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint32_t cols = 32;
    while (cols < 2u * (uint32_t)op.Nmma) cols <<= 1;
    k_gemm_tc<MODE><<<grid, kThreads, smem, s>>>(g, op.img, op.Nmma, op.Kpad, nst, cols, err);
    return cudaGetLastError();
}

}  // namespace

int tc_stages(const TcOperator &op) {
    const int64_t avail = 232448 - 4 * (int64_t)op.Nmma * op.Kpad - (int64_t)sizeof(Bars) - 1024;
    if (avail < 0) return 0;
    const int64_t n = avail / kStageBytes;
    return n > 8 ? 8 : (int)n;
}

size_t tc_smem_bytes(const TcOperator &op) {
    const size_t used = 2 * (size_t)op.Nmma * op.Kpad * 2 + (size_t)tc_stages(op) * kStageBytes + sizeof(Bars);
    // at least 116 KB, so that no two CTAs (and their tensor memory) share an SM
    return used < 118784 ? 118784 : used;
}

cudaError_t launch_gemm_tc(const GemmArgsT<float> &g, const TcOperator &op, int *err, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.M > op.Nmma || op.Nmma > 256 || op.Nmma % 16 || op.Kpad % kStageK || g.K1 + g.K2 > op.Kpad ||
        tc_stages(op) < 2)
        return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (g.N + kTileN - 1) / kTileN;
    const int grid = (int)(ntiles < nsm ? ntiles : nsm);
    switch (g.mode) {
        case GEMM_STORE:
            return launch_mode<GEMM_STORE>(g, op, err, grid, s);
        case GEMM_GRAD:
            return launch_mode<GEMM_GRAD>(g, op, err, grid, s);
        case GEMM_DIV:
            return launch_mode<GEMM_DIV>(g, op, err, grid, s);
        case GEMM_DIV_RK:
            return launch_mode<GEMM_DIV_RK>(g, op, err, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fr
