// Asynchronous-copy plumbing shared by the streaming operator kernels
// (fr_gemm_tc.cu on the tensor cores, fr_gemm_f32.cu on the FP32 pipe):
// shared-memory mbarriers with bounded waits, the proxy fence, 2-D tensor-map
// (TMA) and plain bulk copies into shared memory, and the host encoder of the
// state's tensor maps.  Internal.
//
// Every wait is bounded by clock64 (about 2 s): on expiry the waiting thread
// raises the CTA's abort flag and records an error code in *err (the host
// reads it after the launch), so that no kernel can hang on a copy or an
// arrival that never comes.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace fr {
namespace {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kTileN = 128;   // state columns per tile (one TMA box row)
constexpr int kStageK = 16;   // K rows per stage (one TMA box)

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

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity` to complete.  Returns false
// (and raises *abort and the error code) on expiry, or when another role of
// the CTA has raised *abort.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t *b, uint32_t parity, int *abort, int *err, int code) {
    const uint32_t a = smem_u32(b);
    const long long t0 = clock64();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 31) == 31) {
            if (*(volatile int *)abort) return false;
            if (clock64() - t0 > kWaitCycles) {
                *(volatile int *)abort = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

// Bounded wait that ignores the abort flag: after an abort, the thread that
// issued asynchronous work (bulk copies, MMAs) waits here for exactly that
// work to complete before the CTA releases its shared memory.  Returns false
// (recording `code`) only if the limit expires.
__device__ __forceinline__ bool mbar_drain(uint64_t *b, uint32_t parity, int *err, int code) {
    const uint32_t a = smem_u32(b);
    const long long t0 = clock64();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 31) == 31 && clock64() - t0 > kWaitCycles) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one 2-D tensor-map box (x = column, y = row) into shared memory, completing
// on bar's transaction count
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// a contiguous copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Host: 2-D tensor map of one row-major operand block (rows x cols values,
// row stride ld values), boxes of kStageK rows x kTileN columns, zero fill
// out of bounds (rows past the block read as zeros)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline cudaError_t encode_rows_t(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t es, int64_t cols,
                                 int rows, int64_t ld) {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return cudaErrorNotSupported;
        fn = reinterpret_cast<EncodeTiled>(p);
    }
    const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
    const cuuint64_t stride[1] = {(cuuint64_t)ld * es};
    const cuuint32_t box[2] = {(cuuint32_t)kTileN, (cuuint32_t)kStageK};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = fn(m, dt, 2, const_cast<void *>(base), dim, stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
inline cudaError_t encode_rows(CUtensorMap *m, const float *base, int64_t cols, int rows, int64_t ld) {
    return encode_rows_t(m, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), cols, rows, ld);
}
// the same boxes (16 rows x 128 columns) of FP64 values
inline cudaError_t encode_rows(CUtensorMap *m, const double *base, int64_t cols, int rows, int64_t ld) {
    return encode_rows_t(m, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, sizeof(double), cols, rows, ld);
}

// Tile t covers columns [n0, n1) of one variable block (N = nvb np columns,
// block b = columns [b np, (b+1) np)): the variable block runs fastest, so
// the nvb tiles of one element range are processed together and share the
// geometry factors of a fused epilogue through L2 (the other order, element
// range fastest, measured no faster).
struct TileMap {
    int64_t np, ept;  // elements per block, tiles per block
    int nvb;
    __host__ __device__ __forceinline__ void cols(int64_t t, int64_t &n0, int64_t &n1) const {
        const int64_t eb = t / nvb, vb = t % nvb;
        n0 = vb * np + eb * kTileN;
        const int64_t lim = (vb + 1) * np;
        n1 = n0 + kTileN < lim ? n0 + kTileN : lim;
    }
};

}  // namespace
}  // namespace fr
