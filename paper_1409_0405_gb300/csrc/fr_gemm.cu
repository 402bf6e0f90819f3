// Operator application C <- A [B1; B2] with fused epilogues, in FP64 or
// FP32 (T), the RK register update always in FP64.
//
// Every operator application of an FR step is a constant operator matrix A
// (at most 375 rows, 525 columns here) times a row-major state matrix B whose columns
// run over variables x elements (10^5 - 10^6 columns): the block-by-panel
// shape of Sec. 2.1 (Eq. 1, Fig. 1).  The paper splits B into column slabs,
// one per thread, and keeps A whole; here a CTA owns 128 columns and a
// chunk of RC operator rows, stages that chunk of A in shared memory
// (transposed, so the RC values of one k are contiguous broadcasts), and
// every thread streams its column of B once per chunk, accumulating RC
// outputs in registers.
//
// On GB300 the FP64 pipe issues about 2 FMA per clock per SM, so the FP64
// kernels are bound by FP64 issue, not by HBM (2 flop per 8-byte B element
// per row of A, 2*RC flop per B load): the design goal is to keep the FP64
// pipe fed and to waste no FMA on padding rows, hence RC is chosen per
// operator among the instantiated sizes to divide M with the least waste.
// The FP32 pipe is 64x wider; there the same kernel is bound by issue and
// by the L2 traffic of re-reading B once per row chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "fr_gemm_body.cuh"
#include "fr_kernels.h"

namespace fr {
namespace {

template <typename T, int RC, int MODE>
__global__ void __launch_bounds__(kThreads) k_gemm(const GemmArgsT<T> g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1-D grid, row chunk fastest: the chunks of one column tile run back
    // to back, so that tile of B is read from DRAM once and then from L2
    const int nchunks = (g.M + RC - 1) / RC;
    gemm_block<T, RC, MODE>(g, (int)(blockIdx.x % nchunks) * RC, (int64_t)(blockIdx.x / nchunks),
                            reinterpret_cast<T *>(smem_raw));
}

// Grouped persistent variant: one launch covers many operator applications
// (problems x element types).  begin[d] is the first block index of
// descriptor d (prefix sum of its row chunks x column tiles); the grid
// strides over all blocks.
template <typename T, int RC, int MODE>
__global__ void __launch_bounds__(kThreads) k_gemm_grouped(const GemmArgsT<T> *__restrict__ descs,
                                                           const int64_t *__restrict__ begin, int ndesc,
                                                           int64_t total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    for (int64_t bid = blockIdx.x; bid < total; bid += gridDim.x) {
        int lo = 0, hi = ndesc - 1;
        while (lo < hi) {  // last d with begin[d] <= bid
            const int mid = (lo + hi + 1) >> 1;
            if (begin[mid] <= bid) lo = mid;
            else hi = mid - 1;
        }
        const GemmArgsT<T> &g = descs[lo];
        const int64_t local = bid - begin[lo];
        const int nchunks = (g.M + RC - 1) / RC;
        gemm_block<T, RC, MODE>(g, (int)(local % nchunks) * RC, local / nchunks, sA);
        __syncthreads();  // sA is reloaded by the next block
    }
}

template <typename T, int RC, int MODE>
cudaError_t run(const GemmArgsT<T> &g, cudaStream_t s) {
    const int K = g.K1 + g.K2;
    const size_t smem = gemm_block_smem(RC, (int)sizeof(T), K, g.sp_rc ? g.sp_lmax : 0);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm<T, RC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int64_t blocks = ((g.N + kThreads - 1) / kThreads) * ((g.M + RC - 1) / RC);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_gemm<T, RC, MODE><<<(unsigned)blocks, kThreads, smem, s>>>(g);
    return cudaGetLastError();
}

// row-chunk sizes instantiated; GEMM_GRAD needs multiples of 3
constexpr int kRCs[] = {30, 27, 25, 24, 21, 20, 18, 17, 15, 13, 12, 10, 9, 8, 6, 5, 4, 3};

int pick_rc(int M, bool mult3) {
    int best = -1;
    long best_waste = 1L << 40;
    for (int rc : kRCs) {
        if (mult3 && rc % 3) continue;
        long chunks = (M + rc - 1) / rc;
        long waste = chunks * rc - M;
        // prefer no waste, then fewer chunks (fewer passes over B)
        long score = waste * 1000 + chunks;
        if (score < best_waste) {
            best_waste = score;
            best = rc;
        }
    }
    return best;
}

template <typename T, int MODE>
cudaError_t dispatch(int rc, const GemmArgsT<T> &g, cudaStream_t s) {
    switch (rc) {
#define FR_RC(X) \
    case X:      \
        return run<T, X, MODE>(g, s);
        FR_RC(30) FR_RC(27) FR_RC(24) FR_RC(21) FR_RC(18) FR_RC(15) FR_RC(12) FR_RC(9) FR_RC(6) FR_RC(3)
#undef FR_RC
    }
    if (MODE != GEMM_GRAD) {
        switch (rc) {
#define FR_RC(X) \
    case X:      \
        return run<T, (MODE == GEMM_GRAD ? 3 : X), MODE>(g, s);
            FR_RC(25) FR_RC(20) FR_RC(17) FR_RC(13) FR_RC(10) FR_RC(8) FR_RC(5) FR_RC(4)
#undef FR_RC
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
cudaError_t launch_gemm(const GemmArgsT<T> &g, cudaStream_t s) {
    if (g.N <= 0 || g.M <= 0) return cudaSuccess;
    int rc = pick_rc(g.M, g.mode == GEMM_GRAD);
    if (g.sp_rc) {
        // the compressed operator fixes the chunk size
        if (!g.sp_off || !g.sp_cols || !g.sp_vals || g.sp_lmax <= 0 || (g.mode == GEMM_GRAD && g.sp_rc % 3) ||
            (g.sp_masked && g.sp_rc != 3))
            return cudaErrorInvalidValue;
        rc = g.sp_rc;
    }
    switch (g.mode) {
        case GEMM_STORE:
            return dispatch<T, GEMM_STORE>(rc, g, s);
        case GEMM_GRAD:
            return dispatch<T, GEMM_GRAD>(rc, g, s);
        case GEMM_DIV:
            return dispatch<T, GEMM_DIV>(rc, g, s);
        case GEMM_DIV_RK:
            return dispatch<T, GEMM_DIV_RK>(rc, g, s);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_gemm<double>(const GemmArgsT<double> &, cudaStream_t);
template cudaError_t launch_gemm<float>(const GemmArgsT<float> &, cudaStream_t);

namespace {

template <typename T, int RC, int MODE>
cudaError_t run_grouped(const GemmArgsT<T> *descs, const int64_t *begin, int ndesc, int64_t total, int maxK,
                        int grid, cudaStream_t s) {
    // a dense chunk, or a compressed one with its column list (lmax <= K)
    const size_t smem = gemm_block_smem(RC, (int)sizeof(T), maxK, maxK);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_grouped<T, RC, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (smem > 200 * 1024 || grid <= 0) return cudaErrorInvalidValue;
    k_gemm_grouped<T, RC, MODE><<<grid, kThreads, smem, s>>>(descs, begin, ndesc, total);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t grouped_rc(int rc, const GemmArgsT<T> *descs, const int64_t *begin, int ndesc, int64_t total, int maxK,
                       int grid, cudaStream_t s) {
    switch (rc) {
        case 6: return run_grouped<T, 6, MODE>(descs, begin, ndesc, total, maxK, grid, s);
        case 12: return run_grouped<T, 12, MODE>(descs, begin, ndesc, total, maxK, grid, s);
        case 24: return run_grouped<T, 24, MODE>(descs, begin, ndesc, total, maxK, grid, s);
    }
    if (MODE != GEMM_GRAD) {
        switch (rc) {
            case 8: return run_grouped<T, (MODE == GEMM_GRAD ? 6 : 8), MODE>(descs, begin, ndesc, total, maxK, grid, s);
            case 16: return run_grouped<T, (MODE == GEMM_GRAD ? 6 : 16), MODE>(descs, begin, ndesc, total, maxK, grid, s);
            case 32: return run_grouped<T, (MODE == GEMM_GRAD ? 6 : 32), MODE>(descs, begin, ndesc, total, maxK, grid, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

const int kGroupedRCs[] = {6, 8, 12, 16, 24, 32};

namespace {
template <typename T, int MODE>
cudaError_t configure_mode() {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto fn) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    };
    set(k_gemm_grouped<T, 6, MODE>);
    set(k_gemm_grouped<T, 12, MODE>);
    set(k_gemm_grouped<T, 24, MODE>);
    if (MODE != GEMM_GRAD) {
        set(k_gemm_grouped<T, (MODE == GEMM_GRAD ? 6 : 8), MODE>);
        set(k_gemm_grouped<T, (MODE == GEMM_GRAD ? 6 : 16), MODE>);
        set(k_gemm_grouped<T, (MODE == GEMM_GRAD ? 6 : 32), MODE>);
    }
    return e;
}
}  // namespace

template <typename T>
cudaError_t configure_gemm_grouped() {
    cudaError_t e;
    if ((e = configure_mode<T, GEMM_STORE>()) != cudaSuccess) return e;
    if ((e = configure_mode<T, GEMM_GRAD>()) != cudaSuccess) return e;
    if ((e = configure_mode<T, GEMM_DIV>()) != cudaSuccess) return e;
    return configure_mode<T, GEMM_DIV_RK>();
}
template cudaError_t configure_gemm_grouped<float>();
template cudaError_t configure_gemm_grouped<double>();

int64_t gemm_blocks(int M, int64_t N, int rc) { return ((N + kThreads - 1) / kThreads) * ((M + rc - 1) / rc); }

template <typename T>
cudaError_t launch_gemm_grouped(const GemmArgsT<T> *descs, const int64_t *begin, int ndesc, int64_t total, int mode,
                                int rc, int maxK, int grid, cudaStream_t s) {
    if (ndesc <= 0 || total <= 0) return cudaSuccess;
    switch (mode) {
        case GEMM_STORE: return grouped_rc<T, GEMM_STORE>(rc, descs, begin, ndesc, total, maxK, grid, s);
        case GEMM_GRAD: return grouped_rc<T, GEMM_GRAD>(rc, descs, begin, ndesc, total, maxK, grid, s);
        case GEMM_DIV: return grouped_rc<T, GEMM_DIV>(rc, descs, begin, ndesc, total, maxK, grid, s);
        case GEMM_DIV_RK: return grouped_rc<T, GEMM_DIV_RK>(rc, descs, begin, ndesc, total, maxK, grid, s);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_gemm_grouped<double>(const GemmArgsT<double> *, const int64_t *, int, int64_t, int, int,
                                                 int, int, cudaStream_t);
template cudaError_t launch_gemm_grouped<float>(const GemmArgsT<float> *, const int64_t *, int, int64_t, int, int, int,
                                                int, cudaStream_t);

int sparse_pack(const double *A, int M, int K1, int K2, bool mult3, SparseOp &out, int only_rc) {
    out = SparseOp();
    const int K = K1 + K2;
    if (M <= 0 || K <= 0) return 0;
    const int cand[] = {30, 27, 25, 24, 21, 20, 18, 17, 15, 13, 12, 10, 9, 8, 6, 5, 4, 3};
    long best = -1;
    int best_rc = 0;
    for (int rc : cand) {
        if (mult3 && rc % 3) continue;
        if (only_rc && rc != only_rc) continue;
        long fma = 0;
        for (int m0 = 0; m0 < M; m0 += rc) {
            int cnt = 0;
            for (int k = 0; k < K; ++k) {
                bool nz = false;
                for (int r = 0; r < rc && m0 + r < M && !nz; ++r) nz = A[(size_t)(m0 + r) * K + k] != 0.0;
                cnt += nz;
            }
            fma += (long)cnt * rc;
        }
        if (best < 0 || fma < best) {
            best = fma;
            best_rc = rc;
        }
    }
    const long dense = (long)((M + best_rc - 1) / best_rc) * best_rc * K;
    if (best < 0 || best * 5 > dense * 4) return 0;
    out.rc = best_rc;
    for (int m0 = 0; m0 < M; m0 += best_rc) {
        out.off.push_back((int)out.cols.size());
        bool mid_set = false;
        for (int k = 0; k < K; ++k) {
            bool nz = false;
            for (int r = 0; r < best_rc && m0 + r < M && !nz; ++r) nz = A[(size_t)(m0 + r) * K + k] != 0.0;
            if (!nz) continue;
            if (!mid_set && k >= K1) {
                out.off.push_back((int)out.cols.size());
                mid_set = true;
            }
            out.cols.push_back(k);
            for (int r = 0; r < best_rc; ++r)
                out.vals.push_back(m0 + r < M ? A[(size_t)(m0 + r) * K + k] : 0.0);
        }
        if (!mid_set) out.off.push_back((int)out.cols.size());
        const int len = (int)out.cols.size() - out.off[out.off.size() - 2];
        out.lmax = std::max(out.lmax, len);
    }
    out.off.push_back((int)out.cols.size());
    return out.rc;
}

int sparse_pack_masked(const double *A, int M, int K1, int K2, SparseOp &out) {
    out = SparseOp();
    const int K = K1 + K2;
    if (M <= 0 || K <= 0 || K >= (1 << 24)) return 0;
    long nnz = 0;
    for (size_t i = 0; i < (size_t)M * K; ++i) nnz += A[i] != 0.0;
    const long dense = (long)((M + 2) / 3) * 3 * K;
    if (nnz * 5 > dense * 4) return 0;
    out.rc = 3;
    for (int m0 = 0; m0 < M; m0 += 3) {
        out.off.push_back((int)out.cols.size());
        bool mid_set = false;
        for (int k = 0; k < K; ++k) {
            int mask = 0;
            for (int r = 0; r < 3 && m0 + r < M; ++r)
                if (A[(size_t)(m0 + r) * K + k] != 0.0) mask |= 1 << r;
            if (!mask) continue;
            if (!mid_set && k >= K1) {
                out.off.push_back((int)out.cols.size());
                mid_set = true;
            }
            out.cols.push_back(k | (mask << 24));
            for (int r = 0; r < 3; ++r) out.vals.push_back(m0 + r < M ? A[(size_t)(m0 + r) * K + k] : 0.0);
        }
        if (!mid_set) out.off.push_back((int)out.cols.size());
        out.lmax = std::max(out.lmax, (int)out.cols.size() - out.off[out.off.size() - 2]);
    }
    out.off.push_back((int)out.cols.size());
    return 3;
}

}  // namespace fr
