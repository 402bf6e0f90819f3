// FP64 operator application C <- A [B1; B2] with fused epilogues.
//
// Every operator application of an FR step is a constant operator matrix A
// (at most 225 x 330 here) times a row-major state matrix B whose columns
// run over variables x elements (10^5 - 10^6 columns): the block-by-panel
// shape of Sec. 2.1 (Eq. 1, Fig. 1).  The paper splits B into column slabs,
// one per thread, and keeps A whole; here a CTA owns 128 columns and a
// chunk of RC operator rows, stages that chunk of A in shared memory
// (transposed, so the RC values of one k are contiguous broadcasts), and
// every thread streams its column of B once per chunk, accumulating RC
// outputs in registers.
//
// On GB300 the FP64 pipe issues about 2 FMA per clock per SM, so these
// kernels are bound by FP64 issue, not by HBM (2 flop per 8-byte B element
// per row of A, 2*RC flop per B load): the design goal is to keep the FP64
// pipe fed and to waste no FMA on padding rows, hence RC is chosen per
// operator among the instantiated sizes to divide M with the least waste.
#include <cuda_runtime.h>

#include <cstdio>

#include "fr_kernels.h"

namespace fr {
namespace {

constexpr int kThreads = 128;

template <int RC, int MODE>
__global__ void __launch_bounds__(kThreads) k_gemm(const GemmArgs g) {
    extern __shared__ double sA[];  // [K][RC]
    const int K = g.K1 + g.K2;
    const int m0 = blockIdx.y * RC;
    for (int idx = threadIdx.x; idx < RC * K; idx += kThreads) {
        const int r = idx / K, k = idx - r * K;
        sA[k * RC + r] = (m0 + r < g.M) ? g.A[(size_t)(m0 + r) * K + k] : 0.0;
    }
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (n >= g.N) return;

    double acc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[r] = 0.0;

    {
        const double *b = g.B1 + n;
        const int64_t ld = g.ldb1;
#pragma unroll 2
        for (int k = 0; k < g.K1; ++k) {
            const double bv = __ldg(b + (int64_t)k * ld);
            const double *a = sA + k * RC;
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = fma(a[r], bv, acc[r]);
        }
    }
    if (g.K2 > 0) {
        const double *b = g.B2 + n;
        const int64_t ld = g.ldb2;
        const double *a0 = sA + g.K1 * RC;
#pragma unroll 2
        for (int k = 0; k < g.K2; ++k) {
            const double bv = __ldg(b + (int64_t)k * ld);
            const double *a = a0 + k * RC;
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[r] = fma(a[r], bv, acc[r]);
        }
    }

    if (MODE == GEMM_STORE) {
        const double add = g.add_ref ? g.uref[n / g.np] : 0.0;
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (m0 + r < g.M) g.C[(int64_t)(m0 + r) * g.ldc + n] = acc[r] + add;
    } else if (MODE == GEMM_GRAD) {
        // rows are (j, d) with d fastest; RC and m0 are multiples of 3
        const int64_t e = n % g.np;
#pragma unroll
        for (int jj = 0; jj < RC / 3; ++jj) {
            const int j = m0 / 3 + jj;
            if (3 * j >= g.M) break;
            const double *S = g.S + (int64_t)j * 9 * g.np + e;
            const double ij = g.invJ[(int64_t)j * g.np + e];
            const double g0 = acc[3 * jj], g1 = acc[3 * jj + 1], g2 = acc[3 * jj + 2];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double s0 = S[(0 * 3 + m) * g.np], s1 = S[(1 * 3 + m) * g.np],
                             s2 = S[(2 * 3 + m) * g.np];
                g.C[(int64_t)(3 * j + m) * g.ldc + n] = ij * (s0 * g0 + s1 * g1 + s2 * g2);
            }
        }
    } else {
        const int64_t e = n % g.np;
        const double ur = (MODE == GEMM_DIV_RK) ? g.uref[n / g.np] : 0.0;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int j = m0 + r;
            if (j >= g.M) break;
            const int64_t idx = (int64_t)j * g.ldc + n;
            const double rv = fma(-g.invJ[(int64_t)j * g.np + e], acc[r], g.rfs ? g.rfs[idx] : 0.0);
            if (MODE == GEMM_DIV) {
                g.C[idx] = rv;
            } else {
                const double u = g.U[idx];
                if (g.rk_last) {
                    const double un = g.Uacc[idx] + g.c_acc * rv;
                    g.U[idx] = un;
                    g.Us[idx] = un - ur;
                } else {
                    g.Uacc[idx] = (g.rk_first ? u : g.Uacc[idx]) + g.c_acc * rv;
                    g.Us[idx] = (u - ur) + g.c_stage * rv;
                }
            }
        }
    }
}

template <int RC, int MODE>
cudaError_t run(const GemmArgs &g, cudaStream_t s) {
    const int K = g.K1 + g.K2;
    const size_t smem = (size_t)RC * K * sizeof(double);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm<RC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((g.N + kThreads - 1) / kThreads), (unsigned)((g.M + RC - 1) / RC));
    k_gemm<RC, MODE><<<grid, kThreads, smem, s>>>(g);
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

template <int MODE>
cudaError_t dispatch(int rc, const GemmArgs &g, cudaStream_t s) {
    switch (rc) {
#define FR_RC(X) \
    case X:      \
        return run<X, MODE>(g, s);
        FR_RC(30) FR_RC(27) FR_RC(24) FR_RC(21) FR_RC(18) FR_RC(15) FR_RC(12) FR_RC(9) FR_RC(6) FR_RC(3)
#undef FR_RC
    }
    if (MODE != GEMM_GRAD) {
        switch (rc) {
#define FR_RC(X) \
    case X:      \
        return run<(MODE == GEMM_GRAD ? 3 : X), MODE>(g, s);
            FR_RC(25) FR_RC(20) FR_RC(17) FR_RC(13) FR_RC(10) FR_RC(8) FR_RC(5) FR_RC(4)
#undef FR_RC
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_gemm_f64(const GemmArgs &g, cudaStream_t s) {
    if (g.N <= 0 || g.M <= 0) return cudaSuccess;
    const int rc = pick_rc(g.M, g.mode == GEMM_GRAD);
    switch (g.mode) {
        case GEMM_STORE:
            return dispatch<GEMM_STORE>(rc, g, s);
        case GEMM_GRAD:
            return dispatch<GEMM_GRAD>(rc, g, s);
        case GEMM_DIV:
            return dispatch<GEMM_DIV>(rc, g, s);
        case GEMM_DIV_RK:
            return dispatch<GEMM_DIV_RK>(rc, g, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fr
