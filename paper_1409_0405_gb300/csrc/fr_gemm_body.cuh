// The block body of the operator-application kernel (fr_gemm.cu), shared
// with the batched engine's persistent stage kernel (fr_stage.cu).  Internal.
//
// gemm_block<T, RC, MODE, NC>: one (row chunk, column tile) block of
// C <- A [B1; B2] with the epilogue MODE (see fr_gemm.cu).  NC = true reads
// B through the read-only data cache (B is not written during the kernel);
// the persistent stage kernel, whose later phases read what earlier phases
// of the same launch wrote, uses NC = false (plain, coherent loads).
#pragma once

#include <cuda_runtime.h>

#include "fr_kernels.h"

namespace fr {
namespace {

template <bool NC, typename T>
__device__ __forceinline__ T bload(const T *p) {
    if constexpr (NC) return __ldg(p);
    else return *p;
}

constexpr int kThreads = 128;

// The staged chunk of A keeps the RC values of one column k in a row of
// rc_pad values (fr_kernels.h), loaded with 16-byte vector loads.
// the padded row of column k (values past RC unused)
template <typename T, int RCP>
__device__ __forceinline__ void load_arow(const T *a, T (&av)[RCP]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int v = 0; v < RCP / 4; ++v) {
            const float4 q = reinterpret_cast<const float4 *>(a)[v];
            av[4 * v] = q.x;
            av[4 * v + 1] = q.y;
            av[4 * v + 2] = q.z;
            av[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int v = 0; v < RCP / 2; ++v) {
            const double2 q = reinterpret_cast<const double2 *>(a)[v];
            av[2 * v] = q.x;
            av[2 * v + 1] = q.y;
        }
    }
}

// One (row chunk, column tile) block of C <- A [B1; B2] with the epilogue
// MODE.  Block-uniform: every thread of the block calls it with the same
// (g, m0, tile); it stages the chunk of A in sA and synchronises.
// acc[r] = fma(av[r], bv, acc[r]) for the RC rows; in FP32 two rows per
// paired FMA instruction (fma.rn.f32x2: each lane an ordinary
// round-to-nearest FMA, so the results are those of fmaf)
template <typename T, int RC, int RCP>
__device__ __forceinline__ void fma_rows(T (&acc)[RC], const T (&av)[RCP], T bv) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int r = 0; r + 1 < RC; r += 2)
            asm("{\n\t.reg .b64 d, x, y;\n\tmov.b64 d, {%0, %1};\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %4};\n\t"
                "fma.rn.f32x2 d, x, y, d;\n\tmov.b64 {%0, %1}, d;\n\t}"
                : "+f"(acc[r]), "+f"(acc[r + 1])
                : "f"(av[r]), "f"(av[r + 1]), "f"(bv));
        if constexpr (RC % 2) acc[RC - 1] = fmaf(av[RC - 1], bv, acc[RC - 1]);
    } else {
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[r] = fma(av[r], bv, acc[r]);
    }
}

template <typename T, int RC, int MODE, bool NC = true>
__device__ __forceinline__ void gemm_block(const GemmArgsT<T> &g, int m0, int64_t tile, T *sA) {
    constexpr int RCP = rc_pad(RC, sizeof(T));
    const int K = g.K1 + g.K2;
    // dense: sA[k][r] for every column; compressed: sA[i][r] for the chunk's
    // column list i, the column numbers in sK; rows of RCP values
    int nl1 = g.K1, nl = K;
    int *sK = nullptr;
    if (g.sp_rc) {
        const int c = m0 / RC;
        const int beg = g.sp_off[2 * c], mid = g.sp_off[2 * c + 1], end = g.sp_off[2 * c + 2];
        nl1 = mid - beg;
        nl = end - beg;
        sK = reinterpret_cast<int *>(sA + (size_t)g.sp_lmax * RCP);
        for (int idx = threadIdx.x; idx < RC * nl; idx += kThreads) {
            const int i = idx / RC, r = idx - i * RC;
            sA[i * RCP + r] = g.sp_vals[(size_t)beg * RC + idx];
        }
        for (int idx = threadIdx.x; idx < nl; idx += kThreads) sK[idx] = g.sp_cols[beg + idx];
    } else {
        for (int idx = threadIdx.x; idx < RC * K; idx += kThreads) {
            const int r = idx / K, k = idx - r * K;
            sA[k * RCP + r] = (m0 + r < g.M) ? g.A[(size_t)(m0 + r) * K + k] : T(0);
        }
    }
    __syncthreads();
    const int64_t n = tile * kThreads + threadIdx.x;
    if (n < g.N) {
        T acc[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[r] = T(0);
        if constexpr (RC == 3) {
            if (sK && g.sp_masked) {
                // runs of listed columns with the same row mask, each mask
                // with its own loop (the FMAs of absent rows are not issued,
                // not even predicated off); the column order is unchanged
                const T *b1 = g.B1 + n, *b2 = g.B2 + n;
                const int64_t ld1 = g.ldb1, ld2 = g.ldb2;
                const int K1 = g.K1;
                auto bval = [&](int t) -> T {
                    const int k = sK[t] & 0xFFFFFF;
                    return t < nl1 ? bload<NC>(b1 + (int64_t)k * ld1) : bload<NC>(b2 + (int64_t)(k - K1) * ld2);
                };
                int i = 0;
                while (i < nl) {
                    const int m = sK[i] >> 24;
                    int j = i + 1;
                    while (j < nl && (sK[j] >> 24) == m) ++j;
                    const T *a = sA;
                    switch (m) {
#define FR_RUN(BODY)                               \
    {                                              \
        _Pragma("unroll 2") for (int t = i; t < j; ++t) { \
            const T bv = bval(t);                  \
            BODY                                   \
        }                                          \
    }                                              \
    break;
                        case 1: FR_RUN(acc[0] = fma(a[RCP * t], bv, acc[0]);)
                        case 2: FR_RUN(acc[1] = fma(a[RCP * t + 1], bv, acc[1]);)
                        case 3: FR_RUN(acc[0] = fma(a[RCP * t], bv, acc[0]); acc[1] = fma(a[RCP * t + 1], bv, acc[1]);)
                        case 4: FR_RUN(acc[2] = fma(a[RCP * t + 2], bv, acc[2]);)
                        case 5: FR_RUN(acc[0] = fma(a[RCP * t], bv, acc[0]); acc[2] = fma(a[RCP * t + 2], bv, acc[2]);)
                        case 6: FR_RUN(acc[1] = fma(a[RCP * t + 1], bv, acc[1]); acc[2] = fma(a[RCP * t + 2], bv, acc[2]);)
                        default:
                            FR_RUN(acc[0] = fma(a[RCP * t], bv, acc[0]); acc[1] = fma(a[RCP * t + 1], bv, acc[1]);
                                   acc[2] = fma(a[RCP * t + 2], bv, acc[2]);)
#undef FR_RUN
                    }
                    i = j;
                }
                sK = nullptr;  // done
                nl = -1;
            }
        }
        if (sK) {
            // the chunk's non-zero columns only, in increasing order: the
            // same sums as the dense loop, less the terms whose A is zero
            const T *b1 = g.B1 + n;
#pragma unroll 2
            for (int i = 0; i < nl1; ++i) {
                const T bv = bload<NC>(b1 + (int64_t)sK[i] * g.ldb1);
                T av[RCP];
                load_arow<T, RCP>(sA + i * RCP, av);
                fma_rows<T, RC, RCP>(acc, av, bv);
            }
            const T *b2 = g.B2 + n;
#pragma unroll 2
            for (int i = nl1; i < nl; ++i) {
                const T bv = bload<NC>(b2 + (int64_t)(sK[i] - g.K1) * g.ldb2);
                T av[RCP];
                load_arow<T, RCP>(sA + i * RCP, av);
                fma_rows<T, RC, RCP>(acc, av, bv);
            }
        } else if (nl >= 0) {
            {
                const T *b = g.B1 + n;
                const int64_t ld = g.ldb1;
#pragma unroll 2
                for (int k = 0; k < g.K1; ++k) {
                    const T bv = bload<NC>(b + (int64_t)k * ld);
                    T av[RCP];
                    load_arow<T, RCP>(sA + k * RCP, av);
                    fma_rows<T, RC, RCP>(acc, av, bv);
                }
            }
            if (g.K2 > 0) {
                const T *b = g.B2 + n;
                const int64_t ld = g.ldb2;
                const T *a0 = sA + g.K1 * RCP;
#pragma unroll 2
                for (int k = 0; k < g.K2; ++k) {
                    const T bv = bload<NC>(b + (int64_t)k * ld);
                    T av[RCP];
                    load_arow<T, RCP>(a0 + k * RCP, av);
                    fma_rows<T, RC, RCP>(acc, av, bv);
                }
            }
        }

        if (MODE == GEMM_STORE) {
            const T add = g.add_ref ? T(g.uref[n / g.np]) : T(0);
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
                const T *S = g.S + (int64_t)j * 9 * g.np + e;
                const T ij = g.invJ[(int64_t)j * g.np + e];
                const T g0 = acc[3 * jj], g1 = acc[3 * jj + 1], g2 = acc[3 * jj + 2];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const T s0 = S[(0 * 3 + m) * g.np], s1 = S[(1 * 3 + m) * g.np], s2 = S[(2 * 3 + m) * g.np];
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
                const T rt = -g.invJ[(int64_t)j * g.np + e] * acc[r];
                if (MODE == GEMM_DIV) {
                    g.C[idx] = g.rfs ? T((double)rt + g.rfs[idx]) : rt;
                } else {
                    // FP64 register update (both modes; the arithmetic of
                    // the streaming k_rk_update)
                    // (the addition rounded on its own: no contraction with the
                    // product above, whichever kernel inlines this body)
                    double rv = (double)rt;
                    T rt2 = rt;
                    if (g.rfs) {
                        rv = __dadd_rn(rv, g.rfs[idx]);
                        rt2 = T(rv);
                    }
                    if (g.rk_last) {
                        const double un = g.Uacc[idx] + g.c_acc * rv;
                        g.U[idx] = un;
                        g.Us[idx] = T(un - ur);
                    } else if (g.Us0) {
                        // FP32 storage: the next stage input in T from the
                        // step's centred start state (kept in Us0)
                        T b0;
                        if (g.rk_first) {
                            b0 = g.Us[idx];
                            g.Us0[idx] = b0;
                            g.Uacc[idx] = g.U[idx] + g.c_acc * rv;
                        } else {
                            b0 = g.Us0[idx];
                            g.Uacc[idx] = g.Uacc[idx] + g.c_acc * rv;
                        }
                        g.Us[idx] = b0 + T(g.c_stage) * rt2;
                    } else {
                        const double u = g.U[idx];
                        g.Uacc[idx] = (g.rk_first ? u : g.Uacc[idx]) + g.c_acc * rv;
                        g.Us[idx] = T((u - ur) + g.c_stage * rv);
                    }
                }
            }
        }
    }
}


}  // namespace
}  // namespace fr
