// One RK stage of a batch of FR problems as one persistent launch.
//
// The batched engine (fr_batch.cu) groups every operator application and
// point-wise pass of all problems and element types into work lists.  Here
// all of a stage's work lists run in one cooperative launch: the phases of
// the RHS (interpolation; Navier-Stokes: common solution, corrected
// gradient, gradient at the flux points; transformed flux; common flux;
// divergence with the RK register update) in order, with a grid-wide
// barrier between two phases whose work depends on each other.  Work that
// does not (the interpolation and the Euler flux, both reading only the
// stage input) shares a phase.  Every CTA takes the phase's units
// (operator-kernel blocks of 128 columns x one row chunk, or 128 point-wise
// items) in turn.
//
// Memory: the later phases read what earlier phases of the same launch
// wrote, so the operator blocks load B with plain (coherent) loads, and the
// barrier orders the writes before it and the reads after it: each CTA's
// arrival is released by a device-scope fence, and the thread that sees the
// generation move acquires with another before the CTA proceeds.
//
// Waits are bounded: a barrier wait that runs past kBarrierCycles (~2 s)
// records kStageTimeout in *err and returns; every CTA then leaves, and
// later stage launches return at once until the host clears the error.
#include <cuda_runtime.h>

#include <cstdint>

#include "fr_gemm_body.cuh"
#include "fr_kernels.h"
#include "fr_point_body.cuh"

namespace fr {
namespace {

constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s at 2 GHz

// arrive at and pass the grid barrier; false if a wait ran out (here or in
// another CTA)
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (*(volatile int *)err) break;
                if (clock64() - t0 > kBarrierCycles) {
                    atomicCAS(err, 0, kStageTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)err == 0;
}

// one operator-kernel block of a grouped descriptor list, row chunk RC
template <typename T, int RC, int MODE>
__device__ __noinline__ void gemm_unit_rc(const GemmArgsT<T> *g, int64_t local, T *sA) {
    const int nchunks = (g->M + RC - 1) / RC;
    gemm_block<T, RC, MODE, false>(*g, (int)(local % nchunks) * RC, local / nchunks, sA);
}

template <typename T, int MODE>
__device__ __forceinline__ void gemm_unit(const StagePhase<T> &ph, int64_t bid, T *sA) {
    int lo = 0, hi = ph.ndesc - 1;
    while (lo < hi) {  // last descriptor with begin <= bid
        const int mid = (lo + hi + 1) >> 1;
        if (ph.begin[mid] <= bid) lo = mid;
        else hi = mid - 1;
    }
    const GemmArgsT<T> *g = ph.descs + lo;
    const int64_t local = bid - ph.begin[lo];
    constexpr bool m3 = MODE == GEMM_GRAD;  // row chunks in whole points (multiples of 3)
    // the batch's row chunks are at most kMaxBatchRC (the register budget)
    switch (ph.rc) {
        case 6: gemm_unit_rc<T, 6, MODE>(g, local, sA); break;
        case 12: gemm_unit_rc<T, 12, MODE>(g, local, sA); break;
        case 8: gemm_unit_rc<T, (m3 ? 6 : 8), MODE>(g, local, sA); break;
        default: break;
    }
}

// CTAs per SM the stage kernel is compiled for (its grid is all of them, so
// this is its occupancy): the largest count whose register budget leaves
// the operator blocks (row chunks up to 12) and the phase's point-wise code
// without more than a few spilled words (ptxas -v)
template <typename T, int VIS>
constexpr int stage_min_blocks() {
    return sizeof(T) == 4 ? (VIS == 1 ? 8 : 6) : (VIS == 1 ? 5 : 4);
}

// VIS: 1 Euler, 2 Navier-Stokes (compile time, so that an Euler batch does
// not carry the viscous code's registers)
template <typename T, int VIS>
__global__ void __launch_bounds__(kThreads, stage_min_blocks<T, VIS>()) k_stage(const StagePlan<T> plan, const PhysT<T> phys, unsigned *bar,
                                                    int *err, int skip_block) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    if (*(volatile int *)err) return;             // an earlier stage gave up
    if ((int)blockIdx.x == skip_block) return;    // self-test: never arrives
    for (int p = 0; p < plan.nph; ++p) {
        const StagePhase<T> &ph = plan.ph[p];
        const int64_t gu = ph.ndesc ? ph.total : 0;
        const int64_t fu = (ph.ftotal + kThreads - 1) / kThreads;
        const int64_t cu = (ph.ctotal + kThreads - 1) / kThreads;
        for (int64_t u = blockIdx.x; u < gu + fu + cu; u += gridDim.x) {
            if (u < gu) {
                switch (ph.mode) {
                    case GEMM_STORE: gemm_unit<T, GEMM_STORE>(ph, u, sA); break;
                    case GEMM_GRAD:
                        if constexpr (VIS == 2) gemm_unit<T, GEMM_GRAD>(ph, u, sA);
                        break;
                    case GEMM_DIV_RK: gemm_unit<T, GEMM_DIV_RK>(ph, u, sA); break;
                    default: break;
                }
                __syncthreads();  // sA is reloaded by the next unit
            } else if (u < gu + fu) {
                const int64_t gi = (u - gu) * kThreads + threadIdx.x;
                if (gi < ph.ftotal) {
                    const int i = find_item(ph.fbegin, ph.fn, gi);
                    const FluxItem<T> &it = ph.fitems[i];
                    const int64_t idx = gi - ph.fbegin[i], j = idx / it.np;
                    if (VIS == 2 && ph.xform)
                        flux_at<T, true, VIS>(it.nu, it.ne, it.np, it.U, const_cast<T *>(it.GU), it.S, it.invJ,
                                              it.FT, phys, j, idx - j * it.np);
                    else
                        flux_at<T, false, VIS>(it.nu, it.ne, it.np, it.U, const_cast<T *>(it.GU), it.S, it.invJ,
                                               it.FT, phys, j, idx - j * it.np);
                }
            } else {
                const int64_t gi = (u - gu - fu) * kThreads + threadIdx.x;
                if (gi < ph.ctotal) {
                    const int i = find_item(ph.cbegin, ph.cn, gi);
                    const FaceItem<T> &it = ph.citems[i];
                    if (VIS == 2 && ph.which == 0) common_solution_at(it.P, it.B, it.F, phys, gi - ph.cbegin[i]);
                    else common_flux_at<T, VIS>(it.P, it.B, it.F, phys, gi - ph.cbegin[i]);
                }
            }
        }
        if (p + 1 < plan.nph && !grid_barrier(bar, gridDim.x, err)) return;
    }
}

template <typename T>
size_t stage_smem(const StagePlan<T> &plan) {
    size_t m = 0;
    for (int p = 0; p < plan.nph; ++p) {
        const StagePhase<T> &ph = plan.ph[p];
        if (!ph.ndesc) continue;
        const size_t b = gemm_block_smem(ph.rc, (int)sizeof(T), ph.maxK, ph.maxK);
        if (b > m) m = b;
    }
    return m;
}

template <typename T, int VIS>
cudaError_t configure_stage() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_stage<T, VIS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T, int VIS>
cudaError_t stage_grid_vis(const StagePlan<T> &plan, int *grid) {
    cudaError_t e = configure_stage<T, VIS>();
    if (e != cudaSuccess) return e;
    const size_t smem = stage_smem(plan);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    int per_sm = 0, dev = 0, nsm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<T, VIS>, kThreads, smem)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    *grid = per_sm * nsm;
    return cudaSuccess;
}

template <typename T, int VIS>
cudaError_t launch_stage_vis(const StagePlan<T> &plan, const PhysT<T> &pt, unsigned *bar, int *err, int skip_block,
                             int grid, cudaStream_t s) {
    cudaError_t e = configure_stage<T, VIS>();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = stage_smem(plan);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_stage<T, VIS>, plan, pt, bar, err, skip_block);
}

}  // namespace

template <typename T>
cudaError_t stage_grid(const StagePlan<T> &plan, int viscous, int *grid) {
    return viscous ? stage_grid_vis<T, 2>(plan, grid) : stage_grid_vis<T, 1>(plan, grid);
}

template <typename T>
cudaError_t launch_stage(const StagePlan<T> &plan, const Phys &ph, unsigned *bar, int *err, int skip_block, int grid,
                         cudaStream_t s) {
    const size_t smem = stage_smem(plan);
    if (smem > 200 * 1024 || grid <= 0 || plan.nph <= 0 || plan.nph > kMaxStagePhases) return cudaErrorInvalidValue;
    const PhysT<T> pt = phys_t<T>(ph);
    return ph.viscous ? launch_stage_vis<T, 2>(plan, pt, bar, err, skip_block, grid, s)
                      : launch_stage_vis<T, 1>(plan, pt, bar, err, skip_block, grid, s);
}

template cudaError_t stage_grid<float>(const StagePlan<float> &, int, int *);
template cudaError_t stage_grid<double>(const StagePlan<double> &, int, int *);
template cudaError_t launch_stage<float>(const StagePlan<float> &, const Phys &, unsigned *, int *, int, int,
                                         cudaStream_t);
template cudaError_t launch_stage<double>(const StagePlan<double> &, const Phys &, unsigned *, int *, int, int,
                                          cudaStream_t);

}  // namespace fr
