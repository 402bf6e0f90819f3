// Point-wise kernels of the FR engine (Sec. 2.1: every non-GEMM operation
// concerns a single solution or flux point): transformed fluxes at solution
// points, LDG common solutions and Rusanov/LDG common normal fluxes at
// interface and boundary flux points, layout conversion and reductions.
// The right-hand-side kernels are templated on the arithmetic type T
// (double or float); every constant is converted to T so that the FP32
// mode issues no FP64 arithmetic.
//
// Physics (Sec. 3.4: compressible Navier-Stokes with constant viscosity,
// Rusanov inviscid interface flux; Sec. 3.2: no-slip isothermal wall and
// Riemann-invariant far field):
//   p = (gamma-1)(E - rho|v|^2/2), c = sqrt(gamma p / rho), T = p/rho,
//   tau = mu (grad v + grad v^T - 2/3 div v I),
//   energy viscous flux v.tau + mu gamma/Pr grad e, e = T/(gamma-1),
//   total flux F_inv - F_vis.
// Interface treatment (the paper names no viscous scheme; LDG with a switch
// along s = (1, 0.1 sqrt 2, 0.01 sqrt 3)):  side a is "left" where its
// outward normal n has n.s > 0;  C = (ua+ub)/2 + beta sigma (ua-ub),
// viscous normal flux (Fa+Fb).n/2 - beta sigma (Fa-Fb).n, penalty
// tau (ua - ub), sigma = +1 if a is left else -1.
// Boundary: common solution C_b (wall: (rho, 0, rho e_w); far field: the
// Riemann-invariant ghost), Rusanov against the inviscid ghost (wall:
// (rho, -rho v, rho e_w + rho|v|^2/2)), viscous flux F_vis(C_b, grad u).n,
// penalty tau (u - C_b).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/fr.h"
#include "fr_kernels.h"
#include "fr_point_body.cuh"

namespace fr {
namespace {

template <typename T>
__global__ void k_common_solution(const Pairs P, const Bnd B, const FieldsT<T> F, const PhysT<T> ph) {
    common_solution_at(P, B, F, ph, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void k_common_flux(const Pairs P, const Bnd B, const FieldsT<T> F, const PhysT<T> ph) {
    if (ph.viscous) common_flux_at<T, 2>(P, B, F, ph, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    else common_flux_at<T, 1>(P, B, F, ph, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Diagnostics (FP64 accumulation in both modes).  Block sums of NQ values
// per block of kDiagThreads threads into partial[block][NQ].
constexpr int kDiagThreads = 256;

template <int NQ>
__device__ __forceinline__ void block_sum_store(double (&acc)[NQ], double *partial) {
    __shared__ double sh[NQ][kDiagThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = acc[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double x = 0.0;
        for (int w = 0; w < kDiagThreads / 32; ++w) x += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * NQ + threadIdx.x] = x;
    }
}

// rate of change of the kinetic-energy integral along R:
// sum w J (v . R_m - |v|^2/2 R_rho), u from the FP64 register
template <typename T>
__global__ void k_ke_rate(int nu, int64_t ne, int64_t np, const double *__restrict__ U, const T *__restrict__ R,
                          const double *__restrict__ wJ, double *partial) {
    double acc[1] = {0.0};
    const int64_t tot = (int64_t)nu * np;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx / np, e = idx - j * np;
        if (e >= ne) continue;
        const double *u = U + j * V * np + e;
        const T *r = R + j * V * np + e;
        const double ir = 1.0 / u[0];
        const double v0 = u[np] * ir, v1 = u[2 * np] * ir, v2 = u[3 * np] * ir;
        const double dk = v0 * (double)r[np] + v1 * (double)r[2 * np] + v2 * (double)r[3 * np] -
                          0.5 * (v0 * v0 + v1 * v1 + v2 * v2) * (double)r[0];
        acc[0] += wJ[idx] * dk;
    }
    block_sum_store<1>(acc, partial);
}

// force of the fluid on the no-slip walls: face integral (weights bw |S^T n^|)
// of the common normal momentum flux, inviscid (Rusanov against the wall
// ghost) and viscous (-F_v(C_b, grad u).n + tau (u - C_b)) parts
template <typename T>
__global__ void k_wall_force(const Bnd B, const double *__restrict__ bw, const FieldsT<T> F, const PhysT<T> ph,
                             double *partial) {
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t kb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kb < B.n;
         kb += (int64_t)gridDim.x * blockDim.x) {
        if (B.btag[kb] != FR_BC_WALL) continue;
        const int t = B.bt[kb];
        const int64_t np = F.np[t];
        const int f = B.bf[kb], e = B.be[kb];
        const int64_t o = fpt_off(f, e, np);
        T u[V], ghost[V], cb[V], fi[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = F.UF[t][o + v * np];
        const T n[3] = {T(B.bn[3 * kb]), T(B.bn[3 * kb + 1]), T(B.bn[3 * kb + 2])};
        bc_states(FR_BC_WALL, u, n, ph, ghost, cb);
        rusanov(u, ghost, n, ph.gamma, fi);
        const double wa = bw[kb] * B.bmag[kb];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] += wa * (double)fi[1 + a];
        if (ph.viscous) {
            // the common flux kernel's own viscous normal flux
            T g[3][V], fvn[V];
            load_grad(F.GUF[t], f, e, np, g);
            Prim<T> qc = prim(cb, ph.gamma);
            vis_flux_n(cb, qc, g, ph.mu, ph.kq, n, fvn);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T fv = -fvn[1 + a] + ph.tau * (u[1 + a] - cb[1 + a]);
                acc[3 + a] += wa * (double)fv;
            }
        }
    }
    block_sum_store<6>(acc, partial);
}

__global__ void k_sum_partials(const double *__restrict__ partial, int nblocks, int nq, double *out) {
    if ((int)threadIdx.x < nq) {
        double x = 0.0;
        for (int b = 0; b < nblocks; ++b) x += partial[(int64_t)b * nq + threadIdx.x];
        out[threadIdx.x] = x;
    }
}

template <typename T, bool XFORM>
__global__ void k_flux(int nu, int64_t ne, int64_t np, const T *__restrict__ U, T *__restrict__ GU,
                       const T *__restrict__ S, const T *__restrict__ invJ, T *__restrict__ FT, const PhysT<T> ph,
                       int gj) {
    // 2-D grid: y = solution point, x = element
    if (ph.viscous)
        flux_at<T, XFORM, 2>(nu, ne, np, U, GU, S, invJ, FT, ph, (int64_t)blockIdx.y,
                             (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gj);
    else
        flux_at<T, XFORM, 1>(nu, ne, np, U, GU, S, invJ, FT, ph, (int64_t)blockIdx.y,
                             (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gj);
}

// ---------------------------------------------------------------------------
// grouped variants: one launch over many (problem, element type) segments;
// begin[i] is the first global index of item i (prefix sum of its sizes)
template <typename T, bool XFORM>
__global__ void k_flux_grouped(const FluxItem<T> *__restrict__ items, const int64_t *__restrict__ begin, int n,
                               int64_t total, const PhysT<T> ph) {
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int i = find_item(begin, n, gi);
        const FluxItem<T> &it = items[i];
        const int64_t idx = gi - begin[i], j = idx / it.np;
        if (ph.viscous)
            flux_at<T, XFORM, 2>(it.nu, it.ne, it.np, it.U, const_cast<T *>(it.GU), it.S, it.invJ, it.FT, ph, j,
                                 idx - j * it.np);
        else
            flux_at<T, XFORM, 1>(it.nu, it.ne, it.np, it.U, const_cast<T *>(it.GU), it.S, it.invJ, it.FT, ph, j,
                          idx - j * it.np);
    }
}

template <typename T>
__global__ void k_face_grouped(const FaceItem<T> *__restrict__ items, const int64_t *__restrict__ begin, int n,
                               int64_t total, const PhysT<T> ph, int which) {
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int i = find_item(begin, n, gi);
        const FaceItem<T> &it = items[i];
        if (which == 0) common_solution_at(it.P, it.B, it.F, ph, gi - begin[i]);
        else if (ph.viscous) common_flux_at<T, 2>(it.P, it.B, it.F, ph, gi - begin[i]);
        else common_flux_at<T, 1>(it.P, it.B, it.F, ph, gi - begin[i]);
    }
}

template <typename T>
__global__ void k_center_grouped(const CenterItem<T> *__restrict__ items, const int64_t *__restrict__ begin, int n,
                                 int64_t total) {
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int i = find_item(begin, n, gi);
        const CenterItem<T> &it = items[i];
        const int64_t idx = gi - begin[i];
        const int64_t v = (idx / it.np) % V;
        it.Us[idx] = T(it.U[idx] - it.uref[v]);
    }
}

// reference flux only (set-up, double)
__global__ void k_const_flux(int nu, int64_t ne, int64_t np, const double *__restrict__ S,
                             double *__restrict__ FT, const PhysT<double> ph) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = idx / np, e = idx - j * np;
    if (j >= nu || e >= ne) return;
    double s[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s[k] = S[(j * 9 + k) * np + e];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v)
            FT[((j * 3 + d) * V + v) * np + e] =
                s[d * 3 + 0] * ph.fref[v][0] + s[d * 3 + 1] * ph.fref[v][1] + s[d * 3 + 2] * ph.fref[v][2];
}

__global__ void k_const_common(const Pairs P, const Bnd B, const Fields F, const PhysT<double> ph) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) {
        const PairSides ps = pair_sides(P.code[k]);
        const int ta = ps.ta, tb = ps.tb;
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int64_t oa = fpt_off(ps.fa, P.ea[k], npa), ob = fpt_off(ps.fb, P.eb[k], npb);
        const double *n = P.nrm + 3 * k;
        for (int v = 0; v < V; ++v) {
            const double f = fref_n(ph, v, n);
            F.FC[ta][oa + v * npa] = f * P.maga[k];
            F.FC[tb][ob + v * npb] = -f * P.magb[k];
        }
        return;
    }
    const int64_t kb = k - P.n;
    if (kb < B.n) {
        const int t = B.bt[kb];
        const int64_t np = F.np[t];
        const int64_t o = fpt_off(B.bf[kb], B.be[kb], np);
        const double *n = B.bn + 3 * kb;
        for (int v = 0; v < V; ++v) F.FC[t][o + v * np] = fref_n(ph, v, n) * B.bmag[kb];
    }
}

struct Uref {
    double v[5];
};

template <typename T>
__global__ void k_pub_to_int(int nu, int64_t ne, int64_t np, const double *__restrict__ pub,
                             double *__restrict__ in, T *__restrict__ centred, const Uref uref) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = ne * V * nu;
    if (idx >= tot) return;
    const int64_t e = idx / (V * nu);
    const int64_t r = idx - e * V * nu;
    const int64_t v = r / nu, j = r - v * nu;
    const double x = pub[idx];
    if (in) in[(j * V + v) * np + e] = x;
    if (centred) centred[(j * V + v) * np + e] = T(x - uref.v[v]);
}

// The register kernels below run on a 2-D grid: y = row (j, v) of the
// [nu][V][np] register, x = element; no integer division per thread.
template <typename T>
__global__ void k_center(int64_t np, const double *__restrict__ U, T *__restrict__ Us, const Uref uref) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int row = blockIdx.y;
    const int64_t idx = (int64_t)row * np + e;
    Us[idx] = T(U[idx] - uref.v[row % V]);
}

// RK4 register update from a stored RHS r (the arithmetic of the fused
// GEMM_DIV_RK epilogue, applied as a separate streaming pass)
template <typename T>
__global__ void k_rk_update(int64_t np, const T *__restrict__ R, double *__restrict__ U,
                            double *__restrict__ Uacc, T *__restrict__ Us, const Uref uref, double c_acc,
                            double c_stage, int first, int last, const T *__restrict__ invJ,
                            const double *__restrict__ rfs, T *__restrict__ Us0, int gj) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int row = blockIdx.y;
    const int64_t idx = (int64_t)row * np + e;
    const double ur = uref.v[row % V];
    T rt;
    double rv;
    if (invJ) {
        // R holds the raw divergence-plus-correction product: scale it by
        // -1/J (in T, as the divergence epilogue does) and add rfs
        rt = -invJ[(int64_t)(row / V) * gj * np + e] * R[idx];
        rv = (double)rt;
        if (rfs) {
            rv = __dadd_rn(rv, rfs[idx]);  // as the fused epilogue: no contraction
            rt = T(rv);
        }
    } else {
        rt = R[idx];
        rv = (double)rt;
    }
    if (last) {
        const double un = Uacc[idx] + c_acc * rv;
        U[idx] = un;
        Us[idx] = T(un - ur);
    } else if (Us0) {
        // the next stage input (u_n - uref) + c_stage r formed in T from the
        // step's centred start state (Us at the first stage, kept in Us0):
        // only the FP64 accumulator update runs on the FP64 pipe
        T b0;
        if (first) {
            b0 = Us[idx];
            Us0[idx] = b0;
            Uacc[idx] = U[idx] + c_acc * rv;
        } else {
            b0 = Us0[idx];
            Uacc[idx] = Uacc[idx] + c_acc * rv;
        }
        Us[idx] = b0 + T(c_stage) * rt;
    } else {
        const double u = U[idx];
        Uacc[idx] = (first ? u : Uacc[idx]) + c_acc * rv;
        Us[idx] = T((u - ur) + c_stage * rv);
    }
}

// low-storage (2N) Runge-Kutta stage from a stored RHS r:
// dU = a dU + dt r (dU not read when first), U += b dU, Us = U - uref
template <typename T>
__global__ void k_rk_2n_update(int64_t np, const T *__restrict__ R, double *__restrict__ U,
                               double *__restrict__ dU, T *__restrict__ Us, const Uref uref, double a, double b,
                               double dt, int first) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int row = blockIdx.y;
    const int64_t idx = (int64_t)row * np + e;
    const double du = (first ? 0.0 : a * dU[idx]) + dt * (double)R[idx];
    const double u = U[idx] + b * du;
    dU[idx] = du;
    U[idx] = u;
    Us[idx] = T(u - uref.v[row % V]);
}

// RK45[2R+] stage (Kennedy, Carpenter & Lewis 2000, two registers) from a
// stored RHS r:  the next stage input is formed from the solution register
// before it is advanced, Us = (U - uref) + c_stage r (the last stage: the new
// U - uref), then U += c_acc r; the error register E accumulates
// c_err r (E = c_err r at the first stage; E may be null)
template <typename T>
__global__ void k_rk_2r_update(int64_t np, const T *__restrict__ R, double *__restrict__ U,
                               double *__restrict__ E, T *__restrict__ Us, const Uref uref, double c_stage,
                               double c_acc, double c_err, int first, int last) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int row = blockIdx.y;
    const int64_t idx = (int64_t)row * np + e;
    const double r = (double)R[idx];
    const double u = U[idx];
    const double un = u + c_acc * r;
    const double ur = uref.v[row % V];
    U[idx] = un;
    if (E) E[idx] = (first ? 0.0 : E[idx]) + c_err * r;
    Us[idx] = last ? T(un - ur) : T((u - ur) + c_stage * r);
}

// per-block partial sums of (E / (atol + rtol |U|))^2 over the element
// columns e < ne of one type's [nu][V][np] registers
__global__ void k_err_norm_partial(int nu, int64_t ne, int64_t np, const double *__restrict__ U,
                                   const double *__restrict__ E, double atol, double rtol, double *partial) {
    double acc[1] = {0.0};
    const int64_t tot = (int64_t)nu * V * np;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = idx / np, e = idx - row * np;
        if (e >= ne) continue;
        const double w = E[idx] / (atol + rtol * fabs(U[idx]));
        acc[0] += w * w;
    }
    block_sum_store<1>(acc, partial);
}

// state check after a step: one store of 1 by any thread that finds a bad
// point (no atomics needed; the flag is only ever set).  2-D grid: y = point
// row j, x = element
__global__ void k_state_check(int nu, int64_t ne, int64_t np, const double *__restrict__ U, int *flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (e >= ne || j >= nu) return;
    const double *u = U + (int64_t)j * V * np + e;
    double q[V];
#pragma unroll
    for (int v = 0; v < V; ++v) q[v] = u[v * np];
    // p = (gamma - 1)(E - |m|^2 / (2 rho)) > 0 with rho > 0 (and gamma > 1)
    // is 2 rho E > |m|^2: no division on the FP64 pipe
    const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    const double re = 2.0 * q[0] * q[4];
    bool bad = !(q[0] > 0.0) || !(re > m2) || !isfinite(re) || !isfinite(m2);
#pragma unroll
    for (int v = 0; v < V; ++v) bad = bad || !isfinite(q[v]);
    if (bad) *(volatile int *)flag = 1;
}

__global__ void k_to_float(int64_t n, const double *__restrict__ src, float *__restrict__ dst) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) dst[idx] = (float)src[idx];
}

template <typename T>
__global__ void k_int_to_pub(int nu, int64_t ne, int64_t np, const T *__restrict__ in, double *__restrict__ pub) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = ne * V * nu;
    if (idx >= tot) return;
    const int64_t e = idx / (V * nu);
    const int64_t r = idx - e * V * nu;
    const int64_t v = r / nu, j = r - v * nu;
    pub[idx] = (double)in[(j * V + v) * np + e];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_common_solution(const Pairs &P, const Bnd &B, const FieldsT<T> &F, const Phys &ph,
                                   cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_common_solution<T><<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, phys_t<T>(ph));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ke_rate(int nu, int64_t ne, int64_t np, const double *U, const T *R, const double *wJ,
                           double *partial, int nblocks, cudaStream_t s) {
    k_ke_rate<T><<<nblocks, kDiagThreads, 0, s>>>(nu, ne, np, U, R, wJ, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wall_force(const Bnd &B, const double *bw, const FieldsT<T> &F, const Phys &ph, double *partial,
                              int nblocks, cudaStream_t s) {
    k_wall_force<T><<<nblocks, kDiagThreads, 0, s>>>(B, bw, F, phys_t<T>(ph), partial);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *partial, int nblocks, int nq, double *out, cudaStream_t s) {
    if (nq < 1 || nq > 32) return cudaErrorInvalidValue;
    k_sum_partials<<<1, 32, 0, s>>>(partial, nblocks, nq, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_common_flux(const Pairs &P, const Bnd &B, const FieldsT<T> &F, const Phys &ph,
                               cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_common_flux<T><<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, phys_t<T>(ph));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flux(int nu, int64_t ne, int64_t np, const T *U, T *GU, const T *S, const T *invJ, T *FT,
                        const Phys &ph, cudaStream_t s, int gj) {
    if (ne == 0) return cudaSuccess;
    const dim3 grid(blocks_for(ne, 128), (unsigned)nu);
    if (invJ)
        k_flux<T, true><<<grid, 128, 0, s>>>(nu, ne, np, U, GU, S, invJ, FT, phys_t<T>(ph), gj);
    else
        k_flux<T, false><<<grid, 128, 0, s>>>(nu, ne, np, U, GU, S, invJ, FT, phys_t<T>(ph), gj);
    return cudaGetLastError();
}

cudaError_t launch_const_flux(int nu, int64_t ne, int64_t np, const double *S, double *FT, const Phys &ph,
                              cudaStream_t s) {
    const int64_t n = (int64_t)nu * np;
    if (ne == 0) return cudaSuccess;
    k_const_flux<<<blocks_for(n, 128), 128, 0, s>>>(nu, ne, np, S, FT, phys_t<double>(ph));
    return cudaGetLastError();
}

cudaError_t launch_const_common(const Pairs &P, const Bnd &B, const Fields &F, const Phys &ph, cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_const_common<<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, phys_t<double>(ph));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pub_to_int(int nu, int64_t ne, int64_t np, const double *pub, double *in, cudaStream_t s,
                              T *centred, const double *uref) {
    const int64_t n = ne * V * nu;
    if (n == 0) return cudaSuccess;
    Uref r{{0, 0, 0, 0, 0}};
    if (uref)
        for (int v = 0; v < V; ++v) r.v[v] = uref[v];
    k_pub_to_int<T><<<blocks_for(n, 256), 256, 0, s>>>(nu, ne, np, pub, in, centred, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_center(int nu, int64_t np, const double *U, T *Us, const double *uref, cudaStream_t s) {
    const int64_t n = (int64_t)nu * V * np;
    if (n == 0) return cudaSuccess;
    Uref r{{uref[0], uref[1], uref[2], uref[3], uref[4]}};
    k_center<T><<<dim3(blocks_for(np, 256), (unsigned)(nu * V)), 256, 0, s>>>(np, U, Us, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rk_update(int nu, int64_t np, const T *R, double *U, double *Uacc, T *Us, const double *uref,
                             double c_acc, double c_stage, int first, int last, const T *invJ, const double *rfs,
                             T *Us0, cudaStream_t s, int gj) {
    const int64_t n = (int64_t)nu * V * np;
    if (n == 0) return cudaSuccess;
    Uref r{{uref[0], uref[1], uref[2], uref[3], uref[4]}};
    k_rk_update<T><<<dim3(blocks_for(np, 256), (unsigned)(nu * V)), 256, 0, s>>>(np, R, U, Uacc, Us, r, c_acc,
                                                                                 c_stage, first, last, invJ, rfs,
                                                                                 Us0, gj);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rk_2n_update(int nu, int64_t np, const T *R, double *U, double *dU, T *Us, const double *uref,
                                double a, double b, double dt, int first, cudaStream_t s) {
    const int64_t n = (int64_t)nu * V * np;
    if (n == 0) return cudaSuccess;
    Uref r{{uref[0], uref[1], uref[2], uref[3], uref[4]}};
    k_rk_2n_update<T><<<dim3(blocks_for(np, 256), (unsigned)(nu * V)), 256, 0, s>>>(np, R, U, dU, Us, r, a, b, dt,
                                                                                    first);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rk_2r_update(int nu, int64_t np, const T *R, double *U, double *E, T *Us, const double *uref,
                                double c_stage, double c_acc, double c_err, int first, int last, cudaStream_t s) {
    const int64_t n = (int64_t)nu * V * np;
    if (n == 0) return cudaSuccess;
    Uref r{{uref[0], uref[1], uref[2], uref[3], uref[4]}};
    k_rk_2r_update<T><<<dim3(blocks_for(np, 256), (unsigned)(nu * V)), 256, 0, s>>>(np, R, U, E, Us, r, c_stage,
                                                                                    c_acc, c_err, first, last);
    return cudaGetLastError();
}

cudaError_t launch_err_norm_partial(int nu, int64_t ne, int64_t np, const double *U, const double *E, double atol,
                                    double rtol, double *partial, int nblocks, cudaStream_t s) {
    k_err_norm_partial<<<nblocks, kDiagThreads, 0, s>>>(nu, ne, np, U, E, atol, rtol, partial);
    return cudaGetLastError();
}

cudaError_t launch_state_check(int nu, int64_t ne, int64_t np, const double *U, double gamma, int *flag, int nblocks,
                               cudaStream_t s) {
    (void)gamma;   // the pressure test needs only gamma > 1
    (void)nblocks;  // one thread per point
    if (ne <= 0 || nu <= 0) return cudaSuccess;
    k_state_check<<<dim3(blocks_for(ne, 256), (unsigned)nu), 256, 0, s>>>(nu, ne, np, U, flag);
    return cudaGetLastError();
}

cudaError_t launch_to_float(int64_t n, const double *src, float *dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_float<<<blocks_for(n, 256), 256, 0, s>>>(n, src, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_int_to_pub(int nu, int64_t ne, int64_t np, const T *in, double *pub, cudaStream_t s) {
    const int64_t n = ne * V * nu;
    if (n == 0) return cudaSuccess;
    k_int_to_pub<T><<<blocks_for(n, 256), 256, 0, s>>>(nu, ne, np, in, pub);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flux_grouped(const FluxItem<T> *items, const int64_t *begin, int n, int64_t total, const Phys &ph,
                                int grid, cudaStream_t s, bool xform) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    if (xform)
        k_flux_grouped<T, true><<<grid, 128, 0, s>>>(items, begin, n, total, phys_t<T>(ph));
    else
        k_flux_grouped<T, false><<<grid, 128, 0, s>>>(items, begin, n, total, phys_t<T>(ph));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_face_grouped(const FaceItem<T> *items, const int64_t *begin, int n, int64_t total, const Phys &ph,
                                int which, int grid, cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    k_face_grouped<T><<<grid, 128, 0, s>>>(items, begin, n, total, phys_t<T>(ph), which);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_center_grouped(const CenterItem<T> *items, const int64_t *begin, int n, int64_t total, int grid,
                                  cudaStream_t s) {
    if (n <= 0 || total <= 0) return cudaSuccess;
    k_center_grouped<T><<<grid, 256, 0, s>>>(items, begin, n, total);
    return cudaGetLastError();
}

#define FR_INST(T)                                                                                            \
    template cudaError_t launch_common_solution<T>(const Pairs &, const Bnd &, const FieldsT<T> &, const Phys &, \
                                                   cudaStream_t);                                             \
    template cudaError_t launch_common_flux<T>(const Pairs &, const Bnd &, const FieldsT<T> &, const Phys &,     \
                                               cudaStream_t);                                                 \
    template cudaError_t launch_ke_rate<T>(int, int64_t, int64_t, const double *, const T *, const double *,     \
                                           double *, int, cudaStream_t);                                      \
    template cudaError_t launch_wall_force<T>(const Bnd &, const double *, const FieldsT<T> &, const Phys &,      \
                                              double *, int, cudaStream_t);                                   \
    template cudaError_t launch_flux<T>(int, int64_t, int64_t, const T *, T *, const T *, const T *, T *,       \
                                        const Phys &, cudaStream_t, int);                                     \
    template cudaError_t launch_pub_to_int<T>(int, int64_t, int64_t, const double *, double *, cudaStream_t,    \
                                              T *, const double *);                                           \
    template cudaError_t launch_center<T>(int, int64_t, const double *, T *, const double *, cudaStream_t);     \
    template cudaError_t launch_rk_update<T>(int, int64_t, const T *, double *, double *, T *, const double *,   \
                                             double, double, int, int, const T *, const double *, T *,       \
                                             cudaStream_t, int);                                             \
    template cudaError_t launch_rk_2n_update<T>(int, int64_t, const T *, double *, double *, T *,                \
                                                const double *, double, double, double, int, cudaStream_t);  \
    template cudaError_t launch_rk_2r_update<T>(int, int64_t, const T *, double *, double *, T *,                \
                                                const double *, double, double, double, int, int, cudaStream_t); \
    template cudaError_t launch_int_to_pub<T>(int, int64_t, int64_t, const T *, double *, cudaStream_t);       \
    template cudaError_t launch_flux_grouped<T>(const FluxItem<T> *, const int64_t *, int, int64_t, const Phys &, \
                                                int, cudaStream_t, bool);                                     \
    template cudaError_t launch_face_grouped<T>(const FaceItem<T> *, const int64_t *, int, int64_t, const Phys &, \
                                                int, int, cudaStream_t);                                      \
    template cudaError_t launch_center_grouped<T>(const CenterItem<T> *, const int64_t *, int, int64_t, int,     \
                                                  cudaStream_t);
FR_INST(double)
FR_INST(float)
#undef FR_INST

namespace {

constexpr int kRedThreads = 256;

__global__ void k_reduce_partial(int nu, int64_t ne, int64_t np, const double *__restrict__ U,
                                 const double *__restrict__ wJ, double gamma, double *partial) {
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t tot = (int64_t)nu * np;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx / np, e = idx - j * np;
        if (e >= ne) continue;
        const double w = wJ[idx];
        double u[V];
        for (int v = 0; v < V; ++v) {
            u[v] = U[(j * V + v) * np + e];
            acc[v] += w * u[v];
        }
        const double ke = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
        acc[5] += w * ke;
        const double p = (gamma - 1.0) * (u[4] - ke);
        bool bad = !(u[0] > 0.0) || !(p > 0.0);
        for (int v = 0; v < V; ++v) bad = bad || !isfinite(u[v]);
        acc[6] += bad ? 1.0 : 0.0;
    }
    __shared__ double sh[7][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 7; ++q) {
        double x = acc[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double x = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) x += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * 7 + threadIdx.x] = x;
    }
}

__global__ void k_reduce_final(const double *partial, int nblocks, double *out) {
    if (threadIdx.x < 7) {
        double x = 0;
        for (int b = 0; b < nblocks; ++b) x += partial[(int64_t)b * 7 + threadIdx.x];
        out[threadIdx.x] = x;
    }
}

// FP64 FMA throughput probe: 8 independent chains per thread, no memory
// traffic except one store per thread so the chains are not eliminated.
__global__ void k_fma_probe(int iters, double seed, double *sink) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + c + threadIdx.x * 1e-7;
    const double m = 0.999999999, k = 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, k);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}


}  // namespace

cudaError_t launch_reduce_partial(int nu, int64_t ne, int64_t np, const double *U, const double *wJ,
                                  double gamma, double *partial, int nblocks, cudaStream_t s) {
    k_reduce_partial<<<nblocks, kRedThreads, 0, s>>>(nu, ne, np, U, wJ, gamma, partial);
    return cudaGetLastError();
}

cudaError_t probe_fp64(double *gflops, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int threads = 256, blocks = nsm * 8, iters = 4096;
    double *sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(double) * threads * blocks)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_fma_probe<<<blocks, threads, 0, s>>>(iters, 1.0, sink);  // warm-up
    cudaEventRecord(a, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_fma_probe<<<blocks, threads, 0, s>>>(iters, 1.0 + r, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    const double flops = 2.0 * 8.0 * iters * (double)threads * blocks * reps;
    *gflops = ms > 0 ? flops / (ms * 1e-3) / 1e9 : 0.0;
    return e;
}

cudaError_t launch_reduce_final(const double *partial, int nblocks, double *out, cudaStream_t s) {
    k_reduce_final<<<1, 32, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace fr
