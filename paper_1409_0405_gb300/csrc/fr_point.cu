// Point-wise kernels of the FR engine (Sec. 2.1: every non-GEMM operation
// concerns a single solution or flux point): transformed fluxes at solution
// points, LDG common solutions and Rusanov/LDG common normal fluxes at
// interface and boundary flux points, layout conversion and reductions.
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

namespace fr {
namespace {

constexpr int V = 5;
__constant__ double kSdir[3] = {1.0, 0.14142135623730950488, 0.017320508075688772935};

struct Prim {
    double rho, ir, v[3], p;
};

__device__ __forceinline__ Prim prim(const double *u, double gamma) {
    Prim q;
    q.rho = u[0];
    q.ir = 1.0 / u[0];
    q.v[0] = u[1] * q.ir;
    q.v[1] = u[2] * q.ir;
    q.v[2] = u[3] * q.ir;
    q.p = (gamma - 1.0) * (u[4] - 0.5 * (u[1] * q.v[0] + u[2] * q.v[1] + u[3] * q.v[2]));
    return q;
}

// inviscid flux along direction n (unit or not): F(u).n
__device__ __forceinline__ void inv_flux_n(const double *u, const Prim &q, const double *n, double *f) {
    const double vn = q.v[0] * n[0] + q.v[1] * n[1] + q.v[2] * n[2];
    f[0] = u[0] * vn;
    f[1] = u[1] * vn + q.p * n[0];
    f[2] = u[2] * vn + q.p * n[1];
    f[3] = u[3] * vn + q.p * n[2];
    f[4] = (u[4] + q.p) * vn;
}

// physical viscous flux Fv[var][m] from state u (primitives q) and
// conserved gradient g[m][var]
__device__ __forceinline__ void vis_flux(const double *u, const Prim &q, const double g[3][V], const Phys &ph,
                                         double Fv[V][3]) {
    double gv[3][3];  // gv[a][m] = d v_a / d x_m
    double ge[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double gr = g[m][0];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a][m] = (g[m][1 + a] - q.v[a] * gr) * q.ir;
        ge[m] = (g[m][4] - u[4] * q.ir * gr) * q.ir - (q.v[0] * gv[0][m] + q.v[1] * gv[1][m] + q.v[2] * gv[2][m]);
    }
    const double div = gv[0][0] + gv[1][1] + gv[2][2];
    const double kq = ph.mu * ph.gamma / ph.prandtl;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        Fv[0][m] = 0.0;
        double tv = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double t = ph.mu * (gv[a][m] + gv[m][a]);
            if (a == m) t -= (2.0 / 3.0) * ph.mu * div;
            Fv[1 + a][m] = t;
            tv += q.v[a] * t;
        }
        Fv[4][m] = tv + kq * ge[m];
    }
}

__device__ __forceinline__ void rusanov(const double *ua, const double *ub, const double *n, double gamma,
                                        double *f) {
    Prim qa = prim(ua, gamma), qb = prim(ub, gamma);
    double fa[V], fb[V];
    inv_flux_n(ua, qa, n, fa);
    inv_flux_n(ub, qb, n, fb);
    const double vna = qa.v[0] * n[0] + qa.v[1] * n[1] + qa.v[2] * n[2];
    const double vnb = qb.v[0] * n[0] + qb.v[1] * n[1] + qb.v[2] * n[2];
    const double sa = fabs(vna) + sqrt(gamma * qa.p * qa.ir);
    const double sb = fabs(vnb) + sqrt(gamma * qb.p * qb.ir);
    const double s = fmax(sa, sb);
#pragma unroll
    for (int v = 0; v < V; ++v) f[v] = 0.5 * (fa[v] + fb[v]) - 0.5 * s * (ub[v] - ua[v]);
}

// boundary states: inviscid ghost and common solution
__device__ __forceinline__ void bc_states(int tag, const double *u, const double *n, const Phys &ph,
                                          double *ghost, double *cb) {
    const double g = ph.gamma;
    if (tag == FR_BC_WALL) {
        const double ew = ph.t_wall / (g - 1.0);
        const double ke = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
        ghost[0] = u[0];
        ghost[1] = -u[1];
        ghost[2] = -u[2];
        ghost[3] = -u[3];
        ghost[4] = u[0] * ew + ke;
        cb[0] = u[0];
        cb[1] = 0.0;
        cb[2] = 0.0;
        cb[3] = 0.0;
        cb[4] = u[0] * ew;
        return;
    }
    // Riemann-invariant far field.  With R+ = vn + 2c/(g-1) from the
    // interior and R- = vn_inf - 2c_inf/(g-1) from the far field,
    //   vn_b = (R+ + R-)/2,  c_b = (g-1)(R+ - R-)/4,
    // written without forming R+- (|R+-| ~ 2c/(g-1) >> vn would cancel),
    // and the density from the upwind entropy p/rho^g, written as
    //   rho_b = rho_up (c_b / c_up)^(2/(g-1)).
    Prim q = prim(u, g);
    const double c = sqrt(g * q.p * q.ir);
    const double cinf = sqrt(g * ph.p_inf / ph.rho_inf);
    const double vn = q.v[0] * n[0] + q.v[1] * n[1] + q.v[2] * n[2];
    const double vninf = ph.vinf[0] * n[0] + ph.vinf[1] * n[1] + ph.vinf[2] * n[2];
    const double vnb = 0.5 * (vn + vninf) + (c - cinf) / (g - 1.0);
    const double cbs = 0.5 * (c + cinf) + 0.25 * (g - 1.0) * (vn - vninf);
    double vb[3], rhob;
    const double ex = 2.0 / (g - 1.0);
    if (vnb >= 0.0) {
        rhob = q.rho * pow(cbs / c, ex);
        for (int k = 0; k < 3; ++k) vb[k] = q.v[k] + (vnb - vn) * n[k];
    } else {
        rhob = ph.rho_inf * pow(cbs / cinf, ex);
        for (int k = 0; k < 3; ++k) vb[k] = ph.vinf[k] + (vnb - vninf) * n[k];
    }
    const double pb = rhob * cbs * cbs / g;
    ghost[0] = rhob;
    ghost[1] = rhob * vb[0];
    ghost[2] = rhob * vb[1];
    ghost[3] = rhob * vb[2];
    ghost[4] = pb / (g - 1.0) + 0.5 * rhob * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
    for (int v = 0; v < V; ++v) cb[v] = ghost[v];
}

__device__ __forceinline__ int64_t fpt_off(int f, int e, int64_t np) { return (int64_t)f * V * np + e; }

// ---------------------------------------------------------------------------
__global__ void k_common_solution(const Pairs P, const Bnd B, const Fields F, const Phys ph) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) {
        const int ta = P.ta[k], tb = P.tb[k];
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int64_t oa = fpt_off(P.fa[k], P.ea[k], npa), ob = fpt_off(P.fb[k], P.eb[k], npb);
        const double *UA = F.UF[ta] + oa, *UB = F.UF[tb] + ob;
        const double *n = P.nrm + 3 * k;
        const double sig = (n[0] * kSdir[0] + n[1] * kSdir[1] + n[2] * kSdir[2] > 0.0) ? 1.0 : -1.0;
        const double b = ph.beta * sig;
        double *DA = F.DUF[ta] + oa, *DB = F.DUF[tb] + ob;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double ua = UA[v * npa], ub = UB[v * npb];
            const double C = 0.5 * (ua + ub) + b * (ua - ub);
            DA[v * npa] = C - ua;
            DB[v * npb] = C - ub;
        }
        return;
    }
    const int64_t kb = k - P.n;
    if (kb < B.n) {
        const int t = B.bt[kb];
        const int64_t np = F.np[t];
        const int64_t o = fpt_off(B.bf[kb], B.be[kb], np);
        double u[V], ghost[V], cb[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = F.UF[t][o + v * np];
        bc_states(B.btag[kb], u, B.bn + 3 * kb, ph, ghost, cb);
#pragma unroll
        for (int v = 0; v < V; ++v) F.DUF[t][o + v * np] = cb[v] - u[v];
    }
}

__device__ __forceinline__ void load_grad(const double *G, int f, int e, int64_t np, double g[3][V]) {
    const double *p = G + (int64_t)f * 3 * V * np + e;
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int v = 0; v < V; ++v) g[m][v] = p[(m * V + v) * np];
}

__global__ void k_common_flux(const Pairs P, const Bnd B, const Fields F, const Phys ph) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) {
        const int ta = P.ta[k], tb = P.tb[k];
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int fa = P.fa[k], fb = P.fb[k], ea = P.ea[k], eb = P.eb[k];
        const int64_t oa = fpt_off(fa, ea, npa), ob = fpt_off(fb, eb, npb);
        double ua[V], ub[V], fn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            ua[v] = F.UF[ta][oa + v * npa];
            ub[v] = F.UF[tb][ob + v * npb];
        }
        const double n[3] = {P.nrm[3 * k], P.nrm[3 * k + 1], P.nrm[3 * k + 2]};
        rusanov(ua, ub, n, ph.gamma, fn);
        if (ph.viscous) {
            double ga[3][V], gb[3][V], Fa[V][3], Fb[V][3];
            load_grad(F.GUF[ta], fa, ea, npa, ga);
            load_grad(F.GUF[tb], fb, eb, npb, gb);
            Prim qa = prim(ua, ph.gamma), qb = prim(ub, ph.gamma);
            vis_flux(ua, qa, ga, ph, Fa);
            vis_flux(ub, qb, gb, ph, Fb);
            const double sig = (n[0] * kSdir[0] + n[1] * kSdir[1] + n[2] * kSdir[2] > 0.0) ? 1.0 : -1.0;
            const double b = ph.beta * sig;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const double fva = Fa[v][0] * n[0] + Fa[v][1] * n[1] + Fa[v][2] * n[2];
                const double fvb = Fb[v][0] * n[0] + Fb[v][1] * n[1] + Fb[v][2] * n[2];
                fn[v] = fn[v] - (0.5 * (fva + fvb) - b * (fva - fvb)) + ph.tau * (ua[v] - ub[v]);
            }
        }
        const double ma = P.maga[k], mb = P.magb[k];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const double f = fn[v] - (ph.fref[v][0] * n[0] + ph.fref[v][1] * n[1] + ph.fref[v][2] * n[2]);
            F.FC[ta][oa + v * npa] = f * ma;
            F.FC[tb][ob + v * npb] = -f * mb;
        }
        return;
    }
    const int64_t kb = k - P.n;
    if (kb < B.n) {
        const int t = B.bt[kb];
        const int64_t np = F.np[t];
        const int f = B.bf[kb], e = B.be[kb];
        const int64_t o = fpt_off(f, e, np);
        double u[V], ghost[V], cb[V], fn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = F.UF[t][o + v * np];
        const double n[3] = {B.bn[3 * kb], B.bn[3 * kb + 1], B.bn[3 * kb + 2]};
        bc_states(B.btag[kb], u, n, ph, ghost, cb);
        rusanov(u, ghost, n, ph.gamma, fn);
        if (ph.viscous) {
            double g[3][V], Fv[V][3];
            load_grad(F.GUF[t], f, e, np, g);
            Prim qc = prim(cb, ph.gamma);
            vis_flux(cb, qc, g, ph, Fv);
#pragma unroll
            for (int v = 0; v < V; ++v)
                fn[v] = fn[v] - (Fv[v][0] * n[0] + Fv[v][1] * n[1] + Fv[v][2] * n[2]) + ph.tau * (u[v] - cb[v]);
        }
        const double mg = B.bmag[kb];
#pragma unroll
        for (int v = 0; v < V; ++v)
            F.FC[t][o + v * np] = (fn[v] - (ph.fref[v][0] * n[0] + ph.fref[v][1] * n[1] + ph.fref[v][2] * n[2])) * mg;
    }
}

// transformed flux F~_d = sum_m S[d][m] (F_inv - F_vis)_m at solution points
__global__ void k_flux(int nu, int64_t ne, int64_t np, const double *__restrict__ U,
                       const double *__restrict__ GU, const double *__restrict__ S, double *__restrict__ FT,
                       const Phys ph) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = idx / np, e = idx - j * np;
    if (j >= nu || e >= ne) return;
    double u[V];
#pragma unroll
    for (int v = 0; v < V; ++v) u[v] = U[(j * V + v) * np + e] + ph.uref[v];
    const Prim q = prim(u, ph.gamma);
    double F[V][3];
    // inviscid
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        F[0][m] = u[1 + m];
#pragma unroll
        for (int a = 0; a < 3; ++a) F[1 + a][m] = u[1 + a] * q.v[m] + (a == m ? q.p : 0.0);
        F[4][m] = (u[4] + q.p) * q.v[m];
    }
    if (ph.viscous) {
        double g[3][V], Fv[V][3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int v = 0; v < V; ++v) g[m][v] = GU[((j * 3 + m) * V + v) * np + e];
        vis_flux(u, q, g, ph, Fv);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int m = 0; m < 3; ++m) F[v][m] -= Fv[v][m];
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int m = 0; m < 3; ++m) F[v][m] -= ph.fref[v][m];
    double s[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s[k] = S[(j * 9 + k) * np + e];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v)
            FT[((j * 3 + d) * V + v) * np + e] = s[d * 3 + 0] * F[v][0] + s[d * 3 + 1] * F[v][1] + s[d * 3 + 2] * F[v][2];
}

struct Uref {
    double v[5];
};

__global__ void k_const_flux(int nu, int64_t ne, int64_t np, const double *__restrict__ S,
                             double *__restrict__ FT, const Phys ph) {
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

__global__ void k_const_common(const Pairs P, const Bnd B, const Fields F, const Phys ph) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) {
        const int ta = P.ta[k], tb = P.tb[k];
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int64_t oa = fpt_off(P.fa[k], P.ea[k], npa), ob = fpt_off(P.fb[k], P.eb[k], npb);
        const double *n = P.nrm + 3 * k;
        for (int v = 0; v < V; ++v) {
            const double f = ph.fref[v][0] * n[0] + ph.fref[v][1] * n[1] + ph.fref[v][2] * n[2];
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
        for (int v = 0; v < V; ++v)
            F.FC[t][o + v * np] = (ph.fref[v][0] * n[0] + ph.fref[v][1] * n[1] + ph.fref[v][2] * n[2]) * B.bmag[kb];
    }
}

__global__ void k_pub_to_int(int nu, int64_t ne, int64_t np, const double *__restrict__ pub,
                             double *__restrict__ in, double *__restrict__ centred, const Uref uref) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = ne * V * nu;
    if (idx >= tot) return;
    const int64_t e = idx / (V * nu);
    const int64_t r = idx - e * V * nu;
    const int64_t v = r / nu, j = r - v * nu;
    const double x = pub[idx];
    if (in) in[(j * V + v) * np + e] = x;
    if (centred) centred[(j * V + v) * np + e] = x - uref.v[v];
}

__global__ void k_center(int64_t n, int64_t np, const double *__restrict__ U, double *__restrict__ Us,
                         const Uref uref) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int64_t v = (idx / np) % V;
    Us[idx] = U[idx] - uref.v[v];
}

__global__ void k_int_to_pub(int nu, int64_t ne, int64_t np, const double *__restrict__ in,
                             double *__restrict__ pub) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = ne * V * nu;
    if (idx >= tot) return;
    const int64_t e = idx / (V * nu);
    const int64_t r = idx - e * V * nu;
    const int64_t v = r / nu, j = r - v * nu;
    pub[idx] = in[(j * V + v) * np + e];
}

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

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

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

cudaError_t launch_common_solution(const Pairs &P, const Bnd &B, const Fields &F, const Phys &ph,
                                   cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_common_solution<<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, ph);
    return cudaGetLastError();
}

cudaError_t launch_common_flux(const Pairs &P, const Bnd &B, const Fields &F, const Phys &ph,
                               cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_common_flux<<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, ph);
    return cudaGetLastError();
}

cudaError_t launch_flux(int nu, int64_t ne, int64_t np, const double *U, const double *GU, const double *S,
                        double *FT, const Phys &ph, cudaStream_t s) {
    const int64_t n = (int64_t)nu * np;
    if (ne == 0) return cudaSuccess;
    k_flux<<<blocks_for(n, 128), 128, 0, s>>>(nu, ne, np, U, GU, S, FT, ph);
    return cudaGetLastError();
}

cudaError_t launch_pub_to_int(int nu, int64_t ne, int64_t np, const double *pub, double *in, cudaStream_t s,
                              double *centred, const double *uref) {
    const int64_t n = ne * V * nu;
    if (n == 0) return cudaSuccess;
    Uref r{{0, 0, 0, 0, 0}};
    if (uref)
        for (int v = 0; v < V; ++v) r.v[v] = uref[v];
    k_pub_to_int<<<blocks_for(n, 256), 256, 0, s>>>(nu, ne, np, pub, in, centred, r);
    return cudaGetLastError();
}

cudaError_t launch_const_flux(int nu, int64_t ne, int64_t np, const double *S, double *FT, const Phys &ph,
                              cudaStream_t s) {
    const int64_t n = (int64_t)nu * np;
    if (ne == 0) return cudaSuccess;
    k_const_flux<<<blocks_for(n, 128), 128, 0, s>>>(nu, ne, np, S, FT, ph);
    return cudaGetLastError();
}

cudaError_t launch_const_common(const Pairs &P, const Bnd &B, const Fields &F, const Phys &ph, cudaStream_t s) {
    const int64_t n = P.n + B.n;
    if (n == 0) return cudaSuccess;
    k_const_common<<<blocks_for(n, 128), 128, 0, s>>>(P, B, F, ph);
    return cudaGetLastError();
}

cudaError_t launch_center(int nu, int64_t np, const double *U, double *Us, const double *uref, cudaStream_t s) {
    const int64_t n = (int64_t)nu * V * np;
    if (n == 0) return cudaSuccess;
    Uref r{{uref[0], uref[1], uref[2], uref[3], uref[4]}};
    k_center<<<blocks_for(n, 256), 256, 0, s>>>(n, np, U, Us, r);
    return cudaGetLastError();
}

cudaError_t launch_int_to_pub(int nu, int64_t ne, int64_t np, const double *in, double *pub, cudaStream_t s) {
    const int64_t n = ne * V * nu;
    if (n == 0) return cudaSuccess;
    k_int_to_pub<<<blocks_for(n, 256), 256, 0, s>>>(nu, ne, np, in, pub);
    return cudaGetLastError();
}

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
