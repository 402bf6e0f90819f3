// Point-wise device functions of the FR right-hand side (physics, LDG and
// Rusanov interface values, boundary states, the transformed flux at a
// solution point), shared by the point-wise kernels (fr_point.cu) and the
// batched engine's persistent stage kernel (fr_stage.cu).  Internal; the
// physics and interface conventions are stated in fr_point.cu.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/fr.h"
#include "fr_kernels.h"

namespace fr {
namespace {

constexpr int V = 5;

template <typename T>
struct Prim {
    T rho, ir, v[3], p;
};

template <typename T>
__device__ __forceinline__ Prim<T> prim(const T *u, T gamma) {
    Prim<T> q;
    q.rho = u[0];
    q.ir = T(1) / u[0];
    q.v[0] = u[1] * q.ir;
    q.v[1] = u[2] * q.ir;
    q.v[2] = u[3] * q.ir;
    q.p = (gamma - T(1)) * (u[4] - T(0.5) * (u[1] * q.v[0] + u[2] * q.v[1] + u[3] * q.v[2]));
    return q;
}

// inviscid flux along direction n: F(u).n
template <typename T>
__device__ __forceinline__ void inv_flux_n(const T *u, const Prim<T> &q, const T *n, T *f) {
    const T vn = q.v[0] * n[0] + q.v[1] * n[1] + q.v[2] * n[2];
    f[0] = u[0] * vn;
    f[1] = u[1] * vn + q.p * n[0];
    f[2] = u[2] * vn + q.p * n[1];
    f[3] = u[3] * vn + q.p * n[2];
    f[4] = (u[4] + q.p) * vn;
}

// physical viscous flux Fv[var][m] from state u (primitives q) and
// conserved gradient g[m][var]
template <typename T>
__device__ __forceinline__ void vis_flux(const T *u, const Prim<T> &q, const T g[3][V], T mu, T kq, T Fv[V][3]) {
    T gv[3][3];  // gv[a][m] = d v_a / d x_m
    T ge[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T gr = g[m][0];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a][m] = (g[m][1 + a] - q.v[a] * gr) * q.ir;
        ge[m] = (g[m][4] - u[4] * q.ir * gr) * q.ir - (q.v[0] * gv[0][m] + q.v[1] * gv[1][m] + q.v[2] * gv[2][m]);
    }
    const T div = gv[0][0] + gv[1][1] + gv[2][2];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        Fv[0][m] = T(0);
        T tv = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T t = mu * (gv[a][m] + gv[m][a]);
            if (a == m) t -= T(2.0 / 3.0) * mu * div;
            Fv[1 + a][m] = t;
            tv += q.v[a] * t;
        }
        Fv[4][m] = tv + kq * ge[m];
    }
}

// normal viscous flux F_vis(u, grad u) . n directly (the 3-vector
// tau . n and the energy entry), without forming the full tensor:
//   (tau n)_a = mu (dv_a/dn + sum_m (dv_m/dx_a) n_m - 2/3 div v n_a),
//   energy = v . (tau n) + mu gamma/Pr grad e . n
template <typename T>
__device__ __forceinline__ void vis_flux_n(const T *u, const Prim<T> &q, const T g[3][V], T mu, T kq, const T *n,
                                           T *fn) {
    T gv[3][3];  // gv[a][m] = d v_a / d x_m
    T gen = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T gr = g[m][0];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a][m] = (g[m][1 + a] - q.v[a] * gr) * q.ir;
        const T ge = (g[m][4] - u[4] * q.ir * gr) * q.ir - (q.v[0] * gv[0][m] + q.v[1] * gv[1][m] + q.v[2] * gv[2][m]);
        gen += ge * n[m];
    }
    const T div = gv[0][0] + gv[1][1] + gv[2][2];
    T tv = T(0);
    fn[0] = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T dn = gv[a][0] * n[0] + gv[a][1] * n[1] + gv[a][2] * n[2];
        const T tn = gv[0][a] * n[0] + gv[1][a] * n[1] + gv[2][a] * n[2];
        const T t = mu * (dn + tn - T(2.0 / 3.0) * div * n[a]);
        fn[1 + a] = t;
        tv += q.v[a] * t;
    }
    fn[4] = tv + kq * gen;
}

template <typename T>
__device__ __forceinline__ void rusanov_q(const T *ua, const T *ub, const Prim<T> &qa, const Prim<T> &qb, const T *n,
                                          T gamma, T *f) {
    T fa[V], fb[V];
    inv_flux_n(ua, qa, n, fa);
    inv_flux_n(ub, qb, n, fb);
    const T vna = qa.v[0] * n[0] + qa.v[1] * n[1] + qa.v[2] * n[2];
    const T vnb = qb.v[0] * n[0] + qb.v[1] * n[1] + qb.v[2] * n[2];
    const T sa = fabs(vna) + sqrt(gamma * qa.p * qa.ir);
    const T sb = fabs(vnb) + sqrt(gamma * qb.p * qb.ir);
    const T s = fmax(sa, sb);
#pragma unroll
    for (int v = 0; v < V; ++v) f[v] = T(0.5) * (fa[v] + fb[v]) - T(0.5) * s * (ub[v] - ua[v]);
}

// Rusanov flux from the two states (primitives formed here)
template <typename T>
__device__ __forceinline__ void rusanov(const T *ua, const T *ub, const T *n, T gamma, T *f) {
    rusanov_q(ua, ub, prim(ua, gamma), prim(ub, gamma), n, gamma, f);
}

template <typename T>
struct PhysT {
    T gamma, mu, kq, beta, tau, rho_inf, vinf[3], p_inf, ew, cinf, ex;
    T fref[V][3];
    T uref[V];
    int viscous;
};

template <typename T>
PhysT<T> phys_t(const Phys &p) {
    PhysT<T> q;
    q.gamma = T(p.gamma);
    q.mu = T(p.mu);
    q.kq = T(p.mu * p.gamma / p.prandtl);
    q.beta = T(p.beta);
    q.tau = T(p.tau);
    q.rho_inf = T(p.rho_inf);
    for (int k = 0; k < 3; ++k) q.vinf[k] = T(p.vinf[k]);
    q.p_inf = T(p.p_inf);
    q.ew = T(p.t_wall / (p.gamma - 1.0));
    q.cinf = T(std::sqrt(p.gamma * p.p_inf / p.rho_inf));
    q.ex = T(2.0 / (p.gamma - 1.0));
    for (int v = 0; v < V; ++v) {
        for (int m = 0; m < 3; ++m) q.fref[v][m] = T(p.fref[v][m]);
        q.uref[v] = T(p.uref[v]);
    }
    q.viscous = p.viscous;
    return q;
}

// boundary states: inviscid ghost and common solution
template <typename T>
__device__ __forceinline__ void bc_states(int tag, const T *u, const T *n, const PhysT<T> &ph, T *ghost, T *cb) {
    const T g = ph.gamma;
    if (tag == FR_BC_WALL) {
        const T ke = T(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
        ghost[0] = u[0];
        ghost[1] = -u[1];
        ghost[2] = -u[2];
        ghost[3] = -u[3];
        ghost[4] = u[0] * ph.ew + ke;
        cb[0] = u[0];
        cb[1] = T(0);
        cb[2] = T(0);
        cb[3] = T(0);
        cb[4] = u[0] * ph.ew;
        return;
    }
    // Riemann-invariant far field.  With R+ = vn + 2c/(g-1) from the
    // interior and R- = vn_inf - 2c_inf/(g-1) from the far field,
    //   vn_b = (R+ + R-)/2,  c_b = (g-1)(R+ - R-)/4,
    // written without forming R+- (|R+-| ~ 2c/(g-1) >> vn would cancel),
    // and the density from the upwind entropy p/rho^g, written as
    //   rho_b = rho_up (c_b / c_up)^(2/(g-1)).
    Prim<T> q = prim(u, g);
    const T c = sqrt(g * q.p * q.ir);
    const T vn = q.v[0] * n[0] + q.v[1] * n[1] + q.v[2] * n[2];
    const T vninf = ph.vinf[0] * n[0] + ph.vinf[1] * n[1] + ph.vinf[2] * n[2];
    const T vnb = T(0.5) * (vn + vninf) + (c - ph.cinf) / (g - T(1));
    const T cbs = T(0.5) * (c + ph.cinf) + T(0.25) * (g - T(1)) * (vn - vninf);
    T vb[3], rhob;
    if (vnb >= T(0)) {
        rhob = q.rho * pow(cbs / c, ph.ex);
        for (int k = 0; k < 3; ++k) vb[k] = q.v[k] + (vnb - vn) * n[k];
    } else {
        rhob = ph.rho_inf * pow(cbs / ph.cinf, ph.ex);
        for (int k = 0; k < 3; ++k) vb[k] = ph.vinf[k] + (vnb - vninf) * n[k];
    }
    const T pb = rhob * cbs * cbs / g;
    ghost[0] = rhob;
    ghost[1] = rhob * vb[0];
    ghost[2] = rhob * vb[1];
    ghost[3] = rhob * vb[2];
    ghost[4] = pb / (g - T(1)) + T(0.5) * rhob * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
    for (int v = 0; v < V; ++v) cb[v] = ghost[v];
}

__device__ __forceinline__ int64_t fpt_off(int f, int e, int64_t np) { return (int64_t)f * V * np + e; }

// Face metadata in the arithmetic type: the FP32-storage modes read the
// float copies (no conversions on the FP64 pipe), FP64 the doubles.  The
// LDG switch (+1 where side a's outward normal n has n . s > 0, s = (1,
// 0.1 sqrt 2, 0.01 sqrt 3)) is evaluated once on the host in double.
template <typename T>
__device__ __forceinline__ void pair_normal(const Pairs &P, int64_t k, T *n);
template <>
__device__ __forceinline__ void pair_normal<double>(const Pairs &P, int64_t k, double *n) {
    n[0] = P.nrm[3 * k];
    n[1] = P.nrm[3 * k + 1];
    n[2] = P.nrm[3 * k + 2];
}
template <>
__device__ __forceinline__ void pair_normal<float>(const Pairs &P, int64_t k, float *n) {
    n[0] = P.nrm_f[3 * k];
    n[1] = P.nrm_f[3 * k + 1];
    n[2] = P.nrm_f[3 * k + 2];
}
template <typename T>
__device__ __forceinline__ void pair_mags(const Pairs &P, int64_t k, T &ma, T &mb);
template <>
__device__ __forceinline__ void pair_mags<double>(const Pairs &P, int64_t k, double &ma, double &mb) {
    ma = P.maga[k];
    mb = P.magb[k];
}
template <>
__device__ __forceinline__ void pair_mags<float>(const Pairs &P, int64_t k, float &ma, float &mb) {
    ma = P.maga_f[k];
    mb = P.magb_f[k];
}
template <typename T>
__device__ __forceinline__ void bnd_normal(const Bnd &B, int64_t kb, T *n, T &mag);
template <>
__device__ __forceinline__ void bnd_normal<double>(const Bnd &B, int64_t kb, double *n, double &mag) {
    n[0] = B.bn[3 * kb];
    n[1] = B.bn[3 * kb + 1];
    n[2] = B.bn[3 * kb + 2];
    mag = B.bmag[kb];
}
template <>
__device__ __forceinline__ void bnd_normal<float>(const Bnd &B, int64_t kb, float *n, float &mag) {
    n[0] = B.bn_f[3 * kb];
    n[1] = B.bn_f[3 * kb + 1];
    n[2] = B.bn_f[3 * kb + 2];
    mag = B.bmag_f[kb];
}

// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void common_solution_at(const Pairs &P, const Bnd &B, const FieldsT<T> &F,
                                                   const PhysT<T> &ph, int64_t k) {
    if (k < P.n) {
        const PairSides ps = pair_sides(P.code[k]);
        const int ta = ps.ta, tb = ps.tb;
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int64_t oa = fpt_off(ps.fa, P.ea[k], npa), ob = fpt_off(ps.fb, P.eb[k], npb);
        const T *UA = F.UF[ta] + oa, *UB = F.UF[tb] + ob;
        const T b = ph.beta * T(ps.sgn);
        T *DA = F.DUF[ta] + oa, *DB = F.DUF[tb] + ob;
        if (ph.beta == T(0.5)) {
            // beta = 1/2: the common solution is side a's value where the
            // switch is +1, else side b's, so that side's jump is exactly
            // zero.  The switch is fixed by the geometry and every interior
            // flux point belongs to one pair, so that slot keeps the zero it
            // was allocated with: only the other side's jump is written
            const bool sa = ps.sgn > 0;
            T *D = sa ? DB : DA;
            const int64_t npd = sa ? npb : npa;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T ua = UA[v * npa], ub = UB[v * npb];
                D[v * npd] = sa ? ua - ub : ub - ua;
            }
            return;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T ua = UA[v * npa], ub = UB[v * npb];
            const T C = T(0.5) * (ua + ub) + b * (ua - ub);
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
        T u[V], ghost[V], cb[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = F.UF[t][o + v * np];
        T n[3], mg;
        bnd_normal<T>(B, kb, n, mg);
        bc_states(B.btag[kb], u, n, ph, ghost, cb);
#pragma unroll
        for (int v = 0; v < V; ++v) F.DUF[t][o + v * np] = cb[v] - u[v];
    }
}

template <typename T>
__device__ __forceinline__ void load_grad(const T *G, int f, int e, int64_t np, T g[3][V]) {
    const T *p = G + (int64_t)f * 3 * V * np + e;
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int v = 0; v < V; ++v) g[m][v] = p[(m * V + v) * np];
}

template <typename T>
__device__ __forceinline__ T fref_n(const PhysT<T> &ph, int v, const T *n) {
    return ph.fref[v][0] * n[0] + ph.fref[v][1] * n[1] + ph.fref[v][2] * n[2];
}

// VIS: 0 = viscous terms as ph.viscous says (run time), 1 = inviscid, 2 =
// viscous (known at compile time: the other branch is not compiled)
template <typename T, int VIS = 0>
__device__ __forceinline__ void common_flux_at(const Pairs &P, const Bnd &B, const FieldsT<T> &F, const PhysT<T> &ph,
                                               int64_t k) {
    if (k < P.n) {
        const PairSides ps = pair_sides(P.code[k]);
        const int ta = ps.ta, tb = ps.tb;
        const int64_t npa = F.np[ta], npb = F.np[tb];
        const int fa = ps.fa, fb = ps.fb, ea = P.ea[k], eb = P.eb[k];
        const int64_t oa = fpt_off(fa, ea, npa), ob = fpt_off(fb, eb, npb);
        T ua[V], ub[V], fn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            ua[v] = F.UF[ta][oa + v * npa];
            ub[v] = F.UF[tb][ob + v * npb];
        }
        T n[3];
        pair_normal<T>(P, k, n);
        // primitives once per side, for the Rusanov and the viscous flux
        const Prim<T> qa = prim(ua, ph.gamma), qb = prim(ub, ph.gamma);
        rusanov_q(ua, ub, qa, qb, n, ph.gamma, fn);
        if (VIS == 0 ? ph.viscous != 0 : VIS == 2) {
            if (ph.beta == T(0.5)) {
                // beta = 1/2: the weights 1/2 -+ beta sgn of the two sides'
                // viscous fluxes are 0 and 1, so the common viscous flux is
                // the flux of one side (b where the switch is +1, else a):
                // only that side's gradient is read and its flux formed
                const bool sb = ps.sgn > 0;
                T g[3][V], fv[V];
                load_grad(F.GUF[sb ? tb : ta], sb ? fb : fa, sb ? eb : ea, sb ? npb : npa, g);
                vis_flux_n(sb ? ub : ua, sb ? qb : qa, g, ph.mu, ph.kq, n, fv);
#pragma unroll
                for (int v = 0; v < V; ++v) fn[v] = fn[v] - fv[v] + ph.tau * (ua[v] - ub[v]);
            } else {
                T ga[3][V], gb[3][V], fva[V], fvb[V];
                load_grad(F.GUF[ta], fa, ea, npa, ga);
                load_grad(F.GUF[tb], fb, eb, npb, gb);
                vis_flux_n(ua, qa, ga, ph.mu, ph.kq, n, fva);
                vis_flux_n(ub, qb, gb, ph.mu, ph.kq, n, fvb);
                const T b = ph.beta * T(ps.sgn);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    fn[v] = fn[v] - (T(0.5) * (fva[v] + fvb[v]) - b * (fva[v] - fvb[v])) + ph.tau * (ua[v] - ub[v]);
            }
        }
        T ma, mb;
        pair_mags<T>(P, k, ma, mb);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T f = fn[v] - fref_n(ph, v, n);
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
        T u[V], ghost[V], cb[V], fn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = F.UF[t][o + v * np];
        T n[3], mg;
        bnd_normal<T>(B, kb, n, mg);
        bc_states(B.btag[kb], u, n, ph, ghost, cb);
        rusanov(u, ghost, n, ph.gamma, fn);
        if (VIS == 0 ? ph.viscous != 0 : VIS == 2) {
            T g[3][V], fv[V];
            load_grad(F.GUF[t], f, e, np, g);
            Prim<T> qc = prim(cb, ph.gamma);
            vis_flux_n(cb, qc, g, ph.mu, ph.kq, n, fv);
#pragma unroll
            for (int v = 0; v < V; ++v) fn[v] = fn[v] - fv[v] + ph.tau * (u[v] - cb[v]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) F.FC[t][o + v * np] = (fn[v] - fref_n(ph, v, n)) * mg;
    }
}

// transformed flux F~_d = sum_m S[d][m] (F_inv - F_vis - F_ref)_m at solution points.
// XFORM: GU holds the reference gradient g^_d on entry (rows (j, d)); the
// physical gradient grad_m u = (1/J) sum_d S[d][m] g^_d is formed here,
// written back over it (in place: one thread owns the point's 15 values) and
// used for the viscous flux.  gj: 1 = S [nu][9][np] and 1/J [nu][np] per
// point, 0 = one value per element ([9][np], [np]; elements whose geometry
// factors are the same at every point)
template <typename T, bool XFORM, int VIS = 0>
__device__ __forceinline__ void flux_at(int nu, int64_t ne, int64_t np, const T *__restrict__ U,
                                        T *__restrict__ GU, const T *__restrict__ S, const T *__restrict__ invJ,
                                        T *__restrict__ FT, const PhysT<T> &ph, int64_t j, int64_t e, int gj = 1) {
    if (j >= nu || e >= ne) return;
    const int64_t jg = j * gj;
    T u[V];
#pragma unroll
    for (int v = 0; v < V; ++v) u[v] = U[(j * V + v) * np + e] + ph.uref[v];
    T s[9];
    if (XFORM) {
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = S[(jg * 9 + k) * np + e];
    }
    const Prim<T> q = prim(u, ph.gamma);
    T F[V][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        F[0][m] = u[1 + m];
#pragma unroll
        for (int a = 0; a < 3; ++a) F[1 + a][m] = u[1 + a] * q.v[m] + (a == m ? q.p : T(0));
        F[4][m] = (u[4] + q.p) * q.v[m];
    }
    if (VIS == 0 ? ph.viscous != 0 : VIS == 2) {
        T g[3][V], Fv[V][3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int v = 0; v < V; ++v) g[m][v] = GU[((j * 3 + m) * V + v) * np + e];
        if (XFORM) {
            const T ij = invJ[jg * np + e];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T g0 = g[0][v], g1 = g[1][v], g2 = g[2][v];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    g[m][v] = ij * (s[m] * g0 + s[3 + m] * g1 + s[6 + m] * g2);
                    GU[((j * 3 + m) * V + v) * np + e] = g[m][v];
                }
            }
        }
        vis_flux(u, q, g, ph.mu, ph.kq, Fv);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int m = 0; m < 3; ++m) F[v][m] -= Fv[v][m];
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int m = 0; m < 3; ++m) F[v][m] -= ph.fref[v][m];
    if (!XFORM) {
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = S[(jg * 9 + k) * np + e];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v)
            FT[((j * 3 + d) * V + v) * np + e] = s[d * 3 + 0] * F[v][0] + s[d * 3 + 1] * F[v][1] + s[d * 3 + 2] * F[v][2];
}

__device__ __forceinline__ int find_item(const int64_t *begin, int n, int64_t gi) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= gi) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}


}  // namespace
}  // namespace fr
