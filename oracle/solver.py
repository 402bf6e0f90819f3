"""The oracle's FR right-hand side, RK4 stepper and reductions.

Public state layout (shared with the C ABI): one flat float64 array, tets
first then prisms, each block [elem][var][upt].

RHS (reference-space FR with the DG correction; Sec. 2.1 casts every
operator application as C <- c1 A B + c2 C, Eq. 1):
  1. u_f = M0 u                                   (Table 2's M0)
  2. NS: common solution C at every flux point, Delta = C - u_f
  3. NS: corrected reference gradient  g_d = D_d u + M3 (n^_d Delta),
     physical gradient  grad_m u = (1/J) sum_d S[d][m] g_d
  4. NS: gradient at flux points  M0 grad_m u
  5. transformed flux at solution points  F~_d = sum_m S[d][m] F_m(u, grad u)
  6. common transformed normal flux at flux points  F~c = F_c.n |S^T n^|
  7. R = -(1/J) [ sum_d D_d F~_d + M3 (F~c - sum_d n^_d M0 F~_d) ]
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import physics
from .mesh import Mesh

NVARS = 5

# Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage
# Runge-Kutta: the published rational coefficients (A_i, B_i)
RK4_2N_FRACTIONS = (
    (Fraction(0), Fraction(-567301805773, 1357537059087), Fraction(-2404267990393, 2016746695238),
     Fraction(-3550918686646, 2091501179385), Fraction(-1275806237668, 842570457699)),
    (Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
     Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
     Fraction(2277821191437, 14882151754819)))
RK4_2N_A = [float(x) for x in RK4_2N_FRACTIONS[0]]
RK4_2N_B = [float(x) for x in RK4_2N_FRACTIONS[1]]

# RK45[2R+], the time stepper of the paper's runs (Sec. 3.4; Table 1 lists
# RK45): the five-stage fourth-order scheme RK4(3)5[2R+]C of Kennedy,
# Carpenter & Lewis (2000), with an embedded third-order solution.  Its
# Butcher matrix has the two-register structure A[i][i-1] = a_i and
# A[i][j] = b_j for j < i-1, so only the sub-diagonal a_1..a_4, the weights
# b_1..b_5 and the embedded weights bhat_1..bhat_5 are free.  The published
# rational approximations of those coefficients:
RK45_2R_FRACTIONS = (
    (Fraction(970286171893, 4311952581923), Fraction(6584761158862, 12103376702013),
     Fraction(2251764453980, 15575788980749), Fraction(26877169314380, 34165994151039)),
    (Fraction(1153189308089, 22510343858157), Fraction(1772645290293, 4653164025191),
     Fraction(-1672844663538, 4480602732383), Fraction(2114624349019, 3568978502595),
     Fraction(5198255086312, 14908931495163)),
    (Fraction(1016888040809, 7410784769900), Fraction(11231460423587, 58533540763752),
     Fraction(-1563879915014, 6823010717585), Fraction(606302364029, 971179775848),
     Fraction(1097981568119, 3980877426909)))
RK45_2R_A = [float(x) for x in RK45_2R_FRACTIONS[0]]
RK45_2R_B = [float(x) for x in RK45_2R_FRACTIONS[1]]
RK45_2R_BHAT = [float(x) for x in RK45_2R_FRACTIONS[2]]
# b - bhat in double: the weights of the embedded error estimate
RK45_2R_E = [float(b - bh) for b, bh in zip(RK45_2R_FRACTIONS[1], RK45_2R_FRACTIONS[2])]


def rk45_2r_step(rhs, u, dt, a=None, b=None, e=None):
    """One RK45[2R+] step of du/dt = rhs(u) in its two-register form.

    Register y accumulates the solution, u_n + dt sum_{j<i} b_j k_j; register
    x holds the stage input.  Stage i evaluates k_i = rhs(x), then forms the
    next stage input from y *before* adding b_i k_i to it:
        x <- y + dt a_i k_i   (i < 5),   y <- y + dt b_i k_i,
    which reproduces the stage values of the Butcher matrix above.  The
    third register accumulates the embedded error estimate
        err = u_{n+1} - uhat_{n+1} = dt sum_i (b_i - bhat_i) k_i.
    Returns (u_{n+1}, err).  The coefficients default to the double values
    of the published table; any numeric type that supports + and * works
    (the tests pass Fractions)."""
    a = RK45_2R_A if a is None else a
    b = RK45_2R_B if b is None else b
    e = RK45_2R_E if e is None else e
    y, x = u, u
    err = None
    for i in range(5):
        k = rhs(x)
        if i < 4:
            x = y + (dt * a[i]) * k
        y = y + (dt * b[i]) * k
        err = (dt * e[i]) * k if err is None else err + (dt * e[i]) * k
    return y, err


def rk45_error_norm(u_new, err, atol, rtol):
    """Weighted RMS norm of the embedded error estimate over every value of
    the state: sqrt(mean((err / (atol + rtol |u_{n+1}|))^2)).  (Reading: the
    usual mixed absolute/relative scaling of embedded-pair controllers,
    taken on the new solution only, since the two-register scheme has
    overwritten u_n.)"""
    u_new = np.asarray(u_new, dtype=np.float64)
    w = np.asarray(err, dtype=np.float64) / (atol + rtol * np.abs(u_new))
    return float(np.sqrt(np.mean(w * w)))


# step-size controller of the adaptive RK45[2R+] driver (readings: the
# classic elementary controller for an embedded pair of orders 4(3),
# exponent -1/(3+1), with a safety factor and growth limits)
RK45_SAFETY, RK45_FAC_MIN, RK45_FAC_MAX = 0.9, 0.3, 2.5


def rk45_next_dt(dt, err_norm):
    if err_norm <= 0.0:
        return dt * RK45_FAC_MAX
    fac = RK45_SAFETY * err_norm ** -0.25
    return dt * min(RK45_FAC_MAX, max(RK45_FAC_MIN, fac))


class Solver:
    def __init__(self, mesh, p, gamma=1.4, mu=0.0, prandtl=0.72, viscous=False,
                 ldg_beta=0.5, ldg_tau=0.1, rho_inf=1.0, vel_inf=(1.0, 0.0, 0.0),
                 p_inf=None, t_wall=None):
        self.m = Mesh(mesh, p)
        self.p = p
        self.gamma = gamma
        self.mu = mu
        self.prandtl = prandtl
        self.viscous = viscous
        self.beta = ldg_beta
        self.tau = ldg_tau
        self.rho_inf = rho_inf
        self.vel_inf = np.asarray(vel_inf, dtype=np.float64)
        self.p_inf = (1.0 / gamma if p_inf is None else p_inf)
        self.t_wall = self.p_inf / rho_inf if t_wall is None else t_wall
        m = self.m
        self.types = m.types
        self.nu = {t: m.ops[t].nu for t in self.types}
        self.sizes = {t: m.ne[t] * NVARS * self.nu[t] for t in self.types}
        self.ndof = sum(self.sizes.values())
        self.n_pairs = m.pa.size
        self.na = m.gn[m.pa]
        self.sign = physics.ldg_sign(self.na)

    # -- layout helpers ------------------------------------------------------
    def split(self, flat):
        out, off = {}, 0
        for t in self.types:
            n = self.sizes[t]
            out[t] = flat[off:off + n].reshape(self.m.ne[t], NVARS, self.nu[t])
            off += n
        return out

    def join(self, d):
        return np.concatenate([d[t].reshape(-1) for t in self.types])

    def upts_xyz(self):
        """Physical solution-point coordinates in the public layout with the
        variable axis replaced by x, y, z."""
        return np.concatenate([self.m.upts_x[t].transpose(0, 2, 1).reshape(-1)
                               for t in self.types])

    def upts_xyz_points(self):
        """(n_points, 3) physical coordinates, point order of the public layout."""
        return np.concatenate([self.m.upts_x[t].reshape(-1, 3) for t in self.types])

    def state_from_points(self, q):
        """(n_points, 5) values in upts_xyz_points order -> public layout."""
        out, off = [], 0
        for t in self.types:
            ne, nu = self.m.ne[t], self.nu[t]
            blk = q[off:off + ne * nu].reshape(ne, nu, NVARS).transpose(0, 2, 1)
            out.append(blk.reshape(-1))
            off += ne * nu
        return np.concatenate(out)

    # -- boundary states -------------------------------------------------------
    def _boundary(self, ub, nb):
        """(inviscid ghost, common solution) at boundary flux points."""
        ghost = np.empty_like(ub)
        cb = np.empty_like(ub)
        tags = self.m.btag
        wall = tags == 1
        far = tags == 2
        if np.any(~(wall | far)):
            raise ValueError("unknown boundary tag")
        if np.any(wall):
            g, c = physics.wall_states(ub[wall], self.gamma, self.t_wall)
            ghost[wall], cb[wall] = g, c
        if np.any(far):
            g = physics.farfield_state(ub[far], nb[far], self.gamma, self.rho_inf,
                                       self.vel_inf, self.p_inf)
            ghost[far], cb[far] = g, g
        return ghost, cb

    # -- the right-hand side ---------------------------------------------------
    def rhs(self, u_flat):
        m, g = self.m, self.gamma
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        ops = m.ops
        # 1. interpolate to flux points
        uf = {t: u[t] @ ops[t].M0.T for t in self.types}
        UF = m.to_global(uf)
        ua, ub = UF[m.pa], UF[m.pb]
        na = self.na
        ubnd = UF[m.bg]
        nb = m.gn[m.bg]
        ghost, cb = self._boundary(ubnd, nb)

        grad = {}
        if self.viscous:
            # 2-3. common solution, jumps, corrected physical gradient
            grad = self._gradient(u, UF, ua, ub, ubnd, cb)
            # 4. gradients at flux points
            gradf = {t: np.stack([grad[t][..., k] @ ops[t].M0.T for k in range(3)],
                                 axis=-1) for t in self.types}        # (ne, V, nf, m)
            GF = np.concatenate([gradf[t].transpose(0, 2, 1, 3).reshape(-1, NVARS, 3)
                                 for t in self.types])

        # 5. transformed flux at solution points
        R = {}
        Ft = {}
        for t in self.types:
            up = u[t].transpose(0, 2, 1)                                  # (ne, nu, V)
            F = physics.inviscid_flux(up, g)
            if self.viscous:
                F = F - physics.viscous_flux(up, grad[t].transpose(0, 2, 1, 3), g,
                                             self.mu, self.prandtl)
            Ft[t] = np.einsum("ejdm,ejvm->evjd", m.S[t], F)              # (ne, V, nu, d)

        # 6. common normal flux
        Fc = physics.rusanov(ua, ub, na, g)
        Fcb = physics.rusanov(ubnd, ghost, nb, g)
        if self.viscous:
            fva = physics.viscous_flux(ua, GF[m.pa], g, self.mu, self.prandtl)
            fvb = physics.viscous_flux(ub, GF[m.pb], g, self.mu, self.prandtl)
            Fc = (Fc - physics.ldg_viscous_normal(fva, fvb, na, self.sign, self.beta)
                  + self.tau * (ua - ub))
            fvbnd = physics.viscous_flux(cb, GF[m.bg], g, self.mu, self.prandtl)
            Fcb = (Fcb - np.einsum("...vm,...m->...v", fvbnd, nb)
                   + self.tau * (ubnd - cb))
        FC = np.empty_like(UF)
        FC[m.pa] = Fc * m.gmag[m.pa][:, None]
        FC[m.pb] = -Fc * m.gmag[m.pb][:, None]
        FC[m.bg] = Fcb * m.gmag[m.bg][:, None]
        fc = m.from_global(FC)

        # 7. divergence plus correction, scaled by -1/J
        for t in self.types:
            op = ops[t]
            div = sum(Ft[t][..., d] @ op.D[d].T for d in range(3))
            fn_int = sum(op.fnorm[:, d] * (Ft[t][..., d] @ op.M0.T) for d in range(3))
            R[t] = -(div + (fc[t] - fn_int) @ op.M3.T) / m.J[t][:, None, :]
        return self.join(R)

    def _gradient(self, u, UF, ua, ub, ubnd, cb):
        m, ops = self.m, self.m.ops
        # 2. common solution and jumps
        C = physics.ldg_common_solution(ua, ub, self.sign, self.beta)
        DL = np.empty_like(UF)
        DL[m.pa] = C - ua
        DL[m.pb] = C - ub
        DL[m.bg] = cb - ubnd
        delta = m.from_global(DL)
        # 3. corrected gradient, physical
        grad = {}
        for t in self.types:
            op = ops[t]
            gh = np.stack([u[t] @ op.D[d].T + (op.fnorm[:, d] * delta[t]) @ op.M3.T
                           for d in range(3)], axis=-1)           # (ne, V, nu, d)
            grad[t] = (np.einsum("ejdm,evjd->evjm", m.S[t], gh)
                       / m.J[t][:, None, :, None])                # (ne, V, nu, m)
        return grad

    def gradient(self, u_flat):
        """The corrected physical gradient at the solution points, per type
        (ne, V, nu, 3), as the Navier-Stokes RHS computes it."""
        m = self.m
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        uf = {t: u[t] @ m.ops[t].M0.T for t in self.types}
        UF = m.to_global(uf)
        ua, ub = UF[m.pa], UF[m.pb]
        ubnd = UF[m.bg]
        _, cb = self._boundary(ubnd, m.gn[m.bg])
        return self._gradient(u, UF, ua, ub, ubnd, cb)

    # -- time stepping and reductions ----------------------------------------
    def rk4_step(self, u, dt):
        k1 = self.rhs(u)
        k2 = self.rhs(u + 0.5 * dt * k1)
        k3 = self.rhs(u + 0.5 * dt * k2)
        k4 = self.rhs(u + dt * k3)
        return u + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def rk4_2n_step(self, u, dt):
        """One step of the five-stage fourth-order low-storage Runge-Kutta
        scheme of Carpenter & Kennedy (1994, 2N storage):
        dU <- A_i dU + dt R(U);  U <- U + B_i dU,  i = 1..5 (A_1 = 0)."""
        du = np.zeros_like(u)
        for a, b in zip(RK4_2N_A, RK4_2N_B):
            du = a * du + dt * self.rhs(u)
            u = u + b * du
        return u

    def rk45_step(self, u, dt):
        """One RK45[2R+] step (see rk45_2r_step): (u_{n+1}, error estimate)."""
        return rk45_2r_step(self.rhs, u, dt)

    def rk45_adaptive(self, u, t_span, dt, atol, rtol, max_steps=100000):
        """Advance by exactly t_span with error-controlled RK45[2R+] steps.
        A step is accepted when the weighted error norm is <= 1; either way
        the next step size is rk45_next_dt(dt, norm), and the last step is
        shortened to end at t_span.  Returns (u, next dt, accepted steps,
        rejected steps)."""
        t, acc, rej = 0.0, 0, 0
        while t < t_span and acc + rej < max_steps:
            last = dt >= t_span - t
            h = t_span - t if last else dt
            un, err = self.rk45_step(u, h)
            nrm = rk45_error_norm(un, err, atol, rtol)
            if nrm <= 1.0:
                u, acc = un, acc + 1
                t = t_span if last else t + h
            else:
                rej += 1
            dt = rk45_next_dt(h, nrm)
        return u, dt, acc, rej

    def integrals(self, u_flat):
        """sum_e sum_j w_j J_j u_j per conserved variable."""
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        tot = np.zeros(NVARS)
        for t in self.types:
            wJ = self.m.ops[t].w[None, :] * self.m.J[t]
            tot += np.einsum("ej,evj->v", wJ, u[t])
        return tot

    def kinetic_energy(self, u_flat):
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        ke = 0.0
        for t in self.types:
            wJ = self.m.ops[t].w[None, :] * self.m.J[t]
            k = 0.5 * np.sum(u[t][:, 1:4, :] ** 2, axis=1) / u[t][:, 0, :]
            ke += float(np.sum(wJ * k))
        return ke

    def ke_rate(self, u_flat):
        """Time derivative of the kinetic-energy integral under the
        semi-discrete system du/dt = R(u).  With K = |m|^2 / (2 rho) (m the
        momentum), dK = v.dm - |v|^2/2 drho, so
        dKE/dt = sum_e sum_j w_j J_j (v_j . R_m,j - |v_j|^2/2 R_rho,j).
        The kinetic-energy dissipation rate is its negative."""
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        r = self.split(self.rhs(u_flat))
        tot = 0.0
        for t in self.types:
            wJ = self.m.ops[t].w[None, :] * self.m.J[t]
            v = u[t][:, 1:4, :] / u[t][:, 0:1, :]
            dk = np.sum(v * r[t][:, 1:4, :], axis=1) - 0.5 * np.sum(v * v, axis=1) * r[t][:, 0, :]
            tot += float(np.sum(wJ * dk))
        return tot

    def wall_force(self, u_flat):
        """Force of the fluid on the no-slip walls, as (inviscid, viscous)
        3-vectors: the integral over the wall faces of the common normal
        momentum flux that the RHS uses there (n the fluid's outward normal,
        i.e. into the wall).  Inviscid part: Rusanov against the wall's
        ghost state; viscous part: -F_v(C_b, grad u).n + tau (u - C_b)
        (momentum components).  Face integral: sum over the wall flux points
        of fw |S^T n^| times the value, fw the integral of the flux point's
        face Lagrange polynomial."""
        m, g = self.m, self.gamma
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        UF = m.to_global({t: u[t] @ m.ops[t].M0.T for t in self.types})
        gw = m.bg[m.btag == 1]
        uw, nw = UF[gw], m.gn[gw]
        ghost, cb = physics.wall_states(uw, g, self.t_wall)
        f_inv = physics.rusanov(uw, ghost, nw, g)[:, 1:4]
        f_vis = np.zeros_like(f_inv)
        if self.viscous and gw.size:
            grad = self.gradient(u_flat)
            gradf = {t: np.stack([grad[t][..., k] @ m.ops[t].M0.T for k in range(3)], axis=-1)
                     for t in self.types}
            GF = np.concatenate([gradf[t].transpose(0, 2, 1, 3).reshape(-1, NVARS, 3)
                                 for t in self.types])
            fv = physics.viscous_flux(cb, GF[gw], g, self.mu, self.prandtl)
            f_vis = (-np.einsum("kvm,km->kv", fv, nw) + self.tau * (uw - cb))[:, 1:4]
        gfw = np.concatenate([np.tile(m.ops[t].fw, m.ne[t]) for t in self.types])
        wa = gfw[gw] * m.gmag[gw]
        return wa @ f_inv, wa @ f_vis

    def volume(self):
        return sum(float(np.sum(self.m.ops[t].w[None, :] * self.m.J[t]))
                   for t in self.types)

    def dt_cfl(self, u_flat, cfl):
        """cfl * min_e r_e / max |v| + c, r_e = 3 V_e / A_e."""
        u = self.split(np.asarray(u_flat, dtype=np.float64))
        rmin = np.inf
        smax = 0.0
        for t in self.types:
            op = self.m.ops[t]
            V = np.sum(op.w[None, :] * self.m.J[t], axis=1)
            A = np.sum(op.fw[None, :] * self.m.fmag[t], axis=1)
            rmin = min(rmin, float(np.min(3.0 * V / A)))
            up = u[t].transpose(0, 2, 1)
            _, v, _ = physics.primitives(up, self.gamma)
            s = np.linalg.norm(v, axis=-1) + physics.sound_speed(up, self.gamma)
            smax = max(smax, float(np.max(s)))
        return cfl * rmin / smax
