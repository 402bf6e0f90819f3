"""Point-wise physics of the oracle.

State arrays have the 5 conserved variables (rho, rho u, rho v, rho w, E)
on the last axis; gradients and fluxes are (..., 5, 3) with the spatial
direction last.  Ideal gas p = (gamma-1)(E - rho|v|^2/2), temperature
T = p/rho (gas constant 1), internal energy e = T/(gamma-1).

Readings (the paper fixes Rusanov for the inviscid interface flux, constant
viscosity Navier-Stokes, no-slip isothermal walls and Riemann-invariant far
field; Sec. 3.2 and 3.4):
  * Rusanov: F.n = (F(uL) + F(uR)).n / 2 - s (uR - uL) / 2 with
    s = max(|vL.n| + cL, |vR.n| + cR), c = sqrt(gamma p / rho).
  * viscous flux: tau = mu (grad v + grad v^T - 2/3 div v I), energy flux
    v.tau + mu gamma / Pr grad e; the total flux is F_inv - F_vis.
  * LDG interface treatment (the paper names none): common solution
    C = (uL + uR)/2 + beta (uL - uR), common viscous flux
    (FvL + FvR).n/2 - beta (FvL - FvR).n, penalty tau_ldg (uL - uR) on the
    total normal flux, where L is the side whose outward normal n satisfies
    n . s_dir > 0 with s_dir = (1, 0.1 sqrt 2, 0.01 sqrt 3).
  * boundaries: wall ghost (rhoL, -rhoL vL, rhoL e_w + rhoL |vL|^2/2) for
    Rusanov and common solution (rhoL, 0, rhoL e_w); far-field ghost from
    the Riemann invariants vn +- 2c/(gamma-1), with entropy and tangential
    velocity from the upwind side.  At a boundary the common solution is the
    boundary state C_b, the common viscous flux is F_vis(C_b, grad uL).n and
    the penalty is tau_ldg (uL - C_b).
"""
from __future__ import annotations

import math

import numpy as np

S_DIR = np.array([1.0, 0.1 * math.sqrt(2.0), 0.01 * math.sqrt(3.0)])


def primitives(u, gamma):
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (u[..., 4] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, p


def inviscid_flux(u, gamma):
    """F[..., var, m]."""
    rho, v, p = primitives(u, gamma)
    F = np.empty(u.shape + (3,))
    F[..., 0, :] = u[..., 1:4]
    for a in range(3):
        F[..., 1 + a, :] = u[..., 1 + a, None] * v
        F[..., 1 + a, a] += p
    F[..., 4, :] = (u[..., 4] + p)[..., None] * v
    return F


def viscous_flux(u, grad, gamma, mu, prandtl):
    """Physical viscous flux F_vis[..., var, m] from the state and the
    conserved-variable gradient grad[..., var, m] = d u_var / d x_m."""
    rho, v, p = primitives(u, gamma)
    E = u[..., 4]
    grho = grad[..., 0, :]
    # d v_a / d x_m = (d(rho v_a)/dx_m - v_a d rho/dx_m) / rho
    gv = (grad[..., 1:4, :] - v[..., :, None] * grho[..., None, :]) / rho[..., None, None]
    # e = E/rho - |v|^2/2 ;  d e/dx_m = (dE/dx_m - (E/rho) drho/dx_m)/rho - v_a dv_a/dx_m
    ge = ((grad[..., 4, :] - (E / rho)[..., None] * grho) / rho[..., None]
          - np.einsum("...a,...am->...m", v, gv))
    div = gv[..., 0, 0] + gv[..., 1, 1] + gv[..., 2, 2]
    tau = mu * (gv + np.swapaxes(gv, -1, -2))
    for a in range(3):
        tau[..., a, a] -= 2.0 / 3.0 * mu * div
    Fv = np.zeros(u.shape + (3,))
    Fv[..., 1:4, :] = tau
    Fv[..., 4, :] = np.einsum("...a,...am->...m", v, tau) + mu * gamma / prandtl * ge
    return Fv


def sound_speed(u, gamma):
    rho, v, p = primitives(u, gamma)
    return np.sqrt(gamma * p / rho)


def rusanov(ua, ub, n, gamma):
    """Common inviscid normal flux (along n, the outward normal of side a)."""
    Fa = np.einsum("...vm,...m->...v", inviscid_flux(ua, gamma), n)
    Fb = np.einsum("...vm,...m->...v", inviscid_flux(ub, gamma), n)
    _, va, _ = primitives(ua, gamma)
    _, vb, _ = primitives(ub, gamma)
    sa = np.abs(np.sum(va * n, axis=-1)) + sound_speed(ua, gamma)
    sb = np.abs(np.sum(vb * n, axis=-1)) + sound_speed(ub, gamma)
    s = np.maximum(sa, sb)
    return 0.5 * (Fa + Fb) - 0.5 * s[..., None] * (ub - ua)


def ldg_sign(n):
    """+1 where side a (outward normal n) is the LDG left side, else -1."""
    return np.where(n @ S_DIR > 0.0, 1.0, -1.0)


def ldg_common_solution(ua, ub, sign, beta):
    b = beta * sign[..., None]
    return 0.5 * (ua + ub) + b * (ua - ub)


def ldg_viscous_normal(fva, fvb, n, sign, beta):
    fa = np.einsum("...vm,...m->...v", fva, n)
    fb = np.einsum("...vm,...m->...v", fvb, n)
    return 0.5 * (fa + fb) - beta * sign[..., None] * (fa - fb)


# ---------------------------------------------------------------------------
# boundary states
# ---------------------------------------------------------------------------
def wall_states(ua, gamma, t_wall):
    """(inviscid ghost, common solution) of the no-slip isothermal wall."""
    rho = ua[..., 0]
    e_w = t_wall / (gamma - 1.0)
    ghost = np.empty_like(ua)
    ghost[..., 0] = rho
    ghost[..., 1:4] = -ua[..., 1:4]
    ke = 0.5 * np.sum(ua[..., 1:4] ** 2, axis=-1) / rho
    ghost[..., 4] = rho * e_w + ke
    cb = np.zeros_like(ua)
    cb[..., 0] = rho
    cb[..., 4] = rho * e_w
    return ghost, cb


def farfield_state(ua, n, gamma, rho_inf, vel_inf, p_inf):
    """Riemann-invariant far-field ghost state (also the common solution)."""
    rho, v, p = primitives(ua, gamma)
    c = np.sqrt(gamma * p / rho)
    vinf = np.asarray(vel_inf, dtype=np.float64)
    cinf = math.sqrt(gamma * p_inf / rho_inf)
    vn = np.sum(v * n, axis=-1)
    vninf = n @ vinf
    rp = vn + 2.0 * c / (gamma - 1.0)
    rm = vninf - 2.0 * cinf / (gamma - 1.0)
    vnb = 0.5 * (rp + rm)
    cb = 0.25 * (gamma - 1.0) * (rp - rm)
    outflow = vnb >= 0.0
    s_int = p / rho ** gamma
    s_inf = p_inf / rho_inf ** gamma
    s = np.where(outflow, s_int, s_inf)
    vb = np.where(outflow[..., None], v + (vnb - vn)[..., None] * n,
                  vinf + (vnb - vninf)[..., None] * n)
    rhob = (cb * cb / (gamma * s)) ** (1.0 / (gamma - 1.0))
    pb = rhob * cb * cb / gamma
    g = np.empty_like(ua)
    g[..., 0] = rhob
    g[..., 1:4] = rhob[..., None] * vb
    g[..., 4] = pb / (gamma - 1.0) + 0.5 * rhob * np.sum(vb * vb, axis=-1)
    return g
