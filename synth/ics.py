"""Closed-form flow fields evaluated at caller-supplied points.

All functions take coordinates ``xyz`` of shape (..., 3) and return the
conserved state (rho, rho*u, rho*v, rho*w, E) of shape (..., 5), with the
ideal-gas law p = (gamma-1)(E - rho|v|^2/2).
"""
from __future__ import annotations

import math

import numpy as np


def _conserved(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=-1)


def isentropic_vortex(xyz, t=0.0, gamma=1.4, strength=5.0, center=(0.0, 0.0),
                      vel=(1.0, 1.0, 0.0), period=(10.0, 10.0)):
    """Shu's isentropic vortex (axis along z) advected by the mean flow `vel`.

    With r the distance to the vortex centre (minimum periodic image of the
    centre moved by vel*t):
      du = -b/(2pi) y e^{(1-r^2)/2},  dv = b/(2pi) x e^{(1-r^2)/2},
      T = 1 - (gamma-1) b^2 / (8 gamma pi^2) e^{1-r^2},
      rho = T^{1/(gamma-1)},  p = rho^gamma.
    At time t this is the exact solution of the Euler equations on the
    periodic box (up to the vortex tail cut by the periodic images).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    b = strength
    cx = center[0] + vel[0] * t
    cy = center[1] + vel[1] * t
    dx = xyz[..., 0] - cx
    dy = xyz[..., 1] - cy
    if period[0] > 0:
        dx = dx - period[0] * np.round(dx / period[0])
    if period[1] > 0:
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    u = vel[0] - b / (2.0 * math.pi) * dy * f
    v = vel[1] + b / (2.0 * math.pi) * dx * f
    w = np.full_like(u, vel[2])
    T = 1.0 - (gamma - 1.0) * b * b / (8.0 * gamma * math.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return _conserved(rho, u, v, w, p, gamma)


def taylor_green(xyz, gamma=1.4, mach=0.1):
    """Taylor-Green vortex: rho = 1, u = sin x cos y cos z,
    v = -cos x sin y cos z, w = 0,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16 with p0 = 1/(gamma Ma^2)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p0 = 1.0 / (gamma * mach * mach)
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    rho = np.ones_like(u)
    return _conserved(rho, u, v, w, p, gamma)


def shear_flow(xyz, a=0.3, p=1.0 / 1.4, gamma=1.4):
    """Plane shear u = a y, v = w = 0 with rho = 1 and uniform pressure p."""
    xyz = np.asarray(xyz, dtype=np.float64)
    y = xyz[..., 1]
    one = np.ones_like(y)
    return _conserved(one, a * y, 0.0 * y, 0.0 * y, p * one, gamma)


def shear_wave(xyz, amp=0.01, k=1.0, p=1.0 / 1.4, gamma=1.4):
    """Periodic shear wave u = amp sin(k y), v = w = 0 with rho = 1 and
    uniform pressure p (a steady Euler solution that viscosity decays)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    y = xyz[..., 1]
    one = np.ones_like(y)
    return _conserved(one, amp * np.sin(k * y), 0.0 * y, 0.0 * y, p * one, gamma)


def uniform_state(xyz, rho=1.0, vel=(1.0, 0.0, 0.0), p=None, gamma=1.4,
                  mach=0.2):
    xyz = np.asarray(xyz, dtype=np.float64)
    if p is None:
        p = rho * float(np.dot(vel, vel)) / (gamma * mach * mach)
    one = np.ones(xyz.shape[:-1])
    return _conserved(rho * one, vel[0] * one, vel[1] * one, vel[2] * one,
                      p * one, gamma)


def perturbed_freestream(xyz, seed=2, gamma=1.4, mach=0.2, amp=0.01,
                         lengths=(20.0, 20.0, math.pi), nmodes=8, wall_delta=None):
    """Uniform flow rho=1, v=(1,0,0), p=1/(gamma Ma^2) plus a smooth seeded
    velocity perturbation amp * sum_k a_k d_k sin(k.x + phi_k), with
    sum a_k = 1, random unit directions d_k, random phases, and integer
    wavenumbers per box length (so the field is periodic in every axis).

    wall_delta: if given, the whole velocity is multiplied by
    tanh(y / wall_delta), so the state satisfies the no-slip condition on a
    wall at y = 0 (a boundary-layer profile of thickness ~wall_delta);
    None gives the impulsive start (slip at the wall)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(0.0, 1.0, nmodes)
    a /= a.sum()
    d = rng.normal(size=(nmodes, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    m = rng.integers(1, 4, size=(nmodes, 3))
    phi = rng.uniform(0.0, 2.0 * math.pi, nmodes)
    kvec = 2.0 * math.pi * m / np.asarray(lengths)[None, :]
    dv = np.zeros(xyz.shape[:-1] + (3,))
    for k in range(nmodes):
        s = np.sin(xyz @ kvec[k] + phi[k])
        dv += amp * a[k] * s[..., None] * d[k]
    rho = np.ones(xyz.shape[:-1])
    p = np.full(xyz.shape[:-1], 1.0 / (gamma * mach * mach))
    vel = np.stack([1.0 + dv[..., 0], dv[..., 1], dv[..., 2]], axis=-1)
    if wall_delta is not None:
        vel = vel * np.tanh(xyz[..., 1] / wall_delta)[..., None]
    return _conserved(rho, vel[..., 0], vel[..., 1], vel[..., 2], p, gamma)


def random_smooth_state(xyz, seed=0, gamma=1.4, amp=0.1, lengths=(10.0, 10.0, 10.0)):
    """A smooth, strictly physical random state: rho, v, p each a mean plus
    `amp` times a few seeded periodic Fourier modes."""
    xyz = np.asarray(xyz, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    fields = []
    means = (1.0, 0.5, -0.3, 0.2, 2.0)
    for q in range(5):
        f = np.full(xyz.shape[:-1], means[q])
        for _ in range(3):
            m = rng.integers(0, 3, size=3)
            kvec = 2.0 * math.pi * m / np.asarray(lengths)
            f = f + amp * rng.uniform(-1, 1) * np.sin(xyz @ kvec + rng.uniform(0, 6.3))
        fields.append(f)
    rho, u, v, w, p = fields
    return _conserved(rho, u, v, w, p, gamma)
