"""Pins of the oracle's flow diagnostics (CPU only): the force on no-slip
walls and the time derivative of the kinetic energy.

Wall force: a fluid at rest at uniform pressure p0 pushes a flat wall of
area A with p0 A along the wall's inward normal and exerts no shear; the
plane shear u = a y exerts the viscous shear stress mu a on the wall at
y = 0 (pressure still p0).  Both fields are exactly representable at
p >= 2 (the energy is quadratic in y), the wall's common solution equals
the interior state there, and no element touches both the wall and the
far field, so the discrete values must equal the closed forms to rounding.

Kinetic-energy rate: the directional derivative of the (separately pinned)
kinetic-energy integral along the RHS, by central differences; and the
viscous decay of the periodic shear wave u = A sin y, whose exact rate is
-mu A^2 V / 2 (V the domain volume; no convection, no pressure work),
approached as the mesh is refined.
"""
import math

import numpy as np
import pytest

import synth
from oracle.solver import Solver

GAMMA = 1.4
P0 = 1.0 / GAMMA


def _channel_solver(npl, p, mu=0.01, **kw):
    if npl == "hex":   # hexahedra beside prisms, all layers
        mesh = synth.wall_channel(n_prism_layers=3, n_hex_cols=1, **kw)
    else:
        mesh = synth.wall_channel(n_prism_layers=npl, **kw)
    return Solver(mesh, p, viscous=True, mu=mu, t_wall=P0)


@pytest.mark.parametrize("npl", [2, 0, "hex"])  # prism, tet, hex + prism wall faces
def test_wall_force_at_rest_is_pressure_times_area(npl):
    s = _channel_solver(npl, 2)
    X = s.upts_xyz_points()
    u = s.state_from_points(synth.shear_flow(X, a=0.0, p=P0))
    f_inv, f_vis = s.wall_force(u)
    area = 2.0 * 1.0
    assert abs(f_inv[1] + P0 * area) < 1e-13 * P0 * area
    assert np.max(np.abs(f_inv[[0, 2]])) < 1e-13 * P0 * area
    assert np.max(np.abs(f_vis)) < 1e-13 * P0 * area


@pytest.mark.parametrize("npl", [2, 0, "hex"])
@pytest.mark.parametrize("p", [2, 3])
def test_wall_force_of_plane_shear(npl, p):
    mu, a = 0.01, 0.3
    s = _channel_solver(npl, p, mu=mu)
    u = s.state_from_points(synth.shear_flow(s.upts_xyz_points(), a=a, p=P0))
    f_inv, f_vis = s.wall_force(u)
    area = 2.0 * 1.0
    shear = mu * a * area
    assert abs(f_vis[0] - shear) < 1e-11 * shear
    assert np.max(np.abs(f_vis[1:])) < 1e-11 * shear
    assert abs(f_inv[1] + P0 * area) < 1e-12 * P0 * area
    assert np.max(np.abs(f_inv[[0, 2]])) < 1e-12 * P0 * area


def test_wall_force_without_walls_is_zero():
    s = Solver(synth.vortex_box(), 2)
    u = s.state_from_points(synth.isentropic_vortex(s.upts_xyz_points()))
    f_inv, f_vis = s.wall_force(u)
    assert np.all(f_inv == 0.0) and np.all(f_vis == 0.0)


@pytest.mark.parametrize("viscous", [False, True])
def test_ke_rate_is_the_derivative_of_the_kinetic_energy(viscous):
    kw = dict(viscous=True, mu=0.05) if viscous else {}
    s = Solver(synth.vortex_box(), 2, **kw)
    u = s.state_from_points(synth.isentropic_vortex(s.upts_xyz_points()))
    R = s.rhs(u)
    rate = s.ke_rate(u)
    eps = 1e-4
    fd = (s.kinetic_energy(u + eps * R) - s.kinetic_energy(u - eps * R)) / (2 * eps)
    assert abs(fd - rate) < 1e-7 * abs(rate)


@pytest.mark.parametrize("n, tol", [(4, 1e-2), (6, 3e-3)])
def test_ke_rate_of_decaying_shear_wave(n, tol):
    mu, amp = 0.01, 0.01
    c = np.linspace(0.0, 2.0 * math.pi, n + 1)
    mesh = synth.layered_box((c, c, c), 2, n // 2, (True, True, True), jitter=0.05, seed=5)
    s = Solver(mesh, 4, viscous=True, mu=mu)
    u = s.state_from_points(synth.shear_wave(s.upts_xyz_points(), amp=amp))
    exact = -mu * amp * amp * (2.0 * math.pi) ** 3 / 2.0
    assert abs(s.ke_rate(u) - exact) < tol * abs(exact)


@pytest.mark.parametrize("p", [2, 3])
def test_integrals_and_kinetic_energy_closed_forms(p):
    """On the straight (unjittered) cube [-5,5]^3, tets and prisms: the
    conserved integrals of rho = 1, u = a y, E = e0 + a^2 y^2 / 2 are
    (V, 0, 0, 0, e0 V + a^2 I / 2) and the kinetic energy a^2 I / 2, with
    V = 1000 and I = int y^2 = 10^2 * 2 * 5^3 / 3 (the quadrature is exact
    for these quadratics at p >= 2 on affine elements)."""
    a, e0 = 0.3, 2.5
    s = Solver(synth.vortex_box(jitter=0.0), p)
    X = s.upts_xyz_points()
    q = np.zeros((len(X), 5))
    q[:, 0] = 1.0
    q[:, 1] = a * X[:, 1]
    q[:, 4] = e0 + 0.5 * (a * X[:, 1]) ** 2
    u = s.state_from_points(q)
    V, I = 1000.0, 100.0 * 2.0 * 125.0 / 3.0
    np.testing.assert_allclose(s.integrals(u), [V, 0.0, 0.0, 0.0, e0 * V + 0.5 * a * a * I],
                               rtol=1e-13, atol=1e-10)
    assert abs(s.kinetic_energy(u) - 0.5 * a * a * I) < 1e-12 * I
