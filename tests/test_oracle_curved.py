"""Pins of the oracle's quadratically curved elements (CPU only): 10-node
tets, 18-node prisms and 27-node hexes whose nodes a smooth periodic map
moved off the straight elements.

* Curved nodes placed on the straight elements reproduce the straight
  geometry (points, J, S, normals) and the RHS.
* The curved elements tile the periodic cell: the total volume is exactly
  the cell volume once the quadrature integrates J exactly (p >= 2).
* Free-stream preservation and discrete conservation on the curved meshes
  (p >= 2: J and S of a quadratic map are then in the solution space).
* The isentropic vortex's RHS converges to its exact time derivative at
  the residual order p on curved meshes too.
"""
import math

import numpy as np
import pytest

import synth
from oracle.solver import Solver


def _box(kind, n=4, amp=0.15):
    m0 = synth.vortex_box(n=n) if kind == "pt" else synth.hex_box(n=n, n_hex_cols=n // 2)
    return m0, synth.curve_mesh(m0, amp=amp)


@pytest.mark.parametrize("kind", ["pt", "hp"])
def test_straight_nodes_reproduce_straight_geometry(kind):
    m0, m = _box(kind, amp=0.0)
    s0, s = Solver(m0, 3, viscous=True, mu=0.02), Solver(m, 3, viscous=True, mu=0.02)
    for t in s0.types:
        np.testing.assert_allclose(s.m.upts_x[t], s0.m.upts_x[t], atol=1e-13)
        np.testing.assert_allclose(s.m.J[t], s0.m.J[t], rtol=1e-13)
        np.testing.assert_allclose(s.m.S[t], s0.m.S[t], atol=1e-13)
        np.testing.assert_allclose(s.m.fn[t], s0.m.fn[t], atol=1e-13)
    u = s0.state_from_points(synth.random_smooth_state(s0.upts_xyz_points(), seed=3))
    r0, r = s0.rhs(u), s.rhs(u)
    assert np.max(np.abs(r - r0)) < 1e-12 * np.max(np.abs(r0))


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_curved_elements_tile_the_periodic_cell(kind, p):
    _, m = _box(kind)
    s = Solver(m, p)
    assert abs(s.volume() - 1000.0) < 1e-10
    assert min(float(s.m.J[t].min()) for t in s.types) > 0.0


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_curved_freestream_preservation(kind, p, viscous):
    _, m = _box(kind)
    s = Solver(m, p, viscous=viscous, mu=0.05)
    u = s.state_from_points(synth.uniform_state(s.upts_xyz_points(), vel=(0.3, -0.2, 0.5), p=1.0))
    assert np.max(np.abs(s.rhs(u))) < 1e-12


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("viscous", [False, True])
def test_curved_discrete_conservation(kind, viscous):
    _, m = _box(kind)
    s = Solver(m, 3, viscous=viscous, mu=0.05)
    u = s.state_from_points(synth.random_smooth_state(s.upts_xyz_points(), seed=4))
    r = s.rhs(u)
    assert np.max(np.abs(s.integrals(r)) / s.integrals(np.abs(r))) < 1e-12


def _vortex_dudt(xyz, h=1e-5):
    vel = (1.0, 1.0, 0.0)
    g = np.zeros(xyz.shape[:-1] + (5,))
    for k in range(2):
        d = np.zeros(3)
        d[k] = h
        g -= vel[k] * (synth.isentropic_vortex(xyz + d) - synth.isentropic_vortex(xyz - d)) / (2 * h)
    return g


def test_curved_vortex_residual_converges():
    """p = 2, n = 8 -> 16 on curved prism/tet meshes: order >= p - 0.35."""
    errs = []
    for n in (8, 16):
        _, m = _box("pt", n=n)
        s = Solver(m, 2)
        xyz = s.upts_xyz_points()
        err = s.rhs(s.state_from_points(synth.isentropic_vortex(xyz))) - s.state_from_points(_vortex_dudt(xyz))
        e = s.split(err)
        errs.append(math.sqrt(sum(float(np.sum(s.m.ops[t].w[None, None, :] * s.m.J[t][:, None, :] * e[t] ** 2))
                                  for t in s.types)))
    assert math.log2(errs[0] / errs[1]) >= 2 - 0.35, errs


@pytest.mark.parametrize("kind", ["pt", "hp"])
def test_curved_mesh_generator_shares_face_nodes(kind):
    """The generator's quadratic nodes: the vertex nodes of every element
    are the moved vertices, and two elements sharing an edge give its
    midpoint node the same coordinates (what the face pairing relies on)."""
    m0, m = _box(kind)
    xyz = m0["xyz"]
    lo, hi = xyz.min(0), xyz.max(0)
    L = np.where(m0["period"] > 0, m0["period"], hi - lo)
    phi = lambda x: x + 0.15 * (L / (2 * math.pi)) * np.prod(np.sin(2 * math.pi * (x - lo) / L), axis=-1,
                                                             keepdims=True)
    nv = {"tet": 4, "pri": 6, "hex": 8}
    mids = {}
    for t in ("tet", "pri", "hex"):
        conn = m0.get(t, np.zeros((0, nv[t]), np.int64))
        if not len(conn):
            continue
        nodes = m[t + "_nodes"]
        ref = synth.QUAD_NODES[t]
        # vertex nodes: the first nv reference nodes of tets and hexes are the
        # vertices; for prisms the vertices are nodes 0-2 and 12-14
        vidx = list(range(4)) if t == "tet" else ([0, 1, 2, 12, 13, 14] if t == "pri" else [0, 2, 8, 6, 18, 20, 26, 24])
        np.testing.assert_allclose(nodes[:, vidx], phi(xyz[conn]), atol=1e-12)
        # edge midpoints between two vertices, keyed by the sorted vertex pair
        vref = np.array([ref[i] for i in vidx], dtype=float)
        for q, r in enumerate(ref):
            for a in range(nv[t]):
                for b in range(a + 1, nv[t]):
                    if np.allclose(r, 0.5 * (vref[a] + vref[b])):
                        key = np.sort(conn[:, [a, b]], axis=1)
                        for e in range(len(conn)):
                            k = tuple(key[e])
                            if k in mids:
                                assert np.allclose(mids[k], nodes[e, q], atol=1e-12)
                            else:
                                mids[k] = nodes[e, q]
    assert mids
