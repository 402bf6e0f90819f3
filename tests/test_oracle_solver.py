"""Pins of the oracle's geometry, physics and RHS (CPU only).

They check what the mathematics fixes independently of the oracle's code:
the domain volume, closed element surfaces, free-stream preservation,
discrete conservation, symmetry/renumbering invariance, the Rusanov and
LDG flux identities, the viscous stress from a direct primitive-variable
finite difference, the isentropic vortex's exact time derivative, a
manufactured Navier-Stokes residual derived symbolically, and the RK4
amplification polynomial.
"""
import math

import numpy as np
import pytest

import synth
from oracle import physics
from oracle.solver import Solver

GAMMA = 1.4


def _solver(mesh, p, **kw):
    return Solver(mesh, p, **kw)


def _box(kind, n=4):
    """Periodic [-5,5]^3 test meshes: 'pt' prisms below Kuhn tets, 'hp'
    hexahedra beside prism pairs, 'hex' hexahedra only."""
    if kind == "pt":
        return synth.vortex_box(n=n)
    return synth.hex_box(n=n, n_hex_cols=n // 2 if kind == "hp" else n)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2, 4])
def test_volume_of_jittered_periodic_box(p):
    """Jittered periodic images move together, so the total volume stays
    10^3; sum_j w_j J_j integrates J exactly for p >= 2 on prisms."""
    s = _solver(synth.vortex_box(), p)
    assert abs(s.volume() - 1000.0) < 1e-10


def test_volume_of_boundary_layer_box():
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    s = _solver(m, 2)
    assert abs(s.volume() - 20.0 * 20.0 * math.pi) < 1e-9


@pytest.mark.parametrize("p", [1, 3])
def test_closed_element_surfaces(p):
    """sum over an element's faces of int S^T n^ dS^ = 0."""
    s = _solver(synth.vortex_box(), p)
    for t in s.types:
        op = s.m.ops[t]
        vec = np.einsum("f,ef,efk->ek", op.fw, s.m.fmag[t], s.m.fn[t])
        scale = np.einsum("f,ef->e", op.fw, s.m.fmag[t])
        assert np.max(np.abs(vec) / scale[:, None]) < 1e-13


# --------------------------------------------------------------------------
# point-wise physics
# --------------------------------------------------------------------------
def _rand_states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.normal(size=(n, 3))
    p = rng.uniform(0.5, 3.0, n)
    E = p / (GAMMA - 1) + 0.5 * rho * np.sum(v * v, 1)
    return np.c_[rho, rho[:, None] * v, E]


def _rand_normals(n, seed):
    rng = np.random.default_rng(seed)
    nn = rng.normal(size=(n, 3))
    return nn / np.linalg.norm(nn, axis=1, keepdims=True)


def test_rusanov_consistency_and_antisymmetry():
    u = _rand_states(50, 0)
    w = _rand_states(50, 1)
    n = _rand_normals(50, 2)
    F = physics.inviscid_flux(u, GAMMA)
    np.testing.assert_allclose(physics.rusanov(u, u, n, GAMMA),
                               np.einsum("ivm,im->iv", F, n), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(physics.rusanov(u, w, n, GAMMA),
                               -physics.rusanov(w, u, -n, GAMMA), rtol=1e-13, atol=1e-13)


def test_inviscid_flux_closed_form():
    """F for a single known state written out by hand."""
    rho, v, p = 1.3, np.array([0.4, -0.7, 0.2]), 2.1
    E = p / (GAMMA - 1) + 0.5 * rho * v @ v
    u = np.array([[rho, *(rho * v), E]])
    F = physics.inviscid_flux(u, GAMMA)[0]
    exp = np.zeros((5, 3))
    exp[0] = rho * v
    exp[1:4] = rho * np.outer(v, v) + p * np.eye(3)
    exp[4] = (E + p) * v
    np.testing.assert_allclose(F, exp, rtol=1e-14)


def test_ldg_common_values_antisymmetric():
    u = _rand_states(40, 3)
    w = _rand_states(40, 4)
    n = _rand_normals(40, 5)
    ga = np.random.default_rng(6).normal(size=(40, 5, 3))
    gb = np.random.default_rng(7).normal(size=(40, 5, 3))
    fa = physics.viscous_flux(u, ga, GAMMA, 0.1, 0.72)
    fb = physics.viscous_flux(w, gb, GAMMA, 0.1, 0.72)
    sa, sb = physics.ldg_sign(n), physics.ldg_sign(-n)
    assert np.all(sa == -sb)
    # the common solution does not depend on which side is called a
    np.testing.assert_allclose(physics.ldg_common_solution(u, w, sa, 0.5),
                               physics.ldg_common_solution(w, u, sb, 0.5), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(physics.ldg_viscous_normal(fa, fb, n, sa, 0.5),
                               -physics.ldg_viscous_normal(fb, fa, -n, sb, 0.5), rtol=1e-13, atol=1e-14)
    # beta = 1/2: the common solution is the left state, the flux the right one
    left = sa > 0
    C = physics.ldg_common_solution(u, w, sa, 0.5)
    np.testing.assert_allclose(C[left], u[left], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(C[~left], w[~left], rtol=1e-14, atol=1e-15)


def test_viscous_flux_against_primitive_finite_differences():
    """The chain rule from conserved to primitive gradients: evaluate a
    smooth field, difference rho, v, e directly, build tau by hand."""
    mu, pr = 0.3, 0.72

    def prim(x):
        rho = 1.0 + 0.3 * np.sin(x[..., 0]) * np.cos(0.5 * x[..., 1])
        v = np.stack([np.sin(x[..., 1] + 0.3 * x[..., 2]), 0.5 * np.cos(x[..., 0] * x[..., 2]),
                      0.2 * x[..., 0] * x[..., 1]], -1)
        p = 2.0 + 0.4 * np.cos(x[..., 2] - x[..., 0])
        return rho, v, p

    def cons(x):
        rho, v, p = prim(x)
        return np.concatenate([rho[..., None], rho[..., None] * v,
                               (p / (GAMMA - 1) + 0.5 * rho * np.sum(v * v, -1))[..., None]], -1)

    x0 = np.random.default_rng(8).uniform(-1, 1, size=(20, 3))
    h = 1e-5
    gc = np.zeros((20, 5, 3))
    gv = np.zeros((20, 3, 3))
    ge = np.zeros((20, 3))
    for m in range(3):
        dx = np.zeros(3)
        dx[m] = h
        gc[:, :, m] = (cons(x0 + dx) - cons(x0 - dx)) / (2 * h)
        _, vp, _ = prim(x0 + dx)
        _, vm, _ = prim(x0 - dx)
        gv[:, :, m] = (vp - vm) / (2 * h)
        rp, _, pp = prim(x0 + dx)
        rm, _, pm = prim(x0 - dx)
        ge[:, m] = (pp / rp - pm / rm) / (2 * h) / (GAMMA - 1)
    _, v, _ = prim(x0)
    div = np.trace(gv, axis1=1, axis2=2)
    tau = mu * (gv + gv.transpose(0, 2, 1) - 2.0 / 3.0 * div[:, None, None] * np.eye(3))
    exp = np.zeros((20, 5, 3))
    exp[:, 1:4] = tau
    exp[:, 4] = np.einsum("ia,iam->im", v, tau) + mu * GAMMA / pr * ge
    got = physics.viscous_flux(cons(x0), gc, GAMMA, mu, pr)
    np.testing.assert_allclose(got, exp, atol=1e-8)


def test_farfield_ghost_is_freestream_for_freestream_interior():
    vinf = (1.0, 0.2, -0.1)
    pinf = 1.0 / (GAMMA * 0.2 ** 2)
    u = np.tile(synth.uniform_state(np.zeros((1, 3)), vel=vinf, p=pinf), (30, 1))
    n = _rand_normals(30, 9)
    g = physics.farfield_state(u, n, GAMMA, 1.0, vinf, pinf)
    np.testing.assert_allclose(g, u, rtol=1e-13)


def test_farfield_ghost_keeps_the_characteristic_invariants():
    """Riemann-invariant far field (Sec. 3.2): the ghost state carries the
    outgoing invariant vn + 2c/(g-1) of the interior and the incoming
    vn - 2c/(g-1) of the free stream; its entropy p/rho^g and tangential
    velocity come from the interior at outflow (vn_b >= 0) and from the free
    stream at inflow (computed here from primitives, not from the oracle's
    formula)."""
    rng = np.random.default_rng(12)
    vinf = np.array([1.0, 0.2, -0.1])
    pinf, rinf = 1.0 / (GAMMA * 0.2 ** 2), 1.0
    n = _rand_normals(40, 13)
    rho = 1.0 + 0.1 * rng.standard_normal(40)
    v = vinf + 0.3 * rng.standard_normal((40, 3))
    p = pinf * (1.0 + 0.1 * rng.standard_normal(40))
    u = np.concatenate([rho[:, None], rho[:, None] * v,
                        (p / (GAMMA - 1) + 0.5 * rho * np.sum(v * v, 1))[:, None]], axis=1)
    g = physics.farfield_state(u, n, GAMMA, rinf, vinf, pinf)
    rg = g[:, 0]
    vg = g[:, 1:4] / rg[:, None]
    pg = (GAMMA - 1) * (g[:, 4] - 0.5 * rg * np.sum(vg * vg, 1))
    c, cg, cinf = np.sqrt(GAMMA * p / rho), np.sqrt(GAMMA * pg / rg), math.sqrt(GAMMA * pinf / rinf)
    vn, vng, vninf = np.sum(v * n, 1), np.sum(vg * n, 1), n @ vinf
    k = 2.0 / (GAMMA - 1)
    np.testing.assert_allclose(vng + k * cg, vn + k * c, rtol=1e-12)
    np.testing.assert_allclose(vng - k * cg, vninf - k * cinf, rtol=1e-12, atol=1e-12)
    out = vng >= 0.0
    assert out.any() and (~out).any()
    sg = pg / rg ** GAMMA
    np.testing.assert_allclose(sg[out], (p / rho ** GAMMA)[out], rtol=1e-12)
    np.testing.assert_allclose(sg[~out], np.full((~out).sum(), pinf / rinf ** GAMMA), rtol=1e-12)
    tg = vg - vng[:, None] * n
    np.testing.assert_allclose(tg[out], (v - vn[:, None] * n)[out], atol=1e-12)
    np.testing.assert_allclose(tg[~out], (vinf - vninf[:, None] * n)[~out], atol=1e-12)


def test_wall_ghost_has_zero_mass_flux():
    u = _rand_states(30, 10)
    n = _rand_normals(30, 11)
    ghost, cb = physics.wall_states(u, GAMMA, 1.0)
    Fn = physics.rusanov(u, ghost, n, GAMMA)
    # mass flux of Rusanov: (rho vn - rho vn)/2 - s (rho - rho)/2 = 0
    assert np.max(np.abs(Fn[:, 0])) < 1e-13
    assert np.all(cb[:, 1:4] == 0.0)


# --------------------------------------------------------------------------
# RHS invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["pt", "hp", "hex"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_freestream_preservation_periodic(kind, p, viscous):
    s = _solver(_box(kind), p, viscous=viscous, mu=0.05)
    xyz = s.upts_xyz_points()
    u = s.state_from_points(synth.uniform_state(xyz, vel=(0.3, -0.2, 0.5), p=1.0))
    assert np.max(np.abs(s.rhs(u))) < 1e-12


@pytest.mark.parametrize("viscous", [False, True])
def test_freestream_preservation_farfield_box(viscous):
    """All-far-field box: the free stream is a fixed point of the RHS."""
    m = synth.boundary_layer_box(nx=5, nz=3, n_prism_layers=3, n_tet_layers=3)
    m["bface"][:, 3] = synth.BC_FARFIELD
    pinf = 1.0 / (GAMMA * 0.2 ** 2)
    s = _solver(m, 3, viscous=viscous, mu=1e-3, p_inf=pinf)
    xyz = s.upts_xyz_points()
    u = s.state_from_points(synth.uniform_state(xyz, vel=(1.0, 0.0, 0.0), p=pinf))
    assert np.max(np.abs(s.rhs(u))) < 1e-11 * pinf


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_discrete_conservation(kind, p, viscous):
    s = _solver(_box(kind), p, viscous=viscous, mu=0.05)
    xyz = s.upts_xyz_points()
    u = s.state_from_points(synth.random_smooth_state(xyz, seed=p))
    r = s.rhs(u)
    tot = s.integrals(r)
    scale = s.integrals(np.abs(r))
    assert np.max(np.abs(tot) / scale) < 1e-12


def _permuted_mesh(mesh, perm):
    m = dict(mesh)
    m["xyz"] = mesh["xyz"][:, perm]
    m["period"] = mesh["period"][perm]
    return m


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("p", [2, 3])
def test_axis_permutation_equivariance(kind, p):
    """Cyclically permuting the coordinates of mesh and flow permutes the
    momentum components of the RHS (Euler; every face is re-used under
    another axis, which exercises the face bookkeeping)."""
    mesh = _box(kind)
    perm = [1, 2, 0]
    s1 = _solver(mesh, p)
    s2 = _solver(_permuted_mesh(mesh, perm), p)
    q1 = synth.random_smooth_state(s1.upts_xyz_points(), seed=5)
    u1 = s1.state_from_points(q1)
    q2 = q1.copy()
    q2[:, 1:4] = q1[:, 1:4][:, [1 + perm[k] - 1 for k in range(3)]]
    u2 = s2.state_from_points(q2)
    r1 = s1.split(s1.rhs(u1))
    r2 = s2.split(s2.rhs(u2))
    for t in s1.types:
        np.testing.assert_allclose(r2[t][:, 0], r1[t][:, 0], atol=1e-12)
        np.testing.assert_allclose(r2[t][:, 4], r1[t][:, 4], atol=1e-12)
        np.testing.assert_allclose(r2[t][:, 1:4], r1[t][:, 1:4][:, perm], atol=1e-12)


@pytest.mark.parametrize("kind", ["pt", "hp"])
def test_element_renumbering_invariance(kind):
    """Shuffling element order (and hence face discovery order and the
    a/b roles of every interface) shuffles the NS RHS and nothing else."""
    mesh = _box(kind)
    rng = np.random.default_rng(12)
    m2 = dict(mesh)
    perms = {}
    for t in ("tet", "pri", "hex"):
        if t in mesh and len(mesh[t]):
            perms[t] = rng.permutation(len(mesh[t]))
            m2[t] = mesh[t][perms[t]]
    s1 = _solver(mesh, 2, viscous=True, mu=0.05)
    s2 = _solver(m2, 2, viscous=True, mu=0.05)
    u1 = s1.state_from_points(synth.random_smooth_state(s1.upts_xyz_points(), seed=6))
    u1s = s1.split(u1)
    u2 = s2.join({t: u1s[t][q] for t, q in perms.items()})
    r1 = s1.split(s1.rhs(u1))
    r2 = s2.split(s2.rhs(u2))
    for t, q in perms.items():
        np.testing.assert_allclose(r2[t], r1[t][q], atol=1e-12)


# --------------------------------------------------------------------------
# accuracy
# --------------------------------------------------------------------------
def _l2(s, err):
    e = s.split(err)
    tot = 0.0
    for t in s.types:
        wJ = s.m.ops[t].w[None, :] * s.m.J[t]
        tot += np.sum(wJ[:, None, :] * e[t] ** 2)
    return math.sqrt(tot)


def _vortex_dudt(xyz, h=1e-5):
    """Exact time derivative of the advected vortex: -(vel . grad) u."""
    vel = (1.0, 1.0, 0.0)
    g = np.zeros(xyz.shape[:-1] + (5,))
    for m in range(2):
        d = np.zeros(3)
        d[m] = h
        g -= vel[m] * (synth.isentropic_vortex(xyz + d) - synth.isentropic_vortex(xyz - d)) / (2 * h)
    return g


@pytest.mark.parametrize("p", [2, 3])
def test_vortex_residual_converges(p):
    """The Euler RHS of the exact vortex converges to its exact time
    derivative at the FR/DG residual order p (n = 8 -> 16; coarser meshes
    do not resolve the unit vortex core)."""
    errs = []
    for n in (8, 16):
        s = _solver(synth.vortex_box(n=n), p)
        xyz = s.upts_xyz_points()
        u = s.state_from_points(synth.isentropic_vortex(xyz))
        exact = s.state_from_points(_vortex_dudt(xyz))
        errs.append(_l2(s, s.rhs(u) - exact))
    assert math.log2(errs[0] / errs[1]) >= p - 0.35, errs


def _vortex_solution_error(n, p, T):
    s = _solver(synth.vortex_box(n=n), p)
    xyz = s.upts_xyz_points()
    u = s.state_from_points(synth.isentropic_vortex(xyz))
    nsteps = int(math.ceil(T / (0.1 * s.dt_cfl(u, 1.0))))
    dt = T / nsteps
    for _ in range(nsteps):
        u = s.rk4_step(u, dt)
    return _l2(s, u - s.state_from_points(synth.isentropic_vortex(xyz, t=T)))


def test_vortex_solution_converges():
    """Advect the vortex with RK4 (CFL 0.1) to t = 0.5; at p = 2 the error
    falls by more than 2^2 from n = 4 to n = 8 (pre-asymptotic: the
    asymptotic order p+1 needs finer meshes, see the slow test)."""
    e4, e8 = _vortex_solution_error(4, 2, 0.5), _vortex_solution_error(8, 2, 0.5)
    assert math.log2(e4 / e8) >= 2.0, (e4, e8)


def _vortex_slab(n):
    """Periodic slab [-5,5]^2 x [0, 2h] of n x n x 2 cells (h = 10/n): one
    prism layer under one Kuhn-tet layer, the vortex workload's splitting
    and 5% jitter.  The vortex does not depend on z, so two cell layers
    carry the same solution as the cube at a fraction of the cost."""
    c = np.linspace(-5.0, 5.0, n + 1)
    z = np.linspace(0.0, 2 * 10.0 / n, 3)
    return synth.layered_box((c, c, z), 2, 1, (True, True, True), jitter=0.05, seed=0)


def _slab_error(n, p, T, cfl):
    s = _solver(_vortex_slab(n), p)
    xyz = s.upts_xyz_points()
    u = s.state_from_points(synth.isentropic_vortex(xyz))
    nsteps = int(math.ceil(T / (cfl * s.dt_cfl(u, 1.0))))
    dt = T / nsteps
    for _ in range(nsteps):
        u = s.rk4_step(u, dt)
    err = _l2(s, u - s.state_from_points(synth.isentropic_vortex(xyz, t=T)))
    return err / math.sqrt(s.volume())


@pytest.mark.parametrize("p", [1, 2])
def test_vortex_solution_order_p_plus_one(p):
    """The advected isentropic vortex converges at order p+1 (DG-type FR,
    Sec. 3.4): RK4 to t = 0.5 on the n = 8 and 16 slabs, observed order
    >= p + 1 - 0.5 (errors 1e-3..6e-2, far above the 6e-6 periodic-tail
    floor).  For p = 2 the time step is halved on the finer mesh and the
    error must not move (< 1%): the time error is negligible, the rate is
    spatial.  (Measured on n = 16 -> 32: 2.16 at p = 1, 2.49 at p = 2.)"""
    e8, e16 = _slab_error(8, p, 0.5, 0.25), _slab_error(16, p, 0.5, 0.25)
    assert math.log2(e8 / e16) >= p + 0.5, (e8, e16)
    if p == 2:
        e16h = _slab_error(16, p, 0.5, 0.125)
        assert abs(e16h - e16) < 0.01 * e16, (e16, e16h)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_euler_residual_converges(p):
    """Euler RHS of a smooth periodic field against -div F_inv derived
    symbolically (sympy); observed order >= p - 0.2 on n = 4, 8, 16."""
    _manufactured_rates(p, viscous=False, ns=(4, 8, 16), min_rate=p - 0.2)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_euler_residual_converges_hex_prism(p):
    """The same on hexahedra beside prism pairs (n = 4, 8, 16)."""
    _manufactured_rates(p, viscous=False, ns=(4, 8, 16), min_rate=p - 0.2, kind="hp")


def _manufactured_rates(p, viscous, ns, min_rate, kind="pt"):
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x y z")
    x, y, z = X
    k = 2 * sp.pi / 10
    rho = 1 + sp.Rational(1, 5) * sp.sin(k * x) * sp.cos(k * y)
    vel = [sp.Rational(1, 2) + sp.Rational(1, 4) * sp.sin(k * y + k * z),
           sp.Rational(1, 4) * sp.cos(k * x) * sp.sin(k * z),
           -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.sin(k * (x + y))]
    pr = 2 + sp.Rational(1, 5) * sp.cos(k * (x - z))
    g, Pr = sp.Rational(7, 5), sp.Rational(18, 25)
    mu = sp.Rational(1, 20) if viscous else 0
    E = pr / (g - 1) + rho * sum(v * v for v in vel) / 2
    U = [rho] + [rho * v for v in vel] + [E]
    e = pr / ((g - 1) * rho)
    gv = [[sp.diff(vel[a], X[m]) for m in range(3)] for a in range(3)]
    div = sum(gv[a][a] for a in range(3))
    tau = [[mu * (gv[a][m] + gv[m][a] - (sp.Rational(2, 3) * div if a == m else 0))
            for m in range(3)] for a in range(3)]
    F = []
    for m in range(3):
        Fi = [rho * vel[m]] + [rho * vel[a] * vel[m] + (pr if a == m else 0) for a in range(3)] \
            + [(E + pr) * vel[m]]
        Fv = [0] + [tau[a][m] for a in range(3)] + \
            [sum(vel[a] * tau[a][m] for a in range(3)) + mu * g / Pr * sp.diff(e, X[m])]
        F.append([Fi[q] - Fv[q] for q in range(5)])
    R = [-sum(sp.diff(F[m][q], X[m]) for m in range(3)) for q in range(5)]
    fU = sp.lambdify(X, U, "numpy")
    fR = sp.lambdify(X, R, "numpy")

    def ev(f, xyz):
        out = f(xyz[:, 0], xyz[:, 1], xyz[:, 2])
        return np.stack([np.broadcast_to(np.asarray(c, float), xyz[:, 0].shape) for c in out], -1)

    errs = []
    for n in ns:
        s = _solver(_box(kind, n=n), p, viscous=viscous, mu=float(mu), prandtl=0.72)
        xyz = s.upts_xyz_points()
        u = s.state_from_points(ev(fU, xyz))
        errs.append(_l2(s, s.rhs(u) - s.state_from_points(ev(fR, xyz))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) >= min_rate, (p, errs, rates)


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_navier_stokes_residual_converges(p):
    """NS RHS (mu = 0.05) of the same field against -div(F_inv - F_vis)
    derived symbolically.  The viscous term is a second-order operator, so
    the residual of the interpolated exact field converges at order p - 1;
    a wrong term in the viscous flux, gradient or LDG treatment leaves an
    O(1) residual and a rate near 0.  Observed order >= p - 1.2 on n = 4, 8."""
    _manufactured_rates(p, viscous=True, ns=(4, 8), min_rate=p - 1.2)


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_navier_stokes_residual_converges_hex(p):
    """The same on an all-hexahedral mesh."""
    _manufactured_rates(p, viscous=True, ns=(4, 8), min_rate=p - 1.2, kind="hex")


def test_rk4_amplification(monkeypatch):
    """One step of u' = lam u multiplies u by 1 + z + z^2/2 + z^3/6 + z^4/24."""
    s = _solver(synth.vortex_box(), 1)
    lam = -0.7
    monkeypatch.setattr(s, "rhs", lambda u: lam * u)
    u = np.linspace(1.0, 2.0, s.ndof)
    dt = 0.3
    z = lam * dt
    np.testing.assert_allclose(s.rk4_step(u, dt), u * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24),
                               rtol=1e-15)


def test_rk4_2n_amplification_matches_exp_to_fourth_order():
    """The 2N scheme applied to y' = z y in exact rational arithmetic: its
    amplification polynomial R(z) (degree 5) agrees with exp(z) through z^4,
    i.e. the coefficients satisfy the four order conditions of a linear
    autonomous problem (a mistyped digit anywhere breaks them)."""
    from fractions import Fraction
    from math import factorial
    from oracle.solver import RK4_2N_FRACTIONS
    A, B = RK4_2N_FRACTIONS

    def shift(poly):             # multiply by z
        return [Fraction(0)] + poly

    def add(p, q):
        n = max(len(p), len(q))
        p = p + [Fraction(0)] * (n - len(p))
        q = q + [Fraction(0)] * (n - len(q))
        return [a + b for a, b in zip(p, q)]

    y, du = [Fraction(1)], [Fraction(0)]
    for a, b in zip(A, B):
        du = add([a * c for c in du], shift(y))
        y = add(y, [b * c for c in du])
    for k in range(5):
        assert abs(float(y[k] - Fraction(1, factorial(k)))) < 1e-12, k
    # the z^5 term differs from 1/120 (five stages, order four)
    assert abs(float(y[5]) - 1.0 / 120.0) > 1e-6


def test_rk4_2n_step_order_on_a_scalar_ode():
    """The oracle's step on y' = -y^2 (exact 1/(1+t)): the error falls with
    dt^4."""
    from oracle.solver import RK4_2N_A, RK4_2N_B

    def step(y, dt):
        du = 0.0
        for a, b in zip(RK4_2N_A, RK4_2N_B):
            du = a * du + dt * (-y * y)
            y = y + b * du
        return y

    errs = []
    for n in (10, 20, 40):
        y, dt = 1.0, 1.0 / n
        for _ in range(n):
            y = step(y, dt)
        errs.append(abs(y - 0.5))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.8, rates


# --------------------------------------------------------------------------
# RK45[2R+] (Kennedy, Carpenter & Lewis 2000, RK4(3)5[2R+]C)
# --------------------------------------------------------------------------
def _rk45_tableau():
    """The full Butcher matrix of the two-register structure: A[i][i-1] = a_i,
    A[i][j] = b_j (j < i-1), in exact rationals."""
    from fractions import Fraction
    from oracle.solver import RK45_2R_FRACTIONS
    a, b, bh = RK45_2R_FRACTIONS
    A = [[Fraction(0)] * 5 for _ in range(5)]
    for i in range(1, 5):
        A[i][i - 1] = a[i - 1]
        for j in range(i - 1):
            A[i][j] = b[j]
    return A, list(b), list(bh)


def _order_conditions(A, w):
    """Residuals of the eight Butcher conditions of orders 1-4 for weights w."""
    from fractions import Fraction as Fr
    s = len(w)
    c = [sum(A[i]) for i in range(s)]
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(s)) for i in range(s)]
    dot = lambda x, y: sum(p * q for p, q in zip(x, y))
    return [dot(w, [1] * s) - 1, dot(w, c) - Fr(1, 2),
            dot(w, [x * x for x in c]) - Fr(1, 3), dot(w, Ac) - Fr(1, 6),
            dot(w, [x ** 3 for x in c]) - Fr(1, 4), dot(w, [x * y for x, y in zip(c, Ac)]) - Fr(1, 8),
            dot(w, Ac2) - Fr(1, 12), dot(w, AAc) - Fr(1, 24)]


def test_rk45_2r_coefficients_satisfy_the_order_conditions():
    """b satisfies all eight conditions of order <= 4 and bhat the four of
    order <= 3, to the precision of the published rational approximations
    (~1e-26; a mistyped digit anywhere leaves ~1e-12 or more), while bhat
    misses the order-4 ones (an embedded third-order solution)."""
    A, b, bh = _rk45_tableau()
    rb, rh = _order_conditions(A, b), _order_conditions(A, bh)
    assert max(abs(float(x)) for x in rb) < 1e-20, [float(x) for x in rb]
    assert max(abs(float(x)) for x in rh[:4]) < 1e-20, [float(x) for x in rh]
    assert min(abs(float(x)) for x in rh[4:]) > 1e-3


class _Poly:
    """Polynomial in z with Fraction coefficients (for y' = z y)."""

    def __init__(self, c):
        self.c = list(c)

    def __add__(self, o):
        from fractions import Fraction
        n = max(len(self.c), len(o.c))
        p = self.c + [Fraction(0)] * (n - len(self.c))
        q = o.c + [Fraction(0)] * (n - len(o.c))
        return _Poly([x + y for x, y in zip(p, q)])

    def __rmul__(self, k):
        return _Poly([k * x for x in self.c])


def test_rk45_2r_register_form_amplification_and_error_polynomials():
    """The oracle's two-register step, run in exact rationals on y' = z y:
    its amplification polynomial equals exp(z) through z^4, and its error
    estimate's polynomial dt sum (b - bhat) k vanishes through z^3 (the
    embedded solution is third order) but not at z^4."""
    from fractions import Fraction
    from math import factorial
    from oracle.solver import RK45_2R_FRACTIONS, rk45_2r_step
    a, b, bh = RK45_2R_FRACTIONS
    e = [x - y for x, y in zip(b, bh)]
    y, err = rk45_2r_step(lambda x: _Poly([Fraction(0)] + x.c), _Poly([Fraction(1)]), Fraction(1),
                          a=a, b=b, e=e)
    for k in range(5):
        assert abs(float(y.c[k] - Fraction(1, factorial(k)))) < 1e-20, k
    assert abs(float(y.c[5]) - 1.0 / 120.0) > 1e-6
    for k in range(4):
        assert abs(float(err.c[k])) < 1e-20, k
    assert abs(float(err.c[4])) > 1e-4


def test_rk45_2r_register_form_equals_the_butcher_form_on_a_nonlinear_system():
    """On a nonlinear system the register algorithm gives the stage values
    of the full Butcher matrix: X_i = u + dt sum_j A[i][j] k_j, u_{n+1} =
    u + dt sum b_i k_i, uhat = u + dt sum bhat_i k_i."""
    from oracle.solver import rk45_2r_step
    A, b, bh = _rk45_tableau()
    A = [[float(x) for x in row] for row in A]
    b, bh = [float(x) for x in b], [float(x) for x in bh]

    def f(u):
        return np.array([u[1] * u[2] - 0.3 * u[0], -u[0] * u[2] + np.sin(u[0]), 0.5 * u[0] * u[1] - u[2] ** 2])

    u0, dt = np.array([0.8, -0.4, 1.1]), 0.17
    ks = []
    for i in range(5):
        ks.append(f(u0 + dt * sum(A[i][j] * ks[j] for j in range(i)) if i else u0))
    y_ref = u0 + dt * sum(bi * k for bi, k in zip(b, ks))
    yh_ref = u0 + dt * sum(bi * k for bi, k in zip(bh, ks))
    y, err = rk45_2r_step(f, u0, dt)
    np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(err, y_ref - yh_ref, rtol=0, atol=1e-15)


def test_rk45_2r_orders_on_a_scalar_ode():
    """y' = -y^2 (exact 1/(1+t)): the global error of the oracle's step falls
    with dt^4, and the one-step error estimate with dt^4 (the local error of
    the third-order embedded solution)."""
    from oracle.solver import rk45_2r_step
    f = lambda y: -y * y
    errs, ests = [], []
    for n in (10, 20, 40):
        y, dt = 1.0, 1.0 / n
        for _ in range(n):
            y, _ = rk45_2r_step(f, y, dt)
        errs.append(abs(y - 0.5))
        ests.append(abs(rk45_2r_step(f, 1.0, 1.0 / n)[1]))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    erates = [np.log2(ests[i] / ests[i + 1]) for i in range(2)]
    assert min(rates) > 3.8, rates
    assert min(erates) > 3.7 and max(erates) < 4.3, erates


def test_rk45_adaptive_reaches_the_end_time_within_tolerance(monkeypatch):
    """The adaptive driver on u' = -u^2 per component (exact u0/(1+u0 t)):
    it ends exactly at t_span, the global error follows the tolerance, and
    a large first step is rejected and shrunk."""
    s = _solver(synth.vortex_box(), 1)
    monkeypatch.setattr(s, "rhs", lambda u: -u * u)
    u0 = np.linspace(0.5, 2.0, s.ndof)
    exact = u0 / (1.0 + u0 * 2.0)
    errs = []
    for tol in (1e-6, 1e-8):
        u, dt, acc, rej = s.rk45_adaptive(u0, 2.0, 1.5, tol, tol)
        errs.append(float(np.max(np.abs(u - exact))))
        assert rej >= 1 and acc >= 3
    assert errs[0] < 1e-4 and errs[1] < errs[0] / 10, errs


def test_ldg_beta_half_takes_one_side():
    """With beta = 1/2 the LDG weights 1/2 +- beta are 1 and 0: the common
    solution is the left side's value (side a where the switch is +1) and
    the common viscous flux the right side's, up to rounding.  The face
    kernels of the GPU path rely on this identity to read and form one
    side only; a sign slip of beta or of the switch would swap the sides."""
    rng = np.random.default_rng(3)
    n_pts = 64
    ua, ub = rng.normal(size=(n_pts, 5)), rng.normal(size=(n_pts, 5))
    sign = np.where(rng.random(n_pts) > 0.5, 1.0, -1.0)
    C = physics.ldg_common_solution(ua, ub, sign, 0.5)
    np.testing.assert_allclose(C, np.where(sign[:, None] > 0, ua, ub), rtol=0, atol=1e-15)
    fva, fvb = rng.normal(size=(n_pts, 5, 3)), rng.normal(size=(n_pts, 5, 3))
    nrm = rng.normal(size=(n_pts, 3))
    F = physics.ldg_viscous_normal(fva, fvb, nrm, sign, 0.5)
    fa = np.einsum("pvm,pm->pv", fva, nrm)
    fb = np.einsum("pvm,pm->pv", fvb, nrm)
    np.testing.assert_allclose(F, np.where(sign[:, None] > 0, fb, fa), rtol=0, atol=1e-14)
    # any other beta mixes both sides
    F3 = physics.ldg_viscous_normal(fva, fvb, nrm, sign, 0.3)
    assert np.all(np.abs(F3 - np.where(sign[:, None] > 0, fb, fa)) > 0)
