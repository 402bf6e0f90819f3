"""CUDA path against the oracle, element by element (GPU).

Tolerance: the FP64 path must match the oracle to 1e-12 relative on the
RHS and on states after RK4 steps, per conserved quantity: mass, momentum
(the Euclidean norm of the 3-vector, so the measure does not depend on the
orientation of the axes) and energy, each max over points |gpu - oracle|
divided by max over points |oracle|.  Cases span several GEMM column tiles with ragged
tails, both element types alone and mixed, orders 1..4, Euler and
Navier-Stokes, periodic, wall and far-field boundaries, and the full-size
boundary-layer workload (57,600 prisms + 118,800 tets, p = 4).
"""
import math

import numpy as np
import pytest

import synth
from tests._cases import (GAMMA, bl_params, gpu_rhs, library, make_pair, per_quantity_rel_err,
                          per_var_rel_err, state, to_longdouble)

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    library()


def _check_rhs(sol, ctx, u, tol=TOL):
    ref = sol.rhs(u)
    got = gpu_rhs(ctx, u)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= tol), (err, per_var_rel_err(sol, ref, got))
    return err


def test_solution_points_match_oracle():
    sol, ctx = make_pair(synth.vortex_box(), 3)
    np.testing.assert_allclose(ctx.upts(), sol.upts_xyz(), atol=1e-13)


def test_vortex_euler_p2_rhs():
    """The isentropic-vortex workload: 64 prisms + 192 tets, p = 2, Euler."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    _check_rhs(sol, ctx, state(sol, "vortex"))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_rhs_all_orders_periodic(p, viscous):
    sol, ctx = make_pair(synth.vortex_box(), p, viscous=viscous, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=p))


@pytest.mark.parametrize("p", [2, 4])
def test_rhs_wall_and_farfield_ns(p):
    """No-slip wall, far field and a periodic axis, stretched jittered
    prism layers under Kuhn tets."""
    m = synth.boundary_layer_box(nx=7, nz=3, n_prism_layers=5, n_tet_layers=3)
    sol, ctx = make_pair(m, p, **bl_params(mu=0.01))
    _check_rhs(sol, ctx, state(sol, "bl"))


@pytest.mark.parametrize("precision", ["FR_FP64", "FR_FP32"])
@pytest.mark.parametrize("beta", [0.3, -0.5])
def test_rhs_ldg_beta_general(beta, precision):
    """LDG weights other than beta = 1/2 (where the common viscous flux is
    one side's flux and the kernels read only that side's gradient): both
    sides' viscous fluxes are combined with weights 1/2 -+ beta (walls,
    far field and periodic faces)."""
    from paper_1409_0405_gb300 import fr
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    prm = dict(bl_params(mu=0.01), ldg_beta=beta)
    sol, ctx = make_pair(m, 3, precision=getattr(fr, precision), **prm)
    _check_rhs(sol, ctx, state(sol, "bl"), tol=TOL if precision == "FR_FP64" else 1e-4)


def test_rhs_impulsive_start_within_fp64_floor():
    """The impulsive start (free stream slipping over the no-slip wall) puts
    an O(1) jump at the wall, gradients ~1/h and wall RHS ~mu/h^2, so every
    FP64 evaluation carries rounding amplified by the conditioning.  The
    oracle re-run in numpy extended precision measures that floor; the GPU
    must stay within 8x the FP64 oracle's own distance from it (and within
    1e-11 absolutely)."""
    m = synth.boundary_layer_box(nx=7, nz=3, n_prism_layers=5, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "impulsive")
    r64 = sol.rhs(u)
    rld = to_longdouble(make_pair(m, 3, **bl_params(mu=0.01))[0]).rhs(
        u.astype(np.longdouble)).astype(np.float64)
    got = gpu_rhs(ctx, u)
    floor = per_var_rel_err(sol, rld, r64)
    err = per_var_rel_err(sol, rld, got)
    assert np.all(err <= np.maximum(8.0 * floor, TOL)), (err, floor)
    assert np.all(err <= 1e-11), err


@pytest.mark.parametrize("n,npl", [(5, 2), (6, 0), (3, 3), (7, 3)])
def test_rhs_ragged_and_single_type(n, npl):
    """Element counts that are not multiples of the padding or the column
    tile; tets only (npl = 0) and prisms only (npl = n)."""
    m = synth.vortex_box(n=n, n_prism_layers=npl)
    sol, ctx = make_pair(m, 3, viscous=True, mu=0.02)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=n))


def test_vortex_rk4_100_steps():
    """The vortex workload advanced 100 RK4 steps at CFL 0.1."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 100)
    got = ctx.get_state()
    ref = u
    for _ in range(100):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= TOL), err
    # conserved totals (periodic box) do not drift
    out = ctx.reduce()
    np.testing.assert_allclose(out[:5], sol.integrals(u), rtol=1e-12, atol=1e-9)


def test_vortex_low_storage_rk_steps():
    """fr_step_ls (five-stage 2N Runge-Kutta) against the oracle's scheme:
    the vortex (Euler) for 20 steps and the boundary layer (NS) for 3."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step_ls(dt, 20)
    ref = u
    for _ in range(20):
        ref = sol.rk4_2n_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err
    np.testing.assert_allclose(ctx.reduce()[:5], sol.integrals(u), rtol=1e-12, atol=1e-9)
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step_ls(dt, 3)
    ref = u
    for _ in range(3):
        ref = sol.rk4_2n_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err


def test_ns_boundary_layer_rk4_steps():
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 3)
    ref = u
    for _ in range(3):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err


def test_reductions_match_oracle():
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    ctx.set_state(u)
    out = ctx.reduce()
    np.testing.assert_allclose(out[:5], sol.integrals(u), rtol=1e-13)
    np.testing.assert_allclose(out[5], sol.kinetic_energy(u), rtol=1e-13)
    assert out[6] == 0.0


def _diag_scales(sol, u):
    """Cancellation-free magnitudes of the kinetic-energy rate's terms."""
    uu, rr = sol.split(u), sol.split(sol.rhs(u))
    tot = 0.0
    for t in sol.types:
        wJ = sol.m.ops[t].w[None, :] * sol.m.J[t]
        v = uu[t][:, 1:4, :] / uu[t][:, 0:1, :]
        tot += float(np.sum(wJ * (np.sum(np.abs(v * rr[t][:, 1:4, :]), axis=1)
                                  + 0.5 * np.sum(v * v, axis=1) * np.abs(rr[t][:, 0, :]))))
    return tot


def _check_diagnostics(sol, ctx, u, tol_rate, tol_inv, tol_vis):
    ctx.set_state(u)
    rate, f_inv, f_vis = ctx.diagnostics()
    o_inv, o_vis = sol.wall_force(u)
    assert abs(rate - sol.ke_rate(u)) <= tol_rate * _diag_scales(sol, u)
    assert np.max(np.abs(f_inv - o_inv)) <= tol_inv * max(np.linalg.norm(o_inv), 1e-300)
    assert np.max(np.abs(f_vis - o_vis)) <= tol_vis * max(np.linalg.norm(o_vis), 1e-300)
    # the solution register is untouched
    np.testing.assert_array_equal(ctx.get_state(), u)
    return rate, f_inv, f_vis


@pytest.mark.parametrize("p", [2, 3])
def test_diagnostics_wall_bounded_match_oracle(p):
    """Kinetic-energy rate and wall force (pressure and viscous parts) on
    the wall/far-field box with a wall-consistent boundary-layer state."""
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, p, **bl_params(mu=0.01))
    u = state(sol, "bl")
    _, f_inv, f_vis = _check_diagnostics(sol, ctx, u, 1e-12, 1e-12, 1e-10)
    assert f_inv[1] < 0.0 and f_vis[0] > 0.0   # pressure pushes on, flow drags along


def test_diagnostics_periodic_match_oracle():
    """No walls: zero force; the kinetic-energy rate of the Euler vortex."""
    sol, ctx = make_pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    _, f_inv, f_vis = _check_diagnostics(sol, ctx, u, 1e-12, 0.0, 0.0)
    assert np.all(f_inv == 0.0) and np.all(f_vis == 0.0)


def test_diagnostics_plane_shear_closed_form():
    """Channel with a wall at y = 0 and u = a y: viscous wall force mu a A,
    pressure force -p0 A along y (the oracle pins these to rounding)."""
    mu, a, p0 = 0.01, 0.3, 1.0 / GAMMA
    m = synth.wall_channel(n_prism_layers=2)
    sol, ctx = make_pair(m, 2, viscous=True, mu=mu, p_inf=p0, t_wall=p0)
    u = sol.state_from_points(synth.shear_flow(sol.upts_xyz_points(), a=a, p=p0))
    ctx.set_state(u)
    _, f_inv, f_vis = ctx.diagnostics()
    area = 2.0
    np.testing.assert_allclose(f_vis, [mu * a * area, 0.0, 0.0], rtol=0, atol=1e-11 * mu * a * area)
    np.testing.assert_allclose(f_inv, [0.0, -p0 * area, 0.0], rtol=0, atol=1e-12 * p0 * area)


@pytest.mark.parametrize("prec, tol", [("fp32", 2e-5), ("bf16x3", 5e-4), ("tf32x3", 2e-5)])
def test_diagnostics_reduced_precision(prec, tol):
    from paper_1409_0405_gb300 import fr
    mode = {"fp32": fr.FR_FP32, "bf16x3": fr.FR_BF16X3, "tf32x3": fr.FR_TF32X3}[prec]
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, precision=mode, **bl_params(mu=0.01))
    u = state(sol, "bl")
    _check_diagnostics(sol, ctx, u, tol, tol, 10 * tol)


def test_nonphysical_state_is_reported():
    from paper_1409_0405_gb300 import fr
    sol, ctx = make_pair(synth.vortex_box(), 1)
    u = state(sol, "vortex")
    bad = u.copy()
    bad[0] = -1.0            # negative density at point 0 of element 0
    bad[7] = np.nan          # a non-finite momentum at point 3 of element 0
    ctx.set_state(bad)
    with pytest.raises(fr.FRError) as ei:
        ctx.reduce()
    assert ei.value.code == fr.FR_ERR_NONFINITE
    assert ctx.reduce(check=False)[6] == 2.0


def test_state_roundtrip_and_launch_count():
    sol, ctx = make_pair(synth.vortex_box(), 2, viscous=True, mu=0.01)
    u = state(sol, "smooth", seed=9)
    ctx.set_state(u)
    np.testing.assert_array_equal(ctx.get_state(), u)
    ctx.profile(True)
    ctx.step(1e-4, 2)
    classes, launches = ctx.profile_read()
    # per RK stage: 2 types x (M0, grad, M0 grad, flux, div) + 2 face kernels;
    # per fr_step call: the state check, one launch per type
    assert launches == 2 * 4 * 12 + 2
    assert classes["check"][1] == 2
    assert sum(c for _, c in classes.values()) == launches
    ctx.profile(False)


def test_full_size_boundary_layer_rhs():
    """The full boundary-layer workload: 57,600 prisms + 118,800 tets at
    p = 4, Navier-Stokes, Re = 3900, Ma = 0.2: every output of one RHS."""
    m = synth.boundary_layer_box()
    sol, ctx = make_pair(m, 4, **bl_params())
    u = state(sol, "bl")
    err = _check_rhs(sol, ctx, u)
    assert math.isfinite(float(err.max()))


def test_full_size_boundary_layer_rk4_step():
    """The full boundary-layer workload (57,600 prisms + 118,800 tets, p = 4,
    Navier-Stokes, Re = 3900, Ma = 0.2) advanced one RK4 step: the state
    against the oracle's RK4 step, every value, and the step's increment
    u_1 - u_0 (which carries all of the arithmetic's error) at the RHS
    tolerance as well."""
    m = synth.boundary_layer_box()
    sol, ctx = make_pair(m, 4, **bl_params())
    u = state(sol, "bl")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 1)
    got = ctx.get_state()
    ref = sol.rk4_step(u, dt)
    err = per_quantity_rel_err(sol, ref, got)
    inc = per_quantity_rel_err(sol, ref - u, got - u)
    print("full-size RK4 step: state", err, "increment", inc)
    assert np.all(err <= TOL), err
    assert np.all(inc <= TOL), (inc, per_var_rel_err(sol, ref - u, got - u))


# ---------------------------------------------------------------------------
# FR_FP32: operator applications and point-wise work in FP32, RK registers,
# the reference-flux correction and the reductions in FP64.  Reported against
# the FP64 oracle; the tolerances bound the measured single-precision error.
# ---------------------------------------------------------------------------
FP32_RHS_TOL = 2e-5


@pytest.mark.parametrize("viscous", [False, True])
def test_fp32_rhs_error_periodic(viscous):
    from paper_1409_0405_gb300 import fr
    sol, ctx = make_pair(synth.vortex_box(), 3, viscous=viscous, mu=0.05, precision=fr.FR_FP32)
    u = state(sol, "smooth", seed=4)
    err = per_quantity_rel_err(sol, sol.rhs(u), gpu_rhs(ctx, u))
    print("fp32 rhs error (mass, momentum, energy):", err)
    assert np.all(err <= FP32_RHS_TOL), err


def test_fp32_rhs_error_wall_bounded():
    from paper_1409_0405_gb300 import fr
    m = synth.boundary_layer_box(nx=7, nz=3, n_prism_layers=5, n_tet_layers=3)
    sol, ctx = make_pair(m, 4, **bl_params(), precision=fr.FR_FP32)
    u = state(sol, "bl")
    err = per_quantity_rel_err(sol, sol.rhs(u), gpu_rhs(ctx, u))
    print("fp32 wall-bounded rhs error:", err)
    assert np.all(err <= FP32_RHS_TOL), err


def test_fp32_rk4_vortex_state_error():
    """100 RK4 steps of the vortex in FR_FP32: the state increment
    u(T) - u(0) against the FP64 oracle's."""
    from paper_1409_0405_gb300 import fr
    sol, ctx = make_pair(synth.vortex_box(), 2, precision=fr.FR_FP32)
    u0 = state(sol, "vortex")
    dt = sol.dt_cfl(u0, 0.1)
    ctx.set_state(u0)
    ctx.step(dt, 100)
    got = ctx.get_state()
    ref = u0
    for _ in range(100):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref - u0, got - u0)
    print("fp32 100-step increment error:", err)
    assert np.all(err <= 1e-4), err
    # FP64 reductions of the FP64 register: the FP32 fluxes conserve the
    # totals only to single-precision rounding of the RHS sums
    out = ctx.reduce()
    tot = sol.integrals(u0)
    assert np.max(np.abs(out[:5] - tot)) <= 1e-7 * np.max(np.abs(tot)), (out[:5], tot)


def test_rhs_is_deterministic_and_writes_every_output():
    """Run-twice determinism of the FP64 RHS (bitwise), and every output
    written: an output buffer poisoned with NaN comes back finite."""
    import torch
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    ut = torch.from_numpy(u).cuda()
    outs = []
    for _ in range(2):
        rt = torch.full_like(ut, float("nan"))
        ctx.rhs(ut.data_ptr(), rt.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        outs.append(rt.cpu().numpy())
    assert np.all(np.isfinite(outs[0]))
    np.testing.assert_array_equal(outs[0], outs[1])


def test_checkpoint_resume_is_bitwise():
    """Checkpoint/resume through the public state: 2 + 2 RK4 steps with the
    state read back and set into a fresh context in between equal 4 steps
    bitwise (FP64)."""
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = make_pair(m, 2, **bl_params(mu=0.01))
    u = state(sol, "bl")
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 4)
    full = ctx.get_state()
    ctx.set_state(u)
    ctx.step(dt, 2)
    mid = ctx.get_state()
    _, ctx2 = make_pair(m, 2, **bl_params(mu=0.01))
    ctx2.set_state(mid)
    ctx2.step(dt, 2)
    np.testing.assert_array_equal(ctx2.get_state(), full)
