"""GPU parity on quadratically curved meshes (10-node tets, 18-node
prisms, 27-node hexes; the paper's cylinder mesh is quadratically curved):
the CUDA path's geometry (its own quadratic shape functions) against the
oracle's, through the RHS, RK4 steps and diagnostics."""
import numpy as np
import pytest

import synth
from tests._cases import (bl_params, gpu_rhs, library, make_pair, per_quantity_rel_err,
                          per_var_rel_err, state)

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    library()


def _curved(kind, n=4, amp=0.15):
    m0 = synth.vortex_box(n=n) if kind == "pt" else synth.hex_box(n=n, n_hex_cols=n // 2)
    return synth.curve_mesh(m0, amp=amp)


def _check_rhs(sol, ctx, u, tol=TOL):
    ref = sol.rhs(u)
    got = gpu_rhs(ctx, u)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= tol), (err, per_var_rel_err(sol, ref, got))


def test_curved_solution_points_match_oracle():
    sol, ctx = make_pair(_curved("hp"), 3)
    np.testing.assert_allclose(ctx.upts(), sol.upts_xyz(), atol=1e-13)


@pytest.mark.parametrize("kind", ["pt", "hp"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_curved_rhs_all_orders(kind, p, viscous):
    sol, ctx = make_pair(_curved(kind), p, viscous=viscous, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=p))


def test_curved_straight_nodes_equal_straight_mesh():
    """Quadratic nodes on the straight elements: the same RHS as the
    straight-sided mesh (to rounding of the geometry)."""
    from paper_1409_0405_gb300 import fr
    m0 = synth.hex_box(n=4, n_hex_cols=2)
    sol, c0 = make_pair(m0, 3, viscous=True, mu=0.05)
    c1 = fr.Context(synth.curve_mesh(m0, amp=0.0), 3, viscous=True, mu=0.05)
    u = state(sol, "smooth", seed=7)
    r0, r1 = gpu_rhs(c0, u), gpu_rhs(c1, u)
    assert np.max(np.abs(r1 - r0)) <= 1e-12 * np.max(np.abs(r0))


def test_curved_rk4_steps():
    sol, ctx = make_pair(_curved("pt"), 3, viscous=True, mu=0.02, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 4)
    ref = u
    for _ in range(4):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err


def test_curved_wall_channel_diagnostics():
    """A curved channel (wall at y = 0 stays planar): reductions and the
    kinetic-energy rate and wall force against the oracle."""
    m = synth.curve_mesh(synth.wall_channel(nx=4, ny=4, nz=3, n_prism_layers=2), amp=0.15)
    sol, ctx = make_pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    ctx.set_state(u)
    out = ctx.reduce()
    np.testing.assert_allclose(out[:5], sol.integrals(u), rtol=1e-13)
    rate, f_inv, f_vis = ctx.diagnostics()
    o_inv, o_vis = sol.wall_force(u)
    np.testing.assert_allclose(rate, sol.ke_rate(u), rtol=1e-9)
    assert np.max(np.abs(f_inv - o_inv)) <= 1e-12 * np.linalg.norm(o_inv)
    assert np.max(np.abs(f_vis - o_vis)) <= 1e-10 * np.linalg.norm(o_vis)


@pytest.mark.parametrize("prec, tol", [("fp32", 5e-5), ("tf32x3", 5e-5), ("bf16x3", 3e-3)])
def test_curved_reduced_precision(prec, tol):
    from paper_1409_0405_gb300 import fr
    mode = {"fp32": fr.FR_FP32, "bf16x3": fr.FR_BF16X3, "tf32x3": fr.FR_TF32X3}[prec]
    sol, ctx = make_pair(_curved("pt"), 3, precision=mode, viscous=True, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=3), tol=tol)
    ctx.reduce(check=False)


def test_curved_geometry_arguments():
    """geom_order 2 without the node array of a present type is a mesh error."""
    from paper_1409_0405_gb300 import fr
    m = dict(_curved("pt"))
    del m["pri_nodes"]
    with pytest.raises(fr.FRError) as ei:
        fr.Context(m, 2)
    assert ei.value.code == fr.FR_ERR_MESH
