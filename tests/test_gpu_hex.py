"""GPU parity on meshes with hexahedra (Table 2's third element type; the
paper's hexahedral cylinder mesh, Sec. 3.2): the CUDA path against the
oracle on all-hex and hex/prism meshes, every order, Euler and
Navier-Stokes, periodic and wall-bounded, RHS, RK4 steps, diagnostics, the
reduced-precision modes and batching."""
import numpy as np
import pytest

import synth
from tests._cases import (bl_params, gpu_rhs, library, make_pair, per_quantity_rel_err,
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


def _box(kind, n=4):
    return synth.hex_box(n=n, n_hex_cols=n if kind == "hex" else n // 2)


def _check_rhs(sol, ctx, u, tol=TOL):
    ref = sol.rhs(u)
    got = gpu_rhs(ctx, u)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= tol), (err, per_var_rel_err(sol, ref, got))
    return err


def test_hex_solution_points_match_oracle():
    sol, ctx = make_pair(_box("hp"), 3)
    np.testing.assert_allclose(ctx.upts(), sol.upts_xyz(), atol=1e-13)
    assert ctx.info["n_hex"] == 32 and ctx.info["nu_hex"] == 64 and ctx.info["nf_hex"] == 96


@pytest.mark.parametrize("kind", ["hex", "hp"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_hex_rhs_all_orders_periodic(kind, p, viscous):
    sol, ctx = make_pair(_box(kind), p, viscous=viscous, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=p))


@pytest.mark.parametrize("n", [3, 5])
def test_hex_rhs_ragged(n):
    """Odd element counts (not multiples of the padding or a column tile)."""
    sol, ctx = make_pair(synth.hex_box(n=n, n_hex_cols=n - 1), 2, viscous=True, mu=0.02)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=n))


def _channel():
    return synth.wall_channel(nx=4, ny=3, nz=3, n_prism_layers=3, n_hex_cols=2)


@pytest.mark.parametrize("p", [2, 4])
def test_hex_rhs_wall_bounded_ns(p):
    """Hexahedra and prisms on a no-slip wall under a far field.  The case
    is ill-conditioned for its RHS scale (far-field pressure 17.9, max|R|
    about 3), so the FP64 oracle itself sits ~1e-12 from the exact result:
    the GPU must stay within 8x the oracle's own distance from the
    extended-precision evaluation (and within 1e-11)."""
    sol, ctx = make_pair(_channel(), p, **bl_params(mu=0.01))
    u = state(sol, "bl")
    r64 = sol.rhs(u)
    rld = to_longdouble(make_pair(_channel(), p, **bl_params(mu=0.01))[0]).rhs(
        u.astype(np.longdouble)).astype(np.float64)
    got = gpu_rhs(ctx, u)
    floor = per_var_rel_err(sol, rld, r64)
    err = per_var_rel_err(sol, rld, got)
    assert np.all(err <= np.maximum(8.0 * floor, TOL)), (err, floor)
    assert np.all(err <= 1e-11), err


def test_hex_rk4_steps():
    sol, ctx = make_pair(_box("hp"), 3, viscous=True, mu=0.02, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 4)
    ref = u
    for _ in range(4):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err


def test_hex_reductions_and_diagnostics():
    sol, ctx = make_pair(_channel(), 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    ctx.set_state(u)
    out = ctx.reduce()
    np.testing.assert_allclose(out[:5], sol.integrals(u), rtol=1e-13)
    np.testing.assert_allclose(out[5], sol.kinetic_energy(u), rtol=1e-13)
    rate, f_inv, f_vis = ctx.diagnostics()
    o_inv, o_vis = sol.wall_force(u)
    np.testing.assert_allclose(rate, sol.ke_rate(u), rtol=1e-10)
    assert np.max(np.abs(f_inv - o_inv)) <= 1e-12 * np.linalg.norm(o_inv)
    assert np.max(np.abs(f_vis - o_vis)) <= 1e-10 * np.linalg.norm(o_vis)


def _mode(prec):
    from paper_1409_0405_gb300 import fr
    return {"fp32": fr.FR_FP32, "bf16x3": fr.FR_BF16X3, "tf32x3": fr.FR_TF32X3}[prec]


@pytest.mark.parametrize("prec, tol", [("fp32", 5e-5), ("tf32x3", 5e-5), ("bf16x3", 3e-3)])
@pytest.mark.parametrize("p", [2, 3])
def test_hex_reduced_precision_rhs_periodic(prec, tol, p):
    """Hexahedra beside prisms, Navier-Stokes, a smooth state (the FP32
    rounding floor of a plain evaluation is ~1e-5 here).  Split BF16 keeps
    16 significant bits of each factor and drops the low x low product
    (~2^-16 relative per product); the derivative operators' cancellation
    (sum |a||b| / |sum ab| of order 50 on this state) gives ~1e-3."""
    sol, ctx = make_pair(_box("hp"), p, precision=_mode(prec), viscous=True, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=p), tol=tol)
    ctx.reduce(check=False)


@pytest.mark.parametrize("prec, fac", [("fp32", 10.0), ("tf32x3", 10.0), ("bf16x3", 100.0)])
def test_hex_reduced_precision_rhs_wall_bounded(prec, fac):
    """The ill-conditioned wall case: within a factor of the rounding floor
    of the oracle evaluated in plain single precision."""
    sol, ctx = make_pair(_channel(), 3, precision=_mode(prec), **bl_params(mu=0.01))
    u = state(sol, "bl")
    ref = sol.rhs(u)
    r32 = to_longdouble(make_pair(_channel(), 3, **bl_params(mu=0.01))[0], np.float32).rhs(
        u.astype(np.float32)).astype(np.float64)
    floor = per_quantity_rel_err(sol, ref, r32)
    err = per_quantity_rel_err(sol, ref, gpu_rhs(ctx, u))
    assert np.all(err <= fac * floor), (err, floor)
    ctx.reduce(check=False)


def test_hex_tensor_cores_p4():
    """p = 4 hexahedra on the tensor cores: the gradient operator's 375 rows
    run as two row blocks; split TF32 streams every operator and works
    (checked against the oracle), while split BF16's resident images do
    not fit beside a ring: creation fails cleanly with FR_ERR_UNSUPPORTED."""
    from paper_1409_0405_gb300 import fr
    with pytest.raises(fr.FRError) as ei:
        fr.Context(_box("hex"), 4, precision=fr.FR_BF16X3)
    assert ei.value.code == fr.FR_ERR_UNSUPPORTED
    sol, ctx = make_pair(_box("hp"), 4, precision=fr.FR_TF32X3, viscous=True, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=4), tol=5e-5)
    ctx.reduce(check=False)
    ctx.set_state(state(sol, "smooth", seed=4))
    ctx.step(1e-4, 2)
    ctx.reduce()  # finite, no timeout


def test_hex_batch_matches_per_problem():
    """A batch with hex, hex/prism and prism/tet problems: the grouped,
    graph-replayed launches give bit-identical states to each problem's own
    launch sequence."""
    from paper_1409_0405_gb300 import fr
    probs = [(synth.hex_box(n=3, n_hex_cols=3, seed=21), 2), (synth.hex_box(n=4, n_hex_cols=2, seed=22), 3),
             (synth.vortex_box(n=3, n_prism_layers=1, seed=23), 1), (synth.hex_box(n=2, n_hex_cols=1, seed=24), 4)]
    prm = dict(viscous=False, precision=fr.FR_FP32, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0, rho_inf=1.0)
    states = []
    for batched in (True, False):
        b = fr.Batch([m for m, _ in probs], [p for _, p in probs], **prm)
        for c in b.problems:
            q = synth.isentropic_vortex(c.upts_points())
            out, off = [], 0
            for ne, nu in c.counts():
                if ne:
                    out.append(q[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1).reshape(-1))
                    off += ne * nu
            c.set_state(np.concatenate(out))
        b.step([2e-3] * len(probs), 3, batched=batched)
        states.append([c.get_state() for c in b.problems])
        b.close()
    for a, g in zip(*states):
        np.testing.assert_array_equal(a, g)
