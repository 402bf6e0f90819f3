"""GPU tests of the FR_FP32 mode's streamed operator kernel (fr_gemm_f32.cu):
TMA-streamed state, operator slabs per stage, 4 x 4 register tiles per
lane, zero 4-row blocks skipped per column.

Every output is the FMA chain over the operator's non-zero columns in
increasing order, as in the chunk-staged kernel the batched engine runs,
so a batch's per-problem steps (this kernel) and its batched steps (the
chunk-staged kernel) are bitwise equal; test_gpu_batch checks that for
Euler and Navier-Stokes.  Here: RK4 states against the oracle over orders
1-4, both element types and hexahedra (the p = 4 hexahedral gradient
needs two row passes), ragged column tiles, and the bounded-wait
self-test (GPU)."""
import numpy as np
import pytest

import synth
from tests import _cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 RHS: a few 1e-6 of its scale; over 3 steps the state increment
# carries that error
TOL = 1e-4


def _fr():
    _cases.library()
    from paper_1409_0405_gb300 import fr
    return fr


def _steps(sol, ctx, u, dt, n):
    ctx.set_state(u)
    ctx.step(dt, n)
    got = ctx.get_state()
    ref = u
    for _ in range(n):
        ref = sol.rk4_step(ref, dt)
    return _cases.per_quantity_rel_err(sol, ref - u, got - u)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_fp32_steps_match_oracle(p, viscous):
    fr = _fr()
    mesh = synth.vortex_box(n=4, jitter=0.05, seed=0)
    prm = dict(viscous=viscous, mu=0.01 if viscous else 0.0, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    sol, ctx = _cases.make_pair(mesh, p, precision=fr.FR_FP32, **prm)
    u = _cases.state(sol, "vortex")
    err = _steps(sol, ctx, u, sol.dt_cfl(u, 0.1), 3)
    print(p, viscous, err)
    assert np.all(err < TOL), err
    # the plain RHS (interpolation and gradients on the streamed kernel)
    e1 = _cases.per_quantity_rel_err(sol, sol.rhs(u), _cases.gpu_rhs(ctx, u))
    assert np.all(e1 < TOL), e1
    ctx.reduce()


@pytest.mark.parametrize("p", [2, 4])
def test_fp32_hexahedra_two_row_passes(p):
    """Hexahedra beside prisms, Navier-Stokes: at p = 4 the gradient operator
    has 375 rows, two passes of the streamed kernel."""
    fr = _fr()
    m = synth.hex_box(n=3, n_hex_cols=2)
    sol, ctx = _cases.make_pair(m, p, viscous=True, mu=0.02, precision=fr.FR_FP32)
    u = _cases.state(sol, "smooth", seed=4)
    err = _steps(sol, ctx, u, sol.dt_cfl(u, 0.1), 2)
    print(p, err)
    assert np.all(err < TOL), err
    ctx.reduce()


def test_fp32_ragged_tiles_wall_and_far_field():
    """A boundary-layer box whose element counts leave ragged 128-column
    tiles, with wall and far-field boundaries (Navier-Stokes, p = 3)."""
    fr = _fr()
    m = synth.boundary_layer_box(nx=5, nz=3, n_prism_layers=3, n_tet_layers=2)
    sol, ctx = _cases.make_pair(m, 3, precision=fr.FR_FP32, **_cases.bl_params(mu=0.01))
    assert ctx.info["n_pri"] % 128 and ctx.info["n_tet"] % 128
    u = _cases.state(sol, "bl")
    err = _steps(sol, ctx, u, 0.2 * sol.dt_cfl(u, 0.1), 2)
    print(err)
    assert np.all(err < TOL), err
    ctx.reduce()


def test_fp32_bounded_wait_timeout_is_reported():
    """Failure detection without a GPU fault: the streamed kernel launched
    with its copies withheld lets every bounded wait run out (~2 s),
    reports FR_ERR_TIMEOUT through the context status, which the self-test
    checks and clears; the same context then steps correctly."""
    fr = _fr()
    mesh = synth.vortex_box(n=4, jitter=0.05, seed=0)
    sol, ctx = _cases.make_pair(mesh, 2, precision=fr.FR_FP32, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0)
    u = _cases.state(sol, "vortex")
    ctx.set_state(u)
    ctx.selftest_wait_timeout()
    err = _steps(sol, ctx, u, sol.dt_cfl(u, 0.1), 2)
    assert np.all(err < TOL), err
    ctx.reduce()
