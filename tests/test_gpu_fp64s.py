"""FR_FP64S: FP64 with the operator products of dense-operator element
types (tetrahedra) on the tensor cores by exact splitting (GPU).

The kernel's products are checked against exact products of the FP64
operands (error-free products summed by math.fsum, one rounding), on
operands chosen to stress the split: wide exponent ranges inside a
column, subnormals, zero and non-finite columns, values just below a
power of two (the largest digits), K up to the exactness bound 409, row
blocks and ragged column tiles.  The solver in FR_FP64S is held to the
FP64 path's tolerance against the oracle: 1e-12 relative per conserved
quantity on the RHS and on RK4 states, including the full boundary-layer
workload.
"""
import math

import numpy as np
import pytest

import synth
from tests._cases import bl_params, gpu_rhs, library, make_pair, per_quantity_rel_err, per_var_rel_err, state, \
    to_longdouble

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    library()


def _fr():
    from paper_1409_0405_gb300 import fr
    return fr


def _two_prod(a, b):
    """(p, e) with p + e == a b exactly (Dekker / Veltkamp, no FMA), for
    products well inside the normal range."""
    c = 134217729.0
    p = a * b
    t = c * a
    ah = t - (t - a)
    al = a - ah
    t = c * b
    bh = t - (t - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_matmul(A, B):
    """A B with every output the correctly rounded exact sum."""
    M, K = A.shape
    N = B.shape[1]
    p, e = _two_prod(A[:, :, None], B[None, :, :])
    out = np.empty((M, N))
    for i in range(M):
        terms = np.concatenate([p[i], e[i]], axis=0)  # (2K, N)
        for n in range(N):
            out[i, n] = math.fsum(terms[:, n])
    return out


def _adversarial_B(K, N, rng):
    B = rng.standard_normal((K, N))
    # wide exponent range within a column
    B[:, 0::7] *= 10.0 ** rng.uniform(-12, 12, size=(K, len(range(0, N, 7))))
    # values just below a power of two (the largest digits), both signs
    B[:, 1::7] = np.where(rng.random((K, len(range(1, N, 7)))) < 0.5, -1.0, 1.0) * np.nextafter(2.0, 0.0)
    # one large value over tiny ones
    B[:, 2::7] = 1e-9 * rng.standard_normal((K, len(range(2, N, 7))))
    B[0, 2::7] = 3.0e4
    # exact powers of two and small integers
    B[:, 3::7] = np.ldexp(1.0, rng.integers(-30, 30, size=(K, len(range(3, N, 7)))))
    B[:, 4::7] = rng.integers(-1000, 1000, size=(K, len(range(4, N, 7)))).astype(float)
    # zero column
    if N > 5:
        B[:, 5] = 0.0
    return B


def _run(A, B):
    import torch
    Bt = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Ct = torch.full((A.shape[0], B.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    _fr().gemm_fp64s(A, Bt.data_ptr(), Ct.data_ptr(), B.shape[1], torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return Ct.cpu().numpy()


def _check_products(A, B, got):
    ref = exact_matmul(A, B)
    K = A.shape[1]
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    bound = K * 2.0 ** -52 * scale + 2.0 ** -52 * np.abs(ref) + 1e-300
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    worst = np.max(err / (K * scale + 1e-300))
    assert np.all(err <= bound), worst
    return worst


@pytest.mark.parametrize("M,K,N", [(60, 35, 1000), (105, 95, 386), (35, 165, 130), (7, 409, 256), (3, 1, 2),
                                   (64, 16, 128), (65, 17, 258)])
def test_gemm_fp64s_matches_exact_products(M, K, N):
    rng = np.random.default_rng(M * 1000 + K)
    A = rng.standard_normal((M, K))
    A[:, ::3] *= 10.0 ** rng.uniform(-6, 6, size=(M, len(range(0, K, 3))))
    if M > 2:
        A[1] = 0.0                           # a zero operator row
        A[2, :] = np.nextafter(-4.0, 0.0)    # the largest digits, negative
    B = _adversarial_B(K, N, rng)
    worst = _check_products(A, B, _run(A, B))
    print(f"M={M} K={K} N={N}: max |err| / (K max|A| max|B|) = {worst:.2e}")


def test_gemm_fp64s_subnormals_and_nonfinite_columns():
    rng = np.random.default_rng(7)
    M, K, N = 20, 35, 64
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    B[:, 10] = 1e-310 * rng.standard_normal(K)      # subnormal column
    B[:, 11] = 5e-324                                # the smallest subnormal
    B[3, 12] = np.nan
    B[4, 13] = np.inf
    got = _run(A, B)
    assert np.all(np.isnan(got[:, 12])) and np.all(np.isnan(got[:, 13]))
    keep = [n for n in range(N) if n not in (12, 13)]
    ref = exact_matmul(A, B[:, keep])
    err = np.abs(got[:, keep] - ref)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B[:, keep]), axis=0)[None, :]
    # the reference's own products underflow here: K half-units of 5e-324
    assert np.all(err <= K * 2.0 ** -52 * scale + 2.0 ** -52 * np.abs(ref) + K * 5e-324)


def test_gemm_fp64s_is_deterministic():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 35))
    B = rng.standard_normal((35, 4000))
    np.testing.assert_array_equal(_run(A, B), _run(A, B))


def test_gemm_fp64s_rejects_bad_arguments():
    fr = _fr()
    import torch
    B = torch.zeros((410, 4), dtype=torch.float64, device="cuda")
    C = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FRError) as ei:
        fr.gemm_fp64s(np.ones((2, 410)), B.data_ptr(), C.data_ptr(), 4)
    assert ei.value.code == fr.FR_ERR_ARG
    with pytest.raises(fr.FRError) as ei:
        fr.gemm_fp64s(np.ones((2, 4)), B.data_ptr(), C.data_ptr(), 3)   # odd N
    assert ei.value.code == fr.FR_ERR_ARG
    A = np.ones((2, 4))
    A[0, 0] = np.nan
    with pytest.raises(fr.FRError) as ei:
        fr.gemm_fp64s(A, B.data_ptr(), C.data_ptr(), 4)
    assert ei.value.code == fr.FR_ERR_ARG


# ---------------------------------------------------------------------------
# the solver in FR_FP64S against the oracle (the FP64 path's tolerance)
# ---------------------------------------------------------------------------
def _pair(mesh, p, **kw):
    return make_pair(mesh, p, precision=_fr().FR_FP64S, **kw)


def _check_rhs(sol, ctx, u, tol=TOL):
    ref = sol.rhs(u)
    got = gpu_rhs(ctx, u)
    err = per_quantity_rel_err(sol, ref, got)
    assert np.all(err <= tol), (err, per_var_rel_err(sol, ref, got))
    return err


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("viscous", [False, True])
def test_fp64s_rhs_all_orders_periodic(p, viscous):
    sol, ctx = _pair(synth.vortex_box(), p, viscous=viscous, mu=0.05)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=p))


@pytest.mark.parametrize("p", [2, 4])
def test_fp64s_rhs_wall_and_farfield_ns(p):
    m = synth.boundary_layer_box(nx=7, nz=3, n_prism_layers=5, n_tet_layers=3)
    sol, ctx = _pair(m, p, **bl_params(mu=0.01))
    _check_rhs(sol, ctx, state(sol, "bl"))


@pytest.mark.parametrize("n,npl", [(5, 2), (6, 0), (3, 3), (7, 3)])
def test_fp64s_rhs_ragged_and_single_type(n, npl):
    m = synth.vortex_box(n=n, n_prism_layers=npl)
    sol, ctx = _pair(m, 3, viscous=True, mu=0.02)
    _check_rhs(sol, ctx, state(sol, "smooth", seed=n))


def test_fp64s_rhs_impulsive_start_within_fp64_floor():
    """The wall case whose FP64 evaluations carry conditioning-amplified
    rounding: within 8x the FP64 oracle's distance from an extended-precision
    evaluation (and 1e-11), as the FP64 path."""
    m = synth.boundary_layer_box(nx=7, nz=3, n_prism_layers=5, n_tet_layers=3)
    sol, ctx = _pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "impulsive")
    r64 = sol.rhs(u)
    rld = to_longdouble(make_pair(m, 3, **bl_params(mu=0.01))[0]).rhs(
        u.astype(np.longdouble)).astype(np.float64)
    got = gpu_rhs(ctx, u)
    floor = per_var_rel_err(sol, rld, r64)
    err = per_var_rel_err(sol, rld, got)
    assert np.all(err <= np.maximum(8.0 * floor, TOL)), (err, floor)
    assert np.all(err <= 1e-11), err


def test_fp64s_vortex_rk4_100_steps():
    sol, ctx = _pair(synth.vortex_box(), 2)
    u = state(sol, "vortex")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 100)
    ref = u
    for _ in range(100):
        ref = sol.rk4_step(ref, dt)
    err = per_quantity_rel_err(sol, ref, ctx.get_state())
    assert np.all(err <= TOL), err
    np.testing.assert_allclose(ctx.reduce()[:5], sol.integrals(u), rtol=1e-12, atol=1e-9)


def test_fp64s_ns_rk4_and_rk45_steps():
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = _pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    dt = 0.2 * sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 3)
    ref = u
    for _ in range(3):
        ref = sol.rk4_step(ref, dt)
    assert np.all(per_quantity_rel_err(sol, ref, ctx.get_state()) <= TOL)
    ctx.set_state(u)
    ctx.step_rk45(dt, 3)
    ref = u
    for _ in range(3):
        ref = sol.rk45_step(ref, dt)[0]
    assert np.all(per_quantity_rel_err(sol, ref, ctx.get_state()) <= TOL)


def test_fp64s_close_to_fp64_and_deterministic():
    """FR_FP64S and FR_FP64 RHS agree far below the parity tolerance; two
    FR_FP64S evaluations are bitwise equal."""
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = _pair(m, 4, **bl_params(mu=0.01))
    _, c64 = make_pair(m, 4, **bl_params(mu=0.01))
    u = state(sol, "bl")
    a = gpu_rhs(ctx, u)
    b = gpu_rhs(c64, u)
    np.testing.assert_array_equal(a, gpu_rhs(ctx, u))
    err = per_quantity_rel_err(sol, b, a)
    print("FP64S vs FP64 RHS:", err)
    assert np.all(err <= 2e-13), err


def test_fp64s_partitioned_is_bitwise():
    """Partitions of an FR_FP64S mesh give the single-context RHS bit for
    bit (every output column is computed independently)."""
    fr = _fr()
    m = synth.boundary_layer_box(nx=6, nz=3, n_prism_layers=4, n_tet_layers=3)
    sol, ctx = _pair(m, 3, **bl_params(mu=0.01))
    u = state(sol, "bl")
    ctx.set_state(u)
    ctx.step(1e-4, 2)
    one = ctx.get_state()
    part = fr.PartContext(m, 3, 2, precision=fr.FR_FP64S, **bl_params(mu=0.01))
    part.set_state(u)
    part.step(1e-4, 2)
    np.testing.assert_array_equal(part.get_state(), one)


def test_fp64s_bounded_wait_timeout_is_reported():
    fr = _fr()
    sol, ctx = _pair(synth.vortex_box(), 2)
    ctx.selftest_wait_timeout()
    # the context stays usable
    u = state(sol, "vortex")
    _check_rhs(sol, ctx, u)


def test_fp64s_full_size_boundary_layer_rhs():
    """The full boundary-layer workload (57,600 prisms + 118,800 tets, p = 4,
    Navier-Stokes): every output of one RHS."""
    m = synth.boundary_layer_box()
    sol, ctx = _pair(m, 4, **bl_params())
    err = _check_rhs(sol, ctx, state(sol, "bl"))
    print("FP64S full-size RHS:", err)


def test_fp64s_full_size_boundary_layer_rk4_step():
    m = synth.boundary_layer_box()
    sol, ctx = _pair(m, 4, **bl_params())
    u = state(sol, "bl")
    dt = sol.dt_cfl(u, 0.1)
    ctx.set_state(u)
    ctx.step(dt, 1)
    got = ctx.get_state()
    ref = sol.rk4_step(u, dt)
    err = per_quantity_rel_err(sol, ref, got)
    inc = per_quantity_rel_err(sol, ref - u, got - u)
    print("FP64S full-size RK4 step: state", err, "increment", inc)
    assert np.all(err <= TOL), err
    assert np.all(inc <= TOL), inc
