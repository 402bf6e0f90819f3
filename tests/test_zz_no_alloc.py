"""The allocation-free reduction entry point, fr_reduce_noalloc.

Some callers cannot call cudaMalloc (a device owned by another allocator,
or a path where an allocation is not allowed); this entry point keeps its
scratch in a static device array instead.  The tests call it through the C
ABI on device buffers:

* against the existing context-based fr_reduce on two calls in a row, the
  second over a third of the elements of the first, so that partial sums
  left in the shared array by the larger first call would change the
  second result if the final pass read more slots than the call wrote;
* on a state with a few planted non-physical points (negative density,
  NaN), whose count must match fr_reduce's;
* with an oversized request, which must be rejected before any GPU work.

It lives in a file of its own, collected last, and passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

import synth
from tests._cases import library, make_pair, state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    library()


def _tet_case(n):
    mesh = synth.vortex_box(n=n, n_prism_layers=0)          # one element block (tets)
    sol, ctx = make_pair(mesh, 3, viscous=True, mu=0.01)
    wJ = np.ascontiguousarray(sol.m.ops["tet"].w[None, :] * sol.m.J["tet"])
    return sol, ctx, wJ


def _noalloc(ne, nu, u, wJ):
    import torch
    from paper_1409_0405_gb300 import fr
    ud = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    wd = torch.from_numpy(np.ascontiguousarray(wJ)).cuda()
    out = torch.full((7,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fr.reduce_noalloc(ne, nu, ud.data_ptr(), wd.data_ptr(), 1.4, out.data_ptr(), stream)
    assert rc == fr.FR_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_reduce_noalloc_matches_fr_reduce_twice():
    sol, ctx, wJ = _tet_case(8)                               # 3,072 tets x 20 points: 30 blocks
    ne, nu = ctx.info["n_tet"], ctx.info["nu_tet"]
    u = state(sol, "vortex")
    ctx.set_state(u)
    got = _noalloc(ne, nu, u, wJ)
    ref = ctx.reduce()                                         # existing entry point
    np.testing.assert_allclose(got[:6], ref[:6], rtol=1e-12, atol=1e-12)
    assert got[6] == ref[6] == 0.0

    # second call: another state on the first third of the elements (10
    # blocks), checked against the plain sums of the definition
    ns = ne // 3
    u2 = state(sol, "smooth", seed=3).reshape(ne, 5, nu)[:ns]
    got2 = _noalloc(ns, nu, u2, wJ[:ns])
    direct = np.einsum("ej,evj->v", wJ[:ns], u2)
    ke = np.sum(wJ[:ns] * 0.5 * np.sum(u2[:, 1:4] ** 2, axis=1) / u2[:, 0])
    np.testing.assert_allclose(got2[:5], direct, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(got2[5], ke, rtol=1e-12)
    assert got2[6] == 0.0


def test_reduce_noalloc_counts_nonphysical_points():
    sol, ctx, wJ = _tet_case(5)
    ne, nu = ctx.info["n_tet"], ctx.info["nu_tet"]
    u = state(sol, "vortex").reshape(ne, 5, nu).copy()
    u[3, 0, 2] = -0.5                                          # negative density
    u[40, 4, 7] = np.nan                                       # non-finite energy
    u[41, 1, 0] = np.inf                                       # non-finite momentum
    ctx.set_state(u.reshape(-1))
    ref = ctx.reduce(check=False)
    got = _noalloc(ne, nu, u, wJ)
    assert got[6] == 3.0
    assert ref[6] == got[6]


def test_reduce_noalloc_rejects_oversized_input():
    import torch
    from paper_1409_0405_gb300 import fr
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    too_many = (4096 * 2048) // 4 + 1                          # ne * nu > the maximum for nu = 4
    rc = fr.reduce_noalloc(too_many, 4, buf.data_ptr(), buf.data_ptr(), 1.4, buf.data_ptr())
    assert rc == fr.FR_ERR_ARG
    # ne near 2^63 / nu: ne * nu would overflow int64
    rc = fr.reduce_noalloc((1 << 62) + 1, 4, buf.data_ptr(), buf.data_ptr(), 1.4, buf.data_ptr())
    assert rc == fr.FR_ERR_ARG
    torch.cuda.synchronize()
    assert torch.all(buf == 0)
