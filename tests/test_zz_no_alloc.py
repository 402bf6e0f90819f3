"""The allocation-free reduction entry point, fr_reduce_noalloc.

Some callers cannot call cudaMalloc (a device owned by another allocator,
or a path where an allocation is not allowed); this entry point keeps its
scratch in a static device array instead.  The test calls it through the C
ABI on device buffers and checks it against the existing context-based
fr_reduce on two calls in a row (different states, so stale scratch from
the first call would show up in the second), and checks that an oversized
request is rejected before any GPU work.  It lives in a file of its own,
collected last, and passes alone in a fresh process as well as after the
other tests.
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


def test_reduce_noalloc_matches_fr_reduce_twice():
    import torch
    from paper_1409_0405_gb300 import fr
    mesh = synth.vortex_box(n=5, n_prism_layers=0)          # one element block (tets)
    sol, ctx = make_pair(mesh, 3, viscous=True, mu=0.01)
    ne, nu = ctx.info["n_tet"], ctx.info["nu_tet"]
    wJ = torch.from_numpy(np.ascontiguousarray(sol.m.ops["tet"].w[None, :] * sol.m.J["tet"])).cuda()
    out = torch.full((7,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for kind, seed in (("vortex", 0), ("smooth", 3)):
        u = state(sol, kind, seed=seed)
        ctx.set_state(u)
        ref = ctx.reduce()                                     # existing entry point
        ud = torch.from_numpy(u).cuda()
        rc = fr.reduce_noalloc(ne, nu, ud.data_ptr(), wJ.data_ptr(), 1.4, out.data_ptr(), stream)
        assert rc == fr.FR_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:6], ref[:6], rtol=1e-12, atol=1e-12)
        assert got[6] == ref[6] == 0.0


def test_reduce_noalloc_rejects_oversized_input():
    import torch
    from paper_1409_0405_gb300 import fr
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    too_many = (4096 * 2048) // 4 + 1                          # ne * nu > the maximum for nu = 4
    rc = fr.reduce_noalloc(too_many, 4, buf.data_ptr(), buf.data_ptr(), 1.4, buf.data_ptr())
    assert rc == fr.FR_ERR_ARG
    assert torch.all(buf == 0)
