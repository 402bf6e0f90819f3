"""The C ABI on the CPU: the library builds and loads, exports every entry
point include/fr.h declares, its host-built operators agree with the
oracle's exact ones (two independent constructions), and mesh validation
rejects bad meshes before any device work.  No GPU is needed."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import basis
from tests._cases import library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = library()
    from paper_1409_0405_gb300 import fr
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fr.EXPORTS) == names


def test_strerror():
    lib = library()
    assert lib.fr_strerror(0) == b"success"
    assert b"mesh" in lib.fr_strerror(-2)


@pytest.mark.parametrize("etype", ["tet", "pri", "hex"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_host_operators_match_oracle(etype, p):
    library()
    from paper_1409_0405_gb300 import fr
    op = basis.operators(etype, p)
    np.testing.assert_allclose(fr.operator(etype, p, "UPTS"), op.upts, atol=1e-14)
    np.testing.assert_allclose(fr.operator(etype, p, "FPTS"), op.fpts, atol=1e-14)
    np.testing.assert_allclose(fr.operator(etype, p, "M0"), op.M0, atol=1e-13)
    D = np.stack([op.D[d] for d in range(3)], 1).reshape(-1, op.nu)
    np.testing.assert_allclose(fr.operator(etype, p, "D"), D, atol=1e-12)
    np.testing.assert_allclose(fr.operator(etype, p, "M3"), op.M3, atol=1e-12 * np.abs(op.M3).max())
    np.testing.assert_allclose(fr.operator(etype, p, "W")[:, 0], op.w, atol=1e-14)
    np.testing.assert_allclose(fr.operator(etype, p, "FNORM"), op.fnorm, atol=1e-15)
    np.testing.assert_allclose(fr.operator(etype, p, "FW")[:, 0], op.fw, atol=1e-14)
    # the fused operators are the documented combinations
    AG = fr.operator(etype, p, "AGRAD")
    nu, nf = op.nu, op.nf
    for d in range(3):
        np.testing.assert_allclose(AG[d::3, :nu], op.D[d], atol=1e-12)
        np.testing.assert_allclose(AG[d::3, nu:], op.fnorm[:, d] * op.M3, atol=1e-11)
    AD = fr.operator(etype, p, "ADIV")
    np.testing.assert_allclose(AD[:, 3 * nu:], op.M3, atol=1e-11)
    for d in range(3):
        M132 = op.D[d] - op.M3 @ (op.fnorm[:, d:d + 1] * op.M0)
        np.testing.assert_allclose(AD[:, d:3 * nu:3], M132, atol=1e-11)


def test_operator_bad_arguments():
    lib = library()
    import ctypes as C
    r, c = C.c_int64(), C.c_int64()
    assert lib.fr_operator(3, 2, 0, None, C.byref(r), C.byref(c)) == -1
    assert lib.fr_operator(0, 5, 0, None, C.byref(r), C.byref(c)) == -1
    assert lib.fr_operator(0, 2, 99, None, C.byref(r), C.byref(c)) == -1


def _create_rc(mesh, p=2, **kw):
    from paper_1409_0405_gb300 import fr
    try:
        fr.Context(mesh, p, **kw)
    except fr.FRError as e:
        return e.code
    return 0


def test_mesh_errors_detected_on_host():
    library()
    from paper_1409_0405_gb300 import fr
    m = synth.vortex_box()
    bad = dict(m)
    bad["tet"] = m["tet"].copy()
    bad["tet"][0, [1, 2]] = bad["tet"][0, [2, 1]]           # inverted element
    assert _create_rc(bad) == fr.FR_ERR_MESH
    nop = dict(m)
    nop["period"] = np.zeros(3)                              # free faces, no period
    assert _create_rc(nop) == fr.FR_ERR_MESH
    oob = dict(m)
    oob["pri"] = m["pri"].copy()
    oob["pri"][3, 0] = 10 ** 9                               # node id out of range
    assert _create_rc(oob) == fr.FR_ERR_MESH
    bf = synth.boundary_layer_box(nx=3, nz=2, n_prism_layers=2, n_tet_layers=2)
    bf["bface"] = bf["bface"].copy()
    bf["bface"][0, 3] = 7                                    # unknown tag
    assert _create_rc(bf) == fr.FR_ERR_MESH
    assert _create_rc(m, p=0) == fr.FR_ERR_ARG
    assert _create_rc(m, p=2, precision=7) == fr.FR_ERR_UNSUPPORTED


def test_hex_and_curved_mesh_errors_detected_on_host():
    """Hexahedra and curved meshes: an inverted hex, a stray hex whose faces
    match no neighbour or periodic partner, an unsupported geometry order,
    a curved mesh without the node array of a present type, and a curved
    element folded flat are rejected on the host (FR_ERR_MESH)."""
    library()
    from paper_1409_0405_gb300 import fr
    h = synth.hex_box(n=3, n_hex_cols=2)
    inv = dict(h)
    inv["hex"] = h["hex"].copy()
    inv["hex"][0] = inv["hex"][0][[4, 5, 6, 7, 0, 1, 2, 3]]   # top and bottom swapped
    assert _create_rc(inv) == fr.FR_ERR_MESH
    mix = dict(synth.vortex_box(n=2))
    mix["hex"] = np.asarray(h["hex"][:1])                     # a stray hex: faces match nothing
    mix["xyz"] = np.concatenate([mix["xyz"], h["xyz"]])
    mix["hex"] = mix["hex"] + len(synth.vortex_box(n=2)["xyz"])
    assert _create_rc(mix) == fr.FR_ERR_MESH
    c = synth.curve_mesh(synth.vortex_box(), amp=0.1)
    g3 = dict(c)
    g3["geom_order"] = 3
    assert _create_rc(g3) == fr.FR_ERR_MESH
    nop = dict(c)
    del nop["tet_nodes"]
    assert _create_rc(nop) == fr.FR_ERR_MESH
    fold = dict(c)
    fold["pri_nodes"] = c["pri_nodes"].copy()
    fold["pri_nodes"][0, 12:18] = fold["pri_nodes"][0, 0:6]   # top level onto the bottom one
    assert _create_rc(fold) == fr.FR_ERR_MESH


def test_binding_checks_curved_node_shapes():
    """The binding validates the quadratic node arrays' shapes before any
    pointer reaches the library."""
    library()
    from paper_1409_0405_gb300 import fr
    c = synth.curve_mesh(synth.vortex_box(), amp=0.1)
    bad = dict(c)
    bad["pri_nodes"] = c["pri_nodes"][:, :17]
    with pytest.raises(ValueError):
        fr.Context(bad, 2)
    short = dict(c)
    short["tet_nodes"] = c["tet_nodes"][:-1]
    with pytest.raises(ValueError):
        fr.Context(short, 2)


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    library()
    from paper_1409_0405_gb300 import fr
    assert _create_rc(synth.vortex_box()) == fr.FR_ERR_CUDA


def test_entry_points_reject_bad_arguments_without_a_gpu():
    """Argument checks of the later entry points run before any device
    work: null contexts and pointers, bad element types, orders, sizes and
    steps return FR_ERR_ARG (no GPU touched)."""
    library()
    import ctypes as C
    from paper_1409_0405_gb300 import fr
    lib = fr.load()
    assert lib.fr_step_ls(None, 1e-3, 1, None) == fr.FR_ERR_ARG
    assert lib.fr_step(None, 1e-3, 1, None) == fr.FR_ERR_ARG
    assert lib.fr_diagnostics(None, None, None) == fr.FR_ERR_ARG
    assert lib.fr_selftest_wait_timeout(None, None) == fr.FR_ERR_ARG
    assert lib.fr_closure_set(None, 0, None, 128, None) == fr.FR_ERR_ARG
    assert lib.fr_closure_features(None, None, 0, None, None) == fr.FR_ERR_ARG
    assert lib.fr_closure_sample(None, None, None, None, 0, None, None, None, None, None) == fr.FR_ERR_ARG
    assert lib.fr_transfer_state(None, None, None, None, None) == fr.FR_ERR_ARG
    rows, cols = C.c_int64(), C.c_int64()
    assert lib.fr_transfer(0, 2, 5, None, C.byref(rows), C.byref(cols)) == fr.FR_ERR_ARG
    assert lib.fr_transfer(3, 2, 4, None, C.byref(rows), C.byref(cols)) == fr.FR_ERR_ARG
    assert lib.fr_transfer(-1, 2, 4, None, C.byref(rows), C.byref(cols)) == fr.FR_ERR_ARG
    assert lib.fr_mlp_forward(4, 0, 4, 10, None, None, None, None, None) == fr.FR_ERR_ARG
    assert lib.fr_mlp_grad(4, 8, 4, 0, None, None, None, None, None, None, None) == fr.FR_ERR_ARG
    assert lib.fr_mlp_adam(10, None, None, None, None, 1, 1e-3, None) == fr.FR_ERR_ARG
    assert lib.fr_mlp_nparams(0, 8, 4) == 0 and lib.fr_mlp_workspace(4, 8, 4, 0) == 0
    assert lib.fr_reduce_noalloc(0, 10, None, None, 1.4, None, None) == fr.FR_ERR_ARG
    assert lib.fr_batch_step(None, None, 1, 1, None) == fr.FR_ERR_ARG


def test_tensor_core_precisions_are_accepted_on_the_host():
    """FR_BF16X3, FR_TF32X3 and FR_FP64S pass the host checks (the failure
    without a GPU is the device, not the precision); FR_FP64S + 1 and -1 do
    not."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    library()
    from paper_1409_0405_gb300 import fr
    m = synth.vortex_box()
    assert _create_rc(m, p=2, precision=fr.FR_BF16X3) == fr.FR_ERR_CUDA
    assert _create_rc(m, p=2, precision=fr.FR_TF32X3) == fr.FR_ERR_CUDA
    assert _create_rc(m, p=2, precision=fr.FR_FP64S) == fr.FR_ERR_CUDA
    assert _create_rc(m, p=2, precision=fr.FR_FP64S + 1) == fr.FR_ERR_UNSUPPORTED
    assert _create_rc(m, p=2, precision=-1) == fr.FR_ERR_UNSUPPORTED
