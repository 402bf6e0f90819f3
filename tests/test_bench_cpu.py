"""The bench's measurement arithmetic on CPU (no GPU): how it accounts the
exact-split kernel's tensor work, which launches it groups into the
dominant kernel of a step, the algorithmic bytes of the point-wise
kernels, and when it trusts a committed ncu traffic figure."""
import types

import pytest

import bench
from tests._cases import library


@pytest.fixture(scope="module", autouse=True)
def _lib():
    library()


def _ctx():
    """The full boundary-layer workload's counts (57,600 prisms + 118,800
    tets, p = 4), without a device."""
    c = types.SimpleNamespace(order=4)
    c.info = {"n_tet": 118800, "nu_tet": 35, "nf_tet": 60, "n_pri": 57600, "nu_pri": 75, "nf_pri": 105,
              "n_hex": 0, "nu_hex": 125, "nf_hex": 150, "npairs": 6_590_000}
    return c


def test_exact_split_layout_of_the_p4_operators():
    """Row blocks of at most 64 rows (whole points for the gradient), rows
    and each operand block's K padded to 16; the mostly-zero prism
    operators stay on the FMA kernel."""
    c = _ctx()
    assert bench.x64_layout(c, "M0", "tet") == (1, 64, 48)        # 60 x 35
    assert bench.x64_layout(c, "M0_grad", "tet") == (1, 64, 48)
    assert bench.x64_layout(c, "grad", "tet") == (2, 64, 112)     # 105 x (35 + 60): 2 x 54 rows
    assert bench.x64_layout(c, "div", "tet") == (1, 48, 176)      # 35 x (105 + 60)
    for k in bench.GEMM_CLASSES:
        assert bench.x64_layout(c, k, "pri") is None


def test_exact_split_tensor_flops():
    c = _ctx()
    cols = 5 * 118800
    tiles = -(-cols // 128) * 128
    assert bench.x64_tensor_flops(c, "grad", "tet") == 36 * 2 * tiles * 2 * 64 * 112
    assert bench.x64_tensor_flops(c, "M0_grad", "tet") == 36 * 2 * (-(-3 * cols // 128) * 128) * 64 * 48
    # the FP64-equivalent count is 2 x non-zeros x columns
    from paper_1409_0405_gb300 import fr
    import numpy as np
    nnz = np.count_nonzero(fr.operator(0, 4, "ADIV"))
    assert bench.gemm_flops_type(c, "div", "tet") == 2.0 * nnz * cols


def test_pointwise_bytes():
    c = _ctx()
    assert bench.pointwise_bytes_fp64(c, "flux", "tet") == 8.0 * 118800 * 35 * 44
    assert bench.pointwise_bytes_fp64(c, "common_flux") == 6_590_000 * (8.0 * 40 + 12)
    assert bench.pointwise_bytes_fp64(c, "M0", "tet") is None


def _fakes():
    fr = types.SimpleNamespace(FR_FP64=0, FR_FP64S=4, FR_FP32=1, FR_BF16X3=2, FR_TF32X3=3,
                               peak_fp64=lambda sp: 1057.0)
    from paper_1409_0405_gb300 import fr as real
    fr.operator = real.operator
    props = types.SimpleNamespace(multi_processor_count=152)
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(get_device_properties=lambda i: props))
    return fr, torch


def test_dominant_kernel_is_grouped_by_kernel_function(monkeypatch):
    """Per launch class the exact-split tet gradient is the longest, but
    the prism launches of the FMA kernel add up to more: the entry is the
    FMA kernel's, against the FP64 pipe, over all four of its classes."""
    fr, torch = _fakes()
    monkeypatch.setattr(bench, "dgemm_reference_tflops", lambda t: 1.10)
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6789.0, "bf16_tflops_sustained": 1732.2,
                                                          "sm_max_mhz": 2070.0})
    args = types.SimpleNamespace(steps=2, nx=75)
    ms = {("M0", "tet"): 1.0, ("grad", "tet"): 6.0, ("M0_grad", "tet"): 5.0, ("div", "tet"): 4.0,
          ("M0", "pri"): 2.0, ("grad", "pri"): 5.5, ("M0_grad", "pri"): 5.0, ("div", "pri"): 5.0,
          ("common_flux", "all"): 5.9, ("flux", "tet"): 3.0, ("flux", "pri"): 3.0}
    typed = {k: (v, 8) for k, v in ms.items()}
    c = _ctx()
    r = bench.step_roofline(fr, torch, c, fr.FR_FP64S, {}, typed, args, None, 0)
    assert r["bound"] == "alu" and r["kernel"].startswith("k_gemm FP64 FMA")
    assert r["launches"] == 32
    fl = sum(bench.gemm_flops_type(c, k, "pri") for k in bench.GEMM_CLASSES) * 4 * args.steps
    assert r["achieved"] == pytest.approx(fl / (17.5e-3) / 1e12)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07e9 / 1e12)
    # with the exact-split launches dominant, the entry is the tensor pipe's
    typed2 = dict(typed)
    typed2[("grad", "tet")] = (20.0, 8)
    r2 = bench.step_roofline(fr, torch, c, fr.FR_FP64S, {}, typed2, args, None, 0)
    assert r2["bound"] == "tensor" and r2["kernel"].startswith("k_gemm_x64")
    tf = sum(bench.x64_tensor_flops(c, k, "tet") for k in bench.GEMM_CLASSES) * 4 * args.steps
    assert r2["achieved"] == pytest.approx(tf / 30e-3 / 1e12)
    assert r2["peak"] == 1732.2


def test_traffic_is_read_only_while_the_kernel_source_matches():
    b, src = bench.profiled_traffic("grad", etype="pri")
    assert b == pytest.approx(2.382e9) and src.startswith("profiles/")
    b, src = bench.profiled_traffic("grad", bench.X64_PROFILE, "tet", bench.X64_SOURCES)
    assert b == pytest.approx(1.2149e9)
    # another source file set than the capture's: the figure is withheld
    b, src = bench.profiled_traffic("grad", etype="pri", names=("fr_api.cu",))
    assert b is None and "changed" in src
