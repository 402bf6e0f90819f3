#!/usr/bin/env python3
"""Throughput of the FR right-hand side on the boundary-layer workload.

Workload: compressible Navier-Stokes, p = 4, FP64 (the operator products
of the tetrahedra exact-split on the tensor cores, FR_FP64S; FP64 FMA
throughout and the reduced precisions are reported beside it), on a box
[0,20] x [0,20] x [0,pi] with 32 stretched prism layers (57,600 prisms) on
a no-slip wall under Kuhn tets (118,800 tets), Re = 3900, Ma = 0.2,
uniform inflow plus a 1% seeded velocity perturbation, with a tanh wall
profile of thickness 0.5 so that it satisfies no-slip: 42,390,000 DOF.
One step = one classic RK4 step = 4 RHS evaluations (the whole hot path:
interpolation, common solution, corrected gradients, fluxes, common
fluxes, divergence + correction, register update).

Metric: GDOF/s = DOF x RHS evaluations / second (whole job: with N ranks
each rank advances its own copy of the workload; weak scaling).

--impl reference times the CPU oracle (the plain FP64 numpy solver used as
the correctness reference) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ORDER = 4
GAMMA = 1.4
MACH = 0.2
REYNOLDS = 3900.0
METRIC = "FR RHS GDOF/s, mixed prism/tet p=4, FP64 vs FP32/split/learned; % roofline"
UNIT = "GDOF/s"
WORKLOAD = "boundary-layer box NS p=4 FP64: 57,600 prisms + 118,800 tets, Re=3900, Ma=0.2, RK4"
# a bounded sample of the same workload for the CPU oracle: the same
# generator with 15 instead of 75 cells along x (1/5 of the elements)
CPU_SAMPLE_NX = 15
# the inflow carries a tanh(y/0.5) wall profile so the initial state
# satisfies the no-slip condition
WALL_DELTA = 0.5


def flow_params():
    p_inf = 1.0 / (GAMMA * MACH ** 2)
    return dict(viscous=True, mu=1.0 / REYNOLDS, gamma=GAMMA, prandtl=0.72, ldg_beta=0.5,
                ldg_tau=0.1, rho_inf=1.0, vel_inf=(1.0, 0.0, 0.0), p_inf=p_inf, t_wall=p_inf)


def points_to_public(q, counts):
    """(n_points, 5) values in public point order -> public layout."""
    out, off = [], 0
    for ne, nu in counts:
        if ne == 0:
            continue
        blk = q[off:off + ne * nu].reshape(ne, nu, 5).transpose(0, 2, 1)
        out.append(blk.reshape(-1))
        off += ne * nu
    return np.concatenate(out)


def min_edge(mesh):
    xyz = mesh["xyz"]
    h = np.inf
    for key, pairs in (("tet", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
                       ("pri", [(0, 1), (1, 2), (2, 0), (0, 3), (1, 4), (2, 5)]),
                       ("hex", [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 5), (2, 6), (3, 7)])):
        c = mesh.get(key, ())
        if len(c) == 0:
            continue
        for a, b in pairs:
            h = min(h, float(np.min(np.linalg.norm(xyz[c[:, a]] - xyz[c[:, b]], axis=1))))
    return h


def time_step_size(mesh, order):
    """dt = 0.1 h_min / ((|v| + c) (p+1)^2), a conservative explicit limit."""
    c_inf = 1.0 / MACH
    return 0.1 * min_edge(mesh) / ((1.0 + c_inf) * (order + 1) ** 2)


_NNZ = {}


def _nnz(fr, etype, order, which):
    """Non-zero entries of one of the library's operators (its exact zeros,
    which the FP64 kernels skip, are no algorithmic work)."""
    key = (etype, order, which)
    if key not in _NNZ:
        _NNZ[key] = int(np.count_nonzero(fr.operator(etype, order, which)))
    return _NNZ[key]


def gemm_flops(ctx, kclass):
    """Algorithmic FP64 flops of one launch class, summed over the element
    types, for one RHS evaluation: 2 x (non-zero operator entries) x
    (5 variables x elements) per operator application (x3 columns for M0
    on the gradients)."""
    from paper_1409_0405_gb300 import fr
    i = ctx.info
    p = ctx.order
    tot = 0.0
    for et, name in enumerate(("tet", "pri", "hex")):
        ne = i["n_" + name]
        if ne == 0:
            continue
        cols = 5.0 * ne
        if kclass == "M0":
            tot += 2.0 * _nnz(fr, et, p, "M0") * cols
        elif kclass == "grad":
            tot += 2.0 * _nnz(fr, et, p, "AGRAD") * cols
        elif kclass == "M0_grad":
            tot += 2.0 * _nnz(fr, et, p, "M0") * 3 * cols
        elif kclass == "div":
            tot += 2.0 * _nnz(fr, et, p, "ADIV") * cols
    return tot


def gemm_bytes_f32(ctx, kclass):
    """Algorithmic DRAM bytes of one launch class (all element types) per
    RHS in the FP32-storage modes (4-byte state): operator input and output
    once, plus the epilogue's own reads and writes: the geometry S^T/J for
    the gradient (10 floats per point), and for the divergence with the
    fused RK update (an RK step's average stage) 1/J, the FP64 reference
    term, the FP64 registers read (12 B) and written (12 B incl. the float
    stage input)."""
    i = ctx.info
    tot = 0.0
    for ne, nu, nf in ((i["n_" + t], i["nu_" + t], i["nf_" + t]) for t in ("tet", "pri", "hex")):
        if ne == 0:
            continue
        cols = 5.0 * ne
        if kclass == "M0":
            tot += 4.0 * cols * (nu + nf)
        elif kclass == "grad":
            tot += 4.0 * cols * (nu + nf) + 4.0 * cols * 3 * nu + 4.0 * ne * nu * 10
        elif kclass == "M0_grad":
            tot += 4.0 * 3 * cols * (nu + nf)
        elif kclass == "div":
            tot += 4.0 * cols * (3 * nu + nf) + 4.0 * ne * nu + cols * nu * (8 + 12 + 12)
    return tot


_OPNAME = {"M0": "M0", "grad": "AGRAD", "M0_grad": "M0", "div": "ADIV"}
X64_DIGIT_PAIRS = 36     # digit pairs (levels 0..7) per 16-wide K step of the exact-split kernel
X64_MAX_ROWS = 64        # operator rows per row block (the MMA's N before padding)
X64_MAX_K = 409          # longest K whose level sums stay exact in FP32


def gemm_flops_type(ctx, kclass, etype):
    """gemm_flops for one element type: 2 x non-zero operator entries x
    columns (5 variables x elements; x3 for M0 on the gradients)."""
    from paper_1409_0405_gb300 import fr
    ne = ctx.info["n_" + etype]
    cols = 5.0 * ne * (3 if kclass == "M0_grad" else 1)
    return 2.0 * _nnz(fr, ("tet", "pri", "hex").index(etype), ctx.order, _OPNAME[kclass]) * cols


def x64_layout(ctx, kclass, etype):
    """How FR_FP64S applies one operator: None when the type keeps the FMA
    kernel (the library moves an operator to the exact-split tensor-core
    kernel when at least half of its entries are non-zero and K <= 409),
    else (row blocks, MMA N = rows padded to 16, K padded to 16 per
    operand block) by the library's row-block rule (blocks of at most 64
    rows, as even as possible, whole points of 3 rows for the gradient)."""
    from paper_1409_0405_gb300 import fr
    et = ("tet", "pri", "hex").index(etype)
    A = fr.operator(et, ctx.order, _OPNAME[kclass])
    M, K = A.shape
    if 2 * np.count_nonzero(A) < A.size or K > X64_MAX_K:
        return None
    nu, nf = ctx.info["nu_" + etype], ctx.info["nf_" + etype]
    k1, k2 = {"M0": (nu, 0), "grad": (nu, nf), "M0_grad": (nu, 0), "div": (3 * nu, nf)}[kclass]
    kpad = -(-k1 // 16) * 16 + -(-k2 // 16) * 16
    unit = 3 if kclass == "grad" else 1
    nrb = -(-M // X64_MAX_ROWS)
    rows = -(-M // nrb)
    rows = -(-rows // unit) * unit
    while rows > X64_MAX_ROWS:
        rows -= unit
    nrb = -(-M // rows)
    return nrb, -(-rows // 16) * 16, kpad


def x64_tensor_flops(ctx, kclass, etype):
    """BF16 tensor-core flops of one exact-split launch (one RHS): 36 digit
    pairs x 2 x (state columns padded to the 128-column tile) x (row blocks
    x MMA N) x padded K."""
    nrb, nmma, kpad = x64_layout(ctx, kclass, etype)
    ncols = 5 * ctx.info["n_" + etype] * (3 if kclass == "M0_grad" else 1)
    return X64_DIGIT_PAIRS * 2.0 * (-(-ncols // 128) * 128) * nrb * nmma * kpad


def pointwise_bytes_fp64(ctx, kclass, etype=None):
    """Algorithmic DRAM bytes of one FP64 point-wise launch (one RHS,
    Navier-Stokes): the transformed flux of one type reads the state (5),
    the physical gradient (15) and S (9), and writes F~ (15) doubles per
    point; the common flux
    reads both sides' flux-point states (10), the gradient of the side whose
    viscous flux the LDG flux takes (15: with beta = 1/2 the other side's
    weight is zero), the unit normal and both magnitudes (5), the pair word
    and both element numbers (12 B), and writes both sides' common flux (10)
    per interface pair; the
    common solution reads the states (10) and writes both jumps (10) with the
    pair's normal data."""
    i = ctx.info
    if kclass == "flux":
        pts = i["n_" + etype] * i["nu_" + etype]
        return 8.0 * pts * (5 + 15 + 9 + 15)
    if kclass == "common_flux":
        return i["npairs"] * (8.0 * (10 + 15 + 5 + 10) + 12)
    if kclass == "common_solution":
        return i["npairs"] * (8.0 * (10 + 5 + 10) + 12)
    return None


def kernel_source_sha256(names=("fr_gemm.cu", "fr_gemm_body.cuh")):
    """SHA-256 of the operator kernel's source files, concatenated."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1409_0405_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic(kclass, profile="k_gemm_fp64_boundary_layer_p4_nx15.md", etype=None,
                     names=("fr_gemm.cu", "fr_gemm_body.cuh")):
    """DRAM bytes per launch (dram__bytes_read + dram__bytes_write) of one
    operator class (of one element type when etype is given) at full size,
    as recorded in a committed ncu summary's `bench-traffic` lines (measured
    on a smaller case and scaled by the element count), or None when the
    kernel's source files (names) have changed since that capture (their
    SHA-256 no longer matches) or no line exists."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            txt = f.read()
    except OSError:
        return None, "no profile summary"
    sha = kernel_source_sha256(names)
    for m in re.finditer(r"bench-traffic: class=(\w+)(?: type=(\w+))? sha256=([0-9a-f]+) "
                         r"bytes_per_launch_full_size=([0-9.eE+]+)", txt):
        if m.group(1) != kclass or m.group(2) != etype:
            continue
        if m.group(3) != sha:
            return None, "kernel changed since the ncu capture"
        return float(m.group(4)), f"profiles/{profile}"
    return None, f"no capture for class {kclass}" + (f" ({etype})" if etype else "")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (runs in a child process with one BLAS thread)
# ---------------------------------------------------------------------------
def cpu_oracle_child(nrhs):
    import synth
    from oracle.solver import Solver
    mesh = synth.boundary_layer_box(nx=CPU_SAMPLE_NX)
    prm = flow_params()
    sol = Solver(mesh, ORDER, gamma=prm["gamma"], mu=prm["mu"], prandtl=prm["prandtl"],
                 viscous=True, ldg_beta=prm["ldg_beta"], ldg_tau=prm["ldg_tau"],
                 rho_inf=prm["rho_inf"], vel_inf=prm["vel_inf"], p_inf=prm["p_inf"],
                 t_wall=prm["t_wall"])
    u = sol.state_from_points(synth.perturbed_freestream(sol.upts_xyz_points(), seed=2,
                                                         wall_delta=WALL_DELTA))
    times = []
    for _ in range(nrhs):
        t0 = time.perf_counter()
        r = sol.rhs(u)
        times.append(time.perf_counter() - t0)
    assert np.all(np.isfinite(r))
    nt, npri = len(mesh["tet"]), len(mesh["pri"])
    print(json.dumps({"ndof": sol.ndof, "times": times, "n_tet": nt, "n_pri": npri}))


def run_cpu_oracle(nrhs):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-oracle-child", str(nrhs)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"cpu oracle failed: {r.stderr[-2000:]}")
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return res


def cpu_baseline_entry(nrhs=1):
    res = run_cpu_oracle(nrhs)
    t = statistics.median(res["times"])
    return {"value": res["ndof"] / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one NS p=4 RHS of the same generator at nx={CPU_SAMPLE_NX} "
                       f"({res['n_pri']} prisms + {res['n_tet']} tets, {res['ndof']} DOF), "
                       f"median of {nrhs}, setup excluded, 1 BLAS thread")}


def per_quantity_rel_err(ref, got, counts):
    """[mass, momentum (vector norm), energy]: max |got-ref| / max |ref|
    over all points, public layout."""
    num = np.zeros(3)
    den = np.zeros(3)
    off = 0
    for ne, nu in counts:
        if ne == 0:
            continue
        r = ref[off:off + ne * 5 * nu].reshape(ne, 5, nu)
        g = got[off:off + ne * 5 * nu].reshape(ne, 5, nu)
        for q, sl in enumerate((slice(0, 1), slice(1, 4), slice(4, 5))):
            num[q] = max(num[q], float(np.max(np.linalg.norm(g[:, sl] - r[:, sl], axis=1))))
            den[q] = max(den[q], float(np.max(np.linalg.norm(r[:, sl], axis=1))))
        off += ne * 5 * nu
    return (num / np.where(den > 0, den, 1.0)).tolist()


def precision_mode(fr, torch, mesh, counts, u0, dt, ctx64, precision, args, sp):
    """Time K RK4 steps in another precision mode and measure its error
    against the FP64 path (which matches the FP64 oracle to 1e-12)."""
    ctx = fr.Context(mesh, ORDER, **flow_params(), precision=precision)
    ctx.set_state(u0, sp)
    for _ in range(max(args.warmup, 0)):
        ctx.step(dt, 1, sp)
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step(dt, 1, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    classes, launches = ctx.profile_read()
    ctx.profile(False)
    # errors: one RHS, and the increment of one RK4 step, against FP64
    ud = torch.from_numpy(u0).cuda()
    r64, r32 = torch.empty_like(ud), torch.empty_like(ud)
    ctx64.rhs(ud.data_ptr(), r64.data_ptr(), sp)
    ctx.rhs(ud.data_ptr(), r32.data_ptr(), sp)
    torch.cuda.synchronize()
    rhs_err = per_quantity_rel_err(r64.cpu().numpy(), r32.cpu().numpy(), counts)
    ctx64.set_state(u0, sp)
    ctx64.step(dt, 1, sp)
    s64 = ctx64.get_state(stream=sp)
    ctx.set_state(u0, sp)
    ctx.step(dt, 1, sp)
    s32 = ctx.get_state(stream=sp)
    inc_err = per_quantity_rel_err(s64 - u0, s32 - u0, counts)
    # flow diagnostics of the initial state, against FP64
    ctx64.set_state(u0, sp)
    d64 = ctx64.diagnostics(sp)
    ctx.set_state(u0, sp)
    d32 = ctx.diagnostics(sp)
    diag_err = {"ke_rate": abs(d32[0] - d64[0]) / abs(d64[0]),
                "wall_force_inviscid": float(np.linalg.norm(d32[1] - d64[1]) / np.linalg.norm(d64[1])),
                "wall_force_viscous": float(np.linalg.norm(d32[2] - d64[2]) / np.linalg.norm(d64[2]))}
    out = {"value": ctx64.ndof * 4.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "kernel_ms_per_step": {k: v[0] / args.steps for k, v in classes.items()},
           "gpu_launches": int(launches),
           "rhs_rel_err_vs_fp64": rhs_err, "step_increment_rel_err_vs_fp64": inc_err,
           "diagnostics_rel_err_vs_fp64": diag_err,
           "error_measure": "[mass, momentum vector, energy] max|d|/max|ref|; the FP64 path matches the "
                            "FP64 oracle to 1e-12"}
    gemm = ("M0", "grad", "M0_grad", "div")
    dom = max(gemm, key=lambda k: classes[k][0])
    byts = gemm_bytes_f32(ctx, dom) * 4 * args.steps
    ach = byts / (classes[dom][0] * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    hbm = {"bound": "hbm", "kernel": ("k_gemm_tc" if precision in (fr.FR_BF16X3, fr.FR_TF32X3) else "k_gemm")
           + f" ({dom})", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "traffic": None, "launches": classes[dom][1],
           "avg_launch_ms": classes[dom][0] / max(classes[dom][1], 1),
           "bytes": "operator input + output once, epilogue geometry/registers (bench.gemm_bytes_f32)",
           "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    if precision == fr.FR_FP32:
        # the streamed FP32 operator kernel (register tiles on the FP32
        # pipe) does 2 x (non-zero operator entries) flops per 8 state bytes
        # moved: at these operators' sizes its bound is the FP32 FMA pipe
        # (128 FMA per clock per SM) as much as HBM; both fractions reported
        nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        clk = float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
        fp32_peak = nsm * 128 * 2 * clk
        # the divergence bucket also holds the streaming RK update: the
        # dominant operator class among the other three
        dom = max(("M0", "grad", "M0_grad"), key=lambda k: classes[k][0])
        fl = gemm_flops(ctx, dom) * 4 * args.steps / (classes[dom][0] * 1e-3)
        ach = gemm_bytes_f32(ctx, dom) * 4 * args.steps / (classes[dom][0] * 1e-3) / 1e9
        out["roofline"] = {"bound": "alu", "kernel": f"k_gemm_f32 ({dom})", "achieved": fl / 1e12,
                           "peak": fp32_peak / 1e12, "unit": "TFLOP/s", "frac": fl / fp32_peak,
                           "traffic": None, "launches": classes[dom][1],
                           "avg_launch_ms": classes[dom][0] / max(classes[dom][1], 1),
                           "flops": "2 x non-zero operator entries x columns (bench.gemm_flops)",
                           "peak_source": f"derived: {nsm} SMs x 128 FP32 FMA/clk x 2 flop x {clk / 1e9:.2f} GHz",
                           "hbm_frac": ach / peak}
    else:
        out["roofline"] = hbm
    ctx.close()
    return out


def state_error_study(fr, torch, nsteps, sp):
    """The boundary-layer workload at p = 3 and p = 4: nsteps RK4 steps in
    FP64 (FMA throughout), in FP64 with the exact-split tensor-core
    products and in each reduced-precision mode from the same initial
    state; the final state, its change over the run and the flow
    diagnostics (kinetic-energy rate, wall force) of the final state
    against FP64 (the FP64 path matches the FP64 oracle to 1e-12 per RHS
    and step; the oracle itself would need hours per run at this size)."""
    mesh = synth_mod().boundary_layer_box()
    res = {}
    for order in (3, 4):
        dt = time_step_size(mesh, order)
        runs = {}
        for name, prec in (("fp64", fr.FR_FP64), ("fp64s", fr.FR_FP64S), ("fp32", fr.FR_FP32),
                           ("bf16x3", fr.FR_BF16X3), ("tf32x3", fr.FR_TF32X3)):
            ctx = fr.Context(mesh, order, **flow_params(), precision=prec)
            counts = ctx.counts()
            u0 = points_to_public(synth_mod().perturbed_freestream(ctx.upts_points(), seed=2,
                                                                   wall_delta=WALL_DELTA), counts)
            ctx.set_state(u0, sp)
            t0 = time.perf_counter()
            ctx.step(dt, nsteps, sp)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            finite = ctx.reduce(stream=sp, check=False)[6] == 0.0
            runs[name] = (ctx.get_state(stream=sp), ctx.diagnostics(sp), wall, bool(finite))
            ctx.close()
        s64, d64, _, _ = runs["fp64"]
        ent = {"ndof": int(s64.size), "dt": dt, "steps": nsteps, "fp64_wall_s": runs["fp64"][2],
               "fp64_ke_rate": d64[0], "fp64_wall_force_inviscid": d64[1].tolist(),
               "fp64_wall_force_viscous": d64[2].tolist()}
        for name in ("fp64s", "fp32", "bf16x3", "tf32x3"):
            st, d, wall, finite = runs[name]
            ent[name] = {"state_rel_err": per_quantity_rel_err(s64, st, counts),
                         "change_rel_err": per_quantity_rel_err(s64 - u0, st - u0, counts),
                         "ke_rate_rel_err": abs(d[0] - d64[0]) / abs(d64[0]),
                         "wall_force_viscous_rel_err": float(np.linalg.norm(d[2] - d64[2]) / np.linalg.norm(d64[2])),
                         "wall_force_inviscid_rel_err": float(np.linalg.norm(d[1] - d64[1]) / np.linalg.norm(d64[1])),
                         "wall_s": wall, "finite": finite}
        res[f"p{order}"] = ent
    return res


def synth_mod():
    import synth
    return synth


def batch_mode(fr, torch, args, sp, nprob=64):
    """nprob (default 64) independent periodic isentropic-vortex problems (element counts
    log-uniform in [1k, 80k], prism:tet ratio uniform in [0, 1], order in
    {1..4}, seed 3), FP32 with FP64 RK registers, after autotuning: one
    persistent launch per RK stage replayed from a CUDA graph, against the
    grouped per-class launches and each problem's own launch sequence."""
    import synth
    t0 = time.perf_counter()
    meshes, orders = [], []
    for i in range(nprob):
        m, p = synth.batch_problem_mesh(i)
        meshes.append(m)
        orders.append(p)
    prm = dict(viscous=False, precision=fr.FR_FP32, vel_inf=(1.0, 1.0, 0.0), p_inf=1.0, rho_inf=1.0)
    b = fr.Batch(meshes, orders, **prm)
    dts = []
    for c, m, p in zip(b.problems, meshes, orders):
        q = synth.isentropic_vortex(c.upts_points())
        counts = c.counts()
        c.set_state(points_to_public(q, counts), sp)
        # |v| + c <= 1.6 + 1.2 for the vortex
        dts.append(0.1 * min_edge(m) / (2.8 * (p + 1) ** 2))
    setup_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    b.tune(sp)
    tune_s = time.perf_counter() - t1
    stream = torch.cuda.ExternalStream(sp)

    def timed(batched):
        b.step(dts, max(args.warmup, 1), batched=batched, stream=sp)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(dts, args.steps, batched=batched, stream=sp)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms_b = timed(True)          # one persistent launch per RK stage
    info = b.info()
    ms_g = timed(2)             # one grouped launch per operator class and point-wise pass
    info_g = b.info()
    ms_u = timed(False)         # each problem's own launches
    b.check(sp)                 # raises if a barrier wait of the stage kernel gave up
    finite = all(c.reduce(stream=sp, check=False)[6] == 0.0 for c in b.problems)
    # algorithmic bytes of one RK step (FP32 state, FP64 registers): operator
    # inputs and outputs with their epilogue traffic (gemm_bytes_f32), the
    # flux kernel's U, S and FT (29 floats per point), and per interface
    # pair both sides' u_f read and common flux written (20 floats) plus
    # its metadata (normal and magnitudes in float, six int indices, switch)
    byts = 0.0
    for c in b.problems:
        i = c.info
        pts = sum(i["n_" + t] * i["nu_" + t] for t in ("tet", "pri", "hex"))
        byts += gemm_bytes_f32(c, "M0") + gemm_bytes_f32(c, "div") + 4.0 * 29 * pts
        byts += i["npairs"] * (4.0 * 20 + 4.0 * 5 + 4.0 * 6 + 1)
    byts *= 4
    ach = byts / (ms_b * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    b.close()
    return {"value": info["ndof"] * 4.0 / (ms_b * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_b,
            "schedule": "one persistent cooperative launch per RK stage, CUDA graph",
            "launches_per_step": info["launches_batched"], "stage_grid": info["grid_stage"],
            "grouped_launches_ms_per_step": ms_g, "grouped_launches_per_step": info_g["launches_batched"],
            "per_problem_launches_ms_per_step": ms_u, "speedup_vs_per_problem": ms_u / ms_b,
            "speedup_vs_grouped": ms_g / ms_b,
            "per_problem_launches_per_step": info["launches_per_problem"],
            "roofline": {"bound": "hbm", "kernel": "k_stage (whole RK step)", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "traffic": None,
                         "bytes_per_step": byts,
                         "bytes": "staged pipeline minimum: operators in/out + epilogue registers, flux point "
                                  "data, face gathers and metadata (bench.batch_mode)",
                         "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "ndof": info["ndof"], "problems": nprob, "tuned": {k: info[k] for k in fr.Batch.INFO[4:12]},
            "setup_s": setup_s, "tune_s": tune_s, "state_finite": bool(finite),
            "workload": f"{nprob} periodic isentropic-vortex boxes, Euler, FP32 + FP64 RK, seeds 3/1000+i"}


def _time_steps(torch, step, args, sp):
    """CUDA-event time per call of step() (after warm-up), on stream sp."""
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / args.steps


def rk45_mode(fr, torch, mesh, u0, dt, args, sp, precision):
    """RK45[2R+] (the paper's stepper, Sec. 3.4: five stages in two
    registers plus the embedded error estimate) on the same FP64 workload,
    in the headline's FP64 form: GDOF/s counts its 5 RHS per step; the
    error norm of the last step's embedded estimate (atol = rtol = 1e-6) is
    reported beside it."""
    ctx = fr.Context(mesh, ORDER, **flow_params(), precision=precision)
    ctx.set_state(u0, sp)
    ctx.profile(True)
    ms = _time_steps(torch, lambda: ctx.step_rk45(dt, 1, sp), args, sp)
    classes, launches = ctx.profile_read()
    typed = ctx.profile_read_types()
    ctx.profile(False)
    nprof = args.steps + max(args.warmup, 0)
    roof = step_roofline(fr, torch, ctx, precision, classes, typed, args, sp, torch.cuda.current_device(),
                         nrhs=5 * nprof)
    err = ctx.rk45_error(1e-6, 1e-6, sp)
    ctx.check(sp)
    out = {"value": ctx.ndof * 5.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "rhs_per_step": 5,
           "kernel_ms_per_step": {k: v[0] / (args.steps + max(args.warmup, 0)) for k, v in classes.items()},
           "error_norm_last_step": err, "error_norm_tolerances": [1e-6, 1e-6], "roofline": roof,
           "workload": WORKLOAD.replace("RK4", "RK45[2R+]")}
    ctx.close()
    return out


def partitioned_mode(fr, torch, mesh, u0, dt, ms_single, args, sp, precision):
    """The FP64 workload (in the headline's FP64 form) split into 2 and 4 partitions on this GPU
    (weighted coordinate bisection, tet:pri = 1:2), exchanging cut-face
    flux-point states and gradients through device-local halo buffers every
    RHS: time per RK4 step against the single context, halo sizes, and
    bitwise equality of the states after the timed steps."""
    out = {}
    ref = None
    for n in (2, 4):
        t0 = time.perf_counter()
        pc = fr.PartContext(mesh, ORDER, n, **flow_params(), precision=precision)
        setup_s = time.perf_counter() - t0
        pc.set_state(u0, sp)
        ms = _time_steps(torch, lambda: pc.step(dt, 1, sp), args, sp)
        st = pc.get_state(sp)
        if ref is None:
            ref = st
        info = pc.info
        out[f"{n}_parts"] = {
            "value": pc.ndof * 4.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "overhead_vs_single": ms / ms_single - 1.0,
            "elements": {"tet": info[:, 0].tolist(), "pri": info[:, 1].tolist()},
            "halo_slots": info[:, 3].tolist(), "setup_s": setup_s,
            "state_equal_to_2_parts": bool(np.array_equal(st, ref)),
            "state_finite": bool(pc.reduce(sp)[6] == 0.0)}
        pc.close()
    out["note"] = ("partitions share one GPU (no inter-GPU link is timed); the states after warm-up + timed "
                   "steps of the 2- and 4-partition runs are compared bitwise")
    return out


def p3_modes(fr, torch, mesh, args, sp):
    """The precision study's throughput at p = 3 (the same mesh and flow):
    GDOF/s of an RK4 step in both FP64 forms and in each reduced precision."""
    out = {}
    dt = time_step_size(mesh, 3)
    u0 = None
    for name, prec in (("fp64s", fr.FR_FP64S), ("fp64", fr.FR_FP64), ("fp32", fr.FR_FP32),
                       ("bf16x3", fr.FR_BF16X3), ("tf32x3", fr.FR_TF32X3)):
        ctx = fr.Context(mesh, 3, **flow_params(), precision=prec)
        if u0 is None:
            u0 = points_to_public(synth_mod().perturbed_freestream(ctx.upts_points(), seed=2,
                                                                   wall_delta=WALL_DELTA), ctx.counts())
        ctx.set_state(u0, sp)
        ctx.profile(True)
        ms = _time_steps(torch, lambda: ctx.step(dt, 1, sp), args, sp)
        classes, _ = ctx.profile_read()
        typed = ctx.profile_read_types()
        ctx.profile(False)
        nprof = args.steps + max(args.warmup, 0)
        out[name] = {"value": ctx.ndof * 4.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
                     "ndof": ctx.ndof, "state_finite": bool(ctx.reduce(stream=sp, check=False)[6] == 0.0),
                     "roofline": step_roofline(fr, torch, ctx, prec, classes, typed, args, sp,
                                               torch.cuda.current_device(), nrhs=4 * nprof)}
        ctx.close()
    return out


# ---------------------------------------------------------------------------
# learned closure: Taylor-Green vortex, p=2 + per-element network vs p=4
TGV_CELLS = 24
TGV_MACH = 0.1
TGV_RE = 1600.0
TGV_SNAPSHOTS = 8        # training states along the p=4 run
TGV_STRIDE = 100         # RK4 steps between states
TGV_ITERS = 1000         # full-batch Adam steps per element type
TGV_POST_WINDOWS = 4     # strides after the training window (a posteriori)


def tgv_params(precision):
    return dict(viscous=True, mu=1.0 / TGV_RE, gamma=GAMMA, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1,
                rho_inf=1.0, vel_inf=(0.0, 0.0, 0.0), p_inf=1.0 / (GAMMA * TGV_MACH ** 2),
                precision=precision)


def dgemm_reference_tflops(torch, n=8192, reps=3, device="cuda"):
    """The paper's "reference peak" method (Sec. 4.1): the FP64 rate of a
    large library DGEMM (here cuBLAS through torch.matmul, n x n x n),
    timed with CUDA events after one warm-up call."""
    a = torch.rand(n, n, dtype=torch.float64, device=device)
    b = torch.rand(n, n, dtype=torch.float64, device=device)
    c = torch.matmul(a, b)
    if device != "cuda":
        import time as _t
        t0 = _t.perf_counter()
        for _ in range(reps):
            c = torch.matmul(a, b)
        sec = (_t.perf_counter() - t0) / reps
    else:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            c = torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / reps
    del a, b, c
    return 2.0 * n ** 3 / sec / 1e12


def max_over_ranks(x, world, device="cpu"):
    """The largest x over the ranks of the default process group (x itself
    for one rank): the step time every rank waited for."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gdofs(world, ndof, seconds_per_step, rhs_per_step=4):
    """Whole-job throughput: every rank advances its own copy of the
    workload (weak scaling, replicas), all in the same wall time."""
    return world * ndof * rhs_per_step / seconds_per_step / 1e9


def _tri_area(a, b, c):
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def min_volume_to_area(mesh):
    """min over elements of 3 V / A (V volume, A surface area; planar faces)."""
    x = mesh["xyz"]
    r = np.inf
    t = mesh["tet"]
    if len(t):
        a, b, c, d = (x[t[:, k]] for k in range(4))
        V = np.abs(np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a))) / 6.0
        A = _tri_area(a, b, c) + _tri_area(a, b, d) + _tri_area(a, c, d) + _tri_area(b, c, d)
        r = min(r, float(np.min(3.0 * V / A)))
    pr = mesh["pri"]
    if len(pr):
        v = [x[pr[:, k]] for k in range(6)]
        V = sum(np.abs(np.einsum("ij,ij->i", q[1] - q[0], np.cross(q[2] - q[0], q[3] - q[0]))) / 6.0
                for q in ((v[0], v[1], v[2], v[3]), (v[1], v[2], v[3], v[4]), (v[2], v[3], v[4], v[5])))
        A = _tri_area(v[0], v[1], v[2]) + _tri_area(v[3], v[4], v[5])
        for i, j in ((0, 1), (1, 2), (2, 0)):
            A = A + 0.5 * np.linalg.norm(np.cross(v[j + 3] - v[i], v[i + 3] - v[j]), axis=1)
        r = min(r, float(np.min(3.0 * V / A)))
    return r


HEX_NZ = 29  # 75 x 54 x 29 = 117,450 hexahedra (the paper's hex mesh: 118,070)


def hex_mode(fr, torch, args, sp):
    """The boundary-layer box meshed with hexahedra only (Table 2's third
    type; the paper's cylinder mesh is all-hex): the same 54 stretched and
    uniform layers and flow, 75 x 54 x 29 = 117,450 hexahedra, NS, p = 4,
    FP64, RK4."""
    import synth
    mesh = synth.boundary_layer_box(nx=75, nz=HEX_NZ, all_hex=True)
    ctx = fr.Context(mesh, ORDER, **flow_params())
    u0 = points_to_public(synth.perturbed_freestream(ctx.upts_points(), seed=2, wall_delta=WALL_DELTA),
                          ctx.counts())
    dt = time_step_size(mesh, ORDER)
    ctx.set_state(u0, sp)
    for _ in range(max(args.warmup, 0)):
        ctx.step(dt, 1, sp)
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step(dt, 1, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    classes, launches = ctx.profile_read()
    ctx.profile(False)
    finite = ctx.reduce(stream=sp, check=False)[6] == 0.0
    gemm = ("M0", "grad", "M0_grad", "div")
    gflops = sum(gemm_flops(ctx, k) for k in gemm) * 4 * args.steps
    gms = sum(classes[k][0] for k in gemm)
    dom = max(gemm, key=lambda k: classes[k][0])
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    fp64_peak = nsm * 2 * 2 * clk
    dom_ach = gemm_flops(ctx, dom) * 4 * args.steps / (classes[dom][0] * 1e-3)
    out = {"value": ctx.ndof * 4.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "workload": f"boundary-layer box, hexahedra only: {ctx.info['n_hex']} hexes, NS p=4 FP64, RK4",
           "ndof": ctx.ndof, "kernel_ms_per_step": {k: v[0] / args.steps for k, v in classes.items()},
           "gpu_launches": int(launches), "state_finite": bool(finite),
           "gemm_share": gms / sum(v[0] for v in classes.values()),
           "gemm_fp64_tflops": gflops / (gms * 1e-3) / 1e12,
           "roofline": {"bound": "alu", "kernel": f"k_gemm ({dom})", "achieved": dom_ach / 1e12,
                        "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": dom_ach / fp64_peak,
                        "traffic": None, "launches": classes[dom][1],
                        "peak_source": f"derived: {nsm} SMs x 2 FP64 FMA/clk x 2 flop x {clk / 1e9:.2f} GHz"}}
    ctx.close()
    # the same workload with the operator applications on the tensor cores
    # (split TF32; the p=4 hex gradient runs as two row blocks)
    ct = fr.Context(mesh, ORDER, **flow_params(), precision=fr.FR_TF32X3)
    ct.set_state(u0, sp)
    for _ in range(max(args.warmup, 0)):
        ct.step(dt, 1, sp)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ct.step(dt, 1, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1) / args.steps
    out["tf32x3"] = {"value": ct.ndof * 4.0 / (ms_t * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_t,
                     "state_finite": bool(ct.reduce(stream=sp, check=False)[6] == 0.0)}
    ct.close()
    return out


def learned_mode(fr, torch, args, sp):
    """The learned closure on the Taylor-Green vortex (Re 1600, Ma 0.1,
    periodic [0, 2 pi]^3 of 24^3 cells: 13,824 prisms + 41,472 tets).
    The plain p=4 solve (FP32 RHS, FP64 registers) and the plain p=2 solve
    from the projected initial state run side by side; states along the p=4
    run give training samples (P RHS_4(u_4) - RHS_2(P u_4), the p=4 RHS in
    FP64); one network per element type is trained on the GPU by the
    library's kernels; a second set on the trajectory-consistent target
    P RHS_4(u_4(t)) - RHS_2(u_2(t)), u_2 the plain p=2 solution at the same
    time.  Reported: the RHS error with and without each network on a
    later, held-out state; the kinetic-energy dissipation rate of p=2 with
    and without the networks against p=4, over the training window and over
    the window after it; the p=4 check's decision (the better network is
    kept only if it lowers the dissipation error after the training
    window); and the RHS throughput of each."""
    import synth
    from paper_1409_0405_gb300 import closure
    t_setup = time.perf_counter()
    mesh = synth.tgv_box(n=TGV_CELLS)
    c4 = fr.Context(mesh, 4, **tgv_params(fr.FR_FP64))
    c4f = fr.Context(mesh, 4, **tgv_params(fr.FR_FP32))
    c2 = fr.Context(mesh, 2, **tgv_params(fr.FR_FP64))
    counts4 = c4.counts()
    q = synth.taylor_green(c4.upts_points(), GAMMA, TGV_MACH)
    u0 = points_to_public(q, counts4)
    rho, vel = q[:, 0], q[:, 1:4] / q[:, :1]
    pres = (GAMMA - 1.0) * (q[:, 4] - 0.5 * rho * np.sum(vel ** 2, axis=1))
    lam = float(np.max(np.linalg.norm(vel, axis=1) + np.sqrt(GAMMA * pres / rho)))
    dt = 0.1 * min_volume_to_area(mesh) / lam
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.ExternalStream(sp)
    nwin = TGV_SNAPSHOTS + TGV_POST_WINDOWS

    # p=4 and p=2 side by side from the same (projected) initial state
    t0 = time.perf_counter()
    u4d = torch.from_numpy(u0).cuda()
    u2_0 = torch.empty(c2.ndof, dtype=torch.float64, device="cuda")
    c2.transfer_from(c4, u4d.data_ptr(), u2_0.data_ptr(), sp)
    torch.cuda.synchronize()
    u2_0h = u2_0.cpu().numpy()
    c4f.set_state(u0, sp)
    c2.set_state(u2_0h, sp)
    S4, S2, ke4, ke2 = [], [], [], []
    for k in range(nwin):
        S4.append(torch.from_numpy(c4f.get_state(stream=sp)).cuda())
        S2.append(torch.from_numpy(c2.get_state(stream=sp)).cuda())
        ke4.append(c4f.reduce(stream=sp)[5])
        ke2.append(c2.reduce(stream=sp)[5])
        if k + 1 < nwin:
            c4f.step(dt, TGV_STRIDE, sp)
            c2.step(dt, TGV_STRIDE, sp)
    torch.cuda.synchronize()
    traj_s = time.perf_counter() - t0

    # training (samples, scales, Adam) on the GPU; the last state is held out
    t0 = time.perf_counter()
    cl = closure.Closure(c2, seed=0)
    log = cl.fit(c4, S4[:TGV_SNAPSHOTS], iters=TGV_ITERS, lr=1e-3, log_every=TGV_ITERS // 4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    prior = cl.error(c4, [S4[-1]])

    # a posteriori: p=2 with the network from the same initial state
    def a_posteriori(net):
        """KE along p=2 with the network; NaN after a blown-up step (the
        library reports it; set_state clears the condition)."""
        net.attach()
        c2.set_state(u2_0h, sp)
        ke = []
        for k in range(nwin):
            ke.append(c2.reduce(stream=sp, check=False)[5])
            if k + 1 < nwin:
                try:
                    c2.step(dt, TGV_STRIDE, sp)
                except fr.FRError:
                    ke += [float("nan")] * (nwin - 1 - k)
                    break
        net.detach()
        c2.set_state(u2_0h, sp)
        return ke

    ke2c = a_posteriori(cl)
    # the trajectory-consistent target: features and low-order RHS of the
    # plain p=2 solution at the same time as each p=4 state
    t0 = time.perf_counter()
    cl_t = closure.Closure(c2, seed=0)
    log_t = cl_t.fit(c4, list(zip(S4[:TGV_SNAPSHOTS], S2[:TGV_SNAPSHOTS])), iters=TGV_ITERS, lr=1e-3,
                     log_every=TGV_ITERS // 4)
    torch.cuda.synchronize()
    train_t_s = time.perf_counter() - t0
    prior_t = cl_t.error(c4, [(S4[-1], S2[-1])])
    ke2t = a_posteriori(cl_t)

    def rates(ke):
        ke = np.asarray(ke)
        return -(ke[1:] - ke[:-1]) / (TGV_STRIDE * dt)

    e4, e2, e2c, e2t = rates(ke4), rates(ke2), rates(ke2c), rates(ke2t)
    tr = slice(0, TGV_SNAPSHOTS - 1)
    post = slice(TGV_SNAPSHOTS - 1, nwin - 1)

    def rel(a, w):
        """mean relative dissipation error over the windows (None after a
        blown-up run)"""
        v = float(np.mean(np.abs(a[w] - e4[w]) / np.abs(e4[w])))
        return v if np.isfinite(v) else None

    def key(v):
        return float("inf") if v is None else v

    # the p=4 check: the better of the two networks after the training
    # window, kept only if it beats plain p=2 there
    best = cl if key(rel(e2c, post)) <= key(rel(e2t, post)) else cl_t
    best_post = min(key(rel(e2c, post)), key(rel(e2t, post)))
    keep_net = best_post < key(rel(e2, post))
    best.attach()

    # RHS throughput: p=2 + network, p=2, p=4 (FP64)
    def rhs_ms(ctx, u_dev, n=10):
        r = torch.empty_like(u_dev)
        for _ in range(2):
            ctx.rhs(u_dev.data_ptr(), r.data_ptr(), sp)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(n):
            ctx.rhs(u_dev.data_ptr(), r.data_ptr(), sp)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / n

    c2.profile(True)
    ms2c = rhs_ms(c2, u2_0)
    cls2c, _ = c2.profile_read()
    c2.profile(False)
    best.detach()   # the plain p=2 fallback when the p=4 check is negative
    ms2 = rhs_ms(c2, u2_0)
    ms4 = rhs_ms(c4, u4d)
    closure_ms = cls2c["closure"][0] / max(sum(v[0] for v in cls2c.values()), 1e-30) * ms2c
    nd2, nd4 = c2.ndof, c4.ndof
    for c in (c4, c4f, c2):
        c.close()
    name = {0: "tet", 1: "pri"}
    return {
        "workload": (f"Taylor-Green Re={TGV_RE:g} Ma={TGV_MACH:g}, periodic [0,2pi]^3, {TGV_CELLS}^3 cells "
                     "(lower half 2 prisms/cell, upper half 6 tets/cell), NS, p=2 + MLP 20nu-128-128-5nu "
                     "(BF16 GEMM inputs, FP32 accumulate) vs plain p=4"),
        "dt": dt, "stride_steps": TGV_STRIDE, "train_states": TGV_SNAPSHOTS,
        "train_t": [0.0, dt * TGV_STRIDE * (TGV_SNAPSHOTS - 1)], "end_t": dt * TGV_STRIDE * (nwin - 1),
        "train_iters": TGV_ITERS,
        "loss_log": {name[k]: v for k, v in log.items()},
        "target_rms_per_variable": {name[k]: list(map(float, v)) for k, v in cl.scale.items()},
        "held_out_rhs_rel_rms_err": {name[k]: {"with_network": v[0], "plain_p2": v[1]} for k, v in prior.items()},
        "held_out_t": dt * TGV_STRIDE * (nwin - 1),
        "ke_dissipation_rel_err_vs_p4": {
            "training_window": {"p2": rel(e2, tr), "p2_network": rel(e2c, tr),
                                "p2_network_trajectory_target": rel(e2t, tr)},
            "after_training_window": {"p2": rel(e2, post), "p2_network": rel(e2c, post),
                                      "p2_network_trajectory_target": rel(e2t, post)},
            "p4_rate_end": float(e4[-1]), "measure": "mean over windows of |eps - eps4| / |eps4|, "
                                                     "eps = -dKE/dt over each stride; p=4 in FP32 RHS"},
        "trajectory_target": {
            "target": "P RHS_4(u_4(t)) - RHS_2(u_2(t)), u_2 the plain p=2 solution at the same t (features of u_2)",
            "loss_log": {name[k]: v for k, v in log_t.items()},
            "held_out_rhs_rel_rms_err": {name[k]: {"with_network": v[0], "plain_p2": v[1]}
                                         for k, v in prior_t.items()},
            "training_s": train_t_s},
        "p4_check": {"network_kept": bool(keep_net),
                     "network": "projected target" if best is cl else "trajectory target",
                     "rule": "of the two networks (projected and trajectory-consistent targets) the one with the "
                             "lower dissipation error after the training window, kept only if it beats plain p=2 "
                             "there; otherwise detached (plain p=2 fallback)"},
        "rhs_ms": {"p2_network": ms2c, "p2": ms2, "p4": ms4, "closure_part_of_p2_network": closure_ms},
        "gdof_s": {"p2_network": nd2 / (ms2c * 1e-3) / 1e9, "p2": nd2 / (ms2 * 1e-3) / 1e9,
                   "p4": nd4 / (ms4 * 1e-3) / 1e9},
        "speedup_p2_network_vs_p4": ms4 / ms2c,
        "seconds": {"setup": setup_s, "trajectory": traj_s, "training": train_s},
    }


# ---------------------------------------------------------------------------
GEMM_CLASSES = ("M0", "grad", "M0_grad", "div")
X64_PROFILE = "k_gemm_x64_boundary_layer_p4_nx40.md"
X64_SOURCES = ("fr_gemm_x64.cu", "fr_gemm_body.cuh")


_FP64_PEAKS = {}


def fp64_peaks(fr, torch, local, sp):
    """FP64 denominators: the FMA peak derived from the SM count and the
    maximum SM clock, the library's FMA probe and cuBLAS DGEMM (the paper's
    reference-peak method), in TFLOP/s; measured once per process."""
    if local in _FP64_PEAKS:
        return _FP64_PEAKS[local]
    peaks = measured_peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_ghz = float(peaks.get("sm_max_mhz", 2070.0)) / 1e3
    out = {"derived": nsm * 2 * 2 * clk_ghz / 1e3,
           "source": f"derived: {nsm} SMs x 2 FP64 FMA/clk x 2 flop x {clk_ghz:.2f} GHz (maximum SM clock)"}
    try:
        out["fma_probe"] = fr.peak_fp64(sp) / 1e3
    except Exception:
        out["fma_probe"] = None
    try:
        out["dgemm"] = dgemm_reference_tflops(torch)
    except Exception:
        out["dgemm"] = None
    _FP64_PEAKS[local] = out
    return out


def alu_roofline(flops, ms, n, kernel, p64, traffic=None, traffic_src="n/a"):
    """FP64-pipe roofline entry: flops over ms of device time, n launches."""
    ach = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": p64["derived"], "unit": "TFLOP/s",
            "frac": ach / p64["derived"], "traffic": traffic, "traffic_source": traffic_src,
            "algorithmic_flops_per_launch": flops / max(n, 1),
            "flops": "2 x non-zero operator entries x columns (bench.gemm_flops)",
            "kernel": kernel, "launches": n, "avg_launch_ms": ms / max(n, 1),
            "peak_source": p64["source"],
            "peak_measured_fma_probe": p64["fma_probe"],
            "frac_of_measured_fma_probe": (ach / p64["fma_probe"]) if p64["fma_probe"] else None,
            "reference_peak_cublas_dgemm": p64["dgemm"],
            "frac_of_reference_peak": (ach / p64["dgemm"]) if p64["dgemm"] else None}


def step_roofline(fr, torch, ctx, prec, classes, typed, args, sp, local, nrhs=None):
    """Roofline of the dominant kernel of the timed RK4 steps.

    FR_FP64: the dominant operator class (FP64 pipe; flops = 2 x non-zero
    operator entries x columns).  FR_FP64S: the dominant launch by class and
    element type: an exact-split tensor-core launch against the sustained
    BF16 tensor peak (36 digit-pair MMAs per product, with its FP64-equivalent
    rate beside it), an FMA operator launch against the FP64 pipe, a
    point-wise launch against HBM (algorithmic bytes).  FP32-storage modes:
    the dominant operator class against HBM."""
    peaks = measured_peaks()
    nrhs = 4 * args.steps if nrhs is None else nrhs  # RHS evaluations the profile covers
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    full = args.nx == 75 and ctx.order == ORDER  # the committed traffic captures are of this workload
    if prec == fr.FR_FP64S:
        # launches grouped by kernel: the FMA operator kernel (types whose
        # operators stay on the FP64 pipe), the exact-split kernel (its
        # column-exponent pre-pass is inside the same event pair), and each
        # point-wise kernel
        groups = {}
        for cls, ty in typed:
            if cls in GEMM_CLASSES and ty != "all":
                kern = "k_gemm_x64" if x64_layout(ctx, cls, ty) is not None else "k_gemm"
            else:
                kern = "k_" + cls
            groups.setdefault(kern, []).append((cls, ty))
        kern = max(groups, key=lambda g: sum(typed[k][0] for k in groups[g]))
        keys = groups[kern]
        ms = sum(typed[k][0] for k in keys)
        n = sum(typed[k][1] for k in keys)
        parts = ", ".join(f"{c}/{t}" for c, t in keys)

        def traffic_of(profile=None, names=None):
            if not full:
                return None, "no capture of this workload"
            tot = 0.0
            for c, t in keys:
                kw = {} if profile is None else {"profile": profile, "names": names}
                b, src = profiled_traffic(c, etype=t, **kw)
                if b is None:
                    return None, src
                tot += b * typed[(c, t)][1]
            return tot / max(n, 1), src

        if kern == "k_gemm_x64":
            tfl = sum(x64_tensor_flops(ctx, c, t) for c, t in keys) * nrhs
            fl64 = sum(gemm_flops_type(ctx, c, t) for c, t in keys) * nrhs
            ach = tfl / (ms * 1e-3) / 1e12
            peak = peaks.get("bf16_tflops_sustained")
            src = "measured cuBLAS bf16 GEMM, sustained (MEASURED_PEAKS.json bf16_tflops_sustained)"
            if not peak:
                peak, src = 1700.0, "fallback: 1.7 PFLOP/s bf16 sustained"
            traffic, tsrc = traffic_of(X64_PROFILE, X64_SOURCES)
            p64 = fp64_peaks(fr, torch, local, sp)
            return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": traffic, "traffic_source": tsrc,
                    "kernel": f"k_gemm_x64 ({parts})", "launches": n, "avg_launch_ms": ms / max(n, 1),
                    "algorithmic_tensor_flops_per_launch": tfl / max(n, 1),
                    "flops": "36 digit-pair BF16 MMAs per product: 36 x 2 x 128-padded columns x row "
                             "blocks x MMA N x padded K (bench.x64_tensor_flops)",
                    "peak_source": src,
                    "fp64_equivalent_tflops": fl64 / (ms * 1e-3) / 1e12,
                    "fp64_equivalent_frac_of_fp64_fma_peak": fl64 / (ms * 1e-3) / 1e12 / p64["derived"],
                    "fp64_fma_peak": p64}
        if kern == "k_gemm":
            fl64 = sum(gemm_flops_type(ctx, c, t) for c, t in keys) * nrhs
            traffic, tsrc = traffic_of()
            return alu_roofline(fl64, ms, n, f"k_gemm FP64 FMA ({parts})", fp64_peaks(fr, torch, local, sp),
                                traffic, tsrc)
        b = sum(pointwise_bytes_fp64(ctx, c, t) or 0.0 for c, t in keys)
        if b:
            ach = b * nrhs / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": None, "kernel": f"{kern} ({parts})", "launches": n,
                    "avg_launch_ms": ms / max(n, 1), "algorithmic_bytes_per_launch": b * nrhs / max(n, 1),
                    "bytes": "bench.pointwise_bytes_fp64", "peak_source": hbm_src}
        return {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None, "traffic": None,
                "kernel": kern}
    dom = max(classes, key=lambda k: classes[k][0])
    dom_ms, dom_n = classes[dom]
    if dom in GEMM_CLASSES and prec != fr.FR_FP64:
        byts = gemm_bytes_f32(ctx, dom) * nrhs
        achieved = byts / (dom_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None,
                "kernel": ("k_gemm_tc" if prec in (fr.FR_BF16X3, fr.FR_TF32X3) else "k_gemm") + f" ({dom})",
                "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1), "peak_source": hbm_src}
    if dom in GEMM_CLASSES:
        traffic, tsrc = profiled_traffic(dom) if full else (None, "no capture of this workload")
        return alu_roofline(gemm_flops(ctx, dom) * nrhs, dom_ms, dom_n, f"k_gemm ({dom})",
                            fp64_peaks(fr, torch, local, sp), traffic, tsrc)
    return {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None, "traffic": None,
            "kernel": dom}


def fp64_mode(fr, torch, mesh, counts, u0, dt, ctx_main, prec_main, name, args, sp, local):
    """The other FP64 form of the headline workload (FR_FP64 FMA kernels, or
    FR_FP64S exact-split tensor-core operator products): K timed RK4 steps,
    its roofline, and the RHS and one-step increment differences between
    the two forms (both match the FP64 oracle to 1e-12).  Returns the plain
    FR_FP64 context (the reference of the reduced-precision errors) and the
    entry."""
    prec = fr.FR_FP64 if name == "fp64" else fr.FR_FP64S
    ctx = fr.Context(mesh, ORDER, **flow_params(), precision=prec)
    ctx.set_state(u0, sp)
    for _ in range(max(args.warmup, 0)):
        ctx.step(dt, 1, sp)
    torch.cuda.synchronize()
    stream = torch.cuda.ExternalStream(sp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step(dt, 1, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    classes, launches = ctx.profile_read()
    typed = ctx.profile_read_types()
    ctx.profile(False)
    ud = torch.from_numpy(u0).cuda()
    ra, rb = torch.empty_like(ud), torch.empty_like(ud)
    ctx_main.rhs(ud.data_ptr(), ra.data_ptr(), sp)
    ctx.rhs(ud.data_ptr(), rb.data_ptr(), sp)
    torch.cuda.synchronize()
    rhs_diff = per_quantity_rel_err(ra.cpu().numpy(), rb.cpu().numpy(), counts)
    ctx_main.set_state(u0, sp)
    ctx_main.step(dt, 1, sp)
    sa = ctx_main.get_state(stream=sp)
    ctx.set_state(u0, sp)
    ctx.step(dt, 1, sp)
    sb = ctx.get_state(stream=sp)
    inc_diff = per_quantity_rel_err(sa - u0, sb - u0, counts)
    out = {"value": ctx.ndof * 4.0 / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "gpu_launches": int(launches),
           "kernel_ms_per_step": {k: v[0] / args.steps for k, v in classes.items()},
           "kernel_ms_per_step_by_type": {f"{k}/{t}": v[0] / args.steps for (k, t), v in typed.items()},
           "roofline": step_roofline(fr, torch, ctx, prec, classes, typed, args, sp, local),
           "rhs_rel_diff_vs_headline": rhs_diff, "step_increment_rel_diff_vs_headline": inc_diff,
           "diff_measure": "[mass, momentum vector, energy] max|d|/max|ref|",
           "workload": WORKLOAD + (" [FP64 FMA throughout]" if name == "fp64" else
                                   " [operator products: exact-split FP64 on the tensor cores where dense]")}
    if prec == fr.FR_FP64:
        return ctx, out
    ctx.close()
    return ctx_main, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=75,
                    help="cells along x (75 = the full workload; smaller for profiling)")
    ap.add_argument("--cpu-oracle-child", type=int, default=0)
    ap.add_argument("--fp64-only", action="store_true", help="skip the other modes (precision, batched, learned)")
    ap.add_argument("--state-error-steps", type=int, default=0,
                    help="instead of timing: run this many RK4 steps at p=3 and p=4 in FP64 and each reduced "
                         "precision and print their state and diagnostics errors against FP64")
    ap.add_argument("--precision", default="fp64s", choices=["fp64s", "fp64", "fp32", "bf16x3", "tf32x3"],
                    help="arithmetic of the main timed step (default fp64s: FP64 with the exact-split "
                         "tensor-core operator products, the headline workload; fp64: FP64 FMA throughout)")
    ap.add_argument("--batched-only", type=int, default=0,
                    help="profiling: time only the batched mode on its first N problems and print its entry")
    args = ap.parse_args()

    if args.cpu_oracle_child:
        cpu_oracle_child(args.cpu_oracle_child)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        nrhs = args.warmup + args.steps
        res = run_cpu_oracle(nrhs)
        times = res["times"][args.warmup:] or res["times"]
        t = sum(times) / len(times)
        val = res["ndof"] / t / 1e9
        cb = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": (f"one NS p=4 RHS per step on the nx={CPU_SAMPLE_NX} sample "
                         f"({res['ndof']} DOF), 1 BLAS thread")}
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOAD + f" (oracle sample nx={CPU_SAMPLE_NX})"},
                          "cpu_baseline": cb,
                          "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    # CPU baseline first (child process, before any CUDA work in this one)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.nx == 75:
        try:
            cpu_base = cpu_baseline_entry(1)
        except Exception as e:  # reported, not fatal
            cpu_base = {"error": str(e)[:300]}

    import torch
    import synth
    from paper_1409_0405_gb300 import fr

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    if args.batched_only > 0:
        if rank == 0:
            sp0 = torch.cuda.Stream().cuda_stream
            print(json.dumps({"batched": batch_mode(fr, torch, args, sp0, nprob=args.batched_only)}))
        return

    if args.state_error_steps > 0:
        if rank == 0:
            sp0 = torch.cuda.Stream().cuda_stream
            print(json.dumps({"study": "reduced-precision state error after RK4 steps, boundary-layer workload",
                              "results": state_error_study(fr, torch, args.state_error_steps, sp0)}))
        return

    mesh = synth.boundary_layer_box(nx=args.nx)
    prec = {"fp64s": fr.FR_FP64S, "fp64": fr.FR_FP64, "fp32": fr.FR_FP32, "bf16x3": fr.FR_BF16X3,
            "tf32x3": fr.FR_TF32X3}[args.precision]
    try:
        free0 = torch.cuda.mem_get_info()[0]
    except Exception:
        free0 = None
    ctx = fr.Context(mesh, ORDER, **flow_params(), precision=prec)
    try:
        ctx_gb = (free0 - torch.cuda.mem_get_info()[0]) / 1e9 if free0 is not None else None
    except Exception:
        ctx_gb = None
    counts = ctx.counts()
    u0 = points_to_public(synth.perturbed_freestream(ctx.upts_points(), seed=2,
                                                     wall_delta=WALL_DELTA), counts)
    dt = time_step_size(mesh, ORDER)
    ndof = ctx.ndof

    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    ctx.set_state(u0, sp)
    for _ in range(max(args.warmup, 0)):
        ctx.step(dt, 1, sp)
    torch.cuda.synchronize()

    # --- timed region: K RK4 steps, inputs resident in HBM (all > L2) ---
    gpu_uuid = torch.cuda.get_device_properties(local).uuid
    sampler = ClockSampler(f"GPU-{gpu_uuid}")
    ctx.profile(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with sampler:
        time.sleep(0.3)
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.step(dt, 1, sp)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    classes, launches = ctx.profile_read()
    typed = ctx.profile_read_types()
    ctx.profile(False)
    ms_step = max_over_ranks(ms_total / args.steps, world, "cuda")
    value = job_gdofs(world, ndof, ms_step * 1e-3)
    state_ok = ctx.reduce(stream=sp, check=False)[6] == 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    diag = ctx.diagnostics(sp)
    diag_ms = (time.perf_counter() - t0) * 1e3

    # --- e2e through the C ABI with host buffers ---
    pin_in = torch.from_numpy(u0).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    hin, hout = pin_in.numpy(), pin_out.numpy()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.set_state(hin, sp)
        ctx.step(dt, 1, sp)
        ctx.get_state(hout, sp)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, "cuda")
    e2e_val = job_gdofs(world, ndof, e2e_s)

    # --- other precision modes beside the FP64 line (same mesh, same state) ---
    modes = {}
    fp64_line = args.precision in ("fp64", "fp64s")
    if fp64_line and not args.fp64_only:
        # the other FP64 form beside the headline; the plain FMA context is
        # the reference of the reduced-precision errors (it matches the FP64
        # oracle to 1e-12, as does FR_FP64S)
        other = "fp64" if args.precision == "fp64s" else "fp64s"
        ctx64, modes[other] = fp64_mode(fr, torch, mesh, counts, u0, dt, ctx, prec, other, args, sp, local)
        modes["fp32"] = precision_mode(fr, torch, mesh, counts, u0, dt, ctx64, fr.FR_FP32, args, sp)
        modes["bf16x3"] = precision_mode(fr, torch, mesh, counts, u0, dt, ctx64, fr.FR_BF16X3, args, sp)
        modes["tf32x3"] = precision_mode(fr, torch, mesh, counts, u0, dt, ctx64, fr.FR_TF32X3, args, sp)
        if ctx64 is not ctx:
            ctx64.close()
        modes["rk45"] = rk45_mode(fr, torch, mesh, u0, dt, args, sp, prec)
        modes["partitioned"] = partitioned_mode(fr, torch, mesh, u0, dt, ms_total / args.steps, args, sp, prec)
        if args.nx == 75:
            modes["p3"] = p3_modes(fr, torch, mesh, args, sp)
            modes["batched"] = batch_mode(fr, torch, args, sp)
            modes["learned"] = learned_mode(fr, torch, args, sp)
            modes["hex"] = hex_mode(fr, torch, args, sp)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # --- roofline of the dominant kernel ---
    roof = step_roofline(fr, torch, ctx, prec, classes, typed, args, sp, local)
    gemm_classes = ("M0", "grad", "M0_grad", "div")
    all_gemm = sum(gemm_flops(ctx, k) for k in gemm_classes) * 4 * args.steps
    clocks = sampler.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64s": "f64", "fp64": "f64", "fp32": "f32", "bf16x3": "bf16x3+f32",
                  "tf32x3": "tf32x3+f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.nx == 75 else WORKLOAD + f" (reduced: nx={args.nx})")
                   + {"fp64s": " [operator products: exact-split FP64 on the tensor cores where dense (tets), "
                                "FP64 FMA elsewhere]", "fp64": " [FP64 FMA throughout]"}.get(
                       args.precision, f" [{args.precision} arithmetic]"),
                   "ndof": ndof, "rhs_per_step": 4, "dt": dt,
                   "l2": "inputs > L2 (state 339 MB per register, scratch > 4 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "state_finite_after_timed_steps": bool(state_ok),
                   "device_memory_gb": ctx_gb},
        "roofline": roof,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in classes.items()},
        "kernel_ms_per_step_by_type": {f"{k}/{t}": v[0] / args.steps for (k, t), v in typed.items()},
        "gemm_fp64_tflops": all_gemm / (sum(classes[k][0] for k in gemm_classes) * 1e-3) / 1e12,
        "cpu_baseline": cpu_base,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(ndof * 8),
                "d2h_bytes_per_step": int(ndof * 8), "steps": e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "diagnostics_after_timed_steps": {"ke_rate": diag[0], "wall_force_inviscid": diag[1].tolist(),
                                          "wall_force_viscous": diag[2].tolist(), "host_ms": diag_ms},
        "modes": modes,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
