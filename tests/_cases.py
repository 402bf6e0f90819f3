"""Shared helpers for parity tests: build both sides on the same inputs and
compare element by element.  Inputs come from the seeded generators and the
oracle; nothing here feeds a CUDA result back into an oracle input."""
import numpy as np

import synth
from oracle.solver import Solver

GAMMA = 1.4
# boundary-layer thickness of the wall-consistent initial profile
BL_DELTA = 0.5


def library():
    """Build (incrementally) and load libfr.so."""
    from paper_1409_0405_gb300 import build, fr
    build.build()
    return fr.load()


def bl_params(p_inf=None, mu=1.0 / 3900.0, viscous=True):
    p_inf = 1.0 / (GAMMA * 0.2 ** 2) if p_inf is None else p_inf
    return dict(viscous=viscous, mu=mu, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1,
                rho_inf=1.0, vel_inf=(1.0, 0.0, 0.0), p_inf=p_inf, t_wall=p_inf)


def make_pair(mesh, p, **params):
    """(oracle solver, library context) for the same mesh/order/params."""
    from paper_1409_0405_gb300 import fr
    ctx = fr.Context(mesh, p, **params)
    params = {k: v for k, v in params.items() if k != "precision"}
    sol = Solver(mesh, p, gamma=params.get("gamma", GAMMA), mu=params.get("mu", 0.0),
                 prandtl=params.get("prandtl", 0.72), viscous=bool(params.get("viscous", False)),
                 ldg_beta=params.get("ldg_beta", 0.5), ldg_tau=params.get("ldg_tau", 0.1),
                 rho_inf=params.get("rho_inf", 1.0), vel_inf=params.get("vel_inf", (1.0, 0.0, 0.0)),
                 p_inf=params.get("p_inf"), t_wall=params.get("t_wall"))
    return sol, ctx


def state(sol, kind, seed=0):
    xyz = sol.upts_xyz_points()
    if kind == "vortex":
        q = synth.isentropic_vortex(xyz)
    elif kind == "smooth":
        q = synth.random_smooth_state(xyz, seed=seed)
    elif kind == "bl":
        q = synth.perturbed_freestream(xyz, seed=2, wall_delta=BL_DELTA)
    elif kind == "impulsive":
        q = synth.perturbed_freestream(xyz, seed=2)
    elif kind == "tgv":
        q = synth.taylor_green(xyz)
    else:
        raise ValueError(kind)
    return sol.state_from_points(q)


def per_var_rel_err(sol, ref, got):
    """max |got - ref| / max |ref| for each conserved variable."""
    r = sol.split(np.asarray(ref))
    g = sol.split(np.asarray(got))
    out = []
    for v in range(5):
        num = max(float(np.max(np.abs(g[t][:, v] - r[t][:, v]))) for t in sol.types)
        den = max(float(np.max(np.abs(r[t][:, v]))) for t in sol.types)
        out.append(num / den if den > 0 else num)
    return np.array(out)


def gpu_rhs(ctx, u):
    import torch
    ut = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    rt = torch.empty_like(ut)
    s = torch.cuda.current_stream()
    ctx.rhs(ut.data_ptr(), rt.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    return rt.cpu().numpy()


def to_longdouble(sol, ld=np.longdouble):
    """Switch an oracle instance to numpy extended precision (used only to
    measure the FP64 rounding floor of a case); with ld=np.float32, to
    single precision (the FP32 rounding floor of a plain evaluation)."""
    import copy
    for t in sol.types:
        # copy: the oracle caches its operator objects across solvers
        op = sol.m.ops[t] = copy.copy(sol.m.ops[t])
        for k in ("M0", "D", "M3", "fnorm", "w", "fw"):
            setattr(op, k, getattr(op, k).astype(ld))
        sol.m.J[t] = sol.m.J[t].astype(ld)
        sol.m.S[t] = sol.m.S[t].astype(ld)
    sol.m.gn = sol.m.gn.astype(ld)
    sol.m.gmag = sol.m.gmag.astype(ld)
    sol.na = sol.na.astype(ld)
    return sol


def per_quantity_rel_err(sol, ref, got):
    """Frame-invariant relative error per conserved quantity:
    [mass, momentum (Euclidean norm of the 3-vector), energy], each
    max over points |got - ref| / max over points |ref|."""
    r = sol.split(np.asarray(ref, dtype=np.float64))
    g = sol.split(np.asarray(got, dtype=np.float64))
    out = []
    for sl in (slice(0, 1), slice(1, 4), slice(4, 5)):
        num = max(float(np.max(np.linalg.norm(g[t][:, sl] - r[t][:, sl], axis=1))) for t in sol.types)
        den = max(float(np.max(np.linalg.norm(r[t][:, sl], axis=1))) for t in sol.types)
        out.append(num / den if den > 0 else num)
    return np.array(out)
