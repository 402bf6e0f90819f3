"""Thin ctypes binding of libfr.so (the C ABI declared in include/fr.h).

Argument marshalling only: every step of the FR right-hand side runs in
the library's CUDA kernels.  PyTorch is used by callers for device memory
and streams; this module passes raw pointers.  Loading fails loudly when
the shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfr.so")

FR_OK = 0
FR_ERR_ARG = -1
FR_ERR_MESH = -2
FR_ERR_CUDA = -3
FR_ERR_NONFINITE = -4
FR_ERR_TIMEOUT = -5
FR_ERR_NOMEM = -6
FR_ERR_UNSUPPORTED = -7
FR_FP64 = 0
FR_FP32 = 1
FR_BF16X3 = 2
FR_TF32X3 = 3
FR_FP64S = 4
NVARS = 5

OP_IDS = {"M0": 0, "D": 1, "M3": 2, "AGRAD": 3, "ADIV": 4, "W": 5, "UPTS": 6,
          "FPTS": 7, "FNORM": 8, "FW": 9}

# every entry point declared in include/fr.h
EXPORTS = ("fr_create", "fr_destroy", "fr_ndof", "fr_info", "fr_upts",
           "fr_set_state", "fr_get_state", "fr_rhs", "fr_step", "fr_check", "fr_step_ls", "fr_step_rk45",
           "fr_rk45_error", "fr_rk45_get_error", "fr_step_rk45_adaptive", "fr_reduce",
           "fr_diagnostics", "fr_selftest_wait_timeout", "fr_operator", "fr_profile", "fr_profile_read", "fr_profile_read_types", "fr_peak_fp64", "fr_gemm_fp64s", "fr_strerror",
           "fr_last_error", "fr_reduce_noalloc", "fr_batch_create", "fr_batch_destroy",
           "fr_batch_problem", "fr_batch_tune", "fr_batch_step", "fr_batch_check",
           "fr_batch_selftest_wait_timeout", "fr_batch_info",
           "fr_transfer", "fr_transfer_state", "fr_closure_features", "fr_closure_sample",
           "fr_closure_set", "fr_mlp_nparams", "fr_mlp_workspace", "fr_mlp_forward", "fr_mlp_grad",
           "fr_mlp_adam", "fr_partition", "fr_part_plan", "fr_part_create", "fr_part_destroy",
           "fr_part_info", "fr_part_set_state", "fr_part_get_state", "fr_part_rhs", "fr_part_step",
           "fr_part_reduce", "fr_part_launches", "fr_debug_fail_alloc", "fr_debug_alloc_stats")
KCLASSES = ("M0", "common_solution", "grad", "M0_grad", "flux", "common_flux", "div", "closure", "check")


class FRMesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("n_tet", C.c_int64), ("tet", C.POINTER(C.c_int64)),
                ("n_pri", C.c_int64), ("pri", C.POINTER(C.c_int64)),
                ("n_hex", C.c_int64), ("hex", C.POINTER(C.c_int64)),
                ("n_bface", C.c_int64), ("bface", C.POINTER(C.c_int64)),
                ("period", C.c_double * 3),
                ("geom_order", C.c_int), ("tet_nodes", C.POINTER(C.c_double)),
                ("pri_nodes", C.POINTER(C.c_double)), ("hex_nodes", C.POINTER(C.c_double))]


class FRParams(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mu", C.c_double), ("prandtl", C.c_double),
                ("ldg_beta", C.c_double), ("ldg_tau", C.c_double),
                ("viscous", C.c_int), ("precision", C.c_int),
                ("rho_inf", C.c_double), ("vel_inf", C.c_double * 3),
                ("p_inf", C.c_double), ("t_wall", C.c_double)]


class FRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def load():
    """Load libfr.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run paper_1409_0405_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    lib.fr_create.argtypes = [C.POINTER(FRMesh), C.c_int, C.POINTER(FRParams), C.POINTER(vp)]
    lib.fr_destroy.argtypes = [vp]
    lib.fr_destroy.restype = None
    lib.fr_ndof.argtypes = [vp, i64p]
    lib.fr_info.argtypes = [vp, i64p]
    lib.fr_upts.argtypes = [vp, dp]
    lib.fr_set_state.argtypes = [vp, dp, vp]
    lib.fr_get_state.argtypes = [vp, dp, vp]
    lib.fr_rhs.argtypes = [vp, vp, vp, vp]
    lib.fr_step.argtypes = [vp, C.c_double, C.c_int, vp]
    lib.fr_check.argtypes = [vp, vp]
    lib.fr_check.restype = C.c_int
    lib.fr_step_ls.argtypes = [vp, C.c_double, C.c_int, vp]
    lib.fr_step_ls.restype = C.c_int
    lib.fr_step_rk45.argtypes = [vp, C.c_double, C.c_int, vp]
    lib.fr_step_rk45.restype = C.c_int
    lib.fr_rk45_error.argtypes = [vp, C.c_double, C.c_double, vp, vp]
    lib.fr_rk45_error.restype = C.c_int
    lib.fr_rk45_get_error.argtypes = [vp, vp, vp]
    lib.fr_rk45_get_error.restype = C.c_int
    lib.fr_step_rk45_adaptive.argtypes = [vp, C.c_double, C.c_double, C.c_double, vp, C.c_int, vp, vp]
    lib.fr_step_rk45_adaptive.restype = C.c_int
    lib.fr_reduce.argtypes = [vp, dp, vp]
    lib.fr_diagnostics.argtypes = [vp, dp, vp]
    lib.fr_selftest_wait_timeout.argtypes = [vp, vp]
    lib.fr_operator.argtypes = [C.c_int, C.c_int, C.c_int, dp, i64p, i64p]
    lib.fr_profile.argtypes = [vp, C.c_int]
    lib.fr_profile_read.argtypes = [vp, dp, i64p, i64p]
    lib.fr_profile_read_types.argtypes = [vp, dp, i64p]
    lib.fr_peak_fp64.argtypes = [dp, vp]
    lib.fr_peak_fp64.restype = C.c_int
    lib.fr_gemm_fp64s.argtypes = [C.c_int, C.c_int, dp, C.c_int64, vp, vp, vp]
    lib.fr_gemm_fp64s.restype = C.c_int
    lib.fr_reduce_noalloc.argtypes = [C.c_int64, C.c_int, vp, vp, C.c_double, vp, vp]
    lib.fr_reduce_noalloc.restype = C.c_int
    lib.fr_batch_create.argtypes = [C.c_int, C.POINTER(FRMesh), C.POINTER(C.c_int), C.POINTER(FRParams),
                                    C.POINTER(vp)]
    lib.fr_batch_destroy.argtypes = [vp]
    lib.fr_batch_destroy.restype = None
    lib.fr_batch_problem.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.fr_batch_tune.argtypes = [vp, vp]
    lib.fr_batch_step.argtypes = [vp, dp, C.c_int, C.c_int, vp]
    lib.fr_batch_info.argtypes = [vp, i64p]
    lib.fr_batch_check.argtypes = [vp, vp]
    lib.fr_batch_selftest_wait_timeout.argtypes = [vp, vp]
    for name in ("fr_batch_create", "fr_batch_problem", "fr_batch_tune", "fr_batch_step", "fr_batch_info",
                 "fr_batch_check", "fr_batch_selftest_wait_timeout"):
        getattr(lib, name).restype = C.c_int
    lib.fr_transfer.argtypes = [C.c_int, C.c_int, C.c_int, dp, i64p, i64p]
    lib.fr_transfer_state.argtypes = [vp, vp, vp, vp, vp]
    lib.fr_closure_features.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.fr_closure_sample.argtypes = [vp, vp, vp, vp, C.c_int, dp, vp, vp, vp, vp]
    lib.fr_closure_set.argtypes = [vp, C.c_int, vp, C.c_int, dp]
    lib.fr_mlp_nparams.argtypes = [C.c_int, C.c_int, C.c_int]
    lib.fr_mlp_nparams.restype = C.c_int64
    lib.fr_mlp_workspace.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64]
    lib.fr_mlp_workspace.restype = C.c_int64
    lib.fr_mlp_forward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, vp, vp, vp, vp, vp]
    lib.fr_mlp_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
    lib.fr_mlp_adam.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_int, C.c_float, vp]
    for name in ("fr_transfer", "fr_transfer_state", "fr_closure_features", "fr_closure_sample",
                 "fr_closure_set", "fr_mlp_forward", "fr_mlp_grad", "fr_mlp_adam"):
        getattr(lib, name).restype = C.c_int
    i32p = C.POINTER(C.c_int32)
    lib.fr_partition.argtypes = [C.POINTER(FRMesh), C.c_int, dp, i32p]
    lib.fr_part_plan.argtypes = [C.POINTER(FRMesh), C.c_int, C.c_int, i32p, C.c_int, i64p, i32p, i32p]
    lib.fr_part_create.argtypes = [C.POINTER(FRMesh), C.c_int, C.POINTER(FRParams), C.c_int, i32p, C.POINTER(vp)]
    lib.fr_part_destroy.argtypes = [vp]
    lib.fr_part_destroy.restype = None
    lib.fr_part_info.argtypes = [vp, i64p]
    lib.fr_part_set_state.argtypes = [vp, dp, vp]
    lib.fr_part_get_state.argtypes = [vp, dp, vp]
    lib.fr_part_rhs.argtypes = [vp, vp, vp, vp]
    lib.fr_part_step.argtypes = [vp, C.c_double, C.c_int, vp]
    lib.fr_part_reduce.argtypes = [vp, dp, vp]
    lib.fr_part_launches.argtypes = [vp, i64p]
    for name in ("fr_partition", "fr_part_plan", "fr_part_create", "fr_part_info", "fr_part_set_state",
                 "fr_part_get_state", "fr_part_rhs", "fr_part_step", "fr_part_reduce", "fr_part_launches"):
        getattr(lib, name).restype = C.c_int
    lib.fr_debug_fail_alloc.argtypes = [C.c_int64]
    lib.fr_debug_fail_alloc.restype = C.c_int
    lib.fr_debug_alloc_stats.argtypes = [i64p]
    lib.fr_debug_alloc_stats.restype = C.c_int
    lib.fr_strerror.argtypes = [C.c_int]
    lib.fr_strerror.restype = C.c_char_p
    lib.fr_last_error.argtypes = []
    lib.fr_last_error.restype = C.c_char_p
    for name in ("fr_create", "fr_ndof", "fr_info", "fr_upts", "fr_set_state",
                 "fr_get_state", "fr_rhs", "fr_step", "fr_reduce", "fr_diagnostics", "fr_selftest_wait_timeout",
                 "fr_operator",
                 "fr_profile", "fr_profile_read", "fr_profile_read_types"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


ETYPES = ("tet", "pri", "hex")


def _etype(e):
    return {"tet": 0, "pri": 1, "hex": 2}.get(e, e)


def _check(rc):
    if rc != FR_OK:
        lib = load()
        raise FRError(rc, f"{lib.fr_strerror(rc).decode()}: {lib.fr_last_error().decode()}")


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def operator(etype, order, which):
    """Host-only operator query (no GPU needed): returns a float64 matrix."""
    lib = load()
    rows, cols = C.c_int64(), C.c_int64()
    wid = OP_IDS[which] if isinstance(which, str) else int(which)
    et = _etype(etype)
    _check(lib.fr_operator(et, order, wid, None, C.byref(rows), C.byref(cols)))
    out = np.empty((rows.value, cols.value), dtype=np.float64)
    _check(lib.fr_operator(et, order, wid, _dptr(out), C.byref(rows), C.byref(cols)))
    return out


def gemm_fp64s(A, K_by_N_dev, C_dev, N, stream=None):
    """fr_gemm_fp64s: C = A B through the exact-split tensor-core kernel.

    A: host float64 (M x K); K_by_N_dev / C_dev: device pointers of the
    row-major K x N operand and the M x N result."""
    lib = load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    M, K = A.shape
    _check(lib.fr_gemm_fp64s(int(M), int(K), _dptr(A), int(N), C.c_void_p(K_by_N_dev), C.c_void_p(C_dev),
                             C.c_void_p(stream) if stream else None))


def transfer(etype, p_from, p_to):
    """Host-only order-transfer matrix (nu(p_to) x nu(p_from)), float64."""
    lib = load()
    rows, cols = C.c_int64(), C.c_int64()
    et = _etype(etype)
    _check(lib.fr_transfer(et, int(p_from), int(p_to), None, C.byref(rows), C.byref(cols)))
    out = np.empty((rows.value, cols.value), dtype=np.float64)
    _check(lib.fr_transfer(et, int(p_from), int(p_to), _dptr(out), C.byref(rows), C.byref(cols)))
    return out


def _sp(stream):
    return C.c_void_p(stream) if stream else None


def mlp_nparams(nin, nh, nout):
    return int(load().fr_mlp_nparams(int(nin), int(nh), int(nout)))


def mlp_workspace(nin, nh, nout, n):
    return int(load().fr_mlp_workspace(int(nin), int(nh), int(nout), int(n)))


def mlp_forward(nin, nh, nout, n, x_ptr, p_ptr, y_ptr, ws_ptr, stream=None):
    _check(load().fr_mlp_forward(int(nin), int(nh), int(nout), int(n), C.c_void_p(x_ptr), C.c_void_p(p_ptr),
                                 C.c_void_p(y_ptr), C.c_void_p(ws_ptr), _sp(stream)))


def mlp_grad(nin, nh, nout, n, x_ptr, t_ptr, p_ptr, g_ptr, loss_ptr, ws_ptr, stream=None):
    _check(load().fr_mlp_grad(int(nin), int(nh), int(nout), int(n), C.c_void_p(x_ptr), C.c_void_p(t_ptr),
                              C.c_void_p(p_ptr), C.c_void_p(g_ptr), C.c_void_p(loss_ptr), C.c_void_p(ws_ptr),
                              _sp(stream)))


def mlp_adam(nparams, p_ptr, g_ptr, m_ptr, v_ptr, step, lr, stream=None):
    _check(load().fr_mlp_adam(int(nparams), C.c_void_p(p_ptr), C.c_void_p(g_ptr), C.c_void_p(m_ptr),
                              C.c_void_p(v_ptr), int(step), float(lr), _sp(stream)))


def peak_fp64(stream=None):
    """Measured FP64 FMA throughput of the current GPU in GFLOP/s."""
    lib = load()
    g = C.c_double()
    _check(lib.fr_peak_fp64(C.byref(g), C.c_void_p(stream) if stream else None))
    return g.value


def reduce_noalloc(ne, nu, u_ptr, wj_ptr, gamma, out_ptr, stream=None):
    """fr_reduce_noalloc on raw device pointers (no allocation anywhere);
    returns the library's status code."""
    lib = load()
    return lib.fr_reduce_noalloc(int(ne), int(nu), C.c_void_p(u_ptr), C.c_void_p(wj_ptr), float(gamma),
                                 C.c_void_p(out_ptr), C.c_void_p(stream) if stream else None)


def default_params(viscous=False, mu=0.0, gamma=1.4, prandtl=0.72, ldg_beta=0.5,
                   ldg_tau=0.1, rho_inf=1.0, vel_inf=(1.0, 0.0, 0.0), p_inf=None,
                   t_wall=None, precision=FR_FP64):
    p_inf = 1.0 / gamma if p_inf is None else p_inf
    t_wall = p_inf / rho_inf if t_wall is None else t_wall
    return dict(gamma=gamma, mu=mu, prandtl=prandtl, ldg_beta=ldg_beta, ldg_tau=ldg_tau,
                viscous=int(viscous), precision=precision, rho_inf=rho_inf,
                vel_inf=tuple(vel_inf), p_inf=p_inf, t_wall=t_wall)


def _fr_mesh(mesh, keep):
    """Fill an FRMesh from a mesh dict; arrays are kept alive in `keep`."""
    k = {
        "xyz": np.ascontiguousarray(mesh["xyz"], dtype=np.float64),
        "tet": np.ascontiguousarray(mesh["tet"], dtype=np.int64).reshape(-1, 4),
        "pri": np.ascontiguousarray(mesh["pri"], dtype=np.int64).reshape(-1, 6),
        "hex": np.ascontiguousarray(mesh.get("hex", np.zeros((0, 8))), dtype=np.int64).reshape(-1, 8),
        "bface": np.ascontiguousarray(mesh.get("bface", np.zeros((0, 4))), dtype=np.int64).reshape(-1, 4),
    }
    keep.append(k)
    m = FRMesh()
    m.n_nodes = len(k["xyz"])
    m.xyz = _dptr(k["xyz"])
    m.n_tet = len(k["tet"])
    m.tet = k["tet"].ctypes.data_as(C.POINTER(C.c_int64))
    m.n_pri = len(k["pri"])
    m.pri = k["pri"].ctypes.data_as(C.POINTER(C.c_int64))
    m.n_hex = len(k["hex"])
    m.hex = k["hex"].ctypes.data_as(C.POINTER(C.c_int64))
    m.n_bface = len(k["bface"])
    m.bface = k["bface"].ctypes.data_as(C.POINTER(C.c_int64))
    per = np.asarray(mesh.get("period", np.zeros(3)), dtype=np.float64)
    m.period = (C.c_double * 3)(*per)
    m.geom_order = int(mesh.get("geom_order", 1))
    if m.geom_order == 2:
        for t, nq in (("tet", 10), ("pri", 18), ("hex", 27)):
            if t + "_nodes" not in mesh:
                continue  # left NULL: the library rejects a present type without nodes
            a = np.ascontiguousarray(mesh[t + "_nodes"], dtype=np.float64)
            if a.shape != (len(k[t]), nq, 3):
                raise ValueError(f"{t}_nodes must have shape ({len(k[t])}, {nq}, 3)")
            k[t + "_nodes"] = a
            setattr(m, t + "_nodes", _dptr(a))
    return m


def _fr_params(prm):
    p = FRParams()
    for key, val in prm.items():
        if key == "vel_inf":
            p.vel_inf = (C.c_double * 3)(*val)
        else:
            setattr(p, key, val)
    return p


class Context:
    """One fr_ctx: mesh + order + parameters resident on the current GPU."""

    def __init__(self, mesh, order, _handle=None, _owner=None, **params):
        lib = load()
        prm = default_params(**params)
        self.params = prm
        self._lib = lib
        self._owner = _owner
        if _handle is None:
            self._keep = []
            m = _fr_mesh(mesh, self._keep)
            p = _fr_params(prm)
            h = C.c_void_p()
            _check(lib.fr_create(C.byref(m), int(order), C.byref(p), C.byref(h)))
        else:
            h = _handle
        self._h = h
        n = C.c_int64()
        _check(lib.fr_ndof(h, C.byref(n)))
        self.ndof = n.value
        info = (C.c_int64 * 11)()
        _check(lib.fr_info(h, info))
        self.info = dict(zip(("n_tet", "n_pri", "order", "nu_tet", "nu_pri", "nf_tet",
                              "nf_pri", "npairs", "n_hex", "nu_hex", "nf_hex"), list(info)))
        self.order = int(info[2])

    def close(self):
        if getattr(self, "_h", None):
            if self._owner is None:        # contexts of a batch belong to it
                self._lib.fr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries ---------------------------------------------------------------
    def upts(self):
        """(ndof/5*3,) physical solution-point coordinates, public layout."""
        out = np.empty(self.ndof // NVARS * 3, dtype=np.float64)
        _check(self._lib.fr_upts(self._h, _dptr(out)))
        return out

    def upts_points(self):
        """(n_points, 3) coordinates in public point order."""
        x = self.upts()
        blocks, off = [], 0
        for ne, nu in self.counts():
            if ne == 0:
                continue
            blk = x[off:off + ne * 3 * nu].reshape(ne, 3, nu).transpose(0, 2, 1).reshape(-1, 3)
            blocks.append(blk)
            off += ne * 3 * nu
        return np.concatenate(blocks)

    # -- compute ---------------------------------------------------------------
    def set_state(self, u, stream=None):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == self.ndof
        _check(self._lib.fr_set_state(self._h, _dptr(u), stream))

    def get_state(self, out=None, stream=None):
        out = np.empty(self.ndof, dtype=np.float64) if out is None else out
        _check(self._lib.fr_get_state(self._h, _dptr(out), stream))
        return out

    def rhs(self, u_ptr, r_ptr, stream=None):
        """r = R(u) for device pointers (ints, e.g. tensor.data_ptr())."""
        _check(self._lib.fr_rhs(self._h, C.c_void_p(u_ptr), C.c_void_p(r_ptr),
                                C.c_void_p(stream) if stream else None))

    def step(self, dt, nsteps=1, stream=None):
        _check(self._lib.fr_step(self._h, float(dt), int(nsteps),
                                 C.c_void_p(stream) if stream else None))

    def check(self, stream=None):
        """fr_check: raises FRError (FR_ERR_NONFINITE) after a blown-up step."""
        _check(self._lib.fr_check(self._h, C.c_void_p(stream) if stream else None))

    def step_ls(self, dt, nsteps=1, stream=None):
        """Low-storage (2N) five-stage RK4 steps (fr_step_ls)."""
        _check(self._lib.fr_step_ls(self._h, float(dt), int(nsteps), C.c_void_p(stream) if stream else None))

    def step_rk45(self, dt, nsteps=1, stream=None):
        """Fixed RK45[2R+] steps (fr_step_rk45)."""
        _check(self._lib.fr_step_rk45(self._h, float(dt), int(nsteps), C.c_void_p(stream) if stream else None))

    def rk45_error(self, atol, rtol, stream=None):
        """Weighted RMS norm of the last RK45 step's error estimate."""
        out = C.c_double(0.0)
        _check(self._lib.fr_rk45_error(self._h, float(atol), float(rtol), C.byref(out),
                                       C.c_void_p(stream) if stream else None))
        return out.value

    def rk45_get_error(self, stream=None):
        """The last RK45 step's error register, public layout."""
        out = np.empty(self.ndof, dtype=np.float64)
        _check(self._lib.fr_rk45_get_error(self._h, _dptr(out), C.c_void_p(stream) if stream else None))
        return out

    def step_rk45_adaptive(self, t_span, dt, atol, rtol, max_steps=100000, stream=None):
        """Error-controlled RK45[2R+] over t_span: (next dt, accepted, rejected)."""
        d = C.c_double(float(dt))
        stats = np.zeros(2, dtype=np.int64)
        _check(self._lib.fr_step_rk45_adaptive(self._h, float(t_span), float(atol), float(rtol), C.byref(d),
                                               int(max_steps), stats.ctypes.data_as(C.c_void_p),
                                               C.c_void_p(stream) if stream else None))
        return d.value, int(stats[0]), int(stats[1])

    def profile(self, enable=True):
        _check(self._lib.fr_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{class: (ms, count)} and the total launch count since the reset."""
        ms = np.zeros(len(KCLASSES))
        cnt = np.zeros(len(KCLASSES), dtype=np.int64)
        tot = C.c_int64()
        _check(self._lib.fr_profile_read(self._h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                         C.byref(tot)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KCLASSES)}, tot.value

    def profile_read_types(self):
        """{(class, type): (ms, count)}: type "all" for the launches that span
        every element type, else "tet", "pri" or "hex"; entries with no
        launch are left out."""
        nk = len(KCLASSES)
        ms = np.zeros((len(ETYPES) + 1) * nk)
        cnt = np.zeros((len(ETYPES) + 1) * nk, dtype=np.int64)
        _check(self._lib.fr_profile_read_types(self._h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
        out = {}
        for b, ty in enumerate(("all",) + tuple(ETYPES)):
            for i, k in enumerate(KCLASSES):
                if cnt[b * nk + i]:
                    out[(k, ty)] = (float(ms[b * nk + i]), int(cnt[b * nk + i]))
        return out

    def counts(self):
        """[(elements, solution points per element)] per type, public order."""
        return [(self.info["n_" + t], self.info["nu_" + t]) for t in ETYPES]

    # -- learned closure (device pointers are ints) --------------------------------
    def nu(self, etype):
        return self.info["nu_" + ETYPES[_etype(etype)]]

    def ne(self, etype):
        return self.info["n_" + ETYPES[_etype(etype)]]

    def transfer_from(self, other, u_ptr, out_ptr, stream=None):
        """out (this context's order) = transfer of u (other's order)."""
        _check(self._lib.fr_transfer_state(other._h, self._h, C.c_void_p(u_ptr), C.c_void_p(out_ptr),
                                           _sp(stream)))

    def closure_features(self, u_ptr, etype, x_ptr, stream=None):
        _check(self._lib.fr_closure_features(self._h, C.c_void_p(u_ptr), _etype(etype), C.c_void_p(x_ptr),
                                             _sp(stream)))

    def closure_sample(self, hi, u_hi_ptr, etype, inv_scale=None, x_ptr=None, t_ptr=None, ss_ptr=None,
                       u_lo_ptr=None, stream=None):
        """Features/targets of this (low-order) context from hi's state
        (targets against the RHS of u_lo, or of the projection of u_hi)."""
        isc = None if inv_scale is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(inv_scale, dtype=np.float64), (NVARS,)))
        _check(self._lib.fr_closure_sample(hi._h, self._h, C.c_void_p(u_hi_ptr),
                                           C.c_void_p(u_lo_ptr) if u_lo_ptr else None, _etype(etype),
                                           _dptr(isc) if isc is not None else None,
                                           C.c_void_p(x_ptr) if x_ptr else None,
                                           C.c_void_p(t_ptr) if t_ptr else None,
                                           C.c_void_p(ss_ptr) if ss_ptr else None, _sp(stream)))

    def closure_set(self, etype, params_ptr, nh=128, out_scale=1.0):
        """Attach (params_ptr: device FP32) or detach (None) a network;
        out_scale: one value or one per conserved variable."""
        sc = np.ascontiguousarray(np.broadcast_to(np.asarray(out_scale, dtype=np.float64), (NVARS,)))
        _check(self._lib.fr_closure_set(self._h, _etype(etype), C.c_void_p(params_ptr) if params_ptr else None,
                                        int(nh), _dptr(sc)))

    def reduce(self, stream=None, check=True):
        out = np.empty(7, dtype=np.float64)
        rc = self._lib.fr_reduce(self._h, _dptr(out), C.c_void_p(stream) if stream else None)
        if rc == FR_ERR_NONFINITE and not check:
            return out
        _check(rc)
        return out


    def selftest_wait_timeout(self, stream=None):
        """fr_selftest_wait_timeout (tensor-core precisions)."""
        _check(self._lib.fr_selftest_wait_timeout(self._h, C.c_void_p(stream) if stream else None))

    def diagnostics(self, stream=None):
        """fr_diagnostics: (dKE/dt, inviscid wall force (3,), viscous wall
        force (3,)) of the solution register."""
        out = np.empty(7, dtype=np.float64)
        _check(self._lib.fr_diagnostics(self._h, _dptr(out), C.c_void_p(stream) if stream else None))
        return float(out[0]), out[1:4].copy(), out[4:7].copy()


class Batch:
    """fr_batch: many independent problems advanced with grouped launches."""

    INFO = ("nprob", "ndof", "launches_batched", "launches_per_problem", "rc_m0", "rc_grad",
            "rc_m0grad", "rc_div", "grid_gemm", "grid_div", "grid_flux", "grid_face", "grid_stage",
            "launches_grouped")

    def __init__(self, meshes, orders, **params):
        lib = load()
        self._lib = lib
        prm = default_params(**params)
        keep = []
        arr = (FRMesh * len(meshes))(*[_fr_mesh(m, keep) for m in meshes])
        ords = (C.c_int * len(orders))(*[int(o) for o in orders])
        p = _fr_params(prm)
        h = C.c_void_p()
        _check(lib.fr_batch_create(len(meshes), arr, ords, C.byref(p), C.byref(h)))
        self._h = h
        self.problems = []
        for i in range(len(meshes)):
            ch = C.c_void_p()
            _check(lib.fr_batch_problem(h, i, C.byref(ch)))
            self.problems.append(Context(None, 0, _handle=ch, _owner=self, **params))

    def info(self):
        out = (C.c_int64 * len(self.INFO))()
        _check(self._lib.fr_batch_info(self._h, out))
        return dict(zip(self.INFO, list(out)))

    def tune(self, stream=None):
        _check(self._lib.fr_batch_tune(self._h, C.c_void_p(stream) if stream else None))

    def step(self, dt, nsteps=1, batched=True, stream=None):
        """fr_batch_step: batched True or 1 = one persistent launch per RK
        stage, 2 = grouped launches per class, False or 0 = each problem's
        own launches."""
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self.problems),)))
        mode = int(batched) if not isinstance(batched, bool) else (1 if batched else 0)
        _check(self._lib.fr_batch_step(self._h, _dptr(dts), int(nsteps), mode,
                                       C.c_void_p(stream) if stream else None))

    def check(self, stream=None):
        """fr_batch_check: raises FRError (FR_ERR_TIMEOUT) after a barrier
        wait of the persistent stage kernel ran out."""
        _check(self._lib.fr_batch_check(self._h, C.c_void_p(stream) if stream else None))

    def selftest_wait_timeout(self, stream=None):
        """fr_batch_selftest_wait_timeout (bounded-wait self-test)."""
        _check(self._lib.fr_batch_selftest_wait_timeout(self._h, C.c_void_p(stream) if stream else None))

    def close(self):
        if getattr(self, "_h", None):
            for c in self.problems:
                c._h = None
            self._lib.fr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# partitioned meshes
# ---------------------------------------------------------------------------
def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def partition(mesh, nparts, weights=None):
    """fr_partition (host only): partition of every element, public order."""
    lib = load()
    keep = []
    m = _fr_mesh(mesh, keep)
    n = m.n_tet + m.n_pri + m.n_hex
    out = np.empty(n, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    _check(lib.fr_partition(C.byref(m), int(nparts), _dptr(w) if w is not None else None, _i32p(out)))
    return out


def part_plan(mesh, order, part, rank):
    """fr_part_plan (host only): (counts, send_pts, halo_pts) of one rank."""
    lib = load()
    keep = []
    m = _fr_mesh(mesh, keep)
    part = np.ascontiguousarray(part, dtype=np.int32)
    nparts = int(part.max()) + 1
    counts = np.zeros(nparts, dtype=np.int64)
    _check(lib.fr_part_plan(C.byref(m), int(order), nparts, _i32p(part), int(rank),
                            counts.ctypes.data_as(C.POINTER(C.c_int64)), None, None))
    tot = int(counts.sum())
    send = np.zeros((tot, 3), dtype=np.int32)
    halo = np.zeros((tot, 3), dtype=np.int32)
    _check(lib.fr_part_plan(C.byref(m), int(order), nparts, _i32p(part), int(rank),
                            counts.ctypes.data_as(C.POINTER(C.c_int64)), _i32p(send), _i32p(halo)))
    return counts, send, halo


class PartContext:
    """One fr_part: a mesh split into partitions on the current GPU."""

    def __init__(self, mesh, order, nparts, part=None, **params):
        lib = load()
        self._lib = lib
        prm = default_params(**params)
        self.params = prm
        keep = []
        m = _fr_mesh(mesh, keep)
        p = _fr_params(prm)
        h = C.c_void_p()
        pa = None if part is None else np.ascontiguousarray(part, dtype=np.int32)
        _check(lib.fr_part_create(C.byref(m), int(order), C.byref(p), int(nparts),
                                  _i32p(pa) if pa is not None else None, C.byref(h)))
        self._h = h
        self.nparts = int(nparts)
        info = np.zeros(4 * self.nparts, dtype=np.int64)
        _check(lib.fr_part_info(h, info.ctypes.data_as(C.POINTER(C.c_int64))))
        self.info = info.reshape(self.nparts, 4)   # tets, prisms, hexes, halo slots
        # the unpartitioned public layout's length
        self.ndof = int(sum(self.info[:, t].sum() * 5 * _nupts(t, order) for t in range(3)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fr_part_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, u, stream=None):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(self._lib.fr_part_set_state(self._h, _dptr(u), C.c_void_p(stream) if stream else None))

    def get_state(self, stream=None):
        out = np.empty(self.ndof, dtype=np.float64)
        _check(self._lib.fr_part_get_state(self._h, _dptr(out), C.c_void_p(stream) if stream else None))
        return out

    def rhs(self, u_ptr, r_ptr, stream=None):
        _check(self._lib.fr_part_rhs(self._h, C.c_void_p(u_ptr), C.c_void_p(r_ptr),
                                     C.c_void_p(stream) if stream else None))

    def step(self, dt, nsteps=1, stream=None):
        _check(self._lib.fr_part_step(self._h, float(dt), int(nsteps), C.c_void_p(stream) if stream else None))

    def reduce(self, stream=None):
        out = np.empty(7, dtype=np.float64)
        _check(self._lib.fr_part_reduce(self._h, _dptr(out), C.c_void_p(stream) if stream else None))
        return out

    def launches(self):
        n = C.c_int64()
        _check(self._lib.fr_part_launches(self._h, C.byref(n)))
        return n.value


def _nupts(etype, p):
    return {0: (p + 1) * (p + 2) * (p + 3) // 6, 1: (p + 1) ** 2 * (p + 2) // 2, 2: (p + 1) ** 3}[etype]


def debug_fail_alloc(k):
    """fr_debug_fail_alloc: the k-th device allocation from now fails (0: none)."""
    _check(load().fr_debug_fail_alloc(int(k)))


def debug_alloc_stats():
    """(allocations attempted since the last debug_fail_alloc, live allocations)."""
    out = (C.c_int64 * 2)()
    _check(load().fr_debug_alloc_stats(out))
    return int(out[0]), int(out[1])
