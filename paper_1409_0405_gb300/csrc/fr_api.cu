// C ABI of the FR engine (declared in include/fr.h): context creation,
// device memory, and the RHS / RK4 launch sequences.
//
// One RHS evaluation (Sec. 2.1: operator applications C <- c1 A B + c2 C
// interleaved with point-wise kernels), per element type t:
//   UF_t  = M0 U_t                                   (Table 2's M0)
//   NS:   DUF = C - u_f at every flux point          (common solution)
//         GU_t = (1/J) S^T [D | n^(x)M3] [U_t; DUF_t] (corrected gradient;
//                in the FP32-storage modes the operator kernel stores the
//                reference gradient and the flux kernel applies S^T/J)
//         GUF_t = M0 GU_t
//   FT_t  = S (F_inv - F_vis - F_inf) at solution points
//   FC    = (common normal flux - F_inf.n) |S^T n^| at every flux point
//   R_t   = -(1/J) [M1 - M3 M2 | M3] [FT_t; FC_t]   (+ fused RK4 update;
//           on the tensor cores a streaming pass scales and updates)
// Element types t: tets, prisms, hexes.
// The stage input Us is stored centred, u - u_inf (u_inf the far-field
// conserved state): M0 reproduces and D annihilates constants, so this is
// exact, and the long operator sums then run over small numbers.
// Internal layout of a state-like matrix: [point][variable][element], the
// element index padded to np_t (a multiple of 32) and fastest, so every
// operator application is a plain row-major GEMM over V*np_t columns.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"
#include "fr_kernels.h"

namespace fr {
namespace api {

thread_local std::string g_last_error;

int set_err(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

}  // namespace api
}  // namespace fr

using namespace fr;
using namespace fr::api;

namespace fr {
namespace api {

// Every device allocation of the engine goes through dev_malloc/dev_free,
// which count the live allocations and can be told to fail the k-th
// allocation from now (fr_debug_fail_alloc), so that tests reach every
// FR_ERR_NOMEM path of the set-up code and check that nothing leaks.
std::atomic<int64_t> g_fail_at{0}, g_alloc_seen{0}, g_live{0};

cudaError_t dev_malloc(void **p, size_t bytes) {
    const int64_t k = ++g_alloc_seen;
    if (g_fail_at.load() > 0 && k == g_fail_at.load()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live;
    return e;
}

void dev_free(void *p) {
    if (!p) return;
    if (cudaFree(p) == cudaSuccess) --g_live;
}

constexpr int64_t kPad = 32;
constexpr int kDiagBlocks = 304;  // blocks of the diagnostics reductions (2 per SM)

template <class T>
int dev_alloc(fr_ctx *c, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return FR_OK;
    void *q = nullptr;
    cudaError_t e = dev_malloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(FR_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    e = cudaMemset(q, 0, count * sizeof(T));
    if (e != cudaSuccess) return set_err(FR_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    *p = (T *)q;
    return FR_OK;
}

int dev_alloc_bytes(fr_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return FR_OK;
    cudaError_t e = dev_malloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(FR_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    e = cudaMemset(*p, 0, bytes);
    if (e != cudaSuccess) return set_err(FR_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    return FR_OK;
}

template <class T>
int upload(fr_ctx *c, T **p, const std::vector<T> &h) {
    int rc = dev_alloc(c, p, h.size());
    if (rc) return rc;
    if (h.empty()) return FR_OK;
    cudaError_t e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_err(FR_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    return FR_OK;
}

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FR_OK;
    return set_err(FR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Phys phys_of(const fr_ctx *c) {
    Phys ph{};
    ph.gamma = c->prm.gamma;
    ph.mu = c->prm.mu;
    ph.prandtl = c->prm.prandtl;
    ph.beta = c->prm.ldg_beta;
    ph.tau = c->prm.ldg_tau;
    ph.rho_inf = c->prm.rho_inf;
    for (int k = 0; k < 3; ++k) ph.vinf[k] = c->prm.vel_inf[k];
    ph.p_inf = c->prm.p_inf;
    ph.t_wall = c->prm.t_wall;
    ph.viscous = c->prm.viscous;
    {
        const double r = c->prm.rho_inf, g = c->prm.gamma, pinf = c->prm.p_inf;
        const double *v = c->prm.vel_inf;
        const double E = pinf / (g - 1.0) + 0.5 * r * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int m = 0; m < 3; ++m) {
            ph.fref[0][m] = r * v[m];
            for (int a = 0; a < 3; ++a) ph.fref[1 + a][m] = r * v[a] * v[m] + (a == m ? pinf : 0.0);
            ph.fref[4][m] = (E + pinf) * v[m];
        }
        ph.uref[0] = r;
        for (int a = 0; a < 3; ++a) ph.uref[1 + a] = r * v[a];
        ph.uref[4] = E;
    }
    return ph;
}

template <typename T>
FieldsT<T> fields_of(const fr_ctx *c) {
    FieldsT<T> F{};
    for (int t = 0; t < NT; ++t) {
        F.UF[t] = (const T *)c->T[t].UF;
        F.DUF[t] = (T *)c->T[t].DUF;
        F.GUF[t] = (const T *)c->T[t].GUF;
        F.FC[t] = (T *)c->T[t].FC;
        F.np[t] = c->T[t].np;
    }
    F.UF[HALO] = (const T *)c->UF_h;
    F.DUF[HALO] = (T *)c->DUF_h;
    F.GUF[HALO] = (const T *)c->GUF_h;
    F.FC[HALO] = (T *)c->FC_h;
    F.np[HALO] = c->nhalo_p;
    return F;
}

Pairs pairs_of(const fr_ctx *c) {
    return Pairs{c->npairs, c->pcode, c->ea,    c->eb,     c->nrm,
                 c->maga,   c->magb,  c->nrm_f, c->maga_f, c->magb_f};
}

Bnd bnd_of(const fr_ctx *c) {
    return Bnd{c->nbnd, c->bt, c->bf, c->be, c->btag, c->bn, c->bmag, c->bn_f, c->bmag_f};
}


cudaEvent_t next_event(fr_ctx *c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// One RHS evaluation on the stage input `in[t]`; the final operator
// application either stores R (rk == nullptr) or applies the RK update.

// Arguments of the four operator applications of one element type (shared
// by the per-context launches below and the grouped launches of the batch).
template <typename T>
GemmArgsT<T> args_m0(const fr_ctx *c, int t, const T *in) {
    const DevType &D = c->T[t];
    const Phys ph = phys_of(c);
    GemmArgsT<T> g;
    g.M = D.nf;
    g.N = (int64_t)NV * D.np;
    g.K1 = D.nu;
    g.A = (const T *)D.M0_t;
    g.B1 = in;
    g.ldb1 = g.N;
    g.C = (T *)D.UF;
    g.ldc = g.N;
    g.mode = GEMM_STORE;
    g.np = D.np;
    g.add_ref = 1;  // the stage input is centred; add u_inf back
    for (int v = 0; v < NV; ++v) g.uref[v] = ph.uref[v];
    return g;
}

template <typename T>
GemmArgsT<T> args_grad(const fr_ctx *c, int t, const T *in) {
    const DevType &D = c->T[t];
    GemmArgsT<T> g;
    g.M = 3 * D.nu;
    g.N = (int64_t)NV * D.np;
    g.K1 = D.nu;
    g.K2 = D.nf;
    g.A = (const T *)D.AGRAD_t;
    g.B1 = in;
    g.ldb1 = g.N;
    g.B2 = (const T *)D.DUF;
    g.ldb2 = g.N;
    g.C = (T *)D.GU;  // [nu][3][V][np]: row (j, m), N columns
    g.ldc = g.N;
    g.mode = GEMM_GRAD;
    g.np = D.np;
    g.invJ = (const T *)D.invJ_t;
    g.S = (const T *)D.S_t;
    return g;
}

template <typename T>
GemmArgsT<T> args_m0grad(const fr_ctx *c, int t) {
    const DevType &D = c->T[t];
    GemmArgsT<T> h;
    h.M = D.nf;
    h.N = 3 * (int64_t)NV * D.np;
    h.K1 = D.nu;
    h.A = (const T *)D.M0_t;
    h.B1 = (const T *)D.GU;
    h.ldb1 = h.N;
    h.C = (T *)D.GUF;
    h.ldc = h.N;
    h.np = D.np;  // element stride of the columns (15 blocks of np)
    h.mode = GEMM_STORE;
    return h;
}

template <typename T>
GemmArgsT<T> args_div(const fr_ctx *c, int t, const RKStage *rk) {
    const DevType &D = c->T[t];
    const Phys ph = phys_of(c);
    GemmArgsT<T> g;
    g.M = D.nu;
    g.N = (int64_t)NV * D.np;
    g.K1 = 3 * D.nu;
    g.K2 = D.nf;
    g.A = (const T *)D.ADIV_t;
    g.B1 = (const T *)D.FT;
    g.ldb1 = g.N;
    g.B2 = (const T *)D.FC;
    g.ldb2 = g.N;
    g.ldc = g.N;
    g.np = D.np;
    g.invJ = (const T *)D.invJ_t;
    g.geo_elem = D.geo_elem;
    g.rfs = D.Rfs;
    for (int v = 0; v < NV; ++v) g.uref[v] = ph.uref[v];
    if (rk) {
        g.mode = GEMM_DIV_RK;
        g.U = D.U;
        g.Uacc = D.Uacc;
        g.Us = (T *)D.Us;
        g.Us0 = (T *)D.Us0;  // FP32 storage: stage inputs formed in T
        g.c_acc = rk->c_acc;
        g.c_stage = rk->c_stage;
        g.rk_first = rk->first;
        g.rk_last = rk->last;
    } else {
        g.mode = GEMM_DIV;
        g.C = (T *)D.R;
    }
    return g;
}

// the dense arguments plus the chunk-compressed operator, if there is one
template <typename T>
GemmArgsT<T> with_sparse(const fr_ctx *c, int t, int which, const GemmArgsT<T> &g) {
    GemmArgsT<T> h = g;
    const DevType &D = c->T[t];
    if (D.sp_rc[which]) {
        h.sp_rc = D.sp_rc[which];
        h.sp_lmax = D.sp_lmax[which];
        h.sp_off = D.sp_off[which];
        h.sp_cols = D.sp_cols[which];
        h.sp_vals = (const T *)D.sp_vals[which];
        h.sp_masked = D.sp_masked[which];
    }
    return h;
}

template <>
cudaError_t op_gemm<double>(fr_ctx *c, int t, int which, const GemmArgsT<double> &g, cudaStream_t s) {
    const X64Operator &op = c->T[t].x64[which];
    if (op.img) {
        // the state operand's column exponents, then the exact-split product
        cudaError_t e = launch_colexp(g.B1, g.ldb1, g.K1, g.B2, g.ldb2, g.K2, g.N, c->x64_E, s);
        if (e == cudaSuccess) e = launch_gemm_x64(g, op, c->x64_E, c->tc_err, s);
        ++c->launches;  // the pre-pass
        return e;
    }
    return launch_gemm<double>(with_sparse<double>(c, t, which, g), s);
}

template <>
cudaError_t op_gemm<float>(fr_ctx *c, int t, int which, const GemmArgsT<float> &g, cudaStream_t s) {
    if (is_tc(c)) {
        const DevType &D = c->T[t];
        const int r0 = D.tc_split[which];
        if (!r0) return launch_gemm_tc(g, D.tc[which], c->tc_err, s);
        // row blocks of a split operator (store epilogue): rows [0, r0) and
        // [r0, M) of C from their own images
        if (g.mode != GEMM_STORE) return cudaErrorInvalidValue;
        GemmArgsT<float> g1 = g, g2 = g;
        g1.M = r0;
        g2.M = g.M - r0;
        g2.C = g.C + (int64_t)r0 * g.ldc;
        cudaError_t e = launch_gemm_tc(g1, D.tc[which], c->tc_err, s);
        if (e == cudaSuccess) e = launch_gemm_tc(g2, D.tc2[which], c->tc_err, s);
        ++c->launches;  // the second launch
        return e;
    }
    const F32Operator &op = c->T[t].f32op[which];
    if (op.img && g.mode == GEMM_STORE) {
        const cudaError_t e = launch_gemm_f32(g, op, c->tc_err, s);
        if (e != cudaErrorInvalidValue) return e;
        cudaGetLastError();  // a layout the streamed kernel does not take: the chunk-staged kernel
    }
    return launch_gemm<float>(with_sparse<float>(c, t, which, g), s);
}

// FR_ERR_TIMEOUT if a tensor-core kernel gave up a wait (synchronises)
int check_tc(fr_ctx *c) {
    if (!(is_f32(c) || is_x64(c)) || !c->tc_err) return FR_OK;
    int h = 0;
    int rc = cuda_check(cudaMemcpy(&h, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost), "tensor-core status");
    if (rc) return rc;
    if (h) return set_err(FR_ERR_TIMEOUT, "a tensor-core operator kernel gave up a bounded wait (code " +
                                              std::to_string(h) + ")");
    return FR_OK;
}

// The RHS in three phases, between which a partitioned mesh exchanges its
// halos: (1) interpolation to the flux points; (2) Navier-Stokes only:
// common solution, corrected gradient, gradient at the flux points; (3)
// transformed flux, common normal flux, divergence (+ RK update).
template <typename T>
int phase_interp(fr_ctx *c, T *const in[NT], cudaStream_t s) {
    int rc;
    // 1. interpolate to flux points
    for (int t = 0; t < NT; ++t) {
        if (!c->T[t].present) continue;
        const GemmArgsT<T> g = args_m0<T>(c, t, in[t]);
        if ((rc = cuda_check(launch(c, ktag(K_M0, t), s, [&] { return op_gemm<T>(c, t, 0, g, s); }), "gemm M0"))) return rc;
    }
    return FR_OK;
}

template <typename T>
int phase_grad(fr_ctx *c, T *const in[NT], cudaStream_t s) {
    const Phys ph = phys_of(c);
    const FieldsT<T> F = fields_of<T>(c);
    int rc;
    if (c->prm.viscous) {
        // 2. common solution and jumps
        if ((rc = cuda_check(launch(c, K_COMMON_SOL, s,
                                    [&] { return launch_common_solution<T>(pairs_of(c), bnd_of(c), F, ph, s); }),
                             "common solution")))
            return rc;
        // 3. corrected physical gradient; 4. gradient at flux points.  In
        // the FP32-storage modes the operator kernel stores the reference
        // gradient and the flux kernel (5.), which loads the point's
        // geometry anyway, forms the physical gradient in place before M0 is
        // applied to it (in the operator kernel's epilogue those loads would
        // repeat for every variable and stall it; the FP64 kernel is bound by
        // its FMAs and keeps the fused epilogue)
        const bool tc = is_f32(c);
        for (int t = 0; t < NT; ++t) {
            if (!c->T[t].present) continue;
            GemmArgsT<T> g = args_grad<T>(c, t, in[t]);
            if (tc) g.mode = GEMM_STORE;
            if ((rc = cuda_check(launch(c, ktag(K_GRAD, t), s, [&] { return op_gemm<T>(c, t, 1, g, s); }), "gemm grad")))
                return rc;
            if (tc) {
                DevType &D = c->T[t];
                if ((rc = cuda_check(launch(c, ktag(K_FLUX, t), s,
                                            [&] {
                                                return launch_flux<T>(D.nu, D.ne, D.np, in[t], (T *)D.GU,
                                                                      (const T *)D.S_t, (const T *)D.invJ_t,
                                                                      (T *)D.FT, ph, s, D.geo_elem ? 0 : 1);
                                            }),
                                     "flux")))
                    return rc;
            }
            const GemmArgsT<T> h = args_m0grad<T>(c, t);
            if ((rc = cuda_check(launch(c, ktag(K_M0_GRAD, t), s, [&] { return op_gemm<T>(c, t, 0, h, s); }), "gemm M0 grad")))
                return rc;
        }
    }
    return FR_OK;
}

template <typename T>
int front_stages(fr_ctx *c, T *const in[NT], cudaStream_t s) {
    int rc = phase_interp<T>(c, in, s);
    return rc ? rc : phase_grad<T>(c, in, s);
}

template <typename T>
int phase_div(fr_ctx *c, T *const in[NT], const RKStage *rk, cudaStream_t s) {
    const Phys ph = phys_of(c);
    const FieldsT<T> F = fields_of<T>(c);
    int rc;
    // 5. transformed flux at solution points (done by front_stages for
    // Navier-Stokes in the FP32-storage modes)
    for (int t = 0; t < NT && !(is_f32(c) && c->prm.viscous); ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch(c, ktag(K_FLUX, t), s,
                                    [&] {
                                        return launch_flux<T>(D.nu, D.ne, D.np, in[t], (T *)D.GU, (const T *)D.S_t,
                                                              (const T *)nullptr, (T *)D.FT, ph, s,
                                                              D.geo_elem ? 0 : 1);
                                    }),
                             "flux")))
            return rc;
    }
    // 6. common normal flux at every flux point
    if ((rc = cuda_check(launch(c, K_COMMON_FLUX, s,
                                [&] { return launch_common_flux<T>(pairs_of(c), bnd_of(c), F, ph, s); }),
                         "common flux")))
        return rc;
    // 7. divergence plus correction; with the learned closure on, the
    // network's correction is added by the epilogue with the reference term
    // On the tensor cores an RK stage's operator kernel stores the raw
    // product and a streaming pass scales it by -1/J, adds the
    // reference/closure term and applies the RK update, forming the next
    // stage input in FP32 (per-point loads and the FP64 register arithmetic
    // would otherwise stall the kernel's epilogue on the FP64 pipe).  The
    // FP32 mode does the same with its streamed kernel (fr_gemm_f32.cu); its
    // RK update is the fused epilogue's arithmetic, which the batched
    // launches (chunk-staged kernel, fused epilogue) reproduce bit for bit.
    const bool split_rk = rk && is_f32(c);
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        GemmArgsT<T> g = args_div<T>(c, t, split_rk ? nullptr : rk);
        if (D.cl_on) {
            if ((rc = closure_apply<T>(c, t, in[t], s))) return rc;
            g.rfs = D.cl_add;
        }
        const double *rfs = g.rfs;
        if (split_rk) g.mode = GEMM_STORE;
        if ((rc = cuda_check(launch(c, ktag(K_DIV, t), s, [&] { return op_gemm<T>(c, t, 2, g, s); }), "gemm div"))) return rc;
        if (split_rk &&
            (rc = cuda_check(launch(c, K_DIV, s,
                                    [&] {
                                        return launch_rk_update<T>(D.nu, D.np, (const T *)D.R, D.U, D.Uacc, (T *)D.Us,
                                                                   ph.uref, rk->c_acc, rk->c_stage, rk->first,
                                                                   rk->last, (const T *)D.invJ_t, rfs, (T *)D.Us0, s,
                                                                   D.geo_elem ? 0 : 1);
                                    }),
                             "RK update")))
            return rc;
    }
    return FR_OK;
}

template <typename T>
int rhs_internal(fr_ctx *c, T *const in[NT], const RKStage *rk, cudaStream_t s) {
    int rc = front_stages<T>(c, in, s);
    return rc ? rc : phase_div<T>(c, in, rk, s);
}

int num_sms(int device) {
    static std::atomic<int> cache[64];
    if (device < 0 || device >= 64) device = 0;
    int n = cache[device].load();
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    cache[device] = n;
    return n;
}

int step_guard(const fr_ctx *c) {
    if (c->nf_host && *(volatile const int *)c->nf_host)
        return set_err(FR_ERR_NONFINITE,
                       "an earlier step left a non-finite or non-physical state (fr_set_state clears this)");
    return FR_OK;
}

int step_check(fr_ctx *c, cudaStream_t s) {
    if (!c->nf_dev) return FR_OK;
    // enough CTAs to keep the loads of a streaming read in flight
    const int nb = 16 * num_sms(c->device);
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        int rc = cuda_check(launch(c, K_CHECK, s,
                                   [&] {
                                       return launch_state_check(D.nu, D.ne, D.np, D.U, c->prm.gamma, c->nf_dev, nb,
                                                                 s);
                                   }),
                            "state check");
        if (rc) return rc;
    }
    return FR_OK;
}

int64_t ndof_of(const fr_ctx *c) {
    int64_t n = 0;
    for (int t = 0; t < NT; ++t)
        if (c->T[t].present) n += c->T[t].ne * NV * c->T[t].nu;
    return n;
}

int check_params(int order, const fr_params *prm) {
    if (!prm) return set_err(FR_ERR_ARG, "null params");
    if (order < 1 || order > 4) return set_err(FR_ERR_ARG, "order must be in 1..4");
    if (prm->precision < FR_FP64 || prm->precision > FR_FP64S)
        return set_err(FR_ERR_UNSUPPORTED, "precision must be FR_FP64, FR_FP32, FR_BF16X3, FR_TF32X3 or FR_FP64S");
    if (!(prm->gamma > 1.0) || prm->mu < 0.0 || (prm->viscous && !(prm->prandtl > 0.0)))
        return set_err(FR_ERR_ARG, "invalid gas parameters");
    return FR_OK;
}

int host_setup(const fr_mesh *mesh, int order, HostSetup &h) {
    if (!mesh) return set_err(FR_ERR_ARG, "null mesh");
    if (order < 1 || order > 4) return set_err(FR_ERR_ARG, "order must be in 1..4");
    if (mesh->n_nodes <= 0 || !mesh->xyz) return set_err(FR_ERR_ARG, "mesh has no nodes");
    if (mesh->n_tet < 0 || mesh->n_pri < 0 || mesh->n_hex < 0 || mesh->n_bface < 0)
        return set_err(FR_ERR_ARG, "negative element or face count");
    if (mesh->n_tet + mesh->n_pri + mesh->n_hex == 0) return set_err(FR_ERR_ARG, "mesh has no elements");
    if ((mesh->n_tet && !mesh->tet) || (mesh->n_pri && !mesh->pri) || (mesh->n_hex && !mesh->hex) ||
        (mesh->n_bface && !mesh->bface))
        return set_err(FR_ERR_ARG, "null connectivity array");
    if (mesh->n_tet > (1LL << 30) || mesh->n_pri > (1LL << 30) || mesh->n_hex > (1LL << 30))
        return set_err(FR_ERR_ARG, "element count too large");
    if (order < 1 || order > 4) return set_err(FR_ERR_ARG, "order must be in 1..4");
    std::string err;
    const int64_t ne_in[NT] = {mesh->n_tet, mesh->n_pri, mesh->n_hex};
    for (int t = 0; t < NT; ++t) {
        if (ne_in[t] == 0) continue;  // operators only for the types present
        int rc = build_ref_ops(t, order, h.ops[t], err);
        if (rc) return set_err(rc, err);
    }
    int rc = build_geometry(mesh, h.ops, h.geo, err);
    if (rc) return set_err(rc, err);
    rc = build_faces(mesh, h.ops, h.geo, h.faces, err);
    if (rc) return set_err(rc, err);
    return FR_OK;
}

// Device state of a context from its host set-up: per-type geometry geo,
// the interface pairs and boundary points of `faces`, and nhalo halo slots
// (a partition of a partitioned mesh; 0 otherwise).  ops holds the
// operators of every type present in geo.
int device_setup(fr_ctx *c, int order, const fr_params *prm, const RefOps ops[NT], const TypeGeo geo[NT],
                 const Faces &faces, int64_t nhalo) {
    c->prm = *prm;
    c->order = order;
    int rc;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        return set_err(FR_ERR_CUDA, "no usable CUDA device");
    }
    const int64_t ne[NT] = {geo[0].ne, geo[1].ne, geo[2].ne};
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        D.present = ne[t] > 0;
        if (!D.present) continue;
        D.ne = ne[t];
        D.np = (ne[t] + kPad - 1) / kPad * kPad;
        D.nu = ops[t].nu;
        D.nf = ops[t].nf;
        const size_t su = (size_t)D.nu * NV * D.np, sf = (size_t)D.nf * NV * D.np;
        const size_t es = f32_storage(prm->precision) ? sizeof(float) : sizeof(double);
        if ((rc = dev_alloc(c, &D.U, su)) || (rc = dev_alloc(c, &D.Uacc, su)) ||
            (rc = dev_alloc_bytes(c, &D.Us, su * es)) || (rc = dev_alloc_bytes(c, &D.R, su * es)) ||
            (rc = dev_alloc_bytes(c, &D.UF, sf * es)) || (rc = dev_alloc_bytes(c, &D.FC, sf * es)) ||
            (rc = dev_alloc_bytes(c, &D.FT, 3 * su * es)))
            return rc;
        if (f32_storage(prm->precision) && (rc = dev_alloc_bytes(c, &D.Us0, su * es))) return rc;
        if (prm->viscous) {
            if ((rc = dev_alloc_bytes(c, &D.DUF, sf * es)) || (rc = dev_alloc_bytes(c, &D.GU, 3 * su * es)) ||
                (rc = dev_alloc_bytes(c, &D.GUF, 3 * sf * es)))
                return rc;
        }
        // geometry in the internal layout
        std::vector<double> S((size_t)D.nu * 9 * D.np, 0.0), iJ((size_t)D.nu * D.np, 0.0),
            wJ((size_t)D.nu * D.np, 0.0);
        const TypeGeo &G = geo[t];
        for (int64_t e = 0; e < D.ne; ++e)
            for (int j = 0; j < D.nu; ++j) {
                const size_t ij = (size_t)e * D.nu + j;
                for (int k = 0; k < 9; ++k) S[((size_t)j * 9 + k) * D.np + e] = G.S[9 * ij + k];
                iJ[(size_t)j * D.np + e] = 1.0 / G.J[ij];
                wJ[(size_t)j * D.np + e] = ops[t].W[j] * G.J[ij];
            }
        if ((rc = upload(c, &D.S, S)) || (rc = upload(c, &D.invJ, iJ)) || (rc = upload(c, &D.wJ, wJ)) ||
            (rc = upload(c, &D.M0, ops[t].M0)) || (rc = upload(c, &D.AGRAD, ops[t].AGRAD)) ||
            (rc = upload(c, &D.ADIV, ops[t].ADIV)))
            return rc;
        if (prm->precision == FR_BF16X3 || prm->precision == FR_TF32X3) {
            // the three operators packed for the tensor cores
            const std::vector<double> *opv[3] = {&ops[t].M0, &ops[t].AGRAD, &ops[t].ADIV};
            const int om[3] = {D.nf, 3 * D.nu, D.nu}, ok1[3] = {D.nu, D.nu, 3 * D.nu}, ok2[3] = {0, D.nf, D.nf};
            auto pack = [&](TcOperator &op, const double *A, int M, int K1, int K2) -> int {
                op.tf32 = prm->precision == FR_TF32X3;
                int r;
                if (op.tf32) {
                    std::vector<uint32_t> img;
                    tc_pack_tf32(A, M, K1, K2, img, op.Nmma, op.K1pad, op.Kpad);
                    uint32_t *dimg = nullptr;
                    if ((r = upload(c, &dimg, img))) return r;
                    op.img = (const uint8_t *)dimg;
                } else {
                    std::vector<uint16_t> img;
                    tc_pack(A, M, K1, K2, img, op.Nmma, op.K1pad, op.Kpad);
                    uint16_t *dimg = nullptr;
                    if ((r = upload(c, &dimg, img))) return r;
                    op.img = (const uint8_t *)dimg;
                }
                op.M = M;
                op.K = K1 + K2;
                if (op.Nmma > 256 || tc_stages(op) < 2)
                    return set_err(FR_ERR_UNSUPPORTED, "operator too large for the tensor-core kernel");
                return FR_OK;
            };
            for (int w = 0; w < 3; ++w) {
                const int K = ok1[w] + ok2[w];
                if (om[w] <= 256) {
                    if ((rc = pack(D.tc[w], opv[w]->data(), om[w], ok1[w], ok2[w]))) return rc;
                    continue;
                }
                // two row blocks (store epilogue only: the gradient of an
                // RK step); the first a multiple of 16 rows
                const int r0 = ((om[w] + 1) / 2 + 15) / 16 * 16;
                if ((rc = pack(D.tc[w], opv[w]->data(), r0, ok1[w], ok2[w])) ||
                    (rc = pack(D.tc2[w], opv[w]->data() + (size_t)r0 * K, om[w] - r0, ok1[w], ok2[w])))
                    return rc;
                D.tc_split[w] = r0;
            }
        }
        if (prm->precision == FR_FP64 || prm->precision == FR_FP32 || prm->precision == FR_FP64S) {
            // the operators' exact zeros skipped chunk by chunk (prisms)
            const std::vector<double> *opv[3] = {&ops[t].M0, &ops[t].AGRAD, &ops[t].ADIV};
            const int om[3] = {D.nf, 3 * D.nu, D.nu}, ok1[3] = {D.nu, D.nu, 3 * D.nu}, ok2[3] = {0, D.nf, D.nf};
            for (int w = 0; w < 3; ++w) {
                // FP64 (FMA-bound): exactly the non-zero FMAs, chunk by chunk
                // of 3 rows; FP32 (bound by loads as much as by FMAs): the
                // chunk size with the fewest FMAs over whole column unions
                SparseOp sp;
                const bool masked = !f32_storage(prm->precision);
                if (masked ? !sparse_pack_masked(opv[w]->data(), om[w], ok1[w], ok2[w], sp)
                           : !sparse_pack(opv[w]->data(), om[w], ok1[w], ok2[w], w == 1, sp))
                    continue;
                D.sp_masked[w] = masked;
                if ((rc = upload(c, &D.sp_off[w], sp.off)) || (rc = upload(c, &D.sp_cols[w], sp.cols))) return rc;
                if (prm->precision == FR_FP32) {
                    std::vector<float> vf(sp.vals.begin(), sp.vals.end());
                    float *dv = nullptr;
                    if ((rc = upload(c, &dv, vf))) return rc;
                    D.sp_vals[w] = dv;
                } else {
                    double *dv = nullptr;
                    if ((rc = upload(c, &dv, sp.vals))) return rc;
                    D.sp_vals[w] = dv;
                }
                D.sp_rc[w] = sp.rc;
                D.sp_lmax[w] = sp.lmax;
            }
        }
        if (prm->precision == FR_FP32) {
            // the streamed FP32 kernel's images (fr_gemm_f32.cu)
            const std::vector<double> *opv[3] = {&ops[t].M0, &ops[t].AGRAD, &ops[t].ADIV};
            const int om[3] = {D.nf, 3 * D.nu, D.nu}, ok1[3] = {D.nu, D.nu, 3 * D.nu}, ok2[3] = {0, D.nf, D.nf};
            for (int w = 0; w < 3; ++w) {
                std::vector<int> perm;
                if (w == 1) {  // image row d nu + j holds gradient row 3 j + d
                    perm.resize((size_t)om[1]);
                    for (int d = 0; d < 3; ++d)
                        for (int j = 0; j < D.nu; ++j) perm[(size_t)d * D.nu + j] = 3 * j + d;
                }
                std::vector<float> img;
                std::vector<uint16_t> mask;
                std::vector<int> rowmap;
                F32Operator &op = D.f32op[w];
                f32_pack(opv[w]->data(), om[w], ok1[w], ok2[w], perm, img, mask, rowmap, op);
                float *dimg = nullptr;
                uint16_t *dmask = nullptr;
                int *drow = nullptr;
                if ((rc = upload(c, &dimg, img)) || (rc = upload(c, &dmask, mask)) || (rc = upload(c, &drow, rowmap)))
                    return rc;
                op.img = dimg;
                op.mask = dmask;
                op.rowmap = drow;
            }
        }
        if (prm->precision == FR_FP64S) {
            // the operators of a type whose FMA kernel would run mostly
            // non-zero products (tetrahedra; the prism and hexahedron
            // operators vanish outside their tensor-product structure and
            // keep the zero-skipping FMA kernel) on the tensor cores
            const std::vector<double> *opv[3] = {&ops[t].M0, &ops[t].AGRAD, &ops[t].ADIV};
            const int om[3] = {D.nf, 3 * D.nu, D.nu}, ok1[3] = {D.nu, D.nu, 3 * D.nu}, ok2[3] = {0, D.nf, D.nf};
            for (int w = 0; w < 3; ++w) {
                const size_t cnt = opv[w]->size();
                size_t nnz = 0;
                for (double v : *opv[w]) nnz += v != 0.0;
                if (2 * nnz < cnt) continue;
                std::vector<uint16_t> img;
                std::vector<int> rexp;
                X64Operator &op = D.x64[w];
                if (!x64_pack(opv[w]->data(), om[w], ok1[w], ok2[w], w == 1, img, rexp, op)) continue;
                uint16_t *dimg = nullptr;
                int *dre = nullptr;
                if ((rc = upload(c, &dimg, img)) || (rc = upload(c, &dre, rexp))) return rc;
                op.img = (const uint8_t *)dimg;
                op.rexp = dre;
            }
        }
        if (f32_storage(prm->precision)) {
            // float views of the geometry and operators (rounded once).  In
            // the tensor-core modes, where the flux kernel and the RK update
            // stream the geometry, a type whose float S and 1/J are the same
            // at every solution point of every element keeps one value per
            // element (the same floats: the results do not change)
            int k0 = 0;
            if (prm->precision == FR_BF16X3 || prm->precision == FR_TF32X3) {
                bool same = true;
                for (int64_t e = 0; e < D.ne && same; ++e)
                    for (int j = 1; j < D.nu && same; ++j) {
                        for (int k = 0; k < 9; ++k)
                            same = same && (float)S[((size_t)j * 9 + k) * D.np + e] == (float)S[(size_t)k * D.np + e];
                        same = same && (float)iJ[(size_t)j * D.np + e] == (float)iJ[e];
                    }
                if (same) {
                    std::vector<float> Se((size_t)9 * D.np, 0.f), iJe((size_t)D.np, 0.f);
                    for (size_t i = 0; i < Se.size(); ++i) Se[i] = (float)S[i];   // point 0's rows
                    for (size_t i = 0; i < iJe.size(); ++i) iJe[i] = (float)iJ[i];
                    float *dS = nullptr, *diJ = nullptr;
                    if ((rc = upload(c, &dS, Se)) || (rc = upload(c, &diJ, iJe))) return rc;
                    D.S_t = dS;
                    D.invJ_t = diJ;
                    D.geo_elem = 1;
                    k0 = 2;
                }
            }
            double *src[5] = {D.S, D.invJ, D.M0, D.AGRAD, D.ADIV};
            void **dst[5] = {&D.S_t, &D.invJ_t, &D.M0_t, &D.AGRAD_t, &D.ADIV_t};
            const size_t cnt[5] = {S.size(), iJ.size(), ops[t].M0.size(), ops[t].AGRAD.size(), ops[t].ADIV.size()};
            for (int k = k0; k < 5; ++k) {
                if ((rc = dev_alloc_bytes(c, dst[k], cnt[k] * sizeof(float)))) return rc;
                if ((rc = cuda_check(launch_to_float((int64_t)cnt[k], src[k], (float *)*dst[k], 0), "to float")))
                    return rc;
            }
        } else {
            D.S_t = D.S;
            D.invJ_t = D.invJ;
            D.M0_t = D.M0;
            D.AGRAD_t = D.AGRAD;
            D.ADIV_t = D.ADIV;
        }
        D.xu = G.xu;
    }
    if (nhalo > 0) {
        const size_t es = f32_storage(prm->precision) ? sizeof(float) : sizeof(double);
        c->nhalo = nhalo;
        c->nhalo_p = (nhalo + kPad - 1) / kPad * kPad;
        const size_t sh = (size_t)NV * c->nhalo_p;
        if ((rc = dev_alloc_bytes(c, &c->UF_h, sh * es)) || (rc = dev_alloc_bytes(c, &c->FC_h, sh * es)))
            return rc;
        if (prm->viscous &&
            ((rc = dev_alloc_bytes(c, &c->DUF_h, sh * es)) || (rc = dev_alloc_bytes(c, &c->GUF_h, 3 * sh * es))))
            return rc;
    }
    c->npairs = (int64_t)faces.ta.size();
    c->nbnd = (int64_t)faces.bt.size();
    if ((rc = upload(c, &c->ea, faces.ea)) || (rc = upload(c, &c->eb, faces.eb)) ||
        (rc = upload(c, &c->nrm, faces.n)) || (rc = upload(c, &c->maga, faces.maga)) ||
        (rc = upload(c, &c->magb, faces.magb)) || (rc = upload(c, &c->bt, faces.bt)) ||
        (rc = upload(c, &c->bf, faces.bf)) || (rc = upload(c, &c->be, faces.be)) ||
        (rc = upload(c, &c->btag, faces.btag)) || (rc = upload(c, &c->bn, faces.bn)) ||
        (rc = upload(c, &c->bmag, faces.bmag)))
        return rc;
    {
        std::vector<double> bw(faces.bt.size());
        for (size_t k = 0; k < bw.size(); ++k) bw[k] = ops[faces.bt[k]].FW[faces.bf[k]];
        if ((rc = upload(c, &c->bw, bw))) return rc;
        // LDG switch: +1 where side a's outward normal n has n . s > 0,
        // s = (1, 0.1 sqrt 2, 0.01 sqrt 3) (the dot product in double)
        std::vector<uint32_t> code(faces.ta.size());
        for (size_t k = 0; k < code.size(); ++k) {
            const double *n = &faces.n[3 * k];
            const double d = n[0] * 1.0 + n[1] * 0.14142135623730950488 + n[2] * 0.017320508075688772935;
            if (faces.fa[k] < 0 || faces.fa[k] >= kPairMaxFpt || faces.fb[k] < 0 || faces.fb[k] >= kPairMaxFpt)
                return set_err(FR_ERR_UNSUPPORTED, "more flux points per element than the pair code holds");
            code[k] = pair_code(faces.ta[k], faces.tb[k], faces.fa[k], faces.fb[k], d > 0.0 ? 1 : -1);
        }
        if ((rc = upload(c, &c->pcode, code))) return rc;
        if (f32_storage(prm->precision)) {
            auto to_f = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
            if ((rc = upload(c, &c->nrm_f, to_f(faces.n))) || (rc = upload(c, &c->maga_f, to_f(faces.maga))) ||
                (rc = upload(c, &c->magb_f, to_f(faces.magb))) || (rc = upload(c, &c->bn_f, to_f(faces.bn))) ||
                (rc = upload(c, &c->bmag_f, to_f(faces.bmag))))
                return rc;
        }
    }
    // the discrete divergence of the constant reference flux (zero with exact
    // geometry; ~1e-11 with the geometric factors rounded), evaluated once in
    // FP64 and added back to every RHS since the flux kernels subtract that
    // flux.  Only FR_FP64 needs it: in the FP32-storage modes it lies far
    // below the arithmetic's resolution (the RHS carries ~1e-6 relative
    // rounding), so they skip it and its 8 bytes per output.
    if (!f32_storage(prm->precision)) {
        const Phys ph = phys_of(c);
        const bool f32 = false;
        double *tFT[NT] = {}, *tFC[NT] = {};
        std::vector<void *> tmp;
        for (int t = 0; t < NT; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            if ((rc = dev_alloc(c, &D.Rfs, (size_t)D.nu * NV * D.np))) return rc;
            if (f32) {
                const size_t su = (size_t)D.nu * NV * D.np, sf = (size_t)D.nf * NV * D.np;
                if (dev_malloc((void **)&tFT[t], 3 * su * sizeof(double)) != cudaSuccess ||
                    dev_malloc((void **)&tFC[t], sf * sizeof(double)) != cudaSuccess) {
                    cudaGetLastError();
                    for (double *q : tFT) dev_free(q);
                    for (double *q : tFC) dev_free(q);
                    return set_err(FR_ERR_NOMEM, "set-up scratch");
                }
            } else {
                tFT[t] = (double *)D.FT;
                tFC[t] = (double *)D.FC;
            }
        }
        Fields F{};
        for (int t = 0; t < NT; ++t) {
            F.UF[t] = nullptr;
            F.DUF[t] = nullptr;
            F.GUF[t] = nullptr;
            F.FC[t] = tFC[t];
            F.np[t] = c->T[t].np;
        }
        // the remote side of a cut pair (FP64 here, the context's precision)
        F.UF[HALO] = nullptr;
        F.DUF[HALO] = nullptr;
        F.GUF[HALO] = nullptr;
        F.FC[HALO] = (double *)c->FC_h;
        F.np[HALO] = c->nhalo_p;
        rc = FR_OK;
        for (int t = 0; t < NT && !rc; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            rc = cuda_check(launch_const_flux(D.nu, D.ne, D.np, D.S, tFT[t], ph, 0), "reference flux");
        }
        if (!rc) rc = cuda_check(launch_const_common(pairs_of(c), bnd_of(c), F, ph, 0), "reference common flux");
        for (int t = 0; t < NT && !rc; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            GemmArgs g;
            g.M = D.nu;
            g.N = (int64_t)NV * D.np;
            g.K1 = 3 * D.nu;
            g.K2 = D.nf;
            g.A = D.ADIV;
            g.B1 = tFT[t];
            g.ldb1 = g.N;
            g.B2 = tFC[t];
            g.ldb2 = g.N;
            g.ldc = g.N;
            g.np = D.np;
            g.invJ = D.invJ;
            g.mode = GEMM_DIV;
            g.C = D.Rfs;
            rc = cuda_check(launch_gemm_f64(g, 0), "reference divergence");
        }
        if (f32) {
            cudaDeviceSynchronize();
            for (int t = 0; t < NT; ++t) {
                dev_free(tFT[t]);
                dev_free(tFC[t]);
            }
        }
        if (rc) return rc;
    }
    int nbt = 0;
    for (int t = 0; t < NT; ++t) {
        c->red_blocks[t] = c->T[t].present ? 2 * num_sms(c->device) : 0;
        nbt += c->red_blocks[t];
    }
    if ((rc = dev_alloc(c, &c->red, (size_t)nbt * 7 + 8))) return rc;
    if ((rc = dev_alloc(c, &c->diag, (size_t)kDiagBlocks * (2 + 6) + 8))) return rc;
    if ((rc = dev_alloc(c, &c->tc_err, 1))) return rc;
    if (prm->precision == FR_FP64S) {
        int64_t cols = 0;
        for (int t = 0; t < NT; ++t)
            if (c->T[t].present && 3 * NV * c->T[t].np > cols) cols = 3 * NV * c->T[t].np;
        if ((rc = dev_alloc_bytes(c, (void **)&c->x64_E, (size_t)cols * sizeof(int)))) return rc;
    }
    if (cudaHostAlloc((void **)&c->nf_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        c->nf_host = nullptr;
        return set_err(FR_ERR_NOMEM, "pinned status flag");
    }
    *c->nf_host = 0;
    if ((rc = cuda_check(cudaHostGetDevicePointer((void **)&c->nf_dev, c->nf_host, 0), "status flag address")))
        return rc;
    return cuda_check(cudaDeviceSynchronize(), "fr_create sync");
}

int create_impl(const fr_mesh *mesh, int order, const fr_params *prm, fr_ctx *c) {
    int rc;
    if (!mesh) return set_err(FR_ERR_ARG, "null mesh or params");
    if ((rc = check_params(order, prm))) return rc;
    HostSetup h;
    if ((rc = host_setup(mesh, order, h))) return rc;
    return device_setup(c, order, prm, h.ops, h.geo, h.faces, 0);
}

template <typename T>
int rhs_public(fr_ctx *c, const double *u_dev, double *r_dev, cudaStream_t s) {
    size_t off = 0;
    T *in[NT] = {};
    int rc;
    const Phys ph = phys_of(c);
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_pub_to_int<T>(D.nu, D.ne, D.np, u_dev + off, nullptr, s, (T *)D.Us, ph.uref),
                             "rhs layout in")))
            return rc;
        in[t] = (T *)D.Us;
        off += (size_t)D.ne * NV * D.nu;
    }
    if ((rc = rhs_internal<T>(c, in, nullptr, s))) return rc;
    off = 0;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_int_to_pub<T>(D.nu, D.ne, D.np, (const T *)D.R, r_dev + off, s), "rhs layout out")))
            return rc;
        off += (size_t)D.ne * NV * D.nu;
    }
    return FR_OK;
}

// RHS of the solution register, then the FP64 reductions of fr_diagnostics
template <typename T>
int diagnostics_impl(fr_ctx *c, double *out, cudaStream_t s) {
    const Phys ph = phys_of(c);
    T *in[NT] = {};
    int rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre"))) return rc;
        in[t] = (T *)D.Us;
    }
    if ((rc = rhs_internal<T>(c, in, nullptr, s))) return rc;
    double *part = c->diag, *res = c->diag + (size_t)kDiagBlocks * 8;
    int nb = 0;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_ke_rate<T>(D.nu, D.ne, D.np, D.U, (const T *)D.R, D.wJ, part + nb, kDiagBlocks, s),
                             "kinetic-energy rate")))
            return rc;
        nb += kDiagBlocks;
    }
    if ((rc = cuda_check(launch_sum_partials(part, nb, 1, res, s), "kinetic-energy rate sum"))) return rc;
    double *wpart = part + (size_t)kDiagBlocks * 2;
    if ((rc = cuda_check(launch_wall_force<T>(bnd_of(c), c->bw, fields_of<T>(c), ph, wpart, kDiagBlocks, s),
                         "wall force")))
        return rc;
    if ((rc = cuda_check(launch_sum_partials(wpart, kDiagBlocks, 6, res + 1, s), "wall force sum"))) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(out, res, 7 * sizeof(double), cudaMemcpyDeviceToHost, s), "diagnostics copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(s), "diagnostics sync"))) return rc;
    return check_tc(c);
}

template <typename T>
int step_impl(fr_ctx *c, double dt, int nsteps, cudaStream_t s) {
    const double ca[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
    const double cs[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
    if (nsteps <= 0) return FR_OK;
    // the centred stage input is derived from the FP64 register (fr_rhs
    // reuses its buffer); the last stage of every step keeps it current
    const Phys ph = phys_of(c);
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        int rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre");
        if (rc) return rc;
    }
    for (int it = 0; it < nsteps; ++it)
        for (int st = 0; st < 4; ++st) {
            T *in[NT] = {};
            for (int t = 0; t < NT; ++t)
                if (c->T[t].present) in[t] = (T *)c->T[t].Us;
            RKStage rk{ca[st], cs[st], st == 0, st == 3};
            int rc = rhs_internal<T>(c, in, &rk, s);
            if (rc) return rc;
        }
    return FR_OK;
}

// Five-stage fourth-order low-storage Runge-Kutta (Carpenter & Kennedy
// 1994, 2N storage): dU <- A_i dU + dt R(U); U <- U + B_i dU.  The RHS of
// each stage is stored (R) and a streaming pass applies the update; dU
// lives in the Uacc register.
constexpr double kRk2nA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                              -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
constexpr double kRk2nB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                              1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                              2277821191437.0 / 14882151754819.0};

template <typename T>
int step_2n_impl(fr_ctx *c, double dt, int nsteps, cudaStream_t s) {
    if (nsteps <= 0) return FR_OK;
    const Phys ph = phys_of(c);
    int rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre"))) return rc;
    }
    for (int it = 0; it < nsteps; ++it)
        for (int st = 0; st < 5; ++st) {
            T *in[NT] = {};
            for (int t = 0; t < NT; ++t)
                if (c->T[t].present) in[t] = (T *)c->T[t].Us;
            if ((rc = rhs_internal<T>(c, in, nullptr, s))) return rc;
            for (int t = 0; t < NT; ++t) {
                DevType &D = c->T[t];
                if (!D.present) continue;
                if ((rc = cuda_check(launch(c, K_DIV, s,
                                            [&] {
                                                return launch_rk_2n_update<T>(D.nu, D.np, (const T *)D.R, D.U, D.Uacc,
                                                                              (T *)D.Us, ph.uref, kRk2nA[st],
                                                                              kRk2nB[st], dt, st == 0, s);
                                            }),
                                     "2N update")))
                    return rc;
            }
        }
    return FR_OK;
}

// RK45[2R+] (the paper's stepper, Sec. 3.4): RK4(3)5[2R+]C of Kennedy,
// Carpenter & Lewis (2000), five stages in two registers (U and the stage
// input Us) plus the embedded error estimate E.  The published rational
// coefficients (the same table the oracle states): sub-diagonal a_1..a_4,
// weights b_1..b_5, embedded weights bhat_1..bhat_5.
constexpr double kRk45A[4] = {970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
                              2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0};
constexpr double kRk45B[5] = {1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
                              -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
                              5198255086312.0 / 14908931495163.0};
constexpr double kRk45Bh[5] = {1016888040809.0 / 7410784769900.0, 11231460423587.0 / 58533540763752.0,
                               -1563879915014.0 / 6823010717585.0, 606302364029.0 / 971179775848.0,
                               1097981568119.0 / 3980877426909.0};

// the error register (and, for the adaptive driver, the backup of U):
// allocated by the first call that needs them
int ensure_rk45_regs(fr_ctx *c, bool backup) {
    int rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        const size_t su = (size_t)D.nu * NV * D.np;
        if (!D.E && (rc = dev_alloc(c, &D.E, su))) return rc;
        if (backup && !D.Ubak && (rc = dev_alloc(c, &D.Ubak, su))) return rc;
    }
    return FR_OK;
}

template <typename T>
int step_2r_impl(fr_ctx *c, double dt, int nsteps, cudaStream_t s) {
    if (nsteps <= 0) return FR_OK;
    int rc;
    if ((rc = ensure_rk45_regs(c, false))) return rc;
    const Phys ph = phys_of(c);
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre"))) return rc;
    }
    for (int it = 0; it < nsteps; ++it)
        for (int st = 0; st < 5; ++st) {
            T *in[NT] = {};
            for (int t = 0; t < NT; ++t)
                if (c->T[t].present) in[t] = (T *)c->T[t].Us;
            if ((rc = rhs_internal<T>(c, in, nullptr, s))) return rc;
            const double cs = st < 4 ? dt * kRk45A[st] : 0.0, ca = dt * kRk45B[st],
                         ce = dt * (kRk45B[st] - kRk45Bh[st]);
            for (int t = 0; t < NT; ++t) {
                DevType &D = c->T[t];
                if (!D.present) continue;
                if ((rc = cuda_check(launch(c, K_DIV, s,
                                            [&] {
                                                return launch_rk_2r_update<T>(D.nu, D.np, (const T *)D.R, D.U, D.E,
                                                                              (T *)D.Us, ph.uref, cs, ca, ce, st == 0,
                                                                              st == 4, s);
                                            }),
                                     "2R update")))
                    return rc;
            }
        }
    return FR_OK;
}

// weighted RMS norm of the error register: sqrt(mean((E / (atol + rtol |U|))^2))
// over every value of the state (synchronises)
int rk45_error_norm(fr_ctx *c, double atol, double rtol, double *norm, cudaStream_t s) {
    int rc, nb = 0;
    int64_t nval = 0;
    double *part = c->diag, *res = c->diag + (size_t)kDiagBlocks * 8;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if (!D.E) return set_err(FR_ERR_ARG, "no RK45 step has been taken on this context");
        if ((rc = cuda_check(launch_err_norm_partial(D.nu, D.ne, D.np, D.U, D.E, atol, rtol, part + nb, kDiagBlocks,
                                                     s),
                             "error norm")))
            return rc;
        nb += kDiagBlocks;
        nval += D.ne * NV * D.nu;
    }
    if ((rc = cuda_check(launch_sum_partials(part, nb, 1, res, s), "error norm sum"))) return rc;
    double sum = 0.0;
    if ((rc = cuda_check(cudaMemcpyAsync(&sum, res, sizeof(double), cudaMemcpyDeviceToHost, s), "error norm copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(s), "error norm sync"))) return rc;
    if ((rc = check_tc(c))) return rc;
    *norm = std::sqrt(sum / (double)nval);
    return FR_OK;
}

// step-size controller of the adaptive driver (the oracle's, same readings):
// dt * clamp(0.9 norm^(-1/4), 0.3, 2.5)
double rk45_next_dt(double dt, double norm) {
    if (norm <= 0.0) return dt * 2.5;
    return dt * std::min(2.5, std::max(0.3, 0.9 * std::pow(norm, -0.25)));
}

template <typename T>
int adaptive_impl(fr_ctx *c, double t_span, double atol, double rtol, double *dt_io, int max_steps, int64_t *stats,
                  cudaStream_t s) {
    int rc;
    if ((rc = ensure_rk45_regs(c, true))) return rc;
    double t = 0.0, dt = *dt_io;
    int64_t acc = 0, rej = 0;
    while (t < t_span && acc + rej < max_steps) {
        const bool last = dt >= t_span - t;
        const double h = last ? t_span - t : dt;
        for (int k = 0; k < NT; ++k) {
            DevType &D = c->T[k];
            if (!D.present) continue;
            if ((rc = cuda_check(cudaMemcpyAsync(D.Ubak, D.U, (size_t)D.nu * NV * D.np * sizeof(double),
                                                 cudaMemcpyDeviceToDevice, s),
                                 "backup")))
                return rc;
        }
        if ((rc = step_2r_impl<T>(c, h, 1, s))) return rc;
        double nrm = 0.0;
        if ((rc = rk45_error_norm(c, atol, rtol, &nrm, s))) return rc;
        if (!std::isfinite(nrm)) return set_err(FR_ERR_NONFINITE, "non-finite RK45 error estimate");
        if (nrm <= 1.0) {
            ++acc;
            t = last ? t_span : t + h;
        } else {
            ++rej;
            for (int k = 0; k < NT; ++k) {
                DevType &D = c->T[k];
                if (!D.present) continue;
                if ((rc = cuda_check(cudaMemcpyAsync(D.U, D.Ubak, (size_t)D.nu * NV * D.np * sizeof(double),
                                                     cudaMemcpyDeviceToDevice, s),
                                     "restore")))
                    return rc;
            }
        }
        dt = rk45_next_dt(h, nrm);
    }
    *dt_io = dt;
    if (stats) {
        stats[0] = acc;
        stats[1] = rej;
    }
    // the stage input follows the (possibly restored) solution register
    const Phys ph = phys_of(c);
    for (int k = 0; k < NT; ++k) {
        DevType &D = c->T[k];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre"))) return rc;
    }
    if (t < t_span) return set_err(FR_ERR_ARG, "max_steps reached before t_span");
    return FR_OK;
}

template int step_2r_impl<float>(fr_ctx *, double, int, cudaStream_t);
template int step_2r_impl<double>(fr_ctx *, double, int, cudaStream_t);
template int step_2n_impl<float>(fr_ctx *, double, int, cudaStream_t);
template int step_2n_impl<double>(fr_ctx *, double, int, cudaStream_t);
template int step_impl<float>(fr_ctx *, double, int, cudaStream_t);
template int rhs_public<float>(fr_ctx *, const double *, double *, cudaStream_t);
template int rhs_public<double>(fr_ctx *, const double *, double *, cudaStream_t);
template int phase_interp<float>(fr_ctx *, float *const[NT], cudaStream_t);
template int phase_interp<double>(fr_ctx *, double *const[NT], cudaStream_t);
template int phase_grad<float>(fr_ctx *, float *const[NT], cudaStream_t);
template int phase_grad<double>(fr_ctx *, double *const[NT], cudaStream_t);
template int phase_div<float>(fr_ctx *, float *const[NT], const RKStage *, cudaStream_t);
template int phase_div<double>(fr_ctx *, double *const[NT], const RKStage *, cudaStream_t);
template int front_stages<float>(fr_ctx *, float *const[NT], cudaStream_t);
template int front_stages<double>(fr_ctx *, double *const[NT], cudaStream_t);
template int step_impl<double>(fr_ctx *, double, int, cudaStream_t);
template FieldsT<float> fields_of<float>(const fr_ctx *);
template FieldsT<double> fields_of<double>(const fr_ctx *);
#define FR_ARGS_INST(T)                                                      \
    template GemmArgsT<T> args_m0<T>(const fr_ctx *, int, const T *);     \
    template GemmArgsT<T> args_grad<T>(const fr_ctx *, int, const T *);   \
    template GemmArgsT<T> args_m0grad<T>(const fr_ctx *, int);            \
    template GemmArgsT<T> args_div<T>(const fr_ctx *, int, const RKStage *);
FR_ARGS_INST(float)
FR_ARGS_INST(double)
#undef FR_ARGS_INST

}  // namespace api
}  // namespace fr

extern "C" {

const char *fr_strerror(int code) {
    switch (code) {
        case FR_OK:
            return "success";
        case FR_ERR_ARG:
            return "invalid argument";
        case FR_ERR_MESH:
            return "invalid mesh";
        case FR_ERR_CUDA:
            return "CUDA error";
        case FR_ERR_NONFINITE:
            return "non-finite or non-physical state";
        case FR_ERR_TIMEOUT:
            return "device wait timed out";
        case FR_ERR_NOMEM:
            return "out of memory";
        case FR_ERR_UNSUPPORTED:
            return "unsupported request";
    }
    return "unknown error";
}

const char *fr_last_error(void) { return g_last_error.c_str(); }

int fr_create(const fr_mesh *mesh, int order, const fr_params *params, fr_ctx **out) {
    if (!out) return set_err(FR_ERR_ARG, "null output pointer");
    *out = nullptr;
    fr_ctx *c = new (std::nothrow) fr_ctx();
    if (!c) return set_err(FR_ERR_NOMEM, "host allocation");
    int rc;
    try {
        rc = create_impl(mesh, order, params, c);
    } catch (const std::bad_alloc &) {
        rc = set_err(FR_ERR_NOMEM, "host allocation during set-up");
    } catch (...) {
        rc = set_err(FR_ERR_ARG, "unexpected exception during set-up");
    }
    if (rc) {
        fr_destroy(c);
        return rc;
    }
    *out = c;
    return FR_OK;
}

void fr_destroy(fr_ctx *c) {
    if (!c) return;
    for (void *p : c->allocs) dev_free(p);
    if (c->nf_host) cudaFreeHost(c->nf_host);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

int fr_profile(fr_ctx *c, int enable) {
    if (!c) return set_err(FR_ERR_ARG, "null context");
    c->prof = enable ? 1 : 0;
    c->prof_ev.clear();
    c->ev_used = 0;
    c->launches = 0;
    return FR_OK;
}

int fr_profile_read(fr_ctx *c, double *ms, int64_t *count, int64_t *launches) {
    if (!c || !ms || !count || !launches) return set_err(FR_ERR_ARG, "null argument");
    for (int k = 0; k < K_NCLASS; ++k) {
        ms[k] = 0.0;
        count[k] = 0;
    }
    int rc;
    for (auto &pe : c->prof_ev) {
        if ((rc = cuda_check(cudaEventSynchronize(pe.second.second), "profile sync"))) return rc;
        float t = 0.f;
        if ((rc = cuda_check(cudaEventElapsedTime(&t, pe.second.first, pe.second.second), "profile elapsed")))
            return rc;
        ms[pe.first % K_NCLASS] += t;
        count[pe.first % K_NCLASS] += 1;
    }
    *launches = c->launches;
    return FR_OK;
}

int fr_profile_read_types(fr_ctx *c, double *ms, int64_t *count) {
    if (!c || !ms || !count) return set_err(FR_ERR_ARG, "null argument");
    for (int k = 0; k < (NT + 1) * K_NCLASS; ++k) {
        ms[k] = 0.0;
        count[k] = 0;
    }
    int rc;
    for (auto &pe : c->prof_ev) {
        if ((rc = cuda_check(cudaEventSynchronize(pe.second.second), "profile sync"))) return rc;
        float t = 0.f;
        if ((rc = cuda_check(cudaEventElapsedTime(&t, pe.second.first, pe.second.second), "profile elapsed")))
            return rc;
        ms[pe.first] += t;
        count[pe.first] += 1;
    }
    return FR_OK;
}

int fr_ndof(const fr_ctx *c, int64_t *ndof) {
    if (!c || !ndof) return set_err(FR_ERR_ARG, "null argument");
    *ndof = ndof_of(c);
    return FR_OK;
}

int fr_info(const fr_ctx *c, int64_t *out) {
    if (!c || !out) return set_err(FR_ERR_ARG, "null argument");
    out[0] = c->T[0].ne;
    out[1] = c->T[1].ne;
    out[2] = c->order;
    out[3] = nupts_of(0, c->order);
    out[4] = nupts_of(1, c->order);
    out[5] = nfpts_of(0, c->order);
    out[6] = nfpts_of(1, c->order);
    out[7] = c->npairs;
    out[8] = c->T[2].ne;
    out[9] = nupts_of(2, c->order);
    out[10] = nfpts_of(2, c->order);
    return FR_OK;
}

int fr_upts(const fr_ctx *c, double *xyz) {
    if (!c || !xyz) return set_err(FR_ERR_ARG, "null argument");
    size_t off = 0;
    for (int t = 0; t < NT; ++t) {
        const DevType &D = c->T[t];
        if (!D.present) continue;
        for (int64_t e = 0; e < D.ne; ++e)
            for (int k = 0; k < 3; ++k)
                for (int j = 0; j < D.nu; ++j) xyz[off++] = D.xu[((size_t)e * D.nu + j) * 3 + k];
    }
    return FR_OK;
}

// The device address of a page-locked host buffer mapped into the device's
// address space (cudaHostAlloc / cudaHostRegister memory with unified
// addressing), or nullptr for any other buffer.  The layout kernels read
// or write such a buffer directly over the CPU-GPU link, which moves the
// state faster than one copy engine's bulk copy does; other host memory is
// copied through a device staging buffer.
static const double *mapped_host(const double *u) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, u) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? (const double *)a.devicePointer : nullptr;
}

int fr_set_state(fr_ctx *c, const double *u, void *stream) {
    if (!c || !u) return set_err(FR_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const double *um = mapped_host(u);
    size_t off = 0;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        const size_t n = (size_t)D.ne * NV * D.nu;
        int rc;
        const double *src = um ? um + off : (const double *)D.Uacc;
        // otherwise stage through the accumulator register (overwritten by every step)
        if (!um && (rc = cuda_check(cudaMemcpyAsync(D.Uacc, u + off, n * sizeof(double), cudaMemcpyHostToDevice, s),
                                    "set_state copy")))
            return rc;
        if ((rc = cuda_check(launch_pub_to_int<double>(D.nu, D.ne, D.np, src, D.U, s, nullptr, nullptr),
                             "set_state layout")))
            return rc;
        off += n;
    }
    const int rc = cuda_check(cudaStreamSynchronize(s), "set_state sync");
    if (!rc && c->nf_host) *(volatile int *)c->nf_host = 0;  // a new state: no earlier blow-up applies
    return rc;
}

int fr_get_state(fr_ctx *c, double *u, void *stream) {
    if (!c || !u) return set_err(FR_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    double *um = const_cast<double *>(mapped_host(u));
    size_t off = 0;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        const size_t n = (size_t)D.ne * NV * D.nu;
        int rc;
        if ((rc = cuda_check(launch_int_to_pub<double>(D.nu, D.ne, D.np, D.U, um ? um + off : D.Uacc, s),
                             "get_state layout")))
            return rc;
        if (!um && (rc = cuda_check(cudaMemcpyAsync(u + off, D.Uacc, n * sizeof(double), cudaMemcpyDeviceToHost, s),
                                    "get_state copy")))
            return rc;
        off += n;
    }
    const int rc = cuda_check(cudaStreamSynchronize(s), "get_state sync");
    return rc ? rc : check_tc(c);
}

int fr_rhs(fr_ctx *c, const double *u_dev, double *r_dev, void *stream) {
    if (!c || !u_dev || !r_dev) return set_err(FR_ERR_ARG, "null argument");
    if (u_dev == r_dev) return set_err(FR_ERR_ARG, "u and r may not alias");
    cudaStream_t s = (cudaStream_t)stream;
    return is_f32(c) ? rhs_public<float>(c, u_dev, r_dev, s) : rhs_public<double>(c, u_dev, r_dev, s);
}

int fr_step(fr_ctx *c, double dt, int nsteps, void *stream) {
    if (!c || nsteps < 0 || !std::isfinite(dt)) return set_err(FR_ERR_ARG, "invalid step arguments");
    int rc;
    if ((rc = step_guard(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = is_f32(c) ? step_impl<float>(c, dt, nsteps, s) : step_impl<double>(c, dt, nsteps, s);
    return (rc || nsteps == 0) ? rc : step_check(c, s);
}

int fr_step_ls(fr_ctx *c, double dt, int nsteps, void *stream) {
    if (!c || nsteps < 0 || !std::isfinite(dt)) return set_err(FR_ERR_ARG, "invalid step arguments");
    int rc;
    if ((rc = step_guard(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = is_f32(c) ? step_2n_impl<float>(c, dt, nsteps, s) : step_2n_impl<double>(c, dt, nsteps, s);
    return (rc || nsteps == 0) ? rc : step_check(c, s);
}

int fr_check(fr_ctx *c, void *stream) {
    if (!c) return set_err(FR_ERR_ARG, "null context");
    int rc;
    if ((rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "check sync"))) return rc;
    if ((rc = check_tc(c))) return rc;
    return step_guard(c);
}

int fr_step_rk45(fr_ctx *c, double dt, int nsteps, void *stream) {
    if (!c || nsteps < 0 || !std::isfinite(dt)) return set_err(FR_ERR_ARG, "invalid step arguments");
    int rc;
    if ((rc = step_guard(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = is_f32(c) ? step_2r_impl<float>(c, dt, nsteps, s) : step_2r_impl<double>(c, dt, nsteps, s);
    return (rc || nsteps == 0) ? rc : step_check(c, s);
}

int fr_rk45_error(fr_ctx *c, double atol, double rtol, double *norm, void *stream) {
    if (!c || !norm || !(atol >= 0.0) || !(rtol >= 0.0) || !(atol + rtol > 0.0))
        return set_err(FR_ERR_ARG, "invalid error-norm arguments");
    return rk45_error_norm(c, atol, rtol, norm, (cudaStream_t)stream);
}

int fr_rk45_get_error(fr_ctx *c, double *e, void *stream) {
    if (!c || !e) return set_err(FR_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t off = 0;
    int rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if (!D.E) return set_err(FR_ERR_ARG, "no RK45 step has been taken on this context");
        const size_t n = (size_t)D.ne * NV * D.nu;
        if ((rc = cuda_check(launch_int_to_pub<double>(D.nu, D.ne, D.np, D.E, D.Uacc, s), "error layout")))
            return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(e + off, D.Uacc, n * sizeof(double), cudaMemcpyDeviceToHost, s),
                             "error copy")))
            return rc;
        off += n;
    }
    return cuda_check(cudaStreamSynchronize(s), "error sync");
}

int fr_step_rk45_adaptive(fr_ctx *c, double t_span, double atol, double rtol, double *dt, int max_steps,
                          int64_t *stats, void *stream) {
    if (!c || !dt || !std::isfinite(t_span) || t_span < 0.0 || !(*dt > 0.0) || !std::isfinite(*dt) ||
        max_steps < 1 || !(atol >= 0.0) || !(rtol >= 0.0) || !(atol + rtol > 0.0))
        return set_err(FR_ERR_ARG, "invalid adaptive-step arguments");
    cudaStream_t s = (cudaStream_t)stream;
    return is_f32(c) ? adaptive_impl<float>(c, t_span, atol, rtol, dt, max_steps, stats, s)
                     : adaptive_impl<double>(c, t_span, atol, rtol, dt, max_steps, stats, s);
}

int fr_reduce(fr_ctx *c, double *out, void *stream) {
    if (!c || !out) return set_err(FR_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int off = 0, rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_reduce_partial(D.nu, D.ne, D.np, D.U, D.wJ, c->prm.gamma, c->red + (size_t)off * 7,
                                                   c->red_blocks[t], s),
                             "reduce")))
            return rc;
        off += c->red_blocks[t];
    }
    double *res = c->red + (size_t)off * 7;
    if ((rc = cuda_check(launch_reduce_final(c->red, off, res, s), "reduce final"))) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(out, res, 7 * sizeof(double), cudaMemcpyDeviceToHost, s), "reduce copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(s), "reduce sync"))) return rc;
    if ((rc = check_tc(c))) return rc;
    if (out[6] != 0.0) return set_err(FR_ERR_NONFINITE, "non-finite or non-physical state");
    return FR_OK;
}

int fr_diagnostics(fr_ctx *c, double *out, void *stream) {
    if (!c || !out) return set_err(FR_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    return is_f32(c) ? diagnostics_impl<float>(c, out, s) : diagnostics_impl<double>(c, out, s);
}

int fr_selftest_wait_timeout(fr_ctx *c, void *stream) {
    if (!c) return set_err(FR_ERR_ARG, "null context");
    if (!is_f32(c) && !is_x64(c))
        return set_err(FR_ERR_UNSUPPORTED, "the bounded-wait self-test needs a streamed operator kernel (not FR_FP64)");
    cudaStream_t s = (cudaStream_t)stream;
    int t = 0;
    while (t < NT && !c->T[t].present) ++t;
    int rc;
    if ((rc = check_tc(c))) return rc;  // a status from earlier work is reported, not masked
    DevType &D = c->T[t];
    // M0 on the context's (centred) stage input, its state loads withheld
    if (is_x64(c)) {
        t = 0;
        while (t < NT && !c->T[t].x64[0].img) ++t;
        if (t == NT) return set_err(FR_ERR_UNSUPPORTED, "no element type on the exact-split tensor-core kernel");
        DevType &Dx = c->T[t];
        const GemmArgsT<double> g = args_m0<double>(c, t, (const double *)Dx.Us);
        if ((rc = cuda_check(launch_gemm_x64(g, Dx.x64[0], c->x64_E, c->tc_err, s, 1), "self-test launch")))
            return rc;
    } else {
        const GemmArgsT<float> g = args_m0<float>(c, t, (const float *)D.Us);
        if ((rc = cuda_check(is_tc(c) ? launch_gemm_tc(g, D.tc[0], c->tc_err, s, 1)
                                      : launch_gemm_f32(g, D.f32op[0], c->tc_err, s, 1),
                             "self-test launch")))
            return rc;
    }
    if ((rc = cuda_check(cudaStreamSynchronize(s), "self-test sync"))) return rc;
    const int timed_out = check_tc(c) == FR_ERR_TIMEOUT;
    // clear the status so that the context stays usable
    if ((rc = cuda_check(cudaMemset(c->tc_err, 0, sizeof(int)), "self-test reset"))) return rc;
    if (!timed_out) return set_err(FR_ERR_CUDA, "the withheld loads did not end in a reported timeout");
    return FR_OK;
}

int fr_debug_fail_alloc(int64_t k) {
    if (k < 0) return set_err(FR_ERR_ARG, "k must be >= 0");
    g_alloc_seen = 0;
    g_fail_at = k;
    return FR_OK;
}

int fr_debug_alloc_stats(int64_t *out) {
    if (!out) return set_err(FR_ERR_ARG, "null argument");
    out[0] = g_alloc_seen.load();
    out[1] = g_live.load();
    return FR_OK;
}

int fr_peak_fp64(double *gflops, void *stream) {
    if (!gflops) return set_err(FR_ERR_ARG, "null argument");
    return cuda_check(probe_fp64(gflops, (cudaStream_t)stream), "fp64 probe");
}

int fr_gemm_fp64s(int M, int K, const double *A, int64_t N, const double *B, double *C, void *stream) {
    if (!A || !B || !C || M < 1 || K < 1 || K > kX64MaxK || N < 2 || N % 2 || ((uintptr_t)B % 16))
        return set_err(FR_ERR_ARG, "fr_gemm_fp64s: bad sizes or pointers");
    for (int64_t i = 0; i < (int64_t)M * K; ++i)
        if (!std::isfinite(A[i])) return set_err(FR_ERR_ARG, "fr_gemm_fp64s: A must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    X64Operator op;
    std::vector<uint16_t> img;
    std::vector<int> rexp;
    try {
        if (!x64_pack(A, M, K, 0, false, img, rexp, op)) return set_err(FR_ERR_ARG, "fr_gemm_fp64s: operator");
    } catch (...) {
        return set_err(FR_ERR_NOMEM, "host allocation");
    }
    void *dimg = nullptr, *dre = nullptr, *dE = nullptr, *derr = nullptr;
    auto release = [&] {
        dev_free(dimg);
        dev_free(dre);
        dev_free(dE);
        dev_free(derr);
    };
    if (dev_malloc(&dimg, img.size() * 2) != cudaSuccess || dev_malloc(&dre, rexp.size() * sizeof(int)) != cudaSuccess ||
        dev_malloc(&dE, (size_t)N * sizeof(int)) != cudaSuccess || dev_malloc(&derr, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        release();
        return set_err(FR_ERR_NOMEM, "fr_gemm_fp64s scratch");
    }
    int rc = cuda_check(cudaMemcpyAsync(dimg, img.data(), img.size() * 2, cudaMemcpyHostToDevice, s), "upload");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(dre, rexp.data(), rexp.size() * sizeof(int), cudaMemcpyHostToDevice, s), "upload");
    if (!rc) rc = cuda_check(cudaMemsetAsync(derr, 0, sizeof(int), s), "status");
    op.img = (const uint8_t *)dimg;
    op.rexp = (const int *)dre;
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K1 = K;
    g.B1 = B;
    g.ldb1 = N;
    g.C = C;
    g.ldc = N;
    g.mode = GEMM_STORE;
    g.np = N;
    if (!rc) rc = cuda_check(launch_colexp(B, N, K, nullptr, 0, 0, N, (int *)dE, s), "column exponents");
    if (!rc) rc = cuda_check(launch_gemm_x64(g, op, (const int *)dE, (int *)derr, s), "exact-split product");
    int h = 0;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "fr_gemm_fp64s sync");
    release();
    if (!rc && h) rc = set_err(FR_ERR_TIMEOUT, "the exact-split kernel gave up a bounded wait");
    return rc;
}

int fr_operator(int etype, int order, int which, double *out, int64_t *rows, int64_t *cols) {
    if (!rows || !cols) return set_err(FR_ERR_ARG, "null rows/cols");
    RefOps o;
    std::string err;
    int rc;
    try {
        rc = build_ref_ops(etype, order, o, err);
    } catch (...) {
        return set_err(FR_ERR_NOMEM, "host allocation");
    }
    if (rc) return set_err(rc, err);
    const std::vector<double> *src = nullptr;
    int64_t r = 0, cc = 0;
    switch (which) {
        case 0: src = &o.M0; r = o.nf; cc = o.nu; break;
        case 1: src = &o.D; r = 3 * o.nu; cc = o.nu; break;
        case 2: src = &o.M3; r = o.nu; cc = o.nf; break;
        case 3: src = &o.AGRAD; r = 3 * o.nu; cc = o.nu + o.nf; break;
        case 4: src = &o.ADIV; r = o.nu; cc = 3 * o.nu + o.nf; break;
        case 5: src = &o.W; r = o.nu; cc = 1; break;
        case 6: src = &o.upts; r = o.nu; cc = 3; break;
        case 7: src = &o.fpts; r = o.nf; cc = 3; break;
        case 8: src = &o.fnorm; r = o.nf; cc = 3; break;
        case 9: src = &o.FW; r = o.nf; cc = 1; break;
        default: return set_err(FR_ERR_ARG, "unknown operator id");
    }
    *rows = r;
    *cols = cc;
    if (out) std::memcpy(out, src->data(), sizeof(double) * (size_t)(r * cc));
    return FR_OK;
}

}  // extern "C"
