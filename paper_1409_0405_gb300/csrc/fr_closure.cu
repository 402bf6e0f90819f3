// Learned closure of the low-order FR right-hand side (no counterpart in the
// paper; declared in include/fr.h): order transfer between two contexts on
// one mesh, the per-element features, training samples, and the network's
// correction inside the RHS.
//
// Internal layouts (see fr_api.cu): stage input Us [nu][V][np] (u - u_inf),
// corrected gradient GU [nu][3][V][np], both with the element index
// fastest.  The C ABI's features and network outputs are row-major per
// element: X[e][f], f = v nu + j (state) then 5 nu + m 5 nu + v nu + j
// (gradient); Y[e][v nu + j].  Inside the RHS the network runs
// feature-major on the tensor cores (X[f][e], Y[v nu + j][e] over the padded
// element count): the same values, laid out as the FR state.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"
#include "fr_mlp.h"

namespace fr {
namespace {

// X[e][f] for 32 elements x 32 features per block (tile transpose)
template <typename T>
__global__ void k_features(int nu, int64_t ne, int64_t np, const T *__restrict__ Us, const T *__restrict__ GU,
                           float *__restrict__ X) {
    __shared__ float tile[32][33];
    const int nin = 20 * nu, nv = 5 * nu;
    const int64_t e0 = (int64_t)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int f = f0 + k;
        const int64_t e = e0 + tx;
        float v = 0.f;
        if (f < nin && e < ne) {
            if (f < nv) {
                const int var = f / nu, j = f % nu;
                v = (float)Us[((int64_t)j * 5 + var) * np + e];
            } else {
                const int r = f - nv, m = r / nv, var = (r % nv) / nu, j = r % nu;
                v = (float)GU[(((int64_t)j * 3 + m) * 5 + var) * np + e];
            }
        }
        tile[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t e = e0 + k;
        const int f = f0 + tx;
        if (e < ne && f < nin) X[e * nin + f] = tile[tx][k];
    }
}

// X[f][e] (feature-major, np columns; zero past ne): a coalesced copy
template <typename T>
__global__ void k_features_fm(int nu, int64_t ne, int64_t np, const T *__restrict__ Us, const T *__restrict__ GU,
                              float *__restrict__ X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int f = blockIdx.y, nv = 5 * nu;
    float v = 0.f;
    if (e < ne) {
        if (f < nv) {
            const int var = f / nu, j = f % nu;
            v = (float)Us[((int64_t)j * 5 + var) * np + e];
        } else {
            const int r = f - nv, m = r / nv, var = (r % nv) / nu, j = r % nu;
            v = (float)GU[(((int64_t)j * 3 + m) * 5 + var) * np + e];
        }
    }
    X[(int64_t)f * np + e] = v;
}

struct Scale5 {
    double s[5];
};

// out[r][i] = sum_j R[i][j] in[r][j] over rows r = (e, v) of one type's
// public block
__global__ void k_transfer(int64_t rows, int nto, int nfrom, const double *__restrict__ R,
                           const double *__restrict__ in, double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows * nto) return;
    const int64_t r = k / nto;
    const int i = (int)(k % nto);
    const double *a = R + (int64_t)i * nfrom, *b = in + r * nfrom;
    double s = 0.0;
    for (int j = 0; j < nfrom; ++j) s = fma(a[j], b[j], s);
    out[k] = s;
}

// over one type's public block (i = (e, v, j)): t = inv_scale_v (a - b) as
// float, ss[v] += sum (a - b)^2
__global__ void k_target(int64_t n, int nu, const double *__restrict__ a, const double *__restrict__ b,
                         Scale5 inv_scale, float *__restrict__ t, double *__restrict__ ss) {
    __shared__ double sh[8][5];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double q[5] = {0, 0, 0, 0, 0};
    if (i < n) {
        const int v = (int)((i / nu) % 5);
        const double d = a[i] - b[i];
        if (t) t[i] = (float)(inv_scale.s[v] * d);
        q[v] = d * d;
    }
    if (!ss) return;
#pragma unroll
    for (int v = 0; v < 5; ++v)
        for (int o = 16; o > 0; o >>= 1) q[v] += __shfl_down_sync(0xffffffffu, q[v], o);
    if ((threadIdx.x & 31) == 0)
        for (int v = 0; v < 5; ++v) sh[threadIdx.x >> 5][v] = q[v];
    __syncthreads();
    if (threadIdx.x < 5) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w][threadIdx.x];
        atomicAdd(ss + threadIdx.x, tot);
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace api {

// features of type t from the stage input and the gradient buffer
template <typename T>
cudaError_t launch_features(const DevType &D, const T *in, float *X, cudaStream_t s) {
    dim3 grid(nblk(D.ne, 32), nblk(20 * D.nu, 32));
    k_features<T><<<grid, 256, 0, s>>>(D.nu, D.ne, D.np, in, (const T *)D.GU, X);
    return cudaGetLastError();
}

// features (feature-major) and the three layers on the tensor cores with
// the weight images packed by fr_closure_set, the last writing the RHS
// correction rfs + scale * y in the FR layout: 4 launches
template <typename T>
int closure_apply(fr_ctx *c, int t, const T *in, cudaStream_t s) {
    DevType &D = c->T[t];
    const int nin = 20 * D.nu, nout = 5 * D.nu;
    cudaError_t e = launch(
        c, K_CLOSURE, s,
        [&]() -> cudaError_t {
            k_features_fm<T><<<dim3(nblk(D.np, 256), (unsigned)nin), 256, 0, s>>>(D.nu, D.ne, D.np, in,
                                                                                  (const T *)D.GU, D.cl_X);
            cudaError_t r = cudaGetLastError();
            if (r != cudaSuccess) return r;
            MlpWs w = mlp_ws(nin, D.cl_nh, nout, D.np, D.cl_ws);
            for (int k = 0; k < 3; ++k) w.op[k] = D.cl_op[k];
            ClosureOut co;
            co.add = D.cl_add;
            co.rfs = D.Rfs;
            co.nu = D.nu;
            co.ne = D.ne;
            for (int v = 0; v < 5; ++v) co.scale[v] = D.cl_scale[v];
            return mlp_forward_fm(nin, D.cl_nh, nout, D.np, D.cl_X, D.cl_P, D.cl_Y, w, false, c->tc_err, s, &co);
        },
        4);
    return cuda_check(e, "closure");
}

template int closure_apply<float>(fr_ctx *, int, const float *, cudaStream_t);
template int closure_apply<double>(fr_ctx *, int, const double *, cudaStream_t);

namespace {

// transfer matrices from order p_from into `to` (cached for one p_from)
int ensure_transfer(fr_ctx *to, int p_from) {
    if (to->tr_from == p_from) return FR_OK;
    for (int t = 0; t < NT; ++t) {
        if (!to->T[t].present) continue;
        std::vector<double> R;
        std::string err;
        int rc = build_transfer(t, p_from, to->order, R, err);
        if (rc) return set_err(rc, err);
        if (!to->tr[t]) {
            const size_t bytes = (size_t)nupts_of(t, 4) * nupts_of(t, 4) * sizeof(double);
            void *p = nullptr;
            if ((rc = dev_alloc_bytes(to, &p, bytes))) return rc;
            to->tr[t] = (double *)p;
        }
        if ((rc = cuda_check(cudaMemcpy(to->tr[t], R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice),
                             "transfer upload")))
            return rc;
    }
    to->tr_from = p_from;
    return FR_OK;
}

int check_pair(const fr_ctx *a, const fr_ctx *b) {
    if (!a || !b) return set_err(FR_ERR_ARG, "null context");
    for (int t = 0; t < NT; ++t)
        if (a->T[t].ne != b->T[t].ne) return set_err(FR_ERR_ARG, "contexts have different element counts");
    return FR_OK;
}

int transfer_state(const fr_ctx *from, fr_ctx *to, const double *u, double *out, cudaStream_t s) {
    int rc;
    if ((rc = check_pair(from, to))) return rc;
    if (!u || !out) return set_err(FR_ERR_ARG, "null state pointer");
    if ((rc = ensure_transfer(to, from->order))) return rc;
    size_t off_f = 0, off_t = 0;
    for (int t = 0; t < NT; ++t) {
        const DevType &D = to->T[t];
        if (!D.present) continue;
        const int nf = from->T[t].nu, nt = D.nu;
        const int64_t rows = D.ne * 5;
        k_transfer<<<nblk(rows * nt, 256), 256, 0, s>>>(rows, nt, nf, to->tr[t], u + off_f, out + off_t);
        if ((rc = cuda_check(cudaGetLastError(), "transfer"))) return rc;
        off_f += (size_t)rows * nf;
        off_t += (size_t)rows * nt;
    }
    return FR_OK;
}

template <typename T>
int features_impl(fr_ctx *c, const double *u, int etype, float *X, cudaStream_t s) {
    const Phys ph = phys_of(c);
    size_t off = 0;
    T *in[NT] = {};
    int rc;
    for (int t = 0; t < NT; ++t) {
        DevType &D = c->T[t];
        if (!D.present) continue;
        if ((rc = cuda_check(launch_pub_to_int<T>(D.nu, D.ne, D.np, u + off, nullptr, s, (T *)D.Us, ph.uref),
                             "features layout in")))
            return rc;
        in[t] = (T *)D.Us;
        off += (size_t)D.ne * 5 * D.nu;
    }
    if ((rc = front_stages<T>(c, in, s))) return rc;
    return cuda_check(launch_features<T>(c->T[etype], in[etype], X, s), "features");
}

int check_closure_ctx(const fr_ctx *c, int etype) {
    if (!c) return set_err(FR_ERR_ARG, "null context");
    if (etype < FR_ETYPE_TET || etype > FR_ETYPE_HEX) return set_err(FR_ERR_ARG, "etype must be 0, 1 or 2");
    if (!c->prm.viscous) return set_err(FR_ERR_UNSUPPORTED, "the closure needs a Navier-Stokes context");
    if (!c->T[etype].present) return set_err(FR_ERR_ARG, "no elements of this type");
    return FR_OK;
}

}  // namespace
}  // namespace api
}  // namespace fr

using namespace fr;
using namespace fr::api;

extern "C" {

int fr_transfer(int etype, int p_from, int p_to, double *out, int64_t *rows, int64_t *cols) {
    if (!rows || !cols) return set_err(FR_ERR_ARG, "null argument");
    if (etype < FR_ETYPE_TET || etype > FR_ETYPE_HEX || p_from < 1 || p_from > 4 || p_to < 1 || p_to > 4)
        return set_err(FR_ERR_ARG, "etype must be 0/1/2 and orders 1..4");
    *rows = nupts_of(etype, p_to);
    *cols = nupts_of(etype, p_from);
    if (!out) return FR_OK;
    std::vector<double> R;
    std::string err;
    int rc = build_transfer(etype, p_from, p_to, R, err);
    if (rc) return set_err(rc, err);
    std::copy(R.begin(), R.end(), out);
    return FR_OK;
}

int fr_transfer_state(const fr_ctx *from, fr_ctx *to, const double *u_from_dev, double *u_to_dev, void *stream) {
    return transfer_state(from, to, u_from_dev, u_to_dev, (cudaStream_t)stream);
}

int fr_closure_features(fr_ctx *c, const double *u_dev, int etype, float *x_dev, void *stream) {
    int rc;
    if ((rc = check_closure_ctx(c, etype))) return rc;
    if (!u_dev || !x_dev) return set_err(FR_ERR_ARG, "null pointer");
    const cudaStream_t s = (cudaStream_t)stream;
    return is_f32(c) ? features_impl<float>(c, u_dev, etype, x_dev, s)
                                       : features_impl<double>(c, u_dev, etype, x_dev, s);
}

int fr_closure_sample(fr_ctx *hi, fr_ctx *lo, const double *u_hi_dev, const double *u_lo_dev, int etype,
                      const double *inv_scale, float *x_dev, float *t_dev, double *ss_dev, void *stream) {
    int rc;
    if ((rc = check_closure_ctx(lo, etype)) || (rc = check_pair(hi, lo))) return rc;
    if (!u_hi_dev) return set_err(FR_ERR_ARG, "null state pointer");
    const cudaStream_t s = (cudaStream_t)stream;
    const int64_t nlo = ndof_of(lo), nhi = ndof_of(hi);
    if (!lo->smp_u) {
        void *p[3];
        for (int k = 0; k < 3; ++k)
            if ((rc = dev_alloc_bytes(lo, &p[k], (size_t)nlo * sizeof(double)))) return rc;
        lo->smp_u = (double *)p[0];
        lo->smp_r = (double *)p[1];
        lo->smp_rr = (double *)p[2];
    }
    if (lo->smp_rhi_cap < nhi) {
        void *p = nullptr;
        if ((rc = dev_alloc_bytes(lo, &p, (size_t)nhi * sizeof(double)))) return rc;
        lo->smp_rhi = (double *)p;
        lo->smp_rhi_cap = nhi;
    }
    // RHS_hi and its projection
    rc = is_f32(hi) ? rhs_public<float>(hi, u_hi_dev, lo->smp_rhi, s)
                                      : rhs_public<double>(hi, u_hi_dev, lo->smp_rhi, s);
    if (rc) return rc;
    if ((rc = transfer_state(hi, lo, lo->smp_rhi, lo->smp_rr, s))) return rc;
    // RHS_lo (without a closure) of u_lo, or of the projected state
    const double *ulo = u_lo_dev;
    if (!ulo) {
        if ((rc = transfer_state(hi, lo, u_hi_dev, lo->smp_u, s))) return rc;
        ulo = lo->smp_u;
    }
    int on[NT];
    for (int t = 0; t < NT; ++t) {
        on[t] = lo->T[t].cl_on;
        lo->T[t].cl_on = 0;
    }
    rc = is_f32(lo) ? rhs_public<float>(lo, ulo, lo->smp_r, s)
                                      : rhs_public<double>(lo, ulo, lo->smp_r, s);
    for (int t = 0; t < NT; ++t) lo->T[t].cl_on = on[t];
    if (rc) return rc;
    // the features of the state RHS_lo just ran on (its stage input and
    // gradient are still in the context's buffers)
    const DevType &D = lo->T[etype];
    if (x_dev) {
        rc = is_f32(lo) ? cuda_check(launch_features<float>(D, (const float *)D.Us, x_dev, s), "features")
                                          : cuda_check(launch_features<double>(D, (const double *)D.Us, x_dev, s), "features");
        if (rc) return rc;
    }
    if (t_dev || ss_dev) {
        size_t off = 0;  // start of this type's block in the public layout
        for (int t = 0; t < etype; ++t)
            if (lo->T[t].present) off += (size_t)lo->T[t].ne * 5 * lo->T[t].nu;
        const int64_t n = D.ne * 5 * D.nu;
        Scale5 isc;
        for (int v = 0; v < 5; ++v) isc.s[v] = inv_scale ? inv_scale[v] : 1.0;
        k_target<<<nblk(n, 256), 256, 0, s>>>(n, D.nu, lo->smp_rr + off, lo->smp_r + off, isc, t_dev, ss_dev);
        if ((rc = cuda_check(cudaGetLastError(), "target"))) return rc;
    }
    return FR_OK;
}

int fr_closure_set(fr_ctx *c, int etype, const float *params_dev, int nh, const double *out_scale) {
    int rc;
    if ((rc = check_closure_ctx(c, etype))) return rc;
    DevType &D = c->T[etype];
    if (!params_dev) {
        D.cl_on = 0;
        return FR_OK;
    }
    if (nh <= 0 || nh > 4096) return set_err(FR_ERR_ARG, "hidden width must be in 1..4096");
    if (!out_scale) return set_err(FR_ERR_ARG, "null output scales");
    const int nin = 20 * D.nu, nout = 5 * D.nu;
    if (nh > 256 || nout > 256)
        return set_err(FR_ERR_UNSUPPORTED, "the tensor-core network layers take at most 256 hidden units and "
                                           "256 outputs");
    const MlpLayout L = mlp_layout(nin, nh, nout);
    if (D.cl_cap_nh < nh) {
        void *p[4];
        const size_t sz[4] = {(size_t)L.n * sizeof(float), (size_t)D.np * nin * sizeof(float),
                              (size_t)D.np * nout * sizeof(float),
                              (size_t)mlp_workspace_floats(nin, nh, nout, D.np) * sizeof(float)};
        for (int k = 0; k < 4; ++k)
            if ((rc = dev_alloc_bytes(c, &p[k], sz[k]))) return rc;
        D.cl_P = (float *)p[0];
        D.cl_X = (float *)p[1];
        D.cl_Y = (float *)p[2];
        D.cl_ws = (float *)p[3];
        if (!D.cl_add) {
            void *q = nullptr;
            if ((rc = dev_alloc_bytes(c, &q, (size_t)D.nu * 5 * D.np * sizeof(double)))) return rc;
            D.cl_add = (double *)q;
        }
        D.cl_cap_nh = nh;
    }
    if ((rc = cuda_check(cudaMemcpy(D.cl_P, params_dev, (size_t)L.n * sizeof(float), cudaMemcpyDeviceToDevice),
                         "closure parameters")))
        return rc;
    // the bf16 weight images of the three layers (kept until the next set)
    MlpWs w = mlp_ws(nin, nh, nout, D.np, D.cl_ws);
    if ((rc = cuda_check(mlp_pack_forward(nin, nh, nout, D.cl_P, w, 0), "closure weight images"))) return rc;
    for (int k = 0; k < 3; ++k) D.cl_op[k] = w.op[k];
    if ((rc = cuda_check(cudaDeviceSynchronize(), "closure set"))) return rc;
    D.cl_nh = nh;
    for (int v = 0; v < 5; ++v) D.cl_scale[v] = out_scale[v];
    D.cl_on = 1;
    return FR_OK;
}

int64_t fr_mlp_nparams(int nin, int nh, int nout) {
    if (nin <= 0 || nh <= 0 || nout <= 0) return 0;
    return mlp_layout(nin, nh, nout).n;
}

int64_t fr_mlp_workspace(int nin, int nh, int nout, int64_t n) {
    if (nin <= 0 || nh <= 0 || nout <= 0 || n <= 0) return 0;
    return mlp_workspace_floats(nin, nh, nout, n);
}

namespace {
int check_mlp(int nin, int nh, int nout, int64_t n, const float *ws) {
    if (nin <= 0 || nh <= 0 || nout <= 0 || n <= 0 || n > (1LL << 30)) return set_err(FR_ERR_ARG, "invalid sizes");
    if (nh > 256 || nout > 256)
        return set_err(FR_ERR_UNSUPPORTED, "the tensor-core layers take at most 256 hidden units and 256 outputs");
    if (tc_hi_image_bytes(nh, std::max(nin, nh)) > 196608)
        return set_err(FR_ERR_UNSUPPORTED, "a layer's bf16 weight image exceeds 192 KB of shared memory");
    if ((uintptr_t)ws % 16) return set_err(FR_ERR_ARG, "the workspace must be 16-byte aligned");
    return FR_OK;
}
}  // namespace

int fr_mlp_forward(int nin, int nh, int nout, int64_t n, const float *x, const float *P, float *y, float *ws,
                   void *stream) {
    int rc;
    if ((rc = check_mlp(nin, nh, nout, n, ws))) return rc;
    if (!x || !P || !y || !ws) return set_err(FR_ERR_ARG, "null pointer");
    return cuda_check(mlp_forward(nin, nh, nout, n, x, P, y, ws, (cudaStream_t)stream), "mlp forward");
}

int fr_mlp_grad(int nin, int nh, int nout, int64_t n, const float *x, const float *t, const float *P, float *g,
                float *loss, float *ws, void *stream) {
    int rc;
    if ((rc = check_mlp(nin, nh, nout, n, ws))) return rc;
    if (!x || !t || !P || !g || !loss || !ws) return set_err(FR_ERR_ARG, "null pointer");
    return cuda_check(mlp_grad(nin, nh, nout, n, x, t, P, g, loss, ws, (cudaStream_t)stream), "mlp grad");
}

int fr_mlp_adam(int64_t n, float *P, const float *g, float *m, float *v, int step, float lr, void *stream) {
    if (n <= 0 || step < 1) return set_err(FR_ERR_ARG, "invalid size or step");
    if (!P || !g || !m || !v) return set_err(FR_ERR_ARG, "null pointer");
    return cuda_check(mlp_adam(n, P, g, m, v, step, lr, (cudaStream_t)stream), "mlp adam");
}

}  // extern "C"
