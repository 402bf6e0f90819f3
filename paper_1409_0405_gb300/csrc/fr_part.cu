// Partitioned execution (Sec. 2.5: ranks exchange the interface data of
// their partitions; Sec. 5.2: weighted partitioning of mixed meshes).
//
// A partitioned mesh is a set of partition contexts on the current device,
// each a full FR context of its own elements whose cut interface pairs read
// the remote side from a halo (see host_part.cpp).  Per RHS evaluation the
// partitions exchange, through device-local buffers, what their neighbours
// read across the cut faces:
//   after the interpolation u_f = M0 u        the 5 values of each point,
//   after M0 on the gradients (Navier-Stokes) the 15 gradient values,
// each exchange a pack kernel on the source (its flux points in the plan's
// order, into a contiguous send buffer) followed by a copy into the
// destination's halo slots (on several GPUs, the point-to-point transfer).
// The halo is laid out as the receive buffer, so there is no unpack step.
// The face kernels then compute every cut pair with the same operands and
// the same global pair data as the unpartitioned mesh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fr_ctx.h"
#include "fr_part.h"

using namespace fr;
using namespace fr::api;

struct fr_part {
    int nparts = 0, order = 0;
    fr_params prm{};
    std::vector<fr_ctx *> P;
    std::vector<std::vector<int64_t>> elems[NT];  // elems[t][p]: global ids, increasing
    struct DSeg {
        int src = 0, dst = 0;
        int64_t n = 0, off = 0;
        int *t = nullptr, *f = nullptr, *e = nullptr;
        void *buf = nullptr;  // 15 n values of the arithmetic type
    };
    std::vector<DSeg> segs;
    std::vector<void *> allocs;
    int64_t launches = 0;  // pack kernels (the partitions count their own)
    // fr_part_rhs scratch: per partition its part of u and r in the
    // partition's own public layout, and per (partition, type) the global
    // element ids (device); allocated by the first fr_part_rhs
    std::vector<double *> pu, pr;
    std::vector<int64_t *> gid;  // [p * NT + t]
    bool scratch_ready = false;
};

namespace {

constexpr int V = FR_NVARS;

template <typename T>
__global__ void k_pack(int64_t n, const int *__restrict__ t, const int *__restrict__ f, const int *__restrict__ e,
                       const FieldsT<T> F, int grad, T *__restrict__ buf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ti = t[i];
    const int64_t np = F.np[ti];
    if (grad) {
        const T *src = F.GUF[ti] + (int64_t)f[i] * 3 * V * np + e[i];
#pragma unroll
        for (int q = 0; q < 3 * V; ++q) buf[q * n + i] = src[q * np];
    } else {
        const T *src = F.UF[ti] + (int64_t)f[i] * V * np + e[i];
#pragma unroll
        for (int v = 0; v < V; ++v) buf[v * n + i] = src[v * np];
    }
}

// dst[i][k] = src[gid[i]][k] (gather) or the reverse (scatter), blocks of blk values
__global__ void k_blocks(int64_t n, int64_t blk, const int64_t *__restrict__ gid, const double *__restrict__ src,
                         double *__restrict__ dst, int scatter) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * blk) return;
    const int64_t i = idx / blk, k = idx - i * blk;
    if (scatter)
        dst[gid[i] * blk + k] = src[idx];
    else
        dst[idx] = src[gid[i] * blk + k];
}

int64_t grid_of(int64_t n, int b) { return (n + b - 1) / b; }

template <typename T>
int exchange(fr_part *pp, bool grad, cudaStream_t s) {
    const int rows = grad ? 3 * V : V;
    for (auto &sg : pp->segs) {
        fr_ctx *Q = pp->P[sg.src], *D = pp->P[sg.dst];
        const FieldsT<T> F = fields_of<T>(Q);
        k_pack<T><<<(unsigned)grid_of(sg.n, 256), 256, 0, s>>>(sg.n, sg.t, sg.f, sg.e, F, grad ? 1 : 0, (T *)sg.buf);
        ++pp->launches;
        int rc = cuda_check(cudaGetLastError(), "halo pack");
        if (rc) return rc;
        T *dst = (T *)(grad ? D->GUF_h : D->UF_h) + sg.off;
        rc = cuda_check(cudaMemcpy2DAsync(dst, (size_t)D->nhalo_p * sizeof(T), sg.buf, (size_t)sg.n * sizeof(T),
                                          (size_t)sg.n * sizeof(T), (size_t)rows, cudaMemcpyDeviceToDevice, s),
                        "halo copy");
        if (rc) return rc;
    }
    return FR_OK;
}

template <typename T>
void stage_inputs(fr_ctx *c, T *in[NT]) {
    for (int t = 0; t < NT; ++t) in[t] = c->T[t].present ? (T *)c->T[t].Us : nullptr;
}

// one RHS over every partition with the two exchanges; rk as in rhs_internal
template <typename T>
int part_rhs_stage(fr_part *pp, const RKStage *rk, cudaStream_t s) {
    int rc;
    T *in[NT];
    for (fr_ctx *c : pp->P) {
        stage_inputs<T>(c, in);
        if ((rc = phase_interp<T>(c, in, s))) return rc;
    }
    if ((rc = exchange<T>(pp, false, s))) return rc;
    if (pp->prm.viscous) {
        for (fr_ctx *c : pp->P) {
            stage_inputs<T>(c, in);
            if ((rc = phase_grad<T>(c, in, s))) return rc;
        }
        if ((rc = exchange<T>(pp, true, s))) return rc;
    }
    for (fr_ctx *c : pp->P) {
        stage_inputs<T>(c, in);
        if ((rc = phase_div<T>(c, in, rk, s))) return rc;
    }
    return FR_OK;
}

template <typename T>
int part_center(fr_part *pp, cudaStream_t s) {
    for (fr_ctx *c : pp->P) {
        const Phys ph = phys_of(c);
        for (int t = 0; t < NT; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            int rc = cuda_check(launch_center<T>(D.nu, D.np, D.U, (T *)D.Us, ph.uref, s), "centre");
            if (rc) return rc;
        }
    }
    return FR_OK;
}

template <typename T>
int part_step_impl(fr_part *pp, double dt, int nsteps, cudaStream_t s) {
    if (nsteps <= 0) return FR_OK;
    const double ca[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
    const double cs[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
    int rc;
    if ((rc = part_center<T>(pp, s))) return rc;
    for (int it = 0; it < nsteps; ++it)
        for (int st = 0; st < 4; ++st) {
            RKStage rk{ca[st], cs[st], st == 0, st == 3};
            if ((rc = part_rhs_stage<T>(pp, &rk, s))) return rc;
        }
    return FR_OK;
}

int64_t type_base(const fr_part *pp, int t) {
    // offset of type t's block in the global public layout
    int64_t off = 0;
    for (int k = 0; k < t; ++k) {
        int64_t ne = 0;
        for (auto &v : pp->elems[k]) ne += (int64_t)v.size();
        off += ne * V * nupts_of(k, pp->order);
    }
    return off;
}

int ensure_rhs_scratch(fr_part *pp) {
    if (pp->scratch_ready) return FR_OK;
    const int n = pp->nparts;
    pp->pu.assign(n, nullptr);
    pp->pr.assign(n, nullptr);
    pp->gid.assign((size_t)n * NT, nullptr);
    for (int p = 0; p < n; ++p) {
        const int64_t nd = ndof_of(pp->P[p]);
        for (double **q : {&pp->pu[p], &pp->pr[p]}) {
            if (dev_malloc((void **)q, (size_t)nd * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                *q = nullptr;
                return set_err(FR_ERR_NOMEM, "partition RHS scratch");
            }
            pp->allocs.push_back(*q);
        }
        for (int t = 0; t < NT; ++t) {
            const auto &el = pp->elems[t][p];
            if (el.empty()) continue;
            int64_t *g = nullptr;
            if (dev_malloc((void **)&g, el.size() * sizeof(int64_t)) != cudaSuccess) {
                cudaGetLastError();
                return set_err(FR_ERR_NOMEM, "partition element map");
            }
            pp->allocs.push_back(g);
            pp->gid[(size_t)p * NT + t] = g;
            int rc = cuda_check(cudaMemcpy(g, el.data(), el.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                                "element map upload");
            if (rc) return rc;
        }
    }
    pp->scratch_ready = true;
    return FR_OK;
}

template <typename T>
int part_rhs_impl(fr_part *pp, const double *u_dev, double *r_dev, cudaStream_t s) {
    int rc;
    if ((rc = ensure_rhs_scratch(pp))) return rc;
    for (int p = 0; p < pp->nparts; ++p) {
        fr_ctx *c = pp->P[p];
        const Phys ph = phys_of(c);
        int64_t off = 0;
        for (int t = 0; t < NT; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            const int64_t blk = (int64_t)V * D.nu;
            k_blocks<<<(unsigned)grid_of(D.ne * blk, 256), 256, 0, s>>>(
                D.ne, blk, pp->gid[(size_t)p * NT + t], u_dev + type_base(pp, t), pp->pu[p] + off, 0);
            if ((rc = cuda_check(cudaGetLastError(), "partition gather"))) return rc;
            if ((rc = cuda_check(launch_pub_to_int<T>(D.nu, D.ne, D.np, pp->pu[p] + off, nullptr, s, (T *)D.Us,
                                                      ph.uref),
                                 "rhs layout in")))
                return rc;
            off += D.ne * blk;
        }
    }
    if ((rc = part_rhs_stage<T>(pp, nullptr, s))) return rc;
    for (int p = 0; p < pp->nparts; ++p) {
        fr_ctx *c = pp->P[p];
        int64_t off = 0;
        for (int t = 0; t < NT; ++t) {
            DevType &D = c->T[t];
            if (!D.present) continue;
            const int64_t blk = (int64_t)V * D.nu;
            if ((rc = cuda_check(launch_int_to_pub<T>(D.nu, D.ne, D.np, (const T *)D.R, pp->pr[p] + off, s),
                                 "rhs layout out")))
                return rc;
            k_blocks<<<(unsigned)grid_of(D.ne * blk, 256), 256, 0, s>>>(
                D.ne, blk, pp->gid[(size_t)p * NT + t], pp->pr[p] + off, r_dev + type_base(pp, t), 1);
            if ((rc = cuda_check(cudaGetLastError(), "partition scatter"))) return rc;
            off += D.ne * blk;
        }
    }
    return FR_OK;
}

// host: a partition's part of a global public-layout state and back
void part_slice(const fr_part *pp, int p, const double *g, std::vector<double> &loc, bool to_global,
                double *gout) {
    size_t off = 0;
    for (int t = 0; t < NT; ++t) {
        const auto &el = pp->elems[t][p];
        if (el.empty()) continue;
        const size_t blk = (size_t)V * nupts_of(t, pp->order);
        const int64_t base = type_base(pp, t);
        for (size_t i = 0; i < el.size(); ++i) {
            double *gp = (to_global ? gout : const_cast<double *>(g)) + base + (size_t)el[i] * blk;
            if (to_global)
                std::memcpy(gp, loc.data() + off + i * blk, blk * sizeof(double));
            else
                std::memcpy(loc.data() + off + i * blk, gp, blk * sizeof(double));
        }
        off += el.size() * blk;
    }
}

void part_free(fr_part *pp) {
    if (!pp) return;
    for (fr_ctx *c : pp->P) fr_destroy(c);
    for (void *q : pp->allocs) dev_free(q);
    delete pp;
}

int part_create_impl(const fr_mesh *mesh, int order, const fr_params *prm, int nparts, const int32_t *part,
                     fr_part *pp) {
    int rc;
    if ((rc = check_params(order, prm))) return rc;
    if (nparts < 1 || nparts > 4096) return set_err(FR_ERR_ARG, "nparts must be in 1..4096");
    HostSetup h;
    if ((rc = host_setup(mesh, order, h))) return rc;
    std::string err;
    std::vector<int32_t> own;
    if (!part) {
        const double w[NT] = {1.0, 2.0, 3.0};
        if ((rc = partition_rcb(mesh, nparts, w, own, err))) return set_err(rc, err);
        part = own.data();
    }
    PartPlan pl;
    if ((rc = build_part_plan(h, nparts, part, pl, err))) return set_err(rc, err);
    pp->nparts = nparts;
    pp->order = order;
    pp->prm = *prm;
    for (int t = 0; t < NT; ++t) pp->elems[t] = pl.elems[t];
    for (int p = 0; p < nparts; ++p) {
        fr_ctx *c = new (std::nothrow) fr_ctx();
        if (!c) return set_err(FR_ERR_NOMEM, "host allocation");
        pp->P.push_back(c);
        const auto &L = pl.local[p];
        if ((rc = device_setup(c, order, prm, h.ops, L.geo, L.faces, L.nhalo))) return rc;
    }
    const size_t es = f32_storage(prm->precision) ? sizeof(float) : sizeof(double);
    for (const auto &sg : pl.segs) {
        fr_part::DSeg d;
        d.src = sg.src;
        d.dst = sg.dst;
        d.n = (int64_t)sg.t.size();
        d.off = sg.off;
        int **dst[3] = {&d.t, &d.f, &d.e};
        const std::vector<int> *src[3] = {&sg.t, &sg.f, &sg.e};
        for (int k = 0; k < 3; ++k) {
            if (dev_malloc((void **)dst[k], src[k]->size() * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return set_err(FR_ERR_NOMEM, "exchange plan");
            }
            pp->allocs.push_back(*dst[k]);
            if ((rc = cuda_check(cudaMemcpy(*dst[k], src[k]->data(), src[k]->size() * sizeof(int),
                                            cudaMemcpyHostToDevice),
                                 "exchange plan upload")))
                return rc;
        }
        if (dev_malloc(&d.buf, (size_t)3 * V * d.n * es) != cudaSuccess) {
            cudaGetLastError();
            return set_err(FR_ERR_NOMEM, "exchange buffer");
        }
        pp->allocs.push_back(d.buf);
        pp->segs.push_back(d);
    }
    return cuda_check(cudaDeviceSynchronize(), "fr_part_create sync");
}

}  // namespace

extern "C" {

int fr_partition(const fr_mesh *mesh, int nparts, const double *weights, int32_t *part) {
    if (!mesh || !part || nparts < 1) return set_err(FR_ERR_ARG, "invalid partition arguments");
    if (mesh->n_nodes <= 0 || !mesh->xyz || mesh->n_tet < 0 || mesh->n_pri < 0 || mesh->n_hex < 0 ||
        (mesh->n_tet && !mesh->tet) || (mesh->n_pri && !mesh->pri) || (mesh->n_hex && !mesh->hex))
        return set_err(FR_ERR_ARG, "invalid mesh");
    double w[NT] = {1.0, 2.0, 3.0};
    if (weights)
        for (int t = 0; t < NT; ++t) {
            if (!(weights[t] > 0.0)) return set_err(FR_ERR_ARG, "weights must be positive");
            w[t] = weights[t];
        }
    std::vector<int32_t> out;
    std::string err;
    int rc;
    try {
        rc = partition_rcb(mesh, nparts, w, out, err);
    } catch (const std::bad_alloc &) {
        return set_err(FR_ERR_NOMEM, "host allocation");
    }
    if (rc) return set_err(rc, err);
    std::copy(out.begin(), out.end(), part);
    return FR_OK;
}

int fr_part_plan(const fr_mesh *mesh, int order, int nparts, const int32_t *part, int rank, int64_t *counts,
                 int32_t *send_pts, int32_t *halo_pts) {
    if (!mesh || !part || !counts || nparts < 1 || rank < 0 || rank >= nparts)
        return set_err(FR_ERR_ARG, "invalid plan arguments");
    try {
        HostSetup h;
        int rc;
        if ((rc = host_setup(mesh, order, h))) return rc;
        PartPlan pl;
        std::string err;
        if ((rc = build_part_plan(h, nparts, part, pl, err))) return set_err(rc, err);
        for (int q = 0; q < nparts; ++q) counts[q] = 0;
        // sends of `rank` grouped by destination, halo slots of `rank`
        // grouped by source (both in increasing partner order)
        int64_t ks = 0, kh = 0;
        for (int q = 0; q < nparts; ++q)
            for (const auto &sg : pl.segs) {
                if (sg.src == rank && sg.dst == q) {
                    counts[q] = (int64_t)sg.t.size();
                    for (size_t i = 0; i < sg.t.size() && send_pts; ++i, ++ks) {
                        send_pts[3 * ks] = sg.t[i];
                        send_pts[3 * ks + 1] = sg.e[i];
                        send_pts[3 * ks + 2] = sg.f[i];
                    }
                }
                if (sg.dst == rank && sg.src == q && halo_pts)
                    for (size_t i = 0; i < sg.t.size(); ++i, ++kh) {
                        halo_pts[3 * kh] = sg.t[i];
                        halo_pts[3 * kh + 1] = (int32_t)sg.ge[i];
                        halo_pts[3 * kh + 2] = sg.f[i];
                    }
            }
    } catch (const std::bad_alloc &) {
        return set_err(FR_ERR_NOMEM, "host allocation");
    }
    return FR_OK;
}

int fr_part_create(const fr_mesh *mesh, int order, const fr_params *params, int nparts, const int32_t *part,
                   fr_part **out) {
    if (!out) return set_err(FR_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!mesh) return set_err(FR_ERR_ARG, "null mesh");
    fr_part *pp = new (std::nothrow) fr_part();
    if (!pp) return set_err(FR_ERR_NOMEM, "host allocation");
    int rc;
    try {
        rc = part_create_impl(mesh, order, params, nparts, part, pp);
    } catch (const std::bad_alloc &) {
        rc = set_err(FR_ERR_NOMEM, "host allocation during set-up");
    } catch (...) {
        rc = set_err(FR_ERR_ARG, "unexpected exception during set-up");
    }
    if (rc) {
        part_free(pp);
        return rc;
    }
    *out = pp;
    return FR_OK;
}

void fr_part_destroy(fr_part *pp) { part_free(pp); }

int fr_part_info(const fr_part *pp, int64_t *out) {
    if (!pp || !out) return set_err(FR_ERR_ARG, "null argument");
    for (int p = 0; p < pp->nparts; ++p) {
        for (int t = 0; t < NT; ++t) out[4 * p + t] = (int64_t)pp->elems[t][p].size();
        out[4 * p + 3] = pp->P[p]->nhalo;
    }
    return FR_OK;
}

int fr_part_set_state(fr_part *pp, const double *u, void *stream) {
    if (!pp || !u) return set_err(FR_ERR_ARG, "null argument");
    std::vector<double> loc;
    for (int p = 0; p < pp->nparts; ++p) {
        loc.assign((size_t)ndof_of(pp->P[p]), 0.0);
        part_slice(pp, p, u, loc, false, nullptr);
        int rc = fr_set_state(pp->P[p], loc.data(), stream);
        if (rc) return rc;
    }
    return FR_OK;
}

int fr_part_get_state(fr_part *pp, double *u, void *stream) {
    if (!pp || !u) return set_err(FR_ERR_ARG, "null argument");
    std::vector<double> loc;
    for (int p = 0; p < pp->nparts; ++p) {
        loc.assign((size_t)ndof_of(pp->P[p]), 0.0);
        int rc = fr_get_state(pp->P[p], loc.data(), stream);
        if (rc) return rc;
        part_slice(pp, p, nullptr, loc, true, u);
    }
    return FR_OK;
}

int fr_part_rhs(fr_part *pp, const double *u_dev, double *r_dev, void *stream) {
    if (!pp || !u_dev || !r_dev) return set_err(FR_ERR_ARG, "null argument");
    if (u_dev == r_dev) return set_err(FR_ERR_ARG, "u and r may not alias");
    cudaStream_t s = (cudaStream_t)stream;
    return f32_storage(pp->prm.precision) ? part_rhs_impl<float>(pp, u_dev, r_dev, s)
                                        : part_rhs_impl<double>(pp, u_dev, r_dev, s);
}

int fr_part_step(fr_part *pp, double dt, int nsteps, void *stream) {
    if (!pp || nsteps < 0 || !std::isfinite(dt)) return set_err(FR_ERR_ARG, "invalid step arguments");
    int rc;
    for (fr_ctx *c : pp->P)
        if ((rc = step_guard(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = f32_storage(pp->prm.precision) ? part_step_impl<float>(pp, dt, nsteps, s)
                                      : part_step_impl<double>(pp, dt, nsteps, s);
    for (fr_ctx *c : pp->P)
        if (!rc && nsteps > 0) rc = step_check(c, s);
    return rc;
}

int fr_part_reduce(fr_part *pp, double *out, void *stream) {
    if (!pp || !out) return set_err(FR_ERR_ARG, "null argument");
    for (int k = 0; k < 7; ++k) out[k] = 0.0;
    for (fr_ctx *c : pp->P) {
        double o[7];
        int rc = fr_reduce(c, o, stream);
        if (rc && rc != FR_ERR_NONFINITE) return rc;
        for (int k = 0; k < 7; ++k) out[k] += o[k];
    }
    if (out[6] != 0.0) return set_err(FR_ERR_NONFINITE, "non-finite or non-physical state");
    return FR_OK;
}

int fr_part_launches(const fr_part *pp, int64_t *launches) {
    if (!pp || !launches) return set_err(FR_ERR_ARG, "null argument");
    int64_t n = pp->launches;
    for (fr_ctx *c : pp->P) n += c->launches;
    *launches = n;
    return FR_OK;
}

}  // extern "C"
