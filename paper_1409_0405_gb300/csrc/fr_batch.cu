// Batched engine: many independent FR problems (different meshes, element
// mixes and orders) advanced together.
//
// Every operator application of every problem and element type becomes a
// descriptor in a device-resident work list, and the point-wise flux and
// face kernels walk concatenated segments.  Two schedules of an RK stage:
//  * one persistent cooperative launch per stage (fr_stage.cu): all of the
//    stage's work lists, phase after phase, separated by grid-wide barriers
//    with bounded waits (4 launches per RK step);
//  * one grouped launch per operator class (M0, corrected gradient, M0 on
//    gradients, divergence + RK update) and per point-wise pass.
// One RK step (4 stages) is captured in a CUDA graph and replayed.  The
// row-chunk sizes (the tile shapes of the operator blocks), and the grids
// of the grouped launches, are chosen by timing the candidates on the batch
// itself (fr_batch_tune).
//
// The arithmetic of every output is the same as in the per-problem launch
// sequence (same operators, same summation order), so the two agree bit
// for bit; the batch only changes how the work is scheduled.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"

using namespace fr;
using namespace fr::api;

namespace {

template <typename T>
struct Group {
    int mode = 0, rc = 8, grid = 0, maxK = 0, ndesc = 0;
    int64_t total = 0;
    std::vector<GemmArgsT<T>> h;
    std::vector<int> op;  // per descriptor: etype * 64 + order * 4 + operator (0 M0, 1 AGRAD, 2 ADIV)
    GemmArgsT<T> *d = nullptr;
    int64_t *begin = nullptr;
};

template <typename T>
struct Segs {
    std::vector<T> h;
    std::vector<int64_t> hb;
    T *d = nullptr;
    int64_t *begin = nullptr;
    int64_t total = 0;
    int grid = 0;
};

int dev_put(void **p, const void *src, size_t bytes) {
    if (!*p && dev_malloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(FR_ERR_NOMEM, "batch work-list allocation");
    }
    return cuda_check(cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice), "batch work-list upload");
}

}  // namespace

struct BatchBase {
    virtual ~BatchBase() {}
    virtual int tune(cudaStream_t s) = 0;
    virtual int step(const double *dt, int nsteps, int batched, cudaStream_t s) = 0;
    virtual void info(int64_t *out) const = 0;
    virtual int check(cudaStream_t s) = 0;
    virtual int selftest(cudaStream_t s) = 0;
};

struct fr_batch {
    std::vector<fr_ctx *> ctx;
    BatchBase *impl = nullptr;
};

namespace {

template <typename T>
struct BatchImpl : BatchBase {
    fr_batch *b;
    bool viscous, xform;
    Group<T> m0, grad, m0g, div[4];
    Segs<FluxItem<T>> flux;
    Segs<FaceItem<T>> face;
    Segs<CenterItem<T>> center;
    std::vector<double> dt_cur;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int launches_per_step = 0;
    int nsm = 152;
    // the persistent schedule: one plan per RK stage, the barrier words and
    // status of the stage kernel, its co-resident grid; graph_mode is the
    // schedule the instantiated graph holds (1 persistent, 2 grouped)
    StagePlan<T> plan[4];
    unsigned *bar = nullptr;
    int *serr = nullptr;
    int stage_grid_n = 0, graph_mode = 0, launches_grouped = 0;

    explicit BatchImpl(fr_batch *bb) : b(bb) {
        viscous = bb->ctx[0]->prm.viscous != 0;
        xform = viscous && is_f32(bb->ctx[0]);
    }

    // the operators' exact zeros skipped as in the per-problem launches, in
    // chunks of the group's row-chunk size (compressed per etype, order,
    // operator and chunk size, uploaded once)
    struct SpDev {
        int rc = 0, lmax = 0;
        int *off = nullptr, *cols = nullptr;
        T *vals = nullptr;
    };
    std::map<std::pair<int, int>, SpDev> sp_cache;

    const SpDev &sparse_for(int key, int rc) {
        auto it = sp_cache.find({key, rc});
        if (it != sp_cache.end()) return it->second;
        SpDev &d = sp_cache[{key, rc}];
        const int et = key / 64, order = (key / 4) % 16, which = key % 4;
        RefOps ops;
        std::string err;
        if (build_ref_ops(et, order, ops, err)) return d;
        const int nu = ops.nu, nf = ops.nf;
        const std::vector<double> *A[3] = {&ops.M0, &ops.AGRAD, &ops.ADIV};
        const int M[3] = {nf, 3 * nu, nu}, K1[3] = {nu, nu, 3 * nu}, K2[3] = {0, nf, nf};
        SparseOp sp;
        if (!sparse_pack(A[which]->data(), M[which], K1[which], K2[which], which == 1, sp, rc)) return d;
        std::vector<T> v(sp.vals.begin(), sp.vals.end());
        if (dev_put((void **)&d.off, sp.off.data(), sizeof(int) * sp.off.size()) ||
            dev_put((void **)&d.cols, sp.cols.data(), sizeof(int) * sp.cols.size()) ||
            dev_put((void **)&d.vals, v.data(), sizeof(T) * v.size())) {
            dev_free(d.off);
            dev_free(d.cols);
            dev_free(d.vals);
            d = SpDev();
            return d;
        }
        d.rc = sp.rc;
        d.lmax = sp.lmax;
        return d;
    }

    ~BatchImpl() override {
        for (auto &kv : sp_cache) {
            dev_free(kv.second.off);
            dev_free(kv.second.cols);
            dev_free(kv.second.vals);
        }
        auto fg = [](Group<T> &g) {
            dev_free(g.d);
            dev_free(g.begin);
        };
        fg(m0);
        fg(grad);
        fg(m0g);
        for (auto &g : div) fg(g);
        dev_free(flux.d);
        dev_free(flux.begin);
        dev_free(face.d);
        dev_free(face.begin);
        dev_free(center.d);
        dev_free(center.begin);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        dev_free(bar);
        dev_free(serr);
    }

    // prefix sums of blocks for the group's row-chunk size, uploaded
    int upload_group(Group<T> &g) {
        std::vector<int64_t> bg(g.h.size());
        int64_t tot = 0;
        g.maxK = 0;
        for (size_t i = 0; i < g.h.size(); ++i) {
            bg[i] = tot;
            tot += gemm_blocks(g.h[i].M, g.h[i].N, g.rc);
            g.maxK = std::max(g.maxK, g.h[i].K1 + g.h[i].K2);
            GemmArgsT<T> &a = g.h[i];
            a.sp_rc = 0;
            if (i < g.op.size()) {
                const SpDev &sp = sparse_for(g.op[i], g.rc);
                if (sp.rc == g.rc) {
                    a.sp_rc = sp.rc;
                    a.sp_lmax = sp.lmax;
                    a.sp_off = sp.off;
                    a.sp_cols = sp.cols;
                    a.sp_vals = sp.vals;
                    a.sp_masked = 0;
                }
            }
        }
        g.total = tot;
        g.ndesc = (int)g.h.size();
        if (g.h.empty()) return FR_OK;
        int rc;
        if ((rc = dev_put((void **)&g.d, g.h.data(), sizeof(GemmArgsT<T>) * g.h.size()))) return rc;
        return dev_put((void **)&g.begin, bg.data(), sizeof(int64_t) * bg.size());
    }

    template <typename I>
    int upload_segs(Segs<I> &sg) {
        if (sg.h.empty()) return FR_OK;
        int rc;
        if ((rc = dev_put((void **)&sg.d, sg.h.data(), sizeof(I) * sg.h.size()))) return rc;
        return dev_put((void **)&sg.begin, sg.hb.data(), sizeof(int64_t) * sg.hb.size());
    }

    int build() {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->ctx[0]->device);
        if (int rc = cuda_check(configure_gemm_grouped<T>(), "grouped gemm attributes")) return rc;
        m0.mode = GEMM_STORE;
        // FP32 storage: the reference gradient, transformed by the flux
        // kernel (the arithmetic of the per-problem launches)
        grad.mode = xform ? GEMM_STORE : GEMM_GRAD;
        m0g.mode = GEMM_STORE;
        m0.rc = kMaxBatchRC;
        grad.rc = kMaxBatchRC;
        m0g.rc = kMaxBatchRC;
        for (auto &g : div) {
            g.mode = GEMM_DIV_RK;
            g.rc = kMaxBatchRC;
        }
        for (fr_ctx *c : b->ctx) {
            for (int t = 0; t < NT; ++t) {
                DevType &D = c->T[t];
                if (!D.present) continue;
                const T *in = (const T *)D.Us;
                const int key = t * 64 + c->order * 4;
                m0.h.push_back(args_m0<T>(c, t, in));
                m0.op.push_back(key + 0);
                if (viscous) {
                    grad.h.push_back(args_grad<T>(c, t, in));
                    if (xform) grad.h.back().mode = GEMM_STORE;
                    grad.op.push_back(key + 1);
                    m0g.h.push_back(args_m0grad<T>(c, t));
                    m0g.op.push_back(key + 0);
                }
                flux.hb.push_back(flux.total);
                flux.h.push_back(FluxItem<T>{D.nu, D.ne, D.np, (const T *)D.Us, (const T *)D.GU,
                                             (const T *)D.S_t, (T *)D.FT, xform ? (const T *)D.invJ_t : nullptr});
                flux.total += (int64_t)D.nu * D.np;
                CenterItem<T> ci{(int64_t)D.nu * NVV * D.np, D.np, D.U, (T *)D.Us, {0, 0, 0, 0, 0}};
                const Phys ph = phys_of(c);
                for (int v = 0; v < 5; ++v) ci.uref[v] = ph.uref[v];
                center.hb.push_back(center.total);
                center.h.push_back(ci);
                center.total += ci.n;
            }
            face.hb.push_back(face.total);
            face.h.push_back(FaceItem<T>{pairs_of(c), bnd_of(c), fields_of<T>(c)});
            face.total += c->npairs + c->nbnd;
        }
        flux.grid = face.grid = center.grid = nsm * 16;
        m0.grid = grad.grid = m0g.grid = nsm * 8;
        for (auto &g : div) g.grid = nsm * 8;
        int rc;
        if ((rc = upload_group(m0)) || (rc = upload_group(grad)) || (rc = upload_group(m0g)) ||
            (rc = upload_segs(flux)) || (rc = upload_segs(face)) || (rc = upload_segs(center)))
            return rc;
        {
            // barrier words and status of the stage kernel, zeroed
            const unsigned zb[2] = {0u, 0u};
            const int zi = 0;
            if ((rc = dev_put((void **)&bar, zb, sizeof(zb))) || (rc = dev_put((void **)&serr, &zi, sizeof(int))))
                return rc;
        }
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_err(FR_ERR_CUDA, "batch stream/event creation");
        }
        return FR_OK;
    }

    // divergence descriptors of the four RK stages for the time steps dt
    int set_dt(const double *dt) {
        bool same = dt_cur.size() == b->ctx.size();
        for (size_t i = 0; same && i < b->ctx.size(); ++i) same = dt_cur[i] == dt[i];
        if (same && div[0].d) return FR_OK;
        dt_cur.assign(dt, dt + b->ctx.size());
        for (int st = 0; st < 4; ++st) {
            div[st].h.clear();
            div[st].op.clear();
            for (size_t i = 0; i < b->ctx.size(); ++i) {
                const double h = dt[i];
                const double ca[4] = {h / 6.0, h / 3.0, h / 3.0, h / 6.0};
                const double cs[4] = {0.5 * h, 0.5 * h, h, 0.0};
                RKStage rk{ca[st], cs[st], st == 0, st == 3};
                for (int t = 0; t < NT; ++t)
                    if (b->ctx[i]->T[t].present) {
                        div[st].h.push_back(args_div<T>(b->ctx[i], t, &rk));
                        div[st].op.push_back(t * 64 + b->ctx[i]->order * 4 + 2);
                    }
            }
            int rc = upload_group(div[st]);
            if (rc) return rc;
        }
        return FR_OK;
    }

    int launch_group(const Group<T> &g, cudaStream_t s) {
        return cuda_check(launch_gemm_grouped<T>(g.d, g.begin, g.ndesc, g.total, g.mode, g.rc, g.maxK, g.grid, s),
                          "grouped gemm");
    }

    // one RK stage of the whole batch on stream s; returns launches via n
    int stage(int st, cudaStream_t s, int &n) {
        const Phys ph = phys_of(b->ctx[0]);
        int rc;
        if ((rc = launch_group(m0, s))) return rc;
        ++n;
        auto flux_step = [&]() {
            return cuda_check(launch_flux_grouped<T>(flux.d, flux.begin, (int)flux.h.size(), flux.total, ph,
                                                     flux.grid, s, xform),
                              "grouped flux");
        };
        if (viscous) {
            if ((rc = cuda_check(launch_face_grouped<T>(face.d, face.begin, (int)face.h.size(), face.total, ph, 0,
                                                        face.grid, s),
                                 "grouped common solution")))
                return rc;
            if ((rc = launch_group(grad, s))) return rc;
            // FP32 storage: the flux kernel forms the physical gradient M0 is
            // then applied to
            if (xform && (rc = flux_step())) return rc;
            if ((rc = launch_group(m0g, s))) return rc;
            n += 3;
        }
        if ((!xform && (rc = flux_step())) ||
            (rc = cuda_check(launch_face_grouped<T>(face.d, face.begin, (int)face.h.size(), face.total, ph, 1,
                                                    face.grid, s),
                             "grouped common flux")) ||
            (rc = launch_group(div[st], s)))
            return rc;
        n += 3;
        return FR_OK;
    }

    static StagePhase<T> gemm_phase(const Group<T> &g) {
        StagePhase<T> p;
        p.descs = g.d;
        p.begin = g.begin;
        p.ndesc = g.ndesc;
        p.total = g.total;
        p.mode = g.mode;
        p.rc = g.rc;
        p.maxK = g.maxK;
        return p;
    }
    void add_flux(StagePhase<T> &p, int xf) const {
        p.fitems = flux.d;
        p.fbegin = flux.begin;
        p.fn = (int)flux.h.size();
        p.ftotal = flux.total;
        p.xform = xf;
    }
    void add_face(StagePhase<T> &p, int which) const {
        p.citems = face.d;
        p.cbegin = face.begin;
        p.cn = (int)face.h.size();
        p.ctotal = face.total;
        p.which = which;
    }

    // the phases of stage st (with_div = false: all but the divergence,
    // for the bounded-wait self-test, which must not touch the registers):
    //   Euler       [M0 + flux] [common flux] [divergence + RK]
    //   NS, FP64    [M0] [common solution] [gradient] [M0 on gradients +
    //               flux] [common flux] [divergence + RK]
    //   NS, FP32    as FP64, but the flux (which forms the physical
    //               gradient in place) precedes M0 on the gradients
    StagePlan<T> make_plan(int st, bool with_div) const {
        StagePlan<T> pl;
        int n = 0;
        if (!viscous) {
            pl.ph[n] = gemm_phase(m0);
            add_flux(pl.ph[n++], 0);
        } else {
            pl.ph[n++] = gemm_phase(m0);
            add_face(pl.ph[n++], 0);
            pl.ph[n++] = gemm_phase(grad);
            if (xform) {
                add_flux(pl.ph[n++], 1);
                pl.ph[n++] = gemm_phase(m0g);
            } else {
                pl.ph[n] = gemm_phase(m0g);
                add_flux(pl.ph[n++], 0);
            }
        }
        add_face(pl.ph[n++], 1);
        if (with_div) pl.ph[n++] = gemm_phase(div[st]);
        pl.nph = n;
        return pl;
    }

    int build_plans() {
        for (int st = 0; st < 4; ++st) plan[st] = make_plan(st, true);
        return cuda_check(stage_grid<T>(plan[0], viscous ? 1 : 0, &stage_grid_n), "stage grid");
    }

    int capture(int mode) {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        if (graph) {
            cudaGraphDestroy(graph);
            graph = nullptr;
        }
        int rc;
        if (mode == 1 && (rc = build_plans())) return rc;
        const Phys ph = phys_of(b->ctx[0]);
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_check(cudaGetLastError(), "begin capture");
        int n = 0;
        rc = FR_OK;
        for (int st = 0; st < 4 && !rc; ++st) {
            if (mode == 1) {
                rc = cuda_check(launch_stage<T>(plan[st], ph, bar, serr, -1, stage_grid_n, cap), "stage launch");
                ++n;
            } else {
                rc = stage(st, cap, n);
            }
        }
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_check(e, "end capture");
        if ((rc = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate"))) return rc;
        launches_per_step = n;
        if (mode == 2) launches_grouped = n;
        graph_mode = mode;
        return FR_OK;
    }

    // FR_ERR_TIMEOUT (once; the status and the barrier words are cleared so
    // the batch stays usable) if a barrier wait of the stage kernel ran out
    int check(cudaStream_t s) override {
        int h = 0, rc;
        if ((rc = cuda_check(cudaStreamSynchronize(s), "batch check sync")) ||
            (rc = cuda_check(cudaStreamSynchronize(cap), "batch check sync")) ||
            (rc = cuda_check(cudaMemcpy(&h, serr, sizeof(int), cudaMemcpyDeviceToHost), "batch status")))
            return rc;
        if (!h) return FR_OK;
        if ((rc = cuda_check(cudaMemset(serr, 0, sizeof(int)), "batch status reset")) ||
            (rc = cuda_check(cudaMemset(bar, 0, 2 * sizeof(unsigned)), "batch barrier reset")))
            return rc;
        return set_err(FR_ERR_TIMEOUT, "a grid barrier of the persistent stage kernel gave up (code " +
                                           std::to_string(h) + ")");
    }

    // one stage without its divergence, launched with CTA 0 taking no part:
    // every other CTA's first barrier wait must run out and be reported
    int selftest(cudaStream_t s) override {
        int rc;
        if ((rc = check(s)) && rc != FR_ERR_TIMEOUT) return rc;
        const StagePlan<T> pl = make_plan(0, false);
        int grid = 0;
        if ((rc = cuda_check(stage_grid<T>(pl, viscous ? 1 : 0, &grid), "stage grid"))) return rc;
        if (grid < 2) return set_err(FR_ERR_UNSUPPORTED, "the self-test needs two CTAs");
        if ((rc = cuda_check(launch_stage<T>(pl, phys_of(b->ctx[0]), bar, serr, 0, grid, s), "self-test launch")))
            return rc;
        rc = check(s);
        if (rc == FR_ERR_TIMEOUT) return FR_OK;
        if (rc) return rc;
        return set_err(FR_ERR_CUDA, "the withheld barrier arrival did not end in a reported timeout");
    }

    int step(const double *dt, int nsteps, int batched, cudaStream_t s) override {
        if (nsteps <= 0) return FR_OK;
        if (!batched) {
            for (size_t i = 0; i < b->ctx.size(); ++i) {
                int rc = step_impl<T>(b->ctx[i], dt[i], nsteps, s);
                if (rc) return rc;
            }
            return FR_OK;
        }
        int rc;
        const int mode = batched == 2 ? 2 : 1;
        const bool new_dt = dt_cur.size() != b->ctx.size() ||
                            !std::equal(dt_cur.begin(), dt_cur.end(), dt) || !div[0].d;
        if ((rc = set_dt(dt))) return rc;
        if (!exec || new_dt || graph_mode != mode)
            if ((rc = capture(mode))) return rc;
        // order the internal capture stream after the caller's stream
        if ((rc = cuda_check(cudaEventRecord(ev_in, s), "event")) ||
            (rc = cuda_check(cudaStreamWaitEvent(cap, ev_in, 0), "wait")))
            return rc;
        // the centred stage input is derived from the FP64 registers once
        if ((rc = cuda_check(launch_center_grouped<T>(center.d, center.begin, (int)center.h.size(), center.total,
                                                      center.grid, cap),
                             "grouped centre")))
            return rc;
        for (int it = 0; it < nsteps; ++it)
            if ((rc = cuda_check(cudaGraphLaunch(exec, cap), "graph launch"))) return rc;
        if ((rc = cuda_check(cudaEventRecord(ev_out, cap), "event")) ||
            (rc = cuda_check(cudaStreamWaitEvent(s, ev_out, 0), "wait")))
            return rc;
        return FR_OK;
    }

    // time one grouped launch (milliseconds per launch, best of reps)
    template <class F>
    float time_it(F fn, cudaStream_t s) {
        cudaEvent_t a, c;
        cudaEventCreate(&a);
        cudaEventCreate(&c);
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(a, s);
            if (fn() != FR_OK) {
                best = 1e30f;
                break;
            }
            cudaEventRecord(c, s);
            cudaEventSynchronize(c);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, c);
            best = std::min(best, ms);
        }
        cudaEventDestroy(a);
        cudaEventDestroy(c);
        return best;
    }

    int tune_group(Group<T> &g, cudaStream_t s) {
        if (g.h.empty()) return FR_OK;
        int best_rc = g.rc, best_grid = g.grid;
        float best = 1e30f;
        for (int rc : kGroupedRCs) {
            if (rc > kMaxBatchRC || (g.mode == GEMM_GRAD && rc % 3)) continue;
            if (gemm_block_smem(rc, (int)sizeof(T), g.maxK ? g.maxK : 1, g.maxK ? g.maxK : 1) > 200 * 1024) continue;
            g.rc = rc;
            int e = upload_group(g);
            if (e) return e;
            for (int mult : {2, 4, 8, 16}) {
                g.grid = nsm * mult;
                const float ms = time_it([&] { return launch_group(g, s); }, s);
                if (ms < best) {
                    best = ms;
                    best_rc = rc;
                    best_grid = g.grid;
                }
            }
        }
        g.rc = best_rc;
        g.grid = best_grid;
        return upload_group(g);
    }

    int tune(cudaStream_t s) override {
        int rc;
        const Phys ph = phys_of(b->ctx[0]);
        // the inputs of every class must be valid: centre, then run one stage
        // un-timed to fill the scratch of the later classes
        if (dt_cur.empty()) {
            std::vector<double> z(b->ctx.size(), 0.0);
            if ((rc = set_dt(z.data()))) return rc;
        }
        if ((rc = cuda_check(launch_center_grouped<T>(center.d, center.begin, (int)center.h.size(), center.total,
                                                      center.grid, s),
                             "grouped centre")))
            return rc;
        // the divergence class is tuned in its plain form (writing R), which
        // leaves the RK registers untouched
        Group<T> dv;
        dv.mode = GEMM_DIV;
        for (fr_ctx *c : b->ctx)
            for (int t = 0; t < NT; ++t)
                if (c->T[t].present) {
                    dv.h.push_back(args_div<T>(c, t, nullptr));
                    dv.op.push_back(t * 64 + c->order * 4 + 2);
                }
        dv.rc = 16;
        dv.grid = nsm * 8;
        if ((rc = upload_group(dv))) return rc;
        if ((rc = tune_group(m0, s))) return rc;
        if (viscous) {
            if ((rc = cuda_check(launch_face_grouped<T>(face.d, face.begin, (int)face.h.size(), face.total, ph, 0,
                                                        face.grid, s),
                                 "grouped common solution")))
                return rc;
            if ((rc = tune_group(grad, s)) || (rc = tune_group(m0g, s))) return rc;
        }
        // point-wise grids
        for (Segs<FluxItem<T>> *sg : {&flux}) {
            float best = 1e30f;
            int bg = sg->grid;
            for (int mult : {4, 8, 16, 32}) {
                sg->grid = nsm * mult;
                const float ms = time_it(
                    [&] {
                        return cuda_check(launch_flux_grouped<T>(sg->d, sg->begin, (int)sg->h.size(), sg->total, ph,
                                                                 sg->grid, s),
                                          "flux");
                    },
                    s);
                if (ms < best) {
                    best = ms;
                    bg = sg->grid;
                }
            }
            sg->grid = bg;
        }
        {
            float best = 1e30f;
            int bg = face.grid;
            for (int mult : {4, 8, 16, 32}) {
                face.grid = nsm * mult;
                const float ms = time_it(
                    [&] {
                        return cuda_check(launch_face_grouped<T>(face.d, face.begin, (int)face.h.size(), face.total,
                                                                 ph, 1, face.grid, s),
                                          "face");
                    },
                    s);
                if (ms < best) {
                    best = ms;
                    bg = face.grid;
                }
            }
            face.grid = bg;
        }
        if ((rc = tune_group(dv, s))) {
            dev_free(dv.d);
            dev_free(dv.begin);
            return rc;
        }
        for (auto &g : div) {
            g.rc = dv.rc;
            g.grid = dv.grid;
            if (!g.h.empty() && (rc = upload_group(g))) break;
        }
        dev_free(dv.d);
        dev_free(dv.begin);
        if (rc) return rc;
        // force a new capture with the tuned shapes
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        return cuda_check(cudaStreamSynchronize(s), "tune sync");
    }

    void info(int64_t *out) const override {
        int64_t ndof = 0;
        for (fr_ctx *c : b->ctx)
            for (int t = 0; t < NT; ++t)
                if (c->T[t].present) ndof += c->T[t].ne * NVV * c->T[t].nu;
        out[0] = (int64_t)b->ctx.size();
        out[1] = ndof;
        out[2] = launches_per_step;
        // per-problem launch sequence per stage: per type M0, (gradient, M0
        // on the gradients), flux, divergence and (FP32: the separate RK
        // update), and the face kernels
        int64_t un = 0;
        for (fr_ctx *c : b->ctx) {
            int nt = 0;
            for (int t = 0; t < NT; ++t) nt += c->T[t].present;
            un += 4 * (((viscous ? 5 : 3) + (sizeof(T) == sizeof(float) ? 1 : 0)) * nt + (viscous ? 2 : 1));
        }
        out[3] = un;
        out[4] = m0.rc;
        out[5] = viscous ? grad.rc : 0;
        out[6] = viscous ? m0g.rc : 0;
        out[7] = div[0].rc;
        out[8] = m0.grid;
        out[9] = div[0].grid;
        out[10] = flux.grid;
        out[11] = face.grid;
        out[12] = stage_grid_n;
        out[13] = launches_grouped;
    }
};

}  // namespace

extern "C" {

int fr_batch_create(int nprob, const fr_mesh *meshes, const int *orders, const fr_params *params, fr_batch **out) {
    if (!out || nprob <= 0 || !meshes || !orders || !params) return set_err(FR_ERR_ARG, "invalid batch arguments");
    *out = nullptr;
    if (params->precision != FR_FP64 && params->precision != FR_FP32)
        return set_err(FR_ERR_UNSUPPORTED, "batched launches run FR_FP64 or FR_FP32 operator kernels");
    fr_batch *b = new (std::nothrow) fr_batch();
    if (!b) return set_err(FR_ERR_NOMEM, "host allocation");
    for (int i = 0; i < nprob; ++i) {
        fr_ctx *c = nullptr;
        int rc = fr_create(&meshes[i], orders[i], params, &c);
        if (rc) {
            for (fr_ctx *q : b->ctx) fr_destroy(q);
            delete b;
            return rc;
        }
        b->ctx.push_back(c);
    }
    int rc;
    try {
        if (params->precision == FR_FP32) {
            auto *im = new BatchImpl<float>(b);
            b->impl = im;
            rc = im->build();
        } else {
            auto *im = new BatchImpl<double>(b);
            b->impl = im;
            rc = im->build();
        }
    } catch (...) {
        rc = set_err(FR_ERR_NOMEM, "batch set-up");
    }
    if (rc) {
        fr_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FR_OK;
}

void fr_batch_destroy(fr_batch *b) {
    if (!b) return;
    delete b->impl;
    for (fr_ctx *c : b->ctx) fr_destroy(c);
    delete b;
}

int fr_batch_problem(fr_batch *b, int i, fr_ctx **ctx) {
    if (!b || !ctx || i < 0 || i >= (int)b->ctx.size()) return set_err(FR_ERR_ARG, "invalid problem index");
    *ctx = b->ctx[i];
    return FR_OK;
}

int fr_batch_tune(fr_batch *b, void *stream) {
    if (!b) return set_err(FR_ERR_ARG, "null batch");
    return b->impl->tune((cudaStream_t)stream);
}

int fr_batch_step(fr_batch *b, const double *dt, int nsteps, int batched, void *stream) {
    if (!b || !dt || nsteps < 0) return set_err(FR_ERR_ARG, "invalid step arguments");
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        if (!(dt[i] == dt[i])) return set_err(FR_ERR_ARG, "non-finite time step");
        for (int t = 0; t < NT; ++t)
            if (b->ctx[i]->T[t].cl_on)
                return set_err(FR_ERR_UNSUPPORTED, "batched steps do not apply a learned closure");
    }
    return b->impl->step(dt, nsteps, batched, (cudaStream_t)stream);
}

int fr_batch_check(fr_batch *b, void *stream) {
    if (!b) return set_err(FR_ERR_ARG, "null batch");
    return b->impl->check((cudaStream_t)stream);
}

int fr_batch_selftest_wait_timeout(fr_batch *b, void *stream) {
    if (!b) return set_err(FR_ERR_ARG, "null batch");
    return b->impl->selftest((cudaStream_t)stream);
}

int fr_batch_info(const fr_batch *b, int64_t *out) {
    if (!b || !out) return set_err(FR_ERR_ARG, "null argument");
    b->impl->info(out);
    return FR_OK;
}

}  // extern "C"
